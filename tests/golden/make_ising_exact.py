"""Writes tests/golden/ising_exact_torus.json: the exact density of states of
the 2D Ising model (the q = 2 Potts model) on the L x L torus for L = 16 and
32, from Kaufman's partition function expanded in y = exp(-2K) (Beale's
method; oracle/kaufman.py).  Calls only the oracle.

g(b) counts the configurations with b broken bonds (Potts energy E = b - 2N,
Ising energy 2b - 2N).  Stored per L: the exact counts of b = 0 .. 16 as
decimal strings, ln g(b) for every b (null where g = 0) and the SHA-256 of the
decimal counts joined by commas, with the largest distance of a Fourier
coefficient from its integer (the expansion's own accuracy check).

    python tests/golden/make_ising_exact.py         # L = 16 and 32 (about 5 minutes)
"""
import hashlib
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def main():
    sys.path.insert(0, ROOT)
    from oracle import kaufman

    out = {"source": "oracle/kaufman.py (Kaufman 1949 torus partition function, expanded as in Beale 1996); "
                     "written by tests/golden/make_ising_exact.py", "lattices": {}}
    for L in (16, 32):
        counts, worst = kaufman.ising_counts(L)
        out["lattices"][str(L)] = {
            "L": L, "N": L * L, "max_rounding_residual": worst,
            "low_counts": [str(c) for c in counts[:17]],
            "lng": [math.log(c) if c > 0 else None for c in counts],
            "sha256": hashlib.sha256(",".join(str(c) for c in counts).encode()).hexdigest(),
        }
    with open(os.path.join(HERE, "ising_exact_torus.json"), "w") as f:
        json.dump(out, f)
        f.write("\n")


if __name__ == "__main__":
    main()
