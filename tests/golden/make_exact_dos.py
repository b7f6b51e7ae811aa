"""Writes exact_dos_small.json: exact densities of states of small periodic
Potts lattices, computed by the oracle's brute-force enumeration and its
transfer matrix (this script calls only oracle/).

    python tests/golden/make_exact_dos.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402

CASES = [("brute", 2, 4), ("brute", 3, 3), ("tm", 2, 6), ("tm", 10, 4)]


def main():
    out = {"_source": "oracle/exact_dos.c via oracle/oracle.py (brute force and transfer matrix); "
                      "counts[k] = number of configurations with k broken bonds, E = -2N + k"}
    for kind, q, L in CASES:
        counts = O.exact_counts_brute(q, L) if kind == "brute" else O.exact_counts_tm(q, L)
        out["%s_q%d_L%d" % (kind, q, L)] = {"q": q, "L": L, "counts": [str(c) for c in counts]}
    with open(os.path.join(HERE, "exact_dos_small.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
