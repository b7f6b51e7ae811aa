"""The debug build (librewl_debug.so: every ln g, shadow and histogram index of
the sweeps checked against its array, the production kernel's too, and every
active walker's energy recounted before each window check) on a GPU: parity
cases run in a child process with REWL_DEBUG=1 must report no bounds or
energy error (either would make the run return REWL_ERR_STATE) and still match
the oracle.  The child builds nothing: the debug library is built here first.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r"""
import sys
sys.path.insert(0, %(root)r)
sys.path.insert(0, %(tests)r)
import numpy as np
from oracle import oracle as O
from paper_1312_3004_gb300 import REWL, Batch, _lib
from paper_1312_3004_gb300 import workloads as WL
from tie_trace import TracedPair, differing, gpu_state, oracle_state

assert _lib.load()._name.endswith("librewl_debug.so"), _lib.load()._name
cases = [
    ((10, 20, 8, 0.75, 4, 1e-8, 0.8, 10_000, 3), 8, []),
    ((10, 20, 8, 0.75, 4, 1e-8, 0.8, 10_000, 3), 8, [(_lib.OPT_LANES, 1)]),
    ((3, 5, 3, 0.75, 3, 1e-4, 0.8, 777, 5), 4, [(_lib.OPT_SWEEP_KERNEL, 1)]),
    ((2, 8, 4, 0.75, 2, 1e-6, 0.8, 10_000, 1), 8, [(_lib.OPT_LANES, 8)]),
    ((10, 130, 8, 0.75, 1, 1e-6, 0.8, 2000, 3), 8, []),  # lattices in global memory
]
for args, bits, opts in cases:
    def make(args=args, bits=bits, opts=opts):
        r = REWL(*args, spin_bits=bits)
        for o, v in opts:
            r.set_option(o, v)
        return r
    tp = TracedPair(make, lambda args=args: O.OracleREWL(*args))
    for n in (1, 3):
        tp.run(n)
p = WL.params("potts10_L80")
tp = TracedPair(lambda: REWL(*WL.rewl_args(p, 1), spin_bits=p["spin_bits"]),
                lambda: O.OracleREWL(*WL.rewl_args(p, 1)))
tp.run(1)
args = (4, 6, 3, 0.75, 2, 1e-3, 0.8, 400, 9)
g, o = REWL(*args), O.OracleREWL(*args)
g.run(3); o.run(3)
g.production_start(5); o.production_start(5)
g.production_run(3); o.production_run(3)
assert not differing(gpu_state(g), oracle_state(o)) and np.array_equal(g.heo(), o.heo())
jobs = [dict(q=10, L=12, h=3, overlap=0.75, m=2, lnf_final=1e-6, flatness=0.8, exchange_interval=2000, seed=s)
        for s in (3, 4)]
for lanes in (1, 32):
    b = Batch(jobs, lanes=lanes)
    b.run(3)
    for i, j in enumerate(jobs):
        orc = O.OracleREWL(*WL.rewl_args(j, j["seed"]))
        orc.run(3)
        assert not differing(gpu_state(b.instance(i)), oracle_state(orc))
print("debug build: no bounds or energy error")
"""


def test_debug_build_reports_no_bounds_or_energy_error():
    from paper_1312_3004_gb300 import build

    build.build(debug=True)
    env = dict(os.environ, REWL_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT, "tests": HERE}], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no bounds or energy error" in r.stdout
