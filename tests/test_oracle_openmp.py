"""The OpenMP build of the oracle (used only to time it on all host cores)
gives bit-identical sweeps: the sites of one parity touch disjoint links
(Sec. 2.2), and the random draws are keyed by site, not by visiting order."""
import os
import subprocess
import sys
import tempfile

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = """
import sys, numpy as np
sys.path.insert(0, {root!r})
import oracle
from paper_1212_5221_gb300 import inputs
if {omp}:
    oracle.use_openmp()
U = inputs.links((4, 4, 6, 8), "smooth", 0.4, 3)
oracle.random_gauge_transform(U, 7)
oracle.sweep(U, "landau", "or", 1.7, 3)
oracle.sweep(U, "coulomb", "sr", 0.5, 2, 5, 9)
oracle.anneal(U, "mag", 1.0, 0.5, 2, 11, 13)
np.save({out!r}, U)
"""


def run(omp, out):
    env = dict(os.environ, OMP_NUM_THREADS="4")
    subprocess.run([sys.executable, "-c", CODE.format(root=ROOT, omp=omp, out=out)], check=True, env=env,
                   timeout=600)
    return np.load(out)


def test_openmp_build_bit_identical():
    with tempfile.TemporaryDirectory() as d:
        a = run(False, os.path.join(d, "a.npy"))
        b = run(True, os.path.join(d, "b.npy"))
    assert np.array_equal(a, b)
