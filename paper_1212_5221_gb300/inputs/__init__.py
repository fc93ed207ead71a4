"""Seeded synthetic link fields and job streams.

This module is the one piece of code that the CUDA path's tests and
benchmarks and the FP64 oracle's checks have in common.  It produces
starting configurations only and contains none of the gauge-fixing
arithmetic.  The paper's beta = 5.7 Monte-Carlo configurations are not
available, so these fields stand in for them:

* ``smooth``: links exp(i eps H), H Gaussian traceless Hermitian,
* ``hot``:    Haar-random SU(3) links ("hot gauge field", Sec. 6.5),
* ``unit``:   all links 1.

Links come back as a complex128 array of shape (Nt, Nx, Ny, Nz, 4, 3, 3),
whose memory is the natural "StandardPattern" order of Sec. 4.2.1
(t, x, y, z, mu, i, j, re/im), mu = 0 temporal.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_inputs.c")
_LIB = os.path.join(_HERE, "libgf_inputs.so")
_KINDS = {"unit": 0, "smooth": 1, "hot": 2}
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator (gcc, OpenMP) into this directory."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
           "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gfin_links.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_double, ctypes.c_uint64,
                                   ctypes.c_void_p]
        lib.gfin_links.restype = None
        _lib = lib
    return _lib


def links(dims, kind: str = "smooth", eps: float = 0.3, seed: int = 0,
          t0: int = 0, nt: int | None = None) -> np.ndarray:
    """Links of time-slices [t0, t0+nt) of a lattice dims = (Nt, Nx, Ny, Nz)."""
    dims = tuple(int(d) for d in dims)
    nt = dims[0] - t0 if nt is None else int(nt)
    if not (0 <= t0 and t0 + nt <= dims[0]):
        raise ValueError("slab outside the lattice")
    out = np.empty((nt, dims[1], dims[2], dims[3], 4, 3, 3), dtype=np.complex128)
    d = (ctypes.c_int * 4)(*dims)
    _load().gfin_links(d, t0, nt, _KINDS[kind], float(eps), int(seed) & (2**64 - 1),
                       out.ctypes.data)
    return out


def poisson_jobs(n_jobs: int, rate_per_s: float, seed: int,
                 lattices=((16, 16, 16, 16), (48, 24, 24, 24), (32, 32, 32, 32), (96, 48, 48, 48)),
                 gauges=("landau", "coulomb", "mag")):
    """A Poisson stream of gauge-fixing jobs: arrival time, lattice, gauge, seed.

    Lattices are (Nt, Nx, Ny, Nz); 24^3 x 48 is (48, 24, 24, 24).
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_jobs)
    arrivals = np.cumsum(gaps) - gaps[0]
    li = rng.integers(0, len(lattices), size=n_jobs)
    gi = rng.integers(0, len(gauges), size=n_jobs)
    seeds = rng.integers(0, 2**31 - 1, size=n_jobs)
    return [dict(arrival=float(arrivals[k]), dims=tuple(lattices[li[k]]), gauge=gauges[gi[k]],
                 seed=int(seeds[k])) for k in range(n_jobs)]
