"""ctypes binding to the FP64 CPU oracle (gf_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py.  The product path never imports it.

Links are complex128 arrays of shape (Nt, Nx, Ny, Nz, 4, 3, 3) (the
paper's StandardPattern order, Sec. 4.2.1).  Gauge codes: 0 Landau,
1 Coulomb, 2 MAG.  Algorithm codes: 0 relaxation, 1 overrelaxation,
2 microcanonical, 3 stochastic relaxation, 4 simulated annealing.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

LANDAU, COULOMB, MAG = 0, 1, 2
RELAX, OR, MICRO, SR, SA = 0, 1, 2, 3, 4
GAUGES = {"landau": LANDAU, "coulomb": COULOMB, "mag": MAG}
ALGOS = {"relax": RELAX, "or": OR, "micro": MICRO, "sr": SR, "sa": SA}

_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)
_V = ctypes.c_void_p
_U32 = ctypes.c_uint32
_U64 = ctypes.c_uint64


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_openmp = False


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, IEEE semantics, no FMA contraction).
    openmp=True: the same source with -fopenmp (the sweep visits the sites of a
    parity in parallel), a separate library used only to time the oracle on all
    host cores."""
    lib = _LIB_OMP if openmp else _LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(_SRC):
        return lib
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared"]
                   + (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, lib)
    return lib


def use_openmp():
    """Load the OpenMP build instead of the plain one (before the first call)."""
    global _openmp
    if _lib is not None and not _openmp:
        raise RuntimeError("the plain oracle library is already loaded")
    _openmp = True


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build(openmp=_openmp))
    sig = {
        "or_philox4x32_10": (None, [ctypes.POINTER(_U32), ctypes.POINTER(_U32), ctypes.POINTER(_U32)]),
        "or_u01": (_D, [_U32, _U32]),
        "or_gauge_transform": (None, [_PI, _V, _V]),
        "or_haar_su3": (None, [_U64, _U32, _U32, _V]),
        "or_random_gauge_transform": (None, [_PI, _V, _U64, _U32]),
        "or_reunitarize": (None, [_PI, _V]),
        "or_observables": (None, [_PI, _V, ctypes.c_int, _PD, _PD, _V, _V]),
        "or_plaquette": (_D, [_PI, _V]),
        "or_unitarity": (None, [_PI, _V, _PD, _PD]),
        "or_kp_sample": (ctypes.c_int, [_D, _U64, _U32, _U32, _U32, _U32, _PD]),
        "or_mag_cosbeta": (_D, [_D, _D]),
        "or_site_subgroup_update": (None, [_PI, _V, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, _D, _U32, _U64, _U32]),
        "or_sweep": (None, [_PI, _V, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _U32, _U64,
                            _U32, _V]),
        "or_sweep_trace": (None, [_PI, _V, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _U32, _U64,
                                  _U32, _V, _V, _V]),
        "or_half_sweep": (None, [_PI, _V, ctypes.c_int, ctypes.c_int, _D, ctypes.c_int, _U32, _U64,
                                 _U32, _V]),
        "or_sa_update": (ctypes.c_int, [ctypes.c_int, _PD, _D, _U64, _U32, _U32, _U32, _U32, _PD]),
        "or_anneal": (None, [_PI, _V, ctypes.c_int, _D, _D, ctypes.c_int, _U32, _U64, _U32]),
        "or_step_quaternion": (None, [_PD, ctypes.c_int, _D, _PD]),
        "or_haar_field": (None, [_U64, _U32, ctypes.c_long, _U32, _V]),
        "or_mag_maximiser": (None, [_PD, _PD]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dims(U):
    if U.dtype != np.complex128 or U.ndim != 7 or U.shape[4:] != (4, 3, 3):
        raise ValueError("links must be complex128 of shape (Nt,Nx,Ny,Nz,4,3,3)")
    if not U.flags.c_contiguous:
        raise ValueError("links must be C-contiguous")
    return (ctypes.c_int * 4)(*U.shape[:4])


def _gauge(g):
    return GAUGES[g] if isinstance(g, str) else int(g)


def _algo(a):
    return ALGOS[a] if isinstance(a, str) else int(a)


def philox4x32_10(ctr, key):
    c = (_U32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (_U32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    out = (_U32 * 4)()
    _load().or_philox4x32_10(c, k, out)
    return tuple(out)


def u01(hi, lo):
    return _load().or_u01(hi & 0xFFFFFFFF, lo & 0xFFFFFFFF)


def gauge_transform(U, g):
    """U_mu(x) <- g(x) U_mu(x) g(x+mu)^dag in place; g has shape (Nt,Nx,Ny,Nz,3,3)."""
    g = np.ascontiguousarray(g, dtype=np.complex128)
    if g.shape != U.shape[:4] + (3, 3):
        raise ValueError("g has the wrong shape")
    _load().or_gauge_transform(_dims(U), U.ctypes.data, g.ctypes.data)


def haar_su3(seed, site, copy=0):
    out = np.empty((3, 3), np.complex128)
    _load().or_haar_su3(seed & (2**64 - 1), site, copy, out.ctypes.data)
    return out


def haar_field(seed, site0, n, copy=0):
    """Haar g(x) of the random gauge transformation for sites site0 .. site0+n-1."""
    out = np.empty((n, 3, 3), np.complex128)
    _load().or_haar_field(seed & (2**64 - 1), site0, n, copy, out.ctypes.data)
    return out


def random_gauge_transform(U, seed, copy=0):
    _load().or_random_gauge_transform(_dims(U), U.ctypes.data, seed & (2**64 - 1), copy)


def reunitarize(U):
    _load().or_reunitarize(_dims(U), U.ctypes.data)


def observables(U, gauge):
    """(F, theta, F_t, theta_t): functional, gauge precision, and per time-slice values."""
    Nt = U.shape[0]
    F, th = _D(), _D()
    ft = np.zeros(Nt)
    tt = np.zeros(Nt)
    _load().or_observables(_dims(U), U.ctypes.data, _gauge(gauge), ctypes.byref(F),
                           ctypes.byref(th), ft.ctypes.data, tt.ctypes.data)
    return F.value, th.value, ft, tt


def plaquette(U):
    return _load().or_plaquette(_dims(U), U.ctypes.data)


def unitarity(U):
    m, x = _D(), _D()
    _load().or_unitarity(_dims(U), U.ctypes.data, ctypes.byref(m), ctypes.byref(x))
    return m.value, x.value


def kp_sample(alpha, seed, site, sweep, sub, copy=0):
    x0 = _D()
    n = _load().or_kp_sample(alpha, seed & (2**64 - 1), site, sweep, sub, copy, ctypes.byref(x0))
    return x0.value, n


def mag_cosbeta(kappa, u):
    return _load().or_mag_cosbeta(kappa, u)


def step_quaternion(m, algo, param=1.0):
    """Relaxation / overrelaxation / microcanonical rule applied to a maximiser quaternion."""
    mm = (_D * 4)(*[float(v) for v in m])
    g = (_D * 4)()
    _load().or_step_quaternion(mm, _algo(algo), float(param), g)
    return np.array(list(g))


def mag_maximiser(x):
    xx = (_D * 3)(*[float(v) for v in x])
    m = (_D * 4)()
    _load().or_mag_maximiser(xx, m)
    return np.array(list(m))


def site_subgroup_update(U, site, sub, gauge, algo, param=1.0, sweep=0, seed=0, copy=0):
    _load().or_site_subgroup_update(_dims(U), U.ctypes.data, site, sub, _gauge(gauge),
                                    _algo(algo), param, sweep, seed & (2**64 - 1), copy)


def sweep(U, gauge, algo, param=1.0, n=1, sweep0=0, seed=0, copy=0, slice_active=None):
    """n checkerboard sweeps in place (Alg. 1)."""
    act = None
    if slice_active is not None:
        act = np.ascontiguousarray(slice_active, dtype=np.int32)
        if act.shape != (U.shape[0],):
            raise ValueError("slice_active needs one flag per time-slice")
    _load().or_sweep(_dims(U), U.ctypes.data, _gauge(gauge), _algo(algo), param, n, sweep0,
                     seed & (2**64 - 1), copy, None if act is None else act.ctypes.data)


def sweep_trace(U, gauge, algo, param=1.0, n=1, sweep0=0, seed=0, copy=0, slice_active=None):
    """As sweep(); also returns, for the last sweep, the heat-bath trial count
    and decision margin of every (site, subgroup): arrays of shape (V, 3)
    (1 and inf where no accept/reject decision was taken)."""
    act = None
    if slice_active is not None:
        act = np.ascontiguousarray(slice_active, dtype=np.int32)
        if act.shape != (U.shape[0],):
            raise ValueError("slice_active needs one flag per time-slice")
    V = int(np.prod(U.shape[:4]))
    trials = np.zeros((V, 3), np.int32)
    margin = np.zeros((V, 3), np.float64)
    _load().or_sweep_trace(_dims(U), U.ctypes.data, _gauge(gauge), _algo(algo), param, n, sweep0,
                           seed & (2**64 - 1), copy, None if act is None else act.ctypes.data,
                           trials.ctypes.data, margin.ctypes.data)
    return trials, margin


def half_sweep(U, gauge, algo, param, parity, sweep=0, seed=0, copy=0, slice_active=None):
    """The sites of one parity only (half of a checkerboard sweep), draws of `sweep`."""
    act = None
    if slice_active is not None:
        act = np.ascontiguousarray(slice_active, dtype=np.int32)
        if act.shape != (U.shape[0],):
            raise ValueError("slice_active needs one flag per time-slice")
    _load().or_half_sweep(_dims(U), U.ctypes.data, _gauge(gauge), _algo(algo), param, parity, sweep,
                          seed & (2**64 - 1), copy, None if act is None else act.ctypes.data)


def sa_update(gauge, v, T, seed, site, sweep=0, sub=0, copy=0):
    """The full heat-bath update of one subgroup: from the maximiser direction
    m (Landau/Coulomb, 4 entries) or the Pauli vector x (MAG, 3 entries).
    Returns (g, trials)."""
    vv = (_D * 4)(*([float(a) for a in v] + [0.0] * (4 - len(v))))
    g = (_D * 4)()
    n = _load().or_sa_update(_gauge(gauge), vv, float(T), seed & (2**64 - 1), site, sweep, sub, copy, g)
    return np.array(list(g)), n


def anneal(U, gauge, T0, T1, n, sweep0=0, seed=0, copy=0):
    """n simulated-annealing steps (heat bath + 3 microcanonical sweeps), T linear T0 -> T1."""
    _load().or_anneal(_dims(U), U.ctypes.data, _gauge(gauge), T0, T1, n, sweep0,
                      seed & (2**64 - 1), copy)


def fix(U, gauge, algo="or", param=1.7, theta_target=1e-12, max_sweeps=100000, check=10,
        seed=0, copy=0, sweep0=0):
    """Sweep until theta < theta_target (checked every `check` sweeps).

    For Coulomb each time-slice stops on its own once its theta_t is below the
    target.  Returns (sweeps, F, theta).
    """
    g = _gauge(gauge)
    n = 0
    active = np.ones(U.shape[0], np.int32)
    while True:
        F, th, ft, tt = observables(U, g)
        if g == COULOMB:
            active = (tt >= theta_target).astype(np.int32)
            if not active.any():
                return n, F, th
        elif th < theta_target:
            return n, F, th
        if n >= max_sweeps:
            return n, F, th
        k = min(check, max_sweeps - n)
        sweep(U, g, algo, param, k, sweep0 + n, seed, copy,
              active if g == COULOMB else None)
        n += k
