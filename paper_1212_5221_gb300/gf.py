"""Thin ctypes binding of libgf (include/gf.h): argument marshalling only.

Every function keeps the C name and raises GFError on a non-zero status.
Link arrays are complex128 numpy arrays of shape (Nt, Nx, Ny, Nz, 4, 3, 3)
(the natural order of Sec. 4.2.1) or, for the *_device calls, CUDA tensors
of the same shape.  There is no fallback: if libgf.so is missing or no GPU
is present, the calls fail loudly.

``GaugeField`` is a small convenience wrapper whose device storage and CUDA
stream come from PyTorch (gf_create_ext with a torch buffer and torch's
current stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgf.so")

GF_LANDAU, GF_COULOMB, GF_MAG = 0, 1, 2
GF_FP64, GF_FP32, GF_MIXED, GF_MP = 0, 1, 2, 3
GF_RELAX, GF_OR, GF_MICRO, GF_SR, GF_SA = 0, 1, 2, 3, 4
GF_KERNEL_SWEEP_FP32, GF_KERNEL_SWEEP_FP64, GF_KERNEL_OBSERVABLES, GF_KERNEL_REUNITARIZE, GF_KERNEL_OTHER = range(5)
GF_OK, GF_EINVAL, GF_ENOMEM, GF_ECUDA, GF_ETIMEOUT, GF_ENOTCONV, GF_ENOSYS, GF_ECANCELED = range(8)

GAUGES = {"landau": GF_LANDAU, "coulomb": GF_COULOMB, "mag": GF_MAG}
PRECISIONS = {"fp64": GF_FP64, "fp32": GF_FP32, "mixed": GF_MIXED, "mp": GF_MP}
ALGOS = {"relax": GF_RELAX, "or": GF_OR, "micro": GF_MICRO, "sr": GF_SR, "sa": GF_SA}


class GFError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        self.code = code
        super().__init__(f"{where}: status {code} ({message})")


class gf_fix_params(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("param", ctypes.c_double), ("theta_target", ctypes.c_double),
                ("max_sweeps", ctypes.c_int), ("check_interval", ctypes.c_int),
                ("reunit_interval", ctypes.c_int), ("switch_theta", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class gf_protocol_params(ctypes.Structure):
    _fields_ = [("sa_steps", ctypes.c_int), ("T_start", ctypes.c_double), ("T_end", ctypes.c_double),
                ("sr_sweeps", ctypes.c_int), ("sr_p", ctypes.c_double), ("sr_theta", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("fix", gf_fix_params)]


class gf_job(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("gauge", ctypes.c_int), ("prec", ctypes.c_int),
                ("host_links", ctypes.c_void_p), ("orbit_seed", ctypes.c_uint64), ("fix", gf_fix_params),
                ("host_out", ctypes.c_void_p), ("tag", ctypes.c_uint64), ("anneal", ctypes.c_int),
                ("protocol", gf_protocol_params)]


class gf_job_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("F", ctypes.c_double),
                ("theta", ctypes.c_double), ("sweeps", ctypes.c_int), ("sweeps_fp32", ctypes.c_int),
                ("sweeps_fp64", ctypes.c_int), ("site_updates", ctypes.c_uint64),
                ("footprint", ctypes.c_size_t), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gf_fix_result(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("sweeps_fp32", ctypes.c_int), ("sweeps_fp64", ctypes.c_int),
                ("checks", ctypes.c_int), ("converged", ctypes.c_int), ("seconds", ctypes.c_double),
                ("site_updates", ctypes.c_uint64), ("F_mean", ctypes.c_double), ("theta_max", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
_PI = ctypes.POINTER(ctypes.c_int)
_SIG = {
    "gf_footprint": [_PI, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)],
    "gf_create": [_PI, _I, _I, _P, ctypes.POINTER(_P)],
    "gf_create_batch": [_PI, _I, _I, _I, _P, ctypes.POINTER(_P)],
    "gf_create_ext": [_PI, _I, _I, _I, _P, _P, ctypes.c_size_t, ctypes.POINTER(_P)],
    "gf_load_links": [_P, _I, _P],
    "gf_load_links_slab": [_P, _I, _I, _I, _P],
    "gf_load_links_device": [_P, _I, _P],
    "gf_store_links": [_P, _I, _P],
    "gf_store_links_device": [_P, _I, _P],
    "gf_store_links_slab": [_P, _I, _I, _I, _P],
    "gf_random_gauge_transform": [_P, ctypes.c_uint64],
    "gf_sweep": [_P, _I, _D, _I, ctypes.c_uint64, _P, _P],
    "gf_anneal": [_P, _D, _D, _I, ctypes.c_uint64, _P, _P],
    "gf_reunitarize": [_P],
    "gf_functional_theta": [_P, _P, _P],
    "gf_slice_functional_theta": [_P, _P, _P],
    "gf_promote": [_P],
    "gf_set_active": [_P, _P],
    "gf_get_sweep_index": [_P, ctypes.POINTER(ctypes.c_uint64)],
    "gf_set_sweep_index": [_P, ctypes.c_uint64],
    "gf_set_copy_base": [_P, ctypes.c_uint32],
    "gf_set_links_per_thread": [_P, _I],
    "gf_set_prefetch": [_P, _I],
    "gf_set_graphs": [_P, _I],
    "gf_set_check_log": [_P, ctypes.c_char_p],
    "gf_set_stage_wait_polls": [_P, _I],
    "gf_sweep_async": [_P, _I, ctypes.c_double, _I, ctypes.c_uint64],
    "gf_anneal_async": [_P, ctypes.c_double, ctypes.c_double, _I, ctypes.c_uint64],
    "gf_random_gauge_transform_async": [_P, ctypes.c_uint64],
    "gf_synchronize": [_P],
    "gf_set_fused_observables": [_P, _I],
    "gf_set_sa_micro": [_P, _I],
    "gf_set_sa_trace": [_P, _P],
    "gf_set_slab": [_P, _I, _I],
    "gf_group_sweep": [_P, _I, _I, ctypes.c_double, _I],
    "gf_group_fix": [_P, _I, ctypes.POINTER(gf_fix_params), _P],
    "gf_sweep_half": [_P, _I, ctypes.c_double, _I, _I, ctypes.c_uint64],
    "gf_slab_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "gf_slab_pack": [_P, _I, _I, _P],
    "gf_slab_unpack": [_P, _I, _I, _P],
    "gf_get_links_per_thread": [_P, _PI],
    "gf_autotune": [_P, _I, _PI, _PD],
    "gf_fix": [_P, ctypes.POINTER(gf_fix_params), ctypes.POINTER(gf_fix_result)],
    "gf_protocol": [_P, ctypes.POINTER(gf_protocol_params), ctypes.POINTER(gf_fix_result)],
    "gf_get_info": [_P, _PI, _PI, _PI, _PI, _PI],
    "gf_philox": [ctypes.c_uint64, _P, ctypes.c_size_t, _P],
    "gf_set_profiling": [_P, _I],
    "gf_kernel_stats": [_P, _I, ctypes.POINTER(ctypes.c_uint64), _PD],
    "gf_launch_count": [_P, ctypes.POINTER(ctypes.c_uint64)],
    "gf_functional_theta_noalloc": [_PI, _I, _P, _P, _P, _P, _P, _P],
    "gf_server_create": [ctypes.c_size_t, _I, ctypes.POINTER(_P)],
    "gf_server_create_mock": [ctypes.c_size_t, _I, _D, ctypes.POINTER(_P)],
    "gf_server_submit": [_P, ctypes.POINTER(gf_job)],
    "gf_server_poll": [_P, _P, _I, _I, _PI],
    "gf_server_status": [_P, _PI, _PI, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_size_t)],
    "gf_server_cancel": [_P, ctypes.c_uint64, _PI],
}
_lib = None


def lib():
    """Load libgf.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_1212_5221_gb300.build.build_all()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIG.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _I
        L.gf_destroy.argtypes = [_P]
        L.gf_destroy.restype = None
        L.gf_server_destroy.argtypes = [_P]
        L.gf_server_destroy.restype = None
        L.gf_strerror.argtypes = [_I]
        L.gf_strerror.restype = ctypes.c_char_p
        L.gf_last_error.argtypes = []
        L.gf_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int, where: str):
    if status != GF_OK:
        msg = lib().gf_last_error().decode()
        raise GFError(status, where, msg or lib().gf_strerror(status).decode())


def _dims(dims):
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4:
        raise ValueError("dims must be (Nt, Nx, Ny, Nz)")
    return (ctypes.c_int * 4)(*dims)


def _enum(v, table):
    return table[v] if isinstance(v, str) else int(v)


def _links_arg(U, dims_nt=None):
    if not isinstance(U, np.ndarray) or U.dtype != np.complex128 or not U.flags.c_contiguous:
        raise ValueError("links must be a C-contiguous complex128 numpy array")
    return U.ctypes.data


def gf_strerror(status: int) -> str:
    return lib().gf_strerror(status).decode()


def gf_last_error() -> str:
    return lib().gf_last_error().decode()


def gf_footprint(dims, n_copies=1, gauge="landau", prec="fp64") -> int:
    out = ctypes.c_size_t()
    _check(lib().gf_footprint(_dims(dims), n_copies, _enum(gauge, GAUGES), _enum(prec, PRECISIONS),
                              ctypes.byref(out)), "gf_footprint")
    return out.value


def gf_create(dims, gauge="landau", prec="fp64", stream=None):
    h = _P()
    _check(lib().gf_create(_dims(dims), _enum(gauge, GAUGES), _enum(prec, PRECISIONS), stream,
                           ctypes.byref(h)), "gf_create")
    return h


def gf_create_batch(dims, n_copies, gauge="landau", prec="fp64", stream=None):
    h = _P()
    _check(lib().gf_create_batch(_dims(dims), n_copies, _enum(gauge, GAUGES), _enum(prec, PRECISIONS), stream,
                                 ctypes.byref(h)), "gf_create_batch")
    return h


def gf_create_ext(dims, n_copies, gauge, prec, stream, device_ptr: int, nbytes: int):
    h = _P()
    _check(lib().gf_create_ext(_dims(dims), n_copies, _enum(gauge, GAUGES), _enum(prec, PRECISIONS), stream,
                               _P(device_ptr), nbytes, ctypes.byref(h)), "gf_create_ext")
    return h


def gf_destroy(h):
    if h:
        lib().gf_destroy(h)


def gf_load_links(h, copy, U):
    _check(lib().gf_load_links(h, copy, _links_arg(U)), "gf_load_links")


def gf_load_links_slab(h, copy, t0, nt, U):
    _check(lib().gf_load_links_slab(h, copy, t0, nt, _links_arg(U)), "gf_load_links_slab")


def gf_load_links_device(h, copy, dev_ptr: int):
    _check(lib().gf_load_links_device(h, copy, _P(dev_ptr)), "gf_load_links_device")


def gf_store_links(h, copy, out):
    _check(lib().gf_store_links(h, copy, _links_arg(out)), "gf_store_links")


def gf_store_links_slab(h, copy, t0, nt, out):
    _check(lib().gf_store_links_slab(h, copy, t0, nt, _links_arg(out)), "gf_store_links_slab")


def gf_store_links_device(h, copy, dev_ptr: int):
    _check(lib().gf_store_links_device(h, copy, _P(dev_ptr)), "gf_store_links_device")


def gf_random_gauge_transform(h, seed):
    _check(lib().gf_random_gauge_transform(h, int(seed) & (2**64 - 1)), "gf_random_gauge_transform")


def _ncopies(h):
    n = ctypes.c_int()
    _check(lib().gf_get_info(h, None, ctypes.byref(n), None, None, None), "gf_get_info")
    return n.value


def gf_sweep(h, algo, param=1.0, n_sweeps=1, seed=0, observables=True):
    n = _ncopies(h)
    F = np.zeros(n)
    T = np.zeros(n)
    _check(lib().gf_sweep(h, _enum(algo, ALGOS), float(param), int(n_sweeps), int(seed) & (2**64 - 1),
                          F.ctypes.data if observables else None, T.ctypes.data if observables else None),
           "gf_sweep")
    return (F, T) if observables else None


def gf_anneal(h, T0, T1, n_steps, seed=0, observables=True):
    n = _ncopies(h)
    F = np.zeros(n)
    T = np.zeros(n)
    _check(lib().gf_anneal(h, float(T0), float(T1), int(n_steps), int(seed) & (2**64 - 1),
                           F.ctypes.data if observables else None, T.ctypes.data if observables else None),
           "gf_anneal")
    return (F, T) if observables else None


def gf_reunitarize(h):
    _check(lib().gf_reunitarize(h), "gf_reunitarize")


def gf_functional_theta(h):
    n = _ncopies(h)
    F = np.zeros(n)
    T = np.zeros(n)
    _check(lib().gf_functional_theta(h, F.ctypes.data, T.ctypes.data), "gf_functional_theta")
    return F, T


def gf_slice_functional_theta(h):
    dims = (ctypes.c_int * 4)()
    n = ctypes.c_int()
    _check(lib().gf_get_info(h, dims, ctypes.byref(n), None, None, None), "gf_get_info")
    F = np.zeros((n.value, dims[0]))
    T = np.zeros((n.value, dims[0]))
    _check(lib().gf_slice_functional_theta(h, F.ctypes.data, T.ctypes.data), "gf_slice_functional_theta")
    return F, T


def gf_promote(h):
    _check(lib().gf_promote(h), "gf_promote")


def gf_set_active(h, flags=None):
    arr = None if flags is None else np.ascontiguousarray(flags, dtype=np.int32)
    _check(lib().gf_set_active(h, None if arr is None else arr.ctypes.data), "gf_set_active")


def gf_get_sweep_index(h):
    v = ctypes.c_uint64()
    _check(lib().gf_get_sweep_index(h, ctypes.byref(v)), "gf_get_sweep_index")
    return v.value


def gf_set_sweep_index(h, index):
    _check(lib().gf_set_sweep_index(h, int(index)), "gf_set_sweep_index")


def gf_set_copy_base(h, base):
    _check(lib().gf_set_copy_base(h, int(base)), "gf_set_copy_base")


def gf_set_links_per_thread(h, lpt):
    _check(lib().gf_set_links_per_thread(h, int(lpt)), "gf_set_links_per_thread")


GF_PREFETCH_NONE, GF_PREFETCH_L2, GF_PREFETCH_SMEM = 0, 1, 2
PREFETCH = {"none": 0, "l2": 1, "smem": 2}


def gf_sweep_async(h, algo, param=1.0, n_sweeps=1, seed=0):
    """Enqueue n sweeps on the context's stream and return (gf_synchronize waits)."""
    _check(lib().gf_sweep_async(h, _enum(algo, ALGOS), float(param), int(n_sweeps), int(seed) & (2**64 - 1)),
           "gf_sweep_async")


def gf_anneal_async(h, T0, T1, n_steps, seed=0):
    _check(lib().gf_anneal_async(h, float(T0), float(T1), int(n_steps), int(seed) & (2**64 - 1)), "gf_anneal_async")


def gf_random_gauge_transform_async(h, seed):
    _check(lib().gf_random_gauge_transform_async(h, int(seed) & (2**64 - 1)), "gf_random_gauge_transform_async")


def gf_synchronize(h):
    _check(lib().gf_synchronize(h), "gf_synchronize")


def gf_set_stage_wait_polls(h, polls=-1):
    """Polls of a shared-memory staging wait before it gives up (-1 default, 0 at once)."""
    _check(lib().gf_set_stage_wait_polls(h, int(polls)), "gf_set_stage_wait_polls")


def gf_set_check_log(h, path):
    """Append one JSON line per convergence check of gf_fix / gf_protocol to path (None stops)."""
    _check(lib().gf_set_check_log(h, None if path is None else os.fsencode(path)), "gf_set_check_log")


def gf_set_graphs(h, on=True):
    """Replay blocks of plain overrelaxation sweeps as CUDA graphs (default on)."""
    _check(lib().gf_set_graphs(h, 1 if on else 0), "gf_set_graphs")


def gf_set_prefetch(h, mode=GF_PREFETCH_L2):
    """How the sweep kernels fetch a block's next tile: "none" / "l2" / "smem"
    (or 0 / 1 / 2; True means "l2", False "none")."""
    if isinstance(mode, str):
        mode = PREFETCH[mode]
    elif isinstance(mode, bool):
        mode = GF_PREFETCH_L2 if mode else GF_PREFETCH_NONE
    _check(lib().gf_set_prefetch(h, int(mode)), "gf_set_prefetch")


def gf_set_fused_observables(h, on=True):
    _check(lib().gf_set_fused_observables(h, 1 if on else 0), "gf_set_fused_observables")


def gf_set_sa_micro(h, n_micro=3):
    """Microcanonical sweeps after each heat-bath sweep (3 by default; 0 = heat bath alone)."""
    _check(lib().gf_set_sa_micro(h, int(n_micro)), "gf_set_sa_micro")


def gf_set_sa_trace(h, device_ptr):
    """Record heat-bath trial counts into int32 device memory of n_copies*V*3
    entries ([copy][site][subgroup]); 0 or None turns the record off."""
    _check(lib().gf_set_sa_trace(h, ctypes.c_void_p(int(device_ptr) if device_ptr else 0)), "gf_set_sa_trace")


GF_SLAB_OWNED, GF_SLAB_BOUNDARY, GF_SLAB_INNER = 0, 1, 2
GF_GROUP_MAX = 48


def _group(handles):
    arr = (_P * len(handles))(*handles)
    return arr, len(handles)


def gf_group_sweep(handles, algo="or", param=1.7, n_sweeps=1):
    """n_sweeps sweeps of every context in `handles` (any extents, one gauge), one launch per half-sweep."""
    arr, n = _group(handles)
    _check(lib().gf_group_sweep(arr, n, _enum(algo, ALGOS), float(param), int(n_sweeps)), "gf_group_sweep")


def gf_group_fix(handles, algo="or", param=1.7, theta_target=1e-12, max_sweeps=100000, check_interval=10,
                 reunit_interval=100, switch_theta=1e-8, raise_on_notconv=True):
    """gf_fix of every context in `handles`, sharing the sweep launches; a list of result dicts."""
    arr, n = _group(handles)
    p = gf_fix_params(_enum(algo, ALGOS), float(param), float(theta_target), int(max_sweeps),
                      int(check_interval), int(reunit_interval), float(switch_theta), 0)
    res = (gf_fix_result * n)()
    st = lib().gf_group_fix(arr, n, ctypes.byref(p), res)
    if not (st == GF_ENOTCONV and not raise_on_notconv):
        _check(st, "gf_group_fix")
    return [res[k].as_dict() for k in range(n)]


def gf_set_slab(h, t0, Nt_global):
    """Make the context the time slab owning global slices [t0, t0 + local Nt - 2)."""
    _check(lib().gf_set_slab(h, int(t0), int(Nt_global)), "gf_set_slab")


def gf_sweep_half(h, algo, param, parity, part=GF_SLAB_OWNED, seed=0):
    """One half-sweep of the sites of (global) parity `parity`, enqueued on the context's stream."""
    _check(lib().gf_sweep_half(h, _enum(algo, ALGOS), float(param), int(parity), int(part),
                               int(seed) & (2**64 - 1)), "gf_sweep_half")


def gf_slab_bytes(h):
    v = ctypes.c_size_t()
    _check(lib().gf_slab_bytes(h, ctypes.byref(v)), "gf_slab_bytes")
    return v.value


def gf_slab_pack(h, slice_, parity, buf_ptr: int):
    _check(lib().gf_slab_pack(h, int(slice_), int(parity), ctypes.c_void_p(int(buf_ptr))), "gf_slab_pack")


def gf_slab_unpack(h, slice_, parity, buf_ptr: int):
    _check(lib().gf_slab_unpack(h, int(slice_), int(parity), ctypes.c_void_p(int(buf_ptr))), "gf_slab_unpack")


def gf_get_links_per_thread(h):
    v = ctypes.c_int()
    _check(lib().gf_get_links_per_thread(h, ctypes.byref(v)), "gf_get_links_per_thread")
    return v.value


def gf_autotune(h, algo="or"):
    best = ctypes.c_int()
    ms = ctypes.c_double()
    _check(lib().gf_autotune(h, _enum(algo, ALGOS), ctypes.byref(best), ctypes.byref(ms)), "gf_autotune")
    return best.value, ms.value


def gf_fix(h, algo="or", param=1.7, theta_target=1e-12, max_sweeps=100000, check_interval=10,
           reunit_interval=100, switch_theta=1e-8, seed=0, raise_on_notconv=True):
    p = gf_fix_params(_enum(algo, ALGOS), float(param), float(theta_target), int(max_sweeps),
                      int(check_interval), int(reunit_interval), float(switch_theta), int(seed))
    r = gf_fix_result()
    st = lib().gf_fix(h, ctypes.byref(p), ctypes.byref(r))
    if st == GF_ENOTCONV and not raise_on_notconv:
        return r.as_dict()
    _check(st, "gf_fix")
    return r.as_dict()


def gf_protocol(h, sa_steps, T_start, T_end, sr_sweeps=0, sr_p=0.5, sr_theta=0.0, seed=0, omega=1.35,
                theta_target=1e-12, max_sweeps=100000, check_interval=10, reunit_interval=100,
                switch_theta=1e-8, raise_on_notconv=True):
    fix = gf_fix_params(GF_OR, float(omega), float(theta_target), int(max_sweeps), int(check_interval),
                        int(reunit_interval), float(switch_theta), int(seed))
    p = gf_protocol_params(int(sa_steps), float(T_start), float(T_end), int(sr_sweeps), float(sr_p),
                           float(sr_theta), int(seed), fix)
    r = gf_fix_result()
    st = lib().gf_protocol(h, ctypes.byref(p), ctypes.byref(r))
    if st == GF_ENOTCONV and not raise_on_notconv:
        return r.as_dict()
    _check(st, "gf_protocol")
    return r.as_dict()


def gf_get_info(h):
    dims = (ctypes.c_int * 4)()
    n, g, p, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().gf_get_info(h, dims, ctypes.byref(n), ctypes.byref(g), ctypes.byref(p), ctypes.byref(f)),
           "gf_get_info")
    return dict(dims=tuple(dims), n_copies=n.value, gauge=g.value, precision=p.value, storage_fp64=bool(f.value))


def gf_set_profiling(h, on=True):
    _check(lib().gf_set_profiling(h, 1 if on else 0), "gf_set_profiling")


def gf_kernel_stats(h, kind):
    """(launches, total device ms) of one kernel class since profiling was enabled."""
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(lib().gf_kernel_stats(h, int(kind), ctypes.byref(n), ctypes.byref(ms)), "gf_kernel_stats")
    return n.value, ms.value


def gf_launch_count(h):
    n = ctypes.c_uint64()
    _check(lib().gf_launch_count(h, ctypes.byref(n)), "gf_launch_count")
    return n.value


def gf_functional_theta_noalloc(dims, gauge, device_links_ptr: int, stream=None):
    """F and theta of natural-order FP64 links in device memory, without any
    device allocation (see include/gf.h).  Returns (F, theta, F_t, theta_t)."""
    nt = int(dims[0])
    F, T = ctypes.c_double(), ctypes.c_double()
    Ft, Tt = np.zeros(nt), np.zeros(nt)
    _check(lib().gf_functional_theta_noalloc(_dims(dims), _enum(gauge, GAUGES), _P(device_links_ptr), stream,
                                             ctypes.byref(F), ctypes.byref(T), Ft.ctypes.data, Tt.ctypes.data),
           "gf_functional_theta_noalloc")
    return F.value, T.value, Ft, Tt


def gf_server_create(hbm_bytes, slots):
    h = _P()
    _check(lib().gf_server_create(int(hbm_bytes), int(slots), ctypes.byref(h)), "gf_server_create")
    return h


def gf_server_create_mock(hbm_bytes, slots, seconds_per_gb):
    h = _P()
    _check(lib().gf_server_create_mock(int(hbm_bytes), int(slots), float(seconds_per_gb), ctypes.byref(h)),
           "gf_server_create_mock")
    return h


def gf_server_submit(s, dims, gauge="landau", prec="mixed", host_links=None, orbit_seed=0, tag=0,
                     host_out=None, algo="or", param=1.7, theta_target=1e-12, max_sweeps=100000,
                     check_interval=20, reunit_interval=100, switch_theta=1e-8, anneal=None):
    """Queue a job; host_links / host_out (numpy complex128, natural order) must stay
    alive until the job's result has been polled.  anneal: None (gf_fix), or a dict
    with sa_steps, T_start, T_end, sr_sweeps, sr_p, sr_theta, seed for gf_protocol
    (whose overrelaxation stage takes the other fix arguments)."""
    j = gf_job()
    j.dims[:] = [int(d) for d in dims]
    j.gauge = _enum(gauge, GAUGES)
    j.prec = _enum(prec, PRECISIONS)
    j.host_links = None if host_links is None else _links_arg(host_links)
    j.orbit_seed = int(orbit_seed)
    j.fix = gf_fix_params(_enum(algo, ALGOS), float(param), float(theta_target), int(max_sweeps),
                          int(check_interval), int(reunit_interval), float(switch_theta), 0)
    j.host_out = None if host_out is None else _links_arg(host_out)
    j.tag = int(tag)
    if anneal:
        a = dict(sa_steps=0, T_start=1.45, T_end=0.01, sr_sweeps=0, sr_p=0.5, sr_theta=0.0, seed=0)
        a.update(anneal)
        j.anneal = 1
        j.protocol = gf_protocol_params(int(a["sa_steps"]), float(a["T_start"]), float(a["T_end"]),
                                        int(a["sr_sweeps"]), float(a["sr_p"]), float(a["sr_theta"]),
                                        int(a["seed"]), j.fix)
    _check(lib().gf_server_submit(s, ctypes.byref(j)), "gf_server_submit")


def gf_server_poll(s, max_results=64, wait_ms=0):
    arr = (gf_job_result * max_results)()
    n = ctypes.c_int()
    _check(lib().gf_server_poll(s, arr, max_results, int(wait_ms), ctypes.byref(n)), "gf_server_poll")
    return [arr[k].as_dict() for k in range(n.value)]


def gf_server_status(s):
    q, r = ctypes.c_int(), ctypes.c_int()
    c, b = ctypes.c_uint64(), ctypes.c_size_t()
    _check(lib().gf_server_status(s, ctypes.byref(q), ctypes.byref(r), ctypes.byref(c), ctypes.byref(b)),
           "gf_server_status")
    return dict(queued=q.value, running=r.value, completed=c.value, bytes_in_use=b.value)


def gf_server_cancel(s, tag):
    """Remove the queued jobs with this tag (reported with GF_ECANCELED); returns how many."""
    n = ctypes.c_int()
    _check(lib().gf_server_cancel(s, int(tag), ctypes.byref(n)), "gf_server_cancel")
    return n.value


def gf_server_destroy(s):
    if s:
        lib().gf_server_destroy(s)


def gf_philox(seed, counters):
    """Device Philox4x32-10 of an (n, 4) uint32 array of counters."""
    c = np.ascontiguousarray(counters, dtype=np.uint32)
    if c.ndim != 2 or c.shape[1] != 4:
        raise ValueError("counters must have shape (n, 4)")
    out = np.empty_like(c)
    _check(lib().gf_philox(int(seed) & (2**64 - 1), c.ctypes.data, c.shape[0], out.ctypes.data), "gf_philox")
    return out


_CUDA_STREAM_LEGACY = 0x1  # the CUDA runtime's handle of the legacy default stream


class GaugeField:
    """A context whose device memory and stream are PyTorch's.

    The buffer is a torch uint8 CUDA tensor of gf_footprint bytes and work is
    issued on a torch.cuda.Stream created for the field (or the one given).
    """

    def __init__(self, dims, gauge="landau", prec="fp64", n_copies=1, device=None, stream=None):
        import torch

        self.dims = tuple(int(d) for d in dims)
        self.n_copies = int(n_copies)
        nbytes = gf_footprint(self.dims, self.n_copies, gauge, prec)
        dev = torch.device("cuda" if device is None else device)
        self.buffer = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        ptr = self.buffer.data_ptr()
        aligned = (ptr + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream(dev)
        # torch's default stream has the handle 0, which the C ABI reads as "create a
        # stream of your own": pass the legacy default stream's handle instead, so
        # that the library's work and torch's are ordered on the same stream
        handle = self.stream.cuda_stream or _CUDA_STREAM_LEGACY
        self.h = gf_create_ext(self.dims, self.n_copies, gauge, prec, _P(handle), aligned,
                               nbytes + 256 - (aligned - ptr))

    def close(self):
        if getattr(self, "h", None):
            gf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
