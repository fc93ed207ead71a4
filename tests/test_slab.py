"""The time-slab schedule (Sec. 5) on CPU processes with gloo.

The schedule in paper_1212_5221_gb300.slab drives a backend; here the backend
is the FP64 oracle working on the slab's time-slices of the lattice (each
process keeps a full-size array but only its owned slices and its halo slice
are kept current, and it sweeps only the owned slices).  Two processes
exchanging the boundary links after every half-sweep must reproduce the
oracle's sweeps of the whole lattice link for link, and the reduced F and
theta must equal the whole lattice's.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleSlab:
    """A slab backend on the oracle (test double of the GPU slab)."""

    def __init__(self, orc, U_global, t0, nt, gauge):
        self.orc = orc
        self.U = np.ascontiguousarray(U_global.copy())
        self.Nt = U_global.shape[0]
        self.t0, self.nt, self.gauge = t0, nt, gauge
        self.sweep_index = 0
        c = np.indices(U_global.shape[1:4]).sum(0)
        self.spatial_parity = c % 2

    def _glob(self, l):
        return (self.t0 - 1 + l) % self.Nt

    def _flags(self, part):
        from paper_1212_5221_gb300 import slab

        f = np.zeros(self.Nt, np.int32)
        for k in range(self.nt):
            edge = k in (0, self.nt - 1)
            if part == slab.OWNED or (part == slab.BOUNDARY and edge) or (part == slab.INNER and not edge):
                f[(self.t0 + k) % self.Nt] = 1
        return f

    def half(self, algo, param, parity, part, seed):
        self.orc.half_sweep(self.U, self.gauge, algo, param, parity, self.sweep_index, seed, 0, self._flags(part))

    def _mask(self, l, parity):
        t = self._glob(l)
        return t, (self.spatial_parity + t) % 2 == parity

    def pack(self, l, parity):
        t, m = self._mask(l, parity)
        return torch.from_numpy(np.ascontiguousarray(self.U[t][m][:, 0]).view(np.float64).copy())

    def unpack(self, l, parity, buf):
        t, m = self._mask(l, parity)
        self.U[t][m, 0] = buf.numpy().view(np.complex128).reshape(-1, 3, 3)

    def advance(self):
        self.sweep_index += 1

    def stream_context(self):
        import contextlib

        return contextlib.nullcontext()

    def reunitarize(self):
        self.orc.reunitarize(self.U)

    def slice_observables(self):
        _, _, F_t, th_t = self.orc.observables(self.U, self.gauge)
        idx = [self._glob(l) for l in range(self.nt + 2)]
        return F_t[idx], th_t[idx]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


DIMS = (12, 4, 4, 6)


def _field(gauge, dims=DIMS):
    import oracle
    from paper_1212_5221_gb300 import inputs

    inputs.build()
    U = inputs.links(dims, "smooth", 0.4, 5)
    oracle.random_gauge_transform(U, 17)
    return U


def _program(orc, ts):
    """The work every process runs: OR sweeps, then heat-bath steps."""
    ts.sweep("or", 1.7, 3)
    ts.anneal_step(0.8, seed=41, n_micro=1)
    ts.sweep("sr", 0.5, 1, seed=42)
    return ts.functional_theta()


def _worker(rank, world, port, gauge, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1212_5221_gb300 import slab

        oracle.build()
        U = _field(gauge)
        t0, nt = slab.slab_bounds(DIMS[0], world, rank)
        be = OracleSlab(oracle, U, t0, nt, gauge)
        ts = slab.TimeSlab(be, slab.Ring(), nt, DIMS[0], gauge)
        F, th = _program(oracle, ts)
        q.put((rank, t0, be.U[t0:t0 + nt].copy(), F, th))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("gauge", ["landau", "mag"])
def test_process_slabs_equal_whole_lattice(orc, synth, gauge, world):
    """Two processes (each the other's previous and next) and three (distinct
    neighbours) against the whole lattice."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, gauge, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    W = _field(gauge)
    orc.sweep(W, gauge, "or", 1.7, 3, 0)
    orc.sweep(W, gauge, "sa", 0.8, 1, 3, 41)
    orc.sweep(W, gauge, "micro", 0.0, 1, 4, 41)
    orc.sweep(W, gauge, "sr", 0.5, 1, 5, 42)
    F, th, _, _ = orc.observables(W, gauge)
    for rank, t0, owned, Fr, thr in out:
        assert np.array_equal(owned, W[t0:t0 + owned.shape[0]]), rank
        assert abs(Fr - F) <= 1e-14 * abs(F)
        assert abs(thr - th) <= 1e-12 * abs(th)


def _fix_worker(rank, world, port, gauge, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_1212_5221_gb300 import slab

        oracle.build()
        U = _field(gauge)
        t0, nt = slab.slab_bounds(DIMS[0], world, rank)
        be = OracleSlab(oracle, U, t0, nt, gauge)
        ts = slab.TimeSlab(be, slab.Ring(), nt, DIMS[0], gauge)
        n, F, th = ts.fix("or", FIX["omega"], FIX["theta"], max_sweeps=FIX["max"], check_interval=FIX["check"],
                          reunit_interval=FIX["reunit"])
        q.put((rank, t0, be.U[t0:t0 + nt].copy(), n, F, th))
    finally:
        dist.destroy_process_group()


FIX = dict(omega=1.7, theta=1e-10, max=4000, check=10, reunit=50)


def test_process_slabs_fix(orc, synth):
    """The schedule's convergence loop on two processes: every process stops
    after the same sweep count, decided on the FP64 theta reduced over both;
    that count, the links and F equal the same loop (checks every 10 sweeps,
    re-unitarisation every 50) on the whole lattice."""
    world, gauge = 2, "landau"
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_fix_worker, args=(r, world, port, gauge, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    W = _field(gauge)
    done = since = 0
    while True:
        F, th, _, _ = orc.observables(W, gauge)
        if th < FIX["theta"] or done >= FIX["max"]:
            break
        orc.sweep(W, gauge, "or", FIX["omega"], FIX["check"], done)
        done += FIX["check"]
        since += FIX["check"]
        if since >= FIX["reunit"]:
            orc.reunitarize(W)
            since = 0
    assert th < FIX["theta"] and done > 0
    for rank, t0, owned, n, Fr, thr in out:
        assert n == done, rank
        assert np.array_equal(owned, W[t0:t0 + owned.shape[0]]), rank
        assert abs(Fr - F) <= 1e-14 * abs(F) and abs(thr - th) <= 1e-9 * th


def test_one_process_slab_equals_whole_lattice(orc, synth):
    """World size 1: the process is its own neighbour (halo = its last slice)."""
    from paper_1212_5221_gb300 import slab

    U = _field("landau")
    be = OracleSlab(orc, U, 0, DIMS[0], "landau")
    ts = slab.TimeSlab(be, slab.Ring(), DIMS[0], DIMS[0], "landau")
    F1, th1 = _program(orc, ts)
    W = _field("landau")
    orc.sweep(W, "landau", "or", 1.7, 3, 0)
    orc.sweep(W, "landau", "sa", 0.8, 1, 3, 41)
    orc.sweep(W, "landau", "micro", 0.0, 1, 4, 41)
    orc.sweep(W, "landau", "sr", 0.5, 1, 5, 42)
    assert np.array_equal(be.U, W)
    F, th, _, _ = orc.observables(W, "landau")
    assert abs(F1 - F) <= 1e-14 * abs(F) and abs(th1 - th) <= 1e-12 * abs(th)


def test_slab_bounds():
    from paper_1212_5221_gb300 import slab

    assert slab.slab_bounds(64, 4, 3) == (48, 16)
    for bad in ((10, 4), (6, 2), (8, 8)):
        with pytest.raises(ValueError):
            slab.slab_bounds(bad[0], bad[1], 0)
    U = np.arange(6)[:, None] * np.ones((6, 2))
    assert list(slab.local_slices(U, 0, 2)[:, 0]) == [5, 0, 1, 2]
    assert list(slab.local_slices(U, 4, 2)[:, 0]) == [3, 4, 5, 0]
