"""Time-slab decomposition of one Landau or MAG lattice over several processes
(Sec. 5 of Schroeck & Vogt): the schedule and the communication.

Each process owns nt consecutive time-slices [t0, t0 + nt) and keeps a halo
copy of slice t0 - 1.  A site's update needs U_0(x - 0), which for the first
owned slice lives in the halo; its update then changes that halo link, whose
owner is the previous process.  Every link has exactly one active endpoint in
a half-sweep, so after the half-sweep of parity p two messages travel on the
ring (Sec. 5.1):

  * to the previous process: the halo U_0 of the sites (t0 - 1, x) of parity
    1 - p (changed as down-links of the active sites (t0, x));
  * to the next process: U_0 of the last owned slice at the sites of parity
    p (changed as up-links of those active sites), for its halo.

Each is U_0, rows 0 and 1, of one parity of one slice: 1/12 of a time-slice
(Sec. 5.2).  The first and last owned slices are updated first and their
messages are posted before the inner slices run, so the exchange overlaps
with the inner update (Sec. 5.3).  F and theta are sums over the owned
slices, reduced over the processes in FP64.

Everything device-side (the half-sweeps, packing the messages, the slice
observables) is libgf's; this module only sequences those calls and moves
the buffers with torch.distributed (NCCL for device buffers, gloo on CPU).
The schedule talks to a `backend` with the methods half(algo, param, parity,
part, seed), pack(slice, parity), unpack(slice, parity, buf),
slice_observables(), advance(), reunitarize() and stream_context() (the
stream the messages are ordered on), so the same schedule drives a GPU slab
(`GpuSlab`) or any other implementation of those steps.
"""
from __future__ import annotations

import numpy as np

from . import gf

OWNED, BOUNDARY, INNER = gf.GF_SLAB_OWNED, gf.GF_SLAB_BOUNDARY, gf.GF_SLAB_INNER


def slab_bounds(Nt: int, world: int, rank: int) -> tuple[int, int]:
    """(t0, nt) of rank's slab: Nt split into `world` equal even slabs."""
    if Nt % world or (Nt // world) % 2 or Nt // world < 2:
        raise ValueError(f"Nt = {Nt} does not split into {world} even slabs of >= 2 slices")
    nt = Nt // world
    return rank * nt, nt


def local_slices(U_global: np.ndarray, t0: int, nt: int) -> np.ndarray:
    """The nt + 2 global slices a slab holds, t0 - 1 .. t0 + nt (periodic)."""
    Nt = U_global.shape[0]
    idx = [(t0 - 1 + k) % Nt for k in range(nt + 2)]
    return np.ascontiguousarray(U_global[idx])


class Ring:
    """Neighbour exchange on the ring of processes through torch.distributed.

    start(to_prev, to_next) posts the two sends and two receives and returns
    a handle; finish(handle) waits and returns (from_prev, from_next).  With
    one process the messages go to itself.  For two processes the previous
    and next process coincide: the messages are told apart by their tags
    (gloo) and by their posting order (NCCL matches a pair's operations in
    order), which is the same on every rank: the message to the next process
    first."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0

    def start(self, to_prev, to_next):
        if self.world == 1:
            return (to_next.clone(), to_prev.clone())
        dist = self.dist
        prev = (self.rank - 1) % self.world
        nxt = (self.rank + 1) % self.world
        from_prev = to_next.new_empty(to_next.shape)
        from_next = to_prev.new_empty(to_prev.shape)
        ops = [dist.P2POp(dist.isend, to_next, nxt, self.group, tag=0),
               dist.P2POp(dist.isend, to_prev, prev, self.group, tag=1),
               dist.P2POp(dist.irecv, from_prev, prev, self.group, tag=0),
               dist.P2POp(dist.irecv, from_next, nxt, self.group, tag=1)]
        works = dist.batch_isend_irecv(ops)
        return (works, from_prev, from_next)

    def finish(self, handle):
        if self.world == 1:
            return handle
        works, from_prev, from_next = handle
        for w in works:
            w.wait()
        return from_prev, from_next

    def allreduce_sum(self, values):
        """FP64 sum over the processes (a host float64 array in, the sum out)."""
        import torch

        t = torch.as_tensor(np.asarray(values, np.float64))
        if self.world > 1:
            dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
            t = t.to(dev)
            self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()


class TimeSlab:
    """The schedule of Sec. 5: half-sweeps with the boundary exchange."""

    def __init__(self, backend, ring: Ring, nt: int, Nt_global: int, gauge: str):
        self.b = backend
        self.ring = ring
        self.nt = nt
        self.Nt = Nt_global
        self.gauge = gauge

    def half(self, algo, param, p, seed=0):
        b, nt = self.b, self.nt
        # the messages' buffers, copies and point-to-point operations are
        # ordered on the backend's stream, behind the half-sweeps
        with b.stream_context():
            b.half(algo, param, p, BOUNDARY, seed)
            handle = self.ring.start(b.pack(0, 1 - p), b.pack(nt, p))
            b.half(algo, param, p, INNER, seed)
            from_prev, from_next = self.ring.finish(handle)
            b.unpack(0, p, from_prev)
            b.unpack(nt, 1 - p, from_next)

    def sweep(self, algo, param, n_sweeps=1, seed=0):
        """n checkerboard sweeps (even half, then odd) of the whole lattice."""
        for _ in range(n_sweeps):
            for p in (0, 1):
                self.half(algo, param, p, seed)
            self.b.advance()

    def anneal_step(self, T, seed, n_micro=3):
        """One simulated-annealing step (Sec. 2.3): heat bath + n_micro
        microcanonical sweeps."""
        self.sweep("sa", T, 1, seed)
        self.sweep("micro", 0.0, n_micro, seed)

    def functional_theta(self):
        """(F, theta) of the whole lattice: owned slices summed, reduced in FP64."""
        F_t, th_t = self.b.slice_observables()
        sums = self.ring.allreduce_sum([F_t[1:self.nt + 1].sum(), th_t[1:self.nt + 1].sum()])
        return sums[0] / self.Nt, sums[1] / self.Nt

    def fix(self, algo="or", param=1.7, theta_target=1e-12, max_sweeps=100000, check_interval=20, seed=0,
            reunit_interval=100):
        """Sweep until theta < theta_target (every process decides on the same
        reduced theta); returns (sweeps, F, theta)."""
        n = 0
        since = 0
        while True:
            F, th = self.functional_theta()
            if th < theta_target or n >= max_sweeps:
                return n, F, th
            k = min(check_interval, max_sweeps - n)
            self.sweep(algo, param, k, seed)
            n += k
            since += k
            if reunit_interval and since >= reunit_interval:
                self.b.reunitarize()
                since = 0


class GpuSlab:
    """One process's slab on its GPU: a libgf context in time-slab mode."""

    def __init__(self, dims_global, t0, nt, gauge="landau", prec="fp64", stream=None):
        import torch

        self.torch = torch
        self.dims = (nt + 2,) + tuple(dims_global[1:])
        self.t0, self.nt = t0, nt
        # one stream for the library's work and for the messages: the schedule
        # makes it current around each half-sweep, so torch.distributed orders
        # the boundary messages behind the half-sweeps and copies libgf enqueues
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.field = gf.GaugeField(self.dims, gauge, prec, stream=self.stream)
        self.h = self.field.h
        gf.gf_set_slab(self.h, t0, dims_global[0])
        self.msg_bytes = gf.gf_slab_bytes(self.h)
        self.sweep_index = 0

    def load(self, U_global):
        gf.gf_load_links(self.h, 0, local_slices(U_global, self.t0, self.nt))

    def store_owned(self):
        out = np.empty((self.nt,) + self.dims[1:] + (4, 3, 3), np.complex128)
        gf.gf_store_links_slab(self.h, 0, 1, self.nt, out)
        return out

    def half(self, algo, param, parity, part, seed):
        gf.gf_sweep_half(self.h, algo, param, parity, part, seed)

    def stream_context(self):
        return self.torch.cuda.stream(self.stream)

    def pack(self, slice_, parity):
        with self.torch.cuda.stream(self.stream):
            buf = self.torch.empty(self.msg_bytes, dtype=self.torch.uint8, device="cuda")
        gf.gf_slab_pack(self.h, slice_, parity, buf.data_ptr())
        return buf

    def unpack(self, slice_, parity, buf):
        gf.gf_slab_unpack(self.h, slice_, parity, buf.data_ptr())

    def advance(self):
        self.sweep_index += 1
        gf.gf_set_sweep_index(self.h, self.sweep_index)

    def reunitarize(self):
        gf.gf_reunitarize(self.h)

    def slice_observables(self):
        F_t, th_t = gf.gf_slice_functional_theta(self.h)
        return F_t[0], th_t[0]

    def close(self):
        self.field.close()
