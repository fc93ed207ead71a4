"""The time-slab path (Sec. 5) on one GPU, through the C ABI.

Several slabs of one lattice live in one process on one shared stream and
exchange their boundary messages in memory, in the order the schedule of
paper_1212_5221_gb300.slab uses (every slab updates its boundary slices and
packs its messages, then the inner slices run, then every slab unpacks what
its neighbours sent).  No kernel waits for another, so this is an exact
emulation of the multi-process run.  The result must equal the same sweeps
of the whole lattice in one context bit for bit (same links-per-thread), and
the FP64 oracle to 1e-12.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DIMS = (12, 4, 6, 4)


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_5221_gb300 import build, gf

    build.build_lib()
    return gf


def _field(synth, orc, dims):
    U = synth.links(dims, "smooth", 0.4, 8)
    orc.random_gauge_transform(U, 23)
    return U


def _lockstep(slabs, algo, param, n, seed):
    from paper_1212_5221_gb300 import slab

    W = len(slabs)
    for _ in range(n):
        for p in (0, 1):
            out = []
            for s in slabs:
                s.half(algo, param, p, slab.BOUNDARY, seed)
                out.append((s.pack(0, 1 - p), s.pack(s.nt, p)))
            for s in slabs:
                s.half(algo, param, p, slab.INNER, seed)
            for r, s in enumerate(slabs):
                s.unpack(0, p, out[(r - 1) % W][1])  # the previous slab's message to its next
                s.unpack(s.nt, 1 - p, out[(r + 1) % W][0])  # the next slab's message to its previous
        for s in slabs:
            s.advance()


def _program_slabs(slabs, seed):
    _lockstep(slabs, "or", 1.7, 4, 0)
    _lockstep(slabs, "sa", 0.9, 1, seed)
    _lockstep(slabs, "micro", 0.0, 1, seed)
    _lockstep(slabs, "sr", 0.5, 2, seed)


def _program_whole(gf, h, seed):
    gf.gf_set_sa_micro(h, 1)
    gf.gf_sweep(h, "or", 1.7, 4, 0, observables=False)
    gf.gf_sweep(h, "sa", 0.9, 1, seed, observables=False)
    gf.gf_sweep(h, "sr", 0.5, 2, seed, observables=False)


@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("gauge", ["landau", "mag"])
def test_slabs_equal_whole_lattice(gf, synth, orc, gauge, prec, world):
    from paper_1212_5221_gb300 import slab

    import torch

    lpt = 8 if prec == "fp64" else 4
    U = _field(synth, orc, DIMS)
    slabs = []
    # the emulated processes hand their messages over in memory: one stream
    # orders every slab's packs before the other slabs' unpacks
    stream = torch.cuda.Stream()
    try:
        for r in range(world):
            t0, nt = slab.slab_bounds(DIMS[0], world, r)
            s = slab.GpuSlab(DIMS, t0, nt, gauge, prec, stream=stream)
            gf.gf_set_links_per_thread(s.h, lpt)
            s.load(U)
            slabs.append(s)
        _program_slabs(slabs, 77)
        owned = np.concatenate([s.store_owned() for s in slabs])
        ts = [slab.TimeSlab(s, slab.Ring(), s.nt, DIMS[0], gauge) for s in slabs]
        F_t = np.concatenate([s.slice_observables()[0][1:s.nt + 1] for s in slabs])
        th_t = np.concatenate([s.slice_observables()[1][1:s.nt + 1] for s in slabs])
    finally:
        for s in slabs:
            s.close()
    h = gf.gf_create(DIMS, gauge, prec)
    try:
        gf.gf_set_links_per_thread(h, lpt)
        gf.gf_load_links(h, 0, U)
        _program_whole(gf, h, 77)
        whole = np.empty_like(U)
        gf.gf_store_links(h, 0, whole)
        wF_t, wth_t = gf.gf_slice_functional_theta(h)
    finally:
        gf.gf_destroy(h)
    assert np.array_equal(owned, whole)
    assert np.allclose(F_t, wF_t[0], rtol=1e-13, atol=0) and np.allclose(th_t, wth_t[0], rtol=1e-12, atol=0)
    assert len(ts) == world
    if prec == "fp64":
        W = U.copy()
        orc.sweep(W, gauge, "or", 1.7, 4, 0)
        orc.sweep(W, gauge, "sa", 0.9, 1, 4, 77)
        orc.sweep(W, gauge, "micro", 0.0, 1, 5, 77)
        orc.sweep(W, gauge, "sr", 0.5, 2, 6, 77)
        assert np.abs(owned - W).max() <= 1e-12


def test_time_slab_schedule_one_process_fix(gf, synth, orc):
    """The TimeSlab schedule itself (world size 1: the process is its own
    neighbour) drives a lattice to theta < 1e-12 on the GPU.  Its run equals,
    link for link, the same sequence of sweeps, checks and re-unitarisations
    on one whole-lattice context; the oracle confirms the result: its theta
    of the final links is below 1e-12 and the plaquette is unchanged."""
    from paper_1212_5221_gb300 import slab

    dims = (8, 4, 4, 4)
    U = _field(synth, orc, dims)
    s = slab.GpuSlab(dims, 0, dims[0], "landau", "fp64")
    try:
        gf.gf_set_links_per_thread(s.h, 8)
        s.load(U)
        ts = slab.TimeSlab(s, slab.Ring(), dims[0], dims[0], "landau")
        n, F, th = ts.fix("or", 1.7, 1e-12, max_sweeps=6000, check_interval=20, reunit_interval=100)
        V = s.store_owned()
    finally:
        s.close()
    assert th < 1e-12 and n > 0
    h = gf.gf_create(dims, "landau", "fp64")
    try:
        gf.gf_set_links_per_thread(h, 8)
        gf.gf_load_links(h, 0, U)
        done = since = 0
        while True:
            Fw, Tw = gf.gf_functional_theta(h)
            if Tw[0] < 1e-12 or done >= 6000:
                break
            gf.gf_sweep(h, "or", 1.7, 20, observables=False)
            done += 20
            since += 20
            if since >= 100:
                gf.gf_reunitarize(h)
                since = 0
        W = np.empty_like(U)
        gf.gf_store_links(h, 0, W)
    finally:
        gf.gf_destroy(h)
    assert done == n and np.array_equal(V, W)
    assert abs(F - Fw[0]) <= 1e-13 * abs(F)
    F_o, th_o, _, _ = orc.observables(V, "landau")
    assert th_o < 1e-12 and abs(F_o - F) <= 1e-12 * abs(F)
    assert abs(orc.plaquette(V) - orc.plaquette(U)) < 1e-12


def test_slab_arguments(gf):
    with pytest.raises(gf.GFError):  # Coulomb slices are split as units
        h = gf.gf_create((6, 4, 4, 4), "coulomb", "fp64")
        try:
            gf.gf_set_slab(h, 0, 8)
        finally:
            gf.gf_destroy(h)
    h = gf.gf_create((6, 4, 4, 4), "landau", "fp64")
    try:
        for t0, Nt in ((0, 3), (-1, 8), (8, 8), (0, 2)):
            with pytest.raises(gf.GFError) as e:
                gf.gf_set_slab(h, t0, Nt)
            assert e.value.code == gf.GF_EINVAL
        gf.gf_set_slab(h, 4, 8)
        with pytest.raises(gf.GFError) as e:
            gf.gf_sweep(h, "or", 1.7, 1)
        assert e.value.code == gf.GF_EINVAL
        assert gf.gf_slab_bytes(h) == 6 * 32 * 16
        with pytest.raises(gf.GFError):
            gf.gf_slab_pack(h, 6, 0, 0)
    finally:
        gf.gf_destroy(h)
