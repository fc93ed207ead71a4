"""Several lattices of different extents in one launch (gf_group_sweep,
gf_group_fix), through the C ABI: every member comes out exactly as when it
is swept alone with the same links-per-thread, and a group fix reaches the
oracle's functional member by member."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SPECS = [(4, 4, 4, 4), (6, 4, 6, 10), (8, 8, 8, 8), (4, 6, 8, 4), (10, 6, 4, 6)]


@pytest.fixture(scope="module")
def gf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_5221_gb300 import build, gf

    build.build_lib()
    return gf


def _fields(synth, orc, specs, eps=0.4):
    out = []
    for k, d in enumerate(specs):
        U = synth.links(d, "smooth", eps, 20 + k)
        orc.random_gauge_transform(U, 40 + k)
        out.append(U)
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("gauge", ["landau", "coulomb", "mag"])
def test_group_sweep_equals_alone(gf, synth, orc, gauge, prec):
    fields = _fields(synth, orc, SPECS)
    lpt = 8 if prec == "fp64" else 4
    hs = [gf.gf_create_batch(d, 2 if k == 2 else 1, gauge, prec) for k, d in enumerate(SPECS)]
    try:
        for h, U in zip(hs, fields):
            gf.gf_set_links_per_thread(h, lpt)
            gf.gf_load_links(h, -1, U)
        gf.gf_group_sweep(hs, "or", 1.7, 3)
        got = []
        for k, (h, U) in enumerate(zip(hs, fields)):
            V = np.empty_like(U)
            gf.gf_store_links(h, 0, V)
            got.append(V)
            assert gf.gf_get_sweep_index(h) == 3
    finally:
        for h in hs:
            gf.gf_destroy(h)
    for k, (d, U) in enumerate(zip(SPECS, fields)):
        h = gf.gf_create_batch(d, 2 if k == 2 else 1, gauge, prec)
        try:
            gf.gf_set_links_per_thread(h, lpt)
            gf.gf_load_links(h, -1, U)
            gf.gf_sweep(h, "or", 1.7, 3, observables=False)
            V = np.empty_like(U)
            gf.gf_store_links(h, 0, V)
        finally:
            gf.gf_destroy(h)
        if prec == "fp64" or gauge != "mag":
            assert np.array_equal(got[k], V), (k, np.abs(got[k] - V).max())
        else:  # the FP32 MAG form of two separately compiled kernels rounds alike only to FP32 rounding
            assert np.abs(got[k] - V).max() <= 2e-5, (k, np.abs(got[k] - V).max())
        if prec == "fp64":
            W = U.copy()
            orc.sweep(W, gauge, "or", 1.7, 3)
            assert np.abs(V - W).max() <= 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("gauge", ["landau", "coulomb", "mag"])
def test_group_fix(gf, synth, orc, gauge, prec):
    """Every member reaches theta < 1e-11 (the oracle's theta of the stored
    links agrees); in FP64 each member's run is, link for link, the same
    member fixed alone with the same cadence (sweeps of 10, then the check)."""
    specs = SPECS[:4]
    fields = _fields(synth, orc, specs, 0.3)
    omega = 1.35 if gauge == "mag" else 1.7
    hs = [gf.gf_create(d, gauge, prec) for d in specs]
    out = []
    try:
        for h, U in zip(hs, fields):
            gf.gf_set_links_per_thread(h, 8 if prec == "fp64" else 4)
            gf.gf_load_links(h, 0, U)
        res = gf.gf_group_fix(hs, "or", omega, 1e-11, max_sweeps=40000, check_interval=10, reunit_interval=0)
        for h, U in zip(hs, fields):
            V = np.empty_like(U)
            gf.gf_store_links(h, 0, V)
            out.append(V)
    finally:
        for h in hs:
            gf.gf_destroy(h)
    for k, (d, U, r, V) in enumerate(zip(specs, fields, res, out)):
        assert r["converged"] and r["theta_max"] < 1e-11
        _, th_o, _, tt_o = orc.observables(V, gauge)
        assert (tt_o.max() if gauge == "coulomb" else th_o) < 1.01e-11, k
        if prec != "fp64":
            continue
        h = gf.gf_create(d, gauge, prec)
        try:
            gf.gf_set_links_per_thread(h, 8)
            gf.gf_load_links(h, 0, U)
            n = 0
            act = np.ones(d[0], np.int32)
            while True:
                Ft, Tt = gf.gf_slice_functional_theta(h)
                if gauge == "coulomb":
                    act = (Tt[0] >= 1e-11).astype(np.int32)
                    if not act.any():
                        break
                    gf.gf_set_active(h, act)
                elif Tt[0].mean() < 1e-11:
                    break
                gf.gf_sweep(h, "or", omega, 10, observables=False)
                n += 10
            gf.gf_set_active(h, None)
            W = np.empty_like(U)
            gf.gf_store_links(h, 0, W)
        finally:
            gf.gf_destroy(h)
        assert r["sweeps"] == n and np.array_equal(V, W), k


def test_group_arguments(gf):
    h1 = gf.gf_create((4, 4, 4, 4), "landau", "fp64")
    h2 = gf.gf_create((4, 4, 4, 4), "mag", "fp64")
    h3 = gf.gf_create((4, 4, 4, 4), "landau", "mp")
    try:
        for bad in ([h1, h2], [h1, h1], [h1, h3], []):
            with pytest.raises(gf.GFError) as e:
                gf.gf_group_sweep(bad, "or", 1.7, 1)
            assert e.value.code == gf.GF_EINVAL
        with pytest.raises(gf.GFError):
            gf.gf_group_sweep([h1], "sa", 1.0, 1)
    finally:
        for h in (h1, h2, h3):
            gf.gf_destroy(h)
