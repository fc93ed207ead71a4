"""Host check of the shared-memory staging index arithmetic of the FP32 sweep
(GF_PREFETCH_SMEM).  This mirrors, with the same integer semantics, the
functions `stage_range`, `StageGeom`, `stage_issue` and `load_slot` of
paper_1212_5221_gb300/csrc/gf_sweep.cuh (keep the two in step), and checks on
whole lattices that

* every bulk copy reads inside its source array ([0, Vh) of one slot/chunk),
  writes inside its own region of the stage buffer, and the byte count of a
  stage fits the mbarrier transaction count;
* every read a site makes from the stage buffer lies in the copied range of
  the right region, and every read that falls back to global memory is a
  periodic wrap of a down-link;
* the buffers of a block fit the 227 KB a block may use.

It includes the lattice on which a clip in unsigned arithmetic once produced
a copy far past its array (a down-link range ending below zero).
"""
import pytest

BLOCK = 256


def geom(dims):
    nt, nx, ny, nz = dims
    v3 = nx * ny * nz
    return {"n": dims, "Vh": v3 * nt // 2, "stride": [v3, ny * nz, nz, 1]}


def coords(G, sp, p):
    n = G["n"]
    s0 = 2 * sp
    q1, z0 = divmod(s0, n[3])
    q2, y = divmod(q1, n[2])
    t, x = divmod(q2, n[1])
    b = ((t + x + y) ^ p) & 1
    return [t, x, y, z0 + b], s0 + b


def stage_range(G, sp0, tile, k):
    """lo (int64), clo, chi (uint32) as the C++ computes them."""
    ext, lo = tile, sp0
    if k < 8 and (k & 1):
        mu = k >> 1
        st = G["stride"][mu] if mu < 3 else 0
        lo = sp0 - st // 2 - 1
        ext = tile + 2
    c0 = 0 if lo < 0 else lo
    c1 = lo + ext
    if c1 > G["Vh"]:
        c1 = G["Vh"]
    if c0 > G["Vh"]:
        c0 = G["Vh"]
    if c1 < c0:
        c1 = c0
    assert 0 <= c0 < 2 ** 32 and 0 <= c1 < 2 ** 32
    return lo, c0, c1


def check(dims, lpt, gauge, acc):
    G = geom(dims)
    Vh = G["Vh"]
    tile = BLOCK // (8 // lpt)
    RS = tile + 3
    ACC0 = 24 * RS
    VEC = 24 * RS + 3 * tile
    base = lambda k, c: (k * 3 + c) * RS if k < 8 else ACC0 + c * tile
    stride = lambda k: RS if k < 8 else tile
    extent = lambda k: tile + 2 if k < 8 else tile
    assert RS % 2 == 1
    assert 2 * VEC * 16 + 16 <= 227 * 1024
    use_acc = acc and gauge != "coulomb"
    for p in (0, 1):
        for t in range((Vh + tile - 1) // tile):
            sp0 = t * tile
            copied, total = {}, 0
            for lane in range(32):  # stage_issue
                if not (lane < 24 or (use_acc and lane < 27)):
                    continue
                k = lane // 3 if lane < 24 else 8
                c = lane % 3 if lane < 24 else lane - 24
                if gauge == "coulomb" and k == 1:
                    continue
                lo, clo, chi = stage_range(G, sp0, tile, k)
                if chi <= clo:
                    continue
                assert 0 <= clo < chi <= Vh
                d0 = base(k, c) + (clo - lo)
                assert base(k, c) <= d0 and d0 + (chi - clo) <= base(k, c) + extent(k) <= VEC
                total += (chi - clo) * 16
                copied[(k, c)] = (clo, chi)
            assert total < (1 << 20)
            for local in range(tile):  # load_slot of every valid site
                sp = sp0 + local
                if sp >= Vh:
                    continue
                c4, s = coords(G, sp, p)
                for k in range(9):
                    if (k == 8 and not use_acc) or (gauge == "coulomb" and k == 1):
                        continue
                    idx = sp
                    if k < 8 and (k & 1):
                        mu = k >> 1
                        st = G["stride"][mu]
                        idx = (s - st if c4[mu] > 0 else s + (dims[mu] - 1) * st) >> 1
                    assert 0 <= idx < Vh
                    lo, clo, chi = stage_range(G, sp0, tile, k)
                    if clo <= idx < chi:
                        for c in range(3):
                            assert copied[(k, c)] == (clo, chi)
                            pos = base(k, 0) + (idx - lo) + c * stride(k)
                            assert base(k, c) <= pos < base(k, c) + extent(k)
                    else:
                        assert k < 8 and (k & 1) and c4[k >> 1] == 0, (dims, k, sp)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (6, 4, 4, 2), (4, 4, 6, 8), (6, 4, 6, 10), (8, 8, 8, 8)])
@pytest.mark.parametrize("lpt", [1, 2, 4, 8])
def test_stage_indices_in_bounds(dims, lpt):
    for gauge in ("landau", "coulomb", "mag"):
        for acc in (False, True):
            check(dims, lpt, gauge, acc)


def test_unsigned_clip_regression():
    """The clip taken in unsigned arithmetic (the end of a down-link range
    cast to uint32 before clipping) gives copies far past the array on this
    lattice; the signed clip gives none."""
    G = geom((6, 4, 6, 10))

    def unsigned_clip(sp0, tile, k):
        ext, lo = tile, sp0
        if k < 8 and (k & 1):
            mu = k >> 1
            st = G["stride"][mu] if mu < 3 else 0
            lo, ext = sp0 - st // 2 - 1, tile + 2
        clo = 0 if lo < 0 else lo
        hi = lo + ext
        chi = G["Vh"] if hi > G["Vh"] else hi % 2 ** 32
        return clo, max(chi, clo)

    bad = [(sp0, k) for sp0 in range(0, G["Vh"], 32) for k in range(8) if unsigned_clip(sp0, 32, k)[1] > G["Vh"]]
    assert bad
    assert all(stage_range(G, sp0, 32, k)[2] <= G["Vh"] for sp0, k in bad)
