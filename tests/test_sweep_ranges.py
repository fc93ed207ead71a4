"""The FP64 sweep kernel's distribution of sites over blocks, mirrored on the
CPU: every block takes an equal contiguous range of the (copy, offset)
indices of the launch's sites [sp_lo, sp_lo + sp_n) of each copy and walks it
in tiles.  Every site of the range must be visited exactly once, no site
outside it, and the L2 prefetch of the next tile must stay inside the range.
The host's split of a time slab into boundary and inner launches must cover
the slab's owned sites exactly.  The expressions follow the FP64 branch of
sweep_kernel, the grid size of its launch and gf_sweep_half."""
import numpy as np
import pytest

BLOCK = 256


def blocks_of(sp_n, ncopies, tile, resident):
    ntiles = ((sp_n + tile - 1) // tile) * ncopies
    return min(resident, ntiles) if resident else ntiles


def visit(Vh, ncopies, sp_lo, sp_n, lpt, resident):
    """(copy, site) pairs a launch updates, and the prefetched (copy, lo, n)."""
    tile = BLOCK // (8 // lpt)
    grid = blocks_of(sp_n, ncopies, tile, resident)
    total = sp_n * ncopies
    seen = np.zeros((ncopies + 1, Vh), np.int32)
    pref = []
    for b in range(grid):
        lo, hi = total * b // grid, total * (b + 1) // grid
        c0 = lo // sp_n if sp_n else 0
        s0 = lo - c0 * sp_n
        base = lo
        while base < hi:
            if base + tile < hi:
                nc, ns = c0, s0 + tile
                while ns >= sp_n:
                    ns -= sp_n
                    nc += 1
                n = min(min(tile, sp_n - ns), hi - base - tile)
                pref.append((nc, sp_lo + ns, n))
            for local in range(tile):
                copy, sp = c0, s0 + local
                while sp >= sp_n:
                    sp -= sp_n
                    copy += 1
                sp += sp_lo
                if base + local < hi:
                    assert copy < ncopies and sp < Vh
                    seen[copy, sp] += 1
            s0 += tile
            while s0 >= sp_n:
                s0 -= sp_n
                c0 += 1
            base += tile
    return seen[:ncopies], pref


@pytest.mark.parametrize("lpt", [1, 2, 4, 8])
def test_ranges_visit_every_site_once(lpt):
    rng = np.random.default_rng(10 + lpt)
    for _ in range(25):
        Vh = int(rng.integers(1, 3000))
        ncopies = int(rng.integers(1, 4))
        sp_lo = int(rng.integers(0, Vh))
        sp_n = int(rng.integers(1, Vh - sp_lo + 1))
        resident = int(rng.choice([0, 3, 17, 304]))
        seen, pref = visit(Vh, ncopies, sp_lo, sp_n, lpt, resident)
        want = np.zeros_like(seen)
        want[:, sp_lo:sp_lo + sp_n] = 1
        assert np.array_equal(seen, want)
        for nc, a, n in pref:
            assert 0 <= nc < ncopies and n > 0 and sp_lo <= a and a + n <= sp_lo + sp_n


def test_full_range_is_the_whole_lattice():
    """The default range (0, Vh) gives the original enumeration: every site of
    every copy once."""
    for Vh, ncopies in ((1 << 12, 1), (3000, 3), (257, 2)):
        seen, _ = visit(Vh, ncopies, 0, Vh, 8, 304)
        assert (seen == 1).all()


def slab_launches(nl, V3, part):
    """(sp_lo, sp_n) of the FP64 launches gf_sweep_half makes for a slab part
    (0 owned, 1 boundary, 2 inner) of local extent nl."""
    vs = V3 // 2
    if part == 1:
        return [(t * vs, vs) for t in (1, nl - 2)]
    t0, t1 = (2, nl - 2) if part == 2 else (1, nl - 1)
    return [] if t1 <= t0 else [(t0 * vs, (t1 - t0) * vs)]


@pytest.mark.parametrize("nt", [2, 4, 6, 32])
def test_slab_parts_cover_the_owned_slices(nt):
    """Boundary + inner = owned, disjoint, and each launch's sites are the
    sites of its slices (site sp of a parity lies in slice 2 sp // V3)."""
    nl, V3 = nt + 2, 4 * 6 * 4
    Vh = nl * V3 // 2
    cover = {}
    for part in (0, 1, 2):
        m = np.zeros(Vh, np.int32)
        for lo, n in slab_launches(nl, V3, part):
            assert lo + n <= Vh
            m[lo:lo + n] += 1
        cover[part] = m
    sl = 2 * np.arange(Vh) // V3
    assert np.array_equal(cover[0], ((sl >= 1) & (sl <= nt)).astype(np.int32))
    assert np.array_equal(cover[1], ((sl == 1) | (sl == nt)).astype(np.int32))
    assert np.array_equal(cover[1] + cover[2], cover[0])
