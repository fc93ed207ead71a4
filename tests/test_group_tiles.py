"""The tile arithmetic of the group launch (several lattices in one launch),
mirrored on the CPU: numbering the members' tiles one after the other and
finding a tile's member by binary search of the cumulative counts must visit
every (member, copy, site) exactly once and never leave a member's range.
The expressions follow sweep_group_kernel and the host's tile counts."""
import numpy as np
import pytest

BLOCK = 256


def tiles_of(members, lpt):
    tile = BLOCK // (8 // lpt)
    ends, cum = [], 0
    for Vh, ncopies in members:
        cum += ((Vh + tile - 1) // tile) * ncopies
        ends.append(cum)
    return tile, ends


def member_of(t, ends):
    lo, hi = 0, len(ends) - 1
    while lo < hi:
        mid = (lo + hi) >> 1
        if t < ends[mid]:
            hi = mid
        else:
            lo = mid + 1
    return lo


@pytest.mark.parametrize("lpt", [1, 2, 4, 8])
def test_group_tiles_cover_every_site_once(lpt):
    rng = np.random.default_rng(lpt)
    for _ in range(20):
        n = int(rng.integers(1, 49))
        dims = [tuple(int(2 * rng.integers(1, 9)) for _ in range(4)) for _ in range(n)]
        members = [(int(np.prod(d)) // 2, int(rng.integers(1, 4))) for d in dims]
        tile, ends = tiles_of(members, lpt)
        seen = [np.zeros((c, Vh), np.int32) for Vh, c in members]
        for t in range(ends[-1]):
            m = member_of(t, ends)
            assert t < ends[m] and (m == 0 or t >= ends[m - 1])
            Vh, ncopies = members[m]
            tt = t - (ends[m - 1] if m else 0)
            per_copy = (Vh + tile - 1) // tile
            copy = tt // per_copy
            sp0 = (tt - copy * per_copy) * tile
            assert copy < ncopies and sp0 < Vh
            for local in range(tile):
                sp = sp0 + local
                if sp < Vh:  # the kernel's "valid"
                    seen[m][copy, sp] += 1
        assert all((s == 1).all() for s in seen)
