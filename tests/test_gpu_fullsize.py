"""Sampled parity at the full size of the 64^3 x 256 workload.

The oracle cannot sweep 67 million sites in a test, but every check here
involves only a small part of the lattice that it can reproduce exactly:

* Coulomb: time-slices are independent problems (Sec. 2.1.1), so the pair of
  slices (t, t+1) is cut out as a 2 x 64^3 lattice (slice t placed at the
  index of its own parity), transformed with the Haar g(x) of the full
  lattice's sites, and swept by the oracle; the GPU sweeps all 256 slices in
  one launch per half-sweep.
* Landau: after one sweep, the eight links of an odd site depend only on the
  links within distance two of it; an 8^4 patch around the site (origin of
  even coordinate sum, so parities agree) reproduces them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

DIMS = (256, 64, 64, 64)  # Nt, Nx, Ny, Nz
EPS, FIELD_SEED, ORBIT_SEED = 0.3, 2, 2
V3 = 64 ** 3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    free, _ = torch.cuda.mem_get_info()
    if free < 70e9:
        pytest.skip("needs ~60 GB of free device memory")
    from paper_1212_5221_gb300 import build, gf, inputs
    import oracle

    build.build_all()
    oracle.build()
    return gf, inputs, oracle


def load_full(gf, inputs, h, slab=16):
    for t0 in range(0, DIMS[0], slab):
        U = inputs.links(DIMS, "smooth", EPS, FIELD_SEED, t0=t0, nt=slab)
        gf.gf_load_links_slab(h, 0, t0, slab, U)


def haar_slices(oracle, t0, nt):
    """g(x) of the full lattice's random transformation for slices t0..t0+nt-1."""
    out = []
    for t in range(t0, t0 + nt):
        tt = t % DIMS[0]
        out.append(oracle.haar_field(ORBIT_SEED, tt * V3, V3).reshape(64, 64, 64, 3, 3))
    return np.stack(out)


COULOMB_T = [0, 131, 255]
PATCH_SITES = [(100, 10, 21, 34), (7, 40, 9, 57)]


@pytest.fixture(scope="module")
def coulomb_run(env):
    """One FP64 Coulomb run of the full lattice: 256 slices, 2 sweeps."""
    gf, inputs, oracle = env
    h = gf.gf_create(DIMS, "coulomb", "fp64")
    out = {}
    try:
        load_full(gf, inputs, h)
        gf.gf_random_gauge_transform(h, ORBIT_SEED)
        gf.gf_sweep(h, "or", 1.7, 2, observables=False)
        out["Ft"], out["Tt"] = gf.gf_slice_functional_theta(h)
        for t in COULOMB_T:
            for tt in (t, (t + 1) % DIMS[0]):
                V = np.empty((1, 64, 64, 64, 4, 3, 3), np.complex128)
                gf.gf_store_links_slab(h, 0, tt, 1, V)
                out[tt] = V[0]
    finally:
        gf.gf_destroy(h)
    return out


@pytest.mark.parametrize("t", COULOMB_T)
def test_coulomb_slice_pairs(env, coulomb_run, t):
    gf, inputs, oracle = env
    t1 = (t + 1) % DIMS[0]
    V, V1 = coulomb_run[t][None], coulomb_run[t1][None]
    Ft, Tt = coulomb_run["Ft"], coulomb_run["Tt"]
    # oracle: slices (t, t+1) at indices (t % 2, (t+1) % 2) of a 2 x 64^3 lattice
    j, j1 = t % 2, (t + 1) % 2
    small = np.empty((2, 64, 64, 64, 4, 3, 3), np.complex128)
    small[j] = inputs.links(DIMS, "smooth", EPS, FIELD_SEED, t0=t, nt=1)[0]
    small[j1] = inputs.links(DIMS, "smooth", EPS, FIELD_SEED, t0=t1, nt=1)[0]
    g = np.empty((2, 64, 64, 64, 3, 3), np.complex128)
    g[j] = haar_slices(oracle, t, 1)[0]
    g[j1] = haar_slices(oracle, t1, 1)[0]
    oracle.gauge_transform(small, g)
    oracle.sweep(small, "coulomb", "or", 1.7, 2)
    _, _, oFt, oTt = oracle.observables(small, "coulomb")
    # spatial links of both slices, and U_0 of slice t (its far end is slice t+1)
    assert np.abs(V[0][..., 1:, :, :] - small[j][..., 1:, :, :]).max() <= 1e-12
    assert np.abs(V1[0][..., 1:, :, :] - small[j1][..., 1:, :, :]).max() <= 1e-12
    assert np.abs(V[0][..., 0, :, :] - small[j][..., 0, :, :]).max() <= 1e-12
    assert abs(Ft[0][t] - oFt[j]) <= 1e-12 * abs(oFt[j])
    assert abs(Tt[0][t] - oTt[j]) <= 1e-11 * abs(oTt[j])


@pytest.fixture(scope="module")
def landau_run(env):
    """One mixed-precision Landau run of the full lattice: 1 sweep."""
    gf, inputs, oracle = env
    h = gf.gf_create(DIMS, "landau", "mixed")
    out = {}
    try:
        load_full(gf, inputs, h)
        gf.gf_random_gauge_transform(h, ORBIT_SEED)
        gf.gf_sweep(h, "or", 1.7, 1, observables=False)
        for site in PATCH_SITES:
            Vg = np.empty((2, 64, 64, 64, 4, 3, 3), np.complex128)
            gf.gf_store_links_slab(h, 0, site[0] - 1, 2, Vg)
            out[site] = Vg
    finally:
        gf.gf_destroy(h)
    return out


@pytest.mark.parametrize("site", PATCH_SITES)
def test_landau_mixed_patches(env, landau_run, site):
    gf, inputs, oracle = env
    assert sum(site) % 2 == 1  # odd: updated after its even neighbours
    t = site[0]
    Vg = landau_run[site]
    # 8^4 patch around the site; origin with an even coordinate sum
    o = [c - 4 for c in site]
    if sum(o) % 2:
        o[3] += 1
    loc = [site[d] - o[d] for d in range(4)]
    full = inputs.links(DIMS, "smooth", EPS, FIELD_SEED, t0=o[0], nt=8)
    patch = np.ascontiguousarray(full[:, o[1]:o[1] + 8, o[2]:o[2] + 8, o[3]:o[3] + 8])
    gs = haar_slices(oracle, o[0], 8)[:, o[1]:o[1] + 8, o[2]:o[2] + 8, o[3]:o[3] + 8]
    oracle.gauge_transform(patch, np.ascontiguousarray(gs))
    oracle.sweep(patch, "landau", "or", 1.7, 1)
    for mu in range(4):
        # U_mu(y)
        got = Vg[1][site[1], site[2], site[3], mu]
        want = patch[loc[0], loc[1], loc[2], loc[3], mu]
        assert np.abs(got - want).max() <= 1e-4
        # U_mu(y - mu)
        gy = list(site)
        gy[mu] -= 1
        ly = list(loc)
        ly[mu] -= 1
        got = Vg[gy[0] - (t - 1)][gy[1], gy[2], gy[3], mu]
        want = patch[ly[0], ly[1], ly[2], ly[3], mu]
        assert np.abs(got - want).max() <= 1e-4
