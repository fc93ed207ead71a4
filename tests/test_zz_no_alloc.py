"""gf_functional_theta_noalloc against gf_functional_theta.

The no-allocation entry point serves callers that cannot call cudaMalloc:
it keeps its partial sums in a fixed device array that all calls share.
This test calls it through the C ABI twice in a row, on two different
fields, and checks both results against the context-based reduction; the
second call also shows that the shared array carries nothing over.  It sits
in a file that pytest collects last, and passes run alone or after the rest.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("gauge", ["landau", "coulomb", "mag"])
def test_noalloc_matches_context_reduction(gauge):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_5221_gb300 import build, gf, inputs

    build.build_all()
    dims = (6, 4, 6, 10)
    results = []
    for seed in (3, 4):  # two calls in a row, different inputs
        U = inputs.links(dims, "smooth", 0.4, seed)
        h = gf.gf_create(dims, gauge, "fp64")
        try:
            gf.gf_load_links(h, 0, U)
            gf.gf_random_gauge_transform(h, 10 + seed)
            F_ref, T_ref = gf.gf_functional_theta(h)
            Ft_ref, Tt_ref = gf.gf_slice_functional_theta(h)
            dev = torch.empty(U.size * 2, dtype=torch.float64, device="cuda")
            gf.gf_store_links_device(h, 0, dev.data_ptr())
        finally:
            gf.gf_destroy(h)
        torch.cuda.synchronize()
        F, T, Ft, Tt = gf.gf_functional_theta_noalloc(dims, gauge, dev.data_ptr())
        assert abs(F - F_ref[0]) <= 1e-12 * abs(F_ref[0])
        assert abs(T - T_ref[0]) <= 1e-12 * abs(T_ref[0])
        assert np.allclose(Ft, Ft_ref[0], rtol=1e-12, atol=0)
        assert np.allclose(Tt, Tt_ref[0], rtol=1e-12, atol=0)
        results.append((F, T))
    assert results[0] != results[1]


def test_noalloc_rejects_oversized_and_misaligned():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_5221_gb300 import build, gf

    build.build_all()
    dev = torch.zeros(1024, dtype=torch.float64, device="cuda")
    with pytest.raises(gf.GFError) as e:
        gf.gf_functional_theta_noalloc((2048, 2, 2, 2), "landau", dev.data_ptr())
    assert e.value.code == gf.GF_EINVAL and "GF_NOALLOC_MAX_NT" in str(e.value)
    with pytest.raises(gf.GFError) as e:
        gf.gf_functional_theta_noalloc((2, 2, 2, 2), "landau", dev.data_ptr() + 8)
    assert e.value.code == gf.GF_EINVAL
