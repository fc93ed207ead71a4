"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/gf.h declares, and validates its arguments."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gf():
    from paper_1212_5221_gb300 import build, gf

    build.build_lib()
    return gf


def header_functions():
    text = open(os.path.join(ROOT, "include", "gf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gf_[a-z0-9_]+)\s*\(", text)))


def test_header_symbols_exported(gf):
    lib = gf.lib()
    names = header_functions()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header(gf):
    for name in header_functions():
        assert hasattr(gf, name), name


def test_footprint(gf):
    b64 = gf.gf_footprint((8, 8, 8, 8), 1, "landau", "fp64")
    b32 = gf.gf_footprint((8, 8, 8, 8), 1, "landau", "fp32")
    bmx = gf.gf_footprint((8, 8, 8, 8), 1, "landau", "mixed")
    links32 = 4096 * 4 * 12 * 4
    assert b64 - b32 == pytest.approx(links32, rel=0.01)
    # FP32 copy + accumulated g + the FP64 re-unitarised accumulator (9 complex)
    assert bmx - b64 == pytest.approx(links32 * 5 / 4 + 4096 * 9 * 16, rel=0.01)
    bc = gf.gf_footprint((8, 8, 8, 8), 1, "coulomb", "fp32")
    assert bc - b32 == pytest.approx(links32 / 4, rel=0.01)  # the accumulated g
    assert gf.gf_footprint((8, 8, 8, 8), 16, "mag", "fp32") > 15 * links32


@pytest.mark.parametrize("dims", [(8, 8, 7, 8), (0, 8, 8, 8), (8, 8, 8, 1), (2048, 1024, 1024, 2)])
def test_bad_dims(gf, dims):
    with pytest.raises(gf.GFError) as e:
        gf.gf_footprint(dims)
    assert e.value.code == gf.GF_EINVAL


def test_bad_enums(gf):
    with pytest.raises(gf.GFError) as e:
        gf.gf_footprint((4, 4, 4, 4), 1, 7, 0)
    assert e.value.code == gf.GF_EINVAL
    with pytest.raises(gf.GFError) as e:
        gf.gf_footprint((4, 4, 4, 4), 0, 0, 0)
    assert e.value.code == gf.GF_EINVAL


def test_null_context(gf):
    lib = gf.lib()
    assert lib.gf_reunitarize(None) == gf.GF_EINVAL
    assert lib.gf_sweep(None, 1, 1.7, 1, 0, None, None) == gf.GF_EINVAL
    lib.gf_destroy(None)


def test_strerror(gf):
    for code in range(7):
        assert gf.gf_strerror(code).startswith("GF_")


def test_no_device_is_loud(gf):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gf.GFError) as e:
        gf.gf_create((4, 4, 4, 4))
    assert e.value.code == gf.GF_ENOSYS
