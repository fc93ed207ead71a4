"""The job server's host logic (queue, admission by footprint, slots,
anti-starvation) with its test double, which runs no device code."""
import time

import pytest


@pytest.fixture(scope="module")
def gf():
    from paper_1212_5221_gb300 import build, gf

    build.build_lib()
    return gf


def _fp(gf, dims, gauge="landau", prec="mixed"):
    return gf.gf_footprint(dims, 1, gauge, prec)


def test_mock_server_admission(gf):
    small, big = (8, 8, 8, 8), (16, 16, 16, 16)
    arena = _fp(gf, big) + 2 * _fp(gf, small) + 4096
    s = gf.gf_server_create_mock(arena, 3, 2.0)  # 2 s per GB of footprint
    try:
        jobs = [(k, small if k % 3 else big) for k in range(12)]
        for tag, dims in jobs:
            gf.gf_server_submit(s, dims, "landau", "mixed", tag=tag)
        peak_run, peak_bytes, res = 0, 0, []
        t0 = time.time()
        while len(res) < len(jobs) and time.time() - t0 < 60:
            st = gf.gf_server_status(s)
            peak_run = max(peak_run, st["running"])
            peak_bytes = max(peak_bytes, st["bytes_in_use"])
            res += gf.gf_server_poll(s, 64, 5)
        assert sorted(r["tag"] for r in res) == list(range(12))
        assert all(r["status"] == 0 for r in res)
        assert peak_run <= 3 and peak_bytes <= arena
        assert peak_run >= 2  # jobs ran side by side
        for r in res:
            assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
            assert r["footprint"] >= _fp(gf, small)
        # the big jobs were not starved by the stream of small ones
        assert max(r["t_done"] for r in res if r["tag"] % 3 == 0) < time.time() - t0 + 1
    finally:
        gf.gf_server_destroy(s)


def test_mock_server_rejects_oversize(gf):
    s = gf.gf_server_create_mock(_fp(gf, (8, 8, 8, 8)) + 1024, 1, 0.0)
    try:
        with pytest.raises(gf.GFError) as e:
            gf.gf_server_submit(s, (16, 16, 16, 16), "landau", "mixed")
        assert e.value.code == gf.GF_ENOMEM
        with pytest.raises(gf.GFError) as e:
            gf.gf_server_submit(s, (7, 8, 8, 8), "landau", "mixed")
        assert e.value.code == gf.GF_EINVAL
    finally:
        gf.gf_server_destroy(s)


def test_mock_server_destroy_drains_queue(gf):
    s = gf.gf_server_create_mock(_fp(gf, (8, 8, 8, 8)) * 2, 1, 0.5)
    for k in range(4):
        gf.gf_server_submit(s, (8, 8, 8, 8), "mag", "fp32", tag=k)
    gf.gf_server_destroy(s)  # returns after running all four


def test_mock_server_cancel(gf):
    """Queued jobs can be canceled (reported with GF_ECANCELED); a running job
    completes; an unknown tag cancels nothing."""
    dims = (8, 8, 8, 8)
    s = gf.gf_server_create_mock(_fp(gf, dims) + 4096, 1, 0.5 / (_fp(gf, dims) / 1e9))  # 0.5 s per job
    try:
        for tag in (1, 2, 3, 3):
            gf.gf_server_submit(s, dims, "landau", "mixed", tag=tag)
        t0 = time.time()
        while gf.gf_server_status(s)["running"] == 0 and time.time() - t0 < 10:
            time.sleep(0.01)
        assert gf.gf_server_cancel(s, 3) == 2
        assert gf.gf_server_cancel(s, 99) == 0
        res = []
        while len(res) < 4 and time.time() - t0 < 30:
            res += gf.gf_server_poll(s, 64, 100)
        by = {}
        for r in res:
            by.setdefault(r["tag"], []).append(r["status"])
        assert by[3] == [gf.GF_ECANCELED, gf.GF_ECANCELED]
        assert by[1] == [0] and by[2] == [0]
        assert gf.gf_server_status(s)["completed"] == 4
    finally:
        gf.gf_server_destroy(s)
