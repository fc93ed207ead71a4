"""The job server on the GPU: jobs of different lattices and gauges run
side by side on their own streams, and every job's result is the one the
same job gives when fixed alone."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1212_5221_gb300 import build, gf

    build.build_all()
    return gf


def test_server_results_equal_alone(gf, synth):
    specs = [((8, 8, 8, 8), "landau"), ((4, 4, 6, 8), "coulomb"), ((4, 4, 6, 8), "mag"),
             ((8, 6, 6, 8), "landau"), ((8, 8, 8, 8), "coulomb"), ((6, 6, 6, 6), "mag")] * 2
    fix = dict(theta_target=1e-11, max_sweeps=20000, check_interval=10, switch_theta=1e-8)
    links = [synth.links(d, "smooth", 0.3, k) for k, (d, _) in enumerate(specs)]
    outs = [np.empty_like(u) for u in links]
    arena = sum(gf.gf_footprint(d, 1, g, "mixed") for d, g in specs[:5]) + (1 << 20)
    s = gf.gf_server_create(arena, 4)
    try:
        for k, ((dims, gauge), u) in enumerate(zip(specs, links)):
            gf.gf_server_submit(s, dims, gauge, "mixed", host_links=u, orbit_seed=100 + k, tag=k,
                                host_out=outs[k], param=1.35 if gauge == "mag" else 1.7, **fix)
        res = []
        t0 = time.time()
        while len(res) < len(specs) and time.time() - t0 < 300:
            res += gf.gf_server_poll(s, 64, 50)
    finally:
        gf.gf_server_destroy(s)
    assert len(res) == len(specs)
    by_tag = {r["tag"]: r for r in res}
    # some jobs overlapped in time on the device
    iv = sorted((r["t_admit"], r["t_done"]) for r in res)
    assert any(b[0] < a[1] for a, b in zip(iv, iv[1:]))
    for k, ((dims, gauge), u) in enumerate(zip(specs, links)):
        r = by_tag[k]
        assert r["status"] == 0 and r["theta"] < 1e-11
        h = gf.gf_create(dims, gauge, "mixed")
        try:
            gf.gf_load_links(h, 0, u)
            gf.gf_random_gauge_transform(h, 100 + k)
            r1 = gf.gf_fix(h, "or", 1.35 if gauge == "mag" else 1.7, **fix)
            F, T = gf.gf_functional_theta(h)
            V = np.empty_like(u)
            gf.gf_store_links(h, 0, V)
        finally:
            gf.gf_destroy(h)
        assert r["sweeps"] == r1["sweeps"]
        assert r["F"] == F[0] and r["theta"] == T[0]
        assert np.array_equal(V, outs[k])


def test_server_protocol_job_equals_alone(gf, synth):
    """A MAG job run through the annealing protocol (SA -> SR -> OR, Sec. 6.5)
    in the server, beside plain jobs, gives the links the same protocol gives
    on its own context."""
    dims = (6, 6, 6, 6)
    u = synth.links(dims, "smooth", 0.3, 7)
    other = synth.links((8, 8, 8, 8), "smooth", 0.3, 8)
    out = np.empty_like(u)
    fix = dict(param=1.35, theta_target=1e-11, max_sweeps=20000, check_interval=10, switch_theta=1e-8)
    ann = dict(sa_steps=50, T_start=1.45, T_end=0.01, sr_sweeps=200, sr_p=0.5, sr_theta=1e-6, seed=5)
    s = gf.gf_server_create(gf.gf_footprint(dims, 1, "mag", "mixed") * 3 + (1 << 20), 2)
    try:
        gf.gf_server_submit(s, (8, 8, 8, 8), "landau", "mixed", host_links=other, orbit_seed=3, tag=1,
                            param=1.7, theta_target=1e-11, max_sweeps=20000)
        gf.gf_server_submit(s, dims, "mag", "mixed", host_links=u, orbit_seed=41, tag=2, host_out=out,
                            anneal=ann, **fix)
        res = []
        t0 = time.time()
        while len(res) < 2 and time.time() - t0 < 300:
            res += gf.gf_server_poll(s, 8, 50)
    finally:
        gf.gf_server_destroy(s)
    r = {x["tag"]: x for x in res}[2]
    assert r["status"] == 0 and r["theta"] < 1e-11
    h = gf.gf_create(dims, "mag", "mixed")
    try:
        gf.gf_load_links(h, 0, u)
        gf.gf_random_gauge_transform(h, 41)
        r1 = gf.gf_protocol(h, 50, 1.45, 0.01, sr_sweeps=200, sr_p=0.5, sr_theta=1e-6, seed=5, omega=1.35,
                            theta_target=1e-11, max_sweeps=20000, check_interval=10, switch_theta=1e-8)
        V = np.empty_like(u)
        gf.gf_store_links(h, 0, V)
    finally:
        gf.gf_destroy(h)
    assert r["sweeps"] == r1["sweeps"]
    assert np.array_equal(V, out)
