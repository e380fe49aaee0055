"""Continuous-batching server: trace generation and admission on the host,
and on the GPU: each result is bit for bit the same alone, in a batch of
same-shape requests and beside other requests, the HBM budget is never
exceeded, oversize requests are refused, latency is reported."""
import numpy as np
import pytest

from paper_2403_03488_gb300 import serve


def test_trace_is_seeded_poisson_with_the_configured_mix():
    a = serve.make_trace(4000, 200.0, seed=3)
    b = serve.make_trace(4000, 200.0, seed=3)
    assert a == b
    t = np.array([s["arrival"] for s in a])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    rate = (len(t) - 1) / t[-1]
    assert 185 < rate < 215
    H = np.array([s["H"] for s in a])
    C = np.array([s["C"] for s in a])
    assert H.min() >= 128 and H.max() <= 2048
    assert 0.45 < (C == 3).mean() < 0.55
    assert set(s["sigma"] for s in a) == {15.0, 25.0, 50.0}


def test_scene_pool_requests_are_seeded_crops():
    pool = serve.ScenePool(seed=1, side=256, n_scenes=2)
    spec = dict(rid=0, arrival=0.0, H=100, W=130, C=3, sigma=25.0, seed=11)
    r1, r2 = pool.build(spec), pool.build(spec)
    assert r1.image.shape == (3, 100, 130) and r1.image.dtype == np.float32
    assert np.array_equal(r1.image, r2.image)


def _small_requests(n, seed=0):
    pool = serve.ScenePool(seed=seed, side=384, n_scenes=2)
    specs = serve.make_trace(n, 1000.0, seed=seed, side=(96, 320))
    return [pool.build(s) for s in specs]


@pytest.mark.gpu
@pytest.mark.parametrize("bm3d_bf16", [False, True])
def test_results_same_alone_and_in_the_mix(bm3d_bf16):
    """Also with the tensor-core group transforms, whose persistent CTAs then
    share the SMs with the other requests' kernels."""
    from gpu_util import need_gpu
    need_gpu()
    from paper_2403_03488_gb300 import api
    prec = api.DN_BF16 if bm3d_bf16 else api.DN_FP32
    w = serve.load_weights()
    reqs = _small_requests(10, seed=5)
    alone = []
    for r in reqs:
        srv = serve.Server(w, slots=1, bm3d_precision=prec)
        q = serve.Request(r.rid, r.image, r.sigma)
        srv.run([q], realtime=False, keep_results=True)
        alone.append(q.result)
    mix = [serve.Request(r.rid, r.image, r.sigma) for r in reqs]
    srv = serve.Server(w, slots=8, bm3d_precision=prec)
    st = srv.run(mix, realtime=False, keep_results=True)
    assert st.max_inflight > 1  # the requests really overlapped
    for q, ref in zip(mix, alone):
        assert q.result.shape == ref.shape
        np.testing.assert_array_equal(q.result, ref)


@pytest.mark.gpu
def test_same_shape_requests_are_batched_and_unchanged():
    """Queued requests of equal (C, H, W) go out as one batched launch with
    their own sigmas, and each result is bit for bit its result alone."""
    from gpu_util import need_gpu
    need_gpu()
    w = serve.load_weights()
    pool = serve.ScenePool(seed=9, side=384, n_scenes=2)
    shapes = [(1, 200, 176), (3, 128, 150), (1, 96, 320)]
    sig = [15.0, 25.0, 50.0]
    specs = [dict(rid=i, arrival=0.0, H=shapes[i % 3][1], W=shapes[i % 3][2], C=shapes[i % 3][0],
                  sigma=sig[(i // 3) % 3], seed=500 + i) for i in range(12)]
    reqs = [pool.build(sp) for sp in specs]
    alone = []
    for r in reqs:
        q = serve.Request(r.rid, r.image, r.sigma)
        serve.Server(w, slots=1, max_batch=1).run([q], realtime=False, keep_results=True)
        alone.append(q.result)
    mix = [serve.Request(r.rid, r.image, r.sigma) for r in reqs]
    st = serve.Server(w, slots=2, max_batch=8).run(mix, realtime=False, keep_results=True)
    assert st.max_batch > 1 and st.launches < len(mix)
    for q, ref in zip(mix, alone):
        np.testing.assert_array_equal(q.result, ref)


@pytest.mark.gpu
def test_admission_never_exceeds_budget_and_refuses_oversize():
    from gpu_util import need_gpu
    need_gpu()
    w = serve.load_weights()
    reqs = _small_requests(12, seed=6)
    probe = serve.Server(w)
    fps = sorted(probe.footprint(*r.image.shape) for r in reqs)
    budget = fps[-1] + fps[-2]
    srv = serve.Server(w, budget_bytes=budget, slots=8)
    big = serve.Request(999, np.zeros((3, 1024, 1024), np.float32), 25.0)
    st = srv.run(reqs + [big], realtime=False)
    assert st.max_inflight_bytes <= budget
    assert st.rejected == 1 and big.rejected
    assert len(st.latencies_ms) == len(reqs)


@pytest.mark.gpu
def test_poisson_replay_reports_latency():
    from gpu_util import need_gpu
    need_gpu()
    res = serve.replay(rate=100.0, n=40, side=(128, 384))
    assert res["requests"] == 40 and res["rejected"] == 0
    assert 0 < res["p50_ms"] <= res["p99_ms"]
    assert res["served_mpix_s"] > 0
