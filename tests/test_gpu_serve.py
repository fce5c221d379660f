"""Serving loop on the GPU: each forward+gradient result is the same when the
request runs alone and when it overlaps with others (continuous batching on
several streams inside one arena), and equals the direct model call."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_14782_gb300 import serve
    return serve.LinePool("cuda", sizes=(1000, 3000, 10_000))


def _requests(n):
    from paper_2105_14782_gb300 import serve
    rng = np.random.default_rng(11)
    th = W.theta_points(n, 21)
    return [serve.Request(rid=i, chain=i, n_lines=int(rng.choice([1000, 3000, 10_000])),
                          n_grid=int(rng.integers(2000, 6001)), n_layers=int(rng.integers(20, 41)), theta=th[i])
            for i in range(n)]


def test_same_alone_and_in_the_mix(pool):
    from paper_2105_14782_gb300 import serve
    alone = {}
    s1, _ = serve.make_server(arena_bytes=2 << 30, slots=1, pool=pool)
    for r in _requests(12):
        s1.submit(r)
        s1.drain(timeout_s=120)
        assert r.status == serve.DONE, r.error
        alone[r.rid] = r.result
    s4, _ = serve.make_server(arena_bytes=2 << 30, slots=4, pool=pool)
    mix = _requests(12)
    for r in mix:
        s4.submit(r)
    s4.drain(timeout_s=120)
    assert max(r.t_start for r in mix[:4]) < min(r.t_done for r in mix[:4])  # they overlapped
    for r in mix:
        assert r.status == serve.DONE, r.error
        assert np.all(np.isfinite(r.result))
        np.testing.assert_array_equal(r.result, alone[r.rid])  # deterministic reductions: bit-identical


def test_priority_streams_change_no_result(pool):
    """With short requests on high-priority streams the results are those of the
    server without priorities, bit for bit."""
    from paper_2105_14782_gb300 import serve
    base, prio = _requests(12), _requests(12)
    for reqs, flag in ((base, False), (prio, True)):
        s, _ = serve.make_server(arena_bytes=2 << 30, slots=4, pool=pool, priority=flag, hi_evals=1e9)
        for r in reqs:
            s.submit(r)
        s.drain(timeout_s=120)
    assert not any(r.high_priority for r in base)
    assert any(r.high_priority for r in prio) and not all(r.high_priority for r in prio)
    for a, b in zip(base, prio):
        assert a.status == b.status == serve.DONE
        np.testing.assert_array_equal(a.result, b.result)


def test_matches_direct_model_call(pool):
    from paper_2105_14782_gb300 import serve, xs
    r = _requests(3)[2]
    s, _ = serve.make_server(arena_bytes=1 << 30, slots=2, pool=pool)
    s.submit(r)
    s.drain(timeout_s=120)
    assert r.status == serve.DONE
    P, dP = W.pressure_layers(r.n_layers)
    atm = W.Atmosphere(species=[], vmr=[], nu=W.grid_lognu(r.n_grid), p_bar=P, dp_bar=dP)
    m = xs.EmissionModel(atm, prec=xs.PREC_MIXED, lines=[pool.lists[pool.nearest(r.n_lines)], pool.co],
                         d_obs=np.ones(r.n_grid), sig_obs=np.full(r.n_grid, 0.01))
    logl, g = m.logl_grad(r.theta)
    np.testing.assert_array_equal(r.result, np.concatenate([[logl], g]))


def test_oversized_request_rejected_others_served(pool):
    from paper_2105_14782_gb300 import serve
    s, _ = serve.make_server(arena_bytes=256 << 20, slots=2, pool=pool)
    reqs = _requests(3)
    big = serve.Request(rid=99, chain=0, n_lines=10_000, n_grid=2_000_000, n_layers=200, theta=reqs[0].theta)
    s.submit(big)
    for r in reqs:
        s.submit(r)
    s.drain(timeout_s=120)
    assert big.status == serve.REJECTED
    assert all(r.status == serve.DONE for r in reqs)


def test_modit_requests_beside_line_sum_requests(pool):
    """MODIT requests on grids that resolve the Doppler width run in the mix with
    line-sum requests and equal the direct MODIT model call; a MODIT request on a
    grid coarser than the Doppler width is rejected with the reason."""
    from paper_2105_14782_gb300 import serve, xs
    th = np.array([1300.0, 0.1, -3.5, -3.0, 1.0])  # coolest layer 651 K
    fine = [serve.Request(rid=100 + i, chain=i, n_lines=n, n_grid=g, n_layers=30, theta=th, method="modit")
            for i, (n, g) in enumerate([(3000, 20_000), (1000, 30_000)])]
    coarse = serve.Request(rid=200, chain=9, n_lines=1000, n_grid=3000, n_layers=30, theta=th, method="modit")
    lpf = _requests(4)
    s, _ = serve.make_server(arena_bytes=4 << 30, slots=4, pool=pool, n_gamma=16)
    for r in fine + [coarse] + lpf:
        s.submit(r)
    s.drain(timeout_s=300)
    assert coarse.status == serve.REJECTED and "too coarse for MODIT" in coarse.error, coarse.error
    for r in fine + lpf:
        assert r.status == serve.DONE, r.error
    for r in fine:
        P, dP = W.pressure_layers(r.n_layers)
        atm = W.Atmosphere(species=[], vmr=[], nu=W.grid_lognu(r.n_grid), p_bar=P, dp_bar=dP)
        m = xs.EmissionModel(atm, prec=xs.PREC_MIXED, lines=[pool.lists[pool.nearest(r.n_lines)], pool.co],
                             d_obs=np.ones(r.n_grid), sig_obs=np.full(r.n_grid, 0.01), method="modit", n_gamma=16)
        logl, g = m.logl_grad(r.theta)
        np.testing.assert_array_equal(r.result, np.concatenate([[logl], g]))
