"""Host-side logic of the serving loop (admission by memory and slots, bounded
skip-ahead, rejection, cancellation, injected allocation failure, completion
order), driven by a fake executor: no GPU needed."""
import numpy as np
import pytest

from paper_2105_14782_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    """Each request takes n_lines * 1e-6 s; memory = n_grid * 100 bytes."""

    def __init__(self, clock, fail_hook=None):
        self.clock = clock
        self.fail_hook = fail_hook
        self.launched = []

    def valid(self, r):
        return r.n_grid > 0 and r.n_lines > 0

    def bytes_needed(self, r):
        return r.n_grid * 100 if self.valid(r) else -1

    def launch(self, r, block, slot):
        self.launched.append((r.rid, slot, block))
        r.evals = r.n_lines * r.n_grid
        return self.clock() + r.n_lines * 1e-6

    def ready(self, r):
        return self.clock() >= r.handle

    def collect(self, r):
        return np.array([float(r.rid), r.n_lines, r.n_grid])


def req(i, nl=1000, ng=1000, nlay=10):
    return serve.Request(rid=i, chain=i, n_lines=nl, n_grid=ng, n_layers=nlay, theta=np.zeros(5))


def run_until_idle(s, clk, dt=1e-4, limit=100000):
    for _ in range(limit):
        if not s.busy():
            return
        s.step()
        clk.t += dt
    raise AssertionError("did not drain")


def test_arena_first_fit_and_coalescing():
    a = serve.Arena(10 * 256)
    b1, b2, b3 = a.alloc(256), a.alloc(512), a.alloc(256)
    assert b1 == (0, 256) and b2 == (256, 512) and b3 == (768, 256)
    a.release(b2)
    assert a.free == [(256, 512), (1024, 1536)]
    b4 = a.alloc(300)  # first fit: the hole left by b2, rounded to 512
    assert b4 == (256, 512) and a.free == [(1024, 1536)]
    assert a.alloc(2000) is None
    for b in (b1, b3, b4):
        a.release(b)
    assert a.free == [(0, 10 * 256)] and a.used == 0 and a.largest_free() == 2560


def test_admission_by_slots_and_memory_with_skip_ahead():
    clk = FakeClock()
    s = serve.Scheduler(FakeExecutor(clk), arena_bytes=1_000_000, slots=2, max_skip=4, clock=clk)
    big = s.submit(req(0, ng=9000))    # 900 kB
    big2 = s.submit(req(1, ng=9000))   # does not fit next to the first
    small = s.submit(req(2, ng=500))   # 50 kB: may pass the blocked one
    s.step()
    assert big.status == serve.RUNNING and small.status == serve.RUNNING and big2.status == serve.PENDING
    run_until_idle(s, clk)
    assert all(r.status == serve.DONE for r in (big, big2, small))
    assert s.arena.used == 0 and s.counts["completed"] == 3


def test_rejects_invalid_and_oversized_requests():
    clk = FakeClock()
    s = serve.Scheduler(FakeExecutor(clk), arena_bytes=100_000, slots=2, clock=clk)
    bad = s.submit(req(0, ng=0))
    huge = s.submit(req(1, ng=10_000))
    ok = s.submit(req(2, ng=100))
    assert bad.status == serve.REJECTED and huge.status == serve.REJECTED and "budget" in huge.error
    run_until_idle(s, clk)
    assert ok.status == serve.DONE and s.counts["rejected"] == 2


def test_cancel_pending_request_leaves_others_intact():
    clk = FakeClock()
    s = serve.Scheduler(FakeExecutor(clk), arena_bytes=1_000_000, slots=1, clock=clk)
    a, b, c = (s.submit(req(i)) for i in range(3))
    s.step()
    assert s.cancel(b) and not s.cancel(a)  # a is already running
    run_until_idle(s, clk)
    assert a.status == serve.DONE and c.status == serve.DONE and b.status == serve.CANCELLED
    assert c.result[0] == 2.0


def test_injected_allocation_failure_only_delays_the_victim():
    clk = FakeClock()
    failures = {"left": 3}

    def hook(n):
        if n == 200 * 100 and failures["left"] > 0:  # the 20,000-point request
            failures["left"] -= 1
            return True
        return False

    ex = FakeExecutor(clk, fail_hook=hook)
    s = serve.Scheduler(ex, arena_bytes=1_000_000, slots=2, clock=clk)
    victim = s.submit(req(0, ng=200))
    others = [s.submit(req(i, ng=300)) for i in range(1, 4)]
    run_until_idle(s, clk)
    assert victim.status == serve.DONE and all(o.status == serve.DONE for o in others)
    assert [o.result[0] for o in others] == [1.0, 2.0, 3.0]


def test_closed_loop_keeps_one_request_per_chain():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    s = serve.Scheduler(ex, arena_bytes=50_000_000, slots=4, clock=clk)

    # advance the fake clock inside the loop by patching sleep-free stepping
    orig_step = s.step

    def step():
        clk.t += 1e-3
        return orig_step()

    s.step = step
    finished, wall = serve.closed_loop(s, chains=16, offered_rate=200.0, duration_s=2.0, timeout_s=1e6)
    assert finished and all(r.status == serve.DONE for r in finished)
    by_chain = {}
    for r in sorted(finished, key=lambda r: r.t_submit):
        prev = by_chain.get(r.chain)
        assert prev is None or r.t_submit >= prev.t_done  # at most one outstanding per chain
        by_chain[r.chain] = r
    summ = serve.summarize(finished, wall)
    assert summ["p99_s"] >= summ["p50_s"] > 0


def _stepping(s, clk, dt=1e-3):
    orig = s.step

    def step():
        clk.t += dt
        return orig()

    s.step = step


def test_saturated_closed_loop_cancels_queue_at_window_end():
    clk = FakeClock()
    s = serve.Scheduler(FakeExecutor(clk), arena_bytes=10**12, slots=2, clock=clk)
    _stepping(s, clk)
    # service ~0.1-1 s per request, 64 chains at 1000 req/s offered: saturated
    finished, wall = serve.closed_loop(s, chains=64, offered_rate=1000.0, duration_s=3.0, timeout_s=1e6,
                                       cancel_at_end=True)
    st = serve.summarize(finished, wall)
    assert st["cancelled"] > 0 and st["completed"] > 0
    assert not s.busy() and s.arena.used == 0
    assert wall < 3.0 + 2 * 1.0 + 0.1  # only the running requests were waited for


def test_open_loop_drains_and_counts_all_arrivals():
    clk = FakeClock()
    s = serve.Scheduler(FakeExecutor(clk), arena_bytes=10**12, slots=4, clock=clk)
    _stepping(s, clk)
    sent, wall = serve.open_loop(s, rate=5.0, duration_s=4.0, timeout_s=1e6)
    assert len(sent) > 5 and all(r.status == serve.DONE for r in sent)
    st = serve.summarize(sent, wall)
    assert st["completed"] == len(sent) and st["p99_s"] >= st["p50_s"]


class ReasonExecutor(FakeExecutor):
    def invalid_reason(self, r):
        return "" if r.n_grid > 0 else "grid too coarse for MODIT: test"

    def valid(self, r):
        return self.invalid_reason(r) == ""


def test_rejection_carries_the_executors_reason():
    clk = FakeClock()
    s = serve.Scheduler(ReasonExecutor(clk), arena_bytes=100_000, slots=1, clock=clk)
    bad = s.submit(req(0, ng=0))
    assert bad.status == serve.REJECTED and bad.error == "grid too coarse for MODIT: test"


def test_modit_doppler_width_in_q_steps_matches_the_oracle():
    """beta' = R0 beta/nu_hat (Sec. 2.1.2) from the oracle's per-line Doppler widths
    equals the serving rule's closed form for both species, at any line."""
    oracle = pytest.importorskip("oracle")
    import workloads as W
    N, T = 12_000, 651.0
    R0 = (N - 1) / np.log(W.NU_MAX / W.NU_MIN)
    for lines in (W.water_like(50, seed=5), W.co_like(50, seed=6)):
        _, beta, _ = oracle.line_params(lines, T, 1.0)
        bq = R0 * np.asarray(beta).ravel() / lines.nu_hat
        np.testing.assert_allclose(bq, serve.modit_beta_q(N, T, lines.mass_amu), rtol=1e-12)


def test_coolest_layer_matches_the_oracle_profile():
    oracle = pytest.importorskip("oracle")
    import workloads as W
    P = W.pressure_layers(30)[0]
    for th in ((1300.0, 0.1), (1000.0, 0.2), (1600.0, 0.05)):
        assert serve.coolest_layer_T(th, P) == pytest.approx(float(np.min(oracle.temperatures(th[0], th[1], P))),
                                                             rel=1e-14)


def test_modit_rule_separates_negative_from_nonnegative_cross_sections():
    """The oracle's MODIT cross-section goes negative near lines when the grid is
    coarser than the Doppler width, and stays non-negative in every layer once the
    rule (beta' >= MODIT_MIN_BETA_Q in the coolest layer) admits the grid."""
    oracle = pytest.importorskip("oracle")
    import workloads as W
    P = W.pressure_layers(30)[0]
    th = (1300.0, 0.1)
    T = oracle.temperatures(th[0], th[1], P)
    t_min = serve.coolest_layer_T(th, P)
    species = ((W.water_like(300, seed=5), 18.0), (W.co_like(100, seed=6), 28.0))
    for N, admitted in ((3000, False), (8000, False), (12_000, True), (16_000, True)):
        nu = W.grid_lognu(N)
        bq = min(serve.modit_beta_q(N, t_min, m) for _, m in species)
        assert (bq >= serve.MODIT_MIN_BETA_Q) == admitted
        lo = min(float(np.min(oracle.modit(ll, nu[0], nu[-1], N, T, P, 1.0, n_gamma=16))) for ll, _ in species)
        if admitted:
            assert lo >= 0.0
        elif N == 3000:
            assert lo < 0.0
