"""Continuous-batching server for forward + gradient requests of the emission model.

Many HMC chains send requests of uneven size (line count, grid size, layer count).
Line lists stay resident on the device (a pool registered once); each admitted
request gets a slot (its own CUDA stream) and a contiguous region of one
preallocated device arena holding its workspace and buffers.  Requests are
admitted in arrival order as slots and arena memory free up (a request that does
not fit lets smaller ones behind it go first, up to a bounded skip), so work of
several requests overlaps on the GPU.  Completion is detected by polling CUDA
events; every wait is bounded.

The scheduling core (Arena, Scheduler) is plain host code and runs with any
executor; `LibxsExecutor` launches the work through libxs (xs_model_logl_grad),
with the direct line sum or, per request, MODIT.
"""
from __future__ import annotations

import bisect
import ctypes as C
import heapq
import itertools
import math
import time
from dataclasses import dataclass, field

import numpy as np

import workloads as W

ALIGN = 256

# MODIT (Sec. 2.1.2) multiplies by the Gaussian's transform only up to the Nyquist
# frequency of the q grid, so the grid must resolve the Doppler width (Sec. 4 asks
# for R0 >~ 5e5 to resolve the line profile).  Below about one q step the cut
# transform rings and the cross-section goes negative near lines, which an optical
# depth cannot take.  A MODIT request is admitted only when beta', the Doppler
# width in q steps, is at least this for every species in the coolest layer.
MODIT_MIN_BETA_Q = 1.5
_KB, _AMU, _C = 1.380649e-16, 1.66053906660e-24, 2.99792458e10  # cgs


def modit_beta_q(n_grid, T, mass_amu, nu_min=W.NU_MIN, nu_max=W.NU_MAX):
    """beta' = R0 sqrt(kB T/(M m_u))/c (Sec. 2.1.2), the Doppler width in steps
    of q = R0 ln nu, R0 = (N - 1)/ln(nu_max/nu_min), on an N-point log grid."""
    R0 = (n_grid - 1) / math.log(nu_max / nu_min)
    return R0 * math.sqrt(_KB * T / (mass_amu * _AMU)) / _C


def coolest_layer_T(theta, p_bar):
    """Smallest layer temperature of the power law T0 P^alpha (Sec. 5.2)."""
    return float(np.min(float(theta[0]) * np.asarray(p_bar, dtype=np.float64) ** float(theta[1])))

# request status
PENDING, RUNNING, DONE, REJECTED, FAILED, CANCELLED = "pending", "running", "done", "rejected", "failed", "cancelled"


def _align(v):
    return (int(v) + ALIGN - 1) // ALIGN * ALIGN


class Arena:
    """First-fit allocator over [0, size) bytes with coalescing free list."""

    def __init__(self, size: int, fail_hook=None):
        self.size = int(size)
        self.free = [(0, self.size)]  # sorted (offset, length)
        self.used = 0
        self.fail_hook = fail_hook  # callable(nbytes) -> bool, True makes alloc fail (fault injection)

    def alloc(self, nbytes: int):
        n = _align(nbytes)
        if self.fail_hook is not None and self.fail_hook(n):
            return None
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                self.used += n
                return off, n
        return None

    def release(self, block):
        off, n = block
        i = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(i, (off, n))
        # coalesce with neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)
        self.used -= n

    def largest_free(self):
        return max((ln for _, ln in self.free), default=0)


@dataclass
class Request:
    rid: int
    chain: int
    n_lines: int
    n_grid: int
    n_layers: int
    theta: np.ndarray
    method: str = "lpf"  # cross-section: "lpf" (direct line sum) or "modit"
    high_priority: bool = False  # ran on its slot's high-priority stream
    t_submit: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    status: str = PENDING
    nbytes: int = 0
    block: tuple = None
    slot: int = -1
    result: np.ndarray = None  # [logL, dlogL/dtheta...]
    error: str = ""
    evals: int = 0
    handle: object = None

    @property
    def latency(self):
        return self.t_done - self.t_submit


class Scheduler:
    """Admission by slots and arena memory, completion by polling the executor."""

    def __init__(self, executor, arena_bytes: int, slots: int, max_skip: int = 8, clock=time.perf_counter):
        self.ex = executor
        self.arena = Arena(arena_bytes, fail_hook=getattr(executor, "fail_hook", None))
        self.slots = [None] * slots
        self.queue = []  # FIFO of pending requests
        self.max_skip = max_skip
        self.clock = clock
        self.done = []
        self.counts = {"admitted": 0, "rejected": 0, "failed": 0, "cancelled": 0, "completed": 0}

    def submit(self, req: Request):
        req.t_submit = self.clock()
        req.nbytes = self.ex.bytes_needed(req)
        if req.nbytes <= 0 or req.nbytes > self.arena.size or not self.ex.valid(req):
            req.status = REJECTED
            if req.nbytes <= 0 or not self.ex.valid(req):
                why = getattr(self.ex, "invalid_reason", None)
                req.error = (why(req) if why is not None else "") or "invalid request"
            else:
                req.error = "exceeds device budget"
            req.t_done = req.t_submit
            self.counts["rejected"] += 1
            self.done.append(req)
            return req
        req.status = PENDING
        self.queue.append(req)
        return req

    def cancel(self, req: Request) -> bool:
        if req.status == PENDING and req in self.queue:
            self.queue.remove(req)
            req.status = CANCELLED
            req.t_done = self.clock()
            self.counts["cancelled"] += 1
            self.done.append(req)
            return True
        return False

    def _admit(self):
        progressed = False
        i = 0
        while i < len(self.queue) and i <= self.max_skip:
            free = [k for k, s in enumerate(self.slots) if s is None]
            if not free:
                break
            req = self.queue[i]
            block = self.arena.alloc(req.nbytes)
            if block is None:
                i += 1  # let a smaller request behind it try (bounded skip)
                continue
            self.queue.pop(i)
            k = free[0]
            req.block, req.slot, req.status = block, k, RUNNING
            req.t_start = self.clock()
            try:
                req.handle = self.ex.launch(req, block, k)
            except Exception as e:  # launch failure: free and report, others unaffected
                self.arena.release(block)
                req.status, req.error, req.t_done = FAILED, str(e), self.clock()
                self.counts["failed"] += 1
                self.done.append(req)
                continue
            self.slots[k] = req
            self.counts["admitted"] += 1
            progressed = True
        return progressed

    def _poll(self):
        progressed = False
        for k, req in enumerate(self.slots):
            if req is not None and self.ex.ready(req):
                try:
                    req.result = self.ex.collect(req)
                    req.status = DONE
                    self.counts["completed"] += 1
                except Exception as e:
                    req.status, req.error = FAILED, str(e)
                    self.counts["failed"] += 1
                req.t_done = self.clock()
                self.arena.release(req.block)
                self.slots[k] = None
                self.done.append(req)
                progressed = True
        return progressed

    def step(self):
        a = self._poll()
        b = self._admit()
        return a or b

    def busy(self):
        return bool(self.queue) or any(s is not None for s in self.slots)

    def drain(self, timeout_s: float = 600.0):
        t0 = self.clock()
        while self.busy():
            if not self.step():
                time.sleep(0.0002)
            if self.clock() - t0 > timeout_s:
                raise TimeoutError("drain timed out")


# ------------------------------------------------------------------ libxs executor


class LinePool:
    """Water-like line lists of log-spaced sizes, sorted and resident on the device."""

    SIZES = (1000, 3000, 10_000, 30_000, 100_000, 300_000, 1_000_000)

    def __init__(self, device="cuda", sizes=SIZES, seed=W.SEED_SERVE):
        from . import xs
        self.sizes = list(sizes)
        hosts = {n: W.water_like(n, seed=seed + i) for i, n in enumerate(self.sizes)}
        co = W.co_like(2000, seed=seed + 100)
        self.lists = {n: xs.DeviceLines(h, device) for n, h in hosts.items()}
        self.co = xs.DeviceLines(co, device)
        # lowest and highest centre of each list (MODIT's padded period), from the host copies
        self.spans = {n: (float(np.min(h.nu_hat)), float(np.max(h.nu_hat))) for n, h in hosts.items()}
        self.co_span = (float(np.min(co.nu_hat)), float(np.max(co.nu_hat)))
        # sum over lines of the fraction of a full-band log grid inside each line's
        # wing cut: in-cut pairs of an N-point grid ~ fraction * N (for reporting)
        ref = W.grid_lognu(200_001)
        def frac(c):
            return float(np.sum(np.searchsorted(ref, c + 25.0, "right") - np.searchsorted(ref, c - 25.0, "left"))) / ref.size
        self._frac = {n: frac(np.sort(h.nu_hat)) for n, h in hosts.items()}
        self.co_fraction = frac(np.sort(co.nu_hat))

    def cut_fraction(self, n):
        return self._frac[n]

    def nearest(self, n):
        return min(self.sizes, key=lambda s: abs(math.log(s) - math.log(max(n, 1))))


class LibxsExecutor:
    """Runs a request as xs_model_logl_grad on its slot's stream, inside its arena
    block: [model workspace | grid | P | dP | d_obs | sig_obs | out].  A request
    with method "modit" takes the MODIT cross-section (n_gamma width nodes).
    With hi_streams (one higher-priority stream per slot), line-sum requests of
    fewer than hi_evals Voigt evaluations run on their slot's high-priority stream,
    so that the block scheduler runs their kernels ahead of the long ones."""

    def __init__(self, pool: LinePool, arena_tensor, streams, prec=1, fail_hook=None, n_gamma=16, hi_streams=None,
                 hi_evals=1e11):
        import torch
        from . import xs
        self.torch, self.xs = torch, xs
        self.pool = pool
        self.arena_t = arena_tensor
        self.base = arena_tensor.data_ptr()
        self.streams = streams
        self.hi_streams, self.hi_evals = hi_streams, float(hi_evals)
        self.prec = prec
        self.fail_hook = fail_hook
        self.n_gamma = int(n_gamma)
        self.lib = xs.lib()
        # per-slot pinned host staging, allocated once (grown only for a larger
        # request): a slot's next request starts after its previous one completed,
        # so its copies have drained
        self.stage = [None] * len(streams)
        self.outs = [torch.empty(8, dtype=torch.float64).pin_memory() for _ in streams]

    def _staging(self, slot, n):
        buf = self.stage[slot]
        if buf is None or buf.numel() < n:
            cap = max(n, 4 * 50_000 + 2 * 1000, 0 if buf is None else 2 * buf.numel())
            buf = self.torch.empty(cap, dtype=self.torch.float64).pin_memory()
            self.stage[slot] = buf
        return buf

    def invalid_reason(self, r):
        """Why the request cannot run ("" when it can)."""
        if not (r.n_lines >= 1 and 2 <= r.n_grid <= 2_000_000 and 1 <= r.n_layers <= 1000
                and np.all(np.isfinite(r.theta))):
            return "invalid request"
        if r.method not in ("lpf", "modit"):
            return f"unknown method {r.method!r}"
        if r.method == "modit":
            T_min = coolest_layer_T(r.theta, W.pressure_layers(r.n_layers)[0])
            mass = max(l.mass_amu for l in self._lines(r))
            bq = modit_beta_q(r.n_grid, T_min, mass)
            if not bq >= MODIT_MIN_BETA_Q:
                return (f"grid too coarse for MODIT: Doppler width {bq:.2f} q steps at {T_min:.0f} K "
                        f"(needs {MODIT_MIN_BETA_Q})")
        return ""

    def valid(self, r):
        return self.invalid_reason(r) == ""

    def _lines(self, r):
        return [self.pool.lists[self.pool.nearest(r.n_lines)], self.pool.co]

    def _model(self, r, ptrs=None):
        xs = self.xs
        sp = (xs.XsLinesC * xs.MAX_SPECIES)()
        for i, s in enumerate(self._lines(r)):
            sp[i] = s.struct()
        p = ptrs or {}
        m = xs.XsModelC(2, sp, p.get("nu"), r.n_grid, p.get("P"), p.get("dP"), r.n_layers, 25.0, 1e5, 2.313, 1e-8,
                        p.get("d"), p.get("s"), self.prec)
        if r.method == "modit":
            nu = W.grid_lognu(r.n_grid)  # the request's grid, whose ends MODIT's q axis takes
            nu0, nu1 = float(nu[0]), float(nu[-1])
            m.method, m.n_gamma, m.nu_min, m.nu_max = 1, self.n_gamma, nu0, nu1
            spans = (self.pool.spans[self.pool.nearest(r.n_lines)], self.pool.co_span)
            for i, (lines, span) in enumerate(zip(self._lines(r), spans)):
                m.n_fft[i] = xs.modit_fft_length(nu0, nu1, r.n_grid, lines, span=span)
        return m

    def _layout(self, r):
        # sizing only: the model check wants non-null buffers, any device address will do
        m = self._model(r, {k: self.base for k in ("nu", "P", "dP", "d", "s")})
        ws = self.lib.xs_model_workspace_bytes(C.byref(m))
        N, L = r.n_grid, r.n_layers
        parts = [("ws", ws), ("nu", 8 * N), ("P", 8 * L), ("dP", 8 * L), ("d", 8 * N), ("s", 8 * N), ("out", 8 * 8)]
        off, lay = 0, {}
        for k, n in parts:
            lay[k] = (off, n)
            off += _align(n)
        return lay, off

    def bytes_needed(self, r):
        if not self.valid(r):
            return -1
        return self._layout(r)[1]

    def launch(self, r, block, slot):
        torch = self.torch
        lay, _ = self._layout(r)
        off0 = block[0]
        ptr = {k: self.base + off0 + o for k, (o, n) in lay.items()}
        short = self.hi_streams is not None and r.method == "lpf" and self.work(r) < self.hi_evals
        st = self.hi_streams[slot] if short else self.streams[slot]
        r.high_priority = short
        # request inputs from the host (pinned), copied on the slot's stream
        N, L = r.n_grid, r.n_layers
        nu = W.grid_lognu(N)
        P, dP = W.pressure_layers(L)
        sizes = [N, L, L, N, N]
        host = self._staging(slot, sum(sizes))
        hn = host.numpy()
        o = 0
        for v in (nu, P, dP, np.ones(N), np.full(N, 0.01)):
            hn[o:o + v.size] = v
            o += v.size
        with torch.cuda.stream(st):
            o = 0
            for key, n in zip(("nu", "P", "dP", "d", "s"), sizes):
                dst = self.arena_t.narrow(0, off0 + lay[key][0], 8 * n).view(torch.float64)
                dst.copy_(host[o:o + n], non_blocking=True)
                o += n
        m = self._model(r, ptr)
        th = (C.c_double * 5)(*[float(v) for v in r.theta])
        code = self.lib.xs_model_logl_grad(C.byref(m), th, C.c_void_p(ptr["out"]), None, C.c_void_p(ptr["ws"]),
                                           lay["ws"][1], C.c_void_p(st.cuda_stream))
        if code != 0:
            raise RuntimeError(f"xs_model_logl_grad: {code}")
        out_h = self.outs[slot][:6]
        with torch.cuda.stream(st):
            out_h.copy_(self.arena_t.narrow(0, off0 + lay["out"][0], 48).view(torch.float64), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
        r.evals = 0 if r.method == "modit" else self.work(r)  # MODIT evaluates no Voigt profile
        return (ev, out_h, host)

    def work(self, r):
        """Voigt evaluations of the request's line sum, forward and adjoint."""
        N = r.n_grid
        return 2 * r.n_layers * (self.pool.cut_fraction(self.pool.nearest(r.n_lines)) * N + self.pool.co_fraction * N)

    def ready(self, r):
        return r.handle[0].query()

    def collect(self, r):
        out = r.handle[1].numpy().copy()
        if not np.all(np.isfinite(out)):
            raise RuntimeError("non-finite result")
        return out


# ------------------------------------------------------------------ closed-loop HMC load


def request_stream(n, seed=W.SEED_SERVE):
    nl, ng, nlay = W.serving_requests(n, seed)
    th = W.theta_points(n, seed + 1)
    return [Request(rid=i, chain=-1, n_lines=int(nl[i]), n_grid=int(ng[i]), n_layers=int(nlay[i]), theta=th[i])
            for i in range(n)]


def closed_loop(sched: Scheduler, chains: int, offered_rate: float, duration_s: float, seed=W.SEED_SERVE,
                timeout_s: float = 900.0, cancel_at_end: bool = False):
    """`chains` HMC chains, each with at most one request outstanding; after its
    result a chain thinks Exp(mean chains/offered_rate) before the next one, so the
    offered rate is `offered_rate` when the server keeps up.  With
    `cancel_at_end`, requests still queued when the window closes are cancelled
    (the running ones finish), which bounds the drain of a saturated server."""
    rng = np.random.default_rng(seed + 7)
    reqs = iter(request_stream(100_000, seed))
    think = chains / offered_rate
    t0 = sched.clock()
    wake = [(t0 + rng.exponential(think), c) for c in range(chains)]
    heapq.heapify(wake)
    outstanding = {}
    finished = []
    nd = 0
    while True:
        now = sched.clock()
        if now - t0 > timeout_s:
            raise TimeoutError("closed loop timed out")
        while wake and wake[0][0] <= now and now - t0 < duration_s:
            _, c = heapq.heappop(wake)
            r = next(reqs)
            r.chain = c
            sched.submit(r)
            outstanding[r.rid] = r
        if cancel_at_end and now - t0 >= duration_s and sched.queue:
            for r in list(sched.queue):
                sched.cancel(r)
        progressed = sched.step()
        for r in sched.done[nd:]:
            nd += 1
            if r.rid in outstanding:
                del outstanding[r.rid]
                finished.append(r)
                if r.status != CANCELLED:
                    heapq.heappush(wake, (sched.clock() + rng.exponential(think), r.chain))
        if sched.clock() - t0 >= duration_s and not outstanding:
            break
        if not progressed:
            time.sleep(0.0002)
    return finished, sched.clock() - t0


def open_loop(sched: Scheduler, rate: float, duration_s: float, seed=W.SEED_SERVE, timeout_s: float = 900.0):
    """Poisson arrivals at `rate` req/s for `duration_s`, then drain."""
    rng = np.random.default_rng(seed + 9)
    reqs = iter(request_stream(100_000, seed + 1))
    t0 = sched.clock()
    t_next = t0 + rng.exponential(1.0 / rate)
    sent = []
    while True:
        now = sched.clock()
        if now - t0 > timeout_s:
            raise TimeoutError("open loop timed out")
        while t_next <= now and t_next - t0 < duration_s:
            r = next(reqs)
            r.chain = len(sent)
            sched.submit(r)
            sent.append(r)
            t_next += rng.exponential(1.0 / rate)
        progressed = sched.step()
        if now - t0 >= duration_s and not sched.busy():
            break
        if not progressed:
            time.sleep(0.0002)
    return sent, sched.clock() - t0


def mean_request_evals(pool: LinePool, n=100_000, seed=W.SEED_SERVE):
    """Expected Voigt evaluations (forward + adjoint) of one request of the stream."""
    nl, ng, nlay = W.serving_requests(n, seed)
    fr = np.array([pool.cut_fraction(pool.nearest(int(v))) for v in nl]) + pool.co_fraction
    return float(np.mean(2.0 * nlay * ng * fr))


SIZE_BINS = (0.0, 1e10, 1e11, 1e12, 1e13, float("inf"))


def latency_by_size(finished, bins=SIZE_BINS):
    """p50/p99 latency of completed requests binned by their work (Voigt evaluations)."""
    ok = [r for r in finished if r.status == DONE]
    out = []
    for lo, hi in zip(bins[:-1], bins[1:]):
        lat = np.array([r.latency for r in ok if lo <= r.evals < hi])
        if lat.size:
            out.append({"evals_from": lo, "evals_to": hi, "count": int(lat.size),
                        "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99))})
    return out


def summarize(finished, wall_s):
    ok = [r for r in finished if r.status == DONE]
    lat = np.array([r.latency for r in ok]) if ok else np.array([np.nan])
    return {"completed": len(ok), "rejected": sum(r.status == REJECTED for r in finished),
            "failed": sum(r.status == FAILED for r in finished),
            "cancelled": sum(r.status == CANCELLED for r in finished), "req_per_s": len(ok) / wall_s,
            "evals_per_s": sum(r.evals for r in ok) / wall_s,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(np.mean(lat)), "wall_s": wall_s}


def make_server(arena_bytes=int(40e9), slots=4, prec=1, device="cuda", fail_hook=None, pool=None, n_gamma=16,
                priority=False, hi_evals=1e11):
    """Scheduler + LibxsExecutor over one arena; with priority, short line-sum
    requests (< hi_evals evaluations) run on high-priority streams."""
    import torch
    pool = pool or LinePool(device)
    arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=device)
    streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
    hi = [torch.cuda.Stream(device=device, priority=-1) for _ in range(slots)] if priority else None
    ex = LibxsExecutor(pool, arena, streams, prec=prec, fail_hook=fail_hook, n_gamma=n_gamma, hi_streams=hi,
                       hi_evals=hi_evals)
    return Scheduler(ex, int(arena_bytes), slots), pool
