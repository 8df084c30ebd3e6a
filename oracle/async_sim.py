"""Discrete-event simulation of asynchronous Parareal on a virtual clock (FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

Asynchronous Parareal (§3.2, Eq. (12); Algorithm 2 of §4.1) lets every slice
iterate on whatever version of its predecessor it has received, so the order
of the updates, and therefore kappa(k~) (Proposition 3 of §4.1), depends on
the relative costs of F and G and on the communication delays.  This module
produces such orders without a GPU: workers ("teams"; one per slice is the
paper's one-processor-per-slice setting) advance a shared virtual clock in
units of one fine step, and the states are computed with the propagators of
``heat`` as the updates happen.  A run yields the same event log
(i, k, vF, vG, ...) that ``parareal.async_replay`` consumes.

Update of slice i by its worker, started at time t (Algorithm 2's loop body,
read as in the replay: the fine input is the previous coarse input, so
F(x) - G(x) share x, Eq. (12)):
  * vF := the version of lambda_{i-1} the slice holds (its last coarse input);
    v = F(lambda_{i-1}^{vF}) costs ``f_cost`` units (default n_f);
  * at t + f_cost, vG := the freshest version of lambda_{i-1} visible then
    (never older than vF); if vG > vF, w_new = G(lambda_{i-1}^{vG}) costs
    ``c_G`` more units, else w_new = w_i (nothing new, no solve);
  * lambda_i^{k+1} = (w_new + v) - w_i is published at the end of the update
    and becomes visible to slice i+1 after the injected delay
    d = delays[i-1, k % cols] units (communication delay, §4.1);
  * the worker then picks its next slice.
Visibility: a version published at t with delay d is visible at t + d (at
equal times, publications are seen before decisions).  Only the ``ring``
newest versions of a slice can be read (the storage of a bounded ring).

Work policy (which slices have an update to do), per worker, owned slices
t+1, t+1+T, ... visited round-robin from a cursor:
  * a slice that has not updated yet, or any slice in paper-literal mode, has
    work (Algorithm 2 repeats its loop unconditionally);
  * otherwise a slice has work when a newer predecessor version than its
    coarse input is visible, or when its last update read two different
    versions (vF < vG: the next update, with vF = vG, still changes it);
  * otherwise (last update idempotent, nothing newer visible) it is idle;
  * ``lazy``: a slice whose pending update has vF = vG waits until its
    predecessor is settled (see below).
A worker with no work waits until the next publication or visibility time.

Stop rule (Eq. (22) read per slice, as in the synchronous stop test): after
every publication, stop when every slice has updated at least once and each
is settled or had a last increment max|lambda_i^{k+1} - lambda_i^k| < tol.
Settled = last update idempotent with the predecessor's latest version; when
every slice is settled, lambda_i = F(lambda_{i-1}) for all i (quiescence,
the finite-time termination of Proposition 1 in §3.2).  tol = 0 runs to
quiescence.  Updates in progress at the stop complete and are logged.

Parity unpinned for the instant of the stop of a timed GPU run (it depends
on the device's timing); the schedule rules above are pinned by hand-derived
logs and the states by the finite-termination and per-mode contraction
properties (tests).
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass, field

import numpy as np

from .heat import Propagators

_PUBLISH, _CHOOSE, _DECIDE = 0, 1, 2


@dataclass
class SimEvent:
    i: int          # slice 1..N
    k: int          # version produced
    vF: int         # predecessor version of the fine input
    vG: int         # predecessor version of the coarse input
    worker: int
    t_start: float  # start of the fine propagation
    t_end: float    # publication
    t_vis: float    # visible to the successor
    delta: float    # max-abs increment against version k-1
    cg_iters: int

    def __iter__(self):  # (i, k, vF, vG, ...) as async_replay reads it
        return iter((self.i, self.k, self.vF, self.vG, self.worker, self.t_start, self.t_end,
                     self.t_vis, self.delta, self.cg_iters))

    def __getitem__(self, idx):
        return tuple(self)[idx]


@dataclass
class SimResult:
    events: list                      # SimEvent, in publication order
    lam: np.ndarray                   # each slice's last version, (N+1, M)
    k_i: np.ndarray                   # versions produced per slice, (N,)
    kappa: int                        # kappa(k~) = max_i k_i (§4.1)
    updates: int
    t_stop: float                     # virtual time of the stop decision
    t_end: float                      # last publication (in-flight updates included)
    stop_reason: str                  # "tol", "quiescent" or "limit"
    n_at_stop: int = 0                # events published when the stop was decided
    verify_rounds: int = 0            # residual checks made (verify mode)
    residual: float | None = None     # max_i max|lambda_i - F(lambda_{i-1})| at the last check
    versions: dict = field(default_factory=dict)


def async_simulate(prob: dict, workers: int | None = None, c_G: float = 1.0,
                   f_cost: float | None = None, delays=None, tol=None,
                   paper_literal: bool = False, lazy: bool = False, ring: int = 3,
                   max_updates: int = 100000, verify: bool = False, max_verify: int = 100,
                   u0=None, kappa="from_prob") -> SimResult:
    """Simulate asynchronous Parareal (Eq. (12), Algorithm 2) on a virtual clock.

    workers: number of workers T (default N, one per slice); worker t owns
    slices t+1, t+1+T, ...  c_G, f_cost: costs of one G solve and one F in
    units of one fine step (f_cost defaults to n_f).  delays: (N, cols) array
    of publication delays in the same units (None: no delay).  tol: stop
    tolerance (default prob["tol"]; 0 runs to quiescence).  verify: when the
    increment rule stops the run, check the fixed-point residual
    max_i max|lambda_i - F(lambda_{i-1})| on the latest versions (one batched F,
    f_cost units) and resume, with every slice's increment forgotten, unless it
    is below tol (at most max_verify checks).
    """
    P = Propagators(prob, kappa)
    u0 = prob["u0"] if u0 is None else u0
    N = int(prob["N"])
    T = N if workers is None else max(1, min(int(workers), N))
    tol = float(prob.get("tol", 0.0)) if tol is None else float(tol)
    f_cost = float(prob["f_steps"]) if f_cost is None else float(f_cost)
    c_G = float(c_G)
    if f_cost < 0 or c_G < 0 or ring < 1:
        raise ValueError("costs must be >= 0 and ring >= 1")
    dl = None
    if delays is not None:
        dl = np.asarray(delays, dtype=np.float64)
        if dl.ndim != 2 or dl.shape[0] != N or dl.shape[1] < 1 or np.any(dl < 0):
            raise ValueError("delays must be a non-negative (N, cols) array")

    flat = lambda x: np.asarray(x, dtype=np.float64).reshape(-1)
    # predictor (Algorithm 2 starts from the G chain): version 0 of every slice
    versions = {(0, 0): flat(u0)}
    vis = {(0, 0): 0.0}
    w = [None] * (N + 1)
    for i in range(1, N + 1):
        wi, _ = P.G(versions[(i - 1, 0)])
        w[i] = flat(wi)
        versions[(i, 0)] = w[i].copy()
        vis[(i, 0)] = 0.0
    latest = [0] * (N + 1)      # newest version of each slice (slice 0: 0 forever)
    xver = [0] * (N + 1)        # predecessor version held as the next fine input
    kcount = [0] * (N + 1)
    lastfg = [False] * (N + 1)  # last update had vF == vG
    delta = [np.inf] * (N + 1)

    def freshest_visible(j, now):
        if j == 0:
            return 0
        best = -1
        for v in range(max(0, latest[j] - ring + 1), latest[j] + 1):
            if vis[(j, v)] <= now:
                best = v
        return best

    def settled(i):
        return (not paper_literal) and lastfg[i] and xver[i] == latest[i - 1]

    def has_work(i, now):
        if kcount[i] == 0 or paper_literal:
            return True
        if i > 1 and freshest_visible(i - 1, now) > xver[i]:
            return True
        if lastfg[i]:
            return False
        if not lazy or i == 1:
            return True
        j = i - 1
        return kcount[j] > 0 and lastfg[j] and xver[j] == latest[j - 1]

    def stop_condition():
        quiet, below = True, tol > 0
        for i in range(1, N + 1):
            if kcount[i] < 1:
                return False, ""
            s = settled(i)
            quiet = quiet and s
            if below and not s and not (delta[i] < tol):
                below = False
        return quiet or below, ("quiescent" if quiet else "tol")

    owned = [list(range(t + 1, N + 1, T)) for t in range(T)]
    cursor = [0] * T
    job = [None] * T          # the update in progress of each worker
    wake = [None] * T         # id of the worker's one valid pending decision
    waiting = set()           # idle workers, woken by the next publication
    heap, seq = [], 0

    def push(t, kind, worker):
        nonlocal seq
        heapq.heappush(heap, (t, kind, worker, seq))
        seq += 1
        if kind == _DECIDE:
            wake[worker] = seq - 1

    for t in range(T):
        push(0.0, _DECIDE, t)
    events = []
    stopped, t_stop, reason, t_last, n_at_stop = False, None, "limit", 0.0, 0

    verify_rounds, residual = 0, None
    while True:
        while heap:
            t, kind, wk, sq = heapq.heappop(heap)
            if kind == _DECIDE:
                if stopped or sq != wake[wk]:
                    continue
                wake[wk] = None
                pick = None
                own = owned[wk]
                for c in range(len(own)):
                    i = own[(cursor[wk] + c) % len(own)]
                    if has_work(i, t):
                        pick = i
                        cursor[wk] = (cursor[wk] + c + 1) % len(own)
                        break
                if pick is not None:
                    waiting.discard(wk)
                    job[wk] = dict(i=pick, k=kcount[pick], vF=xver[pick], t0=t)
                    push(t + f_cost, _CHOOSE, wk)
                    continue
                ok, why = stop_condition()
                if ok:
                    stopped, t_stop, reason, n_at_stop = True, t, why, len(events)
                    continue
                # idle: wait for the next visibility instant or publication
                waiting.add(wk)
                future = [tv for tv in vis.values() if tv > t]
                if future:
                    push(min(future), _DECIDE, wk)
            elif kind == _CHOOSE:
                jb = job[wk]
                i, vF = jb["i"], jb["vF"]
                v = flat(P.F(versions[(i - 1, vF)]))
                cand = freshest_visible(i - 1, t)
                vG = cand if cand > vF else vF
                cg = 0
                if vG > vF:
                    wn, cg = P.G(versions[(i - 1, vG)], x0=w[i])
                    wn = flat(wn)
                    t_pub = t + c_G
                else:
                    wn = w[i]
                    t_pub = t
                new = (wn + v) - w[i]
                jb.update(vG=vG, wn=wn, new=new, cg=int(cg))
                push(t_pub, _PUBLISH, wk)
            else:  # _PUBLISH
                jb = job[wk]
                job[wk] = None
                i, k = jb["i"], jb["k"]
                d = float(np.max(np.abs(jb["new"] - versions[(i, k)]))) if jb["new"].size else 0.0
                tv = t + (dl[i - 1, k % dl.shape[1]] if dl is not None else 0.0)
                versions[(i, k + 1)] = jb["new"]
                vis[(i, k + 1)] = tv
                latest[i] = k + 1
                delta[i] = d
                xver[i] = jb["vG"]
                lastfg[i] = jb["vG"] == jb["vF"]
                kcount[i] = k + 1
                w[i] = jb["wn"]
                events.append(SimEvent(i, k + 1, jb["vF"], jb["vG"], wk, jb["t0"], t, tv, d, jb["cg"]))
                t_last = t
                if stopped:
                    continue
                ok, why = stop_condition()
                if ok:
                    stopped, t_stop, reason, n_at_stop = True, t, why, len(events)
                elif len(events) >= max_updates:
                    stopped, t_stop, reason, n_at_stop = True, t, "limit", len(events)
                else:
                    push(t, _DECIDE, wk)
                    for other in sorted(waiting):
                        push(t, _DECIDE, other)
                    waiting.clear()

        if not stopped:
            # every worker idle, nothing in flight and nothing left to become visible
            ok, why = stop_condition()
            if not ok:
                raise RuntimeError("no worker can make progress and the stop rule does not hold")
            t_stop, reason, n_at_stop = t_last, why, len(events)

        if not verify or reason != "tol":
            break
        # residual of the fixed point lambda_i = F(lambda_{i-1}) on the latest
        # versions: one batched F, f_cost units after the last publication
        cur = [versions[(i, latest[i])] for i in range(N + 1)]
        residual = max(float(np.max(np.abs(cur[i] - flat(P.F(cur[i - 1])))))
                       for i in range(1, N + 1))
        verify_rounds += 1
        t_last = max(t_last, t_stop) + f_cost
        if residual < tol or verify_rounds >= max_verify:
            break
        # resume: every unsettled slice must publish again before the rule fires
        for i in range(1, N + 1):
            delta[i] = np.inf
        stopped, t_stop, reason = False, None, "limit"
        waiting.clear()
        for wk in range(T):
            push(t_last, _DECIDE, wk)

    M = versions[(0, 0)].size
    lam = np.zeros((N + 1, M))
    for i in range(N + 1):
        lam[i] = versions[(i, latest[i])]
    k_i = np.array(kcount[1:], dtype=np.int64)
    return SimResult(events=events, lam=lam, k_i=k_i, kappa=int(k_i.max()) if N else 0,
                     updates=len(events), t_stop=t_stop if t_stop is not None else t_last,
                     t_end=t_last, stop_reason=reason, n_at_stop=n_at_stop,
                     verify_rounds=verify_rounds, residual=residual, versions=versions)
