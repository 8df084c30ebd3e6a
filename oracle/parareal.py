"""Serial fine solve, synchronous Parareal and asynchronous replay (FP64).

Indexing (§3.1): the interval [T_0, T_N] is cut into N slices; lambda_i is
the state at T_i, i = 0..N, with lambda_0 = u^(0) fixed.  States are stored
flattened, one row per i: lam has shape (N+1, M).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .heat import Propagators


def _flat(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float64).reshape(-1)


def serial_fine(prob: dict, u0=None, kappa="from_prob") -> np.ndarray:
    """lambda*_0 = u0, lambda*_i = F(lambda*_{i-1}) (§3.1, Eq. (10) and the
    composition F o F o ... o F that Parareal replaces)."""
    P = Propagators(prob, kappa)
    u0 = prob["u0"] if u0 is None else u0
    N = int(prob["N"])
    lam = np.zeros((N + 1, _flat(u0).size))
    lam[0] = _flat(u0)
    for i in range(1, N + 1):
        lam[i] = _flat(P.F(lam[i - 1]))
    return lam


@dataclass
class SyncResult:
    lam: np.ndarray                       # final (N+1, M)
    k: int                                # iterations done after the predictor
    deltas: list = field(default_factory=list)     # per iteration: (N,) max-abs increments
    iterates: list = field(default_factory=list)   # lam^0, lam^1, ... when recorded
    cg_iters: list = field(default_factory=list)   # per iteration: (N,) CG counts (0 = no solve)
    predictor_cg: np.ndarray | None = None
    w: np.ndarray | None = None           # final coarse values w_i


def sync_parareal(prob: dict, u0=None, tol=None, max_iter=None, record=False,
                  kappa="from_prob") -> SyncResult:
    """Synchronous Parareal exactly as Algorithm 1 (§4.1), i.e. Eq. (11) with
    the converged prefix frozen.

    Predictor (Algorithm 1, first lines; §3.1 initial guess):
        lambda_0^0 = u0,  w_i^0 = G(lambda_{i-1}^0),  lambda_i^0 = w_i^0.
    Iteration k = 0, 1, ... (slices in order i = 1..N):
        if i > k:   v_i = F(lambda_{i-1}^k)
                    w_i^{k+1} = G(lambda_{i-1}^{k+1})  if i-1 > k,  else w_i^k
                    lambda_i^{k+1} = (w_i^{k+1} + v_i) - w_i^k
        else:       lambda_i^{k+1} = lambda_i^k
    Convergence test (§5.1, Eq. (22)): delta_i = max_x |lambda_i^{k+1} - lambda_i^k|;
    stop when max_i delta_i < tol (strict), or k = N (finite termination,
    §3.2), or k = max_iter.  tol = 0 runs exactly max_iter iterations.
    The CG start of each coarse solve is the slice's previous coarse value w_i^k
    (the predictor starts from its right-hand side).
    """
    P = Propagators(prob, kappa)
    u0 = prob["u0"] if u0 is None else u0
    N = int(prob["N"])
    tol = float(prob.get("tol", 0.0)) if tol is None else float(tol)
    max_iter = N if max_iter is None else min(int(max_iter), N)
    M = _flat(u0).size
    lam = np.zeros((N + 1, M))
    w = np.zeros((N + 1, M))
    lam[0] = _flat(u0)
    pred_cg = np.zeros(N, dtype=np.int64)
    for i in range(1, N + 1):
        wi, it = P.G(lam[i - 1])
        w[i] = _flat(wi)
        lam[i] = w[i]
        pred_cg[i - 1] = it
    res = SyncResult(lam=lam, k=0, predictor_cg=pred_cg)
    if record:
        res.iterates.append(lam.copy())
    k = 0
    while k < max_iter:
        new = lam.copy()
        cg = np.zeros(N, dtype=np.int64)
        for i in range(1, N + 1):
            if i > k:
                v = _flat(P.F(lam[i - 1]))
                if i - 1 > k:
                    wn, it = P.G(new[i - 1], x0=w[i])
                    wn = _flat(wn)
                    cg[i - 1] = it
                else:
                    wn = w[i]
                new[i] = (wn + v) - w[i]
                w[i] = wn
            # else: frozen, new[i] already equals lam[i]
        delta = np.max(np.abs(new[1:] - lam[1:]), axis=1) if M else np.zeros(N)
        lam = new
        k += 1
        res.deltas.append(delta)
        res.cg_iters.append(cg)
        if record:
            res.iterates.append(lam.copy())
        if np.max(delta) < tol or k == N:
            break
    res.lam = lam
    res.k = k
    res.w = w
    return res


@dataclass
class ReplayResult:
    lam: np.ndarray                 # each slice's last version, (N+1, M)
    versions: dict                  # (i, version) -> state
    deltas: dict                    # (i, version) -> max-abs change vs previous version


def async_replay(prob: dict, events, u0=None, kappa="from_prob") -> ReplayResult:
    """Recompute an asynchronous Parareal run from its event log (Eq. (12), Algorithm 2).

    Each event is (i, k, vF, vG): slice i (1..N) produced its version k
    from version vF of lambda_{i-1} for the fine/correction input and version
    vG for the coarse input (the delays tau_{i-1,2} and tau_{i-1,1}):

        lambda_i^k = (G(lambda_{i-1}^{vG}) + F(lambda_{i-1}^{vF})) - G(lambda_{i-1}^{vF})

    where G(lambda_{i-1}^{vF}) is the slice's stored coarse value w_i from its
    previous event (whose vG equals this vF; Algorithm 2 reuses w_i^{k_i}) or
    from the predictor for k = 1.  When vG = vF the coarse input has not
    changed and the new coarse value is the stored one (no solve), so the
    update is exactly F(lambda_{i-1}^{vF}).  The CG start is the stored w_i.
    Version 0 of every slice is the predictor value; slice 0 is u0 forever.
    """
    P = Propagators(prob, kappa)
    u0 = prob["u0"] if u0 is None else u0
    N = int(prob["N"])
    M = _flat(u0).size
    versions = {(0, 0): _flat(u0)}
    w = {}
    lam0 = _flat(u0)
    for i in range(1, N + 1):
        wi, _ = P.G(lam0)
        w[i] = _flat(wi)
        versions[(i, 0)] = w[i].copy()
        lam0 = w[i]
    by_slice = {i: [] for i in range(1, N + 1)}
    for ev in events:
        i, k, vF, vG = (int(e) for e in ev[:4])
        by_slice[i].append((k, vF, vG))
    deltas = {}
    last = {0: 0}
    for i in range(1, N + 1):
        evs = sorted(by_slice[i])
        prev_vG = 0
        last[i] = 0
        for n_ev, (k, vF, vG) in enumerate(evs, start=1):
            if k != n_ev:
                raise ValueError(f"slice {i}: versions not consecutive at {k}")
            if vF != prev_vG:
                raise ValueError(f"slice {i} v{k}: fine input {vF} != previous coarse input {prev_vG}")
            if (i - 1, vF) not in versions or (i - 1, vG) not in versions or vG < vF:
                raise ValueError(f"slice {i} v{k}: input version missing")
            v = _flat(P.F(versions[(i - 1, vF)]))
            if vG == vF:
                wn = w[i]
            else:
                wn, _ = P.G(versions[(i - 1, vG)], x0=w[i])
                wn = _flat(wn)
            new = (wn + v) - w[i]
            deltas[(i, k)] = float(np.max(np.abs(new - versions[(i, k - 1)]))) if M else 0.0
            versions[(i, k)] = new
            w[i] = wn
            prev_vG = vG
            last[i] = k
    lam = np.zeros((N + 1, M))
    for i in range(N + 1):
        lam[i] = versions[(i, last[i])]
    return ReplayResult(lam=lam, versions=versions, deltas=deltas)
