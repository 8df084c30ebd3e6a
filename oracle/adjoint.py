"""Discrete adjoint of K synchronous Parareal iterations (reverse mode), FP64.

Forward map (Algorithm 1 of §4.1 with the converged prefix frozen, exactly K
iterations, no early stop; Eq. (11)):
    lambda_0 = u0;  w_i^0 = G lambda_{i-1}^0,  lambda_i^0 = w_i^0
    for k = 0..K-1, i = 1..N:
        i > k:  v_i^k = F lambda_{i-1}^k
                w_i^{k+1} = G lambda_{i-1}^{k+1} if i-1 > k else w_i^k
                lambda_i^{k+1} = w_i^{k+1} + v_i^k - w_i^k
        else:   lambda_i^{k+1} = lambda_i^k
    L = 1/2 ||lambda_N^K - u_obs||^2 (the caller supplies dL/dlambda_N).
F = S^{n_f} with S = I - dt A_kappa (explicit) or S = (I + dt A_kappa)^{-1}
(implicit, 1D) and G = (I + dT A_kappa)^{-1} are symmetric, so F^T = F and
G^T = G.  G is taken as the exact solve (CG to the problem's g_rtol, which
callers set tight, or Thomas in 1D).

Diffusivity derivative: <a, A_kappa u> = sum_faces h^-2 kappa_f (a_p-a_q)(u_p-u_q)
with kappa_f = (kappa_p + kappa_q)/2, so each face adds h^-2 (Da)_f (Du)_f / 2 to
both of its nodes (boundary-ring nodes included).  Then
    d<abar, S^n x>/dkappa = -dt sum_j facegrad(S^{n-1-j} abar, S^j x)          (explicit)
    d<abar, S^n x>/dkappa = -dt sum_j facegrad(S^{n-j} abar, S^{j+1} x)        (implicit)
    d<wbar, G b>/dkappa   = -dT facegrad(G wbar, G b).
(implicit: u_{j+1} = S u_j with S = (I + dt A)^{-1}, whose derivative is
-S dt (dA/dkappa) S.)
"""
from __future__ import annotations

import numpy as np

from .heat import Propagators, _h_of_axis, explicit_euler, implicit_euler_1d


def face_grad(a: np.ndarray, u: np.ndarray, h, ring_shape) -> np.ndarray:
    """d<a, A_kappa u>/d(kappa nodes), an array of the ring shape (n+2 per axis)."""
    d = a.ndim
    A = np.pad(a, 1)
    U = np.pad(u, 1)
    g = np.zeros(ring_shape)
    for ax in range(d):
        inner = [slice(1, -1)] * d
        inner[ax] = slice(None)
        Aa, Ua = A[tuple(inner)], U[tuple(inner)]
        hi = [slice(None)] * d
        lo = [slice(None)] * d
        hi[ax] = slice(1, None)
        lo[ax] = slice(None, -1)
        contrib = 0.5 * (Aa[tuple(hi)] - Aa[tuple(lo)]) * (Ua[tuple(hi)] - Ua[tuple(lo)])
        contrib = contrib / _h_of_axis(h, d, ax) ** 2
        ghi = [slice(1, -1)] * d
        glo = [slice(1, -1)] * d
        ghi[ax] = slice(1, None)
        glo[ax] = slice(None, -1)
        g[tuple(glo)] += contrib     # node on the low side of each face
        g[tuple(ghi)] += contrib     # node on the high side
    return g


class _Ops:
    def __init__(self, prob, kappa):
        self.P = Propagators(prob, kappa)
        self.shape = self.P.shape
        self.ring = tuple(s + 2 for s in self.shape)

    def F(self, x):
        return self.P.F(x.reshape(self.shape)).reshape(-1)

    def G(self, x):
        return self.P.G(x.reshape(self.shape))[0].reshape(-1)

    def F_adj(self, x, abar, want_kappa):
        """(F^T abar, d<abar, F x>/dkappa) with the fine states recomputed from x."""
        P = self.P
        if P.f_scheme == "implicit":
            states = [x.reshape(self.shape)]
            for _ in range(P.f_steps):
                states.append(implicit_euler_1d(states[-1], P.dt, P.h, P.kappa, 1))
            a = abar.reshape(self.shape)
            gk = np.zeros(self.ring) if want_kappa else None
            for j in range(P.f_steps - 1, -1, -1):
                a = implicit_euler_1d(a, P.dt, P.h, P.kappa, 1)      # S^T = S
                if want_kappa:
                    gk -= P.dt * face_grad(a, states[j + 1], P.h, self.ring)
            return a.reshape(-1), gk
        states = [x.reshape(self.shape)]
        for _ in range(P.f_steps - 1):
            states.append(explicit_euler(states[-1], P.dt, P.h, P.kappa, 1))
        a = abar.reshape(self.shape)
        gk = np.zeros(self.ring) if want_kappa else None
        for j in range(P.f_steps - 1, -1, -1):
            if want_kappa:
                gk -= P.dt * face_grad(a, states[j], P.h, self.ring)
            a = explicit_euler(a, P.dt, P.h, P.kappa, 1)      # S^T = S
        return a.reshape(-1), gk

    def G_adj(self, b_out, wbar, want_kappa):
        """(G^T wbar, d<wbar, G b>/dkappa) given the forward output w = G b."""
        z = self.G(wbar)
        gk = None
        if want_kappa:
            gk = -self.P.dT * face_grad(z.reshape(self.shape), b_out.reshape(self.shape),
                                        self.P.h, self.ring)
        return z, gk


def adjoint_sync(prob: dict, dL_dlamN, K: int, u0=None, kappa="from_prob"):
    """Gradients (dL/du0, dL/dkappa) of L through K sync iterations.

    Returns (grad_u0 with the state's shape, grad_kappa with the ring shape or
    None for constant kappa, lam_N^K).  Explicit fine propagator only.
    """
    ops = _Ops(prob, kappa)
    if ops.P.f_scheme not in ("explicit", "implicit") or ops.P.g_steps != 1:
        raise ValueError("adjoint oracle covers explicit and 1D implicit fine propagators, one coarse step")
    want_k = ops.P.kappa is not None
    u0 = prob["u0"] if u0 is None else u0
    N = int(prob["N"])
    M = int(np.prod(ops.shape))
    # ---- forward, keeping every iterate
    lam = [np.zeros((N + 1, M))]
    w = [np.zeros((N + 1, M))]
    lam[0][0] = np.asarray(u0, dtype=np.float64).reshape(-1)
    for i in range(1, N + 1):
        w[0][i] = ops.G(lam[0][i - 1])
        lam[0][i] = w[0][i]
    for k in range(K):
        ln = lam[k].copy()
        wn = w[k].copy()
        for i in range(1, N + 1):
            if i > k:
                v = ops.F(lam[k][i - 1])
                if i - 1 > k:
                    wn[i] = ops.G(ln[i - 1])
                ln[i] = (wn[i] + v) - w[k][i]
        lam.append(ln)
        w.append(wn)
    # ---- reverse
    lb = [np.zeros((N + 1, M)) for _ in range(K + 1)]
    wb = [np.zeros((N + 1, M)) for _ in range(K + 1)]
    lb[K][N] = np.asarray(dL_dlamN, dtype=np.float64).reshape(-1)
    gk = np.zeros(ops.ring) if want_k else None
    for k in range(K - 1, -1, -1):
        for i in range(N, 0, -1):
            if i > k:
                g = lb[k + 1][i]
                wb[k + 1][i] += g
                vbar = g
                wb[k][i] -= g
                a, dk = ops.F_adj(lam[k][i - 1], vbar, want_k)
                lb[k][i - 1] += a
                if want_k:
                    gk += dk
                if i - 1 > k:
                    z, dk = ops.G_adj(w[k + 1][i], wb[k + 1][i], want_k)
                    lb[k + 1][i - 1] += z
                    if want_k:
                        gk += dk
                else:
                    wb[k][i] += wb[k + 1][i]
            else:
                lb[k][i] += lb[k + 1][i]
                wb[k][i] += wb[k + 1][i]
        lb[k][0] += lb[k + 1][0]          # lambda_0 is never updated
    # ---- predictor
    for i in range(N, 0, -1):
        wb[0][i] += lb[0][i]
        z, dk = ops.G_adj(w[0][i], wb[0][i], want_k)
        lb[0][i - 1] += z
        if want_k:
            gk += dk
    return lb[0][0].reshape(ops.shape), gk, lam[K][N].reshape(ops.shape)


def adjoint_async(prob: dict, events, dL_dlamN, u0=None, kappa="from_prob"):
    """Gradients (dL/du0, dL/dkappa) of L(lambda_N) through a logged asynchronous run.

    The run is the one its event log defines (Eq. (12), Algorithm 2; see
    parareal.async_replay): version 0 of slice i is the predictor value
    G lambda_{i-1}^0, and event (i, k, vF, vG) makes
        lambda_i^k = G lambda_{i-1}^{vG} + F lambda_{i-1}^{vF} - G lambda_{i-1}^{vF}
    (= F lambda_{i-1}^{vF} when vG = vF), the subtracted coarse value being the
    stored G of the fine input.  lambda_N is slice N's last version.  Reverse
    mode over that graph: slices N..1 (each version depends only on versions of
    the previous slice), events of a slice in reverse order, then the
    predictor chain; with G^T = G and F^T = F,
        lbar(i-1, vG) += G g,   lbar(i-1, vF) += F g - G g,   g = lbar(i, k).
    Returns (grad_u0 (state shape), grad_kappa (ring shape) or None, lambda_N).
    """
    from .parareal import async_replay
    ops = _Ops(prob, kappa)
    if ops.P.f_scheme != "explicit":
        raise ValueError("adjoint oracle covers the explicit fine propagator")
    want_k = ops.P.kappa is not None
    N = int(prob["N"])
    rep = async_replay(prob, events, u0=u0, kappa=kappa)
    ver = rep.versions
    by_slice = {i: [] for i in range(1, N + 1)}
    for ev in events:
        i, k, vF, vG = (int(e) for e in ev[:4])
        by_slice[i].append((k, vF, vG))
    last = {i: (max(k for k, _, _ in by_slice[i]) if by_slice[i] else 0) for i in range(1, N + 1)}
    lbar = {key: np.zeros_like(val) for key, val in ver.items()}
    lbar[(N, last[N])] += np.asarray(dL_dlamN, dtype=np.float64).reshape(-1)
    gk = np.zeros(ops.ring) if want_k else None
    for i in range(N, 0, -1):
        for k, vF, vG in sorted(by_slice[i], reverse=True):
            g = lbar[(i, k)]
            if vG > vF:
                # G's outputs at this event: the new coarse value and the subtracted one
                z, dk_new = ops.G_adj(ops.G(ver[(i - 1, vG)]), g, want_k)
                _, dk_old = ops.G_adj(ops.G(ver[(i - 1, vF)]), g, want_k)
                lbar[(i - 1, vG)] += z
                lbar[(i - 1, vF)] -= z
                if want_k:
                    gk += dk_new - dk_old
            a, dk = ops.F_adj(ver[(i - 1, vF)], g, want_k)
            lbar[(i - 1, vF)] += a
            if want_k:
                gk += dk
        # predictor: lambda_i^0 = G lambda_{i-1}^0
        z, dk = ops.G_adj(ver[(i, 0)], lbar[(i, 0)], want_k)
        lbar[(i - 1, 0)] += z
        if want_k:
            gk += dk
    return lbar[(0, 0)].reshape(ops.shape), gk, ver[(N, last[N])].reshape(ops.shape)


def loss_and_forward(prob: dict, K: int, u_obs, u0=None, kappa="from_prob"):
    """L = 1/2 ||lambda_N^K - u_obs||^2 with K fixed sync iterations (no early stop)."""
    from .parareal import sync_parareal
    res = sync_parareal(prob, u0=u0, tol=0.0, max_iter=K, kappa=kappa)
    r = res.lam[-1] - np.asarray(u_obs).reshape(-1)
    return 0.5 * float(r @ r), res.lam[-1]
