"""Helpers for the GPU parity tests: build pr_problem from a preset dict, move
arrays to the device, and compare with the oracle."""
from __future__ import annotations

import numpy as np

import paper_2110_10762_gb300 as pr


def torch():
    import torch as t
    return t


def dev(a):
    t = torch()
    return t.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).cuda()


def host(x):
    return x.detach().cpu().numpy()


def problem_struct(p: dict, u0_t, kappa_t=None, **over):
    f_scheme = {"explicit": pr.PR_EXPLICIT_EULER, "implicit": pr.PR_IMPLICIT_EULER,
                "cn": pr.PR_CRANK_NICOLSON}[p.get("f_scheme", "explicit")]
    g_solver = pr.PR_SOLVER_THOMAS if p.get("g_solver") == "thomas" else pr.PR_SOLVER_CG
    kw = dict(dim=p["dim"], n=p["n"], T0=0.0, T=p["N"] * p["f_steps"] * p["dt"], N=p["N"],
              u0=u0_t, kappa=kappa_t, f_scheme=f_scheme, f_steps=p["f_steps"],
              f_prec=p.get("f_prec", 64), g_solver=g_solver, g_rtol=p.get("g_rtol", 1e-10),
              g_maxit=p.get("g_maxit", 20000), tol=p.get("tol", 0.0),
              max_iter=p.get("max_iter", 0), f_rtol=p.get("f_rtol") or 0.0,
              f_maxit=p.get("f_maxit") or 0)
    kw.update(over)
    return pr.make_problem(**kw)


class Ctx:
    """Context + problem bound to device tensors kept alive here."""

    def __init__(self, p: dict, **over):
        t = torch()
        self.p = p
        self.u0 = dev(p["u0"])
        self.kappa = dev(p["kappa"]) if p.get("kappa") is not None else None
        self.ctx = pr.parareal_create(0, t.cuda.current_stream())
        self.prob = problem_struct(p, self.u0, self.kappa, **over)
        pr.parareal_set_problem(self.ctx, self.prob)
        # the coarse solver the oracle runs for this problem (Propagators reads the same keys)
        if p.get("g_cheb"):
            pr.parareal_set_option(self.ctx, pr.PR_OPT_G_CHEBYSHEV, p["g_cheb"])
        if p.get("g_cg"):
            pr.parareal_set_option(self.ctx, pr.PR_OPT_G_CG,
                                   {"textbook": 1, "single": 2}[p["g_cg"]])
        self.M = int(np.prod(p["n"]))
        self.N = p["N"]

    def lam(self):
        return torch().zeros((self.N + 1) * self.M, dtype=torch().float64, device="cuda")

    def close(self):
        pr.parareal_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
