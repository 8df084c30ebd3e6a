"""Python binding of the C ABI: same names, argument marshalling only.

Device buffers are passed as CUDA torch tensors (float64, contiguous) or raw
integer addresses; every computation runs in libparareal's CUDA kernels.
A non-OK status raises PararealError, except PR_ENOTCONV, which is returned
(the result is still written).
"""
from __future__ import annotations

import ctypes as C

from . import _abi
from ._abi import (PR_ENOTCONV, PR_OK, pr_async_opts, pr_event, pr_problem, pr_stats)


class PararealError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_abi.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _lib():
    return _abi.load()


def _ptr(x, dtype_check=True):
    """Device address of a CUDA tensor (checked) or an int address; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError(f"expected a torch tensor or an address, got {type(x)}")
    if not x.is_cuda:
        raise ValueError("device buffers must be CUDA tensors")
    if not x.is_contiguous():
        raise ValueError("device buffers must be contiguous")
    if dtype_check and x.dtype != torch.float64:
        raise ValueError(f"expected float64, got {x.dtype}")
    return x.data_ptr()


def _hptr(x):
    """Host address of a CPU tensor / numpy array (float64, contiguous)."""
    import numpy as np
    import torch
    if isinstance(x, torch.Tensor):
        if x.is_cuda or not x.is_contiguous() or x.dtype != torch.float64:
            raise ValueError("host buffers must be contiguous CPU float64 tensors")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"] or x.dtype != np.float64:
            raise ValueError("host arrays must be C-contiguous float64")
        return x.ctypes.data
    raise TypeError(type(x))


def _check(ctx, code):
    if code == PR_OK or code == PR_ENOTCONV:
        return code
    msg = _lib().parareal_last_error(ctx).decode() if ctx else ""
    raise PararealError(code, msg)


def parareal_version() -> str:
    return _lib().parareal_version().decode()


def parareal_last_error(ctx) -> str:
    return _lib().parareal_last_error(ctx).decode()


def parareal_create(device: int = 0, stream=None):
    """Create a context; stream is a torch.cuda.Stream, a raw cudaStream_t or None."""
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    out = C.c_void_p()
    code = _lib().parareal_create(C.byref(out), int(device), stream)
    if code != PR_OK:
        raise PararealError(code, "parareal_create failed")
    return out


def make_problem(dim, n, T0, T, N, u0, kappa=None, f_scheme=_abi.PR_EXPLICIT_EULER,
                 f_steps=1, f_prec=64, g_solver=_abi.PR_SOLVER_CG, g_steps=1, g_rtol=1e-10,
                 g_maxit=20000, tol=0.0, max_iter=0, f_rtol=0.0, f_maxit=0) -> pr_problem:
    """Fill a pr_problem; u0/kappa are CUDA float64 tensors (kept alive by the caller)."""
    p = pr_problem()
    p.dim = int(dim)
    nn = list(n) + [1] * (3 - len(n))
    for a in range(3):
        p.n[a] = int(nn[a])
    p.T0, p.T, p.N = float(T0), float(T), int(N)
    p.u0_dev = _ptr(u0)
    p.kappa_dev = _ptr(kappa)
    p.f_scheme, p.f_steps, p.f_prec = int(f_scheme), int(f_steps), int(f_prec)
    p.g_solver, p.g_steps = int(g_solver), int(g_steps)
    p.g_rtol, p.g_maxit = float(g_rtol), int(g_maxit)
    p.tol, p.max_iter = float(tol), int(max_iter)
    p.f_rtol, p.f_maxit = float(f_rtol), int(f_maxit)
    return p


def parareal_set_problem(ctx, prob: pr_problem):
    return _check(ctx, _lib().parareal_set_problem(ctx, C.byref(prob)))


def parareal_run_sync(ctx, lam_out):
    st = pr_stats()
    code = _check(ctx, _lib().parareal_run_sync(ctx, _ptr(lam_out), C.byref(st)))
    return code, st


def parareal_run_sync_host(ctx, u0_host, lam_out_host):
    st = pr_stats()
    code = _check(ctx, _lib().parareal_run_sync_host(ctx, _hptr(u0_host), _hptr(lam_out_host),
                                                      C.byref(st)))
    return code, st


def parareal_serial_fine(ctx, lam_out):
    st = pr_stats()
    _check(ctx, _lib().parareal_serial_fine(ctx, _ptr(lam_out), C.byref(st)))
    return st


def parareal_fine(ctx, x_in, x_out, count: int):
    return _check(ctx, _lib().parareal_fine(ctx, _ptr(x_in), _ptr(x_out), int(count)))


def parareal_coarse(ctx, x_in, x0, x_out) -> int:
    it = C.c_int(0)
    _check(ctx, _lib().parareal_coarse(ctx, _ptr(x_in), _ptr(x0), _ptr(x_out), C.byref(it)))
    return it.value


def parareal_correct(ctx, w_new, v, w_old, lam_inout) -> float:
    d = C.c_double(0.0)
    _check(ctx, _lib().parareal_correct(ctx, _ptr(w_new), _ptr(v), _ptr(w_old), _ptr(lam_inout),
                                        C.byref(d)))
    return d.value


def make_async_opts(paper_literal=False, timeout_s=60.0, delays=None, delay_unit_ns=0.0,
                    ctas_per_slice=0, quiescence=False, lazy=False,
                    verify=False) -> pr_async_opts:
    o = pr_async_opts()
    o.paper_literal = int(bool(paper_literal))
    o.timeout_s = float(timeout_s)
    if delays is not None:
        import torch
        if delays.dtype != torch.int32 or not delays.is_cuda or delays.dim() != 2:
            raise ValueError("delays must be a 2D CUDA int32 tensor [N, cols]")
        o.delays_dev = delays.data_ptr()
        o.delay_cols = int(delays.shape[1])
    o.delay_unit_ns = float(delay_unit_ns)
    o.ctas_per_slice = int(ctas_per_slice)
    o.quiescence = int(bool(quiescence))
    o.lazy = int(bool(lazy))
    o.verify = int(bool(verify))
    return o


def parareal_run_async(ctx, opts: pr_async_opts, lam_out, log_cap: int = 0):
    """Returns (status, stats, events) with events a list of pr_event; status is
    PR_OK, PR_ETIMEOUT or PR_ELOGFULL (other failures raise PararealError)."""
    st = pr_stats()
    log = (pr_event * max(int(log_cap), 1))()
    n = C.c_size_t(0)
    code = _lib().parareal_run_async(ctx, C.byref(opts), _ptr(lam_out), C.byref(st),
                                     log if log_cap else None, int(log_cap), C.byref(n))
    if code not in (PR_OK, _abi.PR_ETIMEOUT, _abi.PR_ELOGFULL):
        _check(ctx, code)
    # a run stopped by its time limit or by a full log still returns its state and log
    return code, st, [log[i] for i in range(n.value)] if log_cap else []


def parareal_adjoint(ctx, dL_dlamN, K: int, grad_u0, grad_kappa=None):
    return _check(ctx, _lib().parareal_adjoint(ctx, _ptr(dL_dlamN), int(K), _ptr(grad_u0),
                                               _ptr(grad_kappa)))


def parareal_adjoint_async(ctx, log, dL_dlamN, grad_u0, grad_kappa=None, lamN=None):
    """Adjoint of a logged asynchronous run; `log` is the event list returned by
    parareal_run_async (pr_event structs) or any sequence of them."""
    n = len(log)
    arr = (pr_event * max(n, 1))(*log)
    return _check(ctx, _lib().parareal_adjoint_async(ctx, arr, n, _ptr(dL_dlamN), _ptr(grad_u0),
                                                     _ptr(grad_kappa), _ptr(lamN)))


def parareal_set_option(ctx, option: int, value: float):
    return _check(ctx, _lib().parareal_set_option(ctx, int(option), float(value)))


def parareal_slice_stats(ctx, N: int):
    k = (C.c_int * N)()
    d = (C.c_double * N)()
    _check(ctx, _lib().parareal_slice_stats(ctx, k, d))
    return list(k), list(d)


def parareal_coarse_noalloc(dim: int, n, dT: float, b, x0, x_out, rtol: float = 1e-10,
                            maxit: int = 0, stream=None) -> int:
    """Allocation-free coarse solve (kappa = 1) for callers that must not allocate
    device memory; see include/parareal.h.  Returns the CG iteration count.

    The wrapper checks that dim matches len(n) and that b, x0 (if given) and
    x_out hold at least prod(n) float64 values before the library sees the
    pointers (the C entry point cannot know the buffers' lengths).  With
    stream=None the work goes on torch's current stream, like the context path."""
    import torch
    n = [int(v) for v in n]
    if not 1 <= int(dim) == len(n) <= 3:
        raise ValueError("dim must equal len(n) and lie in 1..3 (dim=%r, n=%r)" % (dim, n))
    M = 1
    for v in n:
        M *= v
    for name, t in (("b", b), ("x0", x0), ("x_out", x_out)):
        if t is None and name == "x0":
            continue
        if t is None or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA float64 tensor")
        if t.numel() < M:
            raise ValueError(f"{name} holds {t.numel()} values, fewer than prod(n) = {M}")
    if stream is None:
        stream = torch.cuda.current_stream()
    if not isinstance(stream, int):
        stream = stream.cuda_stream
    nn = (C.c_int * 3)(*(n + [1] * (3 - len(n))))
    it = C.c_int(0)
    code = _lib().parareal_coarse_noalloc(int(dim), nn, float(dT), _ptr(b), _ptr(x0), _ptr(x_out),
                                          float(rtol), int(maxit), C.byref(it), stream)
    if code != PR_OK:
        raise PararealError(code, "parareal_coarse_noalloc failed")
    return it.value


def parareal_probe_fp64(kind: int, iters: int = 1 << 16, stream=None):
    """FP64-pipe throughput of the current device (kind 0: DFMA, 1: DADD), in
    FP64 instructions per second; see include/parareal.h.  Returns (rate, count)."""
    import torch
    scratch = torch.zeros(1, dtype=torch.float64, device="cuda")
    if stream is None:
        stream = torch.cuda.current_stream()
    if not isinstance(stream, int):
        stream = stream.cuda_stream
    rate, ops = C.c_double(0.0), C.c_longlong(0)
    code = _lib().parareal_probe_fp64(int(kind), int(iters), _ptr(scratch), C.byref(rate),
                                      C.byref(ops), stream)
    if code != PR_OK:
        raise PararealError(code, "parareal_probe_fp64 failed")
    return rate.value, ops.value


def parareal_probe_convert(f_in, d_in, stream=None):
    """The library's integer-pipe conversions applied elementwise (see
    include/parareal.h): returns (widen(f_in) as float64, narrow(d_in) as
    float32) for two CUDA tensors of the same length."""
    import torch
    if f_in.dtype != torch.float32 or d_in.dtype != torch.float64 or f_in.numel() != d_in.numel():
        raise ValueError("f_in must be float32 and d_in float64, of equal length")
    f_in, d_in = f_in.contiguous(), d_in.contiguous()
    d_out = torch.empty(f_in.numel(), dtype=torch.float64, device=f_in.device)
    f_out = torch.empty(d_in.numel(), dtype=torch.float32, device=d_in.device)
    if stream is None:
        stream = torch.cuda.current_stream()
    if not isinstance(stream, int):
        stream = stream.cuda_stream
    code = _lib().parareal_probe_convert(_ptr(f_in, False), _ptr(d_out), _ptr(d_in),
                                         _ptr(f_out, False), int(f_in.numel()), stream)
    if code != PR_OK:
        raise PararealError(code, "parareal_probe_convert failed")
    return d_out, f_out


def parareal_destroy(ctx):
    if ctx:
        _lib().parareal_destroy(ctx)
