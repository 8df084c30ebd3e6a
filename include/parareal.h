/*
 * parareal.h — C ABI of the GB300 (sm_103a) Parareal library for the heat
 * equation u_t = div(kappa grad u) with zero Dirichlet boundary.
 *
 * Method: Parareal (§3.1, Eq. (11)) run as Algorithm 1 (§4.1), and
 * asynchronous Parareal (§3.1, Eq. (12)) run as Algorithm 2 (§4.1), with
 * the stopping test of §5.1, Eq. (22).  The problem statement follows §3.1
 * (Eq. (8)-(10)): a time interval [T0, T] cut into N slices, initial values
 * u0, zero Dirichlet boundary, a fine propagator F and a coarse propagator G
 * over one slice, and a tolerance on the max-norm increment.
 *
 * Conventions shared by every entry point
 *  - Grid: dim = 1, 2 or 3; n[a] interior points per axis a (x, y, z);
 *    h_a = 1/(n[a]+1) on the unit interval/square/cube.  A state holds
 *    M = n[0]*n[1]*n[2] doubles (unused n[a] = 1), x fastest, then y, then z.
 *  - Trajectory lam: (N+1) states, row i = state at T_i (row 0 = u0),
 *    contiguous, (N+1)*M doubles, slice index slowest.
 *  - kappa: diffusivity at every node including the boundary ring,
 *    prod(n[a]+2) doubles in the same x-fastest order, or NULL for kappa = 1.
 *    Face values are the mean of the two node values (flux form).
 *  - Pointers named *_dev are device pointers (cudaMalloc / torch CUDA
 *    tensors); *_host are host pointers.  The caller owns every buffer it
 *    passes; the library owns only its context and workspaces.
 *  - Alignment: device arrays must be 16-byte aligned (vector loads).
 *  - Work is issued on the stream given to parareal_create; calls that
 *    return results or statistics synchronise that stream before returning.
 *  - Every function returns PR_OK (0) or a PR_E* code and never throws;
 *    parareal_last_error gives a one-line message for the last failure.
 */
#ifndef PARAREAL_H
#define PARAREAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_ctx pr_ctx; /* opaque; owns workspaces only */

enum pr_status {
  PR_OK = 0,
  PR_EINVAL = 1,    /* invalid argument or problem (sizes, alignment, stability) */
  PR_ENOMEM = 2,    /* device allocation failed */
  PR_ECUDA = 3,     /* a CUDA call failed, or a bounded device wait of the trapezoidal
                       or TMA-fed fine kernels expired (the message names it) */
  PR_ETIMEOUT = 4,  /* an asynchronous run exceeded its wall-clock limit */
  PR_ENOTCONV = 5,  /* max_iter reached before the tolerance; results written */
  PR_ESTATE = 6,    /* call out of order (e.g. run before set_problem) */
  PR_ELOGFULL = 7   /* asynchronous event log capacity exceeded; run stopped */
};

enum pr_scheme { PR_EXPLICIT_EULER = 0, PR_IMPLICIT_EULER = 1, PR_CRANK_NICOLSON = 2 };
enum pr_solver { PR_SOLVER_THOMAS = 0, PR_SOLVER_CG = 1 };

/* Problem statement (§3.1).  Scalars are copied by parareal_set_problem;
 * u0_dev and kappa_dev are borrowed and must stay valid while the context
 * uses this problem.
 *  f_scheme/f_steps: F = f_steps steps of explicit Euler (any dim) or
 *    implicit Euler (dim 1, Thomas) of size dt = (T-T0)/(N*f_steps).
 *  f_scheme PR_CRANK_NICOLSON: the trapezoidal rule of Table 1 (§5.1),
 *    (I + dt/2 A) u' = (I - dt/2 A) u per fine step, unconditionally stable;
 *    dim 1 by the tridiagonal partition solver (exact), dim 2/3 by conjugate
 *    gradients started from the current state and stopped when
 *    ||r||_2 <= f_rtol ||rhs||_2 or after f_maxit iterations.  FP64 only.
 *  Explicit FP64 steps with kappa = 1 run in a scaled form (the state carried
 *    as u / rx^j, one FP64 instruction less per point): the same values up to
 *    rounding.
 *  f_prec: 64 = FP64 fine steps; 32 = FP32 fine steps with FP64 input and
 *    output (the coarse sweep, correction and test stay FP64); in 3D with
 *    kappa = 1 and n[0] % 4 == 0 the middle FP32 steps are fed by TMA.
 *  g_solver: PR_SOLVER_THOMAS (dim 1) or PR_SOLVER_CG; G = one implicit
 *    Euler step of size dT = (T-T0)/N (g_steps must be 1 with CG).
 *  g_rtol/g_maxit: CG stops when ||r||_2 <= g_rtol*||b||_2 or after g_maxit.
 *  tol: stop when max_i max_x |lam_i^{k+1} - lam_i^k| < tol (Eq. (22));
 *    tol = 0 runs exactly max_iter iterations.
 *  max_iter: iteration cap (<= N; finite termination at k = N, §3.2). */
typedef struct pr_problem {
  int dim;
  int n[3];
  double T0, T;
  int N;
  const double* u0_dev;
  const double* kappa_dev;
  int f_scheme;
  int f_steps;
  int f_prec;
  int g_solver;
  int g_steps;
  double g_rtol;
  int g_maxit;
  double tol;
  int max_iter;
  double f_rtol;           /* CG tolerance of the trapezoidal fine steps (<= 0: 1e-12) */
  int f_maxit;             /* CG iteration cap of one fine step (<= 0: 10000) */
} pr_problem;

/* Run statistics. */
typedef struct pr_stats {
  int iterations;          /* sync: k; async: kappa(k~) = max_i k_i (§4.1) */
  int converged;           /* 1 if the tolerance (or finite termination) stopped the run */
  double max_delta;        /* last max_i delta_i */
  long long fine_lups;     /* fine cell updates executed (sum over F applications) */
  long long cg_iterations; /* CG iterations executed by all coarse solves */
  long long coarse_solves; /* number of G applications that ran a solver */
  double t_total_ms;       /* wall time of the run on the device (CUDA events) */
  double t_fine_ms;        /* sync: time in batched F (events); async: 0 */
  double t_coarse_ms;      /* sync: time in predictor + coarse sweeps; async: 0 */
  long long events;        /* async: slice updates published */
  long long launches;      /* CUDA kernel launches issued by the call */
  long long fine_cg_iterations; /* CG iterations of the trapezoidal fine steps (2D/3D) */
  int verify_rounds;       /* async with verify: fixed-point residual checks made */
  double residual;         /* async with verify: max_i max_x |lam_i - F(lam_{i-1})| at the
                              last check (0 otherwise) */
  long long predictor_cg_iterations; /* sync: CG iterations of the predictor's N coarse
                                        solves (included in cg_iterations) */
  double t_predictor_ms;   /* sync: time of the predictor (included in t_coarse_ms) */
} pr_stats;

/* Asynchronous run options (Algorithm 2). */
typedef struct pr_async_opts {
  int paper_literal;        /* 1: a slice re-iterates even when its inputs are unchanged */
  double timeout_s;         /* wall-clock limit of each launch of the persistent kernel
                               (e.g. 60; in verify mode every resumed launch gets it anew) */
  const int32_t* delays_dev;/* NULL, or device int32 [N * delay_cols]: publish delay of
                               slice i's e-th update, in units of delay_unit_ns */
  int delay_cols;           /* columns of delays_dev (events beyond it use column e % delay_cols) */
  double delay_unit_ns;     /* duration of one delay unit */
  int ctas_per_slice;       /* CTAs cooperating on one slice update (0 = automatic: about as
                               many teams as their CG working sets fit in L2, each team
                               owning slices round-robin; at most 8 CTAs when all fit) */
  int quiescence;           /* 1: ignore tol and run until no slice can change */
  int lazy;                 /* 1: after an update whose fine input was older than its coarse
                               input, re-update only when a newer predecessor version
                               appears or the predecessor has settled (skips intermediate
                               updates that a newer version would supersede) */
  int verify;               /* 1: when the increment rule stops the run (not quiescence),
                               check the fixed-point residual max_i max_x |lam_i -
                               F(lam_{i-1})| of the latest versions by one batched F and,
                               unless it is below tol, resume the kernel with every slice's
                               last increment forgotten (so each unsettled slice must
                               publish again); at most 100 checks.  An asynchronous update's
                               increment can be small while the slice is still far from the
                               fixed point (its inputs changed little); the check closes
                               that gap.  The log spans all launches. */
} pr_async_opts;

/* One asynchronous update event (log entry). */
typedef struct pr_event {
  int32_t slice;    /* i in 1..N */
  int32_t version;  /* k_i after the update (1, 2, ...) */
  int32_t vF;       /* version of lam_{i-1} used for F and the subtracted G (tau_{i-1,2}) */
  int32_t vG;       /* version of lam_{i-1} used for the new G (tau_{i-1,1}) */
  int32_t cg_iters; /* CG iterations of the new G (0 when vG == vF) */
  int32_t team;     /* worker team that ran the update */
  double delta;     /* max_x |lam_i^{version} - lam_i^{version-1}| */
  uint64_t t_start; /* %globaltimer ns at update start */
  uint64_t t_end;   /* %globaltimer ns when the new version became visible */
} pr_event;

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  *out receives the context. */
int parareal_create(pr_ctx** out, int device, void* cuda_stream);

/* Validate and bind a problem (§3.1); allocates the workspaces it needs
 * (about 4 N M doubles for the sync path, plus N M floats x 2 for FP32 fine
 * steps and 6 M doubles per team for trapezoidal steps in 2D/3D).  Rejects an
 * unstable explicit step (dt * bound(lambda_max(A)) > 2) with PR_EINVAL. */
int parareal_set_problem(pr_ctx* ctx, const pr_problem* prob);

/* Synchronous Parareal, Algorithm 1 (§4.1) / Eq. (11): predictor G-chain,
 * batched F over the active slices, sequential coarse sweep with the fused
 * correction lam_i = (w_new + v_i) - w_old and per-slice max-norm increment,
 * stop test Eq. (22).  lam_out_dev: (N+1)*M doubles, written with the final
 * iterate (row 0 = u0).  Returns PR_ENOTCONV if max_iter < N stopped it.
 * With trapezoidal fine steps in 2D/3D the plain schedule is used whatever
 * PR_OPT_PIPELINE says (that F is itself a device-wide cooperative launch). */
int parareal_run_sync(pr_ctx* ctx, double* lam_out_dev, pr_stats* stats);

/* Same as parareal_run_sync with host buffers: copies u0_host (M doubles) to
 * the device, runs, and copies the (N+1)*M result into lam_out_host.  The
 * problem's u0_dev is ignored for this call. */
int parareal_run_sync_host(pr_ctx* ctx, const double* u0_host, double* lam_out_host,
                           pr_stats* stats);

/* Asynchronous Parareal, Eq. (12) / Algorithm 2 (§4.1), as one persistent
 * kernel: slice teams publish versions of lam_i through release/acquire
 * flags and take the freshest visible predecessor version, with no global
 * barrier.  lam_out_dev receives each slice's last published version.
 * log_host (capacity log_cap events, may be NULL) receives the event log in
 * publication order; *log_len its length.  Needs the CG coarse solver and
 * explicit fine steps (or trapezoidal steps in 2D/3D); PR_EINVAL otherwise. */
int parareal_run_async(pr_ctx* ctx, const pr_async_opts* opts, double* lam_out_dev,
                       pr_stats* stats, pr_event* log_host, size_t log_cap, size_t* log_len);

/* Serial fine solution lam*_i = F(lam*_{i-1}) (Eq. (10)); (N+1)*M doubles. */
int parareal_serial_fine(pr_ctx* ctx, double* lam_out_dev, pr_stats* stats);

/* F applied to `count` states in_dev[c*M..] -> out_dev[c*M..] (batched over
 * slices, §4.1 F step).  in and out must not overlap. */
int parareal_fine(pr_ctx* ctx, const double* in_dev, double* out_dev, int count);

/* G applied to one state: out = (I + dT A)^{-1} in (one implicit Euler
 * step, §5.1).  x0_dev: CG starting guess (NULL = in).  *cg_iters (host,
 * may be NULL) receives the CG iteration count (0 for Thomas). */
int parareal_coarse(pr_ctx* ctx, const double* in_dev, const double* x0_dev, double* out_dev,
                    int* cg_iters);

/* The fused correction and increment of Algorithm 1 on one state:
 * lam_new = (w_new + v) - w_old (in this operation order, no FMA), written
 * over lam_inout_dev, whose old value gives *delta = max_x |lam_new - lam_old|. */
int parareal_correct(pr_ctx* ctx, const double* w_new_dev, const double* v_dev,
                     const double* w_old_dev, double* lam_inout_dev, double* delta);

/* Discrete adjoint (reverse mode) of K synchronous iterations (Algorithm 1
 * with the prefix frozen, no early stop) of the trajectory map u0 -> lam_N^K,
 * G taken as the exact solve (I + dT A)^{-1} (CG to g_rtol, or the Thomas
 * step in 1D).  Fine steps: FP64 explicit (any dimension) or 1D implicit
 * (the tridiagonal solves run backward: S^-1 is symmetric); one coarse step.  Given
 * dL/dlam_N (M doubles), writes grad_u0_dev (M doubles) and, if non-NULL,
 * grad_kappa_dev (prod(n+2) doubles, one per node including the ring).
 * Fine states are recomputed from slice-boundary checkpoints. */
int parareal_adjoint(pr_ctx* ctx, const double* dL_dlamN_dev, int K, double* grad_u0_dev,
                     double* grad_kappa_dev);

/* Discrete adjoint of a logged asynchronous run (Eq. (12), Algorithm 2): the
 * event log (host array of n_events pr_event, as written by
 * parareal_run_async; only slice, version, vF and vG are read) fixes the
 * computation graph
 *   lam_i^0 = G lam_{i-1}^0,
 *   lam_i^k = G lam_{i-1}^{vG} + F lam_{i-1}^{vF} - G lam_{i-1}^{vF}
 * (= F lam_{i-1}^{vF} when vG = vF), and lam_N = slice N's last version.
 * The run is replayed on the device keeping every version, then reversed
 * slice by slice (G and F are symmetric; G taken as the exact solve, CG to
 * g_rtol).  Given dL/dlam_N (M doubles) writes grad_u0_dev (M doubles),
 * grad_kappa_dev if non-NULL (prod(n+2) doubles) and, if lamN_dev is
 * non-NULL, the replayed lam_N (M doubles).  The log may be in any order;
 * PR_EINVAL when it is not a valid run (versions of a slice not 1, 2, ...;
 * a fine input other than the previous coarse input; an input version never
 * produced).  Workspace: (2 V + E) M doubles for V versions and E events,
 * plus the batched fine states.  FP64 explicit F and CG G only. */
int parareal_adjoint_async(pr_ctx* ctx, const pr_event* log_host, size_t n_events,
                           const double* dL_dlamN_dev, double* grad_u0_dev,
                           double* grad_kappa_dev, double* lamN_dev);

/* Scheduling options (they never change results, only when work runs):
 *  PR_OPT_PIPELINE (0/1, default 0): parareal_run_sync overlaps the fine
 *    propagation of iteration k+1 with the coarse sweep of iteration k (slice
 *    i's fine input lam_{i-1}^{k+1} is final as soon as the sweep has passed
 *    slice i-1, as in the processor schedule of Algorithm 1, §4.1).  The fine
 *    work runs on a low-priority stream in slice chunks; results are bitwise
 *    identical to the plain schedule.  Needs N*M more doubles.
 *  PR_OPT_PIPELINE_CHUNKS (1..1024, default 8): slice chunks per fine batch.
 *  PR_OPT_CG_BLOCKS_PER_SM (0 = automatic): cap on the co-resident blocks per
 *    SM of the coarse CG kernel (leaves room for concurrent fine work).
 * and one that changes the coarse solver (not its stopping rule):
 *  PR_OPT_G_CHEBYSHEV (0 = plain CG, default; m in [2, 64]): the coarse CG
 *    of the synchronous driver, the predictor and the adjoint is
 *    preconditioned by m steps of Chebyshev iteration on the spectrum bounds
 *    of I + dT A (exact for kappa = 1, Rayleigh/Gershgorin bounds otherwise),
 *    computed in FP32; the CG recurrences and the test ||r||_2 <= g_rtol
 *    ||b||_2 stay FP64, so the result meets the same residual bound (and,
 *    I + dT A >= I, lies within 2 g_rtol ||b||_2 of the plain CG result).
 *    Needs M doubles and 4 M floats more.  The asynchronous kernel keeps plain
 *    CG. */
/* and one that changes the coarse CG's recurrence (not its iterates in exact
 * arithmetic, nor its stopping rule):
 *  PR_OPT_G_CG (0 = automatic, default; 1 = textbook; 2 = single-reduction):
 *    the unpreconditioned coarse CG of the synchronous driver, the predictor,
 *    parareal_coarse and the adjoint runs either textbook (Hestenes-Stiefel)
 *    CG, three device-wide barriers and two reductions per iteration, or the
 *    single-reduction recurrence of Chronopoulos and Gear, whose two inner
 *    products r.r and (B r).r are reduced together: two barriers and one
 *    reduction per iteration for one more vector update per point.  Automatic
 *    is textbook (measured faster from 512^2 points up).  The iterates agree to
 *    rounding; the iteration counts to about one. */
/* and one that changes how the fine steps are grouped into launches (the
 * arithmetic of every step is the same):
 *  PR_OPT_F_STEPS_PER_PASS (1 or 2, default 2): the TMA-fed FP32 middle steps
 *    of the mixed form (3D, kappa = 1, n[0] % 4 == 0) run two steps per pass
 *    over the state (temporal blocking: one read and one write of the state per
 *    two steps; the first step's values on the halo the second needs are
 *    recomputed per tile) or one.  Results are bitwise identical. */
enum pr_option {
  PR_OPT_PIPELINE = 1,
  PR_OPT_PIPELINE_CHUNKS = 2,
  PR_OPT_CG_BLOCKS_PER_SM = 3,
  PR_OPT_G_CHEBYSHEV = 4,
  PR_OPT_G_CG = 5,
  PR_OPT_F_STEPS_PER_PASS = 6
};
int parareal_set_option(pr_ctx* ctx, int option, double value);

/* Per-slice statistics of the last run (host arrays of N entries, may be NULL):
 * k_i (async update counts; sync: k for every slice) and delta_i. */
int parareal_slice_stats(pr_ctx* ctx, int* k_host, double* delta_host);

/* Allocation-free coarse solve.  The paper has no counterpart: this is a
 * service for callers that must not allocate device memory while they run
 * (an allocator hook or host callback where cudaMalloc would re-enter or is
 * not allowed, a fixed memory budget checked at start-up, or a loop that
 * cannot pay cudaMalloc/cudaFree's implicit device synchronisation).
 * It solves one backward-Euler step (I + dT A) x = b for kappa = 1 on a
 * dim-dimensional grid with n[0..dim-1] interior points, by the same CG as
 * the coarse propagator (start x0_dev, NULL = b; stop at
 * ||r||_2 <= rtol ||b||_2 or maxit iterations, maxit <= 0 = 20000), on the
 * calling thread's current device and the given stream, without a context.
 *  - Workspace: a static device array inside the library (about 4 MiB, held
 *    by every GPU that loads the library until the process exits); no
 *    cudaMalloc/cudaFree or other allocating call is made.
 *  - Limit: M = prod(n) <= 131072 points; larger grids return PR_EINVAL.
 *  - The first call on a device resolves the array's device address
 *    (cudaGetSymbolAddress) and the launch limit; make that first call
 *    outside any stream capture.
 *  - All calls on a device share the array and it keeps the last call's
 *    contents (nothing of it is read before being rewritten): calls whose
 *    work overlaps on the GPU race.  Serialise them.
 *  - b_dev, x0_dev, x_dev: device, M doubles, 16-byte aligned, caller-owned.
 *    *iters_host (may be NULL) receives the CG iteration count; passing it
 *    synchronises the stream. */
int parareal_coarse_noalloc(int dim, const int* n, double dT, const double* b_dev,
                            const double* x0_dev, double* x_dev, double rtol, int maxit,
                            int* iters_host, void* cuda_stream);

/* FP64-pipe throughput probe (a measurement aid; the paper has no
 * counterpart): runs 4 blocks of 256 threads per SM on the current device,
 * each thread executing `iters` rounds of eight independent FP64 operations
 * (kind 0: DFMA x = x a + b; kind 1: DADD x = x + b), once untimed and once
 * timed with CUDA events on the given stream (synchronised before return).
 * *ops_per_s_host receives FP64 instructions per second of the timed launch,
 * *ops_host (may be NULL) the instruction count.  scratch_dev: one device
 * double, written only if the chains overflow (never for iters <= 2^32).
 * PR_EINVAL for a kind other than 0/1 or iters outside [1, 2^32]. */
int parareal_probe_fp64(int kind, long long iters, double* scratch_dev, double* ops_per_s_host,
                        long long* ops_host, void* cuda_stream);

/* Conversion check (a test aid; the paper has no counterpart).  The coarse
 * solver's vectorised passes convert between FP32 and FP64 with integer
 * operations instead of the conversion instructions, which issue on the FP64
 * pipe; this entry applies those conversions elementwise on the given stream:
 * d_out_dev[i] = widen(f_in_dev[i]) (exact) and f_out_dev[i] =
 * narrow(d_in_dev[i]) (round to nearest, ties to even), n elements, all four
 * device buffers caller-owned.  Asynchronous.  PR_EINVAL for n < 0 or a NULL
 * buffer with n > 0; PR_ECUDA when the launch fails. */
int parareal_probe_convert(const float* f_in_dev, double* d_out_dev, const double* d_in_dev,
                           float* f_out_dev, long long n, void* cuda_stream);

void parareal_destroy(pr_ctx* ctx);
const char* parareal_last_error(const pr_ctx* ctx);
const char* parareal_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PARAREAL_H */
