// Internal declarations shared by the CUDA translation units of libparareal.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/parareal.h"

namespace pr {

// Size limits checked by parareal_set_problem: points per state (the kernels
// index rows and planes with 32-bit integers), slices, and points of the
// stacked (N+1)-state trajectory.
constexpr long long PR_MAX_POINTS = 2147483647LL;
constexpr int PR_MAX_SLICES = 65536;
constexpr long long PR_MAX_TRAJ_POINTS = 1LL << 40;

// Grid geometry of one state (interior points only), x fastest.
struct Geom {
  int dim;
  int nx, ny, nz;
  long long M;      // nx*ny*nz
  double hx, hy, hz;
};

// Coefficients of one constant-coefficient explicit step
//   u' = c0 u + rx (W+E) + ry (S+N) + rz (B+F),  r_a = dt/h_a^2, c0 = 1 - 2 sum r_a
// or, for variable kappa, per-face arrays (see StencilVar).
struct StencilConst {
  double c0, rx, ry, rz;
};

// Variable-kappa step u' = c0[p] u + sum_faces c_f u_q, with face arrays
//   cx: (nz*ny) lines of (nx+1) faces, face xf sits between nodes xf-1 and xf
//   cy: nz planes of (ny+1)*nx, face yf between rows yf-1 and yf
//   cz: (nz+1)*ny*nx
// For F: c_f = dt kappa_f / h^2 and c0 = 1 - sum of the node's faces.
// For G (operator I + dT A): c_f = dT kappa_f / h^2 and c0 = 1 + sum (the
// off-diagonal entries are -c_f).
template <typename T>
struct StencilVar {
  const T* c0;
  const T* cx;
  const T* cy;
  const T* cz;
};

// Partition-method tables for the batched 1D tridiagonal solves (one per
// matrix: fine step and coarse step).  Built on the device by tridiag_setup.
struct TriTables {
  int n = 0;            // unknowns
  int P = 0;            // chunks (lanes used), each with >= 2 rows
  int levels = 0;       // PCR levels of the reduced system (2P rows)
  int cn = 0;           // 1: trapezoidal steps (right-hand side (I - r A) u formed per step)
  double* buf = nullptr;  // device tables (layout in tridiag.cu)
};

}  // namespace pr

struct pr_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int cg_blocks = 0;         // co-resident blocks for the cooperative CG kernel
  bool has_problem = false;
  pr_problem prob{};
  pr::Geom g{};
  double dt = 0, dT = 0;
  bool var_kappa = false;
  pr::StencilConst fst{}, gst{};   // constant-coefficient F step and G operator
  // trapezoidal F: fst is then the right-hand side operator I - dt/2 A and
  // fsys the system operator I + dt/2 A (coarse-operator form)
  pr::StencilConst fsys{};
  // variable-kappa coefficient arrays (device)
  double* fcoef = nullptr;   // F: c0, cx, cy, cz (FP64)
  float* fcoef32 = nullptr;  // F: FP32 copy for the mixed form
  double* gcoef = nullptr;   // G: c0, cx, cy, cz
  float* gcoef32 = nullptr;  // G in FP32 (Chebyshev preconditioner, variable kappa)
  double* fsys0 = nullptr;   // trapezoidal F, variable kappa: diagonal of I + dt/2 A
  pr::StencilVar<double> fvar{}, gvar{}, fsysvar{};
  pr::StencilVar<float> fvar32{}, gvar32{};
  // 1D implicit tables
  pr::TriTables tri_f{}, tri_g{};
  // workspaces
  double* v = nullptr;       // N*M fine outputs v_i (row i-1)
  double* w = nullptr;       // N*M coarse values w_i (row i-1)
  double* tmp = nullptr;     // N*M ping-pong for explicit F
  float* f32a = nullptr;     // N*M FP32 ping-pong (mixed form)
  float* f32b = nullptr;
  // TMA-fed FP32 3D steps (tma_stencil.cu): tensor maps of f32a / f32b
  bool tma_ok = false;
  alignas(64) unsigned char tma_map[2][128] = {};
  alignas(64) unsigned char tma_map2[2][128] = {};  // same buffers, box for two steps per pass
  int opt_f_blocking = 2;    // FP32 TMA fine steps per pass (1 or 2; PR_OPT_F_STEPS_PER_PASS)
  int* tma_err = nullptr;
  double* cg_x = nullptr;    // CG vectors (M each)
  double* cg_r = nullptr;
  double* cg_p = nullptr;
  double* cg_q = nullptr;
  double* cg_w = nullptr;    // single-reduction CG: B r (M)
  double* cg_part = nullptr; // per-block partial sums (2 parities x 3 values x cg_blocks)
  int* cg_iters_dev = nullptr;   // per slot CG iteration counts (N+1)
  unsigned long long* delta_dev = nullptr;  // per slice increments (N), bits of non-negative doubles
  double* u0_stage = nullptr;    // host-API staging (M)
  double* lam_stage = nullptr;   // host-API staging ((N+1)*M)
  size_t lam_stage_bytes = 0;
  // last-run per-slice statistics (host)
  std::vector<int> last_k;
  std::vector<double> last_delta;
  cudaEvent_t ev[6] = {};
  std::string err;
  // options (parareal_set_option)
  int opt_pipeline = 0;      // overlap F of iteration k+1 with the coarse sweep of k
  int opt_chunks = 8;        // slice chunks per pipelined fine batch
  int opt_cg_bps = 0;        // CG blocks per SM (0 = automatic)
  int opt_g_cheb = 0;        // Chebyshev steps of the coarse CG preconditioner (0 = plain CG)
  int opt_g_cg = 0;          // coarse CG recurrence: 0 automatic, 1 textbook, 2 single-reduction
  double g_lo = 0, g_hi = 0; // spectrum bounds of I + dT A
  double* cheb_z = nullptr;  // preconditioned residual (M)
  float* cheb_f32 = nullptr; // FP32 Chebyshev vectors (4 M)
  void* cheb_tmaps = nullptr; // 3D: tensor maps of the three ring vectors and f (4 x 128 B, device)
  int* cheb_err = nullptr;   // 3D TMA-fed steps: 1 after a bounded wait expired
  // pipelined driver resources (created lazily)
  cudaStream_t s_sweep = nullptr, s_fine = nullptr;
  double* v2 = nullptr;      // second fine-output buffer (N*M)
  std::vector<cudaEvent_t> pev;
  // trapezoidal F in 2D/3D (cn.cu): team workspaces and control words
  double* cn_work = nullptr;
  double* cn_part = nullptr;
  unsigned long long* cn_bar = nullptr;
  int* cn_err = nullptr;
  unsigned long long* cn_iters = nullptr;
  int cn_teams = 0, cn_cap = 0;
  // batched coarse solves (gbatch.cu): team workspaces and control words
  double* gb_work = nullptr;
  double* gb_part = nullptr;
  unsigned long long* gb_bar = nullptr;
  int* gb_err = nullptr;
  int gb_teams = 0, gb_cap = 0;
  // async / adjoint workspaces are allocated lazily by their drivers
  void* async_ws = nullptr;
  size_t async_ws_bytes = 0;
  void* adj_ws = nullptr;
  size_t adj_ws_bytes = 0;
};

namespace pr {

int fail(pr_ctx* c, int code, const std::string& msg);
int cuda_fail(pr_ctx* c, cudaError_t e, const char* where);

#define PR_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return pr::cuda_fail(ctx, e_, #call); \
  } while (0)

// ---- explicit fine propagator (stencil.cu)
// Apply `steps` explicit Euler steps to `count` states.  in/out are FP64;
// prec 64 computes in FP64 with the tmp ping-pong buffer, prec 32 computes
// in FP32 through the two FP32 buffers.  Returns a cudaError_t.
cudaError_t explicit_fine(pr_ctx* c, const double* in, double* out, int count, int steps,
                          int prec);
cudaError_t build_var_coefficients(pr_ctx* c);
// Steps between two returns to u in the scaled FP64 explicit form (0: use the
// plain form); the batched kernel and the asynchronous kernel share it.
int scaled_period(double rx);
// One FP64 explicit step u' = S u on `count` states (S is symmetric, so this is
// also the transposed step used by the adjoint).
cudaError_t explicit_step64(pr_ctx* c, const double* in, double* out, int count);

// ---- batched coarse solves over independent systems (gbatch.cu)
// (I + dT A) out[j] = b[j] from x0[j], j < count (device arrays of pointers;
// out[j] aliases neither b[j] nor x0[j]).  Asynchronous on the context stream.
cudaError_t gbatch_solve(pr_ctx* c, const double* const* b_dev, const double* const* x0_dev,
                         double* const* out_dev, int count);
int gbatch_take_error(pr_ctx* c);
void gbatch_free(pr_ctx* c);

// ---- trapezoidal-rule fine propagator in 2D/3D (cn.cu)
cudaError_t cn_alloc(pr_ctx* c);
void cn_free(pr_ctx* c);
// F (f_steps trapezoidal steps) on `count` consecutive states; synchronises the
// stream; cudaErrorTimeout when a team barrier wait expired.
cudaError_t cn_fine(pr_ctx* c, const double* in, double* out, int count);
// CG iterations of the fine steps since the last call (resets the counter).
unsigned long long cn_take_iterations(pr_ctx* c);
// F on `count` consecutive states with the problem's fine scheme (api.cu).
cudaError_t fine_apply(pr_ctx* c, const double* in, double* out, int count);

// ---- TMA-fed FP32 3D step (tma_stencil.cu)
bool tma_prepare(pr_ctx* c);
bool encode_f32_3d_map(void* out, float* base, int nx, int ny, int nz, int box_x, int box_y);
cudaError_t tma_step(pr_ctx* c, const float* src, float* dst, int count);
cudaError_t tma_step2(pr_ctx* c, const float* src, float* dst, int count);
int fine_launch_count(const pr_ctx* c);
int tma_take_error(pr_ctx* c);

// ---- tridiagonal partition solver (tridiag.cu)
// cn: trapezoidal-rule tables (r is then dt/(2 h^2); each solve is preceded by
// forming (I - r A) u).
cudaError_t tri_build(pr_ctx* c, TriTables* t, int n, double r, const double* kappa,
                      bool cn = false);
void tri_free(TriTables* t);
// Solve `steps` times (I + r A) x = b in place for `count` right-hand sides.
cudaError_t tri_solve_steps(pr_ctx* c, const TriTables* t, const double* in, double* out,
                            int count, int steps);

// ---- CG coarse solver (cg.cu)
// Epilogue modes of the cooperative CG kernel.
enum CgMode { CG_PLAIN = 0, CG_PREDICTOR = 1, CG_CORRECT = 2 };
// Launches of one coarse solve in the given mode (the correction runs as a kernel
// of its own after the cooperative solve).
int cg_solve_launches(int mode);
struct CgArgs {
  const double* b;     // right-hand side
  const double* x0;    // start (may equal out for in-place warm start)
  double* out;         // PLAIN: solution; PREDICTOR: w_i; CORRECT: w_i (in: w_old, out: w_new)
  double* lam;         // PREDICTOR: lam_i = x; CORRECT: lam_i in/out
  const double* v;     // CORRECT: fine value v_i
  unsigned long long* delta;  // CORRECT: max |lam_new - lam_old| (double bits), zeroed by the kernel
  int* iters;          // CG iterations (one int)
  int mode;
};
cudaError_t cg_solve(pr_ctx* c, const CgArgs& a);
cudaError_t coarse_bounds(pr_ctx* c);
cudaError_t cheb_alloc(pr_ctx* c);
void cheb_free(pr_ctx* c);
int cg_max_blocks(int num_sms);
cudaError_t correct(pr_ctx* c, const double* w_new, const double* v, const double* w_old,
                    double* lam, unsigned long long* delta);
// Generic dense helpers
cudaError_t vec_copy(pr_ctx* c, double* dst, const double* src, long long n);

// ---- pipelined synchronous driver (pipeline.cu)
int run_sync_pipelined(pr_ctx* c, double* lam, pr_stats* st);
void pipeline_free(pr_ctx* c);

// ---- asynchronous persistent kernel (async.cu)
int run_async(pr_ctx* c, const pr_async_opts* o, double* lam_out, pr_stats* st, pr_event* log,
              size_t log_cap, size_t* log_len);

// ---- adjoint (adjoint.cu)
int run_adjoint(pr_ctx* c, const double* gN, int K, double* grad_u0, double* grad_kappa);
int run_adjoint_async(pr_ctx* c, const pr_event* log, size_t n_events, const double* gN,
                      double* grad_u0, double* grad_kappa, double* lamN);

}  // namespace pr
