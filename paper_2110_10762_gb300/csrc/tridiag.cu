// Batched 1D implicit-Euler solves (I + r A) x = b (§5.1: backward Euler with
// a direct solve per step), as a warp-parallel partition method:
//
//  * the n unknowns are cut into P <= 32 chunks of >= 2 rows, one per lane;
//  * each lane eliminates its chunk interior with the Thomas algorithm, which
//    writes every interior unknown as  x_m = y_m - alpha_m x_s - gamma_m x_e
//    (x_s, x_e: the chunk's first and last unknowns, alpha/gamma: "spikes");
//  * substituting into the chunks' first and last rows gives a tridiagonal
//    system of 2P rows in the chunk end values, solved by parallel cyclic
//    reduction across the lanes with warp shuffles;
//  * each lane then rebuilds its interior from x_s and x_e.
//
// Trapezoidal rule (tables built with cn = 1 and r = dt/(2 h^2)): before each
// solve the lanes form the right-hand side (I - dt/2 A) u in place,
//   rhs_m = e_m u_m - a_m u_{m-1} - c_m u_{m+1},   e_m = 1 - r (k_{m-1/2} + k_{m+1/2}),
// with a, c the off-diagonals of I + dt/2 A.
//
// The matrix is the same for every step and every slice, so all
// matrix-only quantities (Thomas factors, spikes, PCR multipliers) are built
// once by tri_setup; a step then costs about 5 FP64 operations per unknown.
// One warp owns one state (one slice) and keeps it in shared memory across
// all the steps of F, so HBM sees one read and one write per state.
#include "common.cuh"

namespace pr {

namespace {

constexpr int MAXR = 64;  // reduced rows (2 per lane)

struct TriDev {
  int n, P, base, rem, levels, maxL, cn;
  const double *a, *c, *cp, *finv, *alpha, *gamma, *k1, *k2, *binv, *e;
};

__host__ __device__ inline void chunk_of(int j, int base, int rem, int& s, int& L) {
  s = j * base + (j < rem ? j : rem);
  L = base + (j < rem ? 1 : 0);
}

// Matrix-only precomputation; one thread, sequential (n is small).
// kap: ring-node diffusivity (n+2) or NULL; r = step / h^2.
__global__ void tri_setup(int n, int P, int base, int rem, int levels, double r,
                          const double* __restrict__ kap, double* a, double* b, double* c,
                          double* cp, double* finv, double* alpha, double* gamma, double* k1,
                          double* k2, double* binv, double* A, double* B, double* C,
                          double* ee) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int m = 0; m < n; ++m) {
    const double kl = kap ? 0.5 * (kap[m] + kap[m + 1]) : 1.0;      // face m-1/2
    const double kr = kap ? 0.5 * (kap[m + 1] + kap[m + 2]) : 1.0;  // face m+1/2
    a[m] = m > 0 ? -r * kl : 0.0;
    c[m] = m < n - 1 ? -r * kr : 0.0;
    b[m] = 1.0 + r * (kl + kr);
    ee[m] = 1.0 - r * (kl + kr);
  }
  if (n == 1) {
    binv[0] = 1.0 / b[0];
    return;
  }
  const int R = 2 * P;
  for (int j = 0; j < P; ++j) {
    int s, L;
    chunk_of(j, base, rem, s, L);
    const int e = s + L - 1;
    // Thomas factors of the interior block rows s+1..e-1
    for (int m = s + 1; m <= e - 1; ++m) {
      const double den = (m == s + 1) ? b[m] : b[m] - a[m] * cp[m - 1];
      finv[m] = 1.0 / den;
      cp[m] = c[m] * finv[m];
    }
    // spikes: interior solves with right-hand sides a_{s+1} e_first and c_{e-1} e_last
    for (int m = s + 1; m <= e - 1; ++m) {
      const double ra = (m == s + 1) ? a[m] : 0.0;
      const double rg = (m == e - 1) ? c[m] : 0.0;
      alpha[m] = (m == s + 1) ? ra * finv[m] : (ra - a[m] * alpha[m - 1]) * finv[m];
      gamma[m] = (m == s + 1) ? rg * finv[m] : (rg - a[m] * gamma[m - 1]) * finv[m];
    }
    for (int m = e - 2; m >= s + 1; --m) {
      alpha[m] -= cp[m] * alpha[m + 1];
      gamma[m] -= cp[m] * gamma[m + 1];
    }
    // reduced rows 2j (x_s) and 2j+1 (x_e)
    if (L >= 3) {
      A[2 * j] = a[s];
      B[2 * j] = b[s] - c[s] * alpha[s + 1];
      C[2 * j] = -c[s] * gamma[s + 1];
      A[2 * j + 1] = -a[e] * alpha[e - 1];
      B[2 * j + 1] = b[e] - a[e] * gamma[e - 1];
      C[2 * j + 1] = c[e];
    } else {
      A[2 * j] = a[s];
      B[2 * j] = b[s];
      C[2 * j] = c[s];
      A[2 * j + 1] = a[e];
      B[2 * j + 1] = b[e];
      C[2 * j + 1] = c[e];
    }
  }
  // parallel cyclic reduction on the reduced matrix, recording the multipliers
  double nA[MAXR], nB[MAXR], nC[MAXR];
  for (int l = 0, sg = 1; l < levels; ++l, sg *= 2) {
    for (int i = 0; i < R; ++i) {
      const double m1 = (i - sg >= 0) ? A[i] / B[i - sg] : 0.0;
      const double m2 = (i + sg < R) ? C[i] / B[i + sg] : 0.0;
      k1[l * MAXR + i] = m1;
      k2[l * MAXR + i] = m2;
      nA[i] = (i - sg >= 0) ? -A[i - sg] * m1 : 0.0;
      nC[i] = (i + sg < R) ? -C[i + sg] * m2 : 0.0;
      nB[i] = B[i] - ((i - sg >= 0) ? C[i - sg] * m1 : 0.0) - ((i + sg < R) ? A[i + sg] * m2 : 0.0);
    }
    for (int i = 0; i < R; ++i) {
      A[i] = nA[i];
      B[i] = nB[i];
      C[i] = nC[i];
    }
  }
  for (int i = 0; i < R; ++i) binv[i] = 1.0 / B[i];
}

// One warp per state; `steps` solves in a row, state resident in shared memory.
__global__ void __launch_bounds__(32) tri_solve(TriDev t, const double* __restrict__ in,
                                                double* __restrict__ out, long long M, int steps) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x;
  const long long base_off = (long long)blockIdx.x * M;
  const int Ls = t.maxL + 1;  // odd-ish padding against bank conflicts
  const int big = t.rem * (t.base + 1);
  auto pos = [&](int i) {
    int j, off;
    if (i < big) {
      j = i / (t.base + 1);
      off = i - j * (t.base + 1);
    } else {
      j = t.rem + (i - big) / t.base;
      off = i - big - (j - t.rem) * t.base;
    }
    return j * Ls + off;
  };
  if (t.n == 1) {
    if (lane == 0) {
      double x = in[base_off];
      for (int s = 0; s < steps; ++s) x = (t.cn ? t.e[0] * x : x) * t.binv[0];
      out[base_off] = x;
    }
    return;
  }
  for (int i = lane; i < t.n; i += 32) sm[pos(i)] = in[base_off + i];
  __syncwarp();
  int s = 0, L = 0;
  if (lane < t.P) chunk_of(lane, t.base, t.rem, s, L);
  double* xc = sm + lane * Ls;  // this lane's chunk, local index 0..L-1
  for (int step = 0; step < steps; ++step) {
    if (t.cn) {
      // right-hand side (I - dt/2 A) u in place; the chunk's outer neighbours
      // are read before any lane overwrites its chunk
      double left = 0.0, right = 0.0;
      if (lane < t.P) {
        if (s > 0) left = sm[pos(s - 1)];
        if (s + L < t.n) right = sm[pos(s + L)];
      }
      __syncwarp();
      if (lane < t.P) {
        double prev = left;
        for (int m = 0; m < L; ++m) {
          const double cur = xc[m];
          const double nxt = m + 1 < L ? xc[m + 1] : right;
          xc[m] = t.e[s + m] * cur - t.a[s + m] * prev - t.c[s + m] * nxt;
          prev = cur;
        }
      }
      __syncwarp();
    }
    double r0 = 0.0, r1 = 0.0;
    if (lane < t.P) {
      // interior Thomas: forward then back substitution (y over d, in place)
      for (int m = 1; m <= L - 2; ++m) {
        const int gm = s + m;
        const double prev = (m == 1) ? 0.0 : xc[m - 1];
        xc[m] = (xc[m] - t.a[gm] * prev) * t.finv[gm];
      }
      for (int m = L - 3; m >= 1; --m) xc[m] -= t.cp[s + m] * xc[m + 1];
      const int e = s + L - 1;
      r0 = xc[0];
      r1 = xc[L - 1];
      if (L >= 3) {
        r0 -= t.c[s] * xc[1];
        r1 -= t.a[e] * xc[L - 2];
      }
    }
    // PCR over rows 2*lane (r0) and 2*lane+1 (r1)
    for (int l = 0, sg = 1; l < t.levels; ++l, sg *= 2) {
      const int i0 = 2 * lane, i1 = 2 * lane + 1;
      double l0, g0, l1, g1;  // left / right neighbours at distance sg
      if (sg == 1) {
        const double up1 = __shfl_up_sync(0xffffffffu, r1, 1);
        const double dn0 = __shfl_down_sync(0xffffffffu, r0, 1);
        l0 = lane >= 1 ? up1 : 0.0;
        g0 = r1;
        l1 = r0;
        g1 = lane + 1 < 32 ? dn0 : 0.0;
      } else {
        const int d = sg / 2;
        const double u0 = __shfl_up_sync(0xffffffffu, r0, d);
        const double u1 = __shfl_up_sync(0xffffffffu, r1, d);
        const double w0 = __shfl_down_sync(0xffffffffu, r0, d);
        const double w1 = __shfl_down_sync(0xffffffffu, r1, d);
        l0 = lane >= d ? u0 : 0.0;
        l1 = lane >= d ? u1 : 0.0;
        g0 = lane + d < 32 ? w0 : 0.0;
        g1 = lane + d < 32 ? w1 : 0.0;
      }
      if (lane < t.P) {
        r0 = r0 - t.k1[l * MAXR + i0] * l0 - t.k2[l * MAXR + i0] * g0;
        r1 = r1 - t.k1[l * MAXR + i1] * l1 - t.k2[l * MAXR + i1] * g1;
      } else {
        r0 = 0.0;
        r1 = 0.0;
      }
    }
    if (lane < t.P) {
      const double xs = r0 * t.binv[2 * lane];
      const double xe = r1 * t.binv[2 * lane + 1];
      for (int m = 1; m <= L - 2; ++m)
        xc[m] = xc[m] - t.alpha[s + m] * xs - t.gamma[s + m] * xe;
      xc[0] = xs;
      xc[L - 1] = xe;
    }
    __syncwarp();
  }
  for (int i = lane; i < t.n; i += 32) out[base_off + i] = sm[pos(i)];
}

TriDev dev_view(const TriTables* t) {
  TriDev d{};
  d.n = t->n;
  d.P = t->P;
  d.base = t->P ? t->n / t->P : 1;
  d.rem = t->P ? t->n % t->P : 0;
  d.levels = t->levels;
  d.maxL = d.base + (d.rem ? 1 : 0);
  const int n = t->n;
  d.a = t->buf;
  d.c = d.a + n;
  d.cp = d.c + n;
  d.finv = d.cp + n;
  d.alpha = d.finv + n;
  d.gamma = d.alpha + n;
  d.k1 = d.gamma + n;
  d.k2 = d.k1 + (size_t)t->levels * MAXR;
  d.binv = d.k2 + (size_t)t->levels * MAXR;
  d.e = d.binv + MAXR + n + 3 * MAXR;  // after the setup scratch
  d.cn = t->cn;
  return d;
}

}  // namespace

cudaError_t tri_build(pr_ctx* c, TriTables* t, int n, double r, const double* kappa, bool cn) {
  tri_free(t);
  t->n = n;
  t->cn = cn ? 1 : 0;
  t->P = n >= 2 ? (n / 2 < 32 ? n / 2 : 32) : 0;
  int R = 2 * t->P, levels = 0;
  while ((1 << levels) < R) ++levels;
  t->levels = levels;
  const size_t words = 6 * (size_t)n + 2 * (size_t)levels * MAXR + MAXR  // tables
                       + (size_t)n + 3 * MAXR                             // b and reduced scratch
                       + (size_t)n;                                       // e (trapezoidal rhs)
  cudaError_t e = cudaMalloc(&t->buf, words * sizeof(double));
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(t->buf, 0, words * sizeof(double), c->stream);
  if (e != cudaSuccess) return e;
  TriDev d = dev_view(t);
  double* b = const_cast<double*>(d.binv) + MAXR;
  double* A = b + n;
  double* B = A + MAXR;
  double* C = B + MAXR;
  tri_setup<<<1, 1, 0, c->stream>>>(n, t->P, d.base, d.rem, levels, r, kappa,
                                     const_cast<double*>(d.a), b, const_cast<double*>(d.c),
                                     const_cast<double*>(d.cp), const_cast<double*>(d.finv),
                                     const_cast<double*>(d.alpha), const_cast<double*>(d.gamma),
                                     const_cast<double*>(d.k1), const_cast<double*>(d.k2),
                                     const_cast<double*>(d.binv), A, B, C,
                                     const_cast<double*>(d.e));
  return cudaGetLastError();
}

void tri_free(TriTables* t) {
  if (t->buf) cudaFree(t->buf);
  *t = TriTables{};
}

cudaError_t tri_solve_steps(pr_ctx* c, const TriTables* t, const double* in, double* out,
                            int count, int steps) {
  if (count <= 0) return cudaSuccess;
  TriDev d = dev_view(t);
  const int P = d.P > 0 ? d.P : 1;
  const size_t smem = (size_t)P * (d.maxL + 1) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(tri_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  tri_solve<<<count, 32, smem, c->stream>>>(d, in, out, c->g.M, steps);
  return cudaGetLastError();
}

}  // namespace pr
