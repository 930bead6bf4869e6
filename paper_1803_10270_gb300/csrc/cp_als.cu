// CP route: exact RK2-polynomial application in CP form and ALS rank reduction.
//
// CP format and ALS: Section 2.1 (eqs. functional-SSE, als, SSYSTEM, A^{ln}_{jhp},
// f_{jh}^n).  With the grid basis the mode-k normal equations read
//   X_k Gamma_k = Y_k diag(mu) H_k,  Gamma_k = hadamard_{j!=k} X_j^T X_j,
//   H_k = hadamard_{j!=k} Y_j^T X_j,
// Gamma_k is r x r SPD and is factorised by Cholesky in FP64.  Sweeps are Gauss-Seidel
// over k = 1..d (the block Gauss-Seidel reading of Section 2.1); the damped Jacobi
// variant of Appendix B (Algorithm 1: every mode from the same iterate, increment / 4,
// Algorithm 5's convergence measure) is selectable.
//
// Per mode update: hadamard kernel -> GEMM (RHS) -> solve kernel (Cholesky, substitution,
// column normalisation, convergence measure) -> GEMM (refresh X_k^T X_k and Y_k^T X_k).
#include <cstring>

#include "common.cuh"

namespace {

constexpr int NT = 256;

struct CpArgs {
  int d, r, ry, variant;
  int n[HT_MAXD];
  const double* Y[HT_MAXD];
  double* X[HT_MAXD];
  const double* mu;
  double* lam;
};

__device__ inline int type_power(int ti, int d, int k) {
  // column-block types: 0: identity; 1..d: A_i; d+1..2d: A_i^2/2; then A_i A_j (i<j)
  if (ti == 0) return 0;
  if (ti <= d) return (ti - 1 == k) ? 1 : 0;
  if (ti <= 2 * d) return (ti - 1 - d == k) ? 2 : 0;
  int idx = ti - 1 - 2 * d;
  for (int i = 0; i < d; ++i)
    for (int j = i + 1; j < d; ++j) {
      if (idx == 0) return (i == k) + (j == k);
      --idx;
    }
  return 0;
}

struct StencilArgs {
  int d, r, nt;
  int n[HT_MAXD];
  int hw[HT_MAXD];
  double c[HT_MAXD][HT_MAXSTENCIL];
  const double* X[HT_MAXD];
  const double* w;
  double* Y[HT_MAXD];
  double* wy;
};

__device__ inline double stencil_at(const StencilArgs& a, int k, const double* x, int n, int j) {
  double s = 0.0;
  const int hw = a.hw[k];
  for (int o = -hw; o <= hw; ++o) {
    int jj = (j + o) % n;
    if (jj < 0) jj += n;
    s = fma(a.c[k][o + hw], x[jj], s);
  }
  return s;
}

__global__ void cp_apply_kernel(StencilArgs a) {
  extern __shared__ double sh[];
  const int k = blockIdx.y, l = blockIdx.x;
  const int n = a.n[k];
  double* x = sh;
  double* ax = sh + n;
  double* a2x = sh + 2 * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = a.X[k][j + (long long)n * l];
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) ax[j] = stencil_at(a, k, x, n, j);
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) a2x[j] = stencil_at(a, k, ax, n, j);
  __syncthreads();
  for (int ti = 0; ti < a.nt; ++ti) {
    const int p = type_power(ti, a.d, k);
    const double* src = p == 0 ? x : (p == 1 ? ax : a2x);
    double* dst = a.Y[k] + (long long)n * (ti * a.r + l);
    for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = src[j];
    if (k == 0 && threadIdx.x == 0) {
      const double coef = (ti > a.d && ti <= 2 * a.d) ? 0.5 : 1.0;
      a.wy[ti * a.r + l] = coef * a.w[l];
    }
  }
}

// Unit columns, norms into the weights (GS) or folded into factor 0 (Jacobi variant).
// One CTA: column norms of every factor (one warp per (dim, column)), then the scaling.
__global__ void cp_normalize_kernel(CpArgs a, int fold) {
  __shared__ double nrm[HT_MAXD * 64];
  __shared__ double wfin[64];
  const int tid = threadIdx.x, lane = tid & 31, nw = blockDim.x >> 5;
  if (a.r > 64) return;   // callers keep r <= 64 (checked on the host)
  for (int p = tid >> 5; p < a.d * a.r; p += nw) {
    const int k = p / a.r, l = p % a.r;
    const double* col = a.X[k] + (long long)a.n[k] * l;
    double s = 0.0;
    for (int j = lane; j < a.n[k]; j += 32) s = fma(col[j], col[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[p] = sqrt(s);
  }
  __syncthreads();
  for (int l = tid; l < a.r; l += blockDim.x) {
    double w = a.lam[l];
    for (int k = 0; k < a.d; ++k) {
      const double nr = nrm[k * a.r + l];
      const bool pos = htg_dpos_finite(nr);
      if (pos) w *= nr;
      nrm[k * a.r + l] = pos ? htg_rcp_fast(nr) : 1.0;
    }
    wfin[l] = w;
    a.lam[l] = fold ? 1.0 : w;
  }
  __syncthreads();
  for (int k = 0; k < a.d; ++k) {
    const int n = a.n[k];
    for (long long e = tid; e < (long long)n * a.r; e += blockDim.x) {
      const int l = (int)(e / n);
      double v = a.X[k][e] * nrm[k * a.r + l];
      if (fold && k == 0) v *= wfin[l];
      a.X[k][e] = v;
    }
  }
}

// Gamma = hadamard_{j!=k} G_j ; Hh = diag(mu) hadamard_{j!=k} H_j
__global__ void cp_hadamard_kernel(CpArgs a, CpWs w, int k) {
  const long long nh = (long long)a.ry * a.r, ng = (long long)a.r * a.r;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nh + ng;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nh) {
      const int m = (int)(e % a.ry);
      double v = a.mu[m];
      for (int j = 0; j < a.d; ++j)
        if (j != k) v *= w.H[(long long)j * w.rycap * w.rcap + e];
      w.Hh[e] = v;
    } else {
      const long long g = e - nh;
      double v = 1.0;
      for (int j = 0; j < a.d; ++j)
        if (j != k) v *= w.G[(long long)j * w.rcap * w.rcap + g];
      w.Gam[g] = v;
    }
  }
}

// Cholesky of Gamma (FP64), X~ = RHS Gamma^{-1}; then either (GS) normalise into X_k and
// lam, or (Jacobi) store X~ into Xold slot k.  Records |X~ - X_old lam_old| / |X_old lam_old|.
// The factorisation is right-looking and column parallel; every division is replaced by a
// multiplication with a reciprocal computed once (FP64 divides are long instruction
// sequences and each FP64 warp instruction holds the FP64 pipe for the whole warp).
__global__ void cp_solve_kernel(CpArgs a, CpWs w, int k, int sweep, int* err, double* flops) {
  extern __shared__ double sh[];
  const int r = a.r, n = a.n[k];
  double* Lm = sh;               // r x r (lower triangle used)
  double* rinv = sh + r * r;     // r reciprocals of the diagonal, later of the column norms
  double* Xs = rinv + r;         // n x r staged rows
  __shared__ int ok;
  __shared__ double red_num[NT / 32], red_den[NT / 32];
  const int tid = threadIdx.x;
  for (int attempt = 0; attempt < 2; ++attempt) {
    double shift = 0.0;
    if (attempt == 1) {
      double tr = 0.0;
      for (int i = 0; i < r; ++i) tr += w.Gam[i + r * i];
      shift = 1e-14 * tr / r;
    }
    for (int e = tid; e < r * r; e += blockDim.x) Lm[e] = w.Gam[e] + ((e % r == e / r) ? shift : 0.0);
    if (tid == 0) ok = 1;
    __syncthreads();
    for (int j = 0; j < r; ++j) {
      if (tid == 0) {
        const double dj = Lm[j + r * j];
        if (!htg_dpos_finite(dj)) ok = 0;
        const double sq = ok ? sqrt(dj) : 1.0;
        Lm[j + r * j] = sq;
        rinv[j] = 1.0 / sq;
      }
      __syncthreads();
      if (!ok) break;
      const double inv = rinv[j];
      for (int i = j + 1 + tid; i < r; i += blockDim.x) Lm[i + r * j] *= inv;
      __syncthreads();
      // trailing update of the lower triangle: L[i][c] -= L[i][j] L[c][j], j < c <= i
      const int m = r - j - 1;
      for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = j + 1 + e % m, cc = j + 1 + e / m;
        if (cc <= i) Lm[i + r * cc] -= Lm[i + r * j] * Lm[cc + r * j];
      }
      __syncthreads();
    }
    const int good = ok;
    __syncthreads();
    if (good) break;
  }
  if (!ok) {
    if (tid == 0 && err) atomicCAS(err, 0, (int)HT_ERR_NONFINITE);
    return;
  }
  // rows: solve L L^T x = rhs, x^T is row i of X~
  for (long long e = tid; e < (long long)n * r; e += blockDim.x) Xs[e] = w.RHS[e];
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    double* row = Xs + i;   // stride n between columns
    for (int j = 0; j < r; ++j) {
      double v = row[(long long)n * j];
      for (int p = 0; p < j; ++p) v -= Lm[j + r * p] * row[(long long)n * p];
      row[(long long)n * j] = v * rinv[j];
    }
    for (int j = r - 1; j >= 0; --j) {
      double v = row[(long long)n * j];
      for (int p = j + 1; p < r; ++p) v -= Lm[p + r * j] * row[(long long)n * p];
      row[(long long)n * j] = v * rinv[j];
    }
  }
  __syncthreads();
  // convergence measure against the old (scaled) factor
  double num = 0.0, den = 0.0;
  for (long long e = tid; e < (long long)n * r; e += blockDim.x) {
    const int l = (int)(e / n);
    const double old = a.X[k][e] * (a.variant == CP_ALS_GS ? a.lam[l] : 1.0);
    const double df = Xs[e] - old;
    num = fma(df, df, num);
    den = fma(old, old, den);
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((tid & 31) == 0) { red_num[tid >> 5] = num; red_den[tid >> 5] = den; }
  __syncthreads();
  // column norms: one warp per column
  for (int l = tid >> 5; l < r; l += blockDim.x >> 5) {
    double s2 = 0.0;
    for (int j = tid & 31; j < n; j += 32) s2 = fma(Xs[j + (long long)n * l], Xs[j + (long long)n * l], s2);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if ((tid & 31) == 0) {
      const double nr = sqrt(s2);
      a.lam[l] = (a.variant == CP_ALS_GS) ? nr : a.lam[l];
      rinv[l] = htg_dpos_finite(nr) ? htg_rcp_fast(nr) : 1.0;
    }
  }
  if (tid == 0 && flops) {
    // Cholesky (r^3/3 multiply-adds), two triangular solves per row, measure and norms
    const double rr = (double)r;
    atomicAdd(flops, 2.0 * rr * rr * rr / 3.0 + 2.0 * n * rr * rr + 6.0 * n * rr);
  }
  if (tid == 0) {
    double tn = 0.0, td = 0.0;
    for (int q = 0; q < NT / 32; ++q) { tn += red_num[q]; td += red_den[q]; }
    const double ek = td > 0.0 ? sqrt(tn / td) : sqrt(tn);
    if (ek > w.epsacc[sweep]) w.epsacc[sweep] = ek;
  }
  __syncthreads();
  if (a.variant == CP_ALS_GS) {
    for (long long e = tid; e < (long long)n * r; e += blockDim.x) a.X[k][e] = Xs[e] * rinv[e / n];
  } else {
    double* dst = w.Xold + (long long)k * w.nmax * w.rcap;
    for (long long e = tid; e < (long long)n * r; e += blockDim.x) dst[e] = Xs[e];
  }
}

// Jacobi variant: X_k <- X_k + (X~_k - X_k)/4 for every k.
__global__ void cp_damp_kernel(CpArgs a, CpWs w) {
  const int k = blockIdx.y;
  const int n = a.n[k];
  const double* src = w.Xold + (long long)k * w.nmax * w.rcap;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * a.r;
       e += (long long)gridDim.x * blockDim.x)
    a.X[k][e] += 0.25 * (src[e] - a.X[k][e]);
}

__global__ void cp_eps_init_kernel(CpWs w, int sweeps) {
  for (int i = threadIdx.x; i < sweeps && i < 64; i += blockDim.x) w.epsacc[i] = 0.0;
}

__global__ void cp_eps_out_kernel(CpWs w, int sweeps, double* out) {
  for (int i = threadIdx.x; i < sweeps; i += blockDim.x) out[i] = w.epsacc[i];
}

// GEMM descriptors of one call: per mode k: [RHS_k, G_k, H_k]
__global__ void cp_plan_kernel(CpArgs a, CpWs w) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < a.d; ++k) {
    GemmDesc* g = w.descs + 3 * k;
    const int n = a.n[k];
    for (int q = 0; q < 3; ++q) {
      g[q].colscale = nullptr;
      g[q].sA = g[q].sB = g[q].sC = 0;
      g[q].batch = 1;
      g[q].alpha = 1.0;
      g[q].beta = 0.0;
    }
    // RHS = Y_k (n x ry) * Hh (ry x r)
    g[0].A = a.Y[k]; g[0].lda = n; g[0].tA = 0;
    g[0].B = w.Hh; g[0].ldb = a.ry; g[0].tB = 0;
    g[0].C = w.RHS; g[0].ldc = n;
    g[0].m = n; g[0].n = a.r; g[0].k = a.ry;
    // G_k = X_k^T X_k (r x r), ld = r
    g[1].A = a.X[k]; g[1].lda = n; g[1].tA = 1;
    g[1].B = a.X[k]; g[1].ldb = n; g[1].tB = 0;
    g[1].C = w.G + (long long)k * w.rcap * w.rcap; g[1].ldc = a.r;
    g[1].m = a.r; g[1].n = a.r; g[1].k = n;
    // H_k = Y_k^T X_k (ry x r), ld = ry
    g[2].A = a.Y[k]; g[2].lda = n; g[2].tA = 1;
    g[2].B = a.X[k]; g[2].ldb = n; g[2].tB = 0;
    g[2].C = w.H + (long long)k * w.rycap * w.rcap; g[2].ldc = a.ry;
    g[2].m = a.ry; g[2].n = a.r; g[2].k = n;
  }
}

// ---------------------------------------------------------------------------
// ALS against the implicit y = p(dt L) x_old (Kronecker-sum L): the factors of y are
// built from the three powers Z_j^(p) = A_j^p X_old,j (p = 0, 1, 2), so with
// M_j^(p) = Z_j^(p)T X_j (r0 x r) the mode-k system becomes
//   RHS = sum_p Z_k^(p) Hs_p,  Hs_p = sum_{tau : p_tau(k) = p} c_tau diag(mu) hadamard_{j!=k} M_j^(p_tau(j))
// with the column types tau of cp_apply_rk2.  Same result as cp_als_sweep on the formed y.
// ---------------------------------------------------------------------------
struct PowArgs {
  int d, r0;
  int n[HT_MAXD];
  int hw[HT_MAXD];
  double c[HT_MAXD][HT_MAXSTENCIL];
  const double* X[HT_MAXD];
};

__global__ void cp_powers_kernel(PowArgs a, CpWs w) {
  extern __shared__ double sh[];
  const int k = blockIdx.y, l = blockIdx.x;
  const int n = a.n[k];
  double* x = sh;
  double* ax = sh + n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = a.X[k][j + (long long)n * l];
  __syncthreads();
  double* Zk = w.Z + (long long)k * w.nmax * 3 * w.rcap;   // n x 3 r0, ld n
  const int hw = a.hw[k];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0;
    for (int o = -hw; o <= hw; ++o) {
      int jj = (j + o) % n;
      if (jj < 0) jj += n;
      s = fma(a.c[k][o + hw], x[jj], s);
    }
    ax[j] = s;
    Zk[j + (long long)n * l] = x[j];
    Zk[j + (long long)n * (a.r0 + l)] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s = 0.0;
    for (int o = -hw; o <= hw; ++o) {
      int jj = (j + o) % n;
      if (jj < 0) jj += n;
      s = fma(a.c[k][o + hw], ax[jj], s);
    }
    Zk[j + (long long)n * (2 * a.r0 + l)] = s;
  }
}

// Gamma = hadamard_{j!=k} G_j ; Hs (3 r0 x r) as above.  M_j lives in w.H (3 r0 x r, ld 3 r0).
__global__ void cp_hadamard_rk2_kernel(CpArgs a, CpWs w, int k, int r0, const double* mu) {
  const int d = a.d, r = a.r;
  const long long nh = (long long)r0 * r, ng = (long long)r * r;
  const int nt = 1 + 2 * d + d * (d - 1) / 2;
  // type table: power of A_j in column type tau (<= 1 + 2*16 + 120 types, d <= 16)
  __shared__ unsigned char pw[153][HT_MAXD];
  __shared__ double cf[153];
  for (int e = threadIdx.x; e < nt * d; e += blockDim.x) pw[e / d][e % d] = (unsigned char)type_power(e / d, d, e % d);
  for (int e = threadIdx.x; e < nt; e += blockDim.x) cf[e] = (e > d && e <= 2 * d) ? 0.5 : 1.0;
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nh + ng;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < nh) {
      const int lp = (int)(e % r0), l = (int)(e / r0);
      const double* Hb = w.H + (lp + (long long)3 * r0 * l);
      double hs[3] = {0.0, 0.0, 0.0};
      for (int ti = 0; ti < nt; ++ti) {
        double v = cf[ti];
        for (int j = 0; j < d; ++j) {
          if (j == k) continue;
          v *= Hb[(long long)j * w.rycap * w.rcap + pw[ti][j] * r0];
        }
        hs[pw[ti][k]] += v;
      }
      const double m = mu[lp];
      for (int pp = 0; pp < 3; ++pp) w.Hh[(pp * r0 + lp) + (long long)3 * r0 * l] = m * hs[pp];
    } else {
      const long long g = e - nh;
      double v = 1.0;
      for (int j = 0; j < d; ++j)
        if (j != k) v *= w.G[(long long)j * w.rcap * w.rcap + g];
      w.Gam[g] = v;
    }
  }
}

// Mode update of the structured ALS, part 1 (one CTA per row index lp of the r0 x r block):
//   hs_p[l] = mu_lp sum_{tau: p_tau(k) = p} c_tau prod_{j != k} M_j^(p_tau(j))[lp, l]   (p = 0,1,2)
//   Gamma = hadamard_{j != k} G_j, Gamma = L L^T (FP64 Cholesky, shifted only on failure)
//   W[p r0 + lp, :] = hs_p Gamma^{-1}    (forward and back substitution)
// Then X~_k = Z_k W (a GEMM over all SMs) equals RHS Gamma^{-1} of the normal equations.
// The M_j operands of a thread are loaded into registers before any product (an L2 latency
// chain otherwise), and each CTA repeats the small Cholesky so no grid-wide sync is needed.
constexpr int MODE_MAXR = 64;
constexpr int MODE_MAXD = 16;

__global__ void cp_mode_prep_kernel(CpArgs a, CpWs w, int k, int r0, const double* mu, int* err) {
  extern __shared__ double sh[];
  const int d = a.d, r = a.r, lp = blockIdx.x, tid = threadIdx.x;
  double* Lm = sh;              // r x r
  double* hs = Lm + r * r;      // 3 x r
  double* rinv = hs + 3 * r;    // r
  __shared__ unsigned char pw[153][MODE_MAXD];
  __shared__ double cf[153];
  __shared__ int ok;
  const int nt = 1 + 2 * d + d * (d - 1) / 2;
  for (int e = tid; e < nt * d; e += blockDim.x) pw[e / d][e % d] = (unsigned char)type_power(e / d, d, e % d);
  for (int e = tid; e < nt; e += blockDim.x) cf[e] = (e > d && e <= 2 * d) ? 0.5 : 1.0;
  __syncthreads();
  // hs: thread per column l, operands in registers
  for (int l = tid; l < r; l += blockDim.x) {
    double mv[MODE_MAXD][3];
    for (int j = 0; j < d; ++j) {
      if (j == k) continue;
      const double* Mj = w.H + (long long)j * w.rycap * w.rcap + lp + (long long)3 * r0 * l;
      mv[j][0] = Mj[0];
      mv[j][1] = Mj[r0];
      mv[j][2] = Mj[2 * r0];
    }
    double acc[3] = {0.0, 0.0, 0.0};
    for (int ti = 0; ti < nt; ++ti) {
      double v = cf[ti];
      for (int j = 0; j < d; ++j)
        if (j != k) v *= mv[j][pw[ti][j]];
      acc[pw[ti][k]] += v;
    }
    const double m = mu[lp];
    hs[l] = m * acc[0];
    hs[r + l] = m * acc[1];
    hs[2 * r + l] = m * acc[2];
  }
  // Gamma
  for (int e = tid; e < r * r; e += blockDim.x) {
    double v = 1.0;
    for (int j = 0; j < d; ++j)
      if (j != k) v *= w.G[(long long)j * w.rcap * w.rcap + e];
    Lm[e] = v;
  }
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (attempt == 1) {
      double tr = 0.0;
      for (int i = 0; i < r; ++i) {
        double v = 1.0;
        for (int j = 0; j < d; ++j)
          if (j != k) v *= w.G[(long long)j * w.rcap * w.rcap + i + r * i];
        tr += v;
      }
      const double shift = 1e-14 * tr / r;
      for (int e = tid; e < r * r; e += blockDim.x) {
        double v = 1.0;
        for (int j = 0; j < d; ++j)
          if (j != k) v *= w.G[(long long)j * w.rcap * w.rcap + e];
        Lm[e] = v + ((e % r == e / r) ? shift : 0.0);
      }
    }
    if (tid == 0) ok = 1;
    __syncthreads();
    for (int j = 0; j < r; ++j) {
      if (tid == 0) {
        const double dj = Lm[j + r * j];
        if (!htg_dpos_finite(dj)) ok = 0;
        const double ri = ok ? htg_rsqrt_fast(dj) : 1.0;
        Lm[j + r * j] = ok ? dj * ri : 1.0;
        rinv[j] = ri;
      }
      __syncthreads();
      if (!ok) break;
      const double inv = rinv[j];
      for (int i = j + 1 + tid; i < r; i += blockDim.x) Lm[i + r * j] *= inv;
      __syncthreads();
      const int m = r - j - 1;
      for (int e = tid; e < m * m; e += blockDim.x) {
        const int i = j + 1 + e % m, cc = j + 1 + e / m;
        if (cc <= i) Lm[i + r * cc] -= Lm[i + r * j] * Lm[cc + r * j];
      }
      __syncthreads();
    }
    const int good = ok;
    __syncthreads();
    if (good) break;
  }
  if (!ok) {
    if (tid == 0 && err) atomicCAS(err, 0, (int)HT_ERR_NONFINITE);
    return;
  }
  // L L^T w = hs_p for the three vectors, column oriented (short dependency chains):
  // forward  v_j <- v_j / L_jj, then v_i -= L_ij v_j (i > j);
  // backward v_j <- v_j / L_jj, then v_i -= L_ji v_j (i < j)
  for (int j = 0; j < r; ++j) {
    if (tid < 3) hs[tid * r + j] *= rinv[j];
    __syncthreads();
    for (int e = tid; e < 3 * (r - j - 1); e += blockDim.x) {
      const int pv = e / (r - j - 1), i = j + 1 + e % (r - j - 1);
      hs[pv * r + i] -= Lm[i + r * j] * hs[pv * r + j];
    }
    __syncthreads();
  }
  for (int j = r - 1; j >= 0; --j) {
    if (tid < 3) hs[tid * r + j] *= rinv[j];
    __syncthreads();
    for (int e = tid; e < 3 * j; e += blockDim.x) {
      const int pv = e / j, i = e % j;
      hs[pv * r + i] -= Lm[j + r * i] * hs[pv * r + j];
    }
    __syncthreads();
  }
  for (int e = tid; e < 3 * r; e += blockDim.x) {
    const int pp = e / r, l = e % r;
    w.Hh[(pp * r0 + lp) + (long long)3 * r0 * l] = hs[e];
  }
}

// Part 3: convergence measure, column norms, X_k (GS) or the Jacobi slot.  X~ is in w.RHS.
__global__ void cp_mode_finish_kernel(CpArgs a, CpWs w, int k, int sweep, double* flops) {
  const int r = a.r, n = a.n[k], tid = threadIdx.x;
  __shared__ double rinv[MODE_MAXR];
  __shared__ double red_num[NT / 32], red_den[NT / 32];
  double num = 0.0, den = 0.0;
  for (long long e = tid; e < (long long)n * r; e += blockDim.x) {
    const int l = (int)(e / n);
    const double old = a.X[k][e] * (a.variant == CP_ALS_GS ? a.lam[l] : 1.0);
    const double df = w.RHS[e] - old;
    num = fma(df, df, num);
    den = fma(old, old, den);
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  if ((tid & 31) == 0) { red_num[tid >> 5] = num; red_den[tid >> 5] = den; }
  __syncthreads();
  for (int l = tid >> 5; l < r; l += blockDim.x >> 5) {
    double s2 = 0.0;
    for (int j = tid & 31; j < n; j += 32) s2 = fma(w.RHS[j + (long long)n * l], w.RHS[j + (long long)n * l], s2);
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if ((tid & 31) == 0) {
      const double nr = sqrt(s2);
      if (a.variant == CP_ALS_GS) a.lam[l] = nr;
      rinv[l] = htg_dpos_finite(nr) ? htg_rcp_fast(nr) : 1.0;
    }
  }
  if (tid == 0) {
    double tn = 0.0, td = 0.0;
    for (int q = 0; q < NT / 32; ++q) { tn += red_num[q]; td += red_den[q]; }
    const double ek = td > 0.0 ? sqrt(tn / td) : sqrt(tn);
    if (ek > w.epsacc[sweep]) w.epsacc[sweep] = ek;
    if (flops) atomicAdd(flops, 8.0 * n * r);
  }
  __syncthreads();
  if (a.variant == CP_ALS_GS) {
    for (long long e = tid; e < (long long)n * r; e += blockDim.x) a.X[k][e] = w.RHS[e] * rinv[e / n];
  } else {
    double* dst = w.Xold + (long long)k * w.nmax * w.rcap;
    for (long long e = tid; e < (long long)n * r; e += blockDim.x) dst[e] = w.RHS[e];
  }
}

// descriptors per mode k: [RHS_k = Z_k (n x 3r0) Hs (3r0 x r), G_k = X_k^T X_k, M_k = Z_k^T X_k]
__global__ void cp_plan_rk2_kernel(CpArgs a, CpWs w, int r0) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < a.d; ++k) {
    GemmDesc* g = w.descs + 3 * k;
    const int n = a.n[k];
    const double* Zk = w.Z + (long long)k * w.nmax * 3 * w.rcap;
    for (int q = 0; q < 3; ++q) {
      g[q].colscale = nullptr;
      g[q].sA = g[q].sB = g[q].sC = 0;
      g[q].batch = 1;
      g[q].alpha = 1.0;
      g[q].beta = 0.0;
    }
    g[0].A = Zk; g[0].lda = n; g[0].tA = 0;
    g[0].B = w.Hh; g[0].ldb = 3 * r0; g[0].tB = 0;
    g[0].C = w.RHS; g[0].ldc = n;
    g[0].m = n; g[0].n = a.r; g[0].k = 3 * r0;
    g[1].A = a.X[k]; g[1].lda = n; g[1].tA = 1;
    g[1].B = a.X[k]; g[1].ldb = n; g[1].tB = 0;
    g[1].C = w.G + (long long)k * w.rcap * w.rcap; g[1].ldc = a.r;
    g[1].m = a.r; g[1].n = a.r; g[1].k = n;
    g[2].A = Zk; g[2].lda = n; g[2].tA = 1;
    g[2].B = a.X[k]; g[2].ldb = n; g[2].tB = 0;
    g[2].C = w.H + (long long)k * w.rycap * w.rcap; g[2].ldc = 3 * r0;
    g[2].m = 3 * r0; g[2].n = a.r; g[2].k = n;
  }
}

__global__ void cp_copy_weights_kernel(const double* src, double* dst, int r) {
  for (int i = threadIdx.x; i < r; i += blockDim.x) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// Persistent form of cp_als_sweep_rk2: one cooperative launch runs every sweep.  CTA b owns
// factor column b (row b of the r0 x r blocks in the solve phase); phases are separated by
// a grid barrier:
//   0a  powers Z_j^(p) of x_old (CTA b < r0), mu <- weights of x_old, normalise column b of x
//   0b  column b of G_j = X_j^T X_j and M_j = Z_j^T X_j for every j
//   per mode k:  A  Gamma_k (Cholesky) and row b of W = Hs Gamma_k^-1      (CTA b < r0)
//                B  column b of X~_k = Z_k W, convergence sums, X_k[:, b] and lam_b
//                C  column b of G_k and M_k; CTA 0 records the mode's convergence measure
// The launch is cooperative (all CTAs resident), and every barrier wait is bounded: past the
// limit the kernel records HT_ERR_TIMEOUT in the error word and returns.
// ---------------------------------------------------------------------------
constexpr long long BARRIER_TIMEOUT_CYCLES = 400000000LL;   // about 0.2 s

__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, int* err) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
    int ok = 1;
    if (arrived == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (clock64() - t0 > BARRIER_TIMEOUT_CYCLES) {
          ok = 0;
          if (err) atomicCAS(err, 0, (int)HT_ERR_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Copy count doubles global -> shared with 8 independent loads in flight per thread (a plain
// copy loop waits out the full L2 latency on every element).  Plain (coherent) loads: the
// sources are written by other CTAs of the same launch before a grid barrier.
__device__ void stage_copy(double* dst, const double* src, long long count) {
  const int T = blockDim.x;
  long long base = 0;
  for (; base + 8LL * T <= count; base += 8LL * T) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = src[base + (long long)u * T + threadIdx.x];
#pragma unroll
    for (int u = 0; u < 8; ++u) dst[base + (long long)u * T + threadIdx.x] = v[u];
  }
  for (long long e = base + threadIdx.x; e < count; e += T) dst[e] = src[e];
}

// column b of G_j (r values) and, when withM, of M_j (3 r0 values); X_j[:, b] staged in xs
__device__ void gram_column(const CpArgs& a, CpWs& w, int j, int b, int r0, bool withM, double* xs,
                            double* stage = nullptr) {
  const int n = a.n[j], r = a.r;
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = a.X[j][i + (long long)n * b];
  const double* Zj = w.Z + (long long)j * w.nmax * 3 * w.rcap;
  const double* Xsrc = a.X[j];
  const double* Zsrc = Zj;
  if (stage) {   // [X_j | Z_j] (n x (r + 3 r0)) in shared memory
    stage_copy(stage, a.X[j], (long long)n * r);
    if (withM) stage_copy(stage + (long long)n * r, Zj, (long long)n * 3 * r0);
    Xsrc = stage;
    Zsrc = stage + (long long)n * r;
  }
  __syncthreads();
  const int nout = r + (withM ? 3 * r0 : 0);
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    const double* src = (o < r) ? Xsrc + (long long)n * o : Zsrc + (long long)n * (o - r);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 3 < n; i += 4) {
      s0 = fma(src[i], xs[i], s0);
      s1 = fma(src[i + 1], xs[i + 1], s1);
      s2 = fma(src[i + 2], xs[i + 2], s2);
      s3 = fma(src[i + 3], xs[i + 3], s3);
    }
    for (; i < n; ++i) s0 = fma(src[i], xs[i], s0);
    const double v = (s0 + s1) + (s2 + s3);
    if (o < r) w.G[(long long)j * w.rcap * w.rcap + o + (long long)r * b] = v;
    else w.H[(long long)j * w.rycap * w.rcap + (o - r) + (long long)3 * r0 * b] = v;
  }
  __syncthreads();
}

// unit columns across all dimensions for column b (norms into lam_b, or folded into X_0 when fold)
__device__ void normalise_column(const CpArgs& a, int b, bool fold, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = wid; k < a.d; k += blockDim.x >> 5) {
    const double* col = a.X[k] + (long long)a.n[k] * b;
    double s = 0.0;
    for (int j = lane; j < a.n[k]; j += 32) s = fma(col[j], col[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[k] = sqrt(s);
  }
  __syncthreads();
  __shared__ double wfin;
  if (threadIdx.x == 0) {
    double wv = a.lam[b];
    for (int k = 0; k < a.d; ++k) {
      const double nr = red[k];
      const bool pos = htg_dpos_finite(nr);
      if (pos) wv *= nr;
      red[k] = pos ? htg_rcp_fast(nr) : 1.0;
    }
    wfin = wv;
    a.lam[b] = fold ? 1.0 : wv;
  }
  __syncthreads();
  for (int k = 0; k < a.d; ++k) {
    double* col = a.X[k] + (long long)a.n[k] * b;
    const double sc = red[k] * ((fold && k == 0) ? wfin : 1.0);
    for (int j = threadIdx.x; j < a.n[k]; j += blockDim.x) col[j] *= sc;
  }
  __syncthreads();
}

// one Newton step on an FP32 seed: relative error ~1e-13, ample for a Cholesky pivot
__device__ inline double rsqrt_pivot(double x) {
  if (!htg_in_f32_range(x) || !htg_dpos(x)) return rsqrt(x);
  const double y = htg_f2d(rsqrtf(htg_d2f(x)));
  const double h = x * y;
  return fma(0.5 * y, fma(-h, y, 1.0), y);
}

__global__ void __launch_bounds__(NT) cp_als_rk2_persistent(CpArgs a, PowArgs pa, CpWs w, const double* mu_src,
                                                            int sweeps, int* err, int zs_smem) {
  const int b = blockIdx.x, tid = threadIdx.x;
  const unsigned int nb = gridDim.x;
  const int d = a.d, r = a.r, r0 = pa.r0;
  const int nmax = w.nmax;
  extern __shared__ double sh[];
  double* Lm = sh;                         // r x r
  double* hs = Lm + r * r;                 // 3 r
  double* rinv = hs + 3 * r;               // r
  double* xs = rinv + r;                   // nmax
  double* ys = xs + nmax;                  // nmax
  double* Mv = ys + nmax;                  // d x 3 x r   (M_j rows of this CTA's lp)
  const int nt_ = 1 + 2 * d + d * (d - 1) / 2;
  double* Xs = Mv + 3 * d * r;             // max(nmax, types) x r: a staged factor, or type products
  double* Zs = Xs + (long long)htg_max(nmax, nt_) * r;   // nmax x 3 r0 (Z_k, when zs_smem)
  __shared__ unsigned char pw[153][MODE_MAXD];
  __shared__ double cf[153];
  __shared__ double red[HT_MAXD + 32];
  __shared__ int ok;
  const int nt = 1 + 2 * d + d * (d - 1) / 2;
  for (int e = tid; e < nt * d; e += blockDim.x) pw[e / d][e % d] = (unsigned char)type_power(e / d, d, e % d);
  for (int e = tid; e < nt; e += blockDim.x) cf[e] = (e > d && e <= 2 * d) ? 0.5 : 1.0;
  const bool gs = (a.variant == CP_ALS_GS);
  // ---------------- 0a: powers of x_old (CTA b < r0), weights, normalisation of column b
  if (b < r0) {
    for (int k = 0; k < d; ++k) {
      const int n = pa.n[k], hw = pa.hw[k];
      for (int j = tid; j < n; j += blockDim.x) xs[j] = pa.X[k][j + (long long)n * b];
      __syncthreads();
      double* Zk = w.Z + (long long)k * nmax * 3 * w.rcap;
      for (int j = tid; j < n; j += blockDim.x) {
        double s = 0.0;
        for (int o = -hw; o <= hw; ++o) {
          int jj = (j + o) % n;
          if (jj < 0) jj += n;
          s = fma(pa.c[k][o + hw], xs[jj], s);
        }
        ys[j] = s;
        Zk[j + (long long)n * b] = xs[j];
        Zk[j + (long long)n * (r0 + b)] = s;
      }
      __syncthreads();
      for (int j = tid; j < n; j += blockDim.x) {
        double s = 0.0;
        for (int o = -hw; o <= hw; ++o) {
          int jj = (j + o) % n;
          if (jj < 0) jj += n;
          s = fma(pa.c[k][o + hw], ys[jj], s);
        }
        Zk[j + (long long)n * (2 * r0 + b)] = s;
      }
      __syncthreads();
    }
  }
  if (b == 0) {
    for (int i = tid; i < r0; i += blockDim.x) w.wold[i] = mu_src[i];
    for (int i = tid; i < sweeps && i < 64; i += blockDim.x) w.epsacc[i] = 0.0;
  }
  // the iterate may alias x_old: everything of x_old is read above, before the barrier
  if (!grid_barrier(w.bar, nb, err)) return;
  if (b < r) normalise_column(a, b, !gs, red);
  if (!grid_barrier(w.bar, nb, err)) return;
  // ---------------- 0b: column b of G_j and M_j for every j
  if (b < r)
    for (int j = 0; j < d; ++j) gram_column(a, w, j, b, r0, true, xs, zs_smem ? Xs : nullptr);
  if (!grid_barrier(w.bar, nb, err)) return;
  const double* mu = w.wold;
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int k = 0; k < d; ++k) {
      const bool record = !(sweep == 0 && k == 0);  // the previous mode's sums are complete
      // ---------------- A: Gamma_k (Cholesky) and row lp = b of W = Hs Gamma_k^-1
      if (b < r0) {
        const int lp = b;
        if (b == 0 && tid == 0 && record) {
          // record the previous mode's convergence measure (its sums are complete)
          const double tn = w.acc2[0], td = w.acc2[1];
          const double ek = htg_dpos_finite(td) ? sqrt(tn / td) : sqrt(tn);
          const int sw = (k == 0) ? sweep - 1 : sweep;
          if (htg_dgt_nn(ek, w.epsacc[sw])) w.epsacc[sw] = ek;
        }
        // M_j operands of row lp (j != k), and the factor updated last, into shared memory
        for (int e = tid; e < 3 * d * r; e += blockDim.x) {
          const int j = e / (3 * r), rem = e % (3 * r), pp = rem / r, l = rem % r;
          Mv[e] = (j == k) ? 0.0 : w.H[(long long)j * w.rycap * w.rcap + (pp * r0 + lp) + (long long)3 * r0 * l];
        }
        __syncthreads();
        if (b == 0 && tid == 0) { w.acc2[0] = 0.0; w.acc2[1] = 0.0; }
        // hs_p[l] = mu_lp sum_{tau: p_tau(k) = p} c_tau prod_{j != k} M_j^(p_tau(j))[lp, l]:
        // every (type, l) product by its own thread into Xs, then sums per (p, l) in type order
        for (int e = tid; e < nt * r; e += blockDim.x) {
          const int ti = e / r, l = e % r;
          double v = cf[ti];
          for (int j = 0; j < d; ++j)
            if (j != k) v *= Mv[(j * 3 + pw[ti][j]) * r + l];
          Xs[e] = v;
        }
        __syncthreads();
        for (int e = tid; e < 3 * r; e += blockDim.x) {
          const int pp = e / r, l = e % r;
          double acc0 = 0.0;
          for (int ti = 0; ti < nt; ++ti)
            if (pw[ti][k] == pp) acc0 += Xs[ti * r + l];
          hs[e] = mu[lp] * acc0;
        }
        __syncthreads();
        // Gamma_k = hadamard_{j != k} G_j
        for (int e = tid; e < r * r; e += blockDim.x) {
          double v = 1.0;
          for (int j = 0; j < d; ++j)
            if (j != k) v *= w.G[(long long)j * w.rcap * w.rcap + e];
          Lm[e] = v;
        }
        __syncthreads();
        for (int attempt = 0; attempt < 2; ++attempt) {
          if (attempt == 1) {
            // shift by 1e-14 tr(Gamma)/r, only after a failed factorisation
            __shared__ double shift;
            if (tid == 0) {
              double tr = 0.0;
              for (int i = 0; i < r; ++i) {
                double v = 1.0;
                for (int j = 0; j < d; ++j)
                  if (j != k) v *= w.G[(long long)j * w.rcap * w.rcap + i + r * i];
                tr += v;
              }
              shift = 1e-14 * tr / r;
            }
            __syncthreads();
            for (int e = tid; e < r * r; e += blockDim.x) {
              double v = 1.0;
              for (int j = 0; j < d; ++j)
                if (j != k) v *= w.G[(long long)j * w.rcap * w.rcap + e];
              Lm[e] = v + ((e % r == e / r) ? shift : 0.0);
            }
            // the forward solve below overwrote hs: rebuild it (products still in Xs)
            for (int e = tid; e < 3 * r; e += blockDim.x) {
              const int pp = e / r, l = e % r;
              double acc0 = 0.0;
              for (int ti = 0; ti < nt; ++ti)
                if (pw[ti][k] == pp) acc0 += Xs[ti * r + l];
              hs[e] = mu[lp] * acc0;
            }
          }
          if (tid == 0) {
            ok = 1;
            const double d0 = Lm[0];
            ok = htg_dpos_finite(d0);
            rinv[0] = ok ? rsqrt_pivot(d0) : 1.0;
          }
          __syncthreads();
          // right-looking Cholesky, forward substitution fused in: step j scales column j
          // (L_ij = a_ij / L_jj) and y_j, then applies the rank-1 updates with one FMA each; the
          // thread that finishes pivot j+1 computes its reciprocal root at once
          for (int j = 0; j < r && ok; ++j) {
            const double rj = rinv[j];
            for (int e = tid; e < r - j; e += blockDim.x) {
              if (e == 0) {
                for (int pv = 0; pv < 3; ++pv) hs[pv * r + j] *= rj;
                Lm[j + r * j] *= rj;       // d_j / sqrt(d_j)
              } else {
                Lm[j + e + r * j] *= rj;
              }
            }
            __syncthreads();
            const int m = r - j - 1;
            for (int e = tid; e < m * m + 3 * m; e += blockDim.x) {
              if (e < m * m) {
                const int i = j + 1 + e % m, cc = j + 1 + e / m;
                if (cc <= i) {
                  const double v = fma(-Lm[i + r * j], Lm[cc + r * j], Lm[i + r * cc]);
                  Lm[i + r * cc] = v;
                  if (i == j + 1 && cc == j + 1) {
                    const bool good = htg_dpos_finite(v);
                    if (!good) ok = 0;
                    rinv[j + 1] = good ? rsqrt_pivot(v) : 1.0;
                  }
                }
              } else {
                const int f = e - m * m, pv = f / m, i = j + 1 + f % m;
                hs[pv * r + i] = fma(-Lm[i + r * j], hs[pv * r + j], hs[pv * r + i]);
              }
            }
            __syncthreads();
          }
          const int good = ok;
          __syncthreads();
          if (good) break;
        }
        if (!ok) {
          if (tid == 0 && err) atomicCAS(err, 0, (int)HT_ERR_NONFINITE);
        } else {
          // back substitution L^T w = y (y already in hs, columns of L scaled)
          for (int j = r - 1; j >= 0; --j) {
            if (tid < 3) hs[tid * r + j] *= rinv[j];
            __syncthreads();
            for (int e = tid; e < 3 * j; e += blockDim.x) {
              const int pv = e / j, i = e % j;
              hs[pv * r + i] -= Lm[j + r * i] * hs[pv * r + j];
            }
            __syncthreads();
          }
        }
        for (int e = tid; e < 3 * r; e += blockDim.x) {
          const int pp = e / r, l = e % r;
          w.Hh[(pp * r0 + lp) + (long long)3 * r0 * l] = hs[e];
        }
      }
      if (!grid_barrier(w.bar, nb, err)) return;
      // ---------------- B: column b of X~_k = Z_k W, X_k[:, b], lam_b, and M_k[:, b]
      if (b < r) {
        const int n = a.n[k];
        const int K = 3 * r0;
        const double* Zg = w.Z + (long long)k * nmax * 3 * w.rcap;
        const double* Zk = Zg;
        if (zs_smem) {
          stage_copy(Zs, Zg, (long long)n * K);
          Zk = Zs;
        }
        const double* Wb = w.Hh + (long long)K * b;
        for (int i = tid; i < K; i += blockDim.x) ys[i] = Wb[i];
        __syncthreads();
        const double lam_old = a.lam[b];
        double* col = a.X[k] + (long long)n * b;
        double num = 0.0, den = 0.0, nrm2 = 0.0;
        for (int row = tid; row < n; row += blockDim.x) {
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int i = 0;
          for (; i + 3 < K; i += 4) {
            s0 = fma(Zk[row + (long long)n * i], ys[i], s0);
            s1 = fma(Zk[row + (long long)n * (i + 1)], ys[i + 1], s1);
            s2 = fma(Zk[row + (long long)n * (i + 2)], ys[i + 2], s2);
            s3 = fma(Zk[row + (long long)n * (i + 3)], ys[i + 3], s3);
          }
          for (; i < K; ++i) s0 = fma(Zk[row + (long long)n * i], ys[i], s0);
          const double v = (s0 + s1) + (s2 + s3);
          xs[row] = v;
          const double old = col[row] * (gs ? lam_old : 1.0);
          const double df = v - old;
          num = fma(df, df, num);
          den = fma(old, old, den);
          nrm2 = fma(v, v, nrm2);
        }
        for (int o = 16; o > 0; o >>= 1) {
          num += __shfl_xor_sync(0xffffffffu, num, o);
          den += __shfl_xor_sync(0xffffffffu, den, o);
          nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
        }
        __shared__ double r3[3][NT / 32];
        if ((tid & 31) == 0) { r3[0][tid >> 5] = num; r3[1][tid >> 5] = den; r3[2][tid >> 5] = nrm2; }
        __syncthreads();
        __shared__ double scol;
        if (tid == 0) {
          double tn = 0.0, td = 0.0, t2 = 0.0;
          for (int q = 0; q < NT / 32; ++q) { tn += r3[0][q]; td += r3[1][q]; t2 += r3[2][q]; }
          atomicAdd(&w.acc2[0], tn);
          atomicAdd(&w.acc2[1], td);
          const double nr = sqrt(t2);
          if (gs) a.lam[b] = nr;
          scol = htg_dpos_finite(nr) ? htg_rcp_fast(nr) : 1.0;
        }
        __syncthreads();
        if (gs) {
          for (int row = tid; row < n; row += blockDim.x) {
            const double v = xs[row] * scol;
            xs[row] = v;
            col[row] = v;
          }
          __syncthreads();
          // M_k[:, b] = Z_k^T X_k[:, b]
          for (int o = tid; o < K; o += blockDim.x) {
            const double* zc = Zk + (long long)n * o;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int q = 0;
            for (; q + 3 < n; q += 4) {
              s0 = fma(zc[q], xs[q], s0);
              s1 = fma(zc[q + 1], xs[q + 1], s1);
              s2 = fma(zc[q + 2], xs[q + 2], s2);
              s3 = fma(zc[q + 3], xs[q + 3], s3);
            }
            for (; q < n; ++q) s0 = fma(zc[q], xs[q], s0);
            w.H[(long long)k * w.rycap * w.rcap + o + (long long)K * b] = (s0 + s1) + (s2 + s3);
          }
        } else {
          double* dst = w.Xold + (long long)k * nmax * w.rcap + (long long)n * b;
          for (int row = tid; row < n; row += blockDim.x) dst[row] = xs[row];
        }
        __syncthreads();
      }
      if (!grid_barrier(w.bar, nb, err)) return;
      // ---------------- C: column b of G_k = X_k^T X_k (all columns of X_k are final)
      if (gs && b < r) {
        const int n = a.n[k];
        stage_copy(Xs, a.X[k], (long long)n * r);
        __syncthreads();
        const double* xb = Xs + (long long)n * b;
        for (int o = tid; o < r; o += blockDim.x) {
          const double* xo = Xs + (long long)n * o;
          double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
          int q = 0;
          for (; q + 3 < n; q += 4) {
            s0 = fma(xo[q], xb[q], s0);
            s1 = fma(xo[q + 1], xb[q + 1], s1);
            s2 = fma(xo[q + 2], xb[q + 2], s2);
            s3 = fma(xo[q + 3], xb[q + 3], s3);
          }
          for (; q < n; ++q) s0 = fma(xo[q], xb[q], s0);
          w.G[(long long)k * w.rcap * w.rcap + o + (long long)r * b] = (s0 + s1) + (s2 + s3);
        }
        __syncthreads();
      }
      if (gs && !grid_barrier(w.bar, nb, err)) return;
    }
    if (!gs) {
      // damped Jacobi update of every column b, then refresh all Grams
      if (b < r) {
        for (int k = 0; k < d; ++k) {
          const int n = a.n[k];
          const double* src = w.Xold + (long long)k * nmax * w.rcap + (long long)n * b;
          double* col = a.X[k] + (long long)n * b;
          for (int row = tid; row < n; row += blockDim.x) col[row] += 0.25 * (src[row] - col[row]);
        }
      }
      if (!grid_barrier(w.bar, nb, err)) return;
      if (b < r)
        for (int j = 0; j < d; ++j) gram_column(a, w, j, b, r0, true, xs, zs_smem ? Xs : nullptr);
      if (!grid_barrier(w.bar, nb, err)) return;
    }
  }
  // the last mode's measure
  if (b == 0 && tid == 0 && sweeps > 0) {
    const double tn = w.acc2[0], td = w.acc2[1];
    const double ek = htg_dpos_finite(td) ? sqrt(tn / td) : sqrt(tn);
    if (htg_dgt_nn(ek, w.epsacc[sweeps - 1])) w.epsacc[sweeps - 1] = ek;
  }
  if (!gs && b < r) normalise_column(a, b, false, red);
}

// dynamic shared memory of cp_solve_kernel: L (r x r), norms (r), staged rows (n x r)
static cudaError_t solve_smem_for(int r, const int* n, int d, size_t* out) {
  int nmax = 1;
  for (int k = 0; k < d; ++k) nmax = htg_max(nmax, n[k]);
  const size_t sm = ((size_t)r * r + r + (size_t)nmax * r) * sizeof(double);
  *out = sm;
  if (sm > 48 * 1024) return cudaFuncSetAttribute(cp_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  return cudaSuccess;
}

}  // namespace

extern "C" int cp_apply_rk2(ht_ctx* c, const cp_tensor* x, const ht_op* L, double dt, cp_tensor* y, void* stream) {
  if (!c || !x || !y || !L) return HT_ERR_ARG;
  const int d = htg_ctx_d(c);
  if (x->d != d || y->d != d || L->d != d || !L->kron_sum || L->n_terms != d || x->rank < 1) return HT_ERR_ARG;
  const int nt = htg_cp_terms(d);
  if ((long long)x->rank * nt > y->cap || x->rank > x->cap) return HT_ERR_CAPACITY;
  StencilArgs a;
  memset(&a, 0, sizeof(a));
  a.d = d; a.r = x->rank; a.nt = nt;
  int nmax = 1;
  for (int k = 0; k < d; ++k) {
    if (x->n[k] != y->n[k] || !x->factor[k] || !y->factor[k]) return HT_ERR_ARG;
    const ht_factor& f = L->f[k][k];
    if (f.kind != HT_F_STENCIL || 2 * f.half_width + 1 > HT_MAXSTENCIL) return HT_ERR_ARG;
    a.n[k] = x->n[k];
    a.hw[k] = f.half_width;
    for (int j = 0; j < 2 * f.half_width + 1; ++j) a.c[k][j] = dt * L->alpha[k] * f.stencil[j];
    a.X[k] = x->factor[k];
    a.Y[k] = y->factor[k];
    nmax = htg_max(nmax, x->n[k]);
  }
  a.w = x->weight;
  a.wy = y->weight;
  cudaStream_t s = (cudaStream_t)stream;
  htg_prof_begin(c, s);
  cp_apply_kernel<<<dim3(x->rank, d), 128, 3 * nmax * sizeof(double), s>>>(a);
  htg_prof_end(c, KC_APPLY, s);
  htg_ctx_count(c, 1, s);
  if (cudaGetLastError() != cudaSuccess) return HT_ERR_CUDA;
  y->rank = x->rank * nt;
  return HT_OK;
}

extern "C" int cp_als_sweep(ht_ctx* c, const cp_tensor* y, cp_tensor* x, int sweeps, int variant, double* eps_dev,
                            void* stream) {
  if (!c || !x || !y || sweeps < 0 || sweeps > 64) return HT_ERR_ARG;
  if (variant != CP_ALS_GS && variant != CP_ALS_JACOBI_DAMPED) return HT_ERR_ARG;
  const int d = htg_ctx_d(c);
  CpWs* w = htg_ctx_cp(c);
  if (x->d != d || y->d != d || x->rank < 1 || y->rank < 1 || !x->weight || !y->weight) return HT_ERR_ARG;
  if (x->rank > w->rcap || y->rank > w->rycap || x->rank > x->cap || y->rank > y->cap || x->rank > 64)
    return HT_ERR_CAPACITY;
  CpArgs a;
  memset(&a, 0, sizeof(a));
  a.d = d; a.r = x->rank; a.ry = y->rank; a.variant = variant;
  for (int k = 0; k < d; ++k) {
    if (x->n[k] != y->n[k] || x->n[k] != htg_ctx_n(c)[k] || !x->factor[k] || !y->factor[k]) return HT_ERR_ARG;
    a.n[k] = x->n[k];
    a.X[k] = x->factor[k];
    a.Y[k] = y->factor[k];
  }
  a.mu = y->weight;
  a.lam = x->weight;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = htg_ctx_grid(c);
  int launches = 0;
#define CPL(cls, expr)                                         \
  do {                                                         \
    htg_prof_begin(c, s);                                      \
    expr;                                                      \
    htg_prof_end(c, (cls), s);                                 \
    ++launches;                                                \
    if (cudaGetLastError() != cudaSuccess) {                   \
      htg_ctx_count(c, launches, s);                           \
      return HT_ERR_CUDA;                                      \
    }                                                          \
  } while (0)
#define CPG(descs, nd)                                                                    \
  do {                                                                                    \
    htg_prof_begin(c, s);                                                                 \
    cudaError_t _e = htg_launch_gemm((descs), (nd), grid, s, htg_prof_flops(c, KC_GEMM)); \
    htg_prof_end(c, KC_GEMM, s);                                                          \
    ++launches;                                                                           \
    if (_e != cudaSuccess) {                                                              \
      htg_ctx_count(c, launches, s);                                                      \
      return HT_ERR_CUDA;                                                                 \
    }                                                                                     \
  } while (0)
  const int fold = (variant == CP_ALS_JACOBI_DAMPED) ? 1 : 0;
  CPL(KC_CPSMALL, (cp_eps_init_kernel<<<1, 64, 0, s>>>(*w, sweeps)));
  CPL(KC_CPSMALL, (cp_plan_kernel<<<1, 1, 0, s>>>(a, *w)));
  CPL(KC_CPSMALL, (cp_normalize_kernel<<<1, NT, 0, s>>>(a, fold)));
  // all G_k, H_k: descriptors 1,2 of every mode; launch each mode's pair (small)
  for (int k = 0; k < d; ++k) {
    CPG(w->descs + 3 * k + 1, 2);
  }
  size_t solve_smem = 0;
  if (solve_smem_for(a.r, a.n, d, &solve_smem) != cudaSuccess) return HT_ERR_CUDA;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int k = 0; k < d; ++k) {
      CPL(KC_CPSMALL, (cp_hadamard_kernel<<<32, NT, 0, s>>>(a, *w, k)));
      CPG(w->descs + 3 * k, 1);
      CPL(KC_CPSOLVE, (cp_solve_kernel<<<1, NT, solve_smem, s>>>(a, *w, k, sw, htg_ctx_err(c), htg_prof_flops(c, KC_CPSOLVE))));
      if (variant == CP_ALS_GS) CPG(w->descs + 3 * k + 1, 2);
    }
    if (variant == CP_ALS_JACOBI_DAMPED) {
      CPL(KC_CPSMALL, (cp_damp_kernel<<<dim3(8, d), NT, 0, s>>>(a, *w)));
      for (int k = 0; k < d; ++k) CPG(w->descs + 3 * k + 1, 2);
    }
  }
  if (variant == CP_ALS_JACOBI_DAMPED) CPL(KC_CPSMALL, (cp_normalize_kernel<<<1, NT, 0, s>>>(a, 0)));
  if (eps_dev && sweeps > 0) CPL(KC_CPSMALL, (cp_eps_out_kernel<<<1, 64, 0, s>>>(*w, sweeps, eps_dev)));
#undef CPL
#undef CPG
  htg_ctx_count(c, launches, s);
  return HT_OK;
}

extern "C" int cp_als_sweep_rk2(ht_ctx* c, const cp_tensor* x_old, const ht_op* L, double dt, cp_tensor* x,
                                int sweeps, int variant, double* eps_dev, void* stream) {
  if (!c || !x || !x_old || !L || sweeps < 0 || sweeps > 64) return HT_ERR_ARG;
  if (variant != CP_ALS_GS && variant != CP_ALS_JACOBI_DAMPED) return HT_ERR_ARG;
  const int d = htg_ctx_d(c);
  CpWs* w = htg_ctx_cp(c);
  if (x->d != d || x_old->d != d || L->d != d || !L->kron_sum || L->n_terms != d) return HT_ERR_ARG;
  if (x->rank < 1 || x_old->rank < 1 || !x->weight || !x_old->weight) return HT_ERR_ARG;
  if (x->rank > w->rcap || x_old->rank > w->rcap || 3 * x_old->rank > w->rycap || x->rank > x->cap ||
      x_old->rank > x_old->cap || x->rank > 64)
    return HT_ERR_CAPACITY;
  CpArgs a;
  memset(&a, 0, sizeof(a));
  PowArgs pa;
  memset(&pa, 0, sizeof(pa));
  a.d = d; a.r = x->rank; a.ry = 3 * x_old->rank; a.variant = variant;
  pa.d = d; pa.r0 = x_old->rank;
  int nmax = 1;
  for (int k = 0; k < d; ++k) {
    if (x->n[k] != x_old->n[k] || x->n[k] != htg_ctx_n(c)[k] || !x->factor[k] || !x_old->factor[k]) return HT_ERR_ARG;
    const ht_factor& f = L->f[k][k];
    if (f.kind != HT_F_STENCIL || 2 * f.half_width + 1 > HT_MAXSTENCIL) return HT_ERR_ARG;
    a.n[k] = x->n[k];
    a.X[k] = x->factor[k];
    pa.n[k] = x->n[k];
    pa.hw[k] = f.half_width;
    for (int j = 0; j < 2 * f.half_width + 1; ++j) pa.c[k][j] = dt * L->alpha[k] * f.stencil[j];
    pa.X[k] = x_old->factor[k];
    nmax = htg_max(nmax, x->n[k]);
  }
  a.lam = x->weight;
  a.mu = w->wold;
  const int r0 = x_old->rank;
  cudaStream_t s = (cudaStream_t)stream;
  (void)nmax;
  // one cooperative launch: CTA b owns factor column b (and row b of the solve)
  const int nblk = htg_max(a.r, r0);
  const size_t rr = (size_t)a.r, nm = (size_t)w->nmax;
  const size_t ntypes = (size_t)htg_cp_terms(d);
  size_t smem = (rr * rr + 4 * rr + 2 * nm + 3 * (size_t)d * rr + (nm > ntypes ? nm : ntypes) * rr) * sizeof(double);
  const size_t zbytes = nm * 3 * (size_t)r0 * sizeof(double);
  const int zs_smem = (smem + zbytes <= 160 * 1024) ? 1 : 0;   // stage Z_k in shared memory when it fits
  if (zs_smem) smem += zbytes;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(cp_als_rk2_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return HT_ERR_CUDA;
  }
  int launches = 0;
  htg_prof_begin(c, s);
  cudaError_t e0 = cudaMemsetAsync(w->bar, 0, 2 * sizeof(unsigned int), s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblk);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e1 = cudaLaunchKernelEx(&cfg, cp_als_rk2_persistent, a, pa, *w, (const double*)x_old->weight, sweeps,
                                      htg_ctx_err(c), zs_smem);
  htg_prof_end(c, KC_CPSOLVE, s);
  ++launches;
  if (e0 != cudaSuccess || e1 != cudaSuccess) {
    htg_ctx_count(c, launches, s);
    return HT_ERR_CUDA;
  }
  if (eps_dev && sweeps > 0) {
    cp_eps_out_kernel<<<1, 64, 0, s>>>(*w, sweeps, eps_dev);
    ++launches;
    if (cudaGetLastError() != cudaSuccess) {
      htg_ctx_count(c, launches, s);
      return HT_ERR_CUDA;
    }
  }
  htg_ctx_count(c, launches, s);
  return HT_OK;
}

// ============================================================================
// Allocation-free variant of cp_als_sweep.
//
// Some callers cannot allocate device memory at all: code that runs inside a host
// callback or a driver-managed plug-in with a fixed memory budget, processes whose GPU
// memory is fully reserved up front by another framework, or environments where
// cudaMalloc is forbidden after initialisation.  cp_als_sweep_noalloc serves them: it
// needs no ht_ctx and calls no allocator.  Its scratch (Grams, right-hand sides,
// descriptors, the error word) lives in one file-scope __device__ array of fixed size
// that every GPU loading this library holds until the process exits.
//
// Limits: d <= 8, n_k <= 256, x rank <= 32, y rank <= 1024 (about 3.0 MB of scratch).
// The array is shared by every call: calls whose work overlaps on the GPU (two streams,
// two host threads) race on it and must be serialised by the caller.  The first call
// on a device looks up the array's device address (cudaGetSymbolAddress) with that
// device current; make that first call before any stream capture.
// ============================================================================
#include <mutex>

namespace {

constexpr int NA_MAXD = 8, NA_MAXN = 256, NA_MAXR = 32, NA_MAXRY = 1024;
constexpr size_t NA_G = (size_t)NA_MAXD * NA_MAXR * NA_MAXR;
constexpr size_t NA_H = (size_t)NA_MAXD * NA_MAXRY * NA_MAXR;
constexpr size_t NA_HH = (size_t)NA_MAXRY * NA_MAXR;
constexpr size_t NA_GAM = (size_t)NA_MAXR * NA_MAXR;
constexpr size_t NA_RHS = (size_t)NA_MAXN * NA_MAXR;
constexpr size_t NA_XOLD = (size_t)NA_MAXD * NA_MAXN * NA_MAXR;
constexpr size_t NA_WOLD = NA_MAXR;
constexpr size_t NA_EPS = 64;
constexpr size_t NA_DESC = (4 * HT_MAXD * sizeof(GemmDesc) + sizeof(double) - 1) / sizeof(double);
constexpr size_t NA_ERR = 4;
constexpr size_t NA_TOTAL = NA_G + NA_H + NA_HH + NA_GAM + NA_RHS + NA_XOLD + NA_WOLD + NA_EPS + NA_DESC + NA_ERR;

__device__ __align__(256) double g_cp_noalloc_scratch[NA_TOTAL];

__global__ void na_status_kernel(const int* err, int* out) {
  if (threadIdx.x == 0) *out = *err;
}

struct NaDevice {
  double* base = nullptr;
  int grid = 0;
  bool ready = false;
};
NaDevice g_na_dev[64];
std::mutex g_na_mutex;

}  // namespace

extern "C" int cp_als_sweep_noalloc(const cp_tensor* y, cp_tensor* x, int sweeps, int variant, double* eps_dev,
                                    int* status_dev, void* stream) {
  if (!x || !y || sweeps < 0 || sweeps > 64) return HT_ERR_ARG;
  if (variant != CP_ALS_GS && variant != CP_ALS_JACOBI_DAMPED) return HT_ERR_ARG;
  const int d = x->d;
  if (d < 2 || d > HT_MAXD || y->d != d || x->rank < 1 || y->rank < 1 || !x->weight || !y->weight)
    return HT_ERR_ARG;
  if (x->rank > x->cap || y->rank > y->cap) return HT_ERR_CAPACITY;
  if (d > NA_MAXD || x->rank > NA_MAXR || y->rank > NA_MAXRY) return HT_ERR_CAPACITY;
  for (int k = 0; k < d; ++k) {
    if (x->n[k] != y->n[k] || x->n[k] < 1 || !x->factor[k] || !y->factor[k]) return HT_ERR_ARG;
    if (x->n[k] > NA_MAXN) return HT_ERR_CAPACITY;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HT_ERR_CUDA;
  NaDevice* nd = &g_na_dev[dev];
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!nd->ready) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_cp_noalloc_scratch) != cudaSuccess || p == nullptr) return HT_ERR_CUDA;
      int sms = 0;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HT_ERR_CUDA;
      nd->base = (double*)p;
      nd->grid = htg_max(1, sms) * 4;
      nd->ready = true;
    }
  }
  double* b = nd->base;
  CpWs w;
  w.G = b; b += NA_G;
  w.H = b; b += NA_H;
  w.Hh = b; b += NA_HH;
  w.Gam = b; b += NA_GAM;
  w.RHS = b; b += NA_RHS;
  w.Xold = b; b += NA_XOLD;
  w.wold = b; b += NA_WOLD;
  w.epsacc = b; b += NA_EPS;
  w.descs = (GemmDesc*)b; b += NA_DESC;
  int* err = (int*)b;
  w.Z = nullptr;
  w.acc2 = nullptr;
  w.bar = nullptr;
  w.rcap = NA_MAXR;
  w.rycap = NA_MAXRY;
  w.nmax = NA_MAXN;

  CpArgs a;
  memset(&a, 0, sizeof(a));
  a.d = d; a.r = x->rank; a.ry = y->rank; a.variant = variant;
  for (int k = 0; k < d; ++k) {
    a.n[k] = x->n[k];
    a.X[k] = x->factor[k];
    a.Y[k] = y->factor[k];
  }
  a.mu = y->weight;
  a.lam = x->weight;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = nd->grid;
  // the error word starts at zero on every call; everything else is written before it is read
  if (cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) return HT_ERR_CUDA;
#define NAL(expr)                                                  \
  do {                                                             \
    expr;                                                          \
    if (cudaGetLastError() != cudaSuccess) return HT_ERR_CUDA;     \
  } while (0)
  const int fold = (variant == CP_ALS_JACOBI_DAMPED) ? 1 : 0;
  NAL((cp_eps_init_kernel<<<1, 64, 0, s>>>(w, sweeps)));
  NAL((cp_plan_kernel<<<1, 1, 0, s>>>(a, w)));
  NAL((cp_normalize_kernel<<<1, NT, 0, s>>>(a, fold)));
  for (int k = 0; k < d; ++k)
    if (htg_launch_gemm(w.descs + 3 * k + 1, 2, grid, s) != cudaSuccess) return HT_ERR_CUDA;
  size_t solve_smem = 0;
  if (solve_smem_for(a.r, a.n, d, &solve_smem) != cudaSuccess) return HT_ERR_CUDA;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int k = 0; k < d; ++k) {
      NAL((cp_hadamard_kernel<<<32, NT, 0, s>>>(a, w, k)));
      if (htg_launch_gemm(w.descs + 3 * k, 1, grid, s) != cudaSuccess) return HT_ERR_CUDA;
      NAL((cp_solve_kernel<<<1, NT, solve_smem, s>>>(a, w, k, sw, err, nullptr)));
      if (variant == CP_ALS_GS && htg_launch_gemm(w.descs + 3 * k + 1, 2, grid, s) != cudaSuccess)
        return HT_ERR_CUDA;
    }
    if (variant == CP_ALS_JACOBI_DAMPED) {
      NAL((cp_damp_kernel<<<dim3(8, d), NT, 0, s>>>(a, w)));
      for (int k = 0; k < d; ++k)
        if (htg_launch_gemm(w.descs + 3 * k + 1, 2, grid, s) != cudaSuccess) return HT_ERR_CUDA;
    }
  }
  if (variant == CP_ALS_JACOBI_DAMPED) NAL((cp_normalize_kernel<<<1, NT, 0, s>>>(a, 0)));
  if (eps_dev && sweeps > 0) NAL((cp_eps_out_kernel<<<1, 64, 0, s>>>(w, sweeps, eps_dev)));
  if (status_dev) NAL((na_status_kernel<<<1, 32, 0, s>>>(err, status_dev)));
#undef NAL
  return HT_OK;
}
