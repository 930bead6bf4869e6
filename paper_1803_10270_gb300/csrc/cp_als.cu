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
#include <cooperative_groups.h>
#include <cstring>

#include "common.cuh"

namespace cg = cooperative_groups;

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
constexpr int MODE_MAXD = 16;   // largest d of the structured ALS (unrolled Gram loads)

struct PowArgs {
  int d, r0;
  int n[HT_MAXD];
  int hw[HT_MAXD];
  double c[HT_MAXD][HT_MAXSTENCIL];
  const double* X[HT_MAXD];
};

// ---------------------------------------------------------------------------
// Persistent form of cp_als_sweep_rk2: one cooperative launch runs every sweep.  CTA b owns
// factor column b (row b of the r0 x r blocks in the solve phase); phases are separated by
// a grid barrier:
//   0a  powers Z_j^(p) of x_old (CTA b < r0), mu <- weights of x_old, normalise column b of x
//   0b  column b of G_j = X_j^T X_j and M_j = Z_j^T X_j for every j
//   per mode k:  A  Gamma_k (LDL^T) and row b of W = Hs Gamma_k^-1; CTA 0 records the
//                   previous mode's convergence measure                      (CTA b < r0)
//                B  column b of X~_k = Z_k W, convergence sums, X_k[:, b], lam_b and M_k[:, b]
//                C  column b of G_k
// The launch is cooperative (all CTAs resident), and every barrier wait is bounded: past the
// limit the kernel records HT_ERR_TIMEOUT in the error word and returns.
// ---------------------------------------------------------------------------
constexpr long long BARRIER_TIMEOUT_CYCLES = 400000000LL;   // about 0.2 s

// Grid barrier by per-CTA arrival words: CTA b publishes the barrier's sequence number seq in
// flags[b] (no atomics); warp 0 of every CTA polls all words, one lane each, until every one has
// reached seq.  Sequence numbers grow by one per barrier of the launch; the words are zeroed
// before the launch.  The wait is bounded: past the limit the kernel records HT_ERR_TIMEOUT and
// every barrier after it returns false.
__device__ bool grid_barrier(unsigned int* flags, unsigned int nblocks, unsigned int seq, int* err) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      __threadfence();
      *(volatile unsigned int*)(flags + blockIdx.x) = seq;
    }
    __syncwarp();
    int ok = 1;
    const long long t0 = clock64();
    for (unsigned int i = threadIdx.x; i < nblocks && ok; i += 32) {
      while (*(volatile unsigned int*)(flags + i) < seq) {
        if (clock64() - t0 > BARRIER_TIMEOUT_CYCLES) {
          ok = 0;
          break;
        }
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && threadIdx.x == 0 && err) atomicCAS(err, 0, (int)HT_ERR_TIMEOUT);
    __threadfence();
    if (threadIdx.x == 0) ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// Odd leading dimension for a staged n-row matrix: lanes that walk its columns (stride ld)
// then hit distinct shared-memory banks with their 8-byte words.
__device__ inline int odd_ld(int n) { return n | 1; }

// Copy an n x cols column-major matrix (leading dimension lds) to dst (leading dimension ldd),
// 8 independent loads in flight per thread (a plain copy loop waits out the full L2 latency on
// every element).  Plain (coherent) loads: the sources are written by other CTAs of the same
// launch before a grid barrier.
__device__ void stage_pad(double* dst, int ldd, const double* src, int lds, int n, int cols) {
  const unsigned int total = (unsigned int)n * (unsigned int)cols, un = (unsigned int)n;
  const unsigned int T = blockDim.x;
  unsigned int base = 0;
  for (; base + 8u * T <= total; base += 8u * T) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const unsigned int e = base + u * T + threadIdx.x;
      v[u] = src[(e % un) + (long long)lds * (e / un)];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const unsigned int e = base + u * T + threadIdx.x;
      dst[(e % un) + (long long)ldd * (e / un)] = v[u];
    }
  }
  for (unsigned int e = base + threadIdx.x; e < total; e += T)
    dst[(e % un) + (long long)ldd * (e / un)] = src[(e % un) + (long long)lds * (e / un)];
}

// The same copy by asynchronous 8-byte copies (all in flight at once, no register staging);
// row and column advance incrementally (no divisions).  Every thread must call stage_wait()
// before the CTA barrier that publishes dst.  Reads through L1 are safe here: the grid barrier
// ends with a device-scope fence on every SM before anything staged is read.
__device__ void stage_pad_async(double* dst, int ldd, const double* src, int lds, int n, int cols) {
  const int T = blockDim.x;
  int row = threadIdx.x % n, col = threadIdx.x / n;
  const int dr = T % n, dc = T / n;
  while (col < cols) {
    const unsigned int d = (unsigned int)__cvta_generic_to_shared(dst + row + (long long)ldd * col);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src + row + (long long)lds * col) : "memory");
    row += dr;
    col += dc;
    if (row >= n) {
      row -= n;
      ++col;
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ inline void stage_async1(double* dst, const double* src) {
  const unsigned int d = (unsigned int)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ inline void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Parts per output of a split dot product: as many as fill the CTA, at most 8.
__device__ inline int dot_parts(int nout) { return (nout <= NT) ? htg_max(1, htg_min(NT / htg_max(nout, 1), 8)) : 1; }

// out_o = col(o) . x (length n) for o < nout: consecutive lanes take consecutive outputs, each
// output is split into P chunks whose partial sums (pb, nout * P <= max(NT, nout) values) are
// added in chunk order; store(o, value) receives the result.  Two CTA barriers.
template <class Col, class Store>
__device__ void cols_dot(Col col, const double* x, int n, int nout, double* pb, Store store) {
  const int P = dot_parts(nout);
  const int chunk = (n + P - 1) / P;
  for (int e = threadIdx.x; e < nout * P; e += NT) {
    const int o = e % nout, part = e / nout;
    const int q0 = part * chunk, q1 = htg_min(n, q0 + chunk);
    const double* src = col(o);
    double s0 = 0.0, s1 = 0.0;
    int q = q0;
    for (; q + 1 < q1; q += 2) {
      s0 = fma(src[q], x[q], s0);
      s1 = fma(src[q + 1], x[q + 1], s1);
    }
    if (q < q1) s0 = fma(src[q], x[q], s0);
    pb[e] = s0 + s1;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < nout; o += NT) {
    double v = pb[o];
    for (int part = 1; part < P; ++part) v += pb[o + nout * part];
    store(o, v);
  }
  __syncthreads();
}

// out[row] = sum_i S[row + ld i] y[i] for row < n, i < m: consecutive lanes take consecutive
// rows, P chunks of the m terms per row, partial sums added in chunk order.  Two CTA barriers.
__device__ void rows_dot(const double* S, int ld, const double* y, int n, int m, double* pb, double* out) {
  const int P = dot_parts(n);
  const int chunk = (m + P - 1) / P;
  for (int e = threadIdx.x; e < n * P; e += NT) {
    const int row = e % n, part = e / n;
    const int i0 = part * chunk, i1 = htg_min(m, i0 + chunk);
    double s0 = 0.0, s1 = 0.0;
    int i = i0;
    for (; i + 1 < i1; i += 2) {
      s0 = fma(S[row + (long long)ld * i], y[i], s0);
      s1 = fma(S[row + (long long)ld * (i + 1)], y[i + 1], s1);
    }
    if (i < i1) s0 = fma(S[row + (long long)ld * i], y[i], s0);
    pb[e] = s0 + s1;
  }
  __syncthreads();
  for (int row = threadIdx.x; row < n; row += NT) {
    double v = pb[row];
    for (int part = 1; part < P; ++part) v += pb[row + n * part];
    out[row] = v;
  }
  __syncthreads();
}

// column b of G_j (r values) and, when withM, of M_j (3 r0 values); X_j[:, b] staged in xs.
// With stage, [X_j | Z_j] is copied to shared memory with an odd leading dimension first.
__device__ void gram_column(const CpArgs& a, CpWs& w, int j, int b, int r0, bool withM, double* xs, double* pb,
                            double* stage) {
  const int n = a.n[j], r = a.r, K = 3 * r0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = a.X[j][i + (long long)n * b];
  const double* Zj = w.Z + (long long)j * w.nmax * 3 * w.rcap;
  const double* Xsrc = a.X[j];
  const double* Zsrc = Zj;
  int ld = n;
  if (stage) {
    ld = odd_ld(n);
    stage_pad_async(stage, ld, a.X[j], n, n, r);
    if (withM) stage_pad_async(stage + (long long)ld * r, ld, Zj, n, n, K);
    stage_wait();
    Xsrc = stage;
    Zsrc = stage + (long long)ld * r;
  }
  __syncthreads();
  double* Gc = w.G + (long long)j * w.rcap * w.rcap + (long long)r * b;
  double* Hc = w.H + (long long)j * w.rycap * w.rcap + (long long)K * b;
  cols_dot([&](int o) { return (o < r) ? Xsrc + (long long)ld * o : Zsrc + (long long)ld * (o - r); }, xs, n,
           r + (withM ? K : 0), pb, [&](int o, double v) {
             if (o < r) Gc[o] = v;
             else Hc[o - r] = v;
           });
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

// Right-hand sides of row lp for mode k, one per power p of A_k, from the products
// m_p,j = M_j^(p)[lp, l] staged in Mv.  The column types of y = p(dt L) x_old are the monomials
// of p(z_1 + ... + z_d), p(z) = 1 + z + z^2 / 2, each with coefficient 1 / alpha!; grouped by
// the power of z_k they read p(z_k + s) = (1 + s + s^2/2) + z_k (1 + s) + z_k^2 / 2 with
// s = sum_{j != k} z_j.  The truncated product f(e) = prod_{j != k} (m_0,j + m_1,j e + m_2,j e^2 / 2)
// mod e^3 = f0 + f1 e + f2 e^2 holds the degree sums, so
//   hs_0 = mu (f0 + f1 + f2),   hs_1 = mu (f0 + f1),   hs_2 = mu f0 / 2.
__device__ void rk2_rhs_row(const double* Mv, int d, int k, int r, double mu, double* hs, int t0, int nthr) {
  for (int l = t0; l < r; l += nthr) {
    double f0 = 1.0, f1 = 0.0, f2 = 0.0;
    for (int j = 0; j < d; ++j) {
      if (j == k) continue;
      const double m0 = Mv[(j * 3) * r + l], m1 = Mv[(j * 3 + 1) * r + l];
      const double m2h = 0.5 * Mv[(j * 3 + 2) * r + l];
      f2 = fma(f2, m0, fma(f1, m1, f0 * m2h));
      f1 = fma(f1, m0, f0 * m1);
      f0 *= m0;
    }
    hs[l] = mu * ((f0 + f1) + f2);
    hs[r + l] = mu * (f0 + f1);
    hs[2 * r + l] = 0.5 * mu * f0;
  }
}

constexpr int TRI_MAX = 64 * 65 / 2;   // lower-triangle pairs of the largest rank (64)

// offset of column c in the column-ordered lower-triangle pair list of an r x r matrix
__device__ inline int tri_offset(int c, int r) { return c * r - (c * (c - 1)) / 2; }

// LDL^T factorisation (D diagonal, L unit lower) of the SPD r x r matrix in Lm (column-major,
// lower part) with the unit-lower forward solve of the nrhs right-hand sides in hs (vector v at
// hs + v r) fused in.
// Right-looking, two CTA barriers per pivot.  Step j first forms the multipliers L_ij = a_ij / d_j
// of column j once (into Lsc), then applies a_ic -= L_ij a_cj to the trailing lower triangle
// (pairs from tri, i >= c > j) and z_i -= L_ij z_j to the right-hand sides, one FMA per element.
// Meanwhile one thread of the last warp forms the next pivot a_{j+1,j+1} and its reciprocal, and
// the warps on that warp's SM partition (warp index 3 mod 4) take no element work: the pivot
// chain (an FMA, the reciprocal's seed and its correction) never waits behind other warps' FP64
// instructions.  Measured per step (clock64 in CTA 0 at the bench configuration): the pivot
// chain about 650 cycles after the multipliers' barrier, the element threads 300-700; variants
// measured slower: the multiplier formed per element (one product more per element), the pivot
// chain started beside the multipliers behind a named barrier, a division-free scaled
// elimination (no reciprocal on the chain, but a product more per element) with and without the
// trailing entries held in registers, asynchronous copies issued by the element threads during the
// steps, and a look-ahead of the next pivot's entries on the pivot thread.  Column j keeps
// a_ij = L_ij d_j.  A pivot that is not positive and finite leaves dinv = 0 there; every thread
// sees it after the barrier and the result is false.
__device__ bool ldlt_forward(double* Lm, double* Lsc, double* hs, double* dinv, const unsigned short* tri, int r,
                             int nrhs) {
  const int tid = threadIdx.x, wid = tid >> 5;
  constexpr int PIV = NT - 32;              // the pivot thread: lane 0 of the last warp
  constexpr int NE = (NT / 32) * 3 / 4 * 32;   // element threads: the warps with wid % 4 != 3
  const int et = (wid % 4 != 3) ? (wid - wid / 4) * 32 + (tid & 31) : -1;
  if (tid == 0) {
    const double d0 = Lm[0];
    dinv[0] = htg_dpos_finite(d0) ? htg_rcp_fast(d0) : 0.0;
  }
  __syncthreads();
  const int T = r * (r + 1) / 2;
  for (int j = 0; j < r; ++j) {
    const double dj = dinv[j];
    if (!htg_dnz(dj)) return false;   // uniform: written before the last barrier
    const int m = r - 1 - j;
    for (int i = j + 1 + tid; i < r; i += NT) Lsc[i + r * j] = Lm[i + r * j] * dj;
    __syncthreads();
    const int s0 = tri_offset(j + 1, r) + 1;   // the pairs after (j+1, j+1)
    const int ntri = T - s0;
    const int nall = ntri + nrhs * m;
    if (et >= 0) {
      for (int e = et; e < nall; e += NE) {
        if (e < ntri) {
          const unsigned int pr = tri[s0 + e];
          const int i = pr & 0xff, c = pr >> 8;
          Lm[i + r * c] = fma(-Lsc[i + r * j], Lm[c + r * j], Lm[i + r * c]);
        } else {
          const int f = e - ntri, p = f / m, i = j + 1 + f % m;
          hs[p * r + i] = fma(-Lsc[i + r * j], hs[p * r + j], hs[p * r + i]);
        }
      }
    } else if (tid == PIV && m > 0) {
      const int i = j + 1;
      const double v = fma(-Lsc[i + r * j], Lm[i + r * j], Lm[i + r * i]);
      Lm[i + r * i] = v;
      dinv[i] = htg_dpos_finite(v) ? htg_rcp_fast(v) : 0.0;
    }
    __syncthreads();
  }
  return true;
}

// Back substitution D L^T w = z for the nrhs right-hand sides (z in hs, overwritten by w):
// w_i = z_i / d_i - sum_{c > i} L_ci w_c.  For r <= 32 warp p takes sides p, p + 8, ... with lane
// i holding w_i's running value and column i of L (from Lsc) in registers: no CTA barrier inside.
// Otherwise a CTA-wide substitution on the unscaled columns: w_i = (z_i - sum a_ci w_c) / d_i.
__device__ void ldlt_back(const double* Lm, const double* Lsc, double* hs, const double* dinv, int r, int nrhs) {
  const int tid = threadIdx.x;
  if (r <= 32) {
    const int lane = tid & 31;
    for (int wp = tid >> 5; wp < nrhs; wp += NT / 32) {
      double s = (lane < r) ? hs[wp * r + lane] * dinv[lane] : 0.0;
      double col[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) col[c] = (c < r && lane < c) ? Lsc[c + r * lane] : 0.0;
#pragma unroll
      for (int c = 31; c >= 0; --c) {
        if (c < r) {
          const double wc = __shfl_sync(0xffffffffu, s, c);
          if (lane < c) s = fma(-col[c], wc, s);
        }
      }
      if (lane < r) hs[wp * r + lane] = s;
    }
    __syncthreads();
    return;
  }
  for (int j = r - 1; j >= 0; --j) {
    if (tid < nrhs) hs[tid * r + j] *= dinv[j];
    __syncthreads();
    for (int e = tid; e < nrhs * j; e += NT) {
      const int p = e / j, i = e % j;
      hs[p * r + i] = fma(-Lm[j + r * i], hs[p * r + j], hs[p * r + i]);
    }
    __syncthreads();
  }
}

// Shared memory (doubles) of cp_als_rk2_persistent; the Z_k stage is optional.
__host__ __device__ inline long long persistent_smem_doubles(int r, int r0, int d, int nmax, bool with_z) {
  const long long ld = nmax | 1, K = 3LL * r0;
  const long long base = 2LL * r * r + 4LL * r + nmax + (nmax > K ? nmax : K) + 3LL * d * r +
                         (nmax > NT ? nmax : NT) + (long long)d * r * r + ld * r;
  return base + (with_z ? ld * K : 0);
}

__global__ void __launch_bounds__(NT) cp_als_rk2_persistent(CpArgs a, PowArgs pa, CpWs w, const double* mu_src,
                                                            int sweeps, int* err, int zs_smem, double* flops) {
  const int b = blockIdx.x, tid = threadIdx.x;
  const unsigned int nb = gridDim.x;
  const int d = a.d, r = a.r, r0 = pa.r0, K = 3 * r0;
  const int nmax = w.nmax;
  extern __shared__ double sh[];
  double* Lm = sh;                           // r x r: Gamma_k, then its LDL^T factor
  double* Lsc = Lm + r * r;                  // r x r: L of the LDL^T factorisation
  double* hs = Lsc + r * r;                  // 3 r: right-hand sides, then row lp of W
  double* dinv = hs + 3 * r;                 // r: reciprocal pivots
  double* xs = dinv + r;                     // nmax
  double* ys = xs + nmax;                    // max(nmax, 3 r0)
  double* Mv = ys + htg_max(nmax, K);        // d x 3 x r: copy of the M_j^(p) rows of this CTA's lp
  double* pb = Mv + 3 * d * r;               // max(NT, nmax): partial sums of split dot products
  double* Gs = pb + htg_max(NT, nmax);       // d x r x r: copy of the Grams G_j
  double* Xs = Gs + (long long)d * r * r;    // odd_ld(nmax) x r: a staged factor
  double* Zs = Xs + (long long)odd_ld(nmax) * r;   // odd_ld(nmax) x 3 r0: Z_k (when zs_smem)
  __shared__ unsigned short tri[TRI_MAX];
  __shared__ double red[HT_MAXD + 32];
  // lower-triangle pairs (i, c), i >= c, ordered by column then row
  for (int c = tid; c < r; c += blockDim.x) {
    const int o = tri_offset(c, r);
    for (int i = c; i < r; ++i) tri[o + i - c] = (unsigned short)(i | (c << 8));
  }
  const bool gs = (a.variant == CP_ALS_GS);
  unsigned int bseq = 0;   // sequence number of the last grid barrier
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
  if (!grid_barrier(w.bar, nb, ++bseq, err)) return;
  if (b < r) normalise_column(a, b, !gs, red);
  if (!grid_barrier(w.bar, nb, ++bseq, err)) return;
  // ---------------- 0b: column b of G_j and M_j for every j
  if (b < r)
    for (int j = 0; j < d; ++j) gram_column(a, w, j, b, r0, true, xs, pb, zs_smem ? Xs : nullptr);
  if (!grid_barrier(w.bar, nb, ++bseq, err)) return;
  const double* mu = w.wold;
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int k = 0; k < d; ++k) {
      const bool record = !(sweep == 0 && k == 0);  // the previous mode's sums are complete
      // ---------------- A: Gamma_k (LDL^T) and row lp = b of W = Hs Gamma_k^-1
      if (b < r0) {
        const int lp = b;
        // refresh the shared copies of G_j and of the rows lp of M_j^(p) that changed since
        // this CTA last read them: all at the start and after a damped Jacobi sweep, else those
        // of the mode updated last (Gauss-Seidel)
        int j0 = 0, j1 = 0;
        if (k == 0 && (sweep == 0 || !gs)) j1 = d;
        else if (gs) { j0 = (k + d - 1) % d; j1 = j0 + 1; }
        const int nG = r * r, nM = 3 * r;
        for (int j = j0; j < j1; ++j) {
          const double* Gg = w.G + (long long)j * w.rcap * w.rcap;
          const double* Hg = w.H + (long long)j * w.rycap * w.rcap + lp;
          for (int e = tid; e < nG + nM; e += blockDim.x) {
            if (e < nG) {
              stage_async1(Gs + j * nG + e, Gg + e);
            } else {
              const int f = e - nG, pp = f / r, l = f - pp * r;
              stage_async1(Mv + (j * 3 + pp) * r + l, Hg + pp * r0 + (long long)K * l);
            }
          }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        stage_wait();
        __syncthreads();
        // side by side: Gamma_k = hadamard_{j != k} G_j (warps with index != 3 mod 4 but the
        // last), the right-hand sides (the last warp), and in CTA 0 the convergence measure of
        // the previous mode (its sums are complete), recorded off the critical path (warp 3)
        const int wid = tid >> 5;
        if (wid == NT / 32 - 1) {
          rk2_rhs_row(Mv, d, k, r, mu[lp], hs, tid - (NT - 32), 32);
        } else if (wid % 4 != 3) {
          const int gt = (wid - wid / 4) * 32 + (tid & 31);
          for (int e = gt; e < nG; e += (NT / 32 - 2) * 32) {
            double v = 1.0;
            for (int j = 0; j < d; ++j)
              if (j != k) v *= Gs[j * nG + e];
            Lm[e] = v;
          }
        } else if (b == 0 && tid == 96) {
          if (record) {
            const double tn = w.acc2[0], td = w.acc2[1];
            const double ek = htg_dpos_finite(td) ? sqrt(tn / td) : sqrt(tn);
            const int sw = (k == 0) ? sweep - 1 : sweep;
            if (htg_dgt_nn(ek, w.epsacc[sw])) w.epsacc[sw] = ek;
          }
          w.acc2[0] = 0.0;
          w.acc2[1] = 0.0;
        }
        __syncthreads();
        bool ok = ldlt_forward(Lm, Lsc, hs, dinv, tri, r, 3);
        if (!ok) {
          // shift by 1e-14 tr(Gamma)/r, only after a failed factorisation (Section 2.1
          // regularisation of ill-conditioned ALS systems), and start over
          __shared__ double shift;
          if (tid == 0) {
            double tr = 0.0;
            for (int i = 0; i < r; ++i) {
              double v = 1.0;
              for (int j = 0; j < d; ++j)
                if (j != k) v *= Gs[j * nG + i + r * i];
              tr += v;
            }
            shift = 1e-14 * tr / r;
          }
          __syncthreads();
          for (int e = tid; e < nG; e += blockDim.x) {
            double v = 1.0;
            for (int j = 0; j < d; ++j)
              if (j != k) v *= Gs[j * nG + e];
            Lm[e] = v + ((e % r == e / r) ? shift : 0.0);
          }
          rk2_rhs_row(Mv, d, k, r, mu[lp], hs, tid, blockDim.x);
          __syncthreads();
          ok = ldlt_forward(Lm, Lsc, hs, dinv, tri, r, 3);
        }
        if (!ok) {
          if (tid == 0 && err) atomicCAS(err, 0, (int)HT_ERR_NONFINITE);
        } else {
          ldlt_back(Lm, Lsc, hs, dinv, r, 3);
        }
        for (int e = tid; e < 3 * r; e += blockDim.x) {
          const int pp = e / r, l = e % r;
          w.Hh[(pp * r0 + lp) + (long long)K * l] = hs[e];
        }
      }
      if (!grid_barrier(w.bar, nb, ++bseq, err)) return;
      // ---------------- B: column b of X~_k = Z_k W, X_k[:, b], lam_b, and M_k[:, b]
      if (b < r) {
        const int n = a.n[k];
        const double* Zg = w.Z + (long long)k * nmax * 3 * w.rcap;
        const double* Zk = Zg;
        int ldz = n;
        if (zs_smem) {
          ldz = odd_ld(n);
          stage_pad_async(Zs, ldz, Zg, n, n, K);
          Zk = Zs;
        }
        const double* Wb = w.Hh + (long long)K * b;
        for (int i = tid; i < K; i += blockDim.x) stage_async1(ys + i, Wb + i);
        asm volatile("cp.async.commit_group;" ::: "memory");
        // the old column (convergence sums) is fetched now, consumed after the contraction
        double* col = a.X[k] + (long long)n * b;
        const double old_pre = (tid < n) ? col[tid] : 0.0;
        stage_wait();
        __syncthreads();
        rows_dot(Zk, ldz, ys, n, K, pb, xs);
        const double lam_old = a.lam[b];
        double num = 0.0, den = 0.0, nrm2 = 0.0;
        for (int row = tid; row < n; row += blockDim.x) {
          const double v = xs[row];
          const double old = (row == tid ? old_pre : col[row]) * (gs ? lam_old : 1.0);
          const double df = v - old;
          num = fma(df, df, num);
          den = fma(old, old, den);
          nrm2 = fma(v, v, nrm2);
        }
        // only the warps that hold rows reduce (every FP64 warp instruction costs the same)
        const int wr = htg_min(NT / 32, (n + 31) / 32);
        __shared__ double r3[3][NT / 32];
        if ((tid >> 5) < wr) {
          for (int o = 16; o > 0; o >>= 1) {
            num += __shfl_xor_sync(0xffffffffu, num, o);
            den += __shfl_xor_sync(0xffffffffu, den, o);
            nrm2 += __shfl_xor_sync(0xffffffffu, nrm2, o);
          }
          if ((tid & 31) == 0) { r3[0][tid >> 5] = num; r3[1][tid >> 5] = den; r3[2][tid >> 5] = nrm2; }
        }
        __syncthreads();
        __shared__ double scol;
        if (tid == 0) {
          double tn = 0.0, td = 0.0, t2 = 0.0;
          for (int q = 0; q < wr; ++q) { tn += r3[0][q]; td += r3[1][q]; t2 += r3[2][q]; }
          atomicAdd(&w.acc2[0], tn);
          atomicAdd(&w.acc2[1], td);
          double nr = 0.0, inv = 1.0;
          if (htg_dpos_finite(t2)) {
            inv = htg_rsqrt_fast(t2);
            nr = t2 * inv;
          } else {
            nr = sqrt(t2);
          }
          if (gs) a.lam[b] = nr;
          scol = inv;
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
          double* Hc = w.H + (long long)k * w.rycap * w.rcap + (long long)K * b;
          cols_dot([&](int o) { return Zk + (long long)ldz * o; }, xs, n, K, pb,
                   [&](int o, double v) { Hc[o] = v; });
        } else {
          double* dst = w.Xold + (long long)k * nmax * w.rcap + (long long)n * b;
          for (int row = tid; row < n; row += blockDim.x) dst[row] = xs[row];
          __syncthreads();
        }
      }
      if (!grid_barrier(w.bar, nb, ++bseq, err)) return;
      // ---------------- C: column b of G_k = X_k^T X_k (all columns of X_k are final)
      if (gs && b < r) {
        const int n = a.n[k];
        const int ld = odd_ld(n);
        stage_pad_async(Xs, ld, a.X[k], n, n, r);
        stage_wait();
        __syncthreads();
        const double* xb = Xs + (long long)ld * b;
        double* Gc = w.G + (long long)k * w.rcap * w.rcap + (long long)r * b;
        cols_dot([&](int o) { return Xs + (long long)ld * o; }, xb, n, r, pb, [&](int o, double v) { Gc[o] = v; });
      }
      if (gs && !grid_barrier(w.bar, nb, ++bseq, err)) return;
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
      if (!grid_barrier(w.bar, nb, ++bseq, err)) return;
      if (b < r)
        for (int j = 0; j < d; ++j) gram_column(a, w, j, b, r0, true, xs, pb, zs_smem ? Xs : nullptr);
      if (!grid_barrier(w.bar, nb, ++bseq, err)) return;
    }
  }
  if (flops && b == 0 && tid == 0) {
    // FP64 work of the structured algorithm per mode (each item once): Gram of the new factor
    // 2 n r^2, Z_k W and M_k 2 x 2 n (3 r0) r, right-hand sides 10 (d-1) r0 r, Gamma (d-2) r^2,
    // LDL^T r^3 / 3, forward and back substitution for 3 r0 vectors 6 r0 r^2
    double f = 0.0;
    for (int k = 0; k < d; ++k) {
      const double n = a.n[k], rr = r, q0 = r0;
      f += 2.0 * n * rr * rr + 12.0 * n * q0 * rr + 10.0 * (d - 1) * q0 * rr + (d - 2) * rr * rr +
           rr * rr * rr / 3.0 + 6.0 * q0 * rr * rr;
    }
    atomicAdd(flops, f * sweeps);
  }
  // the last mode's measure
  if (b == 0 && tid == 0 && sweeps > 0) {
    const double tn = w.acc2[0], td = w.acc2[1];
    const double ek = htg_dpos_finite(td) ? sqrt(tn / td) : sqrt(tn);
    if (htg_dgt_nn(ek, w.epsacc[sweeps - 1])) w.epsacc[sweeps - 1] = ek;
  }
  if (!gs && b < r) normalise_column(a, b, false, red);
}

// ---------------------------------------------------------------------------
// Thread-block-cluster form of the Gauss-Seidel cp_als_sweep_rk2, for problems whose operands
// fit in shared memory: one cluster of Q <= 16 CTAs (one per SM) runs every sweep.  CTA q owns
// the factor columns b = q, q + Q, ... < r and the solve rows lp = q, q + Q, ... < r0.  What a
// phase hands to the next goes straight into the shared memory of the CTAs that read it
// (distributed shared memory stores), and hardware cluster barriers (release / acquire)
// separate the phases:
//   A  Gamma_k (LDL^T) and the owned rows of W = Hs Gamma_k^-1; W[:, b] to the owner of column
//      b.  Z_k and the owned old columns of X_k are fetched meanwhile, under the pivot chain
//   B  owned columns of X~_k = Z_k W, the convergence sums, X_k[:, b] and lam_b; X_k[:, b] to
//      every CTA
//   C  owned columns of G_k = X_k^T X_k to every CTA; M_k[(p, lp), b] = Z_k[:, p r0 + lp] .
//      X_k[:, b] to the owner of row lp (only the next mode's phase A reads M_k)
// Every CTA holds all Grams G_j (d r^2), the M_j rows of its solve rows, the W columns of its
// factor columns, the current X_k and a staged Z_k.  Against the cooperative form: cluster
// barriers instead of grid barriers, and no L2 round trip between phases.
// ---------------------------------------------------------------------------
constexpr int CLU_MAX = 16;   // CTAs per cluster (the non-portable maximum)

// Cluster size for ranks r, r0: the fewest columns per CTA (ceil(max(r, r0) / 16)), then as few
// CTAs as carry them.
__host__ __device__ inline int clu_ctas(int r, int r0) {
  const int R = r > r0 ? r : r0;
  const int C = (R + CLU_MAX - 1) / CLU_MAX;
  return (R + C - 1) / C;
}

// Shared-memory layout of cp_als_rk2_cluster (offsets in doubles).
struct CluLayout {
  int C, Cr, ldx, K;
  long long gs, lm, lsc, dinv, hs, mv, wc, xk, zs, zt, xo, xn, pb, go, total;
};
__host__ __device__ inline CluLayout clu_layout(int d, int r, int r0, int nmax, int Q) {
  CluLayout L;
  L.C = (r + Q - 1) / Q;      // factor columns per CTA (at most)
  L.Cr = (r0 + Q - 1) / Q;    // solve rows per CTA (at most)
  L.ldx = nmax | 1;           // odd: lanes walking columns of X_k hit distinct banks
  L.K = 3 * r0;
  long long o = 0;
  L.gs = o;   o += (long long)d * r * r;         // G_j, j < d
  L.lm = o;   o += (long long)r * r;             // Gamma_k, then its LDL^T factor
  L.lsc = o;  o += (long long)r * r;             // L
  L.dinv = o; o += r;                            // reciprocal pivots
  L.hs = o;   o += 3LL * r * L.Cr;               // right-hand sides / W rows of the solve rows
  L.mv = o;   o += (long long)L.Cr * d * 3 * r;  // M_j rows (p, lp) of the solve rows
  L.wc = o;   o += (long long)L.C * L.K;         // W columns of the owned factor columns
  L.xk = o;   o += (long long)L.ldx * r;         // X_k
  o += o & 1;                                    // 16-byte starts: bulk-copy destinations
  L.zs = o;   o += (long long)nmax * L.K;        // Z_k (n x K, leading dimension n)
  o += o & 1;
  L.zt = o;   o += (long long)nmax * L.K;        // Z_k^T (K x n, leading dimension K)
  L.xo = o;   o += (long long)nmax * L.C;        // owned columns of X_k before the update
  L.xn = o;   o += (long long)nmax * L.C;        // owned columns after it
  const long long items = htg_max(htg_max(nmax, L.K), r) * L.C;
  L.pb = o;   o += 8 * htg_max((long long)NT, items);   // partial sums (up to 8 parts)
  L.go = o;   o += (long long)(r + L.K) * L.C;   // dot products before they are pushed
  L.total = o;
  return L;
}

// Parts per output of a split dot product of `len` terms over `items` outputs on nthr threads:
// the count (1..8, at most len) that minimises a thread's FP64 instructions,
// ceil(items P / nthr) ceil(len / P).
__device__ inline int balanced_parts(int items, int len, int nthr = NT) {
  int best = 1;
  long long bc = (long long)((items + nthr - 1) / nthr) * len;
  for (int P = 2; P <= 8 && P <= len; ++P) {
    const long long c = (long long)((items * P + nthr - 1) / nthr) * ((len + P - 1) / P);
    if (c < bc) { bc = c; best = P; }
  }
  return best;
}

// sum_{i0 <= i < i1} a[i sa] b[i sb] with four independent partial sums (FP64 latency)
__device__ inline double dot4(const double* a, long long sa, const double* b, int i0, int i1) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = i0;
  for (; i + 3 < i1; i += 4) {
    s0 = fma(a[sa * i], b[i], s0);
    s1 = fma(a[sa * (i + 1)], b[i + 1], s1);
    s2 = fma(a[sa * (i + 2)], b[i + 2], s2);
    s3 = fma(a[sa * (i + 3)], b[i + 3], s3);
  }
  for (; i < i1; ++i) s0 = fma(a[sa * i], b[i], s0);
  return (s0 + s1) + (s2 + s3);
}

// out[o + nout c] = col(o) . xv[:, c] (length n; xv column-major, leading dimension n) for
// o < nout, c < nc, each split into P parts (balanced_parts, computed once per launch):
// consecutive lanes take consecutive outputs, partial sums added in part order.  Work item e =
// f + items part, f = o + nout c; the indices advance without divisions.
template <class Col>
__device__ void cols_dot_multi(Col col, const double* xv, int n, int nout, int nc, int P, double* pb, double* out) {
  const int items = nout * nc;
  const int chunk = (n + P - 1) / P;
  int f = threadIdx.x, part = 0;
  while (f >= items) { f -= items; ++part; }
  for (int e = threadIdx.x; e < items * P; e += NT) {
    int o = f, c = 0;
    while (o >= nout) { o -= nout; ++c; }
    const int q0 = part * chunk;
    pb[e] = dot4(col(o), 1, xv + (long long)n * c, q0, htg_min(n, q0 + chunk));
    f += NT;
    while (f >= items) { f -= items; ++part; }
  }
  __syncthreads();
  for (int g = threadIdx.x; g < items; g += NT) {
    double v = pb[g];
    for (int pp = 1; pp < P; ++pp) v += pb[g + items * pp];
    out[g] = v;
  }
  __syncthreads();
}

// out[row + n c] = sum_i S[row + ld i] Y[i + ldy c] for row < n, c < nc, i < m, each split into P
// parts: consecutive lanes take consecutive rows, partial sums added in part order.
__device__ void rows_dot_multi(const double* S, int ld, const double* Y, int ldy, int n, int m, int nc, int P,
                               double* pb, double* out) {
  const int items = n * nc;
  const int chunk = (m + P - 1) / P;
  int f = threadIdx.x, part = 0;
  while (f >= items) { f -= items; ++part; }
  for (int e = threadIdx.x; e < items * P; e += NT) {
    int row = f, c = 0;
    while (row >= n) { row -= n; ++c; }
    const int i0 = part * chunk;
    pb[e] = dot4(S + row, ld, Y + (long long)ldy * c, i0, htg_min(m, i0 + chunk));
    f += NT;
    while (f >= items) { f -= items; ++part; }
  }
  __syncthreads();
  for (int g = threadIdx.x; g < items; g += NT) {
    double v = pb[g];
    for (int pp = 1; pp < P; ++pp) v += pb[g + items * pp];
    out[g] = v;
  }
  __syncthreads();
}

// The first half of cols_dot_multi on threads t0 .. t0 + nthr - 1 only (no barrier): the P
// partial sums of every output into pb[f + items part], items = nout nc.
template <class Col>
__device__ void cols_dot_parts(Col col, const double* xv, int n, int nout, int nc, int P, double* pb, int t0,
                               int nthr) {
  const int items = nout * nc;
  const int chunk = (n + P - 1) / P;
  const int t = threadIdx.x - t0;
  int f = t, part = 0;
  while (f >= items) { f -= items; ++part; }
  for (int e = t; e < items * P; e += nthr) {
    int o = f, c = 0;
    while (o >= nout) { o -= nout; ++c; }
    const int q0 = part * chunk;
    pb[e] = dot4(col(o), 1, xv + (long long)n * c, q0, htg_min(n, q0 + chunk));
    f += nthr;
    while (f >= items) { f -= items; ++part; }
  }
}

// The first half of rows_dot_multi on threads t0 .. t0 + nthr - 1 only (no barrier): the P
// partial sums of every output into pb[f + items part], items = n nc.
__device__ void rows_dot_parts(const double* S, int ld, const double* Y, int ldy, int n, int m, int nc, int P,
                               double* pb, int t0, int nthr) {
  const int items = n * nc;
  const int chunk = (m + P - 1) / P;
  const int t = threadIdx.x - t0;
  int f = t, part = 0;
  while (f >= items) { f -= items; ++part; }
  for (int e = t; e < items * P; e += nthr) {
    int row = f, c = 0;
    while (row >= n) { row -= n; ++c; }
    const int i0 = part * chunk;
    pb[e] = dot4(S + row, ld, Y + (long long)ldy * c, i0, htg_min(m, i0 + chunk));
    f += nthr;
    while (f >= items) { f -= items; ++part; }
  }
}

// n x cols column-major copy (leading dimensions lds, ldd) through L2 (data other CTAs of this
// launch wrote: an L1 line may hold parts of several CTAs' columns), 8 loads in flight per thread
__device__ void stage_cg(double* dst, int ldd, const double* src, int lds, int n, int cols) {
  const int total = n * cols;
  int base = 0;
  for (; base + 8 * NT <= total; base += 8 * NT) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * NT + (int)threadIdx.x;
      v[u] = __ldcg(src + (e % n) + (long long)lds * (e / n));
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * NT + (int)threadIdx.x;
      dst[(e % n) + (long long)ldd * (e / n)] = v[u];
    }
  }
  for (int e = base + (int)threadIdx.x; e < total; e += NT)
    dst[(e % n) + (long long)ldd * (e / n)] = __ldcg(src + (e % n) + (long long)lds * (e / n));
}

__device__ inline unsigned clu_smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// one-dimensional bulk copy global -> shared, completing on the mbarrier's transaction count
__device__ inline void clu_bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   clu_smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(clu_smem_u32(bar))
               : "memory");
}
constexpr long long CLU_WAIT_CYCLES = 1ll << 31;   // bounded mbarrier wait (about 1 s at 2 GHz)
// bounded wait for the mbarrier phase of the given parity; false when it gave up
__device__ inline bool clu_mbar_wait(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(clu_smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > CLU_WAIT_CYCLES) return false;
  }
}

// (a_n / a_d > b_n / b_d) for non-negative numerators and positive denominators, by cross
// multiplication (no division) and a bit-pattern compare of the non-negative products
__device__ inline bool ratio_gt(double an, double ad, double bn, double bd) { return htg_dgt_nn(an * bd, bn * ad); }

__global__ void __launch_bounds__(NT, 1) cp_als_rk2_cluster(CpArgs a, PowArgs pa, CpWs w, const double* mu_src,
                                                         int sweeps, int* err, double* flops) {
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank(), Q = (int)cluster.num_blocks();
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int d = a.d, r = a.r, r0 = pa.r0, K = 3 * r0, nmax = w.nmax;
  const CluLayout L = clu_layout(d, r, r0, nmax, Q);
  const int ldx = L.ldx;
  extern __shared__ double sh[];
  double* Gs = sh + L.gs;
  double* Lm = sh + L.lm;
  double* Lsc = sh + L.lsc;
  double* dinv = sh + L.dinv;
  double* hs = sh + L.hs;
  double* Mv = sh + L.mv;
  double* Wc = sh + L.wc;
  double* Xk = sh + L.xk;
  double* Zs = sh + L.zs;
  double* ZTs = sh + L.zt;
  double* xo = sh + L.xo;
  double* xn = sh + L.xn;
  double* pb = sh + L.pb;
  double* go = sh + L.go;
  __shared__ unsigned short tri[TRI_MAX];
  __shared__ double red[HT_MAXD + 32];
  __shared__ double part[2 * CLU_MAX];   // CTA 0: every CTA's convergence sums of the last mode
  __shared__ double best[2 * 64];        // CTA 0: per sweep, the largest measure as (num, den)
  __shared__ double mu_own[CLU_MAX];     // weights of x_old at the solve rows
  __shared__ double lamo[CLU_MAX];       // lam of the owned columns before the update
  __shared__ double csum[2 * CLU_MAX];   // per owned column: the convergence sums
  __shared__ double cinv[CLU_MAX];       // per owned column: 1 / |x~|
  __shared__ int Pb[HT_MAXD], Pg[HT_MAXD], Pg2[HT_MAXD], Pm[HT_MAXD], Pm2[HT_MAXD];   // dot-product parts
  __shared__ __align__(8) unsigned long long zbar;        // completion of a mode's bulk prefetch
  const int nc = (q < r) ? (r - q + Q - 1) / Q : 0;      // owned factor columns
  const int nrw = (q < r0) ? (r0 - q + Q - 1) / Q : 0;   // owned solve rows
  for (int c = tid; c < r; c += NT) {
    const int o = tri_offset(c, r);
    for (int i = c; i < r; ++i) tri[o + i - c] = (unsigned short)(i | (c << 8));
  }
  for (int i = tid; i < 2 * CLU_MAX; i += NT) part[i] = 0.0;
  for (int i = tid; i < 64; i += NT) {
    best[2 * i] = 0.0;
    best[2 * i + 1] = 1.0;
  }
  for (int i = tid; i < nrw; i += NT) mu_own[i] = mu_src[q + Q * i];
  for (int k = tid; k < d; k += NT) {
    Pb[k] = balanced_parts(a.n[k] * htg_max(nc, 1), K);
    Pg[k] = balanced_parts(r * htg_max(nc, 1), a.n[k]);
    Pm[k] = balanced_parts(K * htg_max(nc, 1), a.n[k]);
    Pm2[k] = balanced_parts(K * htg_max(nc, 1), a.n[k], NT - 32 * htg_max(nc, 1));
    Pg2[k] = balanced_parts(r * htg_max(nc, 1), a.n[k], NT - 64);
  }
  // Z_k and Z_k^T arrive by two bulk copies per mode when every block is 16-byte aligned and a
  // multiple of 16 bytes (else by 8-byte asynchronous copies)
  const long long zstride = (long long)nmax * 3 * w.rcap;
  bool bulk = (zstride % 2 == 0) && (((unsigned long long)w.Z | (unsigned long long)w.ZT) % 16 == 0);
  for (int k = 0; k < d; ++k) bulk = bulk && ((long long)a.n[k] * K % 2 == 0) && (2LL * a.n[k] * K * 8 < (1 << 20));
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(clu_smem_u32(&zbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (q == 0)
    for (int i = tid; i < r0; i += NT) w.wold[i] = mu_src[i];
  // ---------------- 0a: powers of x_old at the solve rows, all rows of a mode at once (scratch:
  // the Z_k buffer, 2 nrw n <= 3 r0 n doubles)
  for (int k = 0; k < d && nrw > 0; ++k) {
    const int n = pa.n[k], hw = pa.hw[k];
    double* xs = Zs;               // column i: x_old,k[:, q + Q i]
    double* ys = Zs + nrw * n;     // A x
    double* Zk = w.Z + (long long)k * zstride;
    double* ZTk = w.ZT + (long long)k * zstride;   // Z_k^T: K x n, leading dimension K
    for (int e = tid; e < nrw * n; e += NT) xs[e] = pa.X[k][(e % n) + (long long)n * (q + Q * (e / n))];
    __syncthreads();
    for (int e = tid; e < nrw * n; e += NT) {
      const int j = e % n, i = e / n, lp = q + Q * i;
      const double* x = xs + (long long)n * i;
      double s = 0.0;
      for (int o = -hw; o <= hw; ++o) {
        int jj = (j + o) % n;
        if (jj < 0) jj += n;
        s = fma(pa.c[k][o + hw], x[jj], s);
      }
      ys[e] = s;
      Zk[j + (long long)n * lp] = x[j];
      Zk[j + (long long)n * (r0 + lp)] = s;
      ZTk[lp + (long long)K * j] = x[j];
      ZTk[r0 + lp + (long long)K * j] = s;
    }
    __syncthreads();
    for (int e = tid; e < nrw * n; e += NT) {
      const int j = e % n, i = e / n, lp = q + Q * i;
      const double* y = ys + (long long)n * i;
      double s = 0.0;
      for (int o = -hw; o <= hw; ++o) {
        int jj = (j + o) % n;
        if (jj < 0) jj += n;
        s = fma(pa.c[k][o + hw], y[jj], s);
      }
      Zk[j + (long long)n * (2 * r0 + lp)] = s;
      ZTk[2 * r0 + lp + (long long)K * j] = s;
    }
    __syncthreads();
  }
  // owned columns of G_j, from X_j in Xk and its owned columns in xn (columns of Xk), to every CTA
  auto gram_push = [&](int j, int n) {
    cols_dot_multi([&](int o) { return Xk + (long long)ldx * o; }, xn, n, r, nc, Pg[j], pb, go);
    for (int f = tid; f < r * nc; f += NT) {
      const int o = f % r, c = f / r;
      const double v = go[f];
      double* dst = Gs + (long long)j * r * r + (long long)r * (q + Q * c) + o;
      for (int t = 0; t < Q; ++t) *cluster.map_shared_rank(dst, t) = v;
    }
  };
  // M_j[(p, lp), b] = value f = (p r0 + lp) + K c (b = q + Q c) to the owner of solve row lp
  auto m_push = [&](int j, int f, double v) {
    const int oo = f % K, c = f / K, p = oo / r0, lp = oo - p * r0;
    *cluster.map_shared_rank(Mv + ((long long)((lp / Q) * d + j) * 3 + p) * r + (q + Q * c), lp % Q) = v;
  };
  cluster.sync();   // Z complete; all of x_old read (x may alias it)
  for (int i = 0; i < nc; ++i) normalise_column(a, q + Q * i, false, red);
  cluster.sync();   // X normalised
  // ---------------- 0b: owned columns of G_j and M_j for every j (X_j by asynchronous copies, Z_j^T
  // by one bulk copy when aligned)
  unsigned zphase = 0;     // parity of the bulk prefetch's mbarrier phase
  bool waited_ok = true;   // false once a bounded wait gave up
  for (int j = 0; j < d; ++j) {
    const int n = a.n[j];
    if (nc > 0) {
      const double* ZTj = w.ZT + (long long)j * zstride;
      if (bulk) {
        if (tid == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          const unsigned bytes = (unsigned)((long long)n * K * sizeof(double));
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(clu_smem_u32(&zbar)),
                       "r"(bytes)
                       : "memory");
          clu_bulk_g2s(ZTs, ZTj, bytes, &zbar);
        }
      } else {
        stage_cg(ZTs, K, ZTj, K, K, n);
      }
      stage_cg(Xk, ldx, a.X[j], n, n, r);
      if (bulk) {
        if (!clu_mbar_wait(&zbar, zphase)) waited_ok = false;
        zphase ^= 1u;
      }
      __syncthreads();
      for (int e = tid; e < n * nc; e += NT) xn[e] = Xk[(e % n) + (long long)ldx * (q + Q * (e / n))];
      __syncthreads();
      gram_push(j, n);
      rows_dot_multi(ZTs, K, xn, n, K, n, nc, Pm[j], pb, go);   // M_j columns, by rows of Z_j^T
      for (int f = tid; f < K * nc; f += NT) m_push(j, f, go[f]);
      __syncthreads();   // Xk, ZTs and go are rewritten for the next j
    }
  }
  cluster.sync();   // every G_j and M_j row in place
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int k = 0; k < d; ++k) {
      const int n = a.n[k];
      const bool record = !(sweep == 0 && k == 0);   // the previous mode's sums are complete
      // ---------------- A: Gamma_k (LDL^T) and the solve rows of W = Hs Gamma_k^-1
      // Z_k and Z_k^T for phases B and C: two bulk copies issued by one thread (or 8-byte
      // asynchronous copies), and the owned old columns of X_k; all land under the LDL^T pivot
      // chain (nothing may run beside it)
      if (nc > 0) {
        const double* Zk = w.Z + (long long)k * zstride;
        const double* ZTk = w.ZT + (long long)k * zstride;
        if (bulk) {
          if (tid == 0) {
            // the generic-proxy reads of Zs and ZTs (the last phase C) before the async writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const unsigned bytes = (unsigned)((long long)n * K * sizeof(double));
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(clu_smem_u32(&zbar)),
                         "r"(2 * bytes)
                         : "memory");
            clu_bulk_g2s(Zs, Zk, bytes, &zbar);
            clu_bulk_g2s(ZTs, ZTk, bytes, &zbar);
          }
        } else {
          for (int e = tid; e < n * K; e += NT) {
            stage_async1(Zs + e, Zk + e);
            stage_async1(ZTs + e, ZTk + e);
          }
        }
        for (int e = tid; e < n * nc; e += NT)
          stage_async1(xo + e, a.X[k] + (e % n) + (long long)n * (q + Q * (e / n)));
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (tid < nc) lamo[tid] = a.lam[q + Q * tid];
      }
      if (nrw > 0) {
        const int nG = r * r;
        // side by side: Gamma_k (warps 0-2, 4-5), at the first mode the right-hand sides (row i on
        // warp 7 - i % 2; later modes formed them in the previous phase C), CTA 0's record of the
        // previous mode's convergence measure (warp 3).  (Gamma_k on every idle warp, with the
        // factors multiplied as two interleaved partial products, measured slower: 5.4k cycles
        // against 3.4k.)
        if (wid >= NT / 32 - 2) {
          if (sweep == 0 && k == 0)
            for (int i = NT / 32 - 1 - wid; i < nrw; i += 2)
              rk2_rhs_row(Mv + (long long)i * d * 3 * r, d, k, r, mu_own[i], hs + 3LL * r * i, lane, 32);
        } else if (wid % 4 != 3) {
          const int gt = (wid - wid / 4) * 32 + lane;
          for (int e = gt; e < nG; e += (NT / 32 - 3) * 32) {
            double v = 1.0;
            for (int j = 0; j < d; ++j)
              if (j != k) v *= Gs[j * nG + e];
            Lm[e] = v;
          }
        } else if (q == 0 && record) {
          // warp 3: the sums over CTAs (a shuffle tree), then the running maximum of num / den
          double tn = (lane < Q) ? part[2 * lane] : 0.0, td = (lane < Q) ? part[2 * lane + 1] : 0.0;
          for (int o = 16; o > 0; o >>= 1) {
            tn += __shfl_xor_sync(0xffffffffu, tn, o);
            td += __shfl_xor_sync(0xffffffffu, td, o);
          }
          if (lane == 0) {
            if (!htg_dpos_finite(td)) td = 1.0;
            const int sw = (k == 0) ? sweep - 1 : sweep;
            if (ratio_gt(tn, td, best[2 * sw], best[2 * sw + 1])) {
              best[2 * sw] = tn;
              best[2 * sw + 1] = td;
            }
          }
        }
        __syncthreads();
        bool ok = ldlt_forward(Lm, Lsc, hs, dinv, tri, r, 3 * nrw);
        if (!ok) {
          // shift by 1e-14 tr(Gamma)/r, only after a failed factorisation (Section 2.1
          // regularisation of ill-conditioned ALS systems), and start over
          __shared__ double shift;
          if (tid == 0) {
            double tr = 0.0;
            for (int i = 0; i < r; ++i) {
              double v = 1.0;
              for (int j = 0; j < d; ++j)
                if (j != k) v *= Gs[j * nG + i + r * i];
              tr += v;
            }
            shift = 1e-14 * tr / r;
          }
          __syncthreads();
          for (int e = tid; e < nG; e += NT) {
            double v = 1.0;
            for (int j = 0; j < d; ++j)
              if (j != k) v *= Gs[j * nG + e];
            Lm[e] = v + ((e % r == e / r) ? shift : 0.0);
          }
          for (int i = 0; i < nrw; ++i)
            rk2_rhs_row(Mv + (long long)i * d * 3 * r, d, k, r, mu_own[i], hs + 3LL * r * i, tid, NT);
          __syncthreads();
          ok = ldlt_forward(Lm, Lsc, hs, dinv, tri, r, 3 * nrw);
        }
        if (!ok) {
          if (tid == 0 && err) atomicCAS(err, 0, (int)HT_ERR_NONFINITE);
        } else {
          ldlt_back(Lm, Lsc, hs, dinv, r, 3 * nrw);
        }
        // W^(p)[lp, l] to the owner of column l
        for (int e = tid; e < 3 * r * nrw; e += NT) {
          const int i = e / (3 * r), f = e - i * 3 * r, p = f / r, l = f - p * r;
          *cluster.map_shared_rank(Wc + (long long)(l / Q) * K + p * r0 + (q + Q * i), l % Q) = hs[e];
        }
      }
      stage_wait();
      if (nc > 0 && bulk) {
        if (!clu_mbar_wait(&zbar, zphase)) waited_ok = false;
        zphase ^= 1u;
      }
      cluster.sync();
      // ---------------- B: owned columns of X~_k = Z_k W, X_k[:, b] and lam_b; M_k[:, b] to the
      //                  owners of the solve rows
      if (nc > 0) {
        rows_dot_multi(Zs, n, Wc, K, n, K, nc, Pb[k], pb, xn);
        // side by side: warp c < nc reduces column c (convergence sums, |x~|); the other warps form
        // the partial sums of M~_k = Z_k^T X~_k (by rows of Z_k^T), scaled by 1 / |x~| below
        if (wid >= nc) {
          rows_dot_parts(ZTs, K, xn, n, K, n, nc, Pm2[k], pb, 32 * nc, NT - 32 * nc);
        } else {
          const int c = wid;
          const double lam_old = lamo[c];
          double num = 0.0, den = 0.0, nrm2 = 0.0;
          for (int row = lane; row < n; row += 32) {
            const double v = xn[row + n * c];
            const double old = xo[row + n * c] * lam_old;
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
          if (lane == 0) {
            double nr = 0.0, inv = 1.0;
            if (htg_dpos_finite(nrm2)) {
              inv = htg_rsqrt_fast(nrm2);
              nr = nrm2 * inv;
            } else {
              nr = sqrt(nrm2);
            }
            a.lam[q + Q * c] = nr;
            csum[2 * c] = num;
            csum[2 * c + 1] = den;
            cinv[c] = inv;
          }
        }
        __syncthreads();
        {
          const int items = K * nc, P = Pm2[k];
          for (int f = tid; f < items; f += NT) {
            double v = pb[f];
            for (int pp = 1; pp < P; ++pp) v += pb[f + items * pp];
            m_push(k, f, v * cinv[f / K]);
          }
        }
        double* Xg = a.X[k];
        for (int f = tid; f < n * nc; f += NT) {
          const int row = f % n, c = f / n;
          const double v = xn[f] * cinv[c];
          xn[f] = v;
          Xg[row + (long long)n * (q + Q * c)] = v;
          double* dst = Xk + row + (long long)ldx * (q + Q * c);
          for (int t = 0; t < Q; ++t) *cluster.map_shared_rank(dst, t) = v;
        }
        if (tid == 0) {
          double tn = 0.0, td = 0.0;
          for (int c = 0; c < nc; ++c) { tn += csum[2 * c]; td += csum[2 * c + 1]; }
          double* p0 = cluster.map_shared_rank(part, 0);
          p0[2 * q] = tn;
          p0[2 * q + 1] = td;
        }
      }
      cluster.sync();
      // ---------------- C: owned columns of G_k (to every CTA, warps 0-5) and, beside them, the next
      // mode's right-hand sides (warps 6-7: every M_j row they read is in place)
      {
        const bool more = !(sweep == sweeps - 1 && k == d - 1);
        const int kn = (k + 1 == d) ? 0 : k + 1;
        if (wid >= NT / 32 - 2) {
          if (more)
            for (int i = NT / 32 - 1 - wid; i < nrw; i += 2)
              rk2_rhs_row(Mv + (long long)i * d * 3 * r, d, kn, r, mu_own[i], hs + 3LL * r * i, lane, 32);
        } else if (nc > 0) {
          cols_dot_parts([&](int o) { return Xk + (long long)ldx * o; }, xn, n, r, nc, Pg2[k], pb, 0, NT - 64);
        }
        __syncthreads();
        if (nc > 0) {
          const int items = r * nc, P = Pg2[k];
          for (int f = tid; f < items; f += NT) {
            double v = pb[f];
            for (int pp = 1; pp < P; ++pp) v += pb[f + items * pp];
            const int o = f % r, c = f / r;
            double* dst = Gs + (long long)k * r * r + (long long)r * (q + Q * c) + o;
            for (int t = 0; t < Q; ++t) *cluster.map_shared_rank(dst, t) = v;
          }
        }
      }
      cluster.sync();
    }
  }
  if (!waited_ok && err) atomicCAS(err, 0, (int)HT_ERR_TIMEOUT);
  if (flops && q == 0 && tid == 0) {
    // the structured algorithm's FP64 work, as counted by the cooperative form
    double f = 0.0;
    for (int k = 0; k < d; ++k) {
      const double n = a.n[k], rr = r, q0 = r0;
      f += 2.0 * n * rr * rr + 12.0 * n * q0 * rr + 10.0 * (d - 1) * q0 * rr + (d - 2) * rr * rr +
           rr * rr * rr / 3.0 + 6.0 * q0 * rr * rr;
    }
    atomicAdd(flops, f * sweeps);
  }
  // the last mode's sums (arrived before the last cluster barrier), then the per-sweep measures
  if (q == 0 && tid == 0 && sweeps > 0) {
    double tn = 0.0, td = 0.0;
    for (int t = 0; t < Q; ++t) { tn += part[2 * t]; td += part[2 * t + 1]; }
    if (!htg_dpos_finite(td)) td = 1.0;
    const int sw = sweeps - 1;
    if (ratio_gt(tn, td, best[2 * sw], best[2 * sw + 1])) {
      best[2 * sw] = tn;
      best[2 * sw + 1] = td;
    }
    for (int s = 0; s < sweeps && s < 64; ++s) w.epsacc[s] = sqrt(best[2 * s] / best[2 * s + 1]);
  }
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

CpClusterCfg htg_cp_cluster_setup(int device) {
  CpClusterCfg out;
  int optin = 0;
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, cp_als_rk2_cluster) != cudaSuccess) {
    cudaGetLastError();
    return out;
  }
  // every CTA claims its SM's whole shared memory (the HT route's kernels, launched beside this
  // one, then land on other SMs)
  const long long dyn = (long long)optin - (long long)fa.sharedSizeBytes;
  if (dyn < (long long)(16 * 1024)) return out;
  if (cudaFuncSetAttribute(cp_als_rk2_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess ||
      cudaFuncSetAttribute(cp_als_rk2_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return out;
  }
  // the largest cluster (up to 16 CTAs) of which one fits the device: smaller ones fit as well
  for (int q = CLU_MAX; q >= 1; --q) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(q, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = (size_t)dyn;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = q;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, cp_als_rk2_cluster, &cfg) == cudaSuccess && n >= 1) {
      out.max_q = q;
      out.cap_doubles = dyn / (long long)sizeof(double);
      return out;
    }
    cudaGetLastError();
  }
  return out;
}

// CTAs of the cluster form for ranks (r, r0) on this context, 0 when the cooperative form runs
static int cluster_form_ctas(const ht_ctx* c, int r, int r0) {
  const CpClusterCfg* clu = htg_ctx_cp_cluster(c);
  if (htg_ctx_cp_form(c) != 0 || clu->max_q <= 0 || r < 1 || r0 < 1 || r > 64 || r0 > 64) return 0;
  if (r * (r + 1) / 2 > TRI_MAX) return 0;
  const int Q = clu_ctas(r, r0);
  const CluLayout lay = clu_layout(htg_ctx_d(c), r, r0, htg_ctx_cp((ht_ctx*)c)->nmax, Q);
  return (Q <= clu->max_q && lay.total <= clu->cap_doubles) ? Q : 0;
}

extern "C" int cp_als_rk2_cluster_ctas(const ht_ctx* c, int r, int r0, int* ctas) {
  if (!c || !ctas || r < 1 || r0 < 1) return HT_ERR_ARG;
  *ctas = cluster_form_ctas(c, r, r0);
  return HT_OK;
}

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
      x_old->rank > x_old->cap || x->rank > 64 || x_old->rank > 64)
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
  // the cluster form: Gauss-Seidel, and its layout within one CTA's shared memory on a cluster
  // size this device can place (htg_cp_cluster_setup, at context creation)
  const CpClusterCfg* clu = htg_ctx_cp_cluster(c);
  if (variant == CP_ALS_GS) {
    const int Q = cluster_form_ctas(c, a.r, r0);
    if (Q > 0) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(Q);
      cfg.blockDim = dim3(NT);
      cfg.dynamicSmemBytes = (size_t)clu->cap_doubles * sizeof(double);
      cfg.stream = s;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = Q;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int launches = 0;
      htg_prof_begin(c, s);
      const cudaError_t e1 = cudaLaunchKernelEx(&cfg, cp_als_rk2_cluster, a, pa, *w, (const double*)x_old->weight,
                                                sweeps, htg_ctx_err(c), htg_prof_flops(c, KC_CPSOLVE));
      htg_prof_end(c, KC_CPSOLVE, s);
      ++launches;
      if (e1 == cudaSuccess && eps_dev && sweeps > 0) {
        cp_eps_out_kernel<<<1, 64, 0, s>>>(*w, sweeps, eps_dev);
        ++launches;
      }
      htg_ctx_count(c, launches, s);
      return (e1 == cudaSuccess && cudaGetLastError() == cudaSuccess) ? HT_OK : HT_ERR_CUDA;
    }
  }
  // one cooperative launch: CTA b owns factor column b (and row b of the solve)
  const int nblk = htg_max(a.r, r0);
  const size_t nm = (size_t)w->nmax;
  // stage Z_k in shared memory when it fits
  const size_t with_z = (size_t)persistent_smem_doubles(a.r, r0, d, (int)nm, true) * sizeof(double);
  const int zs_smem = (with_z <= 160 * 1024) ? 1 : 0;
  size_t smem = zs_smem ? with_z : (size_t)persistent_smem_doubles(a.r, r0, d, (int)nm, false) * sizeof(double);
  // Claim all of each SM's shared memory: the HT route's kernels, launched beside this one on
  // another stream, then land on other SMs (an SM partition's FP64 pipe shared with their
  // warps lengthens this kernel's latency-bound chains: measured 0.96 ms alone, 1.06 ms side by
  // side before).  The launch has one CTA per factor column, far fewer than SMs.
  {
    int dev = 0, optin = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, cp_als_rk2_persistent) == cudaSuccess && nblk <= nsm && optin > 0) {
      const size_t whole = (size_t)optin - fa.sharedSizeBytes;
      if (whole > smem) smem = whole;
    }
  }
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(cp_als_rk2_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return HT_ERR_CUDA;
  }
  int launches = 0;
  htg_prof_begin(c, s);
  cudaError_t e0 = cudaMemsetAsync(w->bar, 0, 64 * sizeof(unsigned int), s);   // barrier words, one per CTA
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
                                      htg_ctx_err(c), zs_smem, htg_prof_flops(c, KC_CPSOLVE));
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

namespace {
// every CTA but `absent` meets at one grid barrier (sequence number 1)
__global__ void selftest_barrier_kernel(unsigned int* flags, int absent, int* err) {
  if ((int)blockIdx.x == absent) return;
  grid_barrier(flags, gridDim.x, 1u, err);
}
}  // namespace

extern "C" int ht_selftest_grid_barrier(int nblocks, int absent, int device) {
  if (nblocks < 1 || nblocks > 64 || absent >= nblocks) return HT_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return HT_ERR_CUDA;
  void* mem = nullptr;
  if (cudaMalloc(&mem, 2048) != cudaSuccess) return HT_ERR_CUDA;
  unsigned int* flags = (unsigned int*)mem;
  int* err = (int*)((char*)mem + 1024);
  int st = HT_OK;
  if (cudaMemset(mem, 0, 2048) != cudaSuccess) st = HT_ERR_CUDA;
  if (st == HT_OK) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblocks);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = 0;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, selftest_barrier_kernel, flags, absent, err) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
      st = HT_ERR_CUDA;
  }
  int h = 0;
  if (st == HT_OK && cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) st = HT_ERR_CUDA;
  cudaFree(mem);
  return st != HT_OK ? st : h;
}

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
