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
__global__ void cp_normalize_kernel(CpArgs a, int fold) {
  for (int l = threadIdx.x; l < a.r; l += blockDim.x) {
    double w = a.lam[l];
    for (int k = 0; k < a.d; ++k) {
      double* col = a.X[k] + (long long)a.n[k] * l;
      double s = 0.0;
      for (int j = 0; j < a.n[k]; ++j) s = fma(col[j], col[j], s);
      const double nr = sqrt(s);
      if (nr > 0.0) {
        for (int j = 0; j < a.n[k]; ++j) col[j] /= nr;
        w *= nr;
      }
    }
    if (fold) {
      double* col = a.X[0] + (long long)a.n[0] * l;
      for (int j = 0; j < a.n[0]; ++j) col[j] *= w;
      a.lam[l] = 1.0;
    } else {
      a.lam[l] = w;
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
__global__ void cp_solve_kernel(CpArgs a, CpWs w, int k, int sweep, int* err) {
  extern __shared__ double sh[];
  const int r = a.r, n = a.n[k];
  double* Lm = sh;               // r x r
  double* nrm = sh + r * r;      // r
  __shared__ int ok;
  __shared__ double red_num[NT / 32], red_den[NT / 32];
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Lm[e] = w.Gam[e];
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (threadIdx.x == 0) {
      ok = 1;
      if (attempt == 1) {
        double tr = 0.0;
        for (int i = 0; i < r; ++i) tr += w.Gam[i + r * i];
        for (int e = 0; e < r * r; ++e) Lm[e] = w.Gam[e];
        const double sh_ = 1e-14 * tr / r;
        for (int i = 0; i < r; ++i) Lm[i + r * i] += sh_;
      }
      // column-oriented Cholesky, lower triangle: Gamma = L L^T
      for (int j = 0; j < r && ok; ++j) {
        double dj = Lm[j + r * j];
        for (int p = 0; p < j; ++p) dj -= Lm[j + r * p] * Lm[j + r * p];
        if (!(dj > 0.0)) { ok = 0; break; }
        dj = sqrt(dj);
        Lm[j + r * j] = dj;
        for (int i = j + 1; i < r; ++i) {
          double v = Lm[i + r * j];
          for (int p = 0; p < j; ++p) v -= Lm[i + r * p] * Lm[j + r * p];
          Lm[i + r * j] = v / dj;
        }
      }
    }
    __syncthreads();
    const int good = ok;
    __syncthreads();
    if (good) break;
  }
  if (!ok) {
    if (threadIdx.x == 0 && err) atomicCAS(err, 0, (int)HT_ERR_NONFINITE);
    return;
  }
  // rows: solve L L^T x = rhs, x^T is row i of X~ (stored into RHS in place)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double* row = w.RHS + i;   // stride n between columns
    for (int j = 0; j < r; ++j) {
      double v = row[(long long)n * j];
      for (int p = 0; p < j; ++p) v -= Lm[j + r * p] * row[(long long)n * p];
      row[(long long)n * j] = v / Lm[j + r * j];
    }
    for (int j = r - 1; j >= 0; --j) {
      double v = row[(long long)n * j];
      for (int p = j + 1; p < r; ++p) v -= Lm[p + r * j] * row[(long long)n * p];
      row[(long long)n * j] = v / Lm[j + r * j];
    }
  }
  __syncthreads();
  // convergence measure against the old (scaled) factor, then store
  double num = 0.0, den = 0.0;
  for (long long e = threadIdx.x; e < (long long)n * r; e += blockDim.x) {
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
  if ((threadIdx.x & 31) == 0) { red_num[threadIdx.x >> 5] = num; red_den[threadIdx.x >> 5] = den; }
  for (int l = threadIdx.x; l < r; l += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = fma(w.RHS[j + (long long)n * l], w.RHS[j + (long long)n * l], s);
    nrm[l] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tn = 0.0, td = 0.0;
    for (int q = 0; q < NT / 32; ++q) { tn += red_num[q]; td += red_den[q]; }
    const double ek = td > 0.0 ? sqrt(tn / td) : sqrt(tn);
    if (ek > w.epsacc[sweep]) w.epsacc[sweep] = ek;
  }
  if (a.variant == CP_ALS_GS) {
    for (long long e = threadIdx.x; e < (long long)n * r; e += blockDim.x) {
      const int l = (int)(e / n);
      a.X[k][e] = nrm[l] > 0.0 ? w.RHS[e] / nrm[l] : w.RHS[e];
    }
    for (int l = threadIdx.x; l < r; l += blockDim.x) a.lam[l] = nrm[l] > 0.0 ? nrm[l] : 0.0;
  } else {
    double* dst = w.Xold + (long long)k * w.nmax * w.rcap;
    for (long long e = threadIdx.x; e < (long long)n * r; e += blockDim.x) dst[e] = w.RHS[e];
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
  cp_apply_kernel<<<dim3(x->rank, d), 128, 3 * nmax * sizeof(double), s>>>(a);
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
  if (x->rank > w->rcap || y->rank > w->rycap || x->rank > x->cap || y->rank > y->cap) return HT_ERR_CAPACITY;
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
#define CPL(expr)                                              \
  do {                                                         \
    expr;                                                      \
    ++launches;                                                \
    if (cudaGetLastError() != cudaSuccess) {                   \
      htg_ctx_count(c, launches, s);                           \
      return HT_ERR_CUDA;                                      \
    }                                                          \
  } while (0)
  const int fold = (variant == CP_ALS_JACOBI_DAMPED) ? 1 : 0;
  CPL((cp_eps_init_kernel<<<1, 64, 0, s>>>(*w, sweeps)));
  CPL((cp_plan_kernel<<<1, 1, 0, s>>>(a, *w)));
  CPL((cp_normalize_kernel<<<1, 64, 0, s>>>(a, fold)));
  // all G_k, H_k: descriptors 1,2 of every mode; launch each mode's pair (small)
  for (int k = 0; k < d; ++k) {
    if (htg_launch_gemm(w->descs + 3 * k + 1, 2, grid, s) != cudaSuccess) return HT_ERR_CUDA;
    ++launches;
  }
  const size_t solve_smem = ((size_t)a.r * a.r + a.r) * sizeof(double);
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int k = 0; k < d; ++k) {
      CPL((cp_hadamard_kernel<<<32, NT, 0, s>>>(a, *w, k)));
      if (htg_launch_gemm(w->descs + 3 * k, 1, grid, s) != cudaSuccess) return HT_ERR_CUDA;
      ++launches;
      CPL((cp_solve_kernel<<<1, NT, solve_smem, s>>>(a, *w, k, sw, htg_ctx_err(c))));
      if (variant == CP_ALS_GS) {
        if (htg_launch_gemm(w->descs + 3 * k + 1, 2, grid, s) != cudaSuccess) return HT_ERR_CUDA;
        ++launches;
      }
    }
    if (variant == CP_ALS_JACOBI_DAMPED) {
      CPL((cp_damp_kernel<<<dim3(8, d), NT, 0, s>>>(a, *w)));
      for (int k = 0; k < d; ++k) {
        if (htg_launch_gemm(w->descs + 3 * k + 1, 2, grid, s) != cudaSuccess) return HT_ERR_CUDA;
        ++launches;
      }
    }
  }
  if (variant == CP_ALS_JACOBI_DAMPED) CPL((cp_normalize_kernel<<<1, 64, 0, s>>>(a, 0)));
  if (eps_dev && sweeps > 0) CPL((cp_eps_out_kernel<<<1, 64, 0, s>>>(*w, sweeps, eps_dev)));
#undef CPL
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
  NAL((cp_normalize_kernel<<<1, 64, 0, s>>>(a, fold)));
  for (int k = 0; k < d; ++k)
    if (htg_launch_gemm(w.descs + 3 * k + 1, 2, grid, s) != cudaSuccess) return HT_ERR_CUDA;
  const size_t solve_smem = ((size_t)a.r * a.r + a.r) * sizeof(double);
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int k = 0; k < d; ++k) {
      NAL((cp_hadamard_kernel<<<32, NT, 0, s>>>(a, w, k)));
      if (htg_launch_gemm(w.descs + 3 * k, 1, grid, s) != cudaSuccess) return HT_ERR_CUDA;
      NAL((cp_solve_kernel<<<1, NT, solve_smem, s>>>(a, w, k, sw, err)));
      if (variant == CP_ALS_GS && htg_launch_gemm(w.descs + 3 * k + 1, 2, grid, s) != cudaSuccess)
        return HT_ERR_CUDA;
    }
    if (variant == CP_ALS_JACOBI_DAMPED) {
      NAL((cp_damp_kernel<<<dim3(8, d), NT, 0, s>>>(a, w)));
      for (int k = 0; k < d; ++k)
        if (htg_launch_gemm(w.descs + 3 * k + 1, 2, grid, s) != cudaSuccess) return HT_ERR_CUDA;
    }
  }
  if (variant == CP_ALS_JACOBI_DAMPED) NAL((cp_normalize_kernel<<<1, 64, 0, s>>>(a, 0)));
  if (eps_dev && sweeps > 0) NAL((cp_eps_out_kernel<<<1, 64, 0, s>>>(w, sweeps, eps_dev)));
  if (status_dev) NAL((na_status_kernel<<<1, 32, 0, s>>>(err, status_dev)));
#undef NAL
  return HT_OK;
}
