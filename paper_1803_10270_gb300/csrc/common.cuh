// Internal declarations shared by the translation units of the htgpu library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/htgpu.h"

#define HTG_WARP 32
// dynamic shared memory a single-CTA-per-matrix kernel may request (sm_103a allows 227 KB)
#define HTG_SMEM_BYTES (200 * 1024)

// ------------------------------------------------------------------ tree ----
struct TreeInfo {
  int d;
  int nn;                        // 2d - 1
  int lo[HT_MAXNODES], hi[HT_MAXNODES];
  int c1[HT_MAXNODES], c2[HT_MAXNODES];
  int parent[HT_MAXNODES], depth[HT_MAXNODES];
  int max_depth;
};
void htg_build_tree(int d, TreeInfo* t);

// --------------------------------------------------------- work descriptors --
// Batched GEMM: C[b] = alpha * op(A[b]) * op(B[b]) * diag(colscale) + beta * C[b],
// op(A) is m x k, op(B) is k x n, column-major; b = 0..batch-1 with strides sA/sB/sC.
struct GemmDesc {
  const double* A;
  const double* B;
  double* C;
  const double* colscale;   // n values or nullptr
  long long sA, sB, sC;
  int m, n, k;
  int lda, ldb, ldc;
  int batch;
  int tA, tB;
  double alpha, beta;
};

// Householder QR, R factor only.  Input op(A) is m x k (tA: A stored k x m, lda between
// columns of the stored array).  Output R is min(m,k) x k upper trapezoidal written to
// R (ldr); with tR the transpose R^T (k x min(m,k)) is written instead.  scratch holds
// m*k values.  rows_out (optional) receives min(m,k).
struct QrDesc {
  const double* A;
  double* scratch;
  double* R;
  int* rows_out;
  int m, k, lda, ldr;
  int tA, tR;
};

// One-sided Jacobi SVD of M = P^T where P (p x q, ldp) is given.  Rows of M beyond q
// (when q < p) are treated as zero.  Outputs: sigma (p, descending), V (p x p, ldv = p)
// = left singular vectors of P, U (q x p, ldu = q) = right singular vectors of P with
// unit columns (zero for sigma = 0).  work: (max(p,q) + p) * p values.
struct SvdDesc {
  const double* P;
  double* sigma;
  double* V;
  double* U;
  double* work;
  int p, q, ldp;
};

// ------------------------------------------------------------ launchers -----
// All launchers return cudaGetLastError() of their launch.
// flops (device double, or nullptr): the kernels add the FP64 flops they execute.
cudaError_t htg_launch_gemm(const GemmDesc* descs_dev, int ndesc, int grid, cudaStream_t s, double* flops = nullptr);
cudaError_t htg_launch_qr(const QrDesc* descs_dev, int ndesc, cudaStream_t s, double* flops = nullptr);
cudaError_t htg_launch_svd(const SvdDesc* descs_dev, int ndesc, int use_smem, int pmax, int qmax,
                           cudaStream_t s, double* flops = nullptr);

// ------------------------------------------------------------ helpers -------
__host__ __device__ inline int htg_min(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int htg_max(int a, int b) { return a > b ? a : b; }
__host__ __device__ inline int htg_cdiv(int a, int b) { return (a + b - 1) / b; }

// ------------------------------------------------------- FP64 special values ---
// On GB300 a dependent FP64 operation costs about 64 cycles and an FP64 sqrt / divide
// several hundred, against 4.5 / 50-70 cycles in FP32.  These helpers take an FP32 seed
// and refine it with one Newton-Raphson step in FP64 (relative error ~ 1.5 e0^2, e0 the
// seed's error of about 6e-8, i.e. ~1e-14).  Outside the FP32 normal range they fall
// back to the FP64 library functions.
__device__ inline double htg_rsqrt_fast(double x) {
  if (!(x > 1e-36 && x < 1e36)) return rsqrt(x);
  const double y = (double)rsqrtf((float)x);
  const double h = x * y;               // Newton for f(y) = 1/y^2 - x:  y <- y (3 - x y^2) / 2
  return fma(0.5 * y, fma(-h, y, 1.0), y);
}
__device__ inline double htg_rcp_fast(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-36 && ax < 1e36)) return 1.0 / x;
  const double y = (double)(1.0f / (float)x);
  return fma(y, fma(-x, y, 1.0), y);    // Newton for f(y) = 1/y - x:  y <- y (2 - x y)
}

// ------------------------------------------------------------ context access ---
// CP-ALS workspace inside an ht_ctx (sized from the context configuration).
struct CpWs {
  double* G;       // d x rcap^2         factor Grams X_j^T X_j
  double* H;       // d x rycap x rcap   cross Grams Y_j^T X_j
  double* Hh;      // rycap x rcap       diag(mu) * hadamard_{j != k} H_j
  double* Gam;     // rcap^2             hadamard_{j != k} G_j
  double* RHS;     // nmax x rcap        Y_k Hh
  double* Xold;    // HT_MAXD x nmax x rcap   iterate copy (Jacobi variant / eps)
  double* wold;    // rcap
  double* epsacc;  // 64 (per-sweep accumulators)
  GemmDesc* descs; // 4 * HT_MAXD
  double* Z;       // HT_MAXD x nmax x 3 rcap   powers [X, A X, A^2 X] of the step's input
  int rcap, rycap, nmax;
};
CpWs* htg_ctx_cp(ht_ctx* c);
int htg_ctx_d(const ht_ctx* c);
const int* htg_ctx_n(const ht_ctx* c);
int* htg_ctx_err(ht_ctx* c);
int htg_ctx_grid(const ht_ctx* c);
void htg_ctx_count(ht_ctx* c, int launches, cudaStream_t s);
int htg_cp_terms(int d);   // 1 + 2d + d(d-1)/2

// ------------------------------------------------------------ profiling --------
// Kernel classes of the opt-in event profiler (ht_ctx_profile / ht_ctx_profile_read).
enum HtgKernelClass { KC_APPLY = 0, KC_GEMM = 1, KC_QR = 2, KC_SVD = 3, KC_PLAN = 4, KC_CPSMALL = 5,
                      KC_CPSOLVE = 6, KC_COUNT = 7 };
void htg_prof_begin(ht_ctx* c, cudaStream_t s);
void htg_prof_end(ht_ctx* c, int cls, cudaStream_t s);
double* htg_prof_flops(ht_ctx* c, int cls);   // device counter of a class, nullptr when off
