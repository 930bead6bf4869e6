// Internal declarations shared by the translation units of the htgpu library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/htgpu.h"

#define HTG_WARP 32
// dynamic shared memory a single-CTA-per-matrix kernel may request (sm_103a allows 227 KB)
#define HTG_SMEM_BYTES (200 * 1024)
// largest number of column pairs in one Jacobi round (node factors up to 2 * HTG_SVD_MAXP
// columns); their rotation parameters live in static shared memory next to the dynamic part
#define HTG_SVD_MAXP 1024

// ------------------------------------------------------------------ tree ----
struct TreeInfo {
  int d;
  int nn;                        // 2d - 1
  int lo[HT_MAXNODES], hi[HT_MAXNODES];
  int c1[HT_MAXNODES], c2[HT_MAXNODES];
  int parent[HT_MAXNODES], depth[HT_MAXNODES];
  int max_depth;
};
void htg_build_tree(int d, int kind, TreeInfo* t);   // kind: ht_tree_kind

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
// m*k values.  rows_out (optional) receives min(m,k).  With a ticket, tall matrices are
// reduced in row blocks by several CTAs and a combine step (the launch resets the ticket).
struct QrDesc {
  const double* A;
  double* scratch;
  double* R;
  int* rows_out;
  unsigned* ticket;   // zero-initialised counter of the two-stage form (null: one CTA per matrix)
  int m, k, lda, ldr;
  int tA, tR;
};

// One-sided Jacobi SVD of M = P^T where P (p x q, ldp) is given.  Rows of M beyond q
// (when q < p) are treated as zero.  Outputs: sigma (p, descending), V (p x p, ldv = p)
// = left singular vectors of P, U (q x p, ldu = q) = right singular vectors of P with
// unit columns (zero for sigma = 0).  work: 2.5 max(p,q) p + 3.5 p^2 + p + 2 values.
struct SvdDesc {
  const double* P;
  double* sigma;
  double* V;
  double* U;
  double* work;
  int p, q, ldp;
  // Pairs of columns whose squared norms are both below skip2 |P|_F^2 / p are not rotated
  // against each other.  With skip2 |P|_F^2 <= half the truncation threshold (tol |u|)^2 / (2d-3)
  // those columns hold at most half the threshold together, so the rank rule discards all of
  // them, and the tail sums they enter are traces of that block, which rotations within the
  // block do not change.  0: rotate every pair.
  double skip2;
};

// ------------------------------------------------------------ launchers -----
// All launchers return cudaGetLastError() of their launch.
// flops (device double, or nullptr): the kernels add the FP64 flops they execute.
// Batched form (count > 1): instance i (blockIdx.y) reads its ndesc descriptors at
// descs_dev + i * inst_stride bytes.
// tc_min > 0 (HT_PREC_MIXED): the launch skips descriptors of at least tc_min multiply-adds
// (m n k batch), which the tensor-core launch of the same list takes.
cudaError_t htg_launch_gemm(const GemmDesc* descs_dev, int ndesc, int grid, cudaStream_t s, double* flops = nullptr,
                            int count = 1, long long inst_stride = 0, long long tc_min = 0);
// The same descriptor lists in HT_PREC_MIXED's split-FP32 form (the contractions below tc_min
// multiply-adds, all when tc_min <= 0): FP64 operands split into FP32 hi / lo parts, a
// double-float accumulation on the FP32 pipe, at most about 2^-47 (k^2 + 5k + 10) sum |a_i b_i| of
// error, about 2^-47 (k/2 + 10) sum |a_i b_i| in practice.
cudaError_t htg_launch_gemm_f32x2(const GemmDesc* descs_dev, int ndesc, int grid, cudaStream_t s, double* flops,
                                  int count, long long inst_stride, long long tc_min);
// Tensor-core form of the same descriptor lists (HT_PREC_MIXED): `slices` (2..4) BF16 digit planes
// per operand row / column, FP32 accumulation in tensor memory, one CTA per SM (a batch spreads
// them over its instances).  flops (device, or nullptr) accumulates the executed MMA flops.
// err (device, or nullptr): HT_ERR_TIMEOUT when a bounded wait gave up.
// Only descriptors of at least tc_min multiply-adds are taken (0: all).
cudaError_t htg_launch_gemm_tc(const GemmDesc* descs_dev, int ndesc, int sms, int slices, cudaStream_t s,
                               double* flops = nullptr, int count = 1, long long inst_stride = 0, int* err = nullptr,
                               long long tc_min = 0);
// Workspace of the cooperative QR (one instance per launch): per grid position s (the CTAs of a
// matrix sit at consecutive positions) partial dot products in two buffers by column parity
// part[((j & 1) QR_COOP_SLOTS + s) kmax + c] and, after them, the partial Gram blocks of the
// panels' trailing updates part[2 QR_COOP_SLOTS kmax + s QR_COOP_QB (QR_COOP_QB + kmax) + ...];
// per descriptor d totals tot[d kmax + c], the published row j in two buffers by step parity
// rowj[(2 d + (j & 1)) kmax + c], the diagonal of R diag[d kmax + c], the panel's reduced Gram
// block and W wtot[d QR_COOP_QB (QR_COOP_QB + kmax) + ...]; barrier words bar[s] (zeroed by the
// launcher).
constexpr int QR_COOP_QB = 16;       // panel width (columns whose reflectors are applied together)
constexpr int QR_COOP_SLOTS = 256;   // grid positions the workspace serves (at least the SMs)
struct QrCoopWs {
  double* part;
  double* tot;
  double* rowj;
  double* diag;
  unsigned* bar;
  double* wtot;
  int* err;
  int kmax;     // largest k
  int ndmax;    // largest descriptor count of one launch
  int gmax;     // largest CTA group
};
cudaError_t htg_launch_qr(const QrDesc* descs_dev, int ndesc, cudaStream_t s, double* flops = nullptr, int count = 1,
                          long long inst_stride = 0, const QrCoopWs* coop = nullptr);
// Cluster form of the node SVD (wide node factors, one instance per launch): cl CTAs of one
// thread-block cluster share a factor's columns in distributed shared memory.  cl = 0: not
// available (no cluster of 8 or 16 CTAs with the shared memory it needs fits this device).
struct SvdClusterCfg {
  int cl = 0;
  long long cap_doubles = 0;   // shared memory of one CTA of the cluster form, in doubles
  int min_p = 128;             // node factors at least this wide take the cluster form
};
SvdClusterCfg htg_svd_cluster_setup(int device);
// Cluster form of the persistent CP-ALS kernel: the largest cluster (up to 16 CTAs, each with
// its SM's whole shared memory) one of which fits the device, 0 when none does.
struct CpClusterCfg {
  int max_q = 0;
  long long cap_doubles = 0;   // dynamic shared memory of one CTA, in doubles
};
CpClusterCfg htg_cp_cluster_setup(int device);
// whether htg_launch_svd adds the cluster launch (for the launch count)
bool htg_svd_cluster_used(const SvdClusterCfg* clu, int count, int pmax);
// With clu (count = 1 only), node factors the cluster form takes (p >= 128 and fitting its shared
// memory) run in a second launch, one cluster each; the one-CTA kernel skips them.
cudaError_t htg_launch_svd(const SvdDesc* descs_dev, int ndesc, int use_smem, int pmax, int qmax,
                           cudaStream_t s, double* flops = nullptr, int count = 1, long long inst_stride = 0,
                           const SvdClusterCfg* clu = nullptr);

// ------------------------------------------------------------ helpers -------
__host__ __device__ inline int htg_min(int a, int b) { return a < b ? a : b; }
__host__ __device__ inline int htg_max(int a, int b) { return a > b ? a : b; }
__host__ __device__ inline int htg_cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ inline long long htg_max_ll(long long a, long long b) { return a > b ? a : b; }

// HT_PREC_MIXED: contractions of at least this many multiply-adds go to the tensor cores unless the
// context is given a tuned threshold (ht_config.tc_min_work)
// (the autotuner's crossover on GB300 against the FP64 kernel at 16 CTAs per SM: about 2^26)
#define HTG_TC_MIN_WORK_DEFAULT (1ll << 26)

// ------------------------------------------------------- FP64 special values ---
// Measured on GB300 (dependent chains): FP64 FMA 64 cycles, FP64 sqrt 674, divide / rsqrt
// 429, a double<->float conversion about 400 and an FP64 compare-and-select about 800,
// against 4.5 - 70 cycles for their FP32 and integer counterparts.  The helpers below keep
// FP64 compares and conversions out of hot loops: comparisons act on the IEEE bit patterns
// (ordered 64-bit integers), conversions move exponent and mantissa bits with integer
// instructions, and reciprocal (square) roots take an FP32 seed refined by two FP64
// Newton-Raphson steps (each squares the relative error; 2e-7 -> 6e-14 -> rounding level).

// a > 0 (and not -0, NaN counts as positive)
__device__ inline bool htg_dpos(double a) { return __double_as_longlong(a) > 0; }
// a > b for a, b >= 0
__device__ inline bool htg_dgt_nn(double a, double b) { return __double_as_longlong(a) > __double_as_longlong(b); }
// 0 < a < inf (false for NaN, zero, negative)
__device__ inline bool htg_dpos_finite(double a) {
  const long long b = __double_as_longlong(a);
  return b > 0 && b < 0x7FF0000000000000ll;
}
// a != 0 (either sign)
__device__ inline bool htg_dnz(double a) { return (__double_as_longlong(a) << 1) != 0; }
__device__ inline double htg_dabs(double a) { return __longlong_as_double(__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFll); }
// |a| > |b|
__device__ inline bool htg_dabs_gt(double a, double b) {
  return (__double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFll) > (__double_as_longlong(b) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ inline double htg_dmax_nn(double a, double b) { return htg_dgt_nn(a, b) ? a : b; }

// double -> float by truncating the mantissa; |x| outside the FP32 normal range gives +-0 / +-inf
__device__ inline float htg_d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF) - 1023 + 127;
  if (e <= 0) return __int_as_float((int)sign);
  if (e >= 255) return __int_as_float((int)(sign | 0x7F800000u));
  return __int_as_float((int)(sign | ((unsigned int)e << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu)));
}
// float -> double, exact for normal floats and zero (FP32 denormals become 0)
__device__ inline double htg_f2d(float f) {
  const unsigned int u = (unsigned int)__float_as_int(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0) return __longlong_as_double((long long)sign);
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  const unsigned long long ee = (e == 255) ? 0x7FF0000000000000ull : (unsigned long long)(e - 127 + 1023) << 52;
  return __longlong_as_double((long long)(sign | ee | m));
}
// exponent test without FP64 compares: 2^-120 <= |x| < 2^120
__device__ inline bool htg_in_f32_range(double x) {
  const int e = (int)((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7FF) - 1023;
  return e > -120 && e < 120;
}
__device__ inline double htg_rsqrt_fast(double x) {
  if (!htg_in_f32_range(x) || !htg_dpos(x)) return rsqrt(x);
  const double y = htg_f2d(rsqrtf(htg_d2f(x)));
  // with e = 1 - x y^2 (|e| <~ 2^-21 from the FP32 seed of the truncated input):
  // x^-1/2 = y (1 - e)^-1/2 = y (1 + e/2 + 3 e^2/8 + O(e^3)); the O(e^3) term is below 2^-62,
  // so five dependent FP64 operations give the result to rounding (Jacobi rotations need
  // c^2 + s^2 = 1 to rounding)
  const double h = x * y;
  const double e = fma(-h, y, 1.0);
  const double q = fma(0.375, e, 0.5) * e;
  return fma(y, q, y);
}
// float of x 2^k (truncated mantissa) when x 2^k lies in the normal FP32 range, for a power-of-
// two rescaling without an FP64 multiply; *ok = false (and 0 returned) otherwise, x = 0 included
__device__ inline float htg_d2f_shift(double x, int k, bool* ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF) - 1023 + k + 127;
  if ((b << 1) == 0 || e <= 8 || e >= 247) {   // zero, or outside [2^-118, 2^119]
    *ok = false;
    return 0.0f;
  }
  *ok = true;
  return __int_as_float((int)(sign | ((unsigned int)e << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu)));
}
__device__ inline double htg_rcp_fast(double x) {
  if (!htg_in_f32_range(x)) return 1.0 / x;
  // seed: the approximate FP32 reciprocal (one special-function instruction, relative error
  // about 2^-23 on normal inputs; the range test keeps the input and its reciprocal normal)
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(htg_d2f(x)));
  const double y = htg_f2d(yf);
  // with e = 1 - x y (|e| <~ 2^-22): 1/x = y / (1 - e) = y (1 + e + e^2 + O(e^3)); the O(e^3)
  // term is below 2^-64, so three dependent FP64 operations give the reciprocal to rounding
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
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
  double* acc2;    // 2 doubles: per-mode sums of the convergence measure (persistent kernel)
  unsigned int* bar;   // 64 words: grid barrier arrival sequence numbers, one per CTA
  double* ZT;      // HT_MAXD x 3 rcap x nmax   the powers transposed (the cluster form's M_k rows)
  int rcap, rycap, nmax;
};
CpWs* htg_ctx_cp(ht_ctx* c);
int htg_ctx_d(const ht_ctx* c);
const int* htg_ctx_n(const ht_ctx* c);
int* htg_ctx_err(ht_ctx* c);
int htg_ctx_grid(const ht_ctx* c);
int htg_ctx_cp_form(const ht_ctx* c);   // ht_config.cp_form
const CpClusterCfg* htg_ctx_cp_cluster(const ht_ctx* c);
int htg_ctx_cap(const ht_ctx* c);
int htg_ctx_max_terms(const ht_ctx* c);
int htg_ctx_device(const ht_ctx* c);
void** htg_ctx_cn_ws(ht_ctx* c, size_t** bytes);   // lazily allocated Crank-Nicolson ALS workspace
void htg_ctx_count(ht_ctx* c, int launches, cudaStream_t s);
int htg_cp_terms(int d);   // 1 + 2d + d(d-1)/2

// ------------------------------------------------------------ profiling --------
// Kernel classes of the opt-in event profiler (ht_ctx_profile / ht_ctx_profile_read).
// KC_GEMMTC: the tensor-core contractions of HT_PREC_MIXED; their counter holds the executed MMA
// flops (BF16 digit products over whole 128 x 128 tiles), not FP64-equivalent ones.
enum HtgKernelClass { KC_APPLY = 0, KC_GEMM = 1, KC_QR = 2, KC_SVD = 3, KC_PLAN = 4, KC_CPSMALL = 5,
                      KC_CPSOLVE = 6, KC_GEMMTC = 7, KC_COUNT = 8 };
void htg_prof_begin(ht_ctx* c, cudaStream_t s);
void htg_prof_end(ht_ctx* c, int cls, cudaStream_t s);
double* htg_prof_flops(ht_ctx* c, int cls);   // device counter of a class, nullptr when off
