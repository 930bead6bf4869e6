// Householder QR returning the R factor only.
//
// The hierarchical SVD needs, at every node, the triangular factor of the node basis
// (leaves: U_t = Q_t R_t; interior nodes: the (k1 k2) x k matricisation of the
// transfer tensor after absorbing the children's R factors) and the triangular factor
// of the top-down complement factors.  Only R is needed: the orthonormal factors are
// never formed.  Householder reflections keep R backward stable for rank-deficient
// inputs (leaf bases [U, A U, A^2 U] with more columns than grid points are exactly
// rank deficient), where Cholesky-based QR would break down.
//
// One CTA per matrix; the matrix is copied into a scratch buffer and reduced in place
// (L2 resident).  For column j: the norm of the sub-column is reduced across the CTA,
// the reflector v = x - alpha e1 (alpha = -sign(x0)|x|) is formed in place and every
// trailing column (one warp each) gets c <- c - tau (v.c) v with tau = 2 / (v.v).
#include "common.cuh"

namespace {

constexpr int NT = 256;

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int QR_MAX_COLS = 4096;

__global__ void __launch_bounds__(NT) qr_r_kernel(const QrDesc* __restrict__ descs, long long inst_stride,
                                                 long long smem_doubles, double* flops) {
  // batched launches: instance blockIdx.y reads its own descriptor list, inst_stride bytes on
  const QrDesc q = ((const QrDesc*)((const char*)descs + inst_stride * blockIdx.y))[blockIdx.x];
  const int m = q.m, k = q.k;
  if (m <= 0 || k <= 0 || k > QR_MAX_COLS) {
    if (threadIdx.x == 0 && q.rows_out) *q.rows_out = 0;
    return;
  }
  extern __shared__ double diag[];   // min(m,k) values, then the matrix when it fits
  const long long need = (long long)m * k;
  double* S = (need <= smem_doubles - QR_MAX_COLS) ? diag + QR_MAX_COLS : q.scratch;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  // copy op(A) into S (m x k, column major)
  const long long mk = (long long)m * k;
  for (long long e = tid; e < mk; e += NT) {
    const int i = (int)(e % m), c = (int)(e / m);
    S[e] = q.tA ? q.A[c + (long long)q.lda * i] : q.A[i + (long long)q.lda * c];
  }
  __shared__ double red[NT / 32];
  __shared__ double sh_alpha, sh_tau;
  __syncthreads();
  const int rmax = htg_min(m, k);
  for (int j = 0; j < rmax; ++j) {
    double* col = S + (long long)m * j;
    double s = 0.0;
    for (int i = j + 1 + tid; i < m; i += NT) s += col[i] * col[i];
    s = warp_sum(s);
    if (lane == 0) red[wid] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w];
      const double x0 = col[j];
      const double n2 = fma(x0, x0, t);
      double alpha = 0.0, tau = 0.0;
      if (htg_dpos(n2)) {
        const double ri = htg_rsqrt_fast(n2);
        const double nrm = n2 * ri;
        alpha = htg_dpos(x0) ? -nrm : nrm;
        const double v0 = x0 - alpha;
        const double vv = fma(v0, v0, t);
        tau = htg_dpos(vv) ? 2.0 * htg_rcp_fast(vv) : 0.0;
        col[j] = v0;
      }
      sh_alpha = alpha;
      sh_tau = tau;
      diag[j] = alpha;
    }
    __syncthreads();
    const double tau = sh_tau;
    if (htg_dnz(tau)) {
      for (int c = j + 1 + wid; c < k; c += nw) {
        double* cc = S + (long long)m * c;
        double dot = 0.0;
        for (int i = j + lane; i < m; i += 32) dot += col[i] * cc[i];
        dot = warp_sum(dot) * tau;
        for (int i = j + lane; i < m; i += 32) cc[i] -= dot * col[i];
      }
    }
    __syncthreads();
  }
  // write R (rmax x k upper trapezoidal) or its transpose
  const long long rk = (long long)rmax * k;
  for (long long e = tid; e < rk; e += NT) {
    const int r = (int)(e % rmax), c = (int)(e / rmax);
    double v = 0.0;
    if (c == r) v = diag[r];
    else if (c > r) v = S[r + (long long)m * c];
    if (q.tR) q.R[c + (long long)q.ldr * r] = v;
    else q.R[r + (long long)q.ldr * c] = v;
  }
  if (tid == 0 && q.rows_out) *q.rows_out = rmax;
  if (tid == 0 && flops) {
    // norm of the sub-column (2 per entry) + dot and update of every trailing column (4 per entry)
    double f = 0.0;
    for (int j = 0; j < rmax; ++j) f += 2.0 * (m - j) + 4.0 * (double)(m - j) * (k - j - 1);
    atomicAdd(flops, f);
  }
}

}  // namespace

cudaError_t htg_launch_qr(const QrDesc* descs_dev, int ndesc, cudaStream_t s, double* flops, int count,
                          long long inst_stride) {
  if (ndesc <= 0 || count <= 0) return cudaSuccess;
  if (count > 65535) return cudaErrorInvalidValue;
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(qr_r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HTG_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  // diag[] (QR_MAX_COLS values) followed by the staged matrix when it fits
  qr_r_kernel<<<dim3(ndesc, count), NT, HTG_SMEM_BYTES, s>>>(descs_dev, inst_stride,
                                                               (long long)(HTG_SMEM_BYTES / sizeof(double)), flops);
  return cudaGetLastError();
}
