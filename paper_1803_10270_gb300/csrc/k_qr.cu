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
// One CTA per matrix; the matrix is copied into shared memory (or a scratch buffer, L2
// resident, when it does not fit) and reduced in place.  For column j the reflector
// v = x - alpha e1 (alpha = -sign(x0)|x|) is formed in place and every trailing column (one
// warp each) gets c <- c - tau (v.c) v with tau = 2 / (v.v).
#include "common.cuh"

namespace {

constexpr int NT = 256;

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Dynamic shared memory per CTA: 96 KB, so that two CTAs share an SM in batched launches; a
// matrix that does not fit is reduced in its global scratch buffer (L2 resident).
constexpr int QR_SMEM_BYTES = 96 * 1024;

// Householder reflector of column j from x0 = S[j, j] and t = sum_{i > j} S[i, j]^2 (lane 0):
// v = x - alpha e1 with alpha = -sign(x0) |x| stored over S[j, j], alpha into diag[j], and
// tau = 2 / (v.v) (0 when the column is already zero below and on the diagonal).
__device__ inline double reflector(double* colj, int j, double t, double* diag) {
  const double x0 = colj[j];
  const double n2 = fma(x0, x0, t);
  double alpha = 0.0, tau = 0.0;
  if (htg_dpos(n2)) {
    const double ri = htg_rsqrt_fast(n2);
    const double nrm = n2 * ri;
    alpha = htg_dpos(x0) ? -nrm : nrm;
    const double v0 = x0 - alpha;
    const double vv = fma(v0, v0, t);
    tau = htg_dpos(vv) ? 2.0 * htg_rcp_fast(vv) : 0.0;
    colj[j] = v0;
  }
  diag[j] = alpha;
  return tau;
}

// Warp w owns the columns c = w (mod number of warps).  Step j applies reflector j to every
// trailing column c > j (dot product over rows >= j, warp reduction, rank-1 update); the owner
// of column j+1 updates it first and forms reflector j+1 at once (look-ahead), while the other
// warps are still updating their columns, so the reflector's serial FP64 chain (norm, square
// root, reciprocal) stays off the critical path.  One CTA barrier per step.
__global__ void __launch_bounds__(NT) qr_r_kernel(const QrDesc* __restrict__ descs, long long inst_stride,
                                                 long long smem_doubles, double* flops) {
  // batched launches: instance blockIdx.y reads its own descriptor list, inst_stride bytes on
  const QrDesc q = ((const QrDesc*)((const char*)descs + inst_stride * blockIdx.y))[blockIdx.x];
  const int m = q.m, k = q.k;
  const int kd = (k + 1) & ~1;   // diagonal entries, rounded to keep the matrix 16-byte aligned
  if (m <= 0 || k <= 0 || kd > smem_doubles) {
    if (threadIdx.x == 0 && q.rows_out) *q.rows_out = 0;
    return;
  }
  extern __shared__ double diag[];   // the k diagonal entries of R, then the matrix when it fits
  const long long need = (long long)m * k;
  double* S = (need <= smem_doubles - kd) ? diag + kd : q.scratch;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  // copy op(A) into S (m x k, column major)
  const long long mk = (long long)m * k;
  for (long long e = tid; e < mk; e += NT) {
    const int i = (int)(e % m), c = (int)(e / m);
    S[e] = q.tA ? q.A[c + (long long)q.lda * i] : q.A[i + (long long)q.lda * c];
  }
  __shared__ double tau_sh[2];
  __syncthreads();
  const int rmax = htg_min(m, k);
  // reflector 0 by the owner of column 0
  if (wid == 0) {
    double s = 0.0;
    for (int i = 1 + lane; i < m; i += 32) s = fma(S[i], S[i], s);
    s = warp_sum(s);
    if (lane == 0) tau_sh[0] = reflector(S, 0, s, diag);
  }
  __syncthreads();
  for (int j = 0; j < rmax; ++j) {
    const double tau = tau_sh[j & 1];
    const double* v = S + (long long)m * j;
    const int c0 = j + 1 + ((wid - (j + 1)) % nw + nw) % nw;   // this warp's first column > j
    for (int c = c0; c < k; c += nw) {
      double* cc = S + (long long)m * c;
      double dot = 0.0;
      for (int i = j + lane; i < m; i += 32) dot = fma(v[i], cc[i], dot);
      const double wgt = warp_sum(dot) * tau;
      if (c == j + 1 && j + 1 < rmax) {
        // update column j+1 and form reflector j+1 from its new entries
        double ss = 0.0;
        for (int i = j + lane; i < m; i += 32) {
          const double x = fma(-wgt, v[i], cc[i]);
          cc[i] = x;
          if (i > j + 1) ss = fma(x, x, ss);
        }
        ss = warp_sum(ss);
        __syncwarp();
        if (lane == 0) tau_sh[(j + 1) & 1] = reflector(cc, j + 1, ss, diag);
        __syncwarp();
      } else {
        for (int i = j + lane; i < m; i += 32) cc[i] = fma(-wgt, v[i], cc[i]);
      }
    }
    __syncthreads();
  }
  // write R (rmax x k upper trapezoidal) or its transpose
  const long long rk = (long long)rmax * k;
  for (long long e = tid; e < rk; e += NT) {
    const int r = (int)(e % rmax), c = (int)(e / rmax);
    double val = 0.0;
    if (c == r) val = diag[r];
    else if (c > r) val = S[r + (long long)m * c];
    if (q.tR) q.R[c + (long long)q.ldr * r] = val;
    else q.R[r + (long long)q.ldr * c] = val;
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
    cudaError_t e = cudaFuncSetAttribute(qr_r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, QR_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  qr_r_kernel<<<dim3(ndesc, count), NT, QR_SMEM_BYTES, s>>>(descs_dev, inst_stride,
                                                              (long long)(QR_SMEM_BYTES / sizeof(double)), flops);
  return cudaGetLastError();
}
