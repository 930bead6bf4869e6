// One-sided (Hestenes) Jacobi SVD of the small node factors, FP64.
//
// The hierarchical SVD (Section 2.2) needs the leading singular pairs of every node
// matricisation.  Working with the square-root factor P_t = R_t E_t rather than its Gram
// keeps singular values far below sqrt(eps) * sigma_max accurate, which the relative
// truncation tolerance of 1e-8 requires.
//
// M = P^T (rows padded with zeros to max(p,q)) has its p columns orthogonalised by plane
// rotations in the round-robin (Brent-Luk) order: every round rotates p/2 disjoint pairs
// (one warp per pair, lanes over rows), p-1 rounds form a sweep, sweeps repeat until no
// pair has |a.b| > tol |a||b|.  Rotation: zeta = (|b|^2 - |a|^2) / (2 a.b),
// t = sign(zeta) / (|zeta| + hypot(1, zeta)), c = 1/sqrt(1+t^2), s = c t.
// One CTA per matrix; the working copy lives in shared memory when the capacity allows,
// else in the descriptor's global work buffer (L2 resident).
#include "common.cuh"

namespace {

constexpr int NT = 256;
constexpr int MAX_SWEEPS = 40;
constexpr double TOL = 1e-15;

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline int rr_player(int pos, int round, int p2) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (p2 - 1));
}

__global__ void __launch_bounds__(NT) svd_kernel(const SvdDesc* __restrict__ descs, int use_smem) {
  const SvdDesc D = descs[blockIdx.x];
  const int p = D.p, q = D.q;
  if (p <= 0) return;
  const int mr = htg_max(p, q);
  extern __shared__ double smem[];
  double* M = use_smem ? smem : D.work;
  double* V = M + (long long)mr * p;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  for (long long e = tid; e < (long long)mr * p; e += NT) {
    const int i = (int)(e % mr), c = (int)(e / mr);
    M[e] = (i < q) ? D.P[c + (long long)D.ldp * i] : 0.0;
  }
  for (int e = tid; e < p * p; e += NT) V[e] = (e % p == e / p) ? 1.0 : 0.0;
  __shared__ int rotated;
  __syncthreads();
  const int p2 = p + (p & 1);
  if (p > 1) {
    for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
      if (tid == 0) rotated = 0;
      __syncthreads();
      for (int round = 0; round < p2 - 1; ++round) {
        for (int pi = wid; pi < p2 / 2; pi += nw) {
          int a = rr_player(pi, round, p2), b = rr_player(p2 - 1 - pi, round, p2);
          if (a >= p || b >= p) continue;
          if (a > b) { int t = a; a = b; b = t; }
          double* ca = M + (long long)mr * a;
          double* cb = M + (long long)mr * b;
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int i = lane; i < mr; i += 32) {
            const double x = ca[i], y = cb[i];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
          al = warp_sum(al);
          be = warp_sum(be);
          ga = warp_sum(ga);
          if (ga != 0.0 && fabs(ga) > TOL * sqrt(al) * sqrt(be)) {
            const double zeta = (be - al) / (2.0 * ga);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            const double s = c * t;
            for (int i = lane; i < mr; i += 32) {
              const double x = ca[i], y = cb[i];
              ca[i] = c * x - s * y;
              cb[i] = s * x + c * y;
            }
            double* va = V + (long long)p * a;
            double* vb = V + (long long)p * b;
            for (int i = lane; i < p; i += 32) {
              const double x = va[i], y = vb[i];
              va[i] = c * x - s * y;
              vb[i] = s * x + c * y;
            }
            if (lane == 0) rotated = 1;
          }
        }
        __syncthreads();
      }
      const int any = rotated;
      __syncthreads();
      if (!any) break;
    }
  }
  // column norms, then descending order (ties by index)
  double* nrm = V + (long long)p * p;   // p scratch values after V
  for (int c = wid; c < p; c += nw) {
    const double* cc = M + (long long)mr * c;
    double s = 0.0;
    for (int i = lane; i < mr; i += 32) s = fma(cc[i], cc[i], s);
    s = warp_sum(s);
    if (lane == 0) nrm[c] = sqrt(s);
  }
  __syncthreads();
  for (int c = wid; c < p; c += nw) {
    const double sc = nrm[c];
    int rank = 0;
    for (int o = 0; o < p; ++o) {
      const double so = nrm[o];
      rank += (so > sc) || (so == sc && o < c);
    }
    if (lane == 0) D.sigma[rank] = sc;
    for (int i = lane; i < p; i += 32) D.V[i + (long long)p * rank] = V[i + (long long)p * c];
    const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
    for (int i = lane; i < q; i += 32) D.U[i + (long long)q * rank] = M[i + (long long)mr * c] * inv;
  }
}

}  // namespace

cudaError_t htg_launch_svd(const SvdDesc* descs_dev, int ndesc, int use_smem, int pmax, int qmax,
                           cudaStream_t s) {
  if (ndesc <= 0) return cudaSuccess;
  size_t smem = 0;
  if (use_smem) {
    const int mr = htg_max(pmax, qmax);
    smem = ((size_t)mr * pmax + (size_t)pmax * pmax + pmax) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  svd_kernel<<<ndesc, NT, smem, s>>>(descs_dev, use_smem);
  return cudaGetLastError();
}
