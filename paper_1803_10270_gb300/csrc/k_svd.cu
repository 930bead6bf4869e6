// One-sided (Hestenes) Jacobi SVD of the small node factors, FP64.
//
// The hierarchical SVD (Section 2.2) needs the leading singular pairs of every node
// matricisation.  Working with the square-root factor P_t = R_t E_t rather than its Gram
// keeps singular values far below sqrt(eps) * sigma_max accurate, which the relative
// truncation tolerance of 1e-8 requires.
//
// M = P^T (rows padded with zeros to max(p,q)) has its p columns orthogonalised by plane
// rotations in the round-robin (Brent-Luk) order: every round rotates p/2 disjoint pairs
// (a group of lanes per pair, lanes over rows), p-1 rounds form a sweep, sweeps repeat until no
// pair has |a.b| > tol |a||b|, tol = eps * max(m, 8).  Rotation: zeta = (|b|^2 - |a|^2) / (2 a.b),
// t = sign(zeta) / (|zeta| + hypot(1, zeta)), c = 1/sqrt(1+t^2), s = c t.
// One CTA per matrix; the working copy lives in shared memory when the capacity allows,
// else in the descriptor's global work buffer (L2 resident).
#include "common.cuh"

namespace {

constexpr int NT = 512;
constexpr int MAX_SWEEPS = 30;
constexpr double EPS = 2.220446049250313e-16;

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline int rr_player(int pos, int round, int p2) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + round) % (p2 - 1));
}

// FP64 cost model of this kernel: each FP64 warp instruction occupies the SM's FP64 pipe
// for the whole warp whatever the number of active lanes.  A column pair is therefore
// handled by a group of L lanes (L a power of two chosen from the column length): the
// lanes split the rows, reduce their partial dot products with log2(L) shuffles, and every
// group computes its own rotation parameters in the same instructions as the others.
__global__ void __launch_bounds__(NT) svd_kernel(const SvdDesc* __restrict__ descs, long long smem_doubles,
                                                double* flops) {
  const SvdDesc D = descs[blockIdx.x];
  const int p = D.p, q = D.q;
  if (p <= 0) return;
  const int mr = htg_max(p, q);
  extern __shared__ double smem[];
  // working copy in shared memory when the ACTUAL sizes fit, else in the global work buffer
  const long long need = (long long)mr * p + (long long)p * p + p;
  double* M = (need <= smem_doubles) ? smem : D.work;
  double* V = M + (long long)mr * p;
  const int tid = threadIdx.x;
  for (long long e = tid; e < (long long)mr * p; e += NT) {
    const int i = (int)(e % mr), c = (int)(e / mr);
    M[e] = (i < q) ? D.P[c + (long long)D.ldp * i] : 0.0;
  }
  for (int e = tid; e < p * p; e += NT) V[e] = (e % p == e / p) ? 1.0 : 0.0;
  __shared__ int rotated;
  const int p2 = p + (p & 1);
  const int npairs = p2 / 2;
  // lanes per pair: about 8 rows per lane, at most 32, and all pairs of a round in one pass
  int L = 1;
  while (L < 32 && L * 8 < htg_max(mr, p)) L <<= 1;
  while (L > 1 && npairs * L > NT) L >>= 1;
  const int gid = tid / L, gl = tid % L, ngroups = NT / L;
  const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((tid & 31) & ~(L - 1)));
  double myflops = 0.0;
  const double TOL = EPS * (double)htg_max(mr, 8);
  __syncthreads();
  if (p > 1) {
    for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
      if (tid == 0) rotated = 0;
      __syncthreads();
      for (int round = 0; round < p2 - 1; ++round) {
        for (int pi = gid; pi < npairs; pi += ngroups) {
          int a = rr_player(pi, round, p2), b = rr_player(p2 - 1 - pi, round, p2);
          if (a >= p || b >= p) continue;
          if (a > b) { int t = a; a = b; b = t; }
          double* ca = M + (long long)mr * a;
          double* cb = M + (long long)mr * b;
          double al = 0.0, be = 0.0, ga = 0.0;
          for (int i = gl; i < mr; i += L) {
            const double x = ca[i], y = cb[i];
            al = fma(x, x, al);
            be = fma(y, y, be);
            ga = fma(x, y, ga);
          }
          for (int o = L >> 1; o > 0; o >>= 1) {
            al += __shfl_xor_sync(gmask, al, o);
            be += __shfl_xor_sync(gmask, be, o);
            ga += __shfl_xor_sync(gmask, ga, o);
          }
          if (gl == 0) myflops += 6.0 * mr;
          if (ga != 0.0 && ga * ga > TOL * TOL * al * be) {
            // tan of the rotation angle from an FP32 evaluation of
            // zeta = (be - al) / (2 ga), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)); the angle
            // only steers the iteration, while c = (1 + t^2)^(-1/2) (FP64 Newton) and s = c t keep
            // every rotation orthogonal to FP64 accuracy
            const double diff = be - al;
            double t;
            const double ag = fabs(ga), ad = fabs(diff);
            if (ag > 1e-30 && ag < 1e30 && ad < 1e30) {
              const float zf = (float)diff / (2.0f * (float)ga);
              const float azf = fabsf(zf);
              const float tf = (azf > 1e18f) ? 0.5f / zf : copysignf(1.0f, zf) / (azf + sqrtf(fmaf(zf, zf, 1.0f)));
              t = (double)tf;
            } else {
              const double zeta = diff / (2.0 * ga);
              const double az = fabs(zeta);
              t = (az > 1e150) ? 0.5 / zeta : (zeta >= 0.0 ? 1.0 : -1.0) / (az + sqrt(fma(zeta, zeta, 1.0)));
            }
            const double c = htg_rsqrt_fast(fma(t, t, 1.0));
            const double s = c * t;
            for (int i = gl; i < mr; i += L) {
              const double x = ca[i], y = cb[i];
              ca[i] = c * x - s * y;
              cb[i] = s * x + c * y;
            }
            double* va = V + (long long)p * a;
            double* vb = V + (long long)p * b;
            for (int i = gl; i < p; i += L) {
              const double x = va[i], y = vb[i];
              va[i] = c * x - s * y;
              vb[i] = s * x + c * y;
            }
            if (gl == 0) {
              rotated = 1;
              myflops += 6.0 * mr + 6.0 * p;
            }
          }
        }
        __syncthreads();
      }
      const int any = rotated;
      __syncthreads();
      if (!any) break;
    }
  }
  if (flops && gl == 0 && myflops > 0.0) atomicAdd(flops, myflops);
  // column norms, then descending order (ties by index)
  const int lane = tid & 31, wid = tid >> 5, nw = NT / 32;
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
                           cudaStream_t s, double* flops) {
  if (ndesc <= 0) return cudaSuccess;
  (void)use_smem;
  const int mr = htg_max(pmax, qmax);
  size_t smem = ((size_t)mr * pmax + (size_t)pmax * pmax + pmax) * sizeof(double);
  if (smem > HTG_SMEM_BYTES) smem = HTG_SMEM_BYTES;
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HTG_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  svd_kernel<<<ndesc, NT, smem, s>>>(descs_dev, (long long)(smem / sizeof(double)), flops);
  return cudaGetLastError();
}
