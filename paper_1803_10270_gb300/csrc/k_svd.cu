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
// else in the descriptor's global work buffer (L2 resident).  Factors of 128 columns and more
// go to the cluster form further down (one thread-block cluster per matrix).
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

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

// Cost model (measured on GB300): every FP64 warp instruction holds its SM partition's FP64
// pipe for 64 cycles whatever the number of active lanes (FP32: 4.5 cycles latency, 32 lanes
// per clock), FP64 sqrt / divide several hundred.  The SVD therefore runs in phases:
//  1. one-sided Jacobi entirely in FP32 on a scaled copy of M, accumulating V32 (cheap
//     sweeps until |a.b| <= tol32 |a||b|);
//  2. V32 is made orthogonal to FP64 accuracy by two Newton-Schulz steps
//     V <- V (3 I - V^T V) / 2, then G = (M V)^T (M V) is formed in FP64; its off-diagonal
//     part is now ~tol32 relative, so two-sided Jacobi on G (rotations applied to rows, then
//     columns, of G and to V) converges in a few FP64 sweeps while every entry keeps its
//     relative accuracy (no cancellation with small rotation angles);
//  3. U S = M V in FP64, S = column norms, sorted descending.
// Rotation parameters: angle from an FP32 evaluation, c = (1 + t^2)^(-1/2) by an FP64 Newton
// step and s = c t, so each FP64 rotation is orthogonal to FP64 accuracy.

// round-robin pair (a < b) of position pi in a round, or a = -1 for a dummy player
__device__ inline void rr_pair(int pi, int round, int p, int p2, int* a, int* b) {
  int x = rr_player(pi, round, p2), y = rr_player(p2 - 1 - pi, round, p2);
  if (x > y) { int t = x; x = y; y = t; }
  *a = (y >= p) ? -1 : x;
  *b = y;
}

// dst (r x c, ld r) = A (r x k, ld lda) * B (k x c, ld ldb), FP64, whole CTA
__device__ void cta_gemm(double* dst, const double* A, int lda, const double* B, int ldb, int r, int c, int k,
                         bool transA) {
  for (int e = threadIdx.x; e < r * c; e += blockDim.x) {
    const int i = e % r, j = e / r;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int l = 0;
    for (; l + 3 < k; l += 4) {
      const double a0 = transA ? A[l + lda * i] : A[i + lda * l];
      const double a1 = transA ? A[l + 1 + lda * i] : A[i + lda * (l + 1)];
      const double a2 = transA ? A[l + 2 + lda * i] : A[i + lda * (l + 2)];
      const double a3 = transA ? A[l + 3 + lda * i] : A[i + lda * (l + 3)];
      s0 = fma(a0, B[l + ldb * j], s0);
      s1 = fma(a1, B[l + 1 + ldb * j], s1);
      s2 = fma(a2, B[l + 2 + ldb * j], s2);
      s3 = fma(a3, B[l + 3 + ldb * j], s3);
    }
    for (; l < k; ++l) s0 = fma(transA ? A[l + lda * i] : A[i + lda * l], B[l + ldb * j], s0);
    dst[i + r * j] = (s0 + s1) + (s2 + s3);
  }
}

// ------------------------------------------------------------ cluster form -----
// Wide node factors (p >= SVDC_MIN_P columns) are taken by one thread-block cluster of cl CTAs
// (16, else 8): column j of N = M V (its q rows; the rows of M past q are zero and stay zero)
// and of V (p rows) lives in the shared memory of CTA j mod cl, slot j / cl, with |N_j|^2 beside
// it.  Every Brent-Luk round, pair pi goes to CTA pi mod cl, one warp per pair, which reads and
// rotates both columns where they live (distributed shared memory) and writes their new squared
// norms; a cluster barrier ends the round.  The rotations are the one-sided (Hestenes) ones of
// the FP64 phase above, applied to N directly: no FP32 phase and no Gram matrix, so each sweep is
// one pass over the column pairs, and its FP64 work is spread over cl SMs.  A rotated pair's V
// columns (rows q .. q + p - 1, which no dot product reads) are rotated one round late, by the
// same warp at the start of the next round: the round barrier that follows orders them before
// any later rotation of those columns, and a round's critical path is one pair's N work plus at
// most one earlier V update instead of both halves of a rotation.
constexpr int SVDC_MIN_P = 128;
constexpr int CNT = 512;                 // threads per CTA
constexpr int CNW = CNT / 32;            // warps per CTA = pairs one CTA rotates at a time
constexpr int CREG = 15;                 // N entries a lane holds in registers: q <= 32 * CREG
constexpr int SVDC_MAXQ = 32 * CREG;

__host__ __device__ inline long long svdc_smem_doubles(int p, int q, int cl) {
  const long long ncol = (p + cl - 1) / cl;
  return ncol * (long long)(p + q) + ncol + p + 8;
}

// whether the cluster form takes a p x q node factor (the one-CTA kernel skips exactly these);
// min_p: the width from which factors go to the cluster form (SVDC_MIN_P unless tuned)
__host__ __device__ inline bool svdc_takes(int p, int q, int cl, long long cap_doubles, int min_p) {
  return cl > 0 && p >= min_p && p <= SVDC_MAXQ && q >= 1 && q <= SVDC_MAXQ &&
         svdc_smem_doubles(p, q, cl) <= cap_doubles;
}

__device__ inline int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The sweeps, with the KQ = ceil(q / 32) N entries of a lane in registers (a compile-time count,
// so no FP64 instruction is issued for rows past q: an FP64 warp instruction costs the same with
// one lane active as with 32).
template <int KQ>
__device__ void svdc_sweeps(cg::cluster_group& cluster, double* col, double* nrm, double* flag, int p, int q, int cl,
                            double floor2, double skip_abs, int sh2, float rnd2, double* myflops) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int me = (int)cluster.block_rank();
  const int ld = q + p;
  const int p2 = p + (p & 1), npairs = p2 / 2;
  // the pair test |a.b| > tol |a| |b|: tol = eps max(p, q) when the singular values are reported,
  // at least 1e-11 when only the truncation's ranks are wanted (skip_abs > 0): a pair left
  // unrotated at that level moves T(u) by at most about 1e-11 of its smaller column
  const float TOL64F = htg_d2f(skip_abs > 0.0 ? fmax(EPS * (double)htg_max(htg_max(p, q), 8), 1e-11)
                                              : EPS * (double)htg_max(htg_max(p, q), 8));
  __shared__ int rot_sh;
  // this warp's rotation of the previous round whose V columns are still to rotate
  double* pva = nullptr;
  double* pvb = nullptr;
  double pc = 1.0, ps = 0.0;
  auto rotate_v = [&]() {
    if (!pva) return;
    for (int i0 = 0; i0 < p; i0 += 160) {
      double x[5], y[5];
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        const int i = i0 + lane + 32 * u;
        x[u] = (i < p) ? pva[i] : 0.0;
        y[u] = (i < p) ? pvb[i] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 5; ++u) {
        const int i = i0 + lane + 32 * u;
        if (i < p) {
          pva[i] = pc * x[u] - ps * y[u];
          pvb[i] = ps * x[u] + pc * y[u];
        }
      }
    }
    pva = pvb = nullptr;
  };
  for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
    if (tid == 0) rot_sh = 0;
    __syncthreads();
    for (int round = 0; round < p2 - 1; ++round) {
      rotate_v();
      for (int pi = me + cl * wid; pi < npairs; pi += cl * CNW) {
        int a, b;
        rr_pair(pi, round, p, p2, &a, &b);
        if (a < 0) continue;
        double* ca = cluster.map_shared_rank(col + (long long)(a / cl) * ld, a % cl);
        double* cb = cluster.map_shared_rank(col + (long long)(b / cl) * ld, b % cl);
        double* na = cluster.map_shared_rank(nrm + a / cl, a % cl);
        double* nb = cluster.map_shared_rank(nrm + b / cl, b % cl);
        const double al = *na, be = *nb;
        // the rounding floor and the discard-level skip of the one-CTA kernel
        if (!(htg_dgt_nn(al, floor2) && htg_dgt_nn(be, floor2) &&
              (htg_dgt_nn(al, skip_abs) || htg_dgt_nn(be, skip_abs))))
          continue;
        double xa[KQ], xb[KQ];
        double ga = 0.0;
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
          const int i = lane + 32 * k;
          xa[k] = (i < q) ? ca[i] : 0.0;
          xb[k] = (i < q) ? cb[i] : 0.0;
        }
#pragma unroll
        for (int k = 0; k < KQ; ++k) ga = fma(xa[k], xb[k], ga);
        ga = warp_sum(ga);   // the xor butterfly leaves the same value in every lane
        if (lane == 0) *myflops += 2.0 * q;
        // test and angle in FP32 on the values scaled by 2^sh2, c refined in FP64 (as above)
        bool oka, okb, okg;
        const float alf = htg_d2f_shift(al, sh2, &oka), bef = htg_d2f_shift(be, sh2, &okb);
        const float gaf = htg_d2f_shift(ga, sh2, &okg);
        if (!(oka && okb && okg && fabsf(gaf) > (TOL64F * sqrtf(alf)) * sqrtf(bef))) continue;
        // A pair with a column below the discard level (skip_abs > 0: ranks, not singular values,
        // are wanted) moves T(u) by about |a.b| / max(|a|, |b|), the part of the small column along
        // the large one; below 64 eps |P|_F (rnd2, squared and scaled) that is the rounding level of
        // T(u), and the pair stops rotating.  Without this such pairs, coupled through the pairs of
        // two sub-discard columns that never rotate, converged only linearly (a factor of about 0.7
        // per sweep, up to the sweep limit, measured on the kinetic workload's factors).
        if (rnd2 > 0.f && !(htg_dgt_nn(al, skip_abs) && htg_dgt_nn(be, skip_abs)) &&
            gaf * gaf <= rnd2 * fmaxf(alf, bef))
          continue;
        bool okd;
        const float df = htg_d2f_shift(be - al, sh2, &okd);
        const float zf = df / (2.0f * gaf);
        const float azf = fabsf(zf);
        const double t =
            htg_f2d((azf > 1e18f) ? 0.5f / zf : copysignf(1.0f, zf) / (azf + sqrtf(fmaf(zf, zf, 1.0f))));
        const double c = htg_rsqrt_fast(fma(t, t, 1.0)), sn = c * t;
        double sa = 0.0, sb = 0.0;
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
          const int i = lane + 32 * k;
          const double x = c * xa[k] - sn * xb[k];
          const double y = sn * xa[k] + c * xb[k];
          sa = fma(x, x, sa);
          sb = fma(y, y, sb);
          if (i < q) {
            ca[i] = x;
            cb[i] = y;
          }
        }
        // V columns (five entries per lane loaded ahead of their stores) at the next round's start;
        // a warp with a second pair in this round (8-CTA clusters) first rotates the first pair's,
        // whose columns no other warp touches in this round
        rotate_v();
        pva = ca + q;
        pvb = cb + q;
        pc = c;
        ps = sn;
        sa = warp_sum(sa);
        sb = warp_sum(sb);
        if (lane == 0) {
          *na = sa;
          *nb = sb;
          rot_sh = 1;
          *myflops += 12.0 * q + 6.0 * p;
        }
      }
      cluster.sync();   // the round's columns and norms are visible to every CTA
    }
    if (tid == 0) *flag = rot_sh ? 1.0 : 0.0;   // this CTA's flag of the sweep
    cluster.sync();
    const int any = __syncthreads_or(tid < cl ? (*cluster.map_shared_rank(flag, tid) != 0.0) : 0);
    cluster.sync();   // every flag read before the next sweep rewrites it
    if (!any) break;
  }
  rotate_v();
  cluster.sync();   // every V column final
}

__global__ void __launch_bounds__(CNT, 1) svd_cluster_kernel(const SvdDesc* __restrict__ descs, long long cap_doubles,
                                                             double* flops, int min_p) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cl = (int)cluster.num_blocks();
  const int me = (int)cluster.block_rank();
  const SvdDesc D = descs[blockIdx.x / cl];
  const int p = D.p, q = D.q;
  // the same answer in every CTA of the cluster, so either all of them return here or none
  if (!svdc_takes(p, q, cl, cap_doubles, min_p)) return;
  extern __shared__ double smem[];
  const int ncol = (p + cl - 1) / cl, ld = q + p;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // layout (doubles): red[0..7] | columns ncol * ld | nrm ncol | sig p
  double* red = smem;             // [0] max |M| and [1] |M|_F^2 of this CTA's columns, [2] sweep flag
  double* col = smem + 8;
  double* nrm = col + (long long)ncol * ld;
  double* sig = nrm + ncol;
  for (int e = tid; e < ncol * ld; e += CNT) {
    const int s = e / ld, i = e - s * ld, j = s * cl + me;
    double v = 0.0;
    if (j < p) v = (i < q) ? D.P[j + (long long)D.ldp * i] : ((i - q == j) ? 1.0 : 0.0);
    col[e] = v;
  }
  __syncthreads();
  __shared__ double wmax[CNW];
  double am = 0.0;
  for (int s = wid; s < ncol; s += CNW) {
    const double* cc = col + (long long)s * ld;
    double ss = 0.0;
    for (int i = lane; i < q; i += 32) {
      ss = fma(cc[i], cc[i], ss);
      am = htg_dmax_nn(am, htg_dabs(cc[i]));
    }
    ss = warp_sum(ss);
    if (lane == 0) nrm[s] = ss;
  }
  for (int o = 16; o > 0; o >>= 1) am = htg_dmax_nn(am, __shfl_xor_sync(0xffffffffu, am, o));
  if (lane == 0) wmax[wid] = am;
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, f = 0.0;
    for (int w = 0; w < CNW; ++w) a = htg_dmax_nn(a, wmax[w]);
    for (int s = 0; s < ncol; ++s) f += nrm[s];
    red[0] = a;
    red[1] = f;
  }
  cluster.sync();
  // cluster totals, summed in CTA order, so every CTA holds the same values
  double amax = 0.0, fro = 0.0;
  for (int r = 0; r < cl; ++r) {
    const double* rr = cluster.map_shared_rank(red, r);
    amax = htg_dmax_nn(amax, rr[0]);
    fro += rr[1];
  }
  const int sh_e = (amax > 0.0) ? -ilogb(amax) : 0;
  const double floor2 = EPS * EPS * fro;
  const double skip_abs = D.skip2 * fro / (double)p;
  bool okr;
  const float rnd2 = (skip_abs > 0.0) ? htg_d2f_shift(4096.0 * EPS * EPS * fro, 2 * sh_e, &okr) : 0.f;
  double myflops = 0.0;
  switch ((q + 31) / 32) {
#define SVDC_CASE(K) \
  case K: svdc_sweeps<K>(cluster, col, nrm, red + 2, p, q, cl, floor2, skip_abs, 2 * sh_e, rnd2, &myflops); break;
    SVDC_CASE(1) SVDC_CASE(2) SVDC_CASE(3) SVDC_CASE(4) SVDC_CASE(5) SVDC_CASE(6) SVDC_CASE(7) SVDC_CASE(8)
    SVDC_CASE(9) SVDC_CASE(10) SVDC_CASE(11) SVDC_CASE(12) SVDC_CASE(13) SVDC_CASE(14) SVDC_CASE(15)
#undef SVDC_CASE
    default: break;
  }
  // singular values |N_j| of every column, gathered into every CTA
  for (int j = tid; j < p; j += CNT) sig[j] = sqrt(*cluster.map_shared_rank(nrm + j / cl, j % cl));
  cluster.sync();   // no CTA leaves while another still reads its norms
  for (int s = wid; s < ncol; s += CNW) {
    const int j = s * cl + me;
    if (j >= p) continue;
    const double sc = sig[j];
    int rank = 0;
    for (int o = lane; o < p; o += 32) {
      const double so = sig[o];
      rank += htg_dgt_nn(so, sc) || (__double_as_longlong(so) == __double_as_longlong(sc) && o < j);
    }
    rank = warp_sum_int(rank);
    const double* cc = col + (long long)s * ld;
    if (lane == 0) D.sigma[rank] = sc;
    for (int i = lane; i < p; i += 32) D.V[i + (long long)p * rank] = cc[q + i];
    const double inv = htg_dpos_finite(sc) ? 1.0 / sc : 0.0;
    for (int i = lane; i < q; i += 32) D.U[i + (long long)q * rank] = cc[i] * inv;
  }
  if (flops && lane == 0 && myflops > 0.0) atomicAdd(flops, myflops);
}

__global__ void __launch_bounds__(NT) svd_kernel(const SvdDesc* __restrict__ descs, long long inst_stride,
                                                long long smem_doubles, double* flops, int cl, long long cl_cap,
                                                int min_p) {
  // batched launches: instance blockIdx.y reads its own descriptor list, inst_stride bytes on
  const SvdDesc D = ((const SvdDesc*)((const char*)descs + inst_stride * blockIdx.y))[blockIdx.x];
  const int p = D.p, q = D.q;
  if (p <= 0) return;
  if (svdc_takes(p, q, cl, cl_cap, min_p)) return;   // the cluster form's launch takes this factor
  const int mr = htg_max(p, q);
  extern __shared__ double smem[];
  // layout (doubles): M64 mr*p | N mr*p | G p*p | V p*p | T p*p | nrm p | M32 mr*p/2 | V32 p*p/2
  const long long mp = (long long)mr * p, pp = (long long)p * p;
  const long long need = 2 * mp + 3 * pp + p + (mp + 1) / 2 + (pp + 1) / 2 + 2;
  double* base = (need <= smem_doubles) ? smem : D.work;
  double* M = base;
  double* N = M + mp;
  double* G = N + mp;
  double* V = G + pp;
  double* T = V + pp;
  double* nrm = T + pp;
  float* M32 = (float*)(nrm + p);
  float* V32 = M32 + mp + 1;
  const int tid = threadIdx.x;
  __shared__ int rotated;
  __shared__ int sh_e;        // scale = 2^sh_e
  __shared__ int ract;        // id of the last round with a rotation
  __shared__ int nact;        // active rotations of the round (packed form)
  int nrot = 0;               // rotations applied by this thread (flop count)
  __shared__ double red[NT / 32];
  __shared__ double sc_[HTG_SVD_MAXP];
  __shared__ double ss_[HTG_SVD_MAXP];
  __shared__ int act_[HTG_SVD_MAXP];
  for (long long e = tid; e < mp; e += NT) {
    const int i = (int)(e % mr), c = (int)(e / mr);
    M[e] = (i < q) ? D.P[c + (long long)D.ldp * i] : 0.0;
  }
  // scale of the FP32 copy: 2^-e with 2^e about max |M| (keeps FP32 far from over/underflow)
  double amax = 0.0, fro = 0.0;
  for (long long e = tid; e < mp; e += NT) {
    amax = htg_dmax_nn(amax, htg_dabs(M[e]));
    fro = fma(M[e], M[e], fro);
  }
  for (int o = 16; o > 0; o >>= 1) {
    amax = htg_dmax_nn(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    fro += __shfl_xor_sync(0xffffffffu, fro, o);
  }
  __shared__ double red2[NT / 32];
  if ((tid & 31) == 0) { red[tid >> 5] = amax; red2[tid >> 5] = fro; }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, f = 0.0;
    for (int w = 0; w < NT / 32; ++w) { a = htg_dmax_nn(a, red[w]); f += red2[w]; }
    sh_e = (a > 0.0) ? -ilogb(a) : 0;
    red[0] = ldexp(1.0, sh_e);
    red2[0] = f;
  }
  __syncthreads();
  const double scale = red[0];
  const int sh2 = 2 * sh_e;   // Gram entries scale by 2^sh2
  // rounding floor: columns with |col|^2 <= eps^2 |M|_F^2 carry no information and are not
  // rotated (rotating them only reshuffles rounding noise and keeps the sweeps going)
  const double floor2 = EPS * EPS * red2[0];
  // pairs of columns both below the discard level stay unrotated (see SvdDesc::skip2)
  const double skip_abs = D.skip2 * red2[0] / (double)p;
  const float skip32 = htg_d2f(skip_abs * scale * scale);
  const float floor2_32 = htg_d2f(16.0 * 3.55e-15 * red2[0] * scale * scale);   // (4 eps32)^2 |M s|_F^2
  for (long long e = tid; e < mp; e += NT) M32[e] = htg_d2f(M[e] * scale);
  for (long long e = tid; e < pp; e += NT) V32[e] = (e % p == e / p) ? 1.0f : 0.0f;
  const int p2 = p + (p & 1);
  const int npairs = p2 / 2;
  // lanes per pair: enough for one row per lane, as many pairs as fit the CTA
  int L = 1;
  while (L < 32 && L < mr) L <<= 1;
  while (L > 1 && npairs * L > NT) L >>= 1;
  const int gid = tid / L, gl = tid % L, ngroups = NT / L;
  const unsigned gmask = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((tid & 31) & ~(L - 1)));
  double myflops = 0.0;
  __syncthreads();
  // ---------------- phase 1: FP32 one-sided Jacobi
  const float TOL32 = 4.0f * 5.96e-8f * (float)htg_max(mr, 8);
  if (p > 1) {
    for (int sweep = 0; sweep < 20; ++sweep) {
      if (tid == 0) rotated = 0;
      __syncthreads();
      for (int round = 0; round < p2 - 1; ++round) {
        for (int pi = gid; pi < npairs; pi += ngroups) {
          int a, b;
          rr_pair(pi, round, p, p2, &a, &b);
          if (a < 0) continue;
          float* ca = M32 + (long long)mr * a;
          float* cb = M32 + (long long)mr * b;
          float al = 0.f, be = 0.f, ga = 0.f;
          for (int i = gl; i < mr; i += L) {
            const float x = ca[i], y = cb[i];
            al = fmaf(x, x, al);
            be = fmaf(y, y, be);
            ga = fmaf(x, y, ga);
          }
          for (int o = L >> 1; o > 0; o >>= 1) {
            al += __shfl_xor_sync(gmask, al, o);
            be += __shfl_xor_sync(gmask, be, o);
            ga += __shfl_xor_sync(gmask, ga, o);
          }
          if (ga != 0.f && al > floor2_32 && be > floor2_32 && (al > skip32 || be > skip32) &&
              fabsf(ga) > TOL32 * sqrtf(al) * sqrtf(be)) {
            const float zf = (be - al) / (2.0f * ga);
            const float azf = fabsf(zf);
            const float t = (azf > 1e18f) ? 0.5f / zf : copysignf(1.0f, zf) / (azf + sqrtf(fmaf(zf, zf, 1.0f)));
            const float c = rsqrtf(fmaf(t, t, 1.0f)), sn = c * t;
            for (int i = gl; i < mr; i += L) {
              const float x = ca[i], y = cb[i];
              ca[i] = c * x - sn * y;
              cb[i] = sn * x + c * y;
            }
            float* va = V32 + (long long)p * a;
            float* vb = V32 + (long long)p * b;
            for (int i = gl; i < p; i += L) {
              const float x = va[i], y = vb[i];
              va[i] = c * x - sn * y;
              vb[i] = sn * x + c * y;
            }
            if (gl == 0) rotated = 1;
          }
        }
        __syncthreads();
      }
      const int any = rotated;
      __syncthreads();
      if (!any) break;
    }
  }
  // ---------------- phase 2: orthogonal V in FP64, G = (M V)^T (M V)
  for (long long e = tid; e < pp; e += NT) V[e] = htg_f2d(V32[e]);
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    cta_gemm(T, V, p, V, p, p, p, p, true);                 // T = V^T V
    __syncthreads();
    for (long long e = tid; e < pp; e += NT) T[e] = ((e % p == e / p) ? 1.5 : 0.0) - 0.5 * T[e];
    __syncthreads();
    cta_gemm(N, V, p, T, p, p, p, p, false);                // N(p x p) = V (3I - V^T V)/2
    __syncthreads();
    for (long long e = tid; e < pp; e += NT) V[e] = N[e];
    __syncthreads();
  }
  cta_gemm(N, M, mr, V, p, mr, p, p, false);                // N = M V
  __syncthreads();
  cta_gemm(G, N, mr, N, mr, p, p, mr, true);                // G = N^T N
  __syncthreads();
  if (gl == 0 && gid == 0) myflops += 4.0 * p * p * p + 2.0 * mr * p * p + 2.0 * mr * p * p;
  // ---------------- phase 3: FP64 two-sided Jacobi on G (rotations also applied to V)
  bool okr;
  const float rnd2 = (skip_abs > 0.0) ? htg_d2f_shift(4096.0 * EPS * EPS * red2[0], sh2, &okr) : 0.f;
  // at least 1e-11 when only the truncation's ranks are wanted (as in the cluster form)
  const double TOL = (skip_abs > 0.0) ? fmax(EPS * (double)htg_max(mr, 8), 1e-11) : EPS * (double)htg_max(mr, 8);
  const float TOL64F = htg_d2f(TOL);
  if (tid == 0) ract = 0;
  __syncthreads();
  if (p > 1) {
    for (int sweep = 0; sweep < MAX_SWEEPS; ++sweep) {
      if (tid == 0) rotated = 0;
      __syncthreads();
      for (int round = 0; round < p2 - 1; ++round) {
        const int rid = sweep * p2 + round + 1;
        // angles: one thread per pair; with at most 32 pairs the active ones are packed into the
        // first nact slots (warp ballot), so the update passes touch only their rows/columns
        const bool packed = npairs <= 32;
        if (!packed || tid < 32) {
          for (int pi = tid; pi < (packed ? 32 : npairs); pi += NT) {
            int a = -1, b = 0;
            if (pi < npairs) rr_pair(pi, round, p, p2, &a, &b);
            int act = 0;
            double c = 1.0, sn = 0.0;
            if (a >= 0) {
              const double al = G[a + (long long)p * a], be = G[b + (long long)p * b], ga = G[a + (long long)p * b];
              // test and angle in FP32 on the entries scaled by 2^sh2 (|s M| <= 2), rescaled by
              // exponent arithmetic; only c is refined in FP64, so each rotation is orthogonal
              // to FP64 accuracy.  An entry outside the FP32 range means a column below the
              // rounding floor (|s a|^2 < 2^-118, far below eps^2 |s M|_F^2) or a coupling
              // below 2^-118: neither is rotated.
              bool oka, okb, okg;
              const float alf = htg_d2f_shift(al, sh2, &oka), bef = htg_d2f_shift(be, sh2, &okb);
              const float gaf = htg_d2f_shift(ga, sh2, &okg);
              // |ga| > TOL sqrt(al be), with the product formed so that it cannot underflow
              // before the floor test below rejects the pair
              const bool big = oka && okb && okg && fabsf(gaf) > (TOL64F * sqrtf(alf)) * sqrtf(bef);
              // a pair with a column below the discard level also stops once its effect on T(u) is
              // below the rounding level (the rule of the cluster form, svdc_sweeps)
              const bool below = !(htg_dgt_nn(al, skip_abs) && htg_dgt_nn(be, skip_abs));
              const bool moves = !(rnd2 > 0.f && below && gaf * gaf <= rnd2 * fmaxf(alf, bef));
              if (big && moves && htg_dgt_nn(al, floor2) && htg_dgt_nn(be, floor2) &&
                  (htg_dgt_nn(al, skip_abs) || htg_dgt_nn(be, skip_abs))) {
                bool okd;
                const float df = htg_d2f_shift(be - al, sh2, &okd);   // 0 when below the range
                const float zf = df / (2.0f * gaf);
                const float azf = fabsf(zf);
                const double t =
                    htg_f2d((azf > 1e18f) ? 0.5f / zf : copysignf(1.0f, zf) / (azf + sqrtf(fmaf(zf, zf, 1.0f))));
                c = htg_rsqrt_fast(fma(t, t, 1.0));
                sn = c * t;
                act = 1;
                ++nrot;
              }
            }
            if (packed) {
              const unsigned int m = __ballot_sync(0xffffffffu, act);
              if (act) {
                const int pos = __popc(m & ((1u << tid) - 1u));
                sc_[pos] = c;
                ss_[pos] = sn;
                act_[pos] = a | (b << 16);
              }
              if (tid == 0) {
                nact = __popc(m);
                if (m) {
                  rotated = 1;
                  ract = rid;
                }
              }
            } else {
              sc_[pi] = c;
              ss_[pi] = sn;
              act_[pi] = act ? (a | (b << 16)) : -1;
              if (act) {
                rotated = 1;
                ract = rid;
              }
            }
          }
        }
        __syncthreads();
        if (ract != rid) continue;   // no rotation in this round (uniform after the barrier)
        const int ns = packed ? nact : npairs;   // rotation slots
        // rows a, b of G
        for (int e = tid; e < ns * p; e += NT) {
          const int q = e / p, k = e - q * p;
          const int ab = act_[q];
          if (ab < 0) continue;
          const int a = ab & 0xffff, b = ab >> 16;
          const double c = sc_[q], sn = ss_[q];
          const double x = G[a + (long long)p * k], y = G[b + (long long)p * k];
          G[a + (long long)p * k] = c * x - sn * y;
          G[b + (long long)p * k] = sn * x + c * y;
        }
        __syncthreads();
        // columns a, b of G (items e < ns p) and of V (the rest), one rotation each
        for (int e = tid; e < 2 * ns * p; e += NT) {
          const int isV = e >= ns * p;
          const int f = isV ? e - ns * p : e;
          const int q = f / p, k = f - q * p;
          const int ab = act_[q];
          if (ab < 0) continue;
          const int a = ab & 0xffff, b = ab >> 16;
          const double c = sc_[q], sn = ss_[q];
          double* X = isV ? V : G;
          const double x = X[k + (long long)p * a], y = X[k + (long long)p * b];
          X[k + (long long)p * a] = c * x - sn * y;
          X[k + (long long)p * b] = sn * x + c * y;
        }
        __syncthreads();
      }
      const int any = rotated;
      __syncthreads();
      if (!any) break;
    }
  }
  // ---------------- phase 4: U S = M V, sorted by S
  cta_gemm(N, M, mr, V, p, mr, p, p, false);
  if (gl == 0 && gid == 0) myflops += 2.0 * mr * p * p;
  __syncthreads();
  const int lane = tid & 31, wid = tid >> 5, nw = NT / 32;
  for (int c = wid; c < p; c += nw) {
    const double* cc = N + (long long)mr * c;
    double s = 0.0;
    for (int i = lane; i < mr; i += 32) s = fma(cc[i], cc[i], s);
    s = warp_sum(s);
    if (lane == 0) nrm[c] = sqrt(s);
  }
  __syncthreads();
  myflops += 12.0 * p * nrot;
  if (flops && myflops > 0.0) atomicAdd(flops, myflops);
  for (int c = wid; c < p; c += nw) {
    const double sc = nrm[c];
    int rank = 0;
    for (int o = 0; o < p; ++o) {
      const double so = nrm[o];
      rank += htg_dgt_nn(so, sc) || (__double_as_longlong(so) == __double_as_longlong(sc) && o < c);
    }
    if (lane == 0) D.sigma[rank] = sc;
    for (int i = lane; i < p; i += 32) D.V[i + (long long)p * rank] = V[i + (long long)p * c];
    const double inv = htg_dpos_finite(sc) ? 1.0 / sc : 0.0;
    for (int i = lane; i < q; i += 32) D.U[i + (long long)q * rank] = N[i + (long long)mr * c] * inv;
  }
}

}  // namespace

bool htg_svd_cluster_used(const SvdClusterCfg* clu, int count, int pmax) {
  return clu && clu->cl > 0 && count == 1 && pmax >= clu->min_p;
}

SvdClusterCfg htg_svd_cluster_setup(int device) {
  SvdClusterCfg out;
  int optin = 0;
  cudaFuncAttributes fa;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, svd_cluster_kernel) != cudaSuccess) {
    cudaGetLastError();
    return out;
  }
  const long long dyn = (long long)optin - (long long)fa.sharedSizeBytes;
  if (dyn < (long long)(8 * 1024)) return out;
  if (cudaFuncSetAttribute(svd_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess ||
      cudaFuncSetAttribute(svd_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return out;
  }
  // the largest cluster (16 CTAs, else the portable 8) of which one fits the device with the
  // full shared memory per CTA
  const int sizes[2] = {16, 8};
  for (int k = 0; k < 2; ++k) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sizes[k], 1, 1);
    cfg.blockDim = dim3(CNT, 1, 1);
    cfg.dynamicSmemBytes = (size_t)dyn;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = sizes[k];
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, svd_cluster_kernel, &cfg) == cudaSuccess && n >= 1) {
      out.cl = sizes[k];
      out.cap_doubles = dyn / (long long)sizeof(double);
      return out;
    }
    cudaGetLastError();
  }
  return out;
}

cudaError_t htg_launch_svd(const SvdDesc* descs_dev, int ndesc, int use_smem, int pmax, int qmax,
                           cudaStream_t s, double* flops, int count, long long inst_stride, const SvdClusterCfg* clu) {
  if (ndesc <= 0 || count <= 0) return cudaSuccess;
  if (count > 65535) return cudaErrorInvalidValue;
  (void)use_smem;
  // the cluster form's shared memory: enough for the widest factor it may be given
  const bool use_cl = htg_svd_cluster_used(clu, count, pmax);
  const int cl = use_cl ? clu->cl : 0;
  long long cl_cap = 0;
  if (use_cl) {
    cl_cap = svdc_smem_doubles(htg_min(pmax, SVDC_MAXQ), htg_min(htg_max(qmax, 1), SVDC_MAXQ), cl);
    if (cl_cap > clu->cap_doubles) cl_cap = clu->cap_doubles;
  }
  // shared memory sized for p, q <= 40 (about 77 KB dynamic + 21 KB static: two CTAs per SM in
  // batched launches); larger node factors work in their global buffers
  pmax = htg_min(pmax, 40);
  qmax = htg_min(qmax, 40);
  const int mr = htg_max(pmax, qmax);
  const size_t mp = (size_t)mr * pmax, pp = (size_t)pmax * pmax;
  size_t smem = (2 * mp + 3 * pp + pmax + (mp + 1) / 2 + (pp + 1) / 2 + 2) * sizeof(double);
  if (smem > HTG_SMEM_BYTES) smem = HTG_SMEM_BYTES;
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HTG_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  const int min_p = clu ? clu->min_p : SVDC_MIN_P;
  svd_kernel<<<dim3(ndesc, count), NT, smem, s>>>(descs_dev, inst_stride, (long long)(smem / sizeof(double)), flops,
                                                   cl, cl_cap, min_p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !use_cl) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ndesc * cl), 1, 1);
  cfg.blockDim = dim3(CNT, 1, 1);
  cfg.dynamicSmemBytes = (size_t)cl_cap * sizeof(double);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, svd_cluster_kernel, descs_dev, cl_cap, flops, min_p);
}
