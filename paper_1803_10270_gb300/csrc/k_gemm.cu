// Batched small GEMMs for the HT contractions (mode products of transfer tensors,
// leaf projections, factor products).  Sizes are read from device descriptors, so one
// launch serves every node of a tree level whatever the ranks chosen on the device.
//
// Work decomposition: every descriptor contributes batch * tiles(m) * tiles(n) work items
// of a 16 x 16 output tile computed by 64 threads (2 x 2 outputs each); a fixed grid walks
// the items with a grid-stride loop.  FP64 on the CUDA cores: on GB300 the FP64 pipe of an
// SM retires about 2 FMA per clock, so the contractions of these small ranks are bound by
// how many SMs take part; small tiles spread a product over as many SMs as possible.
#include "common.cuh"

namespace {

constexpr int BM = 16, BN = 16, BK = 16, NT = 64;
constexpr int MAXD = 64;

// work of a descriptor in multiply-adds, the quantity the FP64 / tensor-core split compares
__device__ inline long long gemm_work(const GemmDesc& g) {
  return (long long)g.m * g.n * (long long)g.k * g.batch;
}

__global__ void __launch_bounds__(NT) gemm_kernel(const GemmDesc* __restrict__ descs0, long long inst_stride, int ndesc,
                                                  double* flops, long long tc_min) {
  // batched launches: instance blockIdx.y reads its own descriptor list, inst_stride bytes on
  const GemmDesc* __restrict__ descs = (const GemmDesc*)((const char*)descs0 + inst_stride * blockIdx.y);
  __shared__ long long prefix[MAXD + 1];
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  if (tid == 0) {
    long long acc = 0;
    prefix[0] = 0;
    for (int i = 0; i < ndesc; ++i) {
      const GemmDesc& g = descs[i];
      long long items = 0;
      // tc_min > 0: descriptors of at least tc_min multiply-adds belong to the tensor-core launch
      if (g.m > 0 && g.n > 0 && g.batch > 0 && (tc_min <= 0 || gemm_work(g) < tc_min))
        items = (long long)g.batch * htg_cdiv(g.m, BM) * htg_cdiv(g.n, BN);
      acc += items;
      prefix[i + 1] = acc;
    }
  }
  __syncthreads();
  const long long total = prefix[ndesc];
  const int tx = tid % 8, ty = tid / 8;
  for (long long w = blockIdx.x; w < total; w += gridDim.x) {
    int di = 0;
    while (prefix[di + 1] <= w) ++di;
    const GemmDesc g = descs[di];
    long long loc = w - prefix[di];
    const int tm = htg_cdiv(g.m, BM), tn = htg_cdiv(g.n, BN);
    const int tile = (int)(loc % ((long long)tm * tn));
    const int b = (int)(loc / ((long long)tm * tn));
    const int i0 = (tile % tm) * BM, j0 = (tile / tm) * BN;
    if (flops && tid == 0)
      atomicAdd(flops, 2.0 * htg_min(BM, g.m - i0) * htg_min(BN, g.n - j0) * (double)g.k);
    const double* A = g.A + (long long)b * g.sA;
    const double* B = g.B + (long long)b * g.sB;
    double* C = g.C + (long long)b * g.sC;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    const bool has_beta = htg_dnz(g.beta);   // bit test: an FP64 compare costs ~800 cycles here
    // the next k-slice is read from global memory into registers while the current one is
    // multiplied out of shared memory (its loads overlap the FP64 work of the slice)
    constexpr int PER = (BM * BK) / NT;
    double ra[PER], rb[PER];
    auto gload = [&](int l0) {
#pragma unroll
      for (int p = 0; p < PER; ++p) {
        const int e = tid + NT * p;
        int i, l;
        if (!g.tA) { i = e % BM; l = e / BM; } else { l = e % BK; i = e / BK; }
        const int gi = i0 + i, gl = l0 + l;
        ra[p] = (gi < g.m && gl < g.k) ? (g.tA ? A[gl + (long long)g.lda * gi] : A[gi + (long long)g.lda * gl]) : 0.0;
        int j, l2;
        if (!g.tB) { l2 = e % BK; j = e / BK; } else { j = e % BN; l2 = e / BN; }
        const int gj = j0 + j, gl2 = l0 + l2;
        rb[p] = (gj < g.n && gl2 < g.k) ? (g.tB ? B[gj + (long long)g.ldb * gl2] : B[gl2 + (long long)g.ldb * gj]) : 0.0;
      }
    };
    gload(0);
    for (int l0 = 0; l0 < g.k; l0 += BK) {
#pragma unroll
      for (int p = 0; p < PER; ++p) {
        const int e = tid + NT * p;
        if (!g.tA) As[e / BM][e % BM] = ra[p]; else As[e % BK][e / BK] = ra[p];
        if (!g.tB) Bs[e % BK][e / BK] = rb[p]; else Bs[e / BN][e % BN] = rb[p];
      }
      __syncthreads();
      if (l0 + BK < g.k) gload(l0 + BK);
      if (l0 + BK <= g.k) {
#pragma unroll
        for (int l = 0; l < BK; ++l) {
          const double a0 = As[l][ty], a1 = As[l][ty + 8];
          const double b0 = Bs[l][tx], b1 = Bs[l][tx + 8];
          acc[0][0] = fma(a0, b0, acc[0][0]);
          acc[0][1] = fma(a0, b1, acc[0][1]);
          acc[1][0] = fma(a1, b0, acc[1][0]);
          acc[1][1] = fma(a1, b1, acc[1][1]);
        }
      } else {
        // the ragged last slice: only its k - l0 terms (every FP64 warp instruction costs the
        // same, padded or not)
        for (int l = 0; l < g.k - l0; ++l) {
          const double a0 = As[l][ty], a1 = As[l][ty + 8];
          const double b0 = Bs[l][tx], b1 = Bs[l][tx + 8];
          acc[0][0] = fma(a0, b0, acc[0][0]);
          acc[0][1] = fma(a0, b1, acc[0][1]);
          acc[1][0] = fma(a1, b0, acc[1][0]);
          acc[1][1] = fma(a1, b1, acc[1][1]);
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int gi = i0 + ty + 8 * r, gj = j0 + tx + 8 * c;
        if (gi < g.m && gj < g.n) {
          double v = g.alpha * acc[r][c];
          if (g.colscale) v *= g.colscale[gj];
          double* cp = C + gi + (long long)g.ldc * gj;
          if (has_beta) v += g.beta * *cp;
          *cp = v;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- split FP32 form ----
// HT_PREC_MIXED's contractions below the tensor-core threshold, on the FP32 pipe (an SM retires
// 64x as many FP32 as FP64 operations, at a few cycles of latency instead of about a hundred).
// Each FP64 operand x is split by integer operations into x_hi + x_lo, two FP32 values (the
// leading 24 significant bits and the next 24, |x - x_hi - x_lo| < 2^-47 |x|; below 2^-75 x_lo is
// zero, below 2^-125 x_hi is x rounded to FP32, and |x| >= 2^128 is outside the form's range).  A
// product a b is taken as p = a_hi b_hi (rounded), its exact rounding error fma(a_hi, b_hi, -p)
// and the cross terms a_hi b_lo + a_lo b_hi (a_lo b_lo, below 2^-46 |a b|, is dropped); p enters a
// double-float accumulator (hi, lo) by Knuth's error-free TwoSum, the small terms enter lo: the
// compensated dot product of Ogita, Rump and Oishi (2005), on split operands.  Error at most about
// (k^2 + 5 k + 10) 2^-47 sum_i |a_i b_i| (their gamma_k^2 term plus the split and cross terms),
// about (k/2 + 10) 2^-47 sum_i |a_i b_i| with rounding errors of random sign: FP64-like for these
// contractions.  The additions and the product p are the _rn intrinsics, which the compiler never
// contracts into an FMA (a fused t = s_hi + a_hi b_hi would break TwoSum's exactness).  Tiles,
// work items and descriptors as gemm_kernel; alpha, colscale and beta in FP64 on the reassembled
// sum.
__device__ inline void split_hi_lo(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -125 || e > 127) {   // zero, or outside the FP32 normal range: take the FP32 value
    hi = htg_d2f(x);
    lo = 0.0f;
    return;
  }
  hi = __int_as_float((int)(sign | ((unsigned int)(e + 127) << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu)));
  // the low 29 bits of the significand, worth 2^(e - 52) each
  const float r = __uint2float_rz((unsigned int)(b & 0x1FFFFFFFull));
  const int es = e - 52 + 127;
  const float scale = (es >= 1) ? __int_as_float(es << 23) : 0.0f;
  lo = sign ? -(r * scale) : r * scale;
}

// s_hi + s_lo += a b with a = (ah, al), b = (bh, bl)
__device__ inline void acc_term(float ah, float al, float bh, float bl, float& s_hi, float& s_lo) {
  const float p = __fmul_rn(ah, bh);
  float x = fmaf(ah, bh, -p);
  x = fmaf(ah, bl, x);
  x = fmaf(al, bh, x);
  const float t = __fadd_rn(s_hi, p);
  const float bp = __fsub_rn(t, s_hi);
  const float err = __fadd_rn(__fsub_rn(s_hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s_hi = t;
  s_lo = __fadd_rn(s_lo, __fadd_rn(err, x));
}

__global__ void __launch_bounds__(NT) gemm_f32x2_kernel(const GemmDesc* __restrict__ descs0, long long inst_stride,
                                                        int ndesc, double* flops, long long tc_min) {
  const GemmDesc* __restrict__ descs = (const GemmDesc*)((const char*)descs0 + inst_stride * blockIdx.y);
  __shared__ long long prefix[MAXD + 1];
  __shared__ float Ah[BK][BM + 1], Al[BK][BM + 1];
  __shared__ float Bh[BK][BN + 1], Bl[BK][BN + 1];
  const int tid = threadIdx.x;
  if (tid == 0) {
    long long acc = 0;
    prefix[0] = 0;
    for (int i = 0; i < ndesc; ++i) {
      const GemmDesc& g = descs[i];
      long long items = 0;
      if (g.m > 0 && g.n > 0 && g.batch > 0 && (tc_min <= 0 || gemm_work(g) < tc_min))
        items = (long long)g.batch * htg_cdiv(g.m, BM) * htg_cdiv(g.n, BN);
      acc += items;
      prefix[i + 1] = acc;
    }
  }
  __syncthreads();
  const long long total = prefix[ndesc];
  const int tx = tid % 8, ty = tid / 8;
  for (long long w = blockIdx.x; w < total; w += gridDim.x) {
    int di = 0;
    while (prefix[di + 1] <= w) ++di;
    const GemmDesc g = descs[di];
    long long loc = w - prefix[di];
    const int tm = htg_cdiv(g.m, BM), tn = htg_cdiv(g.n, BN);
    const int tile = (int)(loc % ((long long)tm * tn));
    const int b = (int)(loc / ((long long)tm * tn));
    const int i0 = (tile % tm) * BM, j0 = (tile / tm) * BN;
    if (flops && tid == 0)
      atomicAdd(flops, 2.0 * htg_min(BM, g.m - i0) * htg_min(BN, g.n - j0) * (double)g.k);
    const double* A = g.A + (long long)b * g.sA;
    const double* B = g.B + (long long)b * g.sB;
    double* C = g.C + (long long)b * g.sC;
    float sh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, sl[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    const bool has_beta = htg_dnz(g.beta);
    for (int l0 = 0; l0 < g.k; l0 += BK) {
#pragma unroll
      for (int p = 0; p < (BM * BK) / NT; ++p) {
        const int e = tid + NT * p;
        int i, l;
        if (!g.tA) { i = e % BM; l = e / BM; } else { l = e % BK; i = e / BK; }
        const int gi = i0 + i, gl = l0 + l;
        double v = 0.0;
        if (gi < g.m && gl < g.k) v = g.tA ? A[gl + (long long)g.lda * gi] : A[gi + (long long)g.lda * gl];
        split_hi_lo(v, Ah[l][i], Al[l][i]);
        int j, l2;
        if (!g.tB) { l2 = e % BK; j = e / BK; } else { j = e % BN; l2 = e / BN; }
        const int gj = j0 + j, gl2 = l0 + l2;
        double u = 0.0;
        if (gj < g.n && gl2 < g.k) u = g.tB ? B[gj + (long long)g.ldb * gl2] : B[gl2 + (long long)g.ldb * gj];
        split_hi_lo(u, Bh[l2][j], Bl[l2][j]);
      }
      __syncthreads();
      const int lmax = htg_min(BK, g.k - l0);
      for (int l = 0; l < lmax; ++l) {
        const float a0h = Ah[l][ty], a0l = Al[l][ty], a1h = Ah[l][ty + 8], a1l = Al[l][ty + 8];
        const float b0h = Bh[l][tx], b0l = Bl[l][tx], b1h = Bh[l][tx + 8], b1l = Bl[l][tx + 8];
        acc_term(a0h, a0l, b0h, b0l, sh[0][0], sl[0][0]);
        acc_term(a0h, a0l, b1h, b1l, sh[0][1], sl[0][1]);
        acc_term(a1h, a1l, b0h, b0l, sh[1][0], sl[1][0]);
        acc_term(a1h, a1l, b1h, b1l, sh[1][1], sl[1][1]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int gi = i0 + ty + 8 * r, gj = j0 + tx + 8 * c;
        if (gi < g.m && gj < g.n) {
          double v = g.alpha * (htg_f2d(sh[r][c]) + htg_f2d(sl[r][c]));
          if (g.colscale) v *= g.colscale[gj];
          double* cp = C + gi + (long long)g.ldc * gj;
          if (has_beta) v += g.beta * *cp;
          *cp = v;
        }
      }
    }
  }
}

}  // namespace

cudaError_t htg_launch_gemm(const GemmDesc* descs_dev, int ndesc, int grid, cudaStream_t s, double* flops, int count,
                            long long inst_stride, long long tc_min) {
  if (ndesc <= 0 || count <= 0) return cudaSuccess;
  if (ndesc > MAXD || count > 65535) return cudaErrorInvalidValue;
  // One instance: 2 x SMs 64-thread CTAs (grid = 4 x SMs), the grid-stride loop covers any
  // item count.  A batch: instances differ in size, so each gets up to 16 CTAs, as many as
  // stay resident together (32 CTAs of 64 threads per SM)
  const int gx = (count == 1) ? htg_max(1, grid / 2) : htg_max(2, htg_min(16, (grid * 8 + count - 1) / count));
  gemm_kernel<<<dim3(gx, count), NT, 0, s>>>(descs_dev, inst_stride, ndesc, flops, tc_min);
  return cudaGetLastError();
}

cudaError_t htg_launch_gemm_f32x2(const GemmDesc* descs_dev, int ndesc, int grid, cudaStream_t s, double* flops,
                                  int count, long long inst_stride, long long tc_min) {
  if (ndesc <= 0 || count <= 0) return cudaSuccess;
  if (ndesc > MAXD || count > 65535) return cudaErrorInvalidValue;
  const int gx = (count == 1) ? htg_max(1, grid / 2) : htg_max(2, htg_min(16, (grid * 8 + count - 1) / count));
  gemm_f32x2_kernel<<<dim3(gx, count), NT, 0, s>>>(descs_dev, inst_stride, ndesc, flops, tc_min);
  return cudaGetLastError();
}
