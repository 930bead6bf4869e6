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
    for (int l0 = 0; l0 < g.k; l0 += BK) {
#pragma unroll
      for (int p = 0; p < (BM * BK) / NT; ++p) {
        const int e = tid + NT * p;
        int i, l;
        if (!g.tA) { i = e % BM; l = e / BM; } else { l = e % BK; i = e / BK; }
        const int gi = i0 + i, gl = l0 + l;
        double v = 0.0;
        if (gi < g.m && gl < g.k) v = g.tA ? A[gl + (long long)g.lda * gi] : A[gi + (long long)g.lda * gl];
        As[l][i] = v;
        int j, l2;
        if (!g.tB) { l2 = e % BK; j = e / BK; } else { j = e % BN; l2 = e / BN; }
        const int gj = j0 + j, gl2 = l0 + l2;
        double u = 0.0;
        if (gj < g.n && gl2 < g.k) u = g.tB ? B[gj + (long long)g.ldb * gl2] : B[gl2 + (long long)g.ldb * gj];
        Bs[l2][j] = u;
      }
      __syncthreads();
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
