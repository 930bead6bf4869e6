// Batched contractions of the mixed-precision form on the fifth-generation tensor cores
// (tcgen05, BF16 operands, FP32 accumulators in tensor memory), FP64 in and out.
//
// Error-compensated split (an Ozaki-type scheme).  Row i of op(A) is scaled by 2^(8S-2-E_i), E_i
// the largest binary exponent in that row, and rounded to an integer N of at most 8S-1 bits;
// column j of op(B) likewise (exponent F_j, integer M).  N and M are written in balanced base 256,
// N = sum_s d_s 256^(S-1-s) with |d_s| <= 128, so each digit is an exact BF16 value and a product
// of two digits an integer of at most 2^14.  The digit products whose weight reaches 256^-(S-1)
// of the leading one (pairs s + t <= S - 1) are accumulated by tcgen05.mma, one FP32 accumulator
// per group g = s + t, so every partial sum is an integer below 2^24 (exact) for inner dimensions
// up to 1024 / (g + 1) and a rounding 2^-(24+8g) below the leading term beyond.  The epilogue
// combines the groups in 64-bit integers, V = sum_g acc_g 256^(S-1-g), and forms the double
// V 2^(E_i + F_j - 8S - 4) from its bits: no FP64 instruction unless alpha, a column scale or
// beta is present.  The result equals the FP64 product up to a normwise error of about
// 2^-(8S-1) |A_i| |B_j| (rows and columns of op(A), op(B)); S = 4 gives about 5e-10.
//
// Tile: 128 rows x 128 columns of C per work item, the inner dimension in stages of 32 values.
// 256 threads convert a stage into S digit planes per operand in shared memory (the canonical
// K-major layout without swizzle: 8 x 16-byte core matrices, the 8-row groups 512 bytes apart),
// one elected thread issues the MMAs (M = 128, N = 128, K = 16 each) and commits them to an
// mbarrier of the stage; two stages alternate, so the conversion of stage s+1 overlaps the MMAs
// of stage s.  The accumulators (S groups x 128 columns) take the CTA's 512 tensor-memory columns;
// every thread then reads its row (tcgen05.ld, 32 lanes per warp) and writes its outputs.
// Operands are loaded with plain coalesced loads: each value is converted to digits on the way,
// which a bulk tensor copy could not do.
#include "common.cuh"

namespace {

constexpr int TM = 128, TN = 128, KC = 32, NT = 256, MAXD = 64;
constexpr int LBO = 128;                  // bytes between core matrices adjacent along K
constexpr int SBO = (KC / 8) * 128;       // bytes between 8-row groups
constexpr int PLANE = TM * KC * 2;        // bytes of one digit plane (TM = TN)
constexpr uint32_t TMEM_COLS = 512;
// instruction descriptor of kind::f16: D FP32 (bit 4), A and B BF16 (bits 7, 10), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
// bounded waits: about 2^31 SM clocks (1 s at 2 GHz) before an mbarrier wait gives up
constexpr long long WAIT_CYCLES = 1ll << 31;

__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, LBO, SBO (all >> 4), fixed bit 46, no swizzle
__device__ inline uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(LBO >> 4) << 16) | ((uint64_t)(SBO >> 4) << 32) |
         (1ull << 46);
}

__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity; false when it gave up
__device__ inline bool mbar_wait(uint64_t* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}
__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ inline void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accum)
      : "memory");
}
__device__ inline void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ inline void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ inline void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// biased binary exponent of x (0 for zero and subnormals, 2047 for Inf / NaN)
__device__ inline int bexp(double x) { return (int)((((unsigned long long)__double_as_longlong(x)) >> 52) & 0x7FF); }

// the S balanced base-256 digits of round(x 2^(8S-2-(E-1023))), E >= bexp(x) the row's biased
// exponent: |d_0| <= 128, |d_s| <= 128 (s > 0)
template <int S>
__device__ inline void to_digits(double x, int E, int (&dg)[S]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int ef = (int)((b >> 52) & 0x7FF);
  long long n = 0;
  const int sh = 54 - 8 * S + (E - ef);   // >= 6 for S <= 6
  if (ef != 0 && ef != 2047 && sh < 54) {
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    n = (long long)((m + (1ull << (sh - 1))) >> sh);
    if (b >> 63) n = -n;
  }
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int q = (int)((n + 128) & 255) - 128;
    dg[s] = q;
    n = (n - q) >> 8;
  }
  dg[0] = (int)n;
}

// BF16 bit pattern of a small integer (exact: at most 8 significant bits)
__device__ inline uint32_t bf16_bits(int q) { return __float_as_uint((float)q) >> 16; }

// exact double of V 2^sc (V an integer of at most 62 bits); 0 on underflow
__device__ inline double ldexp_ll(long long V, int sc) {
  if (V == 0) return 0.0;
  const unsigned long long sgn = V < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long u = (unsigned long long)(V < 0 ? -V : V);
  const int p = 63 - __clzll((long long)u);      // leading bit
  const int field = p + 1023 + sc;
  if (field <= 0) return __longlong_as_double((long long)sgn);
  if (field >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
  u = (p <= 52) ? (u << (52 - p)) : (u >> (p - 52));
  return __longlong_as_double((long long)(sgn | ((unsigned long long)field << 52) | (u & 0xFFFFFFFFFFFFFull)));
}

// One operand tile (128 rows x KC inner values) of a matrix whose element (r, l) is
// base[r rs + l ks] (exactly one of rs, ks is 1), rows < nr and l < nk valid, converted to S digit
// planes at dst (plane s at dst + s PLANE) with the rows' exponents ex[].
template <int S>
__device__ inline void stage_tile(const double* __restrict__ base, long long rs, long long ks, int nr, int nk,
                                  const int* __restrict__ ex, char* dst) {
  const int tid = threadIdx.x;
#pragma unroll 2
  for (int p = 0; p < (TM * KC / 2) / NT; ++p) {
    int r, kp;
    if (rs == 1) {          // rows contiguous: a warp reads 32 consecutive rows of one column
      r = tid & (TM - 1);
      kp = (tid >> 7) + 2 * p;
    } else {                // inner index contiguous: 16 threads read 32 consecutive values
      kp = tid & 15;
      r = (tid >> 4) + 16 * p;
    }
    const int l = 2 * kp;
    double x0 = 0.0, x1 = 0.0;
    if (r < nr) {
      const double* q = base + (long long)r * rs + (long long)l * ks;
      if (l < nk) x0 = q[0];
      if (l + 1 < nk) x1 = q[ks];
    }
    const int E = ex[r];
    int d0[S], d1[S];
    to_digits<S>(x0, E, d0);
    to_digits<S>(x1, E, d1);
    const int off = (r >> 3) * SBO + (l >> 3) * LBO + (r & 7) * 16 + (l & 7) * 2;
#pragma unroll
    for (int s = 0; s < S; ++s)
      *(uint32_t*)(dst + s * PLANE + off) = bf16_bits(d0[s]) | (bf16_bits(d1[s]) << 16);
  }
}

// per-row largest biased exponent over the whole inner dimension, by shared-memory atomics
__device__ inline void row_exponents(const double* __restrict__ base, long long rs, long long ks, int nr, int nk,
                                     int* ex) {
  const int tid = threadIdx.x;
  if (rs == 1) {
    for (int r = tid & (TM - 1); r < nr; r += TM) {
      int e = 0;
      for (int l = tid >> 7; l < nk; l += NT / TM) e = max(e, bexp(base[r + l * ks]));
      atomicMax(&ex[r], e);
    }
  } else {
    const int lane = tid & 31, w = tid >> 5;
    for (int r = w; r < nr; r += NT / 32) {
      int e = 0;
      for (int l = lane; l < nk; l += 32) e = max(e, bexp(base[(long long)r * rs + l]));
      atomicMax(&ex[r], e);
    }
  }
}

struct TcShared {
  long long prefix[MAXD + 1];
  int exA[TM];
  int exB[TN];
  uint64_t mbar[2];
  uint32_t tmem;
  int stop;
};

template <int S>
__global__ void __launch_bounds__(NT, 1)
    gemm_tc_kernel(const GemmDesc* __restrict__ descs0, long long inst_stride, int ndesc, double* flops, int* err,
                   long long tc_min) {
  extern __shared__ __align__(1024) char smem_raw[];
  char* planes = (char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // stage st: A planes at planes + st (2 S PLANE), B planes after them
  TcShared& sh = *(TcShared*)(planes + 2 * 2 * S * PLANE);
  const GemmDesc* __restrict__ descs = (const GemmDesc*)((const char*)descs0 + inst_stride * blockIdx.y);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    long long acc = 0;
    sh.prefix[0] = 0;
    for (int i = 0; i < ndesc; ++i) {
      const GemmDesc& g = descs[i];
      long long items = 0;
      // descriptors below tc_min multiply-adds belong to the FP64 launch
      if (g.m > 0 && g.n > 0 && g.batch > 0 && (long long)g.m * g.n * (long long)g.k * g.batch >= tc_min)
        items = (long long)g.batch * htg_cdiv(g.m, TM) * htg_cdiv(g.n, TN);
      acc += items;
      sh.prefix[i + 1] = acc;
    }
    sh.stop = 0;
  }
  __syncthreads();
  const long long total = sh.prefix[ndesc];
  if ((long long)blockIdx.x >= total) return;   // no work: no tensor memory taken
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&sh.mbar[0], 1);
    mbar_init(&sh.mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh.tmem;
  unsigned phase = 0u, pending = 0u;   // bit st: the stage's next phase parity / an uncompleted commit
  long long slab_count = 0;
  bool ok = true;

  for (long long w = blockIdx.x; w < total && ok; w += gridDim.x) {
    int di = 0;
    while (sh.prefix[di + 1] <= w) ++di;
    const GemmDesc g = descs[di];
    const long long loc = w - sh.prefix[di];
    const int tm = htg_cdiv(g.m, TM), tn = htg_cdiv(g.n, TN);
    const int tile = (int)(loc % ((long long)tm * tn));
    const int b = (int)(loc / ((long long)tm * tn));
    const int i0 = (tile % tm) * TM, j0 = (tile / tm) * TN;
    const int nr = htg_min(TM, g.m - i0), nc = htg_min(TN, g.n - j0);
    // executed MMA flops: the digit pairs over the whole tile and every stage
    if (flops && tid == 0)
      atomicAdd(flops, (double)(S * (S + 1) / 2) * 2.0 * TM * TN * (double)(KC * htg_max(1, htg_cdiv(g.k, KC))));
    // op(A)(i0 + r, l) = Ab[r rsA + l ksA]; op(B)(l, j0 + c) = Bb[c rsB + l ksB]
    const double* Ab = g.A + (long long)b * g.sA + (g.tA ? (long long)g.lda * i0 : (long long)i0);
    const long long rsA = g.tA ? g.lda : 1, ksA = g.tA ? 1 : g.lda;
    const double* Bb = g.B + (long long)b * g.sB + (g.tB ? (long long)j0 : (long long)g.ldb * j0);
    const long long rsB = g.tB ? 1 : g.ldb, ksB = g.tB ? g.ldb : 1;
    double* C = g.C + (long long)b * g.sC;

    for (int r = tid; r < TM; r += NT) { sh.exA[r] = 0; sh.exB[r] = 0; }
    __syncthreads();
    row_exponents(Ab, rsA, ksA, nr, g.k, sh.exA);
    row_exponents(Bb, rsB, ksB, nc, g.k, sh.exB);
    __syncthreads();

    bool first[S];
#pragma unroll
    for (int q = 0; q < S; ++q) first[q] = true;
    const int nslab = htg_max(1, htg_cdiv(g.k, KC));
    for (int sl = 0; sl < nslab; ++sl) {
      const int st = (int)(slab_count & 1);
      if ((pending >> st) & 1u) {   // the MMAs that last read this stage's planes must be done
        if (tid == 0 && !mbar_wait(&sh.mbar[st], (phase >> st) & 1u)) sh.stop = 1;
        phase ^= 1u << st;
        pending &= ~(1u << st);
        __syncthreads();
        if (sh.stop) { ok = false; break; }
      }
      char* pa = planes + st * (2 * S * PLANE);
      char* pb = pa + S * PLANE;
      const int l0 = sl * KC, nk = htg_max(0, htg_min(KC, g.k - l0));
      stage_tile<S>(Ab + (long long)l0 * ksA, rsA, ksA, nr, nk, sh.exA, pa);
      stage_tile<S>(Bb + (long long)l0 * ksB, rsB, ksB, nc, nk, sh.exB, pb);
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(pa), b0 = smem_u32(pb);
#pragma unroll
        for (int sa = 0; sa < S; ++sa) {
#pragma unroll
          for (int sb = 0; sb + sa < S; ++sb) {
            const int grp = sa + sb;
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              const uint64_t ad = sdesc(a0 + sa * PLANE + kk * 2 * LBO);
              const uint64_t bd = sdesc(b0 + sb * PLANE + kk * 2 * LBO);
              mma_bf16(tmem + (uint32_t)(grp * TN), ad, bd, first[grp] ? 0u : 1u);
              first[grp] = false;
            }
          }
        }
        mma_commit(&sh.mbar[st]);
      }
      pending |= 1u << st;
      ++slab_count;
    }
    if (!ok) break;
    for (int st = 0; st < 2; ++st) {
      if ((pending >> st) & 1u) {
        if (tid == 0 && !mbar_wait(&sh.mbar[st], (phase >> st) & 1u)) sh.stop = 1;
        phase ^= 1u << st;
        pending &= ~(1u << st);
      }
    }
    __syncthreads();
    if (sh.stop) { ok = false; break; }
    tc_fence_after();
    // epilogue: warp w reads lanes 32 (w mod 4) .. +31 (its rows), columns [64 (w / 4), +64)
    const int r = 32 * (warp & 3) + lane;
    const int gi = i0 + r;
    const int eA = sh.exA[r];
    const bool has_beta = htg_dnz(g.beta);
    const bool unit_alpha = __double_as_longlong(g.alpha) == 0x3FF0000000000000ll;
    for (int c0 = 64 * (warp >> 2); c0 < 64 * (warp >> 2) + 64; c0 += 16) {
      if (c0 >= nc) break;   // warp-uniform
      uint32_t acc[S][16];
#pragma unroll
      for (int q = 0; q < S; ++q)
        tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(q * TN + c0), acc[q]);
      tmem_ld_wait();
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int cc = c0 + c;
        if (cc >= nc || r >= nr) continue;
        long long V = 0;
#pragma unroll
        for (int q = 0; q < S; ++q) V += (long long)__float2int_rn(__uint_as_float(acc[q][c])) << (8 * (S - 1 - q));
        const int eB = sh.exB[cc];
        double v;
        if (eA == 2047 || eB == 2047) v = __longlong_as_double(0x7FF8000000000000ll);   // Inf / NaN in
        else v = ldexp_ll(V, (eA - 1023) + (eB - 1023) - 8 * S - 4);
        const int gj = j0 + cc;
        if (!unit_alpha) v *= g.alpha;
        if (g.colscale) v *= g.colscale[gj];
        double* cp = C + gi + (long long)g.ldc * gj;
        if (has_beta) v = fma(g.beta, *cp, v);
        *cp = v;
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (!ok && tid == 0) {
    if (err) atomicCAS(err, 0, (int)HT_ERR_TIMEOUT);
    // let committed MMAs drain (bounded) before the tensor memory is released
    for (int st = 0; st < 2; ++st)
      if ((pending >> st) & 1u) mbar_wait(&sh.mbar[st], (phase >> st) & 1u);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

template <int S>
constexpr int smem_bytes() {
  return 2 * 2 * S * PLANE + (int)sizeof(TcShared) + 1024;
}

template <int S>
cudaError_t launch_s(const GemmDesc* descs_dev, int ndesc, int grid, cudaStream_t s, double* flops, int count,
                     long long inst_stride, int* err, long long tc_min) {
  static int configured[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
  if (dev >= 0 && dev < 64 && !configured[dev]) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<S>());
    if (e != cudaSuccess) return e;
    configured[dev] = 1;
  }
  gemm_tc_kernel<S><<<dim3(grid, count), NT, smem_bytes<S>(), s>>>(descs_dev, inst_stride, ndesc, flops, err, tc_min);
  return cudaGetLastError();
}

}  // namespace

cudaError_t htg_launch_gemm_tc(const GemmDesc* descs_dev, int ndesc, int sms, int slices, cudaStream_t s,
                               double* flops, int count, long long inst_stride, int* err, long long tc_min) {
  if (ndesc <= 0 || count <= 0) return cudaSuccess;
  if (ndesc > MAXD || count > 65535) return cudaErrorInvalidValue;
  // one CTA per SM (512 tensor-memory columns and 2 x 2 S planes of shared memory each); a batch
  // spreads the SMs over its instances
  const int grid = (count == 1) ? htg_max(1, sms) : htg_max(1, htg_min(16, htg_cdiv(sms * 2, count)));
  switch (slices) {
    case 2: return launch_s<2>(descs_dev, ndesc, grid, s, flops, count, inst_stride, err, tc_min);
    case 3: return launch_s<3>(descs_dev, ndesc, grid, s, flops, count, inst_stride, err, tc_min);
    case 4: return launch_s<4>(descs_dev, ndesc, grid, s, flops, count, inst_stride, err, tc_min);
    default: return cudaErrorInvalidValue;
  }
}

// ------------------------------------------------------------- self-test ---------
namespace {
__device__ GemmDesc g_tc_selftest_desc[1];
__device__ int g_tc_selftest_err[1];
}  // namespace

extern "C" int ht_selftest_gemm_mixed(int m, int n, int k, const double* A, int lda, int tA, const double* B, int ldb,
                                      int tB, double* C, int ldc, double alpha, double beta, const double* colscale,
                                      int batch, long long sA, long long sB, long long sC, int slices, void* stream) {
  if (m < 0 || n < 0 || k < 0 || batch < 1 || slices < 1 || slices > 4) return HT_ERR_ARG;
  if (!A || !B || !C || lda < 1 || ldb < 1 || ldc < htg_max(1, m)) return HT_ERR_ARG;
  if (lda < (tA ? htg_max(1, k) : htg_max(1, m)) || ldb < (tB ? htg_max(1, n) : htg_max(1, k))) return HT_ERR_ARG;
  GemmDesc g;
  g.A = A; g.B = B; g.C = C; g.colscale = colscale;
  g.sA = sA; g.sB = sB; g.sC = sC;
  g.m = m; g.n = n; g.k = k;
  g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.batch = batch; g.tA = tA ? 1 : 0; g.tB = tB ? 1 : 0;
  g.alpha = alpha; g.beta = beta;
  cudaStream_t s = (cudaStream_t)stream;
  void* dp = nullptr;
  void* ep = nullptr;
  if (cudaGetSymbolAddress(&dp, g_tc_selftest_desc) != cudaSuccess) return HT_ERR_CUDA;
  if (cudaGetSymbolAddress(&ep, g_tc_selftest_err) != cudaSuccess) return HT_ERR_CUDA;
  if (cudaMemcpyAsync(dp, &g, sizeof(g), cudaMemcpyHostToDevice, s) != cudaSuccess) return HT_ERR_CUDA;
  if (cudaMemsetAsync(ep, 0, sizeof(int), s) != cudaSuccess) return HT_ERR_CUDA;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HT_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t le = (slices == 1) ? htg_launch_gemm_f32x2((const GemmDesc*)dp, 1, 2 * sms, s, nullptr, 1, 0, 0)
                                        : htg_launch_gemm_tc((const GemmDesc*)dp, 1, sms, slices, s, nullptr, 1, 0, (int*)ep);
  if (le != cudaSuccess) return HT_ERR_CUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, ep, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return HT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return HT_ERR_CUDA;
  return h;
}

// ------------------------------------------------------------- tuning ------------
// Mean CUDA-event time of `reps` launches of one synthetic contraction (m x k times k x n, batch
// entries, seeded values) through the FP64 kernel (route 0, ctas_per_sm CTAs per SM) or the
// tensor-core kernel (route 1, `slices` digit planes).  Allocates and frees its own buffers.
extern "C" int ht_tune_time_gemm(int m, int n, int k, int batch, int route, int slices, int ctas_per_sm, int reps,
                                 double* ms_out) {
  if (m < 1 || n < 1 || k < 1 || batch < 1 || reps < 1 || !ms_out || route < 0 || route > 2) return HT_ERR_ARG;
  if (route == 1 && (slices < 2 || slices > 4)) return HT_ERR_ARG;
  if (route != 1 && (ctas_per_sm < 1 || ctas_per_sm > 32)) return HT_ERR_ARG;
  const size_t na = (size_t)m * k * batch, nb = (size_t)k * n * batch, nc = (size_t)m * n * batch;
  double *A = nullptr, *B = nullptr, *Cm = nullptr;
  GemmDesc* dd = nullptr;
  int* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = HT_OK;
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess) return HT_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaMalloc(&A, na * sizeof(double)) != cudaSuccess || cudaMalloc(&B, nb * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&Cm, nc * sizeof(double)) != cudaSuccess || cudaMalloc(&dd, sizeof(GemmDesc)) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    rc = HT_ERR_NOMEM;
  } else {
    // values in [-1, 1) from a byte pattern (their size does not change the timing)
    if (cudaMemset(A, 0x3f, na * sizeof(double)) != cudaSuccess || cudaMemset(B, 0xbf, nb * sizeof(double)) != cudaSuccess ||
        cudaMemset(err, 0, sizeof(int)) != cudaSuccess)
      rc = HT_ERR_CUDA;
    GemmDesc g;
    g.A = A; g.B = B; g.C = Cm; g.colscale = nullptr;
    g.sA = (long long)m * k; g.sB = (long long)k * n; g.sC = (long long)m * n;
    g.m = m; g.n = n; g.k = k; g.lda = m; g.ldb = k; g.ldc = m;
    g.batch = batch; g.tA = 0; g.tB = 0; g.alpha = 1.0; g.beta = 0.0;
    if (rc == HT_OK && cudaMemcpy(dd, &g, sizeof(g), cudaMemcpyHostToDevice) != cudaSuccess) rc = HT_ERR_CUDA;
    if (rc == HT_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = HT_ERR_CUDA;
    auto launch = [&]() -> cudaError_t {
      if (route == 1) return htg_launch_gemm_tc(dd, 1, sms, slices, 0, nullptr, 1, 0, err, 0);
      if (route == 2) return htg_launch_gemm_f32x2(dd, 1, sms * ctas_per_sm, 0, nullptr, 1, 0, 0);
      return htg_launch_gemm(dd, 1, sms * ctas_per_sm, 0, nullptr, 1, 0, 0);
    };
    if (rc == HT_OK) {
      for (int w = 0; w < 2 && rc == HT_OK; ++w)
        if (launch() != cudaSuccess) rc = HT_ERR_CUDA;
      if (rc == HT_OK && cudaEventRecord(e0, 0) != cudaSuccess) rc = HT_ERR_CUDA;
      for (int r = 0; r < reps && rc == HT_OK; ++r)
        if (launch() != cudaSuccess) rc = HT_ERR_CUDA;
      float ms = 0.f;
      if (rc == HT_OK && (cudaEventRecord(e1, 0) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = HT_ERR_CUDA;
      int h = 0;
      if (rc == HT_OK && cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) rc = HT_ERR_CUDA;
      if (rc == HT_OK && h != 0) rc = h;
      if (rc == HT_OK) *ms_out = (double)ms / reps;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(A);
  cudaFree(B);
  cudaFree(Cm);
  cudaFree(dd);
  cudaFree(err);
  return rc;
}
