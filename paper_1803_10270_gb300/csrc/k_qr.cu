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
// For column j the reflector v = x - alpha e1 (alpha = -sign(x0)|x|) is formed in place and
// every trailing column (one warp each) gets c <- c - tau (v.c) v with tau = 2 / (v.v).  A
// matrix is reduced by one CTA, or, when it is tall (m >= 3k) and its row blocks fit in shared
// memory, in two stages (tall-skinny QR): row blocks by separate CTAs, then their stacked
// triangular factors by the last CTA to finish.  An FP64 Householder sweep is bound by the SM's
// FP64 pipe, so the split buys SMs for the few large matrices of a tree level.
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

// Largest number of row blocks (CTAs) per matrix in the two-stage form.
constexpr int QR_MAXSPLIT = 8;

// A launch whose matrices leave SMs idle runs one CTA per SM anyway: it takes 200 KB, so larger
// matrices, row blocks and stacks of the two-stage form stay in shared memory.  Matrices above
// the 96 KB size are the ones split (below it a single sweep is faster).
constexpr int QR_SMEM_WIDE = 200 * 1024;
constexpr long long QR_SPLIT_MIN = QR_SMEM_BYTES / sizeof(double);

// Householder reflector of column j (rows [j, mend)) from x0 = S[j, j] and t = sum_{i > j}
// S[i, j]^2 (lane 0): v = x - alpha e1 with alpha = -sign(x0) |x| stored over S[j, j], alpha into
// diag[j], and tau = 2 / (v.v) (0 when the column is already zero below and on the diagonal).
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

// 2^k as a double (|k| <= 1000)
__device__ inline double pow2(int k) { return __longlong_as_double((long long)(k + 1023) << 52); }

// The reflector by the whole warp (every lane holds t; lane 0's return value is tau).  A column
// whose squared norm leaves [2^-600, 2^600] (a row block holding only far tails of a Gaussian,
// say: entries near 1e-160 have subnormal squares, v.v underflows and tau = 2 / (v.v)
// overflows) is first scaled by an exact power of two, its squared sub-column norm recomputed,
// and the diagonal entry of R scaled back; the scaled vector gives the same reflection.
__device__ inline double warp_reflector(double* colj, int j, int mend, double t, double* diag, int lane) {
  const double x0 = colj[j];
  const double n2 = fma(x0, x0, t);
  const unsigned long long bits = (unsigned long long)__double_as_longlong(n2);
  const int ex = (int)((bits >> 52) & 0x7FF);
  int k = 0;
  if ((bits << 1) != 0) {
    const int e = (ex == 0) ? -1074 : ex - 1023;   // subnormal: the smallest exponent
    if (e < -600 || e > 600) k = -(e / 2);
  }
  if (k == 0) return lane == 0 ? reflector(colj, j, t, diag) : 0.0;
  const double sc = pow2(k);
  for (int i = j + lane; i < mend; i += 32) colj[i] *= sc;
  __syncwarp();
  double tt = 0.0;
  for (int i = j + 1 + lane; i < mend; i += 32) tt = fma(colj[i], colj[i], tt);
  tt = warp_sum(tt);
  double tau = 0.0;
  if (lane == 0) {
    tau = reflector(colj, j, tt, diag);
    diag[j] *= pow2(-k);
  }
  return tau;
}

// Householder reduction of the m x k column-major matrix S (leading dimension ld, in shared
// memory or scratch) to its R factor: diag receives the diagonal, the strict upper triangle
// stays in S.  Step j applies reflector j to every trailing column c > j: a dot product over the
// rows the step touches, a reduction across the lanes that hold the column, a rank-1 update.
// Warp 0 takes column j+1 alone and forms reflector j+1 at once (look-ahead), so the
// reflector's serial FP64 chain (norm, square root, reciprocal) runs while warps 1.. update the
// other columns.  Those hold a column in L = 32, 16 or 8 lanes (32 / L columns per warp), chosen
// per step to minimise the FP64 instructions of the busiest warp: a warp instruction costs its
// SM partition's FP64 pipe the same whatever its active lanes, so short columns (the banded
// combine, late steps) pack several columns per instruction and pay log2 L reduction levels
// instead of 5.  One CTA barrier per step.
//
// band > 0 declares that column c is zero below row (c+1) band - 1 (the interleaved stack of
// triangular factors in the combine stage); reflectors then keep that pattern, and step j works
// on rows [j, min(m, (j+1) band)) only.
__device__ inline int band_rows(int m, int band, int j) {
  return band > 0 ? htg_min(m, (j + 1) * band) : m;
}

constexpr int QR_UPD_WARPS = NT / 32 - 1;   // warps 1.. update the columns after j+1

// log2 of the lanes per column for a step with `rows` rows and nc columns to update: the busiest
// warp issues passes x (2 ceil(rows / L) + log2 L) FP64 instructions, passes = ceil(nc / slots).
__device__ inline int lanes_log2(int rows, int nc) {
  int best = 5, best_cost = 0x7fffffff;
#pragma unroll
  for (int lg = 5; lg >= 3; --lg) {
    const int L = 1 << lg, slots = QR_UPD_WARPS * (32 >> lg);
    const int cost = ((nc + slots - 1) / slots) * (2 * ((rows + L - 1) / L) + lg);
    if (cost < best_cost) {
      best_cost = cost;
      best = lg;
    }
  }
  return best;
}

__device__ void householder_r(double* S, long long ld, int m, int k, int band, double* diag, double* tau_sh) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int rmax = htg_min(m, k);
  // reflector 0 by warp 0
  if (wid == 0 && rmax > 0) {
    const int m0 = band_rows(m, band, 0);
    double s = 0.0;
    for (int i = 1 + lane; i < m0; i += 32) s = fma(S[i], S[i], s);
    s = warp_sum(s);
    const double t0 = warp_reflector(S, 0, m0, s, diag, lane);
    if (lane == 0) tau_sh[0] = t0;
  }
  __syncthreads();
  for (int j = 0; j < rmax; ++j) {
    const double tau = tau_sh[j & 1];
    const double* v = S + ld * j;
    const int mj = band_rows(m, band, j);
    if (wid == 0) {
      if (j + 1 < k) {
        double* cc = S + ld * (j + 1);
        double dot = 0.0;
        for (int i = j + lane; i < mj; i += 32) dot = fma(v[i], cc[i], dot);
        const double wgt = warp_sum(dot) * tau;
        if (j + 1 < rmax) {
          // update column j+1 and form reflector j+1 from its new entries (with band > 0 its
          // support reaches rows [mj, m_{j+1}) that reflector j left untouched)
          const int mj1 = band_rows(m, band, j + 1);
          double ss = 0.0;
          for (int i = j + lane; i < mj1; i += 32) {
            double x = cc[i];
            if (i < mj) {
              x = fma(-wgt, v[i], x);
              cc[i] = x;
            }
            if (i > j + 1) ss = fma(x, x, ss);
          }
          ss = warp_sum(ss);
          __syncwarp();
          const double tj = warp_reflector(cc, j + 1, mj1, ss, diag, lane);
          if (lane == 0) tau_sh[(j + 1) & 1] = tj;
          __syncwarp();
        } else {
          for (int i = j + lane; i < mj; i += 32) cc[i] = fma(-wgt, v[i], cc[i]);
        }
      }
    } else {
      const int nc = k - j - 2;                            // columns j+2 .. k-1
      const int lg = lanes_log2(mj - j, nc);               // uniform over the CTA
      const int L = 1 << lg, grp = lane >> lg, gl = lane & (L - 1);
      const int slots = QR_UPD_WARPS << (5 - lg);
      const int passes = nc > 0 ? (nc + slots - 1) / slots : 0;
      // slot = pass * slots + grp * QR_UPD_WARPS + (wid - 1): consecutive columns on different warps
      for (int p = 0; p < passes; ++p) {
        const int sl = p * slots + grp * QR_UPD_WARPS + (wid - 1);
        const bool act = sl < nc;
        double* cc = S + ld * (j + 2 + (act ? sl : 0));
        double dot = 0.0;
        if (act)
          for (int i = j + gl; i < mj; i += L) dot = fma(v[i], cc[i], dot);
        for (int o = L >> 1; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const double wgt = dot * tau;
        if (act)
          for (int i = j + gl; i < mj; i += L) cc[i] = fma(-wgt, v[i], cc[i]);
      }
    }
    __syncthreads();
  }
}

// Flops of householder_r: the sub-column norm (2 per entry) and the dot and update of every
// trailing column (4 per entry), over the rows each step touches.
__device__ double householder_flops(int m, int k, int band) {
  double f = 0.0;
  const int rmax = htg_min(m, k);
  for (int j = 0; j < rmax; ++j) {
    const double rows = (double)(band_rows(m, band, j) - j);
    f += 2.0 * rows + 4.0 * rows * (k - j - 1);
  }
  return f;
}

// Row blocks of the two-stage form: ns blocks for a matrix that does not fit in shared memory
// (one CTA would sweep it in its L2-resident scratch buffer) when the blocks and the stack of
// their triangular factors do fit and there are at least three rows per column.  A matrix that
// fits stays whole: its sweep is latency bound, and two stages double the serial steps.
// Stage 1 costs about (m / ns) k^2 / 2 and the banded combine about ns k^3 / 6 element
// updates, balanced at ns^2 = 3 m / k.
__device__ inline int qr_splits(int m, int k, int gsplit, long long room) {
  if (gsplit < 2 || m < 3 * k || (long long)(m | 1) * k <= QR_SPLIT_MIN - ((k + 1) & ~1)) return 1;
  int ns = 1;
  while (ns < gsplit && (long long)(ns + 1) * (ns + 1) * k <= 3LL * m) ++ns;
  while (ns > 1 && (long long)((ns * k) | 1) * k > room) --ns;              // stack in shared memory
  if (ns > 1 && (long long)(((m + ns - 1) / ns) | 1) * k > room) ns = 1;    // row block in shared memory
  return ns;
}

// One matrix per CTA (gsplit = 1, or a matrix the split rule keeps whole): the matrix is copied
// into shared memory (or its scratch buffer, L2 resident, when it does not fit) and reduced in
// place.  Two-stage form (TSQR, ns > 1): CTA s of the matrix reduces the row block
// [s mb, (s+1) mb) in shared memory and stores its k x k triangular factor R_s into the scratch
// buffer, interleaved (row r of R_s at stack row r ns + s); the last CTA to finish (a ticket
// counter, no waiting) reduces the ns k x k stack, whose column c is zero below row
// (c+1) ns - 1, with the banded sweep, and writes R.  Q = diag(Q_s) Q_stack, so R is the R
// factor of op(A) up to an orthogonal factor on the left, which the truncation never sees.
// Matrices the cooperative form takes (when the launch offers it): more than 2^16 entries and at
// least twice as tall as wide.  One CTA sweeps such a matrix out of L2 for milliseconds to
// seconds, and the two-stage form cannot hold its row blocks and stack on chip beyond about
// 200 KB x 8 blocks; smaller matrices keep the one-CTA and two-stage forms.
__device__ inline bool qr_coop_eligible(int m, int k) {
  return (long long)m * k > (1LL << 16) && m >= 2 * k;
}

__global__ void __launch_bounds__(NT) qr_r_kernel(const QrDesc* __restrict__ descs, long long inst_stride,
                                                 long long smem_doubles, int gsplit, int coop, double* flops) {
  // batched launches: instance blockIdx.y reads its own descriptor list, inst_stride bytes on
  const QrDesc q = ((const QrDesc*)((const char*)descs + inst_stride * blockIdx.y))[blockIdx.x / gsplit];
  const int part = blockIdx.x % gsplit;
  const int m = q.m, k = q.k;
  const int kd = (k + 1) & ~1;   // diagonal entries, rounded to keep the matrix 16-byte aligned
  if (m <= 0 || k <= 0 || kd > smem_doubles) {
    if (threadIdx.x == 0 && part == 0 && q.rows_out) *q.rows_out = 0;
    return;
  }
  if (coop && qr_coop_eligible(m, k)) return;   // reduced by qr_coop_kernel
  const long long room = smem_doubles - kd;
  const int ns = q.ticket ? qr_splits(m, k, gsplit, room) : 1;
  if (part >= ns) return;
  extern __shared__ double diag[];   // the k diagonal entries of R, then the matrix when it fits
  __shared__ double tau_sh[2];
  __shared__ int last_sh;
  const int tid = threadIdx.x;
  double* S;
  int mw;                            // rows of the matrix this CTA reduces
  long long ld;                      // its leading dimension (odd in shared memory)
  int band = 0;
  double f = 0.0;
  if (ns == 1) {
    mw = m;
    const bool fits = (long long)(m | 1) * k <= room;
    S = fits ? diag + kd : q.scratch;
    ld = fits ? (m | 1) : m;
    for (long long e = tid; e < (long long)m * k; e += NT) {
      const int i = (int)(e % m), c = (int)(e / m);
      S[i + ld * c] = q.tA ? q.A[c + (long long)q.lda * i] : q.A[i + (long long)q.lda * c];
    }
    __syncthreads();
  } else {
    // ---- stage 1: the row block of this CTA
    const int mb = (m + ns - 1) / ns;
    const int r0 = part * mb;
    const int ms = htg_max(0, htg_min(mb, m - r0));
    S = diag + kd;
    ld = ms | 1;
    for (long long e = tid; e < (long long)ms * k; e += NT) {
      const int i = (int)(e % ms), c = (int)(e / ms);
      const long long ig = r0 + i;
      S[i + ld * c] = q.tA ? q.A[c + (long long)q.lda * ig] : q.A[ig + (long long)q.lda * c];
    }
    __syncthreads();
    householder_r(S, ld, ms, k, 0, diag, tau_sh);
    if (tid == 0 && flops) f += householder_flops(ms, k, 0);
    // R_s into the interleaved stack (rows beyond min(ms, k) are zero)
    const int M2 = ns * k, rs = htg_min(ms, k);
    double* stack = q.scratch;
    for (int e = tid; e < k * k; e += NT) {
      const int r = e % k, c = e / k;
      double val = 0.0;
      if (r < rs) val = (c == r) ? diag[r] : (c > r ? S[r + ld * c] : 0.0);
      stack[(long long)(r * ns + part) + (long long)M2 * c] = val;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) last_sh = (atomicAdd(q.ticket, 1u) == (unsigned)(ns - 1));
    __syncthreads();
    if (!last_sh) {
      if (tid == 0 && flops && f > 0.0) atomicAdd(flops, f);
      return;
    }
    // ---- stage 2 (last CTA): the banded stack
    __threadfence();
    if (tid == 0) *q.ticket = 0u;    // ready for the next launch (stream ordered)
    ld = M2 | 1;
    for (int e = tid; e < M2 * k; e += NT) S[(e % M2) + ld * (e / M2)] = __ldcg(stack + e);
    __syncthreads();
    mw = M2;
    band = ns;
  }
  householder_r(S, ld, mw, k, band, diag, tau_sh);
  // write R (rmax x k upper trapezoidal) or its transpose
  const int rmax = htg_min(mw, k);
  const long long rk = (long long)rmax * k;
  for (long long e = tid; e < rk; e += NT) {
    const int r = (int)(e % rmax), c = (int)(e / rmax);
    double val = 0.0;
    if (c == r) val = diag[r];
    else if (c > r) val = S[r + ld * c];
    if (q.tR) q.R[c + (long long)q.ldr * r] = val;
    else q.R[r + (long long)q.ldr * c] = val;
  }
  if (tid == 0 && q.rows_out) *q.rows_out = rmax;
  if (tid == 0 && flops) atomicAdd(flops, f + householder_flops(mw, k, band));
}


// ---------------------------------------------------------------- cooperative form ----
// One CTA per SM, shared out over the launch's wide matrices in proportion to their work m k^2
// (an equal share per matrix left the largest matrix of a level setting the launch time: 33 ms
// for a level whose work split by weight takes about half); CTA g of a matrix's G owns the rows
// [g mb, (g+1) mb).
// Column j: (1) each CTA forms the partial dot products of column j with the columns c >= j
// over its rows >= j (c = j gives the squared norm), and the owner of row j publishes that row;
// (2) after a barrier of the matrix's CTAs, CTA g totals the columns c = j + g (mod G); (3)
// after a second barrier every CTA forms the same reflector from the totals (alpha, and tau
// split as (1 / |x|) (1 / (|x0| + |x|)) so that it does not overflow for tiny columns) and
// updates its own rows: v.c = x.c - alpha c_j, c <- c - tau (v.c) v.  R is the rows j of the
// updated matrix and the alphas.  Barriers are per matrix, by arrival words, each wait bounded
// (HT_ERR_TIMEOUT, and the CTA returns).  A CTA whose row block (its rows x k doubles) fits the
// launch's dynamic shared memory keeps it there for the whole reduction, so the column passes
// (dot products and updates) never leave the SM; otherwise the block lives in the matrix's
// scratch buffer in global memory (an ncu capture of that form measured 76x the matrix's bytes
// of DRAM traffic: one pass over the trailing part per column).
constexpr int QRC_NT = 256;
constexpr int QRC_SMEM_BYTES = 200 * 1024;
constexpr long long QRC_TIMEOUT_CYCLES = 400000000LL;   // about 0.2 s

__device__ bool coop_barrier(unsigned* flags, int G, int g, unsigned seq, int* err) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x < 32) {
    if (threadIdx.x == 0) {
      __threadfence();
      *(volatile unsigned*)(flags + g) = seq;
    }
    __syncwarp();
    int ok = 1;
    const long long t0 = clock64();
    for (int i = threadIdx.x; i < G && ok; i += 32) {
      while (*(volatile unsigned*)(flags + i) < seq) {
        if (clock64() - t0 > QRC_TIMEOUT_CYCLES) {
          ok = 0;
          break;
        }
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && threadIdx.x == 0 && err) atomicCAS(err, 0, (int)HT_ERR_TIMEOUT);
    __threadfence();
    if (threadIdx.x == 0) ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

__global__ void __launch_bounds__(QRC_NT) qr_coop_kernel(const QrDesc* __restrict__ descs, int ndesc, QrCoopWs w,
                                                        int smem_doubles, double* flops) {
  // The launch's CTAs are shared out over the eligible matrices in proportion to their work
  // m k^2: two each, and the rest of the grid by those weights (the same computation in every
  // CTA, so all agree).  Against an equal share of at most 64 CTAs per matrix: the kinetic
  // workload's QR went from 122 to 100 ms per step (its largest matrices got 64-84 CTAs instead
  // of 38); two equal 36864 x 192 matrices (76 CTAs each instead of 64) within run-to-run
  // spread.  CTA g of matrix d's group of G sits at grid position base + g; barrier
  // words and partial sums are indexed by grid position.
  __shared__ int s_d, s_g, s_G, s_base;
  if (threadIdx.x == 0) {
    double wsum = 0.0;
    int ne = 0;
    for (int i = 0; i < ndesc; ++i) {
      const QrDesc qi = descs[i];
      if (qi.m > 0 && qi.k > 0 && qr_coop_eligible(qi.m, qi.k)) {
        wsum += (double)qi.m * qi.k * qi.k;
        ++ne;
      }
    }
    const int spare = htg_max(0, (int)gridDim.x - 2 * ne);
    int base = 0;
    s_d = -1;
    for (int i = 0; i < ndesc; ++i) {
      const QrDesc qi = descs[i];
      int Gi = 0;
      if (qi.m > 0 && qi.k > 0 && qr_coop_eligible(qi.m, qi.k))
        Gi = htg_min(htg_max(2, qi.m / 64), 2 + (int)(spare * ((double)qi.m * qi.k * qi.k / wsum)));
      if ((int)blockIdx.x >= base && (int)blockIdx.x < base + Gi) {
        s_d = i;
        s_g = (int)blockIdx.x - base;
        s_G = Gi;
        s_base = base;
      }
      base += Gi;
    }
  }
  __syncthreads();
  if (s_d < 0) return;   // a CTA beyond the shares (uniform over the CTA)
  const int d = s_d, g = s_g, G = s_G, gbase = s_base;
  const QrDesc q = descs[d];
  const int m = q.m, k = q.k;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = QRC_NT / 32;
  // the matrix's Householder flops, counted once (by its group's first CTA) as the one-CTA form counts them
  if (g == 0 && tid == 0 && flops) atomicAdd(flops, householder_flops(m, k, 0));
  const int mb = (m + G - 1) / G, r0 = htg_min(m, g * mb), r1 = htg_min(m, r0 + mb);
  // the CTA's rows [r0, r1): in shared memory (ld mb) when they fit, else in the scratch buffer
  // (ld m); S points at row r0, so element (i, c) of the matrix is S[(i - r0) + ld c]
  extern __shared__ double qsm[];
  // ... together with the QB x max(k, QRC_NT) staging area of the panel updates
  const bool local = (long long)mb * k + (long long)QR_COOP_QB * htg_max(k, QRC_NT) <= (long long)smem_doubles;
  const long long ld = local ? mb : m;
  double* S = local ? qsm : q.scratch + r0;
  double* part = w.part + ((long long)gbase + g) * w.kmax;
  double* part0 = w.part + (long long)gbase * w.kmax;
  double* tot = w.tot + (long long)d * w.kmax;
  // row j is published into one of two buffers by step parity: a CTA may publish row j+1 while
  // a slower one still reads row j (no barrier between a step's update and the next step's
  // dot products); two steps apart, the next step's first barrier separates them
  double* rowj2 = w.rowj + (long long)d * 2 * w.kmax;
  double* diag = w.diag + (long long)d * w.kmax;
  unsigned* flags = w.bar + gbase;
  __shared__ double wc[1024];                // (v.c) tau for the columns of one step
  __shared__ double sh_v0, sh_alpha;
  for (long long e = tid; e < (long long)(r1 - r0) * k; e += QRC_NT) {
    const int i = r0 + (int)(e % (r1 - r0)), c = (int)(e / (r1 - r0));
    S[(i - r0) + ld * c] = q.tA ? q.A[c + (long long)q.lda * i] : q.A[i + (long long)q.lda * c];
  }
  unsigned seq = 0;
  const int rmax = htg_min(m, k);
  constexpr int QB = QR_COOP_QB;
  const long long slotsz = (long long)QB * (QB + w.kmax);
  // the panels' partial blocks after the column steps' partial sums (QR_COOP_SLOTS x kmax): the
  // launch's matrices run independently, so the two kinds must not share memory
  double* slots = w.part + 2LL * QR_COOP_SLOTS * w.kmax;
  double* wtot = w.wtot + (long long)d * slotsz;   // the panel's reduced [V^T V | V^T C], then W
  double* wsm = local ? qsm + (long long)mb * k : qsm;   // QB x max(k, QRC_NT) staging
  __shared__ double v0s[QB], taus[QB];
  // V(i, p) of the current panel (rows i >= j0): 0 above its diagonal, v0 on it, the reduced
  // column below
  auto vval = [&](int i, int p, int j0) -> double {
    const int jd = j0 + p;
    return (i < jd) ? 0.0 : (i == jd ? v0s[p] : S[(i - r0) + ld * jd]);
  };
  for (int j0 = 0; j0 < rmax; j0 += QB) {
    const int j1 = htg_min(rmax, j0 + QB), pb = j1 - j0;
    // ---- the panel: columns j0 .. j1-1 one at a time, restricted to the panel's columns, one
    // barrier per column: the partial dot products go to one of two buffers by step parity (as
    // row j does), and after the barrier every CTA sums the panel's few columns itself
    __shared__ double ptot[QB];
    for (int j = j0; j < j1; ++j) {
      __syncthreads();
      const int i0 = htg_max(j, r0);
      const double* x = S + ld * j;
      double* partj = part + (long long)(j & 1) * QR_COOP_SLOTS * w.kmax;
      const double* part0j = part0 + (long long)(j & 1) * QR_COOP_SLOTS * w.kmax;
      for (int c = j + wid; c < j1; c += nw) {
        const double* cc = S + ld * c;
        double sdot = 0.0;
        for (int i = i0 + lane; i < r1; i += 32) sdot = fma(x[i - r0], cc[i - r0], sdot);
        sdot = warp_sum(sdot);
        if (lane == 0) partj[c] = sdot;
      }
      double* rowj = rowj2 + (long long)(j & 1) * w.kmax;
      if (j >= r0 && j < r1)
        for (int c = j + tid; c < j1; c += QRC_NT) rowj[c] = S[(j - r0) + ld * c];
      if (!coop_barrier(flags, G, g, ++seq, w.err)) return;
      for (int c = j + wid; c < j1; c += nw) {
        double t = 0.0;
        for (int h = lane; h < G; h += 32) t += __ldcg(part0j + (long long)h * w.kmax + c);
        t = warp_sum(t);
        if (lane == 0) ptot[c - j0] = t;
      }
      __syncthreads();
      // the reflector of column j (every CTA forms the same one)
      const int nc = j1 - j - 1;
      if (tid == 0) {
        const double n2 = ptot[j - j0], x0 = __ldcg(rowj + j);
        double alpha = 0.0, v0 = 0.0, ri = 0.0, rv = 0.0;
        if (htg_dpos(n2)) {
          const double nrm = sqrt(n2);
          alpha = htg_dpos(x0) ? -nrm : nrm;
          v0 = x0 - alpha;
          ri = 1.0 / nrm;
          rv = 1.0 / (fabs(x0) + nrm);      // tau = 2 / (v.v) = ri rv
        }
        sh_v0 = v0;
        sh_alpha = alpha;
        wc[0] = ri;
        wc[1] = rv;
        v0s[j - j0] = v0;
        taus[j - j0] = ri * rv;
        if (j >= r0 && j < r1) diag[j] = alpha;   // read back at the end by this CTA only
      }
      __syncthreads();
      const double ri = wc[0], rv = wc[1], alpha = sh_alpha, v0 = sh_v0;
      __syncthreads();
      for (int t = tid; t < nc; t += QRC_NT) {
        const int c = j + 1 + t;
        const double vc = ptot[c - j0] - alpha * __ldcg(rowj + c);
        wc[t] = (vc * ri) * rv;
      }
      __syncthreads();
      for (long long e = tid; e < (long long)(r1 - i0) * nc; e += QRC_NT) {
        const int i = i0 + (int)(e % (r1 - i0)), c = j + 1 + (int)(e / (r1 - i0));
        const double vi = (i == j) ? v0 : x[i - r0];
        S[(i - r0) + ld * c] = fma(-wc[c - (j + 1)], vi, S[(i - r0) + ld * c]);
      }
    }
    if (j1 >= k) continue;
    // ---- the panel's reflectors applied to the trailing columns at once:
    // H_{j1-1} ... H_{j0} = I - V T^T V^T (T upper triangular, T^-1 = diag(1 / tau) + the strictly
    // upper part of V^T V), so C <- C - V W with (diag(1 / tau) + strict lower of V^T V) W = V^T C
    const int nct = k - j1, ncol = pb + nct;
    const int i0 = htg_max(j0, r0);
    __syncthreads();
    {
      // partial [V^T V | V^T C] over this CTA's rows i >= j0: entry (p, q) at slot[p + QB q].
      // Columns in passes of at most QRC_NT (a thread's QB accumulators stay in registers); a pass
      // with fewer columns than threads splits the rows into P parts.  A row block in L2 goes
      // through shared memory in chunks of rc rows: V's QB columns and the pass's columns, loaded
      // with lanes over rows (coalesced), read with lanes over columns (odd stride: no bank
      // conflicts) and V broadcast.
      const int nrow = htg_max(0, r1 - i0);
      double* slot = slots + ((long long)gbase + g) * slotsz;
      double* stg = wsm + (long long)QB * htg_max(k, QRC_NT);
      for (int qa = 0; qa < ncol; qa += QRC_NT) {
        const int nq = htg_min(QRC_NT, ncol - qa);
        const int P = (nq < QRC_NT) ? htg_max(1, htg_min(8, QRC_NT / nq)) : 1;
        const int qc = qa + tid % nq, rp = tid / nq;
        const bool mine = tid < nq * P;
        double acc[QB];
#pragma unroll
        for (int p = 0; p < QB; ++p) acc[p] = 0.0;
        if (local) {
          if (mine) {
            const int chunk = (nrow + P - 1) / P;
            const int ia = i0 + rp * chunk, ib = htg_min(r1, ia + chunk);
            for (int i = ia; i < ib; ++i) {
              const double xq = (qc < pb) ? vval(i, qc, j0) : S[(i - r0) + ld * (j1 + qc - pb)];
#pragma unroll
              for (int p = 0; p < QB; ++p)
                if (p < pb) acc[p] = fma(vval(i, p, j0), xq, acc[p]);
            }
          }
        } else {
          const int nqp = nq | 1;
          const int avail = smem_doubles - QB * htg_max(k, QRC_NT);
          const int RC = htg_max(1, htg_min(nrow, avail / (nqp + QB)));
          double* Xs = stg;
          double* Vs = stg + (long long)RC * nqp;
          for (int c0 = i0; c0 < r1; c0 += RC) {
            const int rc = htg_min(RC, r1 - c0);
            __syncthreads();   // the previous chunk is consumed
            for (int q = wid; q < nq; q += nw) {
              const int qq = qa + q;
              for (int ri = lane; ri < rc; ri += 32)
                Xs[(long long)ri * nqp + q] = (qq < pb) ? vval(c0 + ri, qq, j0) : S[(c0 + ri - r0) + ld * (j1 + qq - pb)];
            }
            for (int p = wid; p < QB; p += nw)
              for (int ri = lane; ri < rc; ri += 32) Vs[ri * QB + p] = (p < pb) ? vval(c0 + ri, p, j0) : 0.0;
            __syncthreads();
            if (mine) {
              for (int ri = rp; ri < rc; ri += P) {
                const double xq = Xs[(long long)ri * nqp + (qc - qa)];
                const double* vrow = Vs + ri * QB;
#pragma unroll
                for (int p = 0; p < QB; ++p) acc[p] = fma(vrow[p], xq, acc[p]);
              }
            }
          }
        }
        if (P == 1) {
          if (mine) {
#pragma unroll
            for (int p = 0; p < QB; ++p) slot[p + (long long)QB * qc] = acc[p];
          }
        } else {
          __syncthreads();
          if (mine) {
#pragma unroll
            for (int p = 0; p < QB; ++p) wsm[((long long)rp * QB + p) * nq + (qc - qa)] = acc[p];
          }
          __syncthreads();
          for (int t = tid; t < QB * nq; t += QRC_NT) {
            const int p = t % QB, q = t / QB;
            double v = 0.0;
            for (int r2 = 0; r2 < P; ++r2) v += wsm[((long long)r2 * QB + p) * nq + q];
            slot[p + (long long)QB * (qa + q)] = v;
          }
          __syncthreads();
        }
      }
    }
    if (!coop_barrier(flags, G, g, ++seq, w.err)) return;
    // the totals: CTA g sums the columns q = g, g + G, ... over the G slots
    for (int t = tid; t < QB * ((ncol - g + G - 1) / G); t += QRC_NT) {
      const int p = t % QB, qc = g + G * (t / QB);
      const double* src = slots + (long long)gbase * slotsz + p + (long long)QB * qc;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int h = 0;
      for (; h + 3 < G; h += 4) {
        s0 += __ldcg(src + (long long)h * slotsz);
        s1 += __ldcg(src + (long long)(h + 1) * slotsz);
        s2 += __ldcg(src + (long long)(h + 2) * slotsz);
        s3 += __ldcg(src + (long long)(h + 3) * slotsz);
      }
      for (; h < G; ++h) s0 += __ldcg(src + (long long)h * slotsz);
      wtot[p + (long long)QB * qc] = (s0 + s1) + (s2 + s3);
    }
    if (!coop_barrier(flags, G, g, ++seq, w.err)) return;
    // W for this CTA's trailing columns, in place: W_p = tau_p (Y_p - sum_{s<p} (V^T V)_{sp} W_s)
    for (int qc = g + G * tid; qc < ncol; qc += G * QRC_NT) {
      if (qc < pb) continue;
      double wv[QB];
#pragma unroll
      for (int p = 0; p < QB; ++p) {
        if (p < pb) {
          double y = wtot[p + (long long)QB * qc];
          for (int s2 = 0; s2 < p; ++s2) y = fma(-__ldcg(wtot + s2 + (long long)QB * p), wv[s2], y);
          wv[p] = taus[p] * y;
          wtot[p + (long long)QB * qc] = wv[p];
        }
      }
    }
    if (!coop_barrier(flags, G, g, ++seq, w.err)) return;
    // C <- C - V W on this CTA's rows i >= j0: W staged in shared memory, a row's V in registers
    for (int t = tid; t < QB * nct; t += QRC_NT) wsm[t] = __ldcg(wtot + (long long)QB * pb + t);
    __syncthreads();
    // thread -> (row, part of the columns): rows by consecutive threads (coalesced), the columns
    // split in CP parts when the rows are fewer than the threads
    const int rows_cnt = htg_max(0, r1 - i0);
    const int CP = (rows_cnt > 0 && rows_cnt < QRC_NT) ? htg_max(1, htg_min(8, QRC_NT / rows_cnt)) : 1;
    const int cch = (nct + CP - 1) / CP;
    for (int t = tid; t < rows_cnt * CP; t += QRC_NT) {
      const int i = i0 + t % rows_cnt, cpi = t / rows_cnt;
      const int ca = cpi * cch, cb = htg_min(nct, ca + cch);
      double vr[QB];
#pragma unroll
      for (int p = 0; p < QB; ++p) vr[p] = (p < pb) ? vval(i, p, j0) : 0.0;
      double* srow = S + (i - r0);
      for (int c = ca; c < cb; ++c) {
        const double* wcol = wsm + (long long)QB * c;
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int p = 0; p < QB; p += 2) {
          a0 = fma(vr[p], wcol[p], a0);
          a1 = fma(vr[p + 1], wcol[p + 1], a1);
        }
        srow[ld * (j1 + c)] -= a0 + a1;
      }
    }
  }
  // R: rows r < rmax of this CTA (diag from the alphas, upper part from the updated rows)
  __syncthreads();
  for (long long e = tid; e < (long long)(r1 - r0) * k; e += QRC_NT) {
    const int r = r0 + (int)(e % (r1 - r0)), c = (int)(e / (r1 - r0));
    if (r >= rmax) continue;
    double val = 0.0;
    if (c == r) val = diag[r];
    else if (c > r) val = S[(r - r0) + ld * c];
    if (q.tR) q.R[c + (long long)q.ldr * r] = val;
    else q.R[r + (long long)q.ldr * c] = val;
  }
  if (g == 0 && tid == 0 && q.rows_out) *q.rows_out = rmax;
}

}  // namespace

cudaError_t htg_launch_qr(const QrDesc* descs_dev, int ndesc, cudaStream_t s, double* flops, int count,
                          long long inst_stride, const QrCoopWs* coop) {
  if (ndesc <= 0 || count <= 0) return cudaSuccess;
  if (count > 65535) return cudaErrorInvalidValue;
  static bool attr[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(qr_r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, QR_SMEM_WIDE);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr[dev] = true;
  }
  // the split buys idle SMs: a launch whose matrices already outnumber the SMs keeps them whole
  static int sms[64] = {0};
  if (dev >= 0 && dev < 64 && sms[dev] == 0) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
  const int nsm = (dev >= 0 && dev < 64 && sms[dev] > 0) ? sms[dev] : 1;
  const int gsplit = ((long long)ndesc * count < nsm) ? QR_MAXSPLIT : 1;
  const int smem = gsplit > 1 ? QR_SMEM_WIDE : QR_SMEM_BYTES;
  // the cooperative form gives every wide matrix at least two CTAs of a one-per-SM grid
  const bool use_coop = coop && count == 1 && ndesc <= coop->ndmax && 2 * ndesc <= htg_min(nsm, QR_COOP_SLOTS) &&
                        ((long long)QR_COOP_QB * htg_max(coop->kmax, QRC_NT) + QRC_NT + 1 + QR_COOP_QB) *
                                (long long)sizeof(double) <= QRC_SMEM_BYTES;
  qr_r_kernel<<<dim3(ndesc * gsplit, count), NT, smem, s>>>(
      descs_dev, inst_stride, (long long)(smem / sizeof(double)), gsplit, use_coop ? 1 : 0, flops);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !use_coop) return e;
  // the wide matrices: one CTA per SM (all resident, cooperative launch), shared out over the
  // matrices by their work inside the kernel; barrier words and partial sums by grid position
  // (the workspace holds QR_COOP_SLOTS of each)
  const int grid = htg_min(nsm, QR_COOP_SLOTS);
  e = cudaMemsetAsync(coop->bar, 0, (size_t)grid * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  static bool cattr[64] = {false};
  if (dev < 0 || dev >= 64 || !cattr[dev]) {
    e = cudaFuncSetAttribute(qr_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, QRC_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) cattr[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(QRC_NT);
  cfg.dynamicSmemBytes = QRC_SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute lattr[1];
  lattr[0].id = cudaLaunchAttributeCooperative;
  lattr[0].val.cooperative = 1;
  cfg.attrs = lattr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, qr_coop_kernel, descs_dev, ndesc, *coop, (int)(QRC_SMEM_BYTES / sizeof(double)), flops);
}
