// Crank-Nicolson time step solved by CP alternating least squares (Section 3.3, eqs. CNFDE,
// BLs, rRr1, ALS2, ML, MR, eq:77).
//
// With L = sum_q alpha_q prod_k L_k^q the Crank-Nicolson operators are separable,
//   A = I - dt/2 L = sum_{e=0}^{T-1} eta_e prod_k E_k^e,   B = I + dt/2 L = sum_e zeta_e prod_k E_k^e,
// E^0 the identity (eta_0 = zeta_0 = 1), E^e the e-th term of L, eta_e = -dt/2 alpha_e and
// zeta_e = +dt/2 alpha_e.  The step minimises |A x - B x_n| over the factors of the CP tensor x
// (rank r), one dimension q at a time (Gauss-Seidel).  With the other factors fixed the normal
// equations of dimension q are (grid basis: the 1-D integrals of eq:77 are the grid products
// S^{ez}_q = (E_q^e)^T E_q^z)
//   M vec(V) = vec(R),  M = sum_{e,z} eta_e eta_z Gamma^{ez} kron S^{ez}_q     ((n r) x (n r)),
//   R = sum_{e,z} eta_e zeta_z S^{ez}_q Xn_q diag(lam_n) Gn^{ezT},
//   Gamma^{ez} = hadamard_{k != q} (E_k^e X_k)^T (E_k^z X_k),  Gn^{ez} = hadamard_{k != q} (E_k^e X_k)^T (E_k^z Xn_k),
// and V (n x r, vec column major) is the new X_q.  Kernels: the dense 1-D factors E_k^e and the
// products S^{ez}_k once per call; Y^e_k = E_k^e X_k, Yn^e_k = E_k^e Xn_k and their Grams for
// every dimension once, then for dimension q only after it changes; per mode solve the
// Hadamard products, the assembly of M and R (one thread per entry), and a one-CTA Cholesky of
// M with the forward substitution fused in (shared memory when M fits), back substitution,
// and the update of X_q with the increment |X_q^new - X_q^old|^2 of the sweep (the paper's
// convergence measure).
#include <cstring>

#include "common.cuh"

namespace {

constexpr int NT = 256;
constexpr int CN_MAXT = HT_MAXBLOCKTERMS + 1;   // identity + the operator's terms
constexpr int CN_SOLVE_SMEM = 200 * 1024;

struct CnDims {
  int d, T, R, nmax;
  int n[HT_MAXD];
};

// Workspace views: T = max_terms + 1 blocks, R = rank capacity, nmax = largest grid.
struct CnWs {
  double* Ed;    // T x d x nmax^2      E_k^e, column major, ld nmax
  double* S;     // T x T x d x nmax^2  (E_k^e)^T E_k^z
  double* Y;     // T x d x nmax x R    E_k^e X_k   (ld nmax)
  double* Yn;    // T x d x nmax x R    E_k^e Xn_k  (ld nmax)
  double* G;     // d x T x T x R^2     (E_k^e X_k)^T (E_k^z X_k)    (ld R)
  double* Gn;    // d x T x T x R^2     (E_k^e X_k)^T (E_k^z Xn_k)   (ld R)
  double* Gam;   // T x T x R^2         hadamard over k != q of G
  double* Gamn;  // T x T x R^2         hadamard over k != q of Gn
  double* M;     // (nmax R)^2          the system, column major, ld N
  double* Rh;    // nmax R              right-hand side, then the solution
  double* eps;   // 64                  increments per sweep
  double* V;     // d x nmax x R         parallel variant: every mode's solution (ld n_k)
};

struct CnArgs {
  int d, r, rn, T;
  int n[HT_MAXD];
  double eta[CN_MAXT], zeta[CN_MAXT];
  double* X[HT_MAXD];         // x factors (n_k x r, ld n_k), updated in place
  const double* Xn[HT_MAXD];  // x_n factors (n_k x rn, ld n_k)
  double* lam;                // x weights (1 after the call)
  const double* lamn;         // x_n weights
};

__device__ inline long long ed_off(const CnDims& m, int e, int k) {
  return ((long long)e * m.d + k) * m.nmax * m.nmax;
}
__device__ inline long long s_off(const CnDims& m, int e, int z, int k) {
  return (((long long)e * m.T + z) * m.d + k) * m.nmax * m.nmax;
}
__device__ inline long long y_off(const CnDims& m, int e, int k) {
  return ((long long)e * m.d + k) * m.nmax * m.R;
}
__device__ inline long long g_off(const CnDims& m, int k, int e, int z) {
  return (((long long)k * m.T + e) * m.T + z) * m.R * m.R;
}

// E_k^e as dense n_k x n_k matrices ((A u)_i = sum_j A_ij u_j); term e >= 1 is L's term e-1
__global__ void cn_dense_kernel(ht_op L, CnWs w, CnDims m) {
  const long long nn = (long long)m.nmax * m.nmax;
  const long long total = (long long)m.T * m.d * nn;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t / ((long long)m.d * nn));
    const int k = (int)((t / nn) % m.d);
    const int j = (int)((t % nn) / m.nmax), i = (int)(t % m.nmax);
    const int n = m.n[k];
    double v = 0.0;
    if (i < n && j < n) {
      if (e == 0) {
        v = (i == j) ? 1.0 : 0.0;
      } else {
        const ht_factor& f = L.f[e - 1][k];
        switch (f.kind) {
          case HT_F_IDENTITY: v = (i == j) ? 1.0 : 0.0; break;
          case HT_F_STENCIL:
          case HT_F_DIAG_STENCIL: {
            double s = 0.0;
            for (int o = -f.half_width; o <= f.half_width; ++o) {
              int jj = (i + o) % n;
              if (jj < 0) jj += n;
              if (jj == j) s += f.stencil[o + f.half_width];
            }
            v = (f.kind == HT_F_DIAG_STENCIL) ? f.v[i] * s : s;
            break;
          }
          case HT_F_DIAG: v = (i == j) ? f.v[i] : 0.0; break;
          case HT_F_RANK1: v = f.v[i] * f.w[j]; break;
        }
      }
    }
    w.Ed[ed_off(m, e, k) + i + (long long)m.nmax * j] = v;
  }
}

// S^{ez}_k = (E_k^e)^T E_k^z
__global__ void cn_sgram_kernel(CnWs w, CnDims m) {
  const long long nn = (long long)m.nmax * m.nmax;
  const long long total = (long long)m.T * m.T * m.d * nn;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long blk = t / nn;
    const int k = (int)(blk % m.d), z = (int)((blk / m.d) % m.T), e = (int)(blk / ((long long)m.d * m.T));
    const int j = (int)((t % nn) / m.nmax), i = (int)(t % m.nmax);
    const int n = m.n[k];
    double s = 0.0;
    if (i < n && j < n) {
      const double* Ee = w.Ed + ed_off(m, e, k);
      const double* Ez = w.Ed + ed_off(m, z, k);
      for (int p = 0; p < n; ++p) s = fma(Ee[p + (long long)m.nmax * i], Ez[p + (long long)m.nmax * j], s);
    }
    w.S[s_off(m, e, z, k) + i + (long long)m.nmax * j] = s;
  }
}

// fold the weights of x into X_0 (x then carries unit weights); zero the sweep increments
__global__ void cn_fold_kernel(CnArgs a, CnWs w, int sweeps) {
  const int n0 = a.n[0];
  for (int e = threadIdx.x; e < n0 * a.r; e += blockDim.x) a.X[0][e] *= a.lam[e / n0];
  for (int i = threadIdx.x; i < sweeps; i += blockDim.x) w.eps[i] = 0.0;
  __syncthreads();
  for (int l = threadIdx.x; l < a.r; l += blockDim.x) a.lam[l] = 1.0;
}

// Y^e_k = E_k^e X_k (which = 0) or Yn^e_k = E_k^e Xn_k (which = 1) for k0 <= k < k1
__global__ void cn_apply_kernel(CnArgs a, CnWs w, CnDims m, int k0, int k1, int which) {
  const int cols = which ? a.rn : a.r;
  const long long per = (long long)m.nmax * cols;
  const long long total = (long long)a.T * (k1 - k0) * per;
  double* out = which ? w.Yn : w.Y;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(t / ((long long)(k1 - k0) * per));
    const int k = k0 + (int)((t / per) % (k1 - k0));
    const int l = (int)((t % per) / m.nmax), i = (int)(t % m.nmax);
    const int n = a.n[k];
    if (i >= n) continue;
    const double* E = w.Ed + ed_off(m, e, k);
    const double* X = which ? a.Xn[k] : a.X[k];
    double s = 0.0;
    for (int j = 0; j < n; ++j) s = fma(E[i + (long long)m.nmax * j], X[j + (long long)n * l], s);
    out[y_off(m, e, k) + i + (long long)m.nmax * l] = s;
  }
}

// G^{ez}_k = (Y^e_k)^T Y^z_k and Gn^{ez}_k = (Y^e_k)^T Yn^z_k for k0 <= k < k1
__global__ void cn_gram_kernel(CnArgs a, CnWs w, CnDims m, int k0, int k1) {
  const long long rr = (long long)m.R * m.R;
  const long long total = 2LL * (k1 - k0) * a.T * a.T * rr;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int which = (int)(t / ((k1 - k0) * (long long)a.T * a.T * rr));
    const long long u = t % ((k1 - k0) * (long long)a.T * a.T * rr);
    const int k = k0 + (int)(u / ((long long)a.T * a.T * rr));
    const int e = (int)((u / ((long long)a.T * rr)) % a.T), z = (int)((u / rr) % a.T);
    const int mm = (int)((u % rr) / m.R), l = (int)(u % m.R);
    const int cols = which ? a.rn : a.r;
    if (l >= a.r || mm >= cols) continue;
    const int n = a.n[k];
    const double* Ye = w.Y + y_off(m, e, k) + (long long)m.nmax * l;
    const double* Yz = (which ? w.Yn : w.Y) + y_off(m, z, k) + (long long)m.nmax * mm;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(Ye[i], Yz[i], s);
    (which ? w.Gn : w.G)[g_off(m, k, e, z) + l + (long long)m.R * mm] = s;
  }
}

// Gamma^{ez} = hadamard_{k != q} G^{ez}_k and Gamma_n^{ez} likewise
__global__ void cn_gamma_kernel(CnArgs a, CnWs w, CnDims m, int q) {
  const long long rr = (long long)m.R * m.R;
  const long long total = 2LL * a.T * a.T * rr;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int which = (int)(t / ((long long)a.T * a.T * rr));
    const long long u = t % ((long long)a.T * a.T * rr);
    const int e = (int)(u / ((long long)a.T * rr)), z = (int)((u / rr) % a.T);
    const long long off = u % rr;
    double v = 1.0;
    for (int k = 0; k < a.d; ++k)
      if (k != q) v *= (which ? w.Gn : w.G)[g_off(m, k, e, z) + off];
    (which ? w.Gamn : w.Gam)[((long long)e * a.T + z) * rr + off] = v;
  }
}

__device__ inline double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;   // valid in thread 0
}

// M (lower triangle, column major, ld N) and R of the normal equations of dimension q.  The
// first ceil(N^2 / NT) CTAs take one entry of M per thread (T^2 terms); CTA mblocks + row
// then computes R[row] with all its threads over the (e, z, j) terms and a block reduction:
//   R[(i, l)] = sum_{e,z} eta_e zeta_z sum_j S^{ez}_q[i, j] sum_m Xn_q[j, m] lam_n[m] Gn^{ez}[l, m].
__global__ void __launch_bounds__(NT) cn_assemble_kernel(CnArgs a, CnWs w, CnDims m, int q, int mblocks) {
  const int n = a.n[q], r = a.r, N = n * r;
  const long long rr = (long long)m.R * m.R;
  if ((int)blockIdx.x < mblocks) {
    const long long t = (long long)blockIdx.x * NT + threadIdx.x;
    if (t >= (long long)N * N) return;
    const int row = (int)(t % N), col = (int)(t / N);
    if (row < col) return;
    const int i = row % n, l = row / n, j = col % n, mm = col / n;
    double s = 0.0;
    for (int e = 0; e < a.T; ++e)
      for (int z = 0; z < a.T; ++z) {
        const double g = w.Gam[((long long)e * a.T + z) * rr + l + (long long)m.R * mm];
        const double sv = w.S[s_off(m, e, z, q) + i + (long long)m.nmax * j];
        s = fma(a.eta[e] * a.eta[z] * g, sv, s);
      }
    w.M[row + (long long)N * col] = s;
    return;
  }
  __shared__ double red[NT / 32];
  const int row = (int)blockIdx.x - mblocks;
  if (row >= N) return;
  const int i = row % n, l = row / n;
  const double* Xn = a.Xn[q];
  const int terms = a.T * a.T * n;
  double acc = 0.0;
  for (int u = threadIdx.x; u < terms; u += NT) {
    const int j = u % n, ez = u / n, e = ez / a.T, z = ez % a.T;
    const double* Gn = w.Gamn + (long long)ez * rr;
    double p = 0.0;
    for (int mm = 0; mm < a.rn; ++mm) p = fma(Xn[j + (long long)n * mm] * a.lamn[mm], Gn[l + (long long)m.R * mm], p);
    acc = fma(a.eta[e] * a.zeta[z] * w.S[s_off(m, e, z, q) + i + (long long)m.nmax * j], p, acc);
  }
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) w.Rh[row] = tot;
}

// Cholesky M = L L^T (lower, in place) with y = L^-1 R fused in, then L^T v = y; X_q <- v.
// Two columns per step: (1) columns j, j+1 below their 2 x 2 pivot block are scaled (r_j =
// d_j^-1/2, and the second column corrected by l_{j+1,j} first), with y_j, y_{j+1}; (2) the
// rank-2 update a_ic -= l_ij l_cj + l_{i,j+1} l_{c,j+1} of the trailing lower triangle (a warp
// per column on the element warps) and of y; meanwhile one pivot thread, alone on its SM
// partition, applies that update to the next pivot block itself and factors it (look-ahead),
// so the pivots' serial FP64 chain overlaps the update.  Two barriers per two columns.
// (Flattening the triangle over all element threads packed the lanes better but its index
// arithmetic cost more; one column per step took twice the barriers: both measured.)  Shared memory
// when M fits (odd leading dimension), else the global buffer in place.  A pivot that is not
// positive and finite sets HT_ERR_NONFINITE and leaves X_q unchanged.
constexpr int NTS = 512;   // solve threads: 12 element warps hide the column loops' latency (1024: slower, measured)
__global__ void __launch_bounds__(NTS) cn_solve_kernel(CnArgs a, CnWs w, int q, int sweep, int* err,
                                                       long long smem_doubles, int to_v, long long vstride) {
  const int n = a.n[q], r = a.r, N = n * r;
  const int tid = threadIdx.x, wid = tid >> 5;
  constexpr int NT = NTS;
  constexpr int PIV = NT - 32;                     // lane 0 of the last warp (SM partition 3)
  constexpr int NE = (NT / 32) * 3 / 4 * 32;       // element threads: warps with wid % 4 != 3
  const int et = (wid % 4 != 3) ? (wid - wid / 4) * 32 + (tid & 31) : -1;
  extern __shared__ double sh[];
  __shared__ double red[NT / 32];
  double* rinv = sh;                               // N reciprocal square roots of the pivots
  const long long lds = N | 1;
  const bool in_smem = (long long)N + lds * N + N <= smem_doubles;
  double* A = in_smem ? sh + N : w.M;
  const long long ld = in_smem ? lds : N;
  double* y = in_smem ? sh + N + lds * N : w.Rh;
  if (in_smem) {
    for (long long e = tid; e < (long long)N * N; e += NT) {
      const int row = (int)(e % N), col = (int)(e / N);
      if (row >= col) A[row + ld * col] = w.M[e];
    }
    for (int i = tid; i < N; i += NT) y[i] = w.Rh[i];
  }
  __syncthreads();
  // two columns per step: the pivot pair (j, j+1) is factored ahead by the pivot thread
  __shared__ double sh_l10;                        // l_{j+1,j} of the current pair
  if (tid == PIV) {
    const double d0 = A[0];
    const double r0 = htg_dpos_finite(d0) ? htg_rsqrt_fast(d0) : 0.0;
    rinv[0] = r0;
    A[0] = d0 * r0;
    if (N > 1) {
      const double l10 = A[1] * r0;
      const double d1 = fma(-l10, l10, A[1 + ld]);
      const double r1 = htg_dpos_finite(d1) ? htg_rsqrt_fast(d1) : 0.0;
      rinv[1] = r1;
      A[1 + ld] = d1 * r1;
      sh_l10 = l10;
    }
  }
  __syncthreads();
  for (int j = 0; j < N; j += 2) {
    const bool two = j + 1 < N;
    const double r0 = rinv[j], r1 = two ? rinv[j + 1] : 1.0;
    if (!htg_dnz(r0) || !htg_dnz(r1)) {            // uniform: written before the last barrier
      if (tid == 0 && err) atomicCAS(err, 0, (int)HT_ERR_NONFINITE);
      return;
    }
    const double l10 = two ? sh_l10 : 0.0;
    // (1) columns j, j+1 below the pair: l_ij = a_ij r_j, l_{i,j+1} = (a_{i,j+1} - l_ij l10) r_{j+1}
    for (int i = j + 2 + tid; i < N; i += NT) {
      const double lij = A[i + ld * j] * r0;
      A[i + ld * j] = lij;
      if (two) A[i + ld * (j + 1)] = fma(-lij, l10, A[i + ld * (j + 1)]) * r1;
    }
    if (tid == 0) {
      const double y0 = y[j] * r0;
      y[j] = y0;
      if (two) {
        A[(j + 1) + ld * j] = l10;
        y[j + 1] = fma(-l10, y0, y[j + 1]) * r1;
      }
    }
    __syncthreads();
    // (2) rank-2 update of the trailing lower triangle (a warp per column) and of y; the pivot
    // thread updates the next pair's 2 x 2 block itself and factors it (look-ahead)
    const int s0 = two ? j + 2 : j + 1;
    if (et >= 0) {
      const int ew = et >> 5, lane = et & 31;
      for (int c = s0 + ew; c < N; c += NE / 32) {
        const double lc0 = A[c + ld * j];
        const double lc1 = two ? A[c + ld * (j + 1)] : 0.0;
        const int i0 = (c <= s0 + 1) ? s0 + 2 : c;   // the pivot block (rows s0, s0+1) is the pivot thread's
        for (int i = i0 + lane; i < N; i += 32) {
          double v = fma(-A[i + ld * j], lc0, A[i + ld * c]);
          if (two) v = fma(-A[i + ld * (j + 1)], lc1, v);
          A[i + ld * c] = v;
        }
      }
      const double y0 = y[j], y1 = two ? y[j + 1] : 0.0;
      for (int i = s0 + et; i < N; i += NE) {
        double v = fma(-A[i + ld * j], y0, y[i]);
        if (two) v = fma(-A[i + ld * (j + 1)], y1, v);
        y[i] = v;
      }
    } else if (tid == PIV && s0 < N) {
      const int u = s0, w1 = s0 + 1;
      const double luj = A[u + ld * j], luj1 = two ? A[u + ld * (j + 1)] : 0.0;
      double duu = fma(-luj, luj, A[u + ld * u]);
      if (two) duu = fma(-luj1, luj1, duu);
      const double ru = htg_dpos_finite(duu) ? htg_rsqrt_fast(duu) : 0.0;
      rinv[u] = ru;
      A[u + ld * u] = duu * ru;
      if (w1 < N) {
        const double lwj = A[w1 + ld * j], lwj1 = two ? A[w1 + ld * (j + 1)] : 0.0;
        double awu = fma(-lwj, luj, A[w1 + ld * u]);
        double aww = fma(-lwj, lwj, A[w1 + ld * w1]);
        if (two) {
          awu = fma(-lwj1, luj1, awu);
          aww = fma(-lwj1, lwj1, aww);
        }
        const double lwu = awu * ru;
        const double dww = fma(-lwu, lwu, aww);
        const double rw = htg_dpos_finite(dww) ? htg_rsqrt_fast(dww) : 0.0;
        rinv[w1] = rw;
        A[w1 + ld * w1] = dww * rw;
        sh_l10 = lwu;
      }
    }
    __syncthreads();
  }
  for (int j = N - 1; j >= 0; --j) {
    if (tid == 0) y[j] *= rinv[j];
    __syncthreads();
    const double xj = y[j];
    for (int i = tid; i < j; i += NT) y[i] = fma(-A[j + ld * i], xj, y[i]);
    __syncthreads();
  }
  double* Xq = a.X[q];
  // Gauss-Seidel writes X_q; the parallel variant keeps V_q (offset q nmax R, ld n) for the
  // damped update at the end of the sweep
  double* dst = to_v ? w.V + (long long)q * vstride : Xq;
  double inc = 0.0;
  for (int e = tid; e < N; e += NT) {
    const double v = y[e];
    const double dlt = v - Xq[e];
    inc = fma(dlt, dlt, inc);
    dst[e] = v;
  }
  const double tot = block_sum(inc, red);
  if (tid == 0 && htg_dgt_nn(tot, w.eps[sweep])) w.eps[sweep] = tot;
}

// parallel variant (Appendix B, Algorithm 1): X_q <- X_q + (V_q - X_q) / 4 for every q
__global__ void cn_damp_kernel(CnArgs a, CnWs w, long long vstride) {
  for (int k = 0; k < a.d; ++k) {
    const int ne = a.n[k] * a.r;
    const double* V = w.V + (long long)k * vstride;
    double* X = a.X[k];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x)
      X[e] = fma(0.25, V[e] - X[e], X[e]);
  }
}

__global__ void cn_eps_out_kernel(CnWs w, int sweeps, double* out) {
  for (int i = threadIdx.x; i < sweeps; i += blockDim.x) out[i] = w.eps[i];
}

static_assert(sizeof(ht_op) + sizeof(CnWs) + sizeof(CnDims) <= 32000, "kernel parameter space");

bool factor_ok(const ht_factor& f) {
  switch (f.kind) {
    case HT_F_IDENTITY: return true;
    case HT_F_STENCIL: return f.half_width >= 0 && 2 * f.half_width + 1 <= HT_MAXSTENCIL;
    case HT_F_DIAG_STENCIL: return f.v && f.half_width >= 0 && 2 * f.half_width + 1 <= HT_MAXSTENCIL;
    case HT_F_DIAG: return f.v != nullptr;
    case HT_F_RANK1: return f.v && f.w;
  }
  return false;
}

}  // namespace

extern "C" int cp_cn_als_step(ht_ctx* c, const cp_tensor* xn, const ht_op* L, double dt, cp_tensor* x, int sweeps,
                              int variant, double* eps_dev, void* stream) {
  if (!c || !xn || !L || !x || sweeps < 1 || sweeps > 64) return HT_ERR_ARG;
  if (variant != CP_ALS_GS && variant != CP_ALS_JACOBI_DAMPED) return HT_ERR_ARG;
  const int d = htg_ctx_d(c);
  if (x->d != d || xn->d != d || L->d != d || !x->weight || !xn->weight) return HT_ERR_ARG;
  if (L->n_terms < 1 || L->n_terms > HT_MAXBLOCKTERMS) return HT_ERR_ARG;
  if (L->n_terms > htg_ctx_max_terms(c)) return HT_ERR_CAPACITY;
  const int cap = htg_ctx_cap(c);
  if (x->rank < 1 || xn->rank < 1 || x->rank > x->cap || xn->rank > xn->cap) return HT_ERR_ARG;
  if (x->rank > cap || xn->rank > cap) return HT_ERR_CAPACITY;
  for (int k = 0; k < d; ++k)
    if (x->factor[k] == xn->factor[k]) return HT_ERR_ARG;   // x is written while x_n is read
  const int* cn = htg_ctx_n(c);
  int nmax = 1;
  for (int k = 0; k < d; ++k) {
    if (x->n[k] != cn[k] || xn->n[k] != cn[k] || !x->factor[k] || !xn->factor[k]) return HT_ERR_ARG;
    nmax = htg_max(nmax, cn[k]);
    for (int q = 0; q < L->n_terms; ++q)
      if (!factor_ok(L->f[q][k])) return HT_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // workspace for the context's capacities (allocated once; not while a graph is captured)
  const int Tm = htg_ctx_max_terms(c) + 1;
  const long long R = cap, nm = nmax, D = d, T2 = (long long)Tm * Tm;
  const long long counts[12] = {Tm * D * nm * nm, T2 * D * nm * nm, Tm * D * nm * R, Tm * D * nm * R,
                                D * T2 * R * R, D * T2 * R * R, T2 * R * R, T2 * R * R, (nm * R) * (nm * R), nm * R, 64,
                                D * nm * R};
  size_t need = 0;
  for (long long v : counts) need += ((size_t)v * sizeof(double) + 255) & ~(size_t)255;
  size_t* have = nullptr;
  void** slot = htg_ctx_cn_ws(c, &have);
  if (*slot == nullptr || *have < need) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return HT_ERR_ARG;
    if (cudaSetDevice(htg_ctx_device(c)) != cudaSuccess) return HT_ERR_CUDA;
    if (*slot) {
      cudaStreamSynchronize(s);
      cudaFree(*slot);
      *slot = nullptr;
      *have = 0;
    }
    if (cudaMalloc(slot, need) != cudaSuccess) {
      cudaGetLastError();
      *slot = nullptr;
      return HT_ERR_NOMEM;
    }
    *have = need;
  }
  CnWs w;
  {
    char* b = (char*)*slot;
    double** ptrs[12] = {&w.Ed, &w.S, &w.Y, &w.Yn, &w.G, &w.Gn, &w.Gam, &w.Gamn, &w.M, &w.Rh, &w.eps, &w.V};
    for (int i = 0; i < 12; ++i) {
      *ptrs[i] = (double*)b;
      b += ((size_t)counts[i] * sizeof(double) + 255) & ~(size_t)255;
    }
  }
  CnDims m;
  memset(&m, 0, sizeof(m));
  m.d = d; m.T = Tm; m.R = cap; m.nmax = nmax;
  for (int k = 0; k < d; ++k) m.n[k] = cn[k];
  CnArgs a;
  memset(&a, 0, sizeof(a));
  a.d = d; a.r = x->rank; a.rn = xn->rank; a.T = L->n_terms + 1;
  a.eta[0] = a.zeta[0] = 1.0;
  for (int q = 0; q < L->n_terms; ++q) {
    a.eta[q + 1] = -0.5 * dt * L->alpha[q];
    a.zeta[q + 1] = 0.5 * dt * L->alpha[q];
  }
  for (int k = 0; k < d; ++k) {
    a.n[k] = cn[k];
    a.X[k] = x->factor[k];
    a.Xn[k] = xn->factor[k];
  }
  a.lam = x->weight;
  a.lamn = xn->weight;
  const ht_op Lc = *L;
  int launches = 0;
  const int grid = htg_max(1, htg_ctx_grid(c));
  long long solve_smem_doubles = CN_SOLVE_SMEM / (long long)sizeof(double);
  static bool attr_set[64] = {false};
  const int dev = htg_ctx_device(c);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    if (cudaFuncSetAttribute(cn_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CN_SOLVE_SMEM) != cudaSuccess)
      return HT_ERR_CUDA;
    attr_set[dev] = true;
  }
#define CNL(cls, expr)                             \
  do {                                             \
    htg_prof_begin(c, s);                          \
    expr;                                          \
    htg_prof_end(c, (cls), s);                     \
    ++launches;                                    \
    if (cudaGetLastError() != cudaSuccess) {       \
      htg_ctx_count(c, launches, s);               \
      return HT_ERR_CUDA;                          \
    }                                              \
  } while (0)
  CnDims mt = m;
  mt.T = a.T;   // the blocks this operator uses
  CNL(KC_CPSMALL, (cn_dense_kernel<<<grid, NT, 0, s>>>(Lc, w, mt)));
  CNL(KC_CPSMALL, (cn_sgram_kernel<<<grid, NT, 0, s>>>(w, mt)));
  CNL(KC_CPSMALL, (cn_fold_kernel<<<1, NT, 0, s>>>(a, w, sweeps)));
  CNL(KC_CPSMALL, (cn_apply_kernel<<<grid, NT, 0, s>>>(a, w, mt, 0, d, 0)));
  CNL(KC_CPSMALL, (cn_apply_kernel<<<grid, NT, 0, s>>>(a, w, mt, 0, d, 1)));
  CNL(KC_CPSMALL, (cn_gram_kernel<<<grid, NT, 0, s>>>(a, w, mt, 0, d)));
  const bool gs = (variant == CP_ALS_GS);
  const long long vstride = nm * R;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int q = 0; q < d; ++q) {
      CNL(KC_CPSMALL, (cn_gamma_kernel<<<grid, NT, 0, s>>>(a, w, mt, q)));
      const int Nq = cn[q] * a.r;
      const int mblocks = (int)(((long long)Nq * Nq + NT - 1) / NT);
      CNL(KC_CPSMALL, (cn_assemble_kernel<<<mblocks + Nq, NT, 0, s>>>(a, w, mt, q, mblocks)));
      CNL(KC_CPSOLVE, (cn_solve_kernel<<<1, NTS, (size_t)solve_smem_doubles * sizeof(double), s>>>(
                          a, w, q, sw, htg_ctx_err(c), solve_smem_doubles, gs ? 0 : 1, vstride)));
      if (gs) {
        CNL(KC_CPSMALL, (cn_apply_kernel<<<grid, NT, 0, s>>>(a, w, mt, q, q + 1, 0)));
        CNL(KC_CPSMALL, (cn_gram_kernel<<<grid, NT, 0, s>>>(a, w, mt, q, q + 1)));
      }
    }
    if (!gs) {
      // every mode was solved from the same iterate: damped update, then its applications and Grams
      CNL(KC_CPSMALL, (cn_damp_kernel<<<grid, NT, 0, s>>>(a, w, vstride)));
      CNL(KC_CPSMALL, (cn_apply_kernel<<<grid, NT, 0, s>>>(a, w, mt, 0, d, 0)));
      CNL(KC_CPSMALL, (cn_gram_kernel<<<grid, NT, 0, s>>>(a, w, mt, 0, d)));
    }
  }
  if (eps_dev) CNL(KC_CPSMALL, (cn_eps_out_kernel<<<1, 64, 0, s>>>(w, sweeps, eps_dev)));
#undef CNL
  htg_ctx_count(c, launches, s);
  return HT_OK;
}
