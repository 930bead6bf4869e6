// HT apply, HSVD truncation and explicit steps: context, workspace, device planner,
// apply / rank-selection kernels and the C entry points of include/htgpu.h.
//
// Truncation T(u) (root-to-leaves hierarchical SVD; Section 2.2 cites it as the HT rank
// reduction, Section 3.2 uses it after each explicit step) is computed without ever
// forming orthonormal bases:
//   bottom-up  R_leaf = qr_R(U_leaf);  interior: C_t = B_t x1 R_t1 x2 R_t2,  R_t = qr_R(C_t)
//   root       E_t1 = B R_t2^T,  E_t2 = B^T R_t1^T        (square-root factors of the
//                                                          complement Gramians)
//   top-down   P_t = R_t E_t (its SVD gives the singular values of the t-matricisation);
//              children: E_t1 = lq([B_t x2 R_t2 x3 E_t^T]_(1)), E_t2 likewise
//   ranks      smallest k with discarded energy <= (tol |u|)^2 / (2d-3), capped
//   project    X_t = W_k^T R_t,  Y_t = E_t Z_k S_k^{-1}  (P_t = W S Z^T)
//              leaf U <- U Y;  B_t <- B_t x1 X_t1 x2 X_t2 x3 Y_t^T;  root B <- X_t1 B X_t2^T
// With U_t = Q_t R_t this is exactly Q_t W_k (the leading left singular vectors) at every
// node, i.e. the HSVD projections, expressed through R_t, E_t and the small SVDs only.
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <cmath>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

// ------------------------------------------------------------------- tree -----
void htg_build_tree(int d, int kind, TreeInfo* t) {
  memset(t, 0, sizeof(*t));
  t->d = d;
  int n = 1;
  t->lo[0] = 0; t->hi[0] = d; t->parent[0] = -1; t->depth[0] = 0;
  for (int i = 0; i < n; ++i) {
    const int a = t->lo[i], b = t->hi[i];
    if (b - a > 1) {
      const int m = (kind == HT_TREE_LINEAR) ? a + 1 : a + (b - a) / 2;
      t->c1[i] = n; t->c2[i] = n + 1;
      t->lo[n] = a; t->hi[n] = m; t->lo[n + 1] = m; t->hi[n + 1] = b;
      t->parent[n] = t->parent[n + 1] = i;
      t->depth[n] = t->depth[n + 1] = t->depth[i] + 1;
      t->c1[n] = t->c2[n] = t->c1[n + 1] = t->c2[n + 1] = -1;
      n += 2;
    } else {
      t->c1[i] = t->c2[i] = -1;
    }
  }
  t->nn = n;
  int md = 0;
  for (int i = 0; i < n; ++i) md = htg_max(md, t->depth[i]);
  t->max_depth = md;
}

namespace {

constexpr int NN = HT_MAXNODES;
// cooperative QR (k_qr.cu) for contexts whose truncation inputs reach this rank: descriptors
// per launch (a level's complement QRs: 2 per interior node) and CTAs per matrix
constexpr int QR_COOP_MIN_KC = 160;
// contexts whose truncation inputs reach this rank refine X_t Y_t = I in the cluster form
constexpr int BIORTH_CLUSTER_MIN_KC = 160;
constexpr int QR_COOP_NDMAX = 2 * HT_MAXNODES;
constexpr int QR_COOP_GMAX = 64;
constexpr int MAXLEV = HT_MAXD;   // tree depth + 1 (the linear tree of d = 16 is 15 deep)

// Device-side plan: dimensions derived from the device-resident ranks, plus every work
// descriptor of one truncation.  Slots per level follow the host's level lists.
struct Plan {
  int K[NN], Rp[NN], mE[NN], knew[NN];
  QrDesc qr_leaf[HT_MAXD];
  QrDesc qr_orth[MAXLEV][NN];
  QrDesc qr_comp[MAXLEV][2 * NN];
  GemmDesc g_abs1[MAXLEV][NN];
  GemmDesc g_abs2[MAXLEV][NN];
  GemmDesc g_rootE[2];
  GemmDesc g_Pall[NN];        // P_t = R_t E_t for every non-root node (slot t-1)
  SvdDesc svd_all[NN];
  GemmDesc g_T1[MAXLEV][NN];
  GemmDesc g_Epre[MAXLEV][2 * NN];
  GemmDesc g_XY[2 * NN];
  GemmDesc g_bi[2][NN];     // operands of the X_t Y_t = I refinement (biorth_kernel)
  GemmDesc g_proj1[NN];
  GemmDesc g_proj2[NN];
  GemmDesc g_proj3[NN];
  double norm;
};

// Static level lists (host computed, passed by value to the planner).
struct Levels {
  int n_all[MAXLEV];          // non-root nodes per depth
  int all[MAXLEV][NN];
  int n_int[MAXLEV];          // interior non-root nodes per depth
  int inter[MAXLEV][NN];
  int n_leaf;
  int leaf[HT_MAXD];          // leaf nodes in dimension order
  int n_proj1, proj1[NN];     // leaves + interior + root
  int n_proj2, proj2[NN];     // interior + root
  int n_proj3, proj3[NN];     // interior
};

// Workspace pointers per node (capacity sized).
struct WsNode {
  double* Rf;     // R factor          Kc x Kc (leaves: min(n,Kc) x Kc)
  double* Tabs;   // absorb temp / projection T2 / root TR       Kc^3
  double* Cabs;   // absorbed transfer / projection T3           Kc^3
  double* S;      // QR scratch                                   Kc^3
  double* Epre;   // uncompressed complement factor               Kc^3
  double* T1;     // B x3 E^T                                     Kc^3
  double* E;      // compressed complement factor                 Kc x Kc
  double* P;      // R E                                          Kc x Kc
  double* sig;    // singular values                              Kc
  double* W;      // left singular vectors of P                   Kc x Kc
  double* Z;      // right singular vectors of P                  Kc x Kc
  double* SW;     // SVD work                                     6 Kc^2 + Kc + 2
  double* X;      // W_k^T R                                      Kc x Kc
  double* Y;      // E Z_k / s                                    Kc x Kc
  double* invsig; // 1/s_k                                        Kc
  unsigned* tick; // QR tickets: [0] basis (leaf / orthogonalisation), [1] complement factor
};

struct HtView {           // a tensor as the kernels see it
  double* node[NN];
  int* rank;
  int n[HT_MAXD];
};

struct ApplyOp;

// One instance of a batched step as the batched kernels see it (device array, one entry per
// instance): its plan, workspace nodes, views and operators.
enum { VIEW_U = 0, VIEW_APP = 1, VIEW_STAGE = 2, NVIEW = 3 };
struct Inst {
  Plan* P;
  const WsNode* wn;
  HtView view[NVIEW];      // the caller's tensor, the applied-tensor area, the HEUN2 stage area
  const ApplyOp* op[2];    // RK2POLY or EULER operator; HEUN2 second-stage operator
  int* err;
  int cap_in;              // capacity of the truncation input (the applied-tensor area)
  int rmax;
  double rel_tol;
};

}  // namespace

struct ht_ctx {
  ht_config cfg;
  TreeInfo tree;
  Levels lev;
  int Kc;                 // largest truncation input rank
  int cap;                // largest stored rank
  void* ws = nullptr;
  size_t ws_bytes = 0;
  Plan* plan = nullptr;   // device
  int* err = nullptr;     // device error word
  WsNode wn[NN];
  // applied-tensor area (truncation input of ht_step): packed at rank <= Kc
  double* app[NN];
  int* app_rank;
  // second tensor area for HEUN2 (u* and the stage sum), rank <= Kc
  double* stage[NN];
  int* stage_rank;
  WsNode* wn_dev = nullptr;   // device copy of wn[]
  const double** ptr_tbl = nullptr;   // device table of caller pointers (CP factors)
  CpWs cp;
  long long launches = 0;
  // opt-in event profiler
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_pool;
  std::vector<int> prof_cls;        // class of record i (events 2i, 2i+1)
  size_t prof_n = 0;
  double* prof_flops = nullptr;     // device, KC_COUNT counters
  int svd_smem = 0;
  int gemm_grid = 0;
  int sms = 1;                 // streaming multiprocessors of the device
  int slices = 0;              // HT_PREC_MIXED: BF16 digit planes per operand (0: FP64 contractions)
  long long tc_min = 0;        // HT_PREC_MIXED: contractions of at least this many multiply-adds on the tensor cores
  bool tc_reach = false;       // whether a contraction of this context can reach tc_min
  // per contraction list of a single truncation: whether one of its contractions can reach tc_min
  // (bounds from the capacities; a list without a tensor-core launch runs wholly on the CUDA cores)
  enum { TL_ABS1, TL_ABS2, TL_T1, TL_EPRE, TL_LEVEL };   // per depth
  bool tc_lvl[MAXLEV][TL_LEVEL] = {};
  bool tc_rootE = false, tc_Pall = false, tc_XY = false, tc_proj[3] = {false, false, false};
  int svd_min_cols = 128;      // node factors at least this wide take the cluster SVD
  int bi_cl = 0;               // CTAs per node of the cluster form of biorth (0: one CTA per node)
  cudaStream_t last_stream = nullptr;
  ht_batch* batch = nullptr;   // the batch this context is bound to, if any
  QrCoopWs qr_coop;            // cooperative QR workspace (contexts with Kc >= QR_COOP_MIN_KC)
  bool has_coop = false;
  SvdClusterCfg svd_clu;       // cluster form of the node SVD (contexts with Kc >= 128)
  CpClusterCfg cp_clu;         // cluster form of the persistent CP-ALS kernel
  void* cn_ws = nullptr;       // Crank-Nicolson ALS workspace (allocated by its first call)
  size_t cn_bytes = 0;
};

namespace {

// ---------------------------------------------------------------- planner -----
__device__ void fill_gemm(GemmDesc& g, const double* A, int lda, int tA, const double* B, int ldb,
                          int tB, double* C, int ldc, int m, int n, int k) {
  g.A = A; g.B = B; g.C = C; g.colscale = nullptr;
  g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.m = m; g.n = n; g.k = k;
  g.tA = tA; g.tB = tB;
  g.sA = g.sB = g.sC = 0;
  g.batch = 1;
  g.alpha = 1.0; g.beta = 0.0;
}

// skip_tol: the relative tolerance that sets the SVD discard level (SvdDesc::skip2), 0 when every
// singular value is to be resolved (they are reported to the caller)
__device__ void plan_pre_body(Plan* P, const TreeInfo& T, const Levels& L, const HtView& in, const WsNode* wn,
                              int cap_in, double skip_tol, int* err) {
  if (threadIdx.x != 0) return;
  // device-resident ranks are validated against the input capacity: out-of-range ranks are
  // clamped (every later access stays inside the buffers) and reported as HT_ERR_CAPACITY
  bool bad = false;
  for (int t = 0; t < T.nn; ++t) {
    int k = (t == 0) ? 1 : in.rank[t];
    if (k < 1 || k > cap_in) {
      bad = true;
      k = k < 1 ? 1 : cap_in;
    }
    P->K[t] = k;
  }
  if (bad && err) atomicCAS(err, 0, (int)HT_ERR_CAPACITY);
  // R-factor row counts bottom-up
  for (int dep = T.max_depth; dep >= 1; --dep) {
    for (int t = 1; t < T.nn; ++t) {
      if (T.depth[t] != dep) continue;
      if (T.c1[t] < 0) P->Rp[t] = htg_min(in.n[T.lo[t]], P->K[t]);
      else P->Rp[t] = htg_min(P->Rp[T.c1[t]] * P->Rp[T.c2[t]], P->K[t]);
    }
  }
  const int ra = T.c1[0], rb = T.c2[0];
  P->mE[ra] = P->Rp[rb];
  P->mE[rb] = P->Rp[ra];
  for (int dep = 1; dep < T.max_depth; ++dep) {
    for (int t = 1; t < T.nn; ++t) {
      if (T.depth[t] != dep || T.c1[t] < 0) continue;
      const int a = T.c1[t], b = T.c2[t];
      P->mE[a] = htg_min(P->K[a], P->Rp[b] * P->mE[t]);
      P->mE[b] = htg_min(P->K[b], P->Rp[a] * P->mE[t]);
    }
  }
  // leaf QR
  for (int s = 0; s < L.n_leaf; ++s) {
    const int t = L.leaf[s];
    QrDesc& q = P->qr_leaf[s];
    q.A = in.node[t]; q.scratch = wn[t].S; q.R = wn[t].Rf; q.rows_out = nullptr; q.ticket = wn[t].tick;
    q.m = in.n[T.lo[t]]; q.k = P->K[t]; q.lda = q.m; q.ldr = P->Rp[t]; q.tA = 0; q.tR = 0;
  }
  // bottom-up absorb + orthogonalisation QR
  for (int dep = 1; dep < MAXLEV; ++dep) {
    for (int s = 0; s < L.n_int[dep]; ++s) {
      const int t = L.inter[dep][s], a = T.c1[t], b = T.c2[t];
      const int K1 = P->K[a], K2 = P->K[b], K = P->K[t];
      fill_gemm(P->g_abs1[dep][s], wn[a].Rf, P->Rp[a], 0, in.node[t], K1, 0, wn[t].Tabs, P->Rp[a],
                P->Rp[a], K2 * K, K1);
      GemmDesc& g2 = P->g_abs2[dep][s];
      fill_gemm(g2, wn[t].Tabs, P->Rp[a], 0, wn[b].Rf, P->Rp[b], 1, wn[t].Cabs, P->Rp[a],
                P->Rp[a], P->Rp[b], K2);
      g2.batch = K; g2.sA = (long long)P->Rp[a] * K2; g2.sB = 0; g2.sC = (long long)P->Rp[a] * P->Rp[b];
      QrDesc& q = P->qr_orth[dep][s];
      q.A = wn[t].Cabs; q.scratch = wn[t].S; q.R = wn[t].Rf; q.rows_out = nullptr; q.ticket = wn[t].tick;
      q.m = P->Rp[a] * P->Rp[b]; q.k = K; q.lda = q.m; q.ldr = P->Rp[t]; q.tA = 0; q.tR = 0;
    }
  }
  // root complement factors
  {
    const int K1 = P->K[ra], K2 = P->K[rb];
    fill_gemm(P->g_rootE[0], in.node[0], K1, 0, wn[rb].Rf, P->Rp[rb], 1, wn[ra].E, K1, K1, P->Rp[rb], K2);
    fill_gemm(P->g_rootE[1], in.node[0], K1, 1, wn[ra].Rf, P->Rp[ra], 1, wn[rb].E, K2, K2, P->Rp[ra], K1);
  }
  // top-down
  for (int dep = 1; dep < MAXLEV; ++dep) {
    for (int s = 0; s < L.n_all[dep]; ++s) {
      const int t = L.all[dep][s];
      fill_gemm(P->g_Pall[t - 1], wn[t].Rf, P->Rp[t], 0, wn[t].E, P->K[t], 0, wn[t].P, P->Rp[t],
                P->Rp[t], P->mE[t], P->K[t]);
      SvdDesc& v = P->svd_all[t - 1];
      v.P = wn[t].P; v.p = P->Rp[t]; v.q = P->mE[t]; v.ldp = P->Rp[t];
      v.sigma = wn[t].sig; v.V = wn[t].W; v.U = wn[t].Z; v.work = wn[t].SW;
      // |P_t|_F = |u|: with p columns, those with sigma^2 below (tol |u|)^2 / (2p (2d-3)) are
      // discarded by the rank rule whatever their mutual rotation (see SvdDesc::skip2)
      v.skip2 = 0.5 * skip_tol * skip_tol / (double)htg_max(2 * T.d - 3, 1);
      // The root's children have P_t2 = R_t2 B^T R_t1^T = P_t1^T: one SVD serves both (t2's left
      // singular vectors are t1's right ones and vice versa, the singular values shared), so
      // neither P_t2 nor its SVD is formed
      if (t == rb) {
        P->g_Pall[t - 1].m = 0;
        v.p = 0;
      }
    }
    for (int s = 0; s < L.n_int[dep]; ++s) {
      const int t = L.inter[dep][s], a = T.c1[t], b = T.c2[t];
      const int K1 = P->K[a], K2 = P->K[b], K = P->K[t], mE = P->mE[t];
      fill_gemm(P->g_T1[dep][s], in.node[t], K1 * K2, 0, wn[t].E, K, 0, wn[t].T1, K1 * K2, K1 * K2, mE, K);
      GemmDesc& ga = P->g_Epre[dep][2 * s];
      fill_gemm(ga, wn[t].T1, K1, 0, wn[b].Rf, P->Rp[b], 1, wn[a].Epre, K1, K1, P->Rp[b], K2);
      ga.batch = mE; ga.sA = (long long)K1 * K2; ga.sC = (long long)K1 * P->Rp[b];
      GemmDesc& gb = P->g_Epre[dep][2 * s + 1];
      fill_gemm(gb, wn[t].T1, K1, 1, wn[a].Rf, P->Rp[a], 1, wn[b].Epre, K2, K2, P->Rp[a], K1);
      gb.batch = mE; gb.sA = (long long)K1 * K2; gb.sC = (long long)K2 * P->Rp[a];
      QrDesc& qa = P->qr_comp[dep][2 * s];
      qa.A = wn[a].Epre; qa.scratch = wn[a].S; qa.R = wn[a].E; qa.rows_out = nullptr; qa.ticket = wn[a].tick + 1;
      qa.m = P->Rp[b] * mE; qa.k = K1; qa.lda = K1; qa.ldr = K1; qa.tA = 1; qa.tR = 1;
      QrDesc& qb = P->qr_comp[dep][2 * s + 1];
      qb.A = wn[b].Epre; qb.scratch = wn[b].S; qb.R = wn[b].E; qb.rows_out = nullptr; qb.ticket = wn[b].tick + 1;
      qb.m = P->Rp[a] * mE; qb.k = K2; qb.lda = K2; qb.ldr = K2; qb.tA = 1; qb.tR = 1;
    }
  }
}

__global__ void plan_pre_kernel(Plan* P, TreeInfo T, Levels L, HtView in, const WsNode* wn, int cap_in,
                                double skip_tol, int* err) {
  plan_pre_body(P, T, L, in, wn, cap_in, skip_tol, err);
}

__global__ void plan_pre_batch_kernel(const Inst* I, TreeInfo T, Levels L, int in_sel) {
  const Inst& x = I[blockIdx.x];
  plan_pre_body(x.P, T, L, x.view[in_sel], x.wn, x.cap_in, x.rel_tol, x.err);
}

// Rank selection (one CTA) + projection descriptors.
__device__ void rank_select_body(Plan* P, const TreeInfo& T, const Levels& L, const HtView& in, const HtView& out,
                                 const WsNode* wn, double rel_tol, int rmax, double* sigma_out, int sig_stride,
                                 double* norm_out, int* err) {
  __shared__ double s_thr2;
  const int ra = T.c1[0], rb = T.c2[0];
  if (threadIdx.x == 0) {
    const double* sa = wn[ra].sig;
    double nrm2 = 0.0;
    for (int j = 0; j < P->Rp[ra]; ++j) nrm2 += sa[j] * sa[j];
    if (!isfinite(nrm2) && err) atomicCAS(err, 0, (int)HT_ERR_NONFINITE);
    P->norm = sqrt(nrm2);
    if (norm_out) *norm_out = P->norm;
    const int edges = htg_max(2 * T.d - 3, 1);
    s_thr2 = rel_tol * rel_tol * nrm2 / (double)edges;
  }
  __syncthreads();
  const double thr2 = s_thr2;
  const double sfloor = 64.0 * 2.220446049250313e-16 * P->norm;
  for (int t = 1 + threadIdx.x; t < T.nn; t += blockDim.x) {
    const int src = (t == rb) ? ra : t;
    const double* s = wn[src].sig;
    const int p = P->Rp[src];
    double tail = 0.0;
    int k = p;
    // tail(kk) = sum_{j >= kk} s_j^2; smallest kk >= 1 with tail <= thr2
    for (int kk = p; kk >= 1; --kk) {
      if (!htg_dgt_nn(tail, thr2)) k = kk;   // tail <= thr2 (both >= 0), as a bit compare
      else break;
      tail = fma(s[kk - 1], s[kk - 1], tail);
    }
    // (loop above walks kk downward while tail(kk) <= thr2)
    // singular values at the rounding level of |u| are never kept, whatever the tolerance:
    // their vectors are rounding noise, which Y = E Z S^-1 would amplify (dropping them changes
    // T(u) at that level only)
    int knz = 0;
    for (int j = 0; j < p; ++j)
      if (htg_dgt_nn(s[j], sfloor)) knz = j + 1;
    k = htg_min(k, htg_max(1, knz));
    k = htg_max(1, htg_min(k, rmax));
    k = htg_min(k, P->Rp[t]);
    P->knew[t] = k;
    out.rank[t] = k;
    for (int j = 0; j < P->Rp[t]; ++j) {
      const double sj = (j < p) ? s[j] : 0.0;   // the root's second child: its sibling's values
      wn[t].invsig[j] = (j < k && htg_dpos_finite(sj)) ? 1.0 / sj : 0.0;
    }
    if (sigma_out) {
      for (int j = 0; j < sig_stride; ++j)
        sigma_out[(long long)t * sig_stride + j] = (j < P->Rp[t] && j < p) ? s[j] : 0.0;
    }
  }
  if (threadIdx.x == 0) out.rank[0] = 1;
  __syncthreads();
  if (threadIdx.x != 0) return;
  // root children share one rank
  {
    const int k = htg_min(P->knew[ra], P->knew[rb]);
    P->knew[ra] = P->knew[rb] = k;
    out.rank[ra] = out.rank[rb] = k;
    if (sigma_out) {
      for (int j = 0; j < sig_stride; ++j) sigma_out[j] = 0.0;
    }
  }
  // X_t, Y_t
  int i = 0;
  for (int t = 1; t < T.nn; ++t) {
    const int k = P->knew[t];
    // the root's second child: left singular vectors = its sibling's right ones (Rp[rb] rows,
    // leading dimension mE[ra] = Rp[rb]), right ones = the sibling's left ones (Rp[ra] = mE[rb])
    const double* Wt = (t == rb) ? wn[ra].Z : wn[t].W;
    const double* Zt = (t == rb) ? wn[ra].W : wn[t].Z;
    fill_gemm(P->g_XY[i++], Wt, P->Rp[t], 1, wn[t].Rf, P->Rp[t], 0, wn[t].X, k, k, P->K[t], P->Rp[t]);
    GemmDesc& y = P->g_XY[i++];
    fill_gemm(y, wn[t].E, P->K[t], 0, Zt, P->mE[t], 0, wn[t].Y, P->K[t], P->K[t], k, P->mE[t]);
    y.colscale = wn[t].invsig;
    // X_t Y_t = W_k^T W_k S_k Z_k^T Z_k S_k^-1 = I_k in exact arithmetic; rounding in the SVD
    // breaks it by about eps |u| / s_k (Y divides by the kept singular values), and the edge's
    // projector Y X then moves T(u) by that much.  Two Newton steps for the inverse of X_t on
    // the range of Y_t, Y <- Y (2I - X Y) (biorth_kernel), square that error twice; with every
    // direction kept, Y X = I and T(u) = u to rounding.  The descriptors carry the operands
    // (X, Y: k x K and K x k) and the scratch used when they do not fit in shared memory
    // (N = 2I - X Y in SW, Y2 in P: both free once the SVD has run).
    const int K = P->K[t];
    fill_gemm(P->g_bi[0][t - 1], wn[t].X, k, 0, wn[t].Y, K, 0, wn[t].SW, k, k, k, K);
    fill_gemm(P->g_bi[1][t - 1], wn[t].Y, K, 0, wn[t].SW, k, 0, wn[t].P, K, K, k, k);
  }
  // projection
  for (int s = 0; s < L.n_proj1; ++s) {
    const int t = L.proj1[s];
    GemmDesc& g = P->g_proj1[s];
    if (t == 0) {
      fill_gemm(g, wn[ra].X, P->knew[ra], 0, in.node[0], P->K[ra], 0, wn[0].Tabs, P->knew[ra],
                P->knew[ra], P->K[rb], P->K[ra]);
    } else if (T.c1[t] < 0) {
      const int n = in.n[T.lo[t]];
      fill_gemm(g, in.node[t], n, 0, wn[t].Y, P->K[t], 0, out.node[t], n, n, P->knew[t], P->K[t]);
    } else {
      const int a = T.c1[t], b = T.c2[t];
      const int K12 = P->K[a] * P->K[b];
      fill_gemm(g, in.node[t], K12, 0, wn[t].Y, P->K[t], 0, wn[t].Tabs, K12, K12, P->knew[t], P->K[t]);
    }
  }
  for (int s = 0; s < L.n_proj2; ++s) {
    const int t = L.proj2[s];
    GemmDesc& g = P->g_proj2[s];
    if (t == 0) {
      fill_gemm(g, wn[0].Tabs, P->knew[ra], 0, wn[rb].X, P->knew[rb], 1, out.node[0], P->knew[ra],
                P->knew[ra], P->knew[rb], P->K[rb]);
    } else {
      const int a = T.c1[t], b = T.c2[t];
      fill_gemm(g, wn[a].X, P->knew[a], 0, wn[t].Tabs, P->K[a], 0, wn[t].Cabs, P->knew[a],
                P->knew[a], P->K[b] * P->knew[t], P->K[a]);
    }
  }
  for (int s = 0; s < L.n_proj3; ++s) {
    const int t = L.proj3[s];
    const int a = T.c1[t], b = T.c2[t];
    GemmDesc& g = P->g_proj3[s];
    fill_gemm(g, wn[t].Cabs, P->knew[a], 0, wn[b].X, P->knew[b], 1, out.node[t], P->knew[a],
              P->knew[a], P->knew[b], P->K[b]);
    g.batch = P->knew[t];
    g.sA = (long long)P->knew[a] * P->K[b];
    g.sC = (long long)P->knew[a] * P->knew[b];
  }
}

// The two Newton steps Y <- Y (2I - X Y) of every node in one launch (one CTA per node,
// blockIdx.y the instance): X (k x K, ld k) and Y (K x k, ld K) are those of the node's
// descriptors in g_bi[0] (A, B); N = 2I - X Y and Y2 = Y N live in shared memory when
// 3 k K + k^2 doubles fit, else in the node's SW and P buffers (the descriptors' outputs).
constexpr int BIORTH_SMEM = 96 * 1024;
__global__ void __launch_bounds__(256) biorth_kernel(const GemmDesc* d0, const GemmDesc* d1, long long inst_stride,
                                                     double* flops) {
  const GemmDesc g0 = ((const GemmDesc*)((const char*)d0 + inst_stride * blockIdx.y))[blockIdx.x];
  const GemmDesc g1 = ((const GemmDesc*)((const char*)d1 + inst_stride * blockIdx.y))[blockIdx.x];
  const int k = g0.m, K = g0.k;
  if (k <= 0 || K <= 0) return;
  // four products of 2 k^2 K flops each
  if (threadIdx.x == 0 && flops) atomicAdd(flops, 8.0 * k * k * K);
  double* Yg = const_cast<double*>(g0.B);
  extern __shared__ double sh[];
  const long long need = 3LL * k * K + (long long)k * k;
  const bool fits = need <= (long long)(BIORTH_SMEM / sizeof(double));
  const double* X = g0.A;
  const double* Y = Yg;
  double* N = g0.C;
  double* Y2 = g1.C;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (fits) {
    double* Xs = sh;
    double* Ys = Xs + (long long)k * K;
    N = Ys + (long long)K * k;
    Y2 = N + (long long)k * k;
    for (int e = tid; e < k * K; e += nt) {
      Xs[e] = g0.A[e];
      Ys[e] = Yg[e];
    }
    X = Xs;
    Y = Ys;
    __syncthreads();
  }
  for (int it = 0; it < 2; ++it) {
    const double* Yc = (it == 0) ? Y : Y2;
    for (int e = tid; e < k * k; e += nt) {
      const int a = e % k, b = e / k;
      double acc = 0.0;
      for (int c = 0; c < K; ++c) acc = fma(X[a + (long long)k * c], Yc[c + (long long)K * b], acc);
      N[e] = (a == b ? 2.0 : 0.0) - acc;
    }
    __syncthreads();
    double* out = (it == 0) ? Y2 : Yg;
    for (int e = tid; e < K * k; e += nt) {
      const int c = e % K, b = e / K;
      double acc = 0.0;
      for (int a = 0; a < k; ++a) acc = fma(Yc[c + (long long)K * a], N[a + (long long)k * b], acc);
      out[e] = acc;
    }
    __syncthreads();
  }
}

// The same two Newton steps for contexts with wide node factors (ht_config.biorth_form = 1),
// where one CTA per node spends milliseconds on a node's 8 k^2 K flops (k = 64, K = 448: 7.3 M
// multiply-adds, 2.4 ms): each node takes one thread-block cluster of CL CTAs, every product's
// output elements are dealt out over the cluster's threads, and the four products are joined by
// cluster barriers.  Each
// element is summed in the same order as in biorth_kernel, so the results agree bit for bit.
// The operands stay in global memory (L2 resident); N and Y2, written inside the launch, are
// stored and read at L2 (st/ld .cg), so that no CTA reads a line of another CTA's output from
// its own (non-coherent) L1.  One node per cluster: the early return and the barriers are
// uniform over the cluster.
__global__ void __launch_bounds__(256) biorth_cluster_kernel(const GemmDesc* d0, const GemmDesc* d1,
                                                             double* flops) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cl = (int)cluster.num_blocks(), r = (int)cluster.block_rank();
  const int node = (int)blockIdx.x / cl;
  const GemmDesc g0 = d0[node];
  const GemmDesc g1 = d1[node];
  const int k = g0.m, K = g0.k;
  if (k <= 0 || K <= 0) return;
  if (r == 0 && threadIdx.x == 0 && flops) atomicAdd(flops, 8.0 * k * k * K);
  const double* X = g0.A;
  double* Yg = const_cast<double*>(g0.B);
  double* N = g0.C;
  double* Y2 = g1.C;
  const int stride = cl * (int)blockDim.x, e0 = r * (int)blockDim.x + (int)threadIdx.x;
  for (int it = 0; it < 2; ++it) {
    const double* Yc = (it == 0) ? Yg : Y2;
    for (int e = e0; e < k * k; e += stride) {
      const int a = e % k, b = e / k;
      double acc = 0.0;
      // unrolled so that eight iterations' loads are in flight ahead of the (ordered) FMA chain
#pragma unroll 8
      for (int c = 0; c < K; ++c) acc = fma(X[a + (long long)k * c], __ldcg(Yc + c + (long long)K * b), acc);
      __stcg(N + e, (a == b ? 2.0 : 0.0) - acc);
    }
    __threadfence();
    cluster.sync();
    double* out = (it == 0) ? Y2 : Yg;
    for (int e = e0; e < K * k; e += stride) {
      const int c = e % K, b = e / K;
      double acc = 0.0;
#pragma unroll 8
      for (int a = 0; a < k; ++a) acc = fma(__ldcg(Yc + c + (long long)K * a), __ldcg(N + a + (long long)k * b), acc);
      __stcg(out + e, acc);
    }
    __threadfence();
    cluster.sync();
  }
}

// The largest cluster (16 CTAs, else the portable 8) of biorth_cluster_kernel one of which fits
// the device; 0 when none does (biorth_kernel then serves).
static int biorth_cluster_setup() {
  if (cudaFuncSetAttribute(biorth_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int sizes[2] = {16, 8};
  for (int i = 0; i < 2; ++i) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(sizes[i], 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = sizes[i];
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, biorth_cluster_kernel, &cfg) == cudaSuccess && n >= 1) return sizes[i];
    cudaGetLastError();
  }
  return 0;
}

static cudaError_t launch_biorth(const ht_ctx* c, const Plan* P, int nodes, int count, long long st, double* flops,
                                 cudaStream_t s) {
  if (nodes <= 0 || count <= 0) return cudaSuccess;
  if (c->bi_cl > 0 && count == 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nodes * c->bi_cl), 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c->bi_cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, biorth_cluster_kernel, (const GemmDesc*)P->g_bi[0], (const GemmDesc*)P->g_bi[1],
                              flops);
  }
  biorth_kernel<<<dim3(nodes, count), 256, BIORTH_SMEM, s>>>(P->g_bi[0], P->g_bi[1], st, flops);
  return cudaGetLastError();
}

__global__ void rank_select_kernel(Plan* P, TreeInfo T, Levels L, HtView in, HtView out, const WsNode* wn,
                                   double rel_tol, int rmax, double* sigma_out, int sig_stride, double* norm_out,
                                   int* err) {
  rank_select_body(P, T, L, in, out, wn, rel_tol, rmax, sigma_out, sig_stride, norm_out, err);
}

__global__ void rank_select_batch_kernel(const Inst* I, TreeInfo T, Levels L, int in_sel, int out_sel) {
  const Inst& x = I[blockIdx.x];
  rank_select_body(x.P, T, L, x.view[in_sel], x.view[out_sel], x.wn, x.rel_tol, x.rmax, nullptr, 0, nullptr, x.err);
}

// ------------------------------------------------------------ apply kernels ---
struct ApplyFactor {   // one 1-D factor as the apply kernel sees it
  int kind, hw;
  double c[HT_MAXSTENCIL];
  const double* v;
  const double* w;
};
constexpr int MAXBLK = HT_MAXBLOCKTERMS + 2;   // identity + terms (+ the stage block of HEUN2)
// Block-diagonal assembly: block b of the result is F_b applied to source tensor src[b]
// (0 or 1) with root weight coef[b].  RK2POLY instead uses the binomial block pattern of
// a single source with factor f[0][dim] = dt * L_dim.
// mode APPLY_POLY: sum over npoly sources s of q_s(S) u_s, q_s(z) = sum_{j <= deg[s]} pc[s][j] z^j,
// S = sum_i f[0][i] (a Kronecker sum, the 1-D factors dt L_i): the exact form with the binomial
// block pattern (HT_APPLY_RK2POLY is the one-source case with q = 1 + z + z^2/2).
constexpr int APPLY_POLY = 100;
struct ApplyOp {
  int nb;                            // number of blocks (block-diagonal modes)
  int mode;                          // APPLY_POLY or block diagonal (any other value)
  int src[MAXBLK];
  double coef[MAXBLK];
  int npoly;                         // APPLY_POLY: sources (1 or 2, views in0 / in1)
  int deg[2];
  double pc[2][3];
  ApplyFactor f[MAXBLK][HT_MAXD];
};

// y = A x for one factor on a column of length n; x in shared memory
__device__ double apply_factor_at(const ApplyFactor& F, const double* x, int n, int j, double xsum) {
  switch (F.kind) {
    case HT_F_IDENTITY: return x[j];
    case HT_F_STENCIL: {
      double s = 0.0;
      for (int o = -F.hw; o <= F.hw; ++o) {
        int jj = (j + o) % n;
        if (jj < 0) jj += n;
        s = fma(F.c[o + F.hw], x[jj], s);
      }
      return s;
    }
    case HT_F_DIAG: return F.v[j] * x[j];
    case HT_F_RANK1: return F.v[j] * xsum;
    case HT_F_DIAG_STENCIL: {
      double s = 0.0;
      for (int o = -F.hw; o <= F.hw; ++o) {
        int jj = (j + o) % n;
        if (jj < 0) jj += n;
        s = fma(F.c[o + F.hw], x[jj], s);
      }
      return F.v[j] * s;
    }
  }
  return 0.0;
}

// Leaves: for each leaf (blockIdx.y), every input column (blockIdx.x-strided) of every block
// is loaded to shared memory and the block's 1-D factor is applied to it.
// RK2POLY: [U, A U, A^2 U] with A = dt * L_i.
__device__ void apply_leaf_body(const ApplyOp& op, const TreeInfo& T, const Levels& L, const HtView& in0,
                                const HtView& in1, const HtView& out) {
  extern __shared__ double sh[];
  const int leaf = L.leaf[blockIdx.y];
  const int dim = T.lo[leaf];
  const int n = out.n[dim];
  double* x = sh;          // n
  double* y = sh + n;      // n
  __shared__ double red[32];
  if (op.mode == APPLY_POLY) {
    // columns [U_s, A U_s, .., A^deg_s U_s] of every source s, one after the other
    const ApplyFactor& F = op.f[0][dim];
    int off = 0;
    for (int sidx = 0; sidx < op.npoly; ++sidx) {
      const HtView& sv = sidx == 0 ? in0 : in1;
      const int K = sv.rank[leaf], dg = op.deg[sidx];
      for (int c = blockIdx.x; c < K; c += gridDim.x) {
        const double* src = sv.node[leaf] + (long long)n * c;
        for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = src[j];
        __syncthreads();
        double* o0 = out.node[leaf] + (long long)n * (off + c);
        double* o1 = out.node[leaf] + (long long)n * (off + K + c);
        double* o2 = out.node[leaf] + (long long)n * (off + 2 * K + c);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          o0[j] = x[j];
          if (dg >= 1) {
            const double v = apply_factor_at(F, x, n, j, 0.0);
            y[j] = v;
            o1[j] = v;
          }
        }
        __syncthreads();
        if (dg >= 2)
          for (int j = threadIdx.x; j < n; j += blockDim.x) o2[j] = apply_factor_at(F, y, n, j, 0.0);
        __syncthreads();
      }
      off += (dg + 1) * K;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out.rank[leaf] = off;
    return;
  }
  int off = 0;
  for (int b = 0; b < op.nb; ++b) {
    const HtView& sv = op.src[b] == 0 ? in0 : in1;
    const int K = sv.rank[leaf];
    const ApplyFactor& F = op.f[b][dim];
    for (int c = blockIdx.x; c < K; c += gridDim.x) {
      const double* src = sv.node[leaf] + (long long)n * c;
      for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = src[j];
      __syncthreads();
      double xsum = 0.0;
      if (F.kind == HT_F_RANK1) {
        double s = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) s = fma(F.w[j], x[j], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        double tt = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += red[w];
        xsum = tt;
      }
      double* o = out.node[leaf] + (long long)n * (off + c);
      for (int j = threadIdx.x; j < n; j += blockDim.x) o[j] = apply_factor_at(F, x, n, j, xsum);
      __syncthreads();
    }
    off += K;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out.rank[leaf] = off;
}

__device__ inline double binom3(int j, int j1) {   // C(j, j1) for j <= 2
  return (j == 2 && j1 == 1) ? 2.0 : 1.0;
}

// Transfer tensors: binomial block pattern (RK2POLY) or block diagonal (other modes).
__device__ inline int find_block(const int* offs, int nb, int i, int* local) {
  int b = 0;
  while (b + 1 < nb && offs[b + 1] <= i) ++b;
  *local = i - offs[b];
  return b;
}

__device__ void apply_xfer_body(const ApplyOp& op, const TreeInfo& T, const Levels& L, const HtView& in0,
                                const HtView& in1, const HtView& out) {
  const int t = L.proj2[blockIdx.y];   // interior nodes and the root
  const int a = T.c1[t], b = T.c2[t];
  int oa[MAXBLK + 1], ob[MAXBLK + 1], ot[MAXBLK + 1];
  int bs[MAXBLK], bj[MAXBLK];   // APPLY_POLY: source and power of each block
  int nb = op.nb;
  if (op.mode == APPLY_POLY) {
    nb = 0;
    oa[0] = ob[0] = ot[0] = 0;
    for (int sidx = 0; sidx < op.npoly; ++sidx) {
      const HtView& sv = sidx == 0 ? in0 : in1;
      for (int j = 0; j <= op.deg[sidx]; ++j) {
        bs[nb] = sidx;
        bj[nb] = j;
        oa[nb + 1] = oa[nb] + sv.rank[a];
        ob[nb + 1] = ob[nb] + sv.rank[b];
        ot[nb + 1] = ot[nb] + (t == 0 ? 1 : sv.rank[t]);
        ++nb;
      }
    }
  } else {
    oa[0] = ob[0] = ot[0] = 0;
    for (int j = 0; j < nb; ++j) {
      const HtView& sv = op.src[j] == 0 ? in0 : in1;
      oa[j + 1] = oa[j] + sv.rank[a];
      ob[j + 1] = ob[j] + sv.rank[b];
      ot[j + 1] = ot[j] + (t == 0 ? 1 : sv.rank[t]);
    }
  }
  const int M1 = oa[nb], M2 = ob[nb], M3 = (t == 0) ? 1 : ot[nb];
  const long long total = (long long)M1 * M2 * M3;
  double* O = out.node[t];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int i1 = (int)(e % M1);
    const int i2 = (int)((e / M1) % M2);
    const int i3 = (int)(e / ((long long)M1 * M2));
    int aa, bb, cc = 0;
    const int j1 = find_block(oa, nb, i1, &aa);
    const int j2 = find_block(ob, nb, i2, &bb);
    double v = 0.0;
    if (op.mode == APPLY_POLY) {
      // blocks j1, j2 (j3) are (source, power) pairs: nonzero only within one source, with
      // power(j3) = power(j1) + power(j2) (root: the polynomial coefficient of that power)
      const int sidx = bs[j1];
      if (bs[j2] == sidx) {
        const HtView& sv = sidx == 0 ? in0 : in1;
        const int K1 = sv.rank[a], K2 = sv.rank[b];
        const int p1 = bj[j1], p2 = bj[j2], pw = p1 + p2;
        if (t == 0) {
          if (pw <= op.deg[sidx]) v = op.pc[sidx][pw] * binom3(pw, p1) * sv.node[0][aa + (long long)K1 * bb];
        } else {
          const int j3 = find_block(ot, nb, i3, &cc);
          if (bs[j3] == sidx && bj[j3] == pw)
            v = binom3(pw, p1) * sv.node[t][aa + (long long)K1 * (bb + (long long)K2 * cc)];
        }
      }
    } else if (j1 == j2) {
      const HtView& sv = op.src[j1] == 0 ? in0 : in1;
      const int K1 = sv.rank[a], K2 = sv.rank[b];
      if (t == 0) {
        v = op.coef[j1] * sv.node[0][aa + (long long)K1 * bb];
      } else {
        const int j3 = find_block(ot, nb, i3, &cc);
        if (j3 == j1) v = sv.node[t][aa + (long long)K1 * (bb + (long long)K2 * cc)];
      }
    }
    O[e] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && t != 0) out.rank[t] = ot[nb];
}

// the operator travels as a kernel parameter (at most 32764 bytes on this architecture)
static_assert(sizeof(ApplyOp) + sizeof(TreeInfo) + sizeof(Levels) + 3 * sizeof(HtView) <= 32000,
              "apply kernel parameters exceed the parameter space");

__global__ void apply_leaf_kernel(ApplyOp op, TreeInfo T, Levels L, HtView in0, HtView in1, HtView out) {
  apply_leaf_body(op, T, L, in0, in1, out);
}

__global__ void apply_xfer_kernel(ApplyOp op, TreeInfo T, Levels L, HtView in0, HtView in1, HtView out) {
  apply_xfer_body(op, T, L, in0, in1, out);
}

// batched forms: instance blockIdx.z, its operator op_sel and views in0_sel, in1_sel, out_sel
__global__ void apply_leaf_batch_kernel(const Inst* I, TreeInfo T, Levels L, int op_sel, int in0_sel, int in1_sel,
                                        int out_sel) {
  const Inst& x = I[blockIdx.z];
  apply_leaf_body(*x.op[op_sel], T, L, x.view[in0_sel], x.view[in1_sel], x.view[out_sel]);
}

__global__ void apply_xfer_batch_kernel(const Inst* I, TreeInfo T, Levels L, int op_sel, int in0_sel, int in1_sel,
                                        int out_sel) {
  const Inst& x = I[blockIdx.z];
  apply_xfer_body(*x.op[op_sel], T, L, x.view[in0_sel], x.view[in1_sel], x.view[out_sel]);
}

// ------------------------------------------------------------ misc kernels ----
__global__ void from_cp_kernel(TreeInfo T, HtView out, const double* const* fac, const double* w, int r) {
  const int t = blockIdx.y;
  double* O = out.node[t];
  if (T.c1[t] < 0) {
    const int n = out.n[T.lo[t]];
    const double* F = fac[T.lo[t]];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * r;
         e += (long long)gridDim.x * blockDim.x)
      O[e] = F[e];
  } else if (t == 0) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)r * r;
         e += (long long)gridDim.x * blockDim.x)
      O[e] = (e % r == e / r) ? w[e % r] : 0.0;
  } else {
    const long long r2 = (long long)r * r;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < r2 * r;
         e += (long long)gridDim.x * blockDim.x) {
      const long long a = e % r, b = (e / r) % r, c = e / r2;
      O[e] = (a == b && b == c) ? 1.0 : 0.0;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out.rank[t] = (t == 0) ? 1 : r;
}

// <u, w> (or the mass when w == nullptr: contraction with all-ones vectors), one CTA.
// G_leaf = U^T W; G_t[k,l] = sum B_u[a,b,k] G_a[a,a'] G_b[b,b'] B_w[a',b',l]; root likewise.
__global__ void inner_kernel(TreeInfo T, HtView u, HtView w, int use_ones, double* gbuf, long long gstride,
                             double* tmp, double* out) {
  for (int dep = T.max_depth; dep >= 0; --dep) {
    for (int t = 0; t < T.nn; ++t) {
      if (T.depth[t] != dep) continue;
      double* G = gbuf + gstride * t;
      const int ku = (t == 0) ? 1 : u.rank[t];
      const int kw = use_ones ? 1 : ((t == 0) ? 1 : w.rank[t]);
      if (T.c1[t] < 0) {
        const int n = u.n[T.lo[t]];
        for (int e = threadIdx.x; e < ku * kw; e += blockDim.x) {
          const int k = e % ku, l = e / ku;
          double s = 0.0;
          for (int j = 0; j < n; ++j)
            s += u.node[t][j + (long long)n * k] * (use_ones ? 1.0 : w.node[t][j + (long long)n * l]);
          G[e] = s;
        }
      } else {
        const int a = T.c1[t], b = T.c2[t];
        const int A1 = u.rank[a], A2 = u.rank[b];
        const int W1 = use_ones ? 1 : w.rank[a], W2 = use_ones ? 1 : w.rank[b];
        const double* Ga = gbuf + gstride * a;
        const double* Gb = gbuf + gstride * b;
        const double* Bu = u.node[t];
        const double* Bw = use_ones ? nullptr : w.node[t];
        // tmp[a', b', k] = sum_{a,b} Ga[a,a'] Gb[b,b'] Bu[a,b,k]
        for (long long e = threadIdx.x; e < (long long)W1 * W2 * ku; e += blockDim.x) {
          const int ap = (int)(e % W1), bp = (int)((e / W1) % W2), k = (int)(e / ((long long)W1 * W2));
          double s = 0.0;
          for (int bb = 0; bb < A2; ++bb) {
            double sa = 0.0;
            for (int aa = 0; aa < A1; ++aa)
              sa += Ga[aa + (long long)A1 * ap] * Bu[aa + (long long)A1 * (bb + (long long)A2 * k)];
            s += Gb[bb + (long long)A2 * bp] * sa;
          }
          tmp[e] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ku * kw; e += blockDim.x) {
          const int k = e % ku, l = e / ku;
          double s = 0.0;
          for (int ap = 0; ap < W1; ++ap)
            for (int bp = 0; bp < W2; ++bp) {
              const double bw = use_ones ? 1.0 : Bw[ap + (long long)W1 * (bp + (long long)W2 * l)];
              s += tmp[ap + (long long)W1 * (bp + (long long)W2 * k)] * bw;
            }
          G[e] = s;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) *out = gbuf[0];
}

}  // namespace

// ================================================================ host side =====
#define HTG_LAUNCH(ctx, cls, s, expr)          \
  do {                                         \
    htg_prof_begin((ctx), (s));                \
    cudaError_t _e = (expr);                   \
    htg_prof_end((ctx), (cls), (s));           \
    (ctx)->launches++;                         \
    if (_e != cudaSuccess) return HT_ERR_CUDA; \
  } while (0)

static void build_levels(const TreeInfo& T, Levels* L) {
  memset(L, 0, sizeof(*L));
  for (int dep = 1; dep <= T.max_depth; ++dep) {
    for (int t = 1; t < T.nn; ++t) {
      if (T.depth[t] != dep) continue;
      L->all[dep][L->n_all[dep]++] = t;
      if (T.c1[t] >= 0) L->inter[dep][L->n_int[dep]++] = t;
    }
  }
  for (int i = 0; i < T.d; ++i)
    for (int t = 0; t < T.nn; ++t)
      if (T.c1[t] < 0 && T.lo[t] == i) L->leaf[L->n_leaf++] = t;
  for (int t = 0; t < T.nn; ++t) L->proj1[L->n_proj1++] = t;
  for (int t = 0; t < T.nn; ++t)
    if (T.c1[t] >= 0) L->proj2[L->n_proj2++] = t;
  for (int t = 1; t < T.nn; ++t)
    if (T.c1[t] >= 0) L->proj3[L->n_proj3++] = t;
}

static bool cfg_valid(const ht_config* c) {
  if (!c || c->d < 2 || c->d > HT_MAXD || c->cap < 1 || c->max_terms < 1 || c->max_terms > HT_MAXTERMS)
    return false;
  for (int i = 0; i < c->d; ++i)
    if (c->n[i] < 1) return false;
  if (c->tree != HT_TREE_BALANCED && c->tree != HT_TREE_LINEAR) return false;
  if (c->tc_min_work < -1 || c->gemm_ctas_per_sm < 0 || c->gemm_ctas_per_sm > 32) return false;
  if (c->svd_cluster_min_cols != 0 && (c->svd_cluster_min_cols < 32 || c->svd_cluster_min_cols > 480)) return false;
  if (c->cp_form != 0 && c->cp_form != 1) return false;
  if (c->biorth_form != 0 && c->biorth_form != 1) return false;
  if (c->precision == HT_PREC_MIXED)
    return c->mixed_slices == 0 || (c->mixed_slices >= 2 && c->mixed_slices <= 4);
  return c->precision == HT_PREC_FP64;
}

static int trunc_input_cap(const ht_config* c) {
  // RK2POLY raises ranks by 3; HEUN2 stage sums reach (terms + 2) * cap
  return htg_max(3, c->max_terms + 2) * c->cap;
}

struct WsLayout {
  size_t off_plan, off_err, off_tick, off_app_rank, off_stage_rank, off_wn, off_ptrs, off_cp[12], off_prof;
  size_t off_coop[6];           // cooperative QR: part, tot, rowj, diag, bar, wtot (0 when not used)
  size_t node_off[NN][16];
  size_t app_off[NN], stage_off[NN];
  size_t total;
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static void layout(const ht_config* c, const TreeInfo& T, WsLayout* W) {
  const size_t Kc = (size_t)trunc_input_cap(c);
  size_t off = 0;
  W->off_plan = off; off = align_up(off + sizeof(Plan));
  W->off_err = off; off = align_up(off + 64);
  W->off_tick = off; off = align_up(off + 2 * NN * sizeof(unsigned));
  for (int j = 0; j < 6; ++j) W->off_coop[j] = 0;
  if ((size_t)Kc >= (size_t)QR_COOP_MIN_KC) {
    const size_t nd = QR_COOP_NDMAX, sl = QR_COOP_SLOTS, qb = QR_COOP_QB;
    const size_t slot = qb * (qb + Kc);   // a panel's partial block
    const size_t sz[6] = {sl * (2 * Kc + slot) * sizeof(double), nd * Kc * sizeof(double), 2 * nd * Kc * sizeof(double),
                          nd * Kc * sizeof(double), sl * sizeof(unsigned), nd * slot * sizeof(double)};
    for (int j = 0; j < 6; ++j) {
      W->off_coop[j] = off;
      off = align_up(off + sz[j]);
    }
  }
  W->off_app_rank = off; off = align_up(off + NN * sizeof(int));
  W->off_stage_rank = off; off = align_up(off + NN * sizeof(int));
  W->off_wn = off; off = align_up(off + NN * sizeof(WsNode));
  W->off_prof = off; off = align_up(off + KC_COUNT * sizeof(double));
  W->off_ptrs = off; off = align_up(off + 4 * HT_MAXD * sizeof(void*));
  {
    const size_t rc = (size_t)c->cap, ry = rc * (size_t)htg_cp_terms(c->d);
    size_t nmax = 1;
    for (int i = 0; i < c->d; ++i) nmax = nmax > (size_t)c->n[i] ? nmax : (size_t)c->n[i];
    const size_t cps[12] = {c->d * rc * rc, c->d * ry * rc, ry * rc, rc * rc, nmax * rc,
                            HT_MAXD * nmax * rc, rc, 64, (4 * HT_MAXD * sizeof(GemmDesc)) / sizeof(double) + 1,
                            HT_MAXD * nmax * 3 * rc, 4 + 32,   // acc2 (4 doubles) + 64 barrier words
                            HT_MAXD * nmax * 3 * rc};          // ZT
    for (int j = 0; j < 12; ++j) {
      W->off_cp[j] = off;
      off = align_up(off + cps[j] * sizeof(double));
    }
  }
  size_t nmax = 1;
  for (int i = 0; i < c->d; ++i) nmax = nmax > (size_t)c->n[i] ? nmax : (size_t)c->n[i];
  size_t K3 = Kc * Kc * Kc;
  if (K3 < nmax * Kc) K3 = nmax * Kc;             // leaf QR scratch (n x Kc)
  if (K3 < (size_t)NN * Kc * Kc) K3 = (size_t)NN * Kc * Kc;   // per-node Grams of ht_inner
  const size_t K2 = Kc * Kc;
  const size_t sizes[15] = {K2, K3, K3, K3, K3, K3, K2, K2, Kc, K2, K2, 6 * K2 + Kc + 8, K2, K2, Kc};
  for (int t = 0; t < T.nn; ++t) {
    for (int j = 0; j < 15; ++j) {
      // leaves never hold an absorbed transfer (Tabs, Cabs) or B x3 E^T (T1); the root has no
      // QR and no absorbed transfer (Cabs, S)
      const bool unused = (T.c1[t] < 0 && (j == 1 || j == 2 || j == 5)) || (t == 0 && (j == 2 || j == 3));
      W->node_off[t][j] = off;
      off = align_up(off + (unused ? 8 : sizes[j]) * sizeof(double));
    }
  }
  for (int t = 0; t < T.nn; ++t) {
    size_t sz = (T.c1[t] < 0) ? (size_t)c->n[T.lo[t]] * Kc : (t == 0 ? K2 : K3);
    W->app_off[t] = off; off = align_up(off + sz * sizeof(double));
    W->stage_off[t] = off; off = align_up(off + sz * sizeof(double));
  }
  W->total = off;
}

extern "C" size_t ht_workspace_bytes(const ht_config* cfg) {
  if (!cfg_valid(cfg)) return 0;
  TreeInfo T;
  htg_build_tree(cfg->d, cfg->tree, &T);
  WsLayout W;
  layout(cfg, T, &W);
  return W.total;
}

// Upper bounds of the work (multiply-adds m n k batch) of every contraction list a truncation of
// this context issues, from the planner's shapes with every input rank at the capacity Kc, the
// R-factor rows Rp bounded by the grid and by the children's Rp, the complement columns mE by the
// sibling's Rp, and the new ranks by cap; a list whose bound stays below tc_min never reaches
// the tensor cores, so its tensor-core launch (which would find no work) is left out.
static void tc_list_bounds(ht_ctx* c, const ht_config* cfg) {
  const TreeInfo& T = c->tree;
  const double Kc = c->Kc, cap = c->cap, tcm = (double)c->tc_min;
  double Rp[NN] = {0}, mE[NN] = {0}, kn[NN] = {0};
  for (int dep = T.max_depth; dep >= 1; --dep)
    for (int t = 1; t < T.nn; ++t) {
      if (T.depth[t] != dep) continue;
      Rp[t] = (T.c1[t] < 0) ? std::min(Kc, (double)cfg->n[T.lo[t]]) : std::min(Kc, Rp[T.c1[t]] * Rp[T.c2[t]]);
    }
  const int ra = T.c1[0], rb = T.c2[0];
  mE[ra] = Rp[rb];
  mE[rb] = Rp[ra];
  for (int dep = 1; dep < T.max_depth; ++dep)
    for (int t = 1; t < T.nn; ++t) {
      if (T.depth[t] != dep || T.c1[t] < 0) continue;
      mE[T.c1[t]] = std::min(Kc, Rp[T.c2[t]] * mE[t]);
      mE[T.c2[t]] = std::min(Kc, Rp[T.c1[t]] * mE[t]);
    }
  for (int t = 1; t < T.nn; ++t) kn[t] = std::min(cap, Rp[t]);
  double w_rootE = std::max(Kc * Rp[rb] * Kc, Kc * Rp[ra] * Kc), w_Pall = 0, w_XY = 0, w_p1 = 0, w_p2 = 0, w_p3 = 0;
  for (int dep = 0; dep < MAXLEV; ++dep)
    for (int j = 0; j < ht_ctx::TL_LEVEL; ++j) c->tc_lvl[dep][j] = false;
  w_p1 = kn[ra] * Kc * Kc;            // the root's projection
  w_p2 = kn[ra] * kn[rb] * Kc;
  for (int t = 1; t < T.nn; ++t) {
    w_Pall = std::max(w_Pall, Rp[t] * mE[t] * Kc);
    w_XY = std::max(w_XY, std::max(kn[t] * Kc * Rp[t], Kc * kn[t] * mE[t]));
    if (T.c1[t] < 0) {
      w_p1 = std::max(w_p1, (double)cfg->n[T.lo[t]] * kn[t] * Kc);
      continue;
    }
    const int a = T.c1[t], b = T.c2[t], dep = T.depth[t];
    w_p1 = std::max(w_p1, Kc * Kc * kn[t] * Kc);
    w_p2 = std::max(w_p2, kn[a] * Kc * kn[t] * Kc);
    w_p3 = std::max(w_p3, kn[a] * kn[b] * Kc * kn[t]);
    bool* f = c->tc_lvl[dep];
    f[ht_ctx::TL_ABS1] = f[ht_ctx::TL_ABS1] || Rp[a] * Kc * Kc * Kc >= tcm;
    f[ht_ctx::TL_ABS2] = f[ht_ctx::TL_ABS2] || Rp[a] * Rp[b] * Kc * Kc >= tcm;
    f[ht_ctx::TL_T1] = f[ht_ctx::TL_T1] || Kc * Kc * mE[t] * Kc >= tcm;
    f[ht_ctx::TL_EPRE] = f[ht_ctx::TL_EPRE] || std::max(Rp[a], Rp[b]) * Kc * Kc * mE[t] >= tcm;
  }
  c->tc_rootE = w_rootE >= tcm;
  c->tc_Pall = w_Pall >= tcm;
  c->tc_XY = w_XY >= tcm;
  c->tc_proj[0] = w_p1 >= tcm;
  c->tc_proj[1] = w_p2 >= tcm;
  c->tc_proj[2] = w_p3 >= tcm;
}

extern "C" int ht_ctx_create(ht_ctx** out, const ht_config* cfg) {
  if (!out) return HT_ERR_ARG;
  *out = nullptr;
  if (!cfg_valid(cfg)) return HT_ERR_ARG;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return HT_ERR_CUDA;
  ht_ctx* c = new ht_ctx();
  c->cfg = *cfg;
  htg_build_tree(cfg->d, cfg->tree, &c->tree);
  build_levels(c->tree, &c->lev);
  c->Kc = trunc_input_cap(cfg);
  c->cap = cfg->cap;
  c->svd_min_cols = cfg->svd_cluster_min_cols ? cfg->svd_cluster_min_cols : 128;
  if (c->Kc > 2 * HTG_SVD_MAXP) { delete c; return HT_ERR_CAPACITY; }
  WsLayout W;
  layout(cfg, c->tree, &W);
  c->ws_bytes = W.total;
  if (cudaMalloc(&c->ws, W.total) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return HT_ERR_NOMEM;
  }
  char* base = (char*)c->ws;
  c->plan = (Plan*)(base + W.off_plan);
  c->err = (int*)(base + W.off_err);
  c->app_rank = (int*)(base + W.off_app_rank);
  c->stage_rank = (int*)(base + W.off_stage_rank);
  for (int t = 0; t < c->tree.nn; ++t) {
    double** f[15] = {&c->wn[t].Rf, &c->wn[t].Tabs, &c->wn[t].Cabs, &c->wn[t].S, &c->wn[t].Epre,
                      &c->wn[t].T1, &c->wn[t].E, &c->wn[t].P, &c->wn[t].sig, &c->wn[t].W,
                      &c->wn[t].Z, &c->wn[t].SW, &c->wn[t].X, &c->wn[t].Y, &c->wn[t].invsig};
    for (int j = 0; j < 15; ++j) *f[j] = (double*)(base + W.node_off[t][j]);
    c->wn[t].tick = (unsigned*)(base + W.off_tick) + 2 * t;
    c->app[t] = (double*)(base + W.app_off[t]);
    c->stage[t] = (double*)(base + W.stage_off[t]);
  }
  c->wn_dev = (WsNode*)(base + W.off_wn);
  if (W.off_coop[0]) {
    c->has_coop = true;
    c->qr_coop.part = (double*)(base + W.off_coop[0]);
    c->qr_coop.tot = (double*)(base + W.off_coop[1]);
    c->qr_coop.rowj = (double*)(base + W.off_coop[2]);
    c->qr_coop.diag = (double*)(base + W.off_coop[3]);
    c->qr_coop.bar = (unsigned*)(base + W.off_coop[4]);
    c->qr_coop.wtot = (double*)(base + W.off_coop[5]);
    c->qr_coop.err = c->err;
    c->qr_coop.kmax = c->Kc;
    c->qr_coop.ndmax = QR_COOP_NDMAX;
    c->qr_coop.gmax = QR_COOP_GMAX;
  }
  c->prof_flops = (double*)(base + W.off_prof);
  c->ptr_tbl = (const double**)(base + W.off_ptrs);
  {
    double** cpf[8] = {&c->cp.G, &c->cp.H, &c->cp.Hh, &c->cp.Gam, &c->cp.RHS, &c->cp.Xold, &c->cp.wold, &c->cp.epsacc};
    for (int j = 0; j < 8; ++j) *cpf[j] = (double*)(base + W.off_cp[j]);
    c->cp.descs = (GemmDesc*)(base + W.off_cp[8]);
    c->cp.Z = (double*)(base + W.off_cp[9]);
    c->cp.acc2 = (double*)(base + W.off_cp[10]);
    c->cp.bar = (unsigned int*)(base + W.off_cp[10] + 4 * sizeof(double));
    c->cp.ZT = (double*)(base + W.off_cp[11]);
    c->cp.rcap = cfg->cap;
    c->cp.rycap = cfg->cap * htg_cp_terms(cfg->d);
    int nmax = 1;
    for (int i = 0; i < cfg->d; ++i) nmax = htg_max(nmax, cfg->n[i]);
    c->cp.nmax = nmax;
  }
  if (cudaMemset(c->err, 0, 64) != cudaSuccess ||
      cudaMemset(base + W.off_tick, 0, 2 * NN * sizeof(unsigned)) != cudaSuccess ||
      cudaMemcpy(c->wn_dev, c->wn, sizeof(WsNode) * NN, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return HT_ERR_CUDA;
  }
  if (cudaFuncSetAttribute(biorth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BIORTH_SMEM) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return HT_ERR_CUDA;
  }
  c->cp_clu = htg_cp_cluster_setup(cfg->device);
  // wide node factors, on request: the cluster form of the X_t Y_t = I refinement
  if (cfg->biorth_form == 1 && c->Kc >= BIORTH_CLUSTER_MIN_KC) c->bi_cl = biorth_cluster_setup();
  // wide node factors: the cluster form of the SVD, when a cluster fits this device
  if (c->Kc >= c->svd_min_cols) {
    c->svd_clu = htg_svd_cluster_setup(cfg->device);
    c->svd_clu.min_p = c->svd_min_cols;
  }
  // SVD working copy in shared memory when the capacity allows
  const size_t Kc = (size_t)c->Kc;
  c->svd_smem = ((2 * Kc * Kc + Kc) * sizeof(double) <= 200 * 1024) ? 1 : 0;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg->device);
  // FP64 contraction CTAs per SM: the autotuner's measurement on GB300 (small tiles of 64 threads
  // over many SMs hide the FP64 pipe's latency: 16 per SM were 1.4-2.4x faster than 4 on the
  // contractions of contexts with Kc >= 96, 8 per SM best below)
  c->gemm_grid = htg_max(1, sms) * (cfg->gemm_ctas_per_sm ? cfg->gemm_ctas_per_sm : (c->Kc >= 96 ? 16 : 8));
  c->sms = htg_max(1, sms);
  c->slices = (cfg->precision == HT_PREC_MIXED) ? (cfg->mixed_slices ? cfg->mixed_slices : 4) : 0;
  if (c->slices) {
    // the largest contraction a truncation of this context can issue: an absorbed or projected
    // transfer tensor (Kc^4 multiply-adds) or a leaf projection (n Kc^2)
    int nmax = 1;
    for (int i = 0; i < cfg->d; ++i) nmax = htg_max(nmax, cfg->n[i]);
    const double kc = (double)c->Kc;
    const double wmax = kc * kc * kc * kc > (double)nmax * kc * kc ? kc * kc * kc * kc : (double)nmax * kc * kc;
    c->tc_min = (cfg->tc_min_work == -1) ? 0 : (cfg->tc_min_work ? cfg->tc_min_work : HTG_TC_MIN_WORK_DEFAULT);
    c->tc_reach = (double)c->tc_min <= wmax;
    tc_list_bounds(c, cfg);
  }
  *out = c;
  return HT_OK;
}

extern "C" void ht_ctx_destroy(ht_ctx* ctx) {
  if (!ctx) return;
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->cn_ws) cudaFree(ctx->cn_ws);
  delete ctx;
}

extern "C" long long ht_ctx_launches(const ht_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" int ht_biorth_cluster_ctas(const ht_ctx* ctx, int* ctas) {
  if (!ctx || !ctas) return HT_ERR_ARG;
  *ctas = ctx->bi_cl;
  return HT_OK;
}

extern "C" int ht_ctx_check(ht_ctx* ctx, void* stream) {
  if (!ctx) return HT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  if (cudaMemcpyAsync(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return HT_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return HT_ERR_CUDA;
  if (h != 0) cudaMemsetAsync(ctx->err, 0, sizeof(int), s);
  return h;
}

extern "C" const char* ht_status_string(int s) {
  switch (s) {
    case HT_OK: return "HT_OK";
    case HT_ERR_ARG: return "HT_ERR_ARG";
    case HT_ERR_CAPACITY: return "HT_ERR_CAPACITY";
    case HT_ERR_CUDA: return "HT_ERR_CUDA";
    case HT_ERR_NONFINITE: return "HT_ERR_NONFINITE";
    case HT_ERR_TIMEOUT: return "HT_ERR_TIMEOUT";
    case HT_ERR_NOMEM: return "HT_ERR_NOMEM";
  }
  return "HT_ERR_UNKNOWN";
}

extern "C" int ht_tree_info(int d, int kind, int* lo, int* hi, int* c1, int* c2, int* parent, int* depth) {
  if (d < 2 || d > HT_MAXD || (kind != HT_TREE_BALANCED && kind != HT_TREE_LINEAR)) return HT_ERR_ARG;
  TreeInfo T;
  htg_build_tree(d, kind, &T);
  for (int t = 0; t < T.nn; ++t) {
    if (lo) lo[t] = T.lo[t];
    if (hi) hi[t] = T.hi[t];
    if (c1) c1[t] = T.c1[t];
    if (c2) c2[t] = T.c2[t];
    if (parent) parent[t] = T.parent[t];
    if (depth) depth[t] = T.depth[t];
  }
  return HT_OK;
}

static bool tensor_matches(const ht_ctx* c, const ht_tensor* u) {
  if (!u || u->d != c->cfg.d || !u->rank || u->cap < 1) return false;
  for (int i = 0; i < u->d; ++i)
    if (u->n[i] != c->cfg.n[i]) return false;
  for (int t = 0; t < c->tree.nn; ++t)
    if (!u->node[t]) return false;
  return true;
}

static HtView view_of(const ht_tensor* u) {
  HtView v;
  memset(&v, 0, sizeof(v));
  for (int t = 0; t < HT_MAXNODES; ++t) v.node[t] = u->node[t];
  v.rank = u->rank;
  for (int i = 0; i < HT_MAXD; ++i) v.n[i] = u->n[i];
  return v;
}

static HtView view_ws(ht_ctx* c, double* const* nodes, int* rank) {
  HtView v;
  memset(&v, 0, sizeof(v));
  for (int t = 0; t < c->tree.nn; ++t) v.node[t] = nodes[t];
  v.rank = rank;
  for (int i = 0; i < c->cfg.d; ++i) v.n[i] = c->cfg.n[i];
  return v;
}


// ---------------------------------------------------------------- truncation --
// Launch sequence of one truncation (the HSVD of Section 2.2 in R-factor form) for `count`
// instances: instance i's descriptors sit in plan P + i.  pre() and sel() launch the planner and
// the rank selection (single-instance or batched kernels).
template <class Pre, class Sel>
static int truncate_launches(ht_ctx* c, Plan* P, int count, int Kc, int svd_smem, Pre pre, Sel sel, cudaStream_t s) {
  const TreeInfo& T = c->tree;
  const Levels& L = c->lev;
  const int g = c->gemm_grid;
  const long long st = (long long)sizeof(Plan);
  // the dense contractions: FP64 CUDA-core tiles; in HT_PREC_MIXED those of at least tc_min
  // multiply-adds (decided per descriptor on the device) on the tensor cores, the rest in the
  // split-FP32 form on the CUDA cores (the same tiles, FP64-like accuracy on the FP32 pipe)
  const bool tc_on = c->slices && c->tc_reach;
  const long long tcm = tc_on ? htg_max_ll(1, c->tc_min) : 0;
  auto gemm64 = [&](const GemmDesc* d, int nd, bool tc_here) -> cudaError_t {
    const long long cut = tc_here ? tcm : 0;   // 0: every descriptor on the CUDA cores
    return c->slices ? htg_launch_gemm_f32x2(d, nd, g, s, htg_prof_flops(c, KC_GEMM), count, st, cut)
                     : htg_launch_gemm(d, nd, g, s, htg_prof_flops(c, KC_GEMM), count, st, cut);
  };
  auto gemmtc = [&](const GemmDesc* d, int nd) -> cudaError_t {
    return htg_launch_gemm_tc(d, nd, c->sms, c->slices, s, htg_prof_flops(c, KC_GEMMTC), count, st, c->err, tcm);
  };
  // FLAG: whether the list can reach the tensor cores (single truncations; a batch launches both
  // kernels for every list); without them the CUDA-core kernel takes every descriptor
#define HTG_GEMM(DESCS, ND, FLAG)                                                            \
  do {                                                                                       \
    const bool tc_here = tc_on && (count > 1 || (FLAG));                                     \
    if (!(tc_here && c->tc_min == 0)) HTG_LAUNCH(c, KC_GEMM, s, gemm64(DESCS, ND, tc_here)); \
    if (tc_here) HTG_LAUNCH(c, KC_GEMMTC, s, gemmtc(DESCS, ND));                             \
  } while (0)
  HTG_LAUNCH(c, KC_PLAN, s, pre());
  const QrCoopWs* coop = (c->has_coop && count == 1) ? &c->qr_coop : nullptr;
  const int coop_extra = coop ? 1 : 0;   // the cooperative QR launch beside each QR launch
  HTG_LAUNCH(c, KC_QR, s, htg_launch_qr(P->qr_leaf, L.n_leaf, s, htg_prof_flops(c, KC_QR), count, st, coop));
  c->launches += coop_extra;
  for (int dep = T.max_depth - 1; dep >= 1; --dep) {
    if (L.n_int[dep] == 0) continue;
    HTG_GEMM(P->g_abs1[dep], L.n_int[dep], c->tc_lvl[dep][ht_ctx::TL_ABS1]);
    HTG_GEMM(P->g_abs2[dep], L.n_int[dep], c->tc_lvl[dep][ht_ctx::TL_ABS2]);
    HTG_LAUNCH(c, KC_QR, s, htg_launch_qr(P->qr_orth[dep], L.n_int[dep], s, htg_prof_flops(c, KC_QR), count, st, coop));
    c->launches += coop_extra;
  }
  HTG_GEMM(P->g_rootE, 2, c->tc_rootE);
  // top-down complement factors: E of a child needs only E, B and R of its parent, never the
  // parent's SVD, so every node SVD runs afterwards in a single launch
  for (int dep = 1; dep < T.max_depth; ++dep) {
    if (L.n_int[dep] == 0) continue;
    HTG_GEMM(P->g_T1[dep], L.n_int[dep], c->tc_lvl[dep][ht_ctx::TL_T1]);
    HTG_GEMM(P->g_Epre[dep], 2 * L.n_int[dep], c->tc_lvl[dep][ht_ctx::TL_EPRE]);
    HTG_LAUNCH(c, KC_QR, s, htg_launch_qr(P->qr_comp[dep], 2 * L.n_int[dep], s, htg_prof_flops(c, KC_QR), count, st, coop));
    c->launches += coop_extra;
  }
  HTG_GEMM(P->g_Pall, T.nn - 1, c->tc_Pall);
  const SvdClusterCfg* clu = (count == 1) ? &c->svd_clu : nullptr;
  HTG_LAUNCH(c, KC_SVD, s,
             htg_launch_svd(P->svd_all, T.nn - 1, svd_smem, Kc, Kc, s, htg_prof_flops(c, KC_SVD), count, st, clu));
  c->launches += htg_svd_cluster_used(clu, count, Kc) ? 1 : 0;
  HTG_LAUNCH(c, KC_PLAN, s, sel());
  HTG_GEMM(P->g_XY, 2 * (T.nn - 1), c->tc_XY);
  HTG_LAUNCH(c, KC_GEMM, s, launch_biorth(c, P, T.nn - 1, count, st, htg_prof_flops(c, KC_GEMM), s));
  HTG_GEMM(P->g_proj1, L.n_proj1, c->tc_proj[0]);
  HTG_GEMM(P->g_proj2, L.n_proj2, c->tc_proj[1]);
  if (L.n_proj3 > 0)
    HTG_GEMM(P->g_proj3, L.n_proj3, c->tc_proj[2]);
  c->last_stream = s;
  return HT_OK;
}

static int run_truncate(ht_ctx* c, const HtView& in, int cap_in, const HtView& out, double rel_tol, int rmax,
                        double* sigma_dev, int sig_stride, double* norm_dev, cudaStream_t s) {
  const TreeInfo& T = c->tree;
  const Levels& L = c->lev;
  Plan* P = c->plan;
  const WsNode* wn = c->wn_dev;
  int* err = c->err;
  auto pre = [&]() {
    plan_pre_kernel<<<1, 1, 0, s>>>(P, T, L, in, wn, cap_in, sigma_dev ? 0.0 : rel_tol, err);
    return cudaGetLastError();
  };
  auto sel = [&]() {
    rank_select_kernel<<<1, 32, 0, s>>>(P, T, L, in, out, wn, rel_tol, rmax, sigma_dev, sig_stride, norm_dev, err);
    return cudaGetLastError();
  };
  return truncate_launches(c, P, 1, c->Kc, c->svd_smem, pre, sel, s);
}

static int copy_tensor_to(ht_ctx* c, const ht_tensor* u, double* const* dst, int* dst_rank, cudaStream_t s) {
  const TreeInfo& T = c->tree;
  for (int t = 0; t < T.nn; ++t) {
    size_t sz;
    if (T.c1[t] < 0) sz = (size_t)u->n[T.lo[t]] * u->cap;
    else if (t == 0) sz = (size_t)u->cap * u->cap;
    else sz = (size_t)u->cap * u->cap * u->cap;
    if (cudaMemcpyAsync(dst[t], u->node[t], sz * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return HT_ERR_CUDA;
  }
  if (cudaMemcpyAsync(dst_rank, u->rank, NN * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HT_ERR_CUDA;
  return HT_OK;
}

extern "C" int ht_truncate(ht_ctx* c, const ht_tensor* u, double rel_tol, int rmax, ht_tensor* out,
                           double* sigma_dev, int sig_stride, double* norm_dev, void* stream) {
  if (!c || !tensor_matches(c, u) || !tensor_matches(c, out)) return HT_ERR_ARG;
  if (rmax < 1 || !(rel_tol >= 0.0) || (sigma_dev && sig_stride < 1)) return HT_ERR_ARG;
  if (u->cap > c->Kc || out->cap < rmax) return HT_ERR_CAPACITY;
  if (sigma_dev && sig_stride < htg_min(u->cap, c->Kc)) return HT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  bool alias = false;
  for (int t = 0; t < c->tree.nn; ++t)
    if (u->node[t] == out->node[t]) alias = true;
  HtView in = view_of(u);
  if (alias) {
    int st = copy_tensor_to(c, u, c->stage, c->stage_rank, s);
    if (st != HT_OK) return st;
    in = view_ws(c, c->stage, c->stage_rank);
  }
  return run_truncate(c, in, u->cap, view_of(out), rel_tol, rmax, sigma_dev, sig_stride, norm_dev, s);
}

// ---------------------------------------------------------------- apply -------
static bool build_apply(const ht_ctx* c, const ht_op* L, double dt, int mode, ApplyOp* op) {
  memset(op, 0, sizeof(*op));
  const int d = c->cfg.d;
  if (!L || L->d != d || L->n_terms < 1 || L->n_terms > HT_MAXTERMS) return false;
  auto conv = [&](const ht_factor& f, double scale, ApplyFactor* o) -> bool {
    o->kind = f.kind;
    o->hw = 0;
    if (f.kind == HT_F_IDENTITY) {
      o->kind = HT_F_STENCIL;   // identity as a width-0 stencil carrying the scale
      o->c[0] = scale;
      return true;
    }
    if (f.kind == HT_F_STENCIL || f.kind == HT_F_DIAG_STENCIL) {
      if (f.half_width < 0 || 2 * f.half_width + 1 > HT_MAXSTENCIL) return false;
      if (f.kind == HT_F_DIAG_STENCIL && !f.v) return false;
      o->hw = f.half_width;
      for (int j = 0; j < 2 * f.half_width + 1; ++j) o->c[j] = scale * f.stencil[j];
      o->v = f.v;
      return true;
    }
    if (f.kind == HT_F_DIAG || f.kind == HT_F_RANK1) {
      if (!f.v || (f.kind == HT_F_RANK1 && !f.w)) return false;
      if (scale != 1.0) return false;   // scales of DIAG/RANK1 factors go into alpha
      o->v = f.v;
      o->w = f.w;
      return true;
    }
    return false;
  };
  op->mode = mode;
  if (mode == HT_APPLY_RK2POLY) {
    if (!L->kron_sum || L->n_terms != d) return false;
    for (int i = 0; i < d; ++i) {
      if (L->f[i][i].kind != HT_F_STENCIL) return false;
      for (int j = 0; j < d; ++j)
        if (j != i && L->f[i][j].kind != HT_F_IDENTITY) return false;
      if (!conv(L->f[i][i], dt * L->alpha[i], &op->f[0][i])) return false;
    }
    // p(z) = 1 + z + z^2/2 of one source
    op->mode = APPLY_POLY;
    op->npoly = 1;
    op->deg[0] = 2;
    op->pc[0][0] = 1.0;
    op->pc[0][1] = 1.0;
    op->pc[0][2] = 0.5;
    op->nb = 3;
    return true;
  }
  if (L->n_terms > HT_MAXBLOCKTERMS) return false;
  int b = 0;
  ht_factor ident;
  memset(&ident, 0, sizeof(ident));
  if (mode == HT_APPLY_EULER) {
    op->src[b] = 0;
    op->coef[b] = 1.0;
    for (int i = 0; i < d; ++i) conv(ident, 1.0, &op->f[b][i]);
    ++b;
  }
  const double sc = (mode == HT_APPLY_EULER) ? dt : 1.0;
  for (int q = 0; q < L->n_terms; ++q) {
    op->src[b] = 0;
    op->coef[b] = sc * L->alpha[q];
    for (int i = 0; i < d; ++i)
      if (!conv(L->f[q][i], 1.0, &op->f[b][i])) return false;
    ++b;
  }
  op->nb = b;
  return true;
}

static int launch_apply(ht_ctx* c, const ApplyOp& op, const HtView& in0, const HtView& in1,
                        const HtView& out, int max_cols, cudaStream_t s) {
  const TreeInfo& T = c->tree;
  const Levels& L = c->lev;
  int nmax = 1;
  for (int i = 0; i < c->cfg.d; ++i) nmax = htg_max(nmax, c->cfg.n[i]);
  dim3 gl(htg_max(1, htg_min(max_cols, 64)), L.n_leaf);
  const size_t smem = 2 * (size_t)nmax * sizeof(double);
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(apply_leaf_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return HT_ERR_CUDA;
  }
  HTG_LAUNCH(c, KC_APPLY, s, (apply_leaf_kernel<<<gl, 128, smem, s>>>(op, T, L, in0, in1, out), cudaGetLastError()));
  dim3 gx(c->gemm_grid, L.n_proj2);
  HTG_LAUNCH(c, KC_APPLY, s, (apply_xfer_kernel<<<gx, 256, 0, s>>>(op, T, L, in0, in1, out), cudaGetLastError()));
  c->last_stream = s;
  return HT_OK;
}

extern "C" int ht_apply(ht_ctx* c, const ht_tensor* u, const ht_op* L, double dt, int mode, ht_tensor* v,
                        void* stream) {
  if (!c || !tensor_matches(c, u) || !tensor_matches(c, v)) return HT_ERR_ARG;
  if (mode < HT_APPLY_L || mode > HT_APPLY_RK2POLY) return HT_ERR_ARG;
  for (int t = 0; t < c->tree.nn; ++t)
    if (u->node[t] == v->node[t]) return HT_ERR_ARG;
  ApplyOp op;
  if (!build_apply(c, L, dt, mode, &op)) return HT_ERR_ARG;
  const int mult = (mode == HT_APPLY_RK2POLY) ? 3 : op.nb;
  if ((long long)mult * u->cap > v->cap) return HT_ERR_CAPACITY;
  HtView in = view_of(u);
  return launch_apply(c, op, in, in, view_of(v), u->cap, (cudaStream_t)stream);
}

extern "C" int ht_step(ht_ctx* c, ht_tensor* u, const ht_op* L, double dt, double rel_tol, int rmax,
                       int scheme, void* stream) {
  if (!c || !tensor_matches(c, u)) return HT_ERR_ARG;
  if (rmax < 1 || rmax > u->cap || !(rel_tol >= 0.0)) return HT_ERR_ARG;
  if (u->cap > c->cap) return HT_ERR_CAPACITY;
  cudaStream_t s = (cudaStream_t)stream;
  HtView uv = view_of(u);
  HtView app = view_ws(c, c->app, c->app_rank);
  if (scheme == HT_SCHEME_RK2POLY) {
    ApplyOp op;
    if (!build_apply(c, L, dt, HT_APPLY_RK2POLY, &op)) return HT_ERR_ARG;
    int st = launch_apply(c, op, uv, uv, app, u->cap, s);
    if (st != HT_OK) return st;
    return run_truncate(c, app, c->Kc, uv, rel_tol, rmax, nullptr, 0, nullptr, s);
  }
  if (scheme == HT_SCHEME_HEUN2) {
    ApplyOp op;
    if (!build_apply(c, L, dt, HT_APPLY_EULER, &op)) return HT_ERR_ARG;
    if ((long long)(op.nb + 1) * u->cap > c->Kc) return HT_ERR_CAPACITY;
    HtView stg = view_ws(c, c->stage, c->stage_rank);
    // u* = T(u + dt L u) into the stage area
    int st = launch_apply(c, op, uv, uv, app, u->cap, s);
    if (st != HT_OK) return st;
    st = run_truncate(c, app, c->Kc, stg, rel_tol, rmax, nullptr, 0, nullptr, s);
    if (st != HT_OK) return st;
    // u <- T(u/2 + (u* + dt L u*)/2): blocks [u | u* | A^q u*]
    ApplyOp op2;
    memset(&op2, 0, sizeof(op2));
    op2.mode = HT_APPLY_EULER;
    op2.nb = op.nb + 1;
    op2.src[0] = 0;
    op2.coef[0] = 0.5;
    for (int i = 0; i < c->cfg.d; ++i) op2.f[0][i] = op.f[0][i];   // identity
    for (int b = 0; b < op.nb; ++b) {
      op2.src[b + 1] = 1;
      op2.coef[b + 1] = 0.5 * op.coef[b];
      for (int i = 0; i < c->cfg.d; ++i) op2.f[b + 1][i] = op.f[b][i];
    }
    st = launch_apply(c, op2, uv, stg, app, u->cap, s);
    if (st != HT_OK) return st;
    return run_truncate(c, app, c->Kc, uv, rel_tol, rmax, nullptr, 0, nullptr, s);
  }
  return HT_ERR_ARG;
}

extern "C" int ht_step_ab2(ht_ctx* c, ht_tensor* u, ht_tensor* u_prev, const ht_op* L, double dt, double rel_tol,
                           int rmax, void* stream) {
  if (!c || !tensor_matches(c, u) || !tensor_matches(c, u_prev) || u->cap != u_prev->cap) return HT_ERR_ARG;
  for (int t = 0; t < c->tree.nn; ++t)
    if (u->node[t] == u_prev->node[t]) return HT_ERR_ARG;
  if (u->rank == u_prev->rank) return HT_ERR_ARG;
  if (rmax < 1 || rmax > u->cap || !(rel_tol >= 0.0)) return HT_ERR_ARG;
  if (u->cap > c->cap || 4LL * u->cap > c->Kc) return HT_ERR_CAPACITY;
  ApplyOp op;
  if (!build_apply(c, L, dt, HT_APPLY_RK2POLY, &op)) return HT_ERR_ARG;   // the factors dt L_i
  // (1 + 3/2 S) u + (-1/2 S) u_prev, S = dt L (eq. AB2_)
  op.npoly = 2;
  op.deg[0] = op.deg[1] = 1;
  op.pc[0][0] = 1.0;
  op.pc[0][1] = 1.5;
  op.pc[1][0] = 0.0;
  op.pc[1][1] = -0.5;
  op.pc[0][2] = op.pc[1][2] = 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  HtView uv = view_of(u);
  HtView app = view_ws(c, c->app, c->app_rank);
  int st = launch_apply(c, op, uv, view_of(u_prev), app, u->cap, s);
  if (st != HT_OK) return st;
  st = copy_tensor_to(c, u, u_prev->node, u_prev->rank, s);   // u_prev <- u (u is read no more)
  if (st != HT_OK) return st;
  return run_truncate(c, app, c->Kc, uv, rel_tol, rmax, nullptr, 0, nullptr, s);
}

// block-diagonal sum a * in0 + b * in1 (identity factors, root coefficients a, b)
static void sum_op(const ht_ctx* c, double a, double b, ApplyOp* op) {
  memset(op, 0, sizeof(*op));
  op->mode = HT_APPLY_L;
  op->nb = 2;
  op->src[0] = 0;
  op->src[1] = 1;
  op->coef[0] = a;
  op->coef[1] = b;
  for (int blk = 0; blk < 2; ++blk)
    for (int i = 0; i < c->cfg.d; ++i) {
      op->f[blk][i].kind = HT_F_STENCIL;   // identity: a width-0 stencil
      op->f[blk][i].hw = 0;
      op->f[blk][i].c[0] = 1.0;
    }
}

extern "C" int ht_add(ht_ctx* c, double a, const ht_tensor* u, double b, const ht_tensor* w, ht_tensor* out,
                      void* stream) {
  if (!c || !tensor_matches(c, u) || !tensor_matches(c, w) || !tensor_matches(c, out)) return HT_ERR_ARG;
  for (int t = 0; t < c->tree.nn; ++t)
    if (out->node[t] == u->node[t] || out->node[t] == w->node[t]) return HT_ERR_ARG;
  if (out->rank == u->rank || out->rank == w->rank) return HT_ERR_ARG;
  if ((long long)u->cap + w->cap > out->cap) return HT_ERR_CAPACITY;
  ApplyOp op;
  sum_op(c, a, b, &op);
  return launch_apply(c, op, view_of(u), view_of(w), view_of(out), htg_max(u->cap, w->cap), (cudaStream_t)stream);
}

extern "C" int ht_step_ab2_split(ht_ctx* c, ht_tensor* u, ht_tensor* u_prev, const ht_op* L, double dt,
                                 double rel_tol, int rmax, int variant, void* stream) {
  if (!c || !tensor_matches(c, u) || !tensor_matches(c, u_prev) || u->cap != u_prev->cap) return HT_ERR_ARG;
  for (int t = 0; t < c->tree.nn; ++t)
    if (u->node[t] == u_prev->node[t]) return HT_ERR_ARG;
  if (u->rank == u_prev->rank) return HT_ERR_ARG;
  if (rmax < 1 || rmax > u->cap || !(rel_tol >= 0.0)) return HT_ERR_ARG;
  if (variant != HT_AB2_SPLIT_ARGUMENT && variant != HT_AB2_SPLIT_DIFFERENCE) return HT_ERR_ARG;
  if (u->cap > c->cap || 3LL * u->cap > c->Kc) return HT_ERR_CAPACITY;
  ApplyOp opS;   // S x = dt L x exactly: the blocks [X, S X] with root coefficients (0, 1)
  if (!build_apply(c, L, dt, HT_APPLY_RK2POLY, &opS)) return HT_ERR_ARG;
  opS.npoly = 1;
  opS.deg[0] = 1;
  opS.pc[0][0] = 0.0;
  opS.pc[0][1] = 1.0;
  opS.pc[0][2] = 0.0;
  cudaStream_t s = (cudaStream_t)stream;
  const HtView uv = view_of(u), pv = view_of(u_prev);
  const HtView app = view_ws(c, c->app, c->app_rank), stg = view_ws(c, c->stage, c->stage_rank);
  const int cap = u->cap, Kc = c->Kc;
  ApplyOp opA;
  int st;
#define HTG_TRY(x) do { st = (x); if (st != HT_OK) return st; } while (0)
  if (variant == HT_AB2_SPLIT_ARGUMENT) {
    // w = T(3u - u_prev) -> stage;  v = T(S w) -> u_prev;  u <- T(u + v/2), u_prev <- u
    sum_op(c, 3.0, -1.0, &opA);
    HTG_TRY(launch_apply(c, opA, uv, pv, app, cap, s));
    HTG_TRY(run_truncate(c, app, Kc, stg, rel_tol, rmax, nullptr, 0, nullptr, s));
    HTG_TRY(launch_apply(c, opS, stg, stg, app, cap, s));
    HTG_TRY(run_truncate(c, app, Kc, pv, rel_tol, rmax, nullptr, 0, nullptr, s));
    sum_op(c, 1.0, 0.5, &opA);
    HTG_TRY(launch_apply(c, opA, uv, pv, app, cap, s));
  } else {
    // w = T(u - u_prev) -> u_prev;  a = T(S u) -> stage;  b = T(S w) -> u_prev;
    // u <- T(u + (a + b/2)), u_prev <- u
    sum_op(c, 1.0, -1.0, &opA);
    HTG_TRY(launch_apply(c, opA, uv, pv, app, cap, s));
    HTG_TRY(run_truncate(c, app, Kc, pv, rel_tol, rmax, nullptr, 0, nullptr, s));
    HTG_TRY(launch_apply(c, opS, uv, uv, app, cap, s));
    HTG_TRY(run_truncate(c, app, Kc, stg, rel_tol, rmax, nullptr, 0, nullptr, s));
    HTG_TRY(launch_apply(c, opS, pv, pv, app, cap, s));
    HTG_TRY(run_truncate(c, app, Kc, pv, rel_tol, rmax, nullptr, 0, nullptr, s));
    sum_op(c, 1.0, 0.5, &opA);
    HTG_TRY(launch_apply(c, opA, stg, pv, app, cap, s));      // a + b/2 (ranks <= 2 rmax)
    sum_op(c, 1.0, 1.0, &opA);
    HTG_TRY(launch_apply(c, opA, uv, app, stg, 2 * cap, s));  // u + (a + b/2) (ranks <= 3 rmax)
  }
  HTG_TRY(copy_tensor_to(c, u, u_prev->node, u_prev->rank, s));   // u_prev <- u
  const HtView& fin = (variant == HT_AB2_SPLIT_ARGUMENT) ? app : stg;
  HTG_TRY(run_truncate(c, fin, Kc, uv, rel_tol, rmax, nullptr, 0, nullptr, s));
#undef HTG_TRY
  return HT_OK;
}

// ---------------------------------------------------------------- batches -----
struct ht_batch {
  int count = 0;
  std::vector<ht_ctx*> ctx;
  std::vector<Plan*> own_plan;     // each context's own plan, restored by ht_batch_destroy
  void* mem = nullptr;             // device: plans | instances | operators (2 per instance)
  Plan* plans = nullptr;
  Inst* inst = nullptr;
  ApplyOp* ops = nullptr;
  void* host = nullptr;            // pinned staging of instances and operators
  Inst* inst_h = nullptr;
  ApplyOp* ops_h = nullptr;
  cudaEvent_t up_done = nullptr;   // the last upload from the staging buffers
  bool uploaded = false;
  std::vector<Inst> inst_new;
  std::vector<ApplyOp> ops_new;
  std::vector<int> ucap;           // rank capacity of each bound tensor
  int Kc = 0, nmax = 1, max_cols = 1;
};

static void batch_free(ht_batch* b) {
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (i < b->own_plan.size() && b->own_plan[i]) b->ctx[i]->plan = b->own_plan[i];
    b->ctx[i]->batch = nullptr;
  }
  if (b->up_done) cudaEventDestroy(b->up_done);
  if (b->host) cudaFreeHost(b->host);
  if (b->mem) cudaFree(b->mem);
  delete b;
}

extern "C" int ht_batch_create(ht_batch** out, int count, ht_ctx* const* ctxs, ht_tensor* const* us) {
  if (!out) return HT_ERR_ARG;
  *out = nullptr;
  if (count < 1 || count > 65535 || !ctxs || !us) return HT_ERR_ARG;
  const int d = ctxs[0] ? ctxs[0]->cfg.d : 0;
  const int dev = ctxs[0] ? ctxs[0]->cfg.device : 0;
  const int tree = ctxs[0] ? ctxs[0]->cfg.tree : 0;
  for (int i = 0; i < count; ++i) {
    ht_ctx* c = ctxs[i];
    if (!c || c->cfg.d != d || c->cfg.device != dev || c->cfg.tree != tree || c->batch || !tensor_matches(c, us[i]))
      return HT_ERR_ARG;
    if (c->slices != ctxs[0]->slices) return HT_ERR_ARG;   // one precision form per batch
    if (us[i]->cap > c->cap) return HT_ERR_CAPACITY;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return HT_ERR_ARG;   // each instance needs its own workspace
  }
  if (cudaSetDevice(dev) != cudaSuccess) return HT_ERR_CUDA;
  ht_batch* b = new ht_batch();
  b->count = count;
  const size_t plan_b = align_up((size_t)count * sizeof(Plan));
  const size_t inst_b = align_up((size_t)count * sizeof(Inst));
  const size_t ops_b = align_up(2 * (size_t)count * sizeof(ApplyOp));
  if (cudaMalloc(&b->mem, plan_b + inst_b + ops_b) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return HT_ERR_NOMEM;
  }
  char* base = (char*)b->mem;
  b->plans = (Plan*)base;
  b->inst = (Inst*)(base + plan_b);
  b->ops = (ApplyOp*)(base + plan_b + inst_b);
  if (cudaMallocHost(&b->host, inst_b + ops_b) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(b->mem);
    delete b;
    return HT_ERR_NOMEM;
  }
  b->inst_h = (Inst*)b->host;
  b->ops_h = (ApplyOp*)((char*)b->host + inst_b);
  if (cudaEventCreateWithFlags(&b->up_done, cudaEventDisableTiming) != cudaSuccess) {
    b->up_done = nullptr;
    batch_free(b);
    return HT_ERR_CUDA;
  }
  b->inst_new.resize(count);
  b->ops_new.resize(2 * (size_t)count);
  for (int i = 0; i < count; ++i) {
    ht_ctx* c = ctxs[i];
    b->ctx.push_back(c);
    b->own_plan.push_back(c->plan);
    c->plan = b->plans + i;
    c->batch = b;
    Inst& x = b->inst_new[i];
    memset(&x, 0, sizeof(x));
    x.P = b->plans + i;
    x.wn = c->wn_dev;
    x.view[VIEW_U] = view_of(us[i]);
    x.view[VIEW_APP] = view_ws(c, c->app, c->app_rank);
    x.view[VIEW_STAGE] = view_ws(c, c->stage, c->stage_rank);
    x.op[0] = b->ops + 2 * i;
    x.op[1] = b->ops + 2 * i + 1;
    x.err = c->err;
    x.cap_in = c->Kc;
    b->Kc = htg_max(b->Kc, c->Kc);
    b->ucap.push_back(us[i]->cap);
    b->max_cols = htg_max(b->max_cols, us[i]->cap);
    for (int k = 0; k < d; ++k) b->nmax = htg_max(b->nmax, c->cfg.n[k]);
  }
  *out = b;
  return HT_OK;
}

extern "C" void ht_batch_destroy(ht_batch* b) {
  if (!b) return;
  if (!b->ctx.empty()) cudaSetDevice(b->ctx[0]->cfg.device);
  batch_free(b);
}

extern "C" int ht_batch_step(ht_batch* b, const ht_op* const* Ls, const double* dts, const double* rel_tols,
                             const int* rmaxs, int scheme, void* stream) {
  if (!b || !Ls || !dts || !rel_tols || !rmaxs) return HT_ERR_ARG;
  if (scheme != HT_SCHEME_RK2POLY && scheme != HT_SCHEME_HEUN2) return HT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int cnt = b->count;
  // operators and scalars of this call
  for (int i = 0; i < cnt; ++i) {
    ht_ctx* c = b->ctx[i];
    Inst& x = b->inst_new[i];
    const int ucap = b->ucap[i];
    if (rmaxs[i] < 1 || rmaxs[i] > ucap || !(rel_tols[i] >= 0.0)) return HT_ERR_ARG;
    x.rmax = rmaxs[i];
    x.rel_tol = rel_tols[i];
    ApplyOp& op = b->ops_new[2 * i];
    ApplyOp& op2 = b->ops_new[2 * i + 1];
    memset(&op2, 0, sizeof(op2));
    if (scheme == HT_SCHEME_RK2POLY) {
      if (!build_apply(c, Ls[i], dts[i], HT_APPLY_RK2POLY, &op)) return HT_ERR_ARG;
    } else {
      if (!build_apply(c, Ls[i], dts[i], HT_APPLY_EULER, &op)) return HT_ERR_ARG;
      if ((long long)(op.nb + 1) * ucap > c->Kc) return HT_ERR_CAPACITY;
      // second stage blocks [u | u* | A^q u*], as in ht_step
      op2.mode = HT_APPLY_EULER;
      op2.nb = op.nb + 1;
      op2.src[0] = 0;
      op2.coef[0] = 0.5;
      for (int k = 0; k < c->cfg.d; ++k) op2.f[0][k] = op.f[0][k];
      for (int q = 0; q < op.nb; ++q) {
        op2.src[q + 1] = 1;
        op2.coef[q + 1] = 0.5 * op.coef[q];
        for (int k = 0; k < c->cfg.d; ++k) op2.f[q + 1][k] = op.f[q][k];
      }
    }
  }
  const size_t ib = (size_t)cnt * sizeof(Inst), ob = 2 * (size_t)cnt * sizeof(ApplyOp);
  const bool same = b->uploaded && memcmp(b->inst_h, b->inst_new.data(), ib) == 0 &&
                    memcmp(b->ops_h, b->ops_new.data(), ob) == 0;
  if (!same) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return HT_ERR_CUDA;
    if (cs != cudaStreamCaptureStatusNone) return HT_ERR_ARG;
    // the staging buffers are rewritten only after the previous upload has run
    if (cudaEventSynchronize(b->up_done) != cudaSuccess) return HT_ERR_CUDA;
    memcpy(b->inst_h, b->inst_new.data(), ib);
    memcpy(b->ops_h, b->ops_new.data(), ob);
    if (cudaMemcpyAsync(b->inst, b->inst_h, ib, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b->ops, b->ops_h, ob, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(b->up_done, s) != cudaSuccess)
      return HT_ERR_CUDA;
    b->uploaded = true;
  }
  ht_ctx* c0 = b->ctx[0];
  const TreeInfo& T = c0->tree;
  const Levels& L = c0->lev;
  const Inst* I = b->inst;
  const size_t smem = 2 * (size_t)b->nmax * sizeof(double);
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(apply_leaf_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return HT_ERR_CUDA;
  const dim3 gl(htg_max(1, htg_min(b->max_cols, 64)), L.n_leaf, cnt);
  const dim3 gx(htg_max(1, c0->gemm_grid / cnt), L.n_proj2, cnt);
  auto apply = [&](int op_sel, int in0, int in1, int outv) -> int {
    HTG_LAUNCH(c0, KC_APPLY, s, (apply_leaf_batch_kernel<<<gl, 128, smem, s>>>(I, T, L, op_sel, in0, in1, outv),
                                 cudaGetLastError()));
    HTG_LAUNCH(c0, KC_APPLY, s, (apply_xfer_batch_kernel<<<gx, 256, 0, s>>>(I, T, L, op_sel, in0, in1, outv),
                                 cudaGetLastError()));
    return HT_OK;
  };
  auto truncate = [&](int inv, int outv) -> int {
    auto pre = [&]() {
      plan_pre_batch_kernel<<<cnt, 1, 0, s>>>(I, T, L, inv);
      return cudaGetLastError();
    };
    auto sel = [&]() {
      rank_select_batch_kernel<<<cnt, 32, 0, s>>>(I, T, L, inv, outv);
      return cudaGetLastError();
    };
    return truncate_launches(c0, b->plans, cnt, b->Kc, c0->svd_smem, pre, sel, s);
  };
  int st;
  if (scheme == HT_SCHEME_RK2POLY) {
    if ((st = apply(0, VIEW_U, VIEW_U, VIEW_APP)) != HT_OK) return st;
    return truncate(VIEW_APP, VIEW_U);
  }
  if ((st = apply(0, VIEW_U, VIEW_U, VIEW_APP)) != HT_OK) return st;
  if ((st = truncate(VIEW_APP, VIEW_STAGE)) != HT_OK) return st;
  if ((st = apply(1, VIEW_U, VIEW_STAGE, VIEW_APP)) != HT_OK) return st;
  return truncate(VIEW_APP, VIEW_U);
}

// ---------------------------------------------------------------- misc --------
extern "C" int ht_from_cp(ht_ctx* c, const cp_tensor* x, ht_tensor* out, void* stream) {
  if (!c || !x || !tensor_matches(c, out) || x->d != c->cfg.d || x->rank < 1 || !x->weight) return HT_ERR_ARG;
  if (x->rank > out->cap) return HT_ERR_CAPACITY;
  for (int i = 0; i < x->d; ++i)
    if (x->n[i] != c->cfg.n[i] || !x->factor[i]) return HT_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const double* fp[HT_MAXD];
  for (int i = 0; i < HT_MAXD; ++i) fp[i] = (i < x->d) ? x->factor[i] : nullptr;
  const double** tbl = c->ptr_tbl;
  if (cudaMemcpyAsync((void*)tbl, fp, sizeof(fp), cudaMemcpyHostToDevice, s) != cudaSuccess) return HT_ERR_CUDA;
  dim3 g(64, c->tree.nn);
  HTG_LAUNCH(c, KC_APPLY, s, (from_cp_kernel<<<g, 256, 0, s>>>(c->tree, view_of(out), tbl, x->weight, x->rank),
                       cudaGetLastError()));
  c->last_stream = s;
  return HT_OK;
}

static int run_inner(ht_ctx* c, const ht_tensor* u, const ht_tensor* w, double* out_dev, cudaStream_t s) {
  // Grams per node in the workspace's per-node E buffers (Kc x Kc), temp in T1 of the root
  double* gbuf = c->wn[0].Epre;   // nn * Kc^2 fits in Kc^3 for Kc >= 2d - 1
  const long long gstride = (long long)c->Kc * c->Kc;
  if ((long long)c->tree.nn * gstride > (long long)c->Kc * c->Kc * c->Kc) return HT_ERR_CAPACITY;
  HtView uw = view_of(u);
  HtView ww = w ? view_of(w) : uw;
  HTG_LAUNCH(c, KC_PLAN, s, (inner_kernel<<<1, 256, 0, s>>>(c->tree, uw, ww, w ? 0 : 1, gbuf, gstride, c->wn[0].T1, out_dev),
                       cudaGetLastError()));
  c->last_stream = s;
  return HT_OK;
}

extern "C" int ht_mass(ht_ctx* c, const ht_tensor* u, double* out_dev, void* stream) {
  if (!c || !tensor_matches(c, u) || !out_dev) return HT_ERR_ARG;
  if (u->cap > c->Kc) return HT_ERR_CAPACITY;
  return run_inner(c, u, nullptr, out_dev, (cudaStream_t)stream);
}

extern "C" int ht_inner(ht_ctx* c, const ht_tensor* u, const ht_tensor* w, double* out_dev, void* stream) {
  if (!c || !tensor_matches(c, u) || !tensor_matches(c, w) || !out_dev) return HT_ERR_ARG;
  if (u->cap > c->Kc || w->cap > c->Kc) return HT_ERR_CAPACITY;
  return run_inner(c, u, w, out_dev, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- accessors -----
CpWs* htg_ctx_cp(ht_ctx* c) { return &c->cp; }
int htg_ctx_d(const ht_ctx* c) { return c->cfg.d; }
const int* htg_ctx_n(const ht_ctx* c) { return c->cfg.n; }
int* htg_ctx_err(ht_ctx* c) { return c->err; }
int htg_ctx_grid(const ht_ctx* c) { return c->gemm_grid; }
int htg_ctx_cp_form(const ht_ctx* c) { return c->cfg.cp_form; }
const CpClusterCfg* htg_ctx_cp_cluster(const ht_ctx* c) { return &c->cp_clu; }
int htg_ctx_cap(const ht_ctx* c) { return c->cfg.cap; }
int htg_ctx_max_terms(const ht_ctx* c) { return c->cfg.max_terms; }
int htg_ctx_device(const ht_ctx* c) { return c->cfg.device; }
void** htg_ctx_cn_ws(ht_ctx* c, size_t** bytes) {
  *bytes = &c->cn_bytes;
  return &c->cn_ws;
}
void htg_ctx_count(ht_ctx* c, int launches, cudaStream_t s) {
  c->launches += launches;
  c->last_stream = s;
}
int htg_cp_terms(int d) { return 1 + 2 * d + d * (d - 1) / 2; }

// ---------------------------------------------------------------- profiler ------
void htg_prof_begin(ht_ctx* c, cudaStream_t s) {
  if (!c || !c->prof_on) return;
  if (c->prof_pool.size() < 2 * (c->prof_n + 1)) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { c->prof_on = false; return; }
      c->prof_pool.push_back(e);
    }
  }
  cudaEventRecord(c->prof_pool[2 * c->prof_n], s);
}

void htg_prof_end(ht_ctx* c, int cls, cudaStream_t s) {
  if (!c || !c->prof_on) return;
  cudaEventRecord(c->prof_pool[2 * c->prof_n + 1], s);
  if (c->prof_cls.size() <= c->prof_n) c->prof_cls.push_back(cls);
  else c->prof_cls[c->prof_n] = cls;
  c->prof_n++;
}

double* htg_prof_flops(ht_ctx* c, int cls) {
  return (c && c->prof_on && cls >= 0 && cls < KC_COUNT) ? c->prof_flops + cls : nullptr;
}

extern "C" int ht_ctx_profile(ht_ctx* c, int on) {
  if (!c) return HT_ERR_ARG;
  if (cudaSetDevice(c->cfg.device) != cudaSuccess) return HT_ERR_CUDA;
  if (on) {
    if (cudaMemset(c->prof_flops, 0, KC_COUNT * sizeof(double)) != cudaSuccess) return HT_ERR_CUDA;
    c->prof_n = 0;
  }
  c->prof_on = on != 0;
  return HT_OK;
}

extern "C" int ht_ctx_profile_read(ht_ctx* c, double* ms, long long* launches, double* flops) {
  if (!c) return HT_ERR_ARG;
  double tms[KC_COUNT] = {0};
  long long cnt[KC_COUNT] = {0};
  for (size_t i = 0; i < c->prof_n; ++i) {
    if (cudaEventSynchronize(c->prof_pool[2 * i + 1]) != cudaSuccess) return HT_ERR_CUDA;
    float e = 0.f;
    if (cudaEventElapsedTime(&e, c->prof_pool[2 * i], c->prof_pool[2 * i + 1]) != cudaSuccess) return HT_ERR_CUDA;
    tms[c->prof_cls[i]] += e;
    cnt[c->prof_cls[i]] += 1;
  }
  double fl[KC_COUNT] = {0};
  if (cudaMemcpy(fl, c->prof_flops, sizeof(fl), cudaMemcpyDeviceToHost) != cudaSuccess) return HT_ERR_CUDA;
  for (int k = 0; k < KC_COUNT; ++k) {
    if (ms) ms[k] = tms[k];
    if (launches) launches[k] = cnt[k];
    if (flops) flops[k] = fl[k];
  }
  return HT_OK;
}
