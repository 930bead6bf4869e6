/*
 * htgpu.h -- C ABI of the GB300 (sm_103a) library for explicit time steps of
 * d-dimensional linear PDEs u_t = L u whose solution is held in hierarchical Tucker
 * (HT) format on a balanced binary dimension tree, or in canonical (CP) format.
 *
 * Method (arXiv:1803.10270):
 *  - HT format, Section 2.2, eqs. HTD / coreT: leaf bases U_i (n_i x k) and transfer
 *    tensors B_t (k_t1 x k_t2 x k_t), root B (k_t1 x k_t2).
 *  - Separable operator, Section 3, eq. Lz: L = sum_q alpha_q L_1^q ... L_d^q.
 *  - Explicit stepping with rank reduction, Section 3.2 (eq. AB2_ and the text after
 *    it): the step needs operator application, addition and rank reduction by the
 *    hierarchical SVD (HT) or by alternating least squares (CP).
 *  - CP format and ALS, Section 2.1, eqs. functional-SSE, als, SSYSTEM, A^{ln}_{jhp}.
 *
 * Conventions shared by every entry point
 *  - All array arguments named "device" are device pointers owned by the caller.
 *    The library owns only the workspace inside an ht_ctx.
 *  - Every call is asynchronous on the given CUDA stream (cudaStream_t passed as
 *    void*; NULL = legacy default stream) and never synchronises the host, so a
 *    sequence of calls can be captured in a CUDA graph.  Ranks stay in device memory.
 *  - Floating-point data are FP64 in memory in every precision mode.
 *  - Return value: HT_OK (0) or a negative ht_status.  Argument errors are detected on
 *    the host before anything is launched.  Numerical problems found on the device
 *    (non-finite values, a bounded wait that gave up) set a device error word that
 *    ht_ctx_check() reads (synchronising) and clears.
 *
 * Tree and node numbering
 *  HT_TREE_BALANCED: the dimension range [a, b) of a node splits at a + floor((b-a)/2); for
 *  d = 6 this is {1,2,3}|{4,5,6}, then {1}|{2,3} and {4}|{5,6} (Section 2.2, eq. HTD).
 *  HT_TREE_LINEAR: [a, b) splits at a + 1 ({a} | [a+1, b)), the degenerate tree of the
 *  tensor-train format (Section 2.2 names TT as the special case of HT on such a tree): the
 *  interior node [i, d) holds the TT core of dimension i, contracted with leaf i.  Nodes are
 *  numbered breadth first from the root (node 0); 2d-1 nodes, d leaves.  ht_tree_info()
 *  returns the numbering.  A tensor's buffers follow the tree of the context it is used with.
 *
 * Storage of an HT tensor (packed with the CURRENT ranks, first index fastest)
 *  leaf t of dimension i:  U[j + n_i * a],             0 <= a < k_t
 *  interior t (t1, t2):    B[a + k_t1 * (b + k_t2 * c)]
 *  root (t1, t2):          B[a + k_t1 * b]
 *  Buffers are sized for the capacity cap: n_i*cap, cap^3 and cap^2 doubles.
 */
#ifndef HTGPU_H
#define HTGPU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HT_MAXD 16
#define HT_MAXNODES (2 * HT_MAXD - 1)
#define HT_MAXTERMS 16   /* a Kronecker-sum operator has one term per dimension */
#define HT_MAXBLOCKTERMS 10  /* terms of a general (block-diagonal) application (the 3-D
                                variable-coefficient advection operator has 9) */
#define HT_MAXSTENCIL 9

typedef enum ht_status {
  HT_OK = 0,
  HT_ERR_ARG = -1,        /* bad argument: d, n, ranks, pointers, modes */
  HT_ERR_CAPACITY = -2,   /* a result rank could exceed a buffer or workspace capacity */
  HT_ERR_CUDA = -3,       /* a CUDA runtime call failed */
  HT_ERR_NONFINITE = -4,  /* NaN/Inf met on the device (reported by ht_ctx_check) */
  HT_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up (reported by ht_ctx_check) */
  HT_ERR_NOMEM = -6       /* workspace allocation failed */
} ht_status;

typedef enum ht_precision {
  HT_PREC_FP64 = 0,   /* every operation in FP64 */
  HT_PREC_MIXED = 1   /* the dense contractions of the HSVD truncation (transfer-tensor absorption,
                         the complement / square-root factors, the node factors P_t = R_t E_t, the
                         projections) run on the tensor cores: each FP64 operand row / column is
                         split into ht_config.mixed_slices BF16 digit planes, accumulated in FP32
                         (tcgen05, tensor memory), normwise error about 2^-(8 slices - 1); those
                         below ht_config.tc_min_work multiply-adds in a split-FP32 form on the CUDA
                         cores (FP32 hi / lo operand parts, the compensated dot product of Ogita,
                         Rump and Oishi: error at most about (k^2 + 5k + 10) 2^-47, in practice
                         about (k/2 + 10) 2^-47, of the sum of |products|); the QR
                         R factors, node SVDs, truncation thresholds, the X_t Y_t = I refinement
                         of the kept subspaces, the apply and the CP route stay FP64 */
} ht_precision;

/* ---------------------------------------------------------------- tensors ---- */
typedef struct ht_tensor {
  int d;                          /* number of dimensions, 2 <= d <= HT_MAXD */
  int n[HT_MAXD];                 /* grid points per dimension, 1 <= n_i */
  int cap;                        /* rank capacity of every non-root node */
  double* node[HT_MAXNODES];      /* device buffers per node (see storage above) */
  int* rank;                      /* device, HT_MAXNODES ints; rank[0] = 1 */
} ht_tensor;

typedef struct cp_tensor {
  int d;                          /* number of dimensions */
  int n[HT_MAXD];                 /* grid points per dimension */
  int rank;                       /* current rank r (host value) */
  int cap;                        /* column capacity of every factor buffer */
  double* factor[HT_MAXD];        /* device, n_k x cap column-major, first r columns used */
  double* weight;                 /* device, cap values lambda_l */
} cp_tensor;

/* ------------------------------------------------------------- operators ---- */
typedef enum ht_factor_kind {
  HT_F_IDENTITY = 0,   /* identity */
  HT_F_STENCIL = 1,    /* periodic constant band: (A u)_j = sum_{s=-w}^{w} c_{s+w} u_{j+s mod n} */
  HT_F_DIAG = 2,       /* (A u)_j = v_j u_j, v a device vector of n values */
  HT_F_RANK1 = 3,      /* (A u)_j = m_j sum_l w_l u_l, m and w device vectors of n values */
  HT_F_DIAG_STENCIL = 4   /* (A u)_j = v_j sum_{s=-w}^{w} c_{s+w} u_{j+s mod n}: a diagonal times a
                             periodic band, e.g. z_k d/dz_k of the variable-coefficient advection
                             operator (Section 4.1, Table tab:ordering0); v a device vector */
} ht_factor_kind;

typedef struct ht_factor {
  int kind;                        /* ht_factor_kind */
  int half_width;                  /* STENCIL, DIAG_STENCIL: w, 0 <= w <= (HT_MAXSTENCIL-1)/2 */
  double stencil[HT_MAXSTENCIL];   /* STENCIL, DIAG_STENCIL: 2w+1 coefficients (host values) */
  const double* v;                 /* DIAG, DIAG_STENCIL: device values; RANK1: device m */
  const double* w;                 /* RANK1: device w */
} ht_factor;

/* Separable operator L = sum_q alpha_q A_1^q x ... x A_d^q  (eq. Lz).
 * kron_sum = 1 declares that term q acts on dimension q only (n_terms = d,
 * f[q][i] = identity for i != q), i.e. L = sum_i L_i; this enables the exact
 * rank-3k form of the RK2 polynomial p(dt L) = 1 + dt L + dt^2 L^2 / 2. */
typedef struct ht_op {
  int d;
  int n_terms;                             /* 1 <= n_terms <= HT_MAXTERMS; the general (block-
                                              diagonal) forms take at most HT_MAXBLOCKTERMS */
  int kron_sum;
  double alpha[HT_MAXTERMS];
  ht_factor f[HT_MAXTERMS][HT_MAXD];
} ht_op;

/* ---------------------------------------------------------------- context --- */
typedef struct ht_ctx ht_ctx;

typedef enum ht_tree_kind {
  HT_TREE_BALANCED = 0,    /* balanced binary dimension tree (eq. HTD) */
  HT_TREE_LINEAR = 1       /* {a} | [a+1, b) at every node: the tensor-train tree */
} ht_tree_kind;

typedef struct ht_config {
  int d;                   /* dimensions of the tensors this context serves */
  int n[HT_MAXD];          /* grid points per dimension */
  int cap;                 /* largest input rank capacity */
  int max_terms;           /* largest operator term count used with ht_step/ht_apply */
  int precision;           /* ht_precision */
  int device;              /* CUDA device ordinal */
  int tree;                /* ht_tree_kind */
  int mixed_slices;        /* HT_PREC_MIXED: BF16 digit planes per contraction operand, 2..4 (0 = 4);
                              ignored in HT_PREC_FP64 */
  /* Tuning (0 = the library default; the package's autotuner measures them per GPU): */
  long long tc_min_work;   /* HT_PREC_MIXED: contractions of at least this many multiply-adds
                              (m n k batch, decided on the device per contraction) run on the tensor
                              cores, smaller ones in the split-FP32 form on the CUDA cores; a list of
                              contractions that cannot reach it at the context's capacities makes no
                              tensor-core launch; -1: all on the tensor cores */
  int gemm_ctas_per_sm;    /* CTAs per SM of the CUDA-core contraction launches (FP64 or split-FP32),
                              1..32 (default 16, or 8 for truncation inputs below rank 96) */
  int svd_cluster_min_cols;/* node factors at least this wide use the thread-block-cluster SVD,
                              32..480 (default 128) */
  int cp_form;             /* cp_als_sweep_rk2 (Gauss-Seidel): 0 = one thread-block cluster of up to
                              16 CTAs whenever the problem fits its shared memory (ranks <= 64), else
                              the cooperative grid form; 1 = always the cooperative grid form */
  int biorth_form;         /* the refinement X_t Y_t = I of the projections (two Newton steps, four
                              products of 2 k^2 K flops per node): 0 = one CTA per node; 1 = one
                              thread-block cluster of 16 (else 8) CTAs per node in contexts whose
                              truncation inputs reach rank 160 (one CTA per node below that).  Both
                              forms sum every element in the same order: the results agree bit for
                              bit.  Measured on GB300: the cluster form takes the rank-192 wide-factor
                              truncation from 93 to 86 ms, but the kinetic HEUN2 step (rank 64,
                              5 terms) from 105.9 to 106.9 ms, so it is not the default */
} ht_config;

/* Context management, status codes, the profiler and the tree query below are infrastructure
 * around the method: no passage of the paper defines them.
 *
 * Workspace bytes a context with this configuration allocates (0 on bad config). */
size_t ht_workspace_bytes(const ht_config* cfg);

/* Create a context: allocates the workspace on cfg->device with cudaMalloc.
 * *out receives the context.  Errors: HT_ERR_ARG, HT_ERR_NOMEM, HT_ERR_CUDA. */
int ht_ctx_create(ht_ctx** out, const ht_config* cfg);

/* Free the workspace and the context (NULL is accepted). */
void ht_ctx_destroy(ht_ctx* ctx);

/* Synchronise the context's last stream, read and clear the device error word.
 * Returns HT_OK, HT_ERR_NONFINITE or HT_ERR_TIMEOUT. */
int ht_ctx_check(ht_ctx* ctx, void* stream);

/* Number of kernel launches the context issued since creation (host counter). */
long long ht_ctx_launches(const ht_ctx* ctx);

/* CTAs per node of the cluster form of the X_t Y_t = I refinement on this context (16 or 8),
 * or 0 when it runs one CTA per node (ht_config.biorth_form = 0, truncation inputs below rank
 * 160, or no cluster placeable on the device; batched steps always take one CTA per node and
 * instance).  Errors: HT_ERR_ARG. */
int ht_biorth_cluster_ctas(const ht_ctx* ctx, int* ctas);

/* Opt-in event profiler (off by default).  on = 1 clears the accumulators and starts
 * recording a CUDA event pair on the launching stream around every kernel launch of the
 * context; the FP64-bound kernels also add the FP64 flops they execute to a device
 * counter per kernel class.  on = 0 stops recording.  Not for use inside stream capture. */
int ht_ctx_profile(ht_ctx* ctx, int on);

/* Per kernel class (8 classes: apply, gemm, qr, svd, plan/rank, cp small kernels,
 * cp solve, tensor-core gemm) the summed event time in ms, the launch count and the counted
 * flops (FP64 flops; for the tensor-core class the executed BF16 MMA flops).
 * Synchronises on the recorded events.  Any output pointer may be NULL. */
int ht_ctx_profile_read(ht_ctx* ctx, double* ms, long long* launches, double* flops);

/* Human-readable name of a status code. */
const char* ht_status_string(int status);

/* Node numbering of the dimension tree for d dimensions (Section 2.2, eq. HTD): kind
 * HT_TREE_BALANCED, or HT_TREE_LINEAR for the tensor-train format.  Each output array holds
 * 2d-1 ints: lo/hi = dimension range [lo, hi), c1/c2 = children (-1 for leaves),
 * parent (-1 for the root), depth.  Returns HT_ERR_ARG for d outside [2, HT_MAXD] or an
 * unknown kind. */
int ht_tree_info(int d, int kind, int* lo, int* hi, int* c1, int* c2, int* parent, int* depth);

/* ------------------------------------------------------------- HT calls ----- */
typedef enum ht_apply_mode {
  HT_APPLY_L = 0,          /* v = L u                        rank n_terms * k */
  HT_APPLY_EULER = 1,      /* v = u + dt L u                 rank (n_terms+1) * k */
  HT_APPLY_RK2POLY = 2     /* v = (1 + dt L + dt^2 L^2 / 2) u, kron_sum operators only, rank 3k */
} ht_apply_mode;

/* Operator application (eq. Lz; Section 3.2).  The result is exact (no truncation):
 * leaves [A_i^q U_i]_q, block-structured transfer tensors.  v->cap must hold the
 * raised rank of every node (checked against u->cap on the host).  u and v must not
 * alias.  Errors: HT_ERR_ARG, HT_ERR_CAPACITY, HT_ERR_CUDA. */
int ht_apply(ht_ctx* ctx, const ht_tensor* u, const ht_op* L, double dt, int mode,
             ht_tensor* v, void* stream);

/* HSVD truncation T(u) (root-to-leaves hierarchical SVD; Section 2.2 and 3.2).
 * Rank of node t: the smallest k whose discarded singular-value energy is at most
 * (rel_tol * |u|)^2 / (2d-3), then min(k, rmax); both root children share the rank.
 * Writes T(u) into out (out->cap >= rmax; out may equal u).  sigma_dev (device,
 * HT_MAXNODES * sig_stride doubles, or NULL) receives each node's singular values
 * (descending, zero padded; sig_stride >= the node's input rank).  norm_dev (device,
 * 1 double, or NULL) receives |u|.  When sigma_dev is NULL (and in ht_step / ht_batch_step)
 * the node SVDs leave unrotated any pair of columns whose squared norms are both below
 * (rel_tol |u|)^2 / (2 p (2d-3)) (p columns in the node factor): together such columns hold at
 * most half the truncation threshold, so all of them are discarded, and the discarded energy
 * is the trace of that block, which such rotations do not change; ranks and T(u) are those of
 * the fully resolved SVDs.  Errors: HT_ERR_ARG, HT_ERR_CAPACITY, HT_ERR_CUDA. */
int ht_truncate(ht_ctx* ctx, const ht_tensor* u, double rel_tol, int rmax, ht_tensor* out,
                double* sigma_dev, int sig_stride, double* norm_dev, void* stream);

typedef enum ht_scheme {
  HT_SCHEME_RK2POLY = 0,   /* u <- T(p(dt L) u), kron_sum operators */
  HT_SCHEME_HEUN2 = 1      /* u* = T(u + dt L u); u <- T(u/2 + (u* + dt L u*)/2) */
} ht_scheme;

/* One explicit time step in place (Section 3.2).  Errors as ht_apply/ht_truncate. */
int ht_step(ht_ctx* ctx, ht_tensor* u, const ht_op* L, double dt, double rel_tol, int rmax,
            int scheme, void* stream);

/* ---------------------------------------------------------- batched steps -- */
/* Many independent instances of the explicit step (Section 3.2, one per instance), each with
 * its own context (grid sizes, rank capacity and workspace may differ) and its own tensor, all
 * with the same d and so the same dimension tree.  Every launch of a batched step covers all
 * instances: the planner, each level's QRs and contractions, the node SVDs, the rank choice and
 * the projections run once per step for the whole batch (instance = a grid dimension), so the
 * per-instance results are those of ht_step on that instance: bit for bit while a launch's
 * matrices (instances x matrices of a tree level) are fewer than the SMs; a larger batch keeps
 * every QR in one CTA where a lone step may reduce a large one in row blocks (the same R up to
 * rounding and an orthogonal factor the truncation does not see).
 *
 * ht_batch_create binds count contexts and tensors (caller-owned, distinct, same d, device, tree and
 * precision form (precision and mixed_slices);
 * us[i] must fit ctxs[i] as for ht_step).  A bound context's device plan lives in the batch
 * until ht_batch_destroy; the context may still be used alone in between, but not concurrently
 * with a batched step.  Errors: HT_ERR_ARG, HT_ERR_CAPACITY, HT_ERR_NOMEM, HT_ERR_CUDA. */
typedef struct ht_batch ht_batch;
int ht_batch_create(ht_batch** out, int count, ht_ctx* const* ctxs, ht_tensor* const* us);
void ht_batch_destroy(ht_batch* b);

/* One step of every bound instance in place: u_i <- step(u_i; Ls[i], dts[i], rel_tols[i],
 * rmaxs[i]) with the scheme of ht_step (HT_SCHEME_RK2POLY or HT_SCHEME_HEUN2).  Operators and
 * scalars are copied to the device only when they differ from the previous call's (the first
 * call always copies; the copy is ordered on the stream); a call that needs such a copy while
 * the stream is being captured returns HT_ERR_ARG, so make one call before capturing a graph.
 * Device errors of instance i are reported by ht_ctx_check(ctxs[i]).  Errors: HT_ERR_ARG,
 * HT_ERR_CAPACITY, HT_ERR_CUDA. */
int ht_batch_step(ht_batch* b, const ht_op* const* Ls, const double* dts, const double* rel_tols,
                  const int* rmaxs, int scheme, void* stream);

/* The paper's two-step explicit scheme (eq. AB2_, Section 3.2) for Kronecker-sum operators:
 * u_next = T(u + dt (3/2 L u - 1/2 L u_prev)) = T((1 + 3/2 dt L) u + (-1/2 dt L) u_prev), the sum
 * formed exactly (rank 2k + 2k_prev, block-diagonal transfers) and truncated once as in
 * ht_truncate; then u_prev <- u and u <- u_next, in place.  u and u_prev: distinct buffers
 * and rank arrays, equal capacity.  Start a run with u_prev = u_0 and u = one ht_step of u_0.
 * The context needs a truncation input of 4 cap (max_terms >= 2).  Errors as ht_step. */
int ht_step_ab2(ht_ctx* ctx, ht_tensor* u, ht_tensor* u_prev, const ht_op* L, double dt, double rel_tol,
                int rmax, void* stream);

/* Addition of HT tensors (one of the three operations an explicit step needs, Section 3.2):
 * out = a u + b w exactly, ranks adding (k_u + k_w at every node), block-diagonal transfer
 * tensors.  out->cap >= u->cap + w->cap; out must not share buffers or rank arrays with u or w.
 * Errors: HT_ERR_ARG, HT_ERR_CAPACITY, HT_ERR_CUDA. */
int ht_add(ht_ctx* ctx, double a, const ht_tensor* u, double b, const ht_tensor* w, ht_tensor* out, void* stream);

typedef enum ht_ab2_split {
  HT_AB2_SPLIT_ARGUMENT = 0,    /* w = T(3u - u_prev); v = T(dt L w); u_next = T(u + v/2) */
  HT_AB2_SPLIT_DIFFERENCE = 1   /* w = T(u - u_prev); a = T(dt L u); b = T(dt L w); u_next = T(u + a + b/2) */
} ht_ab2_split;

/* The AB2 step (eq. AB2_) evaluated as a sequence of simple tensor operations, each followed by
 * its own HSVD truncation (rel_tol, rmax), as the paragraph after eq. AB2_ (Section 3.2) proposes
 * to save memory: HT_AB2_SPLIT_ARGUMENT reduces the argument 3u - u_prev of L, then L of it;
 * HT_AB2_SPLIT_DIFFERENCE takes the passage's w = f_{n+1} - f_n literally (dt/2 L (3u - u_prev) =
 * dt L u + dt L w / 2).  Kronecker-sum operators; in place, u_prev <- u and u <- u_next, as
 * ht_step_ab2 (which forms the exact sum and truncates once).  The context needs a truncation
 * input of 3 cap.  Errors as ht_step_ab2. */
int ht_step_ab2_split(ht_ctx* ctx, ht_tensor* u, ht_tensor* u_prev, const ht_op* L, double dt, double rel_tol,
                      int rmax, int variant, void* stream);

/* Exact HT form of a CP tensor (footnote to eq. HTD: a CP tensor is the diagonal case):
 * leaves = factors, interior B = delta_abc, root = diag(weights).  out->cap >= x->rank. */
int ht_from_cp(ht_ctx* ctx, const cp_tensor* x, ht_tensor* out, void* stream);

/* Scalars: sum of all entries (discrete mass) and <u, w>, written to device doubles (the
 * scalar products of the HT toolkit, Section 2.2; the mass is the density moment Section 4.2
 * checks).  Errors: HT_ERR_ARG, HT_ERR_CAPACITY (tensor capacity above the context's). */
int ht_mass(ht_ctx* ctx, const ht_tensor* u, double* out_dev, void* stream);
int ht_inner(ht_ctx* ctx, const ht_tensor* u, const ht_tensor* w, double* out_dev, void* stream);

/* ------------------------------------------------------------- CP calls ----- */
typedef enum cp_variant {
  CP_ALS_GS = 0,              /* Gauss-Seidel over k = 1..d (Section 3.1) */
  CP_ALS_JACOBI_DAMPED = 1    /* all modes from one iterate, increment / 4 (Appendix B, Alg. 1) */
} cp_variant;

/* ALS rank reduction (eqs. SSYSTEM, A^{ln}_{jhp}): x <- argmin |y - x| by `sweeps`
 * sweeps from the initial x (rank x->rank).  Mode update: X_k Gamma_k = Y_k diag(mu) H_k
 * with Gamma_k = hadamard_{j!=k} X_j^T X_j and H_k = hadamard_{j!=k} Y_j^T X_j, solved by
 * an FP64 Cholesky factorisation.  Factor columns are normalised into x->weight after
 * each mode solve.  eps_dev (device, `sweeps` doubles, or NULL) receives Algorithm 5's
 * max_k |X_k^new - X_k^old| / |X_k^old| per sweep.  Errors: HT_ERR_ARG, HT_ERR_CAPACITY. */
int cp_als_sweep(ht_ctx* ctx, const cp_tensor* y, cp_tensor* x, int sweeps, int variant,
                 double* eps_dev, void* stream);

/* y = p(dt L) x exactly in CP form for a kron_sum operator (the separable operator of eq. Lz
 * applied in CP format, the explicit step of Section 3.2): 1 + 2d + d(d-1)/2 rank-1
 * terms per term of x (identity, dt A_i, dt^2 A_i^2 / 2, dt^2 A_i A_j for i < j).
 * y->cap >= x->rank * (1 + 2d + d(d-1)/2).  Sets y->rank on the host. */
int cp_apply_rk2(ht_ctx* ctx, const cp_tensor* x, const ht_op* L, double dt, cp_tensor* y,
                 void* stream);

/* ALS rank reduction towards the implicit y = p(dt L) x_old (kron_sum L), without forming y:
 * the same result as cp_apply_rk2 followed by cp_als_sweep (Section 3.2: explicit step
 * then ALS rank reduction; Section 2.1 normal equations).  The factors of y are built
 * from the powers A_j^p X_old,j (p <= 2), so the right-hand side of mode k contracts
 * over 3 r0 columns instead of r0 (1 + 2d + d(d-1)/2).  x holds the initial iterate
 * (rank x->rank) and receives the fit; x_old (rank r0) may alias x (it is read first).
 * One launch runs every sweep: Gauss-Seidel sweeps on one thread-block cluster when the
 * problem fits its shared memory (ht_config.cp_form), else on a cooperative grid with
 * one CTA per factor column.  The two forms compute the same quantities in different
 * summation orders (they agree to rounding).
 * Errors: HT_ERR_ARG, HT_ERR_CAPACITY (x rank > 64 or above the context capacity). */
int cp_als_sweep_rk2(ht_ctx* ctx, const cp_tensor* x_old, const ht_op* L, double dt, cp_tensor* x,
                     int sweeps, int variant, double* eps_dev, void* stream);

/* Which form cp_als_sweep_rk2 takes on this context for ranks r (x) and r0 (x_old) in the
 * Gauss-Seidel variant: *ctas receives the CTAs of its thread-block cluster, or 0 for the
 * cooperative grid form (ht_config.cp_form = 1, ranks above 64, a layout beyond one CTA's
 * shared memory, or no cluster of that size placeable on the device).  The damped Jacobi
 * variant always takes the grid form.  Errors: HT_ERR_ARG. */
int cp_als_rk2_cluster_ctas(const ht_ctx* ctx, int r, int r0, int* ctas);

/* ----------------------------------------------------- allocation-free ---- */
/* The paper has no counterpart: this is a deployment variant of cp_als_sweep (same arguments
 * and results; see its declaration above) that allocates nothing and needs no ht_ctx.
 * Who needs it: code running where cudaMalloc is unavailable or forbidden -- inside
 * host callbacks or plug-ins with a fixed memory budget, or processes whose device
 * memory is reserved up front by another framework.
 * Same arguments and results as cp_als_sweep, plus status_dev (device int, or NULL)
 * which receives the device error word (HT_OK or HT_ERR_NONFINITE) at the end.
 * Scratch: one file-scope __device__ array of about 3.0 MB that every GPU loading the
 * library holds until exit.  Limits: d <= 8, n_k <= 256, x rank <= 32, y rank <= 1024;
 * larger sizes return HT_ERR_CAPACITY before anything is launched.  Allocates nothing
 * (no cudaMalloc/cudaFree, no allocating library routine).  The first call on a device
 * looks up the array's address with that device current: make it before any stream
 * capture.  All calls share the array, so calls that overlap on the GPU race and must
 * be serialised by the caller.  Errors: HT_ERR_ARG, HT_ERR_CAPACITY, HT_ERR_CUDA. */
int cp_als_sweep_noalloc(const cp_tensor* y, cp_tensor* x, int sweeps, int variant, double* eps_dev,
                         int* status_dev, void* stream);

/* ------------------------------------------------------------ diagnostics -- */
/* One Crank-Nicolson step solved in CP format by alternating least squares (Section 3.3, eqs.
 * CNFDE, BLs, rRr1, ALS2, ML, MR): x minimises |A x - B x_n| with A = I - dt/2 L and
 * B = I + dt/2 L, over the factors of x at its current rank, Gauss-Seidel over the dimensions,
 * `sweeps` sweeps (1..64); variant CP_ALS_GS solves the dimensions in turn (Gauss-Seidel),
 * CP_ALS_JACOBI_DAMPED solves all from the same iterate and moves each factor a quarter of the
 * way (the parallel ALS of Appendix B, Algorithm 1).  Mode q solves the (n_q r) x (n_q r) normal equations
 * M vec(X_q) = vec(R) (eq. ALS2 on the grid basis; M = sum_{e,z} eta_e eta_z Gamma^{ez} kron
 * (E_q^e)^T E_q^z, eq. ML) by Cholesky.  x: the initial guess on entry (e.g. a copy of x_n),
 * the result on return; its weights are folded into its first factor, so they are 1 on
 * return.  x_n: read only, must not share factor buffers with x.  L: any separable operator
 * (n_terms <= min(HT_MAXBLOCKTERMS, the context's max_terms); every factor kind).  eps_dev
 * (optional, device): per sweep the largest |X_q^new - X_q^old|^2 (the paper's convergence
 * measure).  Ranks <= the context's cap.  The first call on a context allocates its workspace
 * (about (T^2 d + T d) n^2 + (n cap)^2 doubles, T = max_terms + 1): make it before capturing a
 * graph (a capture that would allocate returns HT_ERR_ARG).  A system that is not positive
 * definite sets HT_ERR_NONFINITE (ht_ctx_check) and leaves that factor unchanged.  Errors:
 * HT_ERR_ARG, HT_ERR_CAPACITY, HT_ERR_NOMEM, HT_ERR_CUDA. */
int cp_cn_als_step(ht_ctx* ctx, const cp_tensor* x_n, const ht_op* L, double dt, cp_tensor* x, int sweeps,
                   int variant, double* eps_dev, void* stream);

/* Self-test of the bounded grid barrier that the cooperative grid form of the persistent ALS
 * kernel (cp_als_sweep_rk2) uses between its phases.  The paper has no counterpart.  Launches nblocks (1..64) cooperative CTAs
 * on `device` that meet at one barrier; CTA `absent` (or none when absent < 0) skips it, so the
 * others wait out the bounded limit (about 0.2 s of SM clock) and report instead of hanging.
 * Synchronising (allocates and frees its own 2 KB).  Returns HT_OK when every CTA passed, the
 * device-reported HT_ERR_TIMEOUT when the barrier gave up, or HT_ERR_ARG / HT_ERR_CUDA. */
int ht_selftest_grid_barrier(int nblocks, int absent, int device);

/* Self-test of the library's FP64 reciprocal and reciprocal square root (an FP32 seed refined
 * by the truncated series 1/(1-e) = 1 + e + e^2 and (1-e)^-1/2 = 1 + e/2 + 3e^2/8; used by the
 * QR, SVD and ALS kernels).  The paper has no counterpart.  For each of the n device doubles
 * x_dev[i] writes out_dev[4i .. 4i+3] = (library reciprocal, CUDA 1.0 / x, library rsqrt, CUDA
 * rsqrt) (device, 4n doubles).  Asynchronous on stream.  Errors: HT_ERR_ARG, HT_ERR_CUDA. */
int ht_selftest_fastmath(const double* x_dev, double* out_dev, int n, void* stream);

/* Self-test of the contraction kernels of HT_PREC_MIXED contexts: C[b] = alpha op(A[b])
 * op(B[b]) diag(colscale) + beta C[b] for b < batch (column-major; op(A) m x k, op(B) k x n; tA/tB
 * select the stored transposes; strides sA, sB, sC between batch entries; colscale: device, n
 * values, or NULL).  slices 2..4: the tensor-core kernel of the large contractions, from that many
 * BF16 digit planes per operand with FP32 accumulation in tensor memory; element (i, j) is within
 * about 2^-(8 slices - 1) k max_l |op(A)_il| max_l |op(B)_lj| of the exact product.  slices 1: the
 * split-FP32 CUDA-core kernel of the small ones (FP32 hi / lo parts, double-float accumulation);
 * element (i, j) is within about (k^2 + 5k + 10) 2^-47 sum_l |op(A)_il op(B)_lj| of the exact
 * product (about (k/2 + 10) 2^-47 of it with rounding errors of random sign; operands of magnitude
 * 2^128 or more are outside its range).  The paper has no counterpart: the
 * precision scheme is this library's.  Synchronising.  Returns HT_OK, HT_ERR_TIMEOUT (a bounded
 * wait gave up), HT_ERR_ARG or HT_ERR_CUDA. */
/* Tuning probe (used by the package's autotuner; the paper has no counterpart): mean CUDA-event
 * time in ms of `reps` launches of one synthetic contraction (op(A) m x k, op(B) k x n, `batch`
 * entries) through the FP64 CUDA-core kernel (route 0, ctas_per_sm CTAs per SM, 1..32), the
 * tensor-core split kernel (route 1, `slices` digit planes, 2..4) or the split-FP32 CUDA-core
 * kernel of the mixed form's small contractions (route 2, ctas_per_sm as route 0), written to
 * *ms_out.
 * Synchronising; allocates and frees its own device buffers.  Errors: HT_ERR_ARG, HT_ERR_NOMEM,
 * HT_ERR_CUDA, HT_ERR_TIMEOUT. */
int ht_tune_time_gemm(int m, int n, int k, int batch, int route, int slices, int ctas_per_sm, int reps,
                      double* ms_out);

int ht_selftest_gemm_mixed(int m, int n, int k, const double* A, int lda, int tA, const double* B, int ldb, int tB,
                           double* C, int ldc, double alpha, double beta, const double* colscale, int batch,
                           long long sA, long long sB, long long sC, int slices, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HTGPU_H */
