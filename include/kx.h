/*
 * kx.h -- C ABI of the GB300 screened Fock exchange library.
 *
 * The library builds the exchange matrix of Challacombe & Bock, "An N-Body
 * Solution to the Problem of Fock Exchange" (Eqs. 5-6), in the unscaled form
 *
 *     K_{mu nu} = sum_{lambda sigma} (mu lambda | nu sigma) P_{lambda sigma}
 *
 * (the paper's -1/2 is left to the caller), over uncontracted Cartesian
 * Gaussian shells (one primitive per shell, l = 0, 1, 2).  Shells are put in
 * Hilbert-curve order, recursively bisected (Eq. 1), annotated with
 * Frobenius-norm quadtrees (Eq. 2), and the hextree of Eq. 7 is traversed
 * level by level on the GPU with the metric query of Eq. 8: a task
 * (A,B,C,D) -- mu in A, lambda in B, nu in C, sigma in D -- is culled when
 *
 *     beta = (||Q_AB||_F * ||P_BD||_F) * ||Q_CD||_F <= tau,
 *
 * with Q_{mu lambda} = (mu lambda|mu lambda)^{1/2}.  Surviving shell
 * quartets are evaluated by McMurchie-Davidson kernels and contracted into K.
 *
 * Conventions
 *   - Cartesian components: x power descending, then y (p: x y z;
 *     d: xx xy xz yy yz zz).  Each component of a shell carries
 *     N(a,l) = (2a/pi)^{3/4} (4a)^{l/2} / sqrt((2l-1)!!).
 *   - Coordinates in bohr, exponents in bohr^-2.
 *   - Matrices are dense, row-major FP64 in *user* function order (shells in
 *   input order, functions of a shell contiguous).
 *   - All device work runs on the stream given to kx_create, in order.
 *
 * Errors: every call returns KX_OK or a KX_E* code; kx_last_error() gives a
 * one-line message.  No call aborts the process, and no call leaves the
 * CUDA context unusable on an error it detects.  Device waits are bounded.
 */
#ifndef KX_H
#define KX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    KX_OK = 0,
    KX_EINVAL = 1,     /* bad argument (null pointer, size, l > 2, ...) */
    KX_ESTATE = 2,     /* called out of order (e.g. exchange before tree) */
    KX_ENOMEM = 3,     /* device or host allocation failed */
    KX_ECUDA = 4,      /* a CUDA runtime call failed */
    KX_ECAPACITY = 5,  /* a caller buffer or a size limit was too small */
    KX_ETIMEOUT = 6,   /* a bounded device wait gave up */
    KX_ENOTIMPL = 7    /* option not available in this build */
};

/* Precision of the ERI stage.  KX_FP64: every shell quartet in FP64.
 * KX_MIXED: quartets with beta <= split_threshold in FP32 (FP32 Boys
 * table, pair data, P copy and accumulation), the rest in FP64.
 * KX_MIXED_DW: the same split, with the quartets above it in double-word
 * FP32 arithmetic (each value an unevaluated sum of two floats, about 48
 * significant bits, all on the FP32 pipe) wherever the class has such a
 * kernel (la+lb+lc+ld <= 5) and in FP64 otherwise; split_threshold = 0
 * puts every quartet of those classes in double-word arithmetic.  K is
 * accumulated in FP64 in every mode. */
enum { KX_FP64 = 0, KX_MIXED = 1, KX_MIXED_DW = 2 };

typedef struct kx_ctx kx_ctx;          /* opaque, owned by the library */

/* Molecule and shell list (host memory, copied by kx_create). */
typedef struct {
    int32_t n_atom;
    int32_t n_shell;             /* 1 .. 65535 (per system) */
    const double* xyz;           /* [n_atom][3] atom centres, bohr */
    const int32_t* shell_atom;   /* [n_shell] atom of each shell */
    const int32_t* shell_l;      /* [n_shell] angular momentum, 0..2 */
    const double* shell_alpha;   /* [n_shell] exponent > 0, bohr^-2 */
} kx_basis;

/* Options of one exchange build. */
typedef struct {
    double tau;                  /* Eq. 8 threshold tau_2e >= 0 (keep iff beta > tau) */
    double split_threshold;      /* KX_MIXED(_DW): shell quartets with beta > split run in FP64
                                    (double-word FP32 in KX_MIXED_DW) */
    int32_t precision;           /* KX_FP64, KX_MIXED or KX_MIXED_DW */
    int32_t shell_screen;        /* 1: apply Eq. 8 again to each shell quartet of a leaf */
    int32_t keep_worklist;       /* 1: retain the leaf-quartet list for kx_get_worklist */
    int32_t profile;             /* 1: time every ERI class launch (see kx_get_profile) */
    int64_t chunk_records;       /* shell quartets per evaluation chunk, 0 = default */
    int32_t symmetric;           /* 1: P is symmetric, so K = K^T: only the K blocks (A,C)
                                    with A <= C (tree order; shells a <= c inside a
                                    diagonal block) are built and the rest mirrored */
    int32_t row_leaf_lo;         /* K row-block shard: only tasks whose row block A lies in */
    int32_t row_leaf_hi;         /* the leaves [row_leaf_lo, row_leaf_hi) are traversed and
                                    evaluated (0, 0 = every leaf); see kx_row_work */
    int32_t reserved;            /* 0 */
    double split_budget;         /* KX_MIXED(_DW), > 0: split_threshold is ignored and the split is
                                    chosen per build from the FP32 error model so that the
                                    estimated max|dK| of the FP32 quartets stays within this
                                    budget (kx_stats.split_used, fp32_err_estimate) */
} kx_opts;

/* Counters and stage times of the last build. */
typedef struct {
    int64_t n_leaf_quartets;     /* leaf-block quartets surviving Eq. 8 */
    int64_t n_shell_quartets;    /* shell quartets evaluated */
    int64_t n_shell_quartets_fp64;
    int64_t n_candidates;        /* shell quartets screened at the shell level */
    int64_t n_shell_quartets_dw; /* KX_MIXED_DW: shell quartets in double-word FP32 */
    int64_t n_tasks[32];         /* tasks surviving at each traversal level */
    int32_t depth;               /* deepest traversal level */
    int32_t n_chunks;
    int32_t n_launches;          /* kernels launched by the build */
    int32_t pad;
    double flops_fp64;           /* algorithmic FLOPs of the ERI+contraction stage */
    double flops_fp32;
    double flops_dw;
    double ms_norms;             /* P norms and pyramid */
    double ms_traverse;          /* levels 0 .. depth-1 */
    double ms_expand;            /* last level + shell screen + class binning */
    double ms_eri;               /* ERI evaluation + contraction */
    double ms_eri_kernel_max;    /* longest single ERI class launch */
    double ms_total;
    double split_used;           /* KX_MIXED(_DW): the split threshold of the build (the
                                    planner's choice when split_budget > 0) */
    double fp32_err_bound;       /* split_budget > 0: eps32 * (largest sum over one sampled K shell
                                    block of c_max[class] * beta of its FP32 quartets), a
                                    bound on max|dK| from FP32 rounding under the
                                    per-quartet error model */
    double fp32_err_estimate;    /* split_budget > 0: 5 eps32 * sqrt(largest sum over one sampled K
                                    shell block of (c_rms[class] * beta)^2), a 5-sigma
                                    estimate of that error for independent roundings */
} kx_stats;

/* Fills the defaults: tau = 1e-10, split 1e-5, FP64, shell screen on,
 * no worklist retention, default chunking, no symmetry. */
void kx_default_opts(kx_opts* o);

/* Creates a context on CUDA device `device` (made current by the call) whose
 * work is ordered on `cuda_stream` (a cudaStream_t; NULL = legacy default
 * stream).  Copies the basis.  Runs the Hilbert ordering of the atoms
 * (Sec. "Exchange as hextree traversal": locality-preserving space-filling
 * curve) on the device.  *out is NULL on failure. */
int kx_create(kx_ctx** out, const kx_basis* basis, int device, void* cuda_stream);

/* Shell-pair Schwarz factors for Eq. 8: s2(a,b) = sum_{mu in a, lambda in b}
 * (mu lambda|mu lambda), FP64 on the device.  When tau_ovlp > 0, pairs whose
 * every overlap |(phi_mu, phi_nu)| is below tau_ovlp are set empty (Eq. 4);
 * 0 disables that prune.  Geometry-only: call once per context. */
int kx_build_schwarz(kx_ctx* c, double tau_ovlp);

/* Ragged bisection of the shell index space (Eq. 1) into leaves of at most
 * leaf_max_functions functions (a single shell is always a leaf; the paper
 * uses 10), and the Schwarz norm pyramid over it (Eq. 2).  perm, if not
 * NULL, is a host array [n_shell] giving the user shell at each tree
 * position and replaces the Hilbert order (in a batch it must map every
 * system's range of positions onto that system's shells).  Requires
 * kx_build_schwarz. */
int kx_build_tree(kx_ctx* c, int32_t leaf_max_functions, const int32_t* perm);

/* One exchange build (Eqs. 6-8).  P and K are DEVICE pointers to row-major
 * FP64 matrices of n_fn x n_fn in user function order with leading
 * dimensions ldp, ldk >= n_fn; the caller owns both.  K is overwritten.  P
 * need not be symmetric.  st may be NULL.  Asynchronous on the context's
 * stream except for a few small size read-backs.  Single-system contexts
 * only (KX_EINVAL on a batch: see kx_exchange_batch). */
int kx_exchange(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o,
                double* K, int64_t ldk, kx_stats* st);

/* kx_exchange with HOST buffers: copies P in, builds K, copies K out, and
 * returns after K is on the host.  Device buffers are cached in the context. */
int kx_exchange_host(kx_ctx* c, const double* P_host, int64_t ldp, const kx_opts* o,
                     double* K_host, int64_t ldk, kx_stats* st);

/* Survivor counts of one build without building it: the traversal (Eqs.
 * 7-8) and the shell-level screen of kx_exchange for the same P and
 * options, but no integral is evaluated and K is not touched.  Fills
 * n_leaf_quartets, n_tasks, depth, n_candidates, n_shell_quartets,
 * n_shell_quartets_fp64 / _dw (KX_MIXED(_DW): those above split_threshold)
 * and flops_fp64/flops_fp32/flops_dw (the ERI stage's algorithmic FLOPs), exactly as the
 * build would report them; the time fields hold the traversal and screen.
 * P: DEVICE, as for kx_exchange (ldp >= n_fn), or packed per system with
 * ldp = 0 on a batch context.  st is required.  Synchronous. */
int kx_count(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, kx_stats* st);

/* The split threshold of a mixed build from an error budget (a growth
 * direction beyond the paper, whose integrals are all FP64).  An FP32 shell quartet
 * q of bound beta_q (Eq. 8) perturbs its K shell block (a,c) by at most
 * c_max eps32 beta_q and by c_rms eps32 beta_q in root-mean-square, with
 * per-class constants measured on GB300 (eps32 = 2^-24).  A statistics
 * variant of the build's count pass sums, for a sample of K shell blocks
 * (every diagonal block, every pair of tree neighbours, 4 n_shell seeded
 * random blocks), the FP32 quartets' c_max beta and (c_rms beta)^2 in bins
 * of log2 beta.  The split is the largest tau * 2^(k/4) whose estimate
 * 5 eps32 max_ac sqrt(sum (c_rms beta)^2) over those blocks is at most
 * `budget`: st->split_used, st->fp32_err_estimate (that estimate) and
 * st->fp32_err_bound (eps32 max_ac sum c_max beta, the bound under the
 * per-quartet model).  0 when even the smallest split exceeds the budget.
 * P and o as for kx_count (o->split_threshold and precision are ignored).
 * Single-system contexts (KX_ENOTIMPL on a batch).  Synchronous.
 * kx_exchange, kx_count and kx_graph_plan run this first when
 * o->split_budget > 0 and build with the split it chooses. */
int kx_split_plan(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double budget, kx_stats* st);

/* K row-block shards (several GPUs).  The leaf quartets are independent,
 * so the build splits by the row block A of K (mu in A): a build with
 * kx_opts.row_leaf_lo/hi traverses (Eqs. 7-8) and evaluates only the tasks
 * whose A lies in those leaves, and writes only their contributions (its
 * rows, and in a symmetric build the mirrored columns of those rows); K is
 * zero elsewhere.  Summing the K of the shards [b_0, b_1), [b_1, b_2), ...
 * gives the K of the whole build (every entry comes from exactly one
 * shard), and the union of their worklists is its worklist.
 *
 * kx_row_work: work[leaf] (host array of the leaf count of kx_get_leaves)
 * = algorithmic FLOPs of the ERI stage of the tasks with that row leaf, in
 * the build with these options (its traversal and count pass, no K);
 * P as for kx_count.  Synchronous. */
int kx_row_work(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double* work);

/* Contiguous shards of balanced work: bounds[0] = 0 < bounds[1] < ... <
 * bounds[n_shards] = n_leaf, each boundary the leaf boundary whose prefix
 * sum of work is nearest j/n_shards of the total (equal leaf counts when
 * all work is zero).  Host only (no device, no context); KX_EINVAL unless
 * 1 <= n_shards <= n_leaf and every work[i] is finite and >= 0. */
int kx_shard_bounds(const double* work, int32_t n_leaf, int32_t n_shards, int32_t* bounds);

/* ------------------------------------------------------------------------
 * Batches of independent systems (a growth direction beyond the paper: many
 * uneven systems in one traversal and one set of class-kernel launches).
 * The systems are concatenated in input order: atoms, shells and functions
 * of system y follow those of systems 0..y-1, and the tree positions of
 * system y form the range of its shells.  Every system gets its own Hilbert
 * order (Sec. "Exchange as hextree traversal") and its own bisection tree
 * (Eq. 1); level k of the forest holds the level-k nodes of every system,
 * system-major, so kx_get_leaves and kx_get_worklist report leaf ordinals of
 * the forest.  A task never mixes systems: the level-0 tasks are (Y,Y,Y,Y),
 * one per system Y, and children stay inside their parent's system.
 * ------------------------------------------------------------------------ */

/* Creates a context holding n_sys (1..65535) systems bases[0..n_sys-1]
 * (host; each as for kx_create).  kx_build_schwarz and kx_build_tree then
 * apply to every system.  kx_create(out, b, ...) is
 * kx_create_batch(out, 1, b, ...). */
int kx_create_batch(kx_ctx** out, int32_t n_sys, const kx_basis* bases, int device, void* cuda_stream);

/* One exchange build of every system of the batch (Eqs. 6-8 per system).
 * P and K are DEVICE arrays of kx_packed_size(c) doubles: system y's
 * n_y x n_y matrix (row-major, its own user function order) starts at
 * sum_{z<y} n_z^2.  K is overwritten.  Works on single-system contexts
 * too (packed = dense n_fn x n_fn). */
int kx_exchange_batch(kx_ctx* c, const double* P, const kx_opts* o, double* K, kx_stats* st);

/* kx_exchange_batch with HOST buffers (copies inside, returns when K is on
 * the host). */
int kx_exchange_batch_host(kx_ctx* c, const double* P_host, const kx_opts* o, double* K_host,
                           kx_stats* st);

/* Doubles of a packed P or K: sum over the systems of n_y^2. */
int64_t kx_packed_size(const kx_ctx* c);

/* Launch-shape autotuner of the class kernels: one kx_exchange_batch build
 * (P, K packed, K written) during which every (precision, class) stream with
 * at least 16384 shell quartets is timed, on up to 2^19 of its quartets
 * accumulated into a scratch K, with 64, 128 and 256 threads per block and
 * with one thread per quartet or a persistent grid of 1x or 2x the blocks
 * that fit on an SM; the fastest shape is kept for later builds of this
 * context.  *n_tuned = streams tuned (may be NULL). */
int kx_autotune(kx_ctx* c, const double* P, const kx_opts* o, double* K, kx_stats* st, int32_t* n_tuned);

/* Current launch shape of the 243 streams (threads per block; persistent
 * blocks per SM, 0 = one thread per quartet; kernel variant: 0 for every
 * stream except the classes with la+lb+lc+ld >= 7, where FP64 has 0 the
 * rolled kernel, 1 the shared-memory kernel and 2 the shared-memory kernel
 * with the ket Hermite set pruned per ket component, and FP32 has 0 the
 * shared-memory kernel and 1 its ket-pruned form; the double-word streams
 * have one kernel each).  Host arrays of 243 entries, may be NULL. */
int kx_get_launch_shapes(const kx_ctx* c, int32_t* threads, int32_t* blocks_per_sm, int32_t* variant);

/* Sets the launch shape of stream s = precision * 81 + class: threads a
 * multiple of 32 in [32, 256], blocks_per_sm >= 0, variant 0, 1 or 2 (1 and 2
 * only where those kernels exist).  KX_EINVAL otherwise.  Discards a captured
 * plan. */
int kx_set_launch_shape(kx_ctx* c, int32_t s, int32_t threads, int32_t blocks_per_sm, int32_t variant);

/* Captured build.  kx_graph_plan runs one kx_exchange_batch build (P, K
 * packed, K written), sizes every buffer from it with `headroom` (0.25 = 25 %
 * more frontier tasks, leaf quartets and shell quartets per chunk than this
 * build needed), and records a whole build of the same options into one
 * CUDA graph in which every launch takes its sizes from device memory: the
 * traversal and screen kernels stride over device counts with persistent
 * grids, the class kernels read their quartet ranges from the device.
 * kx_graph_launch replays it: reads the CURRENT contents of the P array given
 * to kx_graph_plan and overwrites that K (the addresses are part of the
 * graph), ordered on the context's stream.  A count beyond its capacity (or
 * quartets of a class stream that was empty in the planning build) is
 * detected on the device, nothing is written out of bounds, and the replay
 * returns KX_ECAPACITY with K incomplete: plan again.  No kernel of the
 * graph waits on another block, so no replay can time out.  Any other build
 * on the context, kx_build_schwarz or kx_build_tree discards the plan. */
int kx_graph_plan(kx_ctx* c, const double* P, const kx_opts* o, double* K, double headroom, kx_stats* st);
int kx_graph_launch(kx_ctx* c, kx_stats* st);

/* Number of basis functions (summed over the systems of a batch). */
int64_t kx_n_functions(const kx_ctx* c);

/* Tree order: perm[i] = user shell at tree position i (host array). */
int kx_get_order(const kx_ctx* c, int32_t* perm);

/* Leaves of the bisection, left to right: [lo, hi) tree positions (host
 * arrays of capacity cap).  *n_leaf and *depth always set. */
int kx_get_leaves(const kx_ctx* c, int32_t* lo, int32_t* hi, int32_t cap,
                  int32_t* n_leaf, int32_t* depth);

/* Leaf quartets (A,B,C,D) kept by the last kx_exchange that had
 * keep_worklist = 1 (or by kx_traverse / kx_cull_kept), as leaf ordinals, into host out[cap][4].  With
 * n_filter > 0 only quartets whose A is in a_filter[] are returned.
 * *n = number matching (entries beyond cap are not written; KX_ECAPACITY
 * then).  Without a filter the list comes in kept order (the order of
 * kx_leaf_features); with one the order is unspecified. */
int kx_get_worklist(kx_ctx* c, const int32_t* a_filter, int32_t n_filter,
                    int32_t* out, int64_t cap, int64_t* n);

/* Shell-level tables in USER shell order (host arrays [n_shell][n_shell]):
 * s2 = squared Schwarz norms (after any Eq. 4 prune), pq = squared
 * Frobenius norms of the P shell blocks of the last kx_exchange (may be
 * NULL).  For a batch: one dense block per system, system y's
 * [n_shell_y][n_shell_y] block (its own user shell order) starting at
 * sum_{z<y} n_shell_z^2. */
int kx_get_norms(kx_ctx* c, double* s2, double* pq);

/* Per-stream totals of the last kx_exchange run with profile = 1, for the
 * 243 streams s = precision * 81 + class (precision 0 = FP64, 1 = FP32,
 * 2 = double-word FP32; class = ((la*3 + lb)*3 + lc)*3 + ld): ms = summed
 * CUDA-event time of the stream's kernel launches, n = shell quartets,
 * flops = algorithmic FLOPs, launches = kernel launches.  Host arrays of
 * 243 entries (any may be NULL). */
int kx_get_profile(const kx_ctx* c, double* ms, int64_t* n, double* flops, int32_t* launches);

/* Throughput probe on `device`, timed with CUDA events (best of five after
 * a warm-up launch).  precision KX_FP64 or KX_MIXED (= FP32): independent
 * fused multiply-add chains on the plain FMA pipe; KX_PROBE_FP64_MMA: FP64
 * tensor-core (DMMA, mma.sync m8n8k4) chains; KX_PROBE_DW: double-word FP32
 * multiply-add chains (the arithmetic of KX_MIXED_DW).  *gflops = measured
 * GFLOP/s (2 per multiply-add).  Not part of the exchange build; used to state
 * roofline fractions and to decide where tensor cores would pay. */
#define KX_PROBE_FP64_MMA 2
#define KX_PROBE_DW 3
int kx_peak_probe(int device, int precision, double* gflops);

/* ------------------------------------------------------------------------
 * Learned culling (a growth direction beyond the paper).  A small network
 * predicts, from ten descriptors of a leaf quartet, log10 of the Frobenius
 * norm of its contribution to K; a leaf quartet whose exact Eq. 8 bound is
 * at most 10 tau is dropped when the predicted contributions of such
 * quartets fit a per-K-block budget (kx_cull_kept), so any quartet whose
 * bound exceeds 10 tau is always evaluated.  The pieces
 * below compose: kx_traverse -> kx_leaf_features -> kx_mlp_infer_bf16 ->
 * kx_cull_kept -> kx_evaluate_kept.  The context-bound calls of this block
 * (and kx_traverse_level_noalloc) take single-system contexts; on a batch
 * they return KX_ENOTIMPL.
 * ------------------------------------------------------------------------ */
#define KX_NFEAT 10
#define KX_MLP_HIDDEN 64
/* parameters (FP32): mu[10], 1/sigma[10], W1[64][10], b1[64], W2[64][64],
 * b2[64], W3[64][64], b3[64], W4[64], b4 */
#define KX_MLP_NPARAM 9109

/* The traversal of kx_exchange (Eqs. 7-8) without the ERI stage: computes
 * the P norms of P (device) and keeps every surviving leaf quartet on the
 * device; *n_leaves = their number. */
int kx_traverse(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, int64_t* n_leaves);

/* Descriptors of the kept leaf quartets (A,B,C,D), in kept order, into the
 * DEVICE array feat[n][10] (FP32): log10 ||Q_AB||, log10 ||Q_CD||,
 * log10 ||P_BD||, log10 beta, |c_A - c_C|, |c_B - c_D|, distance between
 * the bra and ket centroids (bohr), largest block radius, largest l, log10
 * of the smallest exponent.  *n = kept count (KX_ECAPACITY if > cap). */
int kx_leaf_features(kx_ctx* c, float* feat, int64_t cap, int64_t* n);

/* Drops kept leaf quartet i = (A,B,C,D) when its bound is at most 10 tau
 * and pred[i] + log10(m_AC) < log10_budget, m_AC being the number of kept
 * quartets of bound <= 10 tau that share its K block (A,C): the predicted
 * sum of what any K block loses stays below the budget.  pred: DEVICE
 * array in kept order (log10 contributions, any safety margin added by the
 * caller).  Keeps the order of the rest; *n_kept = what remains. */
int kx_cull_kept(kx_ctx* c, const float* pred, double tau, double log10_budget, int64_t* n_kept);

/* The ERI stage (shell screen, class kernels, K accumulation) over the kept
 * leaf quartets; P and K device, K overwritten. */
int kx_evaluate_kept(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double* K, int64_t ldk,
                     kx_stats* st);

/* The ERI stage over an explicit list of leaf quartets (host int32[n][4],
 * leaf ordinals).  For a list whose (A,C) are pairwise distinct every
 * quartet owns its K block, so kx_block_norms then returns the exact norm
 * of each quartet's contribution (the training targets). */
int kx_exchange_leaves(kx_ctx* c, const double* P, int64_t ldp, const int32_t* leaves, int64_t n,
                       const kx_opts* o, double* K, int64_t ldk, kx_stats* st);

/* ||K_AC||_F for every leaf quartet of leaves (host int32[n][4]) from the
 * DEVICE matrix K; norms host double[n]. */
int kx_block_norms(kx_ctx* c, const double* K, int64_t ldk, const int32_t* leaves, int64_t n,
                   double* norms);

/* MLP inference with BF16 weights and activations and FP32 accumulation:
 * pred[i] for the n feature rows (DEVICE arrays), on `stream`. */
int kx_mlp_infer_bf16(const float* params, const float* feat, int64_t n, float* pred, void* stream);

/* Loss 0.5 * mean((y - target)^2) over the n rows and its gradient with
 * respect to every trained parameter (FP32, DEVICE arrays; the two
 * normalisation vectors get zero gradient); *loss on the host. */
int kx_mlp_loss_grad(const float* params, const float* feat, const float* target, int64_t n,
                     float* grad, double* loss, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with
 * `step` >= 1) on the trained parameters; m and v are DEVICE state. */
int kx_mlp_adam(float* params, const float* grad, float* m, float* v, float lr, int32_t step,
                void* stream);

/* Largest frontier, in tasks, that kx_traverse_level_noalloc accepts. */
#define KX_NOALLOC_MAX_TASKS (1 << 18)

/* One level of the hextree traversal that allocates no device memory.
 *
 * This entry point has no counterpart in the paper.  It exists for callers
 * that cannot let a library allocate: programs that hand all device memory
 * to their own allocator at start-up (a framework's caching pool, or a fixed
 * budget reserved once) and must not see cudaMalloc/cudaFree calls behind
 * their back, and programs with a no-allocation-after-initialisation rule
 * (a cudaMalloc or cudaFree can stall the whole device).
 *
 * It expands the n level-`level` tasks of `front` (DEVICE array of n tasks,
 * each four uint16 node ids A, B, C, D of that level, as in the traversal of
 * kx_exchange) into the level-(level+1) tasks whose Eq. 8 bound exceeds tau,
 * written to `next` (DEVICE array with room for cap tasks) in the order the
 * traversal uses; *n_next (host) receives their number.  Starting from the
 * single task (0,0,0,0) at level 0 and calling it for levels 0 .. depth-1
 * yields the leaf-quartet worklist of kx_exchange for the same tau and the
 * same `symmetric` option.  The root task itself is not tested, as in
 * kx_exchange when depth >= 1; a tree of depth 0 (a single leaf) has no
 * level to walk (KX_EINVAL), and there kx_exchange keeps the root task iff
 * its own bound exceeds tau, a test left to the caller.
 *
 * Requirements: a tree (kx_build_tree) and the P norms of a previous
 * kx_exchange on this context.  The norms of that call's P are used, and so
 * is its `symmetric` option: after a symmetric build, a task whose K block
 * is diagonal (A == C) keeps only the children with A' <= C', as in the
 * traversal of that build.
 * Scratch: a file-scope device array of 4.5 MiB, holding counts,
 * offsets, masks and scan sums for up to KX_NOALLOC_MAX_TASKS tasks, that
 * every GPU which loads the library keeps until the process exits.  The
 * first call on a device (made current by the call) looks up that array's
 * device address; make that first call before any stream capture on the
 * device.  The address is kept for the life of the process: after a
 * cudaDeviceReset (or any other teardown of the device's primary context)
 * the kept address is stale, so do not call this entry point again in that
 * process.  All calls share the array and it keeps the last call's contents
 * (the call itself clears what must start at zero), so calls that overlap
 * on the GPU -- other streams, threads or contexts on the same device --
 * race and must be serialised by the caller.  Returns after the count is on
 * the host.
 *
 * Errors: KX_ECAPACITY when n > KX_NOALLOC_MAX_TASKS (nothing is run) or
 * when the next frontier exceeds cap (the first cap tasks are written and
 * *n_next holds the full count); KX_ESTATE without tree or P norms;
 * KX_EINVAL for a bad level, pointer, size or tau, and when a task of
 * `front` names a node id at or beyond the node count of level `level`
 * (such tasks are skipped on the device without touching any table, the
 * others are expanded and *n_next counts their children). */
int kx_traverse_level_noalloc(kx_ctx* c, int32_t level, const uint16_t* front, int64_t n,
                              double tau, uint16_t* next, int64_t cap, int64_t* n_next);

/* Algorithmic FLOPs of one shell quartet of class cls = ((la*3 + lb)*3 +
 * lc)*3 + ld, as the build counts them (*total), and the part of it that
 * does not involve P (*integral: P-Q, the prefactor, the Boys function and
 * the Hermite recursion of R; the rest is the contraction with P through
 * the Hermite sets).  An integral block shared by several symmetric images
 * (the index swaps of Eq. 9) could save the integral part of all but one,
 * never the contraction.  Host only; KX_EINVAL for a bad class or pointer. */
int kx_class_flops(int32_t cls, double* total, double* integral);

/* Last error message of the context (never NULL). */
const char* kx_last_error(const kx_ctx* c);

/* Frees the context and all its device memory (NULL is ignored). */
void kx_destroy(kx_ctx* c);

#ifdef __cplusplus
}
#endif
#endif /* KX_H */
