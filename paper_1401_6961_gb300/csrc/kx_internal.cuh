// kx_internal.cuh -- internal types and device helpers of the exchange library.
//
// Index spaces used throughout:
//   user shell      the order of kx_basis (P and K rows/columns follow it)
//   tree position   Hilbert-ordered shells (atom-major, input order inside an
//                   atom); the bisection tree of Eq. 1 is built over it
//   level node      the nodes of traversal level k: a left-to-right partition
//                   of the tree positions.  A leaf that stops splitting
//                   before the deepest level is carried down unchanged (its
//                   only child is itself), so every level partitions all
//                   shells and level `depth` is the leaf partition.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/kx.h"

namespace kx {

constexpr int LMAX = 2;
constexpr int NCLASS = 81;          // (la,lb,lc,ld), l <= 2
// class-kernel streams s = precision * NCLASS + class: precision 0 = FP64,
// 1 = FP32, 2 = double-word FP32 (KX_MIXED_DW above the split)
constexpr int NPREC = 3;
constexpr int NSTREAM = NPREC * NCLASS;
// double-word kernels exist for the classes with la+lb+lc+ld <= DW_LMAX
constexpr int DW_LMAX = 5;
// split planning: bins of log2 beta per octave (candidate splits tau 2^(k/4))
constexpr int PLAN_BINS_PER_OCTAVE = 4;
__host__ __device__ constexpr int class_l(int cls) { return cls / 27 + (cls / 9) % 3 + (cls / 3) % 3 + cls % 3; }
constexpr int NPAIRCLASS = 9;       // (la,lb)
constexpr int MAX_LEVELS = 32;
constexpr double PI = 3.14159265358979323846;
// Boys table: F_m(T_i), T_i = i / BOYS_DENS for T < BOYS_TMAX, m = 0..BOYS_M
// (orders up to 8 plus the 6 extra Taylor orders).
constexpr int BOYS_M = 14;
constexpr int BOYS_DENS = 32;
constexpr double BOYS_TMAX = 40.0;
constexpr int BOYS_NPTS = 40 * BOYS_DENS + 2;
// layout of the small device counter array of a context
constexpr int CTR_CAND = 8;                        // shell quartets screened
constexpr int CTR_FILTER = CTR_CAND + 1;           // worklist export count
constexpr int CTR_END = CTR_FILTER + 1;            // per-stream end offsets
constexpr int CTR_ERR = CTR_END + NSTREAM;         // write-guard violations
constexpr int NCOUNTERS = 512;

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
// Hermite functions with t+u+v <= L
__host__ __device__ constexpr int nherm(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
// linear index of (t,u,v): block of total n = t+u+v, then s = u+v, then v
__host__ __device__ constexpr int hidx(int t, int u, int v) {
    return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}
// Cartesian component k of angular momentum l (x power descending, then y)
__host__ __device__ constexpr int cart_x(int l, int k) {
    return l == 0 ? 0 : (l == 1 ? (k == 0 ? 1 : 0) : (k == 0 ? 2 : (k <= 2 ? 1 : 0)));
}
__host__ __device__ constexpr int cart_y(int l, int k) {
    return l == 0 ? 0 : (l == 1 ? (k == 1 ? 1 : 0) : (k == 1 ? 1 : (k == 3 ? 2 : (k == 4 ? 1 : 0))));
}
__host__ __device__ constexpr int cart_z(int l, int k) { return l - cart_x(l, k) - cart_y(l, k); }

// size of the per-dimension E table of a pair (la,lb): [i<=la][j<=lb][t<=la+lb]
__host__ __device__ constexpr int etab(int la, int lb) { return (la + 1) * (lb + 1) * (la + lb + 1); }
__host__ __device__ constexpr int eidx(int la, int lb, int i, int j, int t) {
    return (i * (lb + 1) + j) * (la + lb + 1) + t;
}
// FP64 pair record: p, Px, Py, Pz, prefactor, Ex[], Ey[], Ez[] (padded to even)
__host__ __device__ constexpr int pair_stride(int la, int lb) {
    return ((5 + 3 * etab(la, lb)) + 1) & ~1;
}
// FP32 pair record (64 bytes, four 16-byte loads): p, 1/(2p), prefactor,
// P as hi+lo floats (so that P-Q keeps its digits when P ~ Q), P-A, P-B, pad.
// The FP32 kernels rebuild the E coefficients from it in registers.
constexpr int PAIR32_STRIDE = 16;
enum { P32_P = 0, P32_INV2P = 1, P32_KAB = 2, P32_PHI = 3, P32_PLO = 6, P32_PA = 9, P32_PB = 12 };
// row length of the FP32 Boys table (orders 0..BOYS_M, padded for 16-byte loads)
constexpr int BOYS32_ROW = 16;

// Shell pair metadata shared by the FP64 and FP32 pair tables.  P and K
// entries of one system are addressed affinely in user function indices:
// X(mu,nu) = X[x0 + mu * ld + nu] (see MatFrame); a pair (a,b) carries the
// row bases it needs as a bra.
struct PairMeta {
    int64_t prow_b;   // P offset of row fb, column 0 (p0 + fb * ldp)
    int64_t krow_a;   // K offset of row fa, column 0 (k0 + fa * ldk)
    int32_t fa, fb;   // user function offsets of the two shells
    int32_t ldp, ldk; // leading dimensions of the pair's system
};

// One square diagonal block of a block-diagonal table: entries (i,j) with
// base <= i, j < base + n sit at off + (i - base) * n + (j - base), i.e. at
// t0() + i * n + j.  A single system is one block with base 0.
struct Seg {
    int64_t off;
    int32_t base, n;
    __host__ __device__ int64_t t0() const { return off - (int64_t)base * (n + 1); }
};

// P and K addressing of one system for one build: X(mu,nu) at
// x0 + mu * ld + nu (mu, nu user function indices of the system).
struct MatFrame {
    int64_t p0, k0;
    int32_t ldp, ldk;
};

// block of a flat table index (binary search over the blocks' offsets)
__host__ __device__ inline int seg_find(const Seg* __restrict__ seg, int nseg, int64_t e) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (seg[m].off <= e) lo = m; else hi = m - 1;
    }
    return lo;
}
// (i, j) of flat index e of a block-diagonal table
__host__ __device__ inline void seg_pair(const Seg* __restrict__ seg, int nseg, int64_t e, int& i, int& j) {
    const Seg s = seg[seg_find(seg, nseg, e)];
    const int64_t r = e - s.off;
    i = s.base + (int)(r / s.n);
    j = s.base + (int)(r % s.n);
}

// Shell quartet record: slots in the bra (la,lb) and ket (lc,ld) pair tables.
struct Quartet {
    int32_t ab, cd;
};

// A traversal task: node ids of level k (tree positions fit in 16 bits).
struct Task {
    uint16_t a, b, c, d;
};

struct LevelInfo {
    int32_t n;        // nodes at this level
    int32_t off;      // offset of the level in the flat node arrays
};

// Device-side view of a level's dense norm tables.
struct NormLevel {
    const double* s;  // ||Q_XY||_F, n x n
    const double* p;  // ||P_XY||_F, n x n
    int32_t n;
};

}  // namespace kx

// ---------------------------------------------------------------------------
// context (host side)
// ---------------------------------------------------------------------------

struct kx_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err = "no error";

    // systems: a context holds n_sys independent systems, each contiguous
    // in atoms, shells (user order and tree positions) and functions; every
    // table is block-diagonal over them (one block for a single system)
    int n_sys = 1;
    std::vector<int32_t> sys_atom, sys_shell;   // [n_sys + 1] offsets
    std::vector<int64_t> sys_fn, sys_mat;       // [n_sys + 1]; sys_mat: packed P/K (sum of n_fn^2)
    std::vector<kx::Seg> sseg;                  // shell-pair blocks, [n_sys]
    int64_t sp_total = 0;                       // entries of a shell-pair table
    kx::Seg* d_sseg = nullptr;
    int32_t* d_tsys = nullptr;                  // system of every tree position
    std::vector<kx::Seg> lseg;                  // level blocks, [(depth + 1) * n_sys], off absolute
    kx::Seg* d_lseg = nullptr;
    int32_t* d_node_sys = nullptr;              // system of every node (flat over levels)
    kx::MatFrame* d_mframe = nullptr;           // [n_sys], per build
    kx::Seg* d_fseg = nullptr;                  // function blocks of the systems, off = packed offset
    int32_t* d_ftpos = nullptr;                 // tree position of every function's shell (user order)
    bool packed = false;                        // the current build's P/K are packed per system
    int build_sym = 0;                          // the current build is symmetric (kx_opts.symmetric)

    // basis (host copies)
    int n_atom = 0, n_shell = 0;
    int64_t n_fn = 0;
    std::vector<double> xyz;
    std::vector<int32_t> shell_atom, shell_l;
    std::vector<double> shell_alpha;
    std::vector<int64_t> fn_off;          // user shell -> first function

    // order and tree
    std::vector<int32_t> perm;            // tree position -> user shell
    bool have_order = false, have_schwarz = false, have_tree = false;
    int depth = 0;                        // deepest level
    int leaf_max = 10;
    std::vector<kx::LevelInfo> levels;    // 0..depth
    std::vector<int32_t> node_lo, node_hi, node_child;   // flat over levels; child = first child
    std::vector<int32_t> node_nchild;

    // device: basis in tree order
    int32_t* d_tl = nullptr;              // l by tree position
    double* d_tctr = nullptr;             // centre [3] by tree position
    double* d_talpha = nullptr;
    int32_t* d_tfoff = nullptr;           // user function offset by tree position
    int32_t* d_perm = nullptr;

    // device: shell-pair tables in tree order (n_shell^2)
    double* d_s2 = nullptr;               // squared Schwarz norms
    double* d_snorm = nullptr;            // sqrt(s2)
    float* d_slog = nullptr;              // log2(sqrt(s2)), -inf for 0
    double* d_pq = nullptr;               // squared P shell-block norms (per build)
    double* d_pnorm = nullptr;
    float* d_plog = nullptr;

    // device: tree + pyramids
    int32_t* d_node_lo = nullptr;
    int32_t* d_node_hi = nullptr;
    int32_t* d_node_child = nullptr;
    int32_t* d_node_nchild = nullptr;
    std::vector<int64_t> pyr_off;         // offset of level k in the pyramid arrays
    double* d_sq_s = nullptr;             // squared ||Q|| per level (dense)
    double* d_sq_p = nullptr;
    double* d_nrm_s = nullptr;            // sqrt of the above
    double* d_nrm_p = nullptr;
    int32_t* d_leaf_lo = nullptr;         // leaves (level depth) as tree ranges
    int32_t* d_leaf_hi = nullptr;

    // device: Boys table (FP64, FP32 and double-word copies of one table)
    double* d_boys64 = nullptr;
    float* d_boys32 = nullptr;
    float2* d_boysdw = nullptr;

    // device: pair tables, rebuilt per build
    int32_t* d_pairmap = nullptr;         // tree (a,b) -> slot in its class, -1 if absent
    kx::PairMeta* d_pairmeta[kx::NPAIRCLASS] = {};
    double* d_pair64[kx::NPAIRCLASS] = {};
    float* d_pair32[kx::NPAIRCLASS] = {};
    float2* d_pairdw[kx::NPAIRCLASS] = {};      // the FP64 records as double words (KX_MIXED_DW builds)
    int64_t pairdw_cap[kx::NPAIRCLASS] = {};
    int64_t pair_cap[kx::NPAIRCLASS] = {};
    int64_t n_pairs[kx::NPAIRCLASS] = {};

    // device: scratch (grow-only)
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    kx::Task* d_front[2] = {nullptr, nullptr};
    size_t front_cap[2] = {0, 0};
    uint16_t* d_mask = nullptr;
    size_t mask_cap = 0;
    int64_t* d_scan = nullptr;
    size_t scan_cap = 0;
    kx::Quartet* d_rec = nullptr;
    size_t rec_cap = 0;
    int64_t* d_bin = nullptr;             // per (stream, block) counts and offsets
    size_t bin_cap = 0;
    unsigned long long* d_counters = nullptr;   // small device counters
    kx::Task* d_keep = nullptr;                 // retained leaf worklist
    size_t keep_cap = 0, keep_n = 0;
    bool keep_valid = false;

    // FP32 and double-word copies of P for the mixed-precision kernels (same layout as P)
    float* d_P32 = nullptr;
    size_t P32_cap = 0;
    float2* d_Pdw = nullptr;
    size_t Pdw_cap = 0;
    // scan temporaries
    int64_t* d_scantmp = nullptr;
    size_t scantmp_cap = 0;

    // host-buffer entry point
    double* d_hostP = nullptr;
    double* d_hostK = nullptr;
    size_t host_cap = 0;

    double tau_ovlp = 0.0;
    double kept_tau = 0.0;                // tau of the traversal that made the kept list
    float* d_leafdesc = nullptr;          // per-leaf centroid, radius, max l, min exponent
    size_t leafdesc_cap = 0;
    kx::Task* d_list = nullptr;           // explicit leaf lists and compaction scratch
    size_t list_cap = 0;
    bool have_pq = false;
    int64_t launches = 0;                 // kernels launched by the current build
    // launch shape of every (precision, class) stream: threads per block and
    // persistent blocks per SM (0 = one thread per record); see kx_autotune
    int eri_threads[kx::NSTREAM] = {};
    int eri_bpsm[kx::NSTREAM] = {};
    int eri_variant[kx::NSTREAM] = {};       // kernel variant of the stream
    bool eri_smem_set[kx::NSTREAM][3] = {};  // dynamic shared memory limit raised, per variant
    int n_sm = 0;
    bool tuned[kx::NSTREAM] = {};
    // what the last eager build saw (sizes for a captured plan)
    int64_t plan_max_rec = 0;             // largest record count of one leaf chunk
    double rec_per_leaf = 48.0;           // shell-quartet records per leaf quartet (last build, with margin):
                                          // sizes the leaf chunks of eager builds
    int64_t last_lq = 1 << 16;            // leaf quartets per chunk of the last eager build
    uint8_t plan_active[kx::NSTREAM] = {};
    // autotuning inside an eager build (kx_autotune)
    bool tuning = false;
    double* d_tuneK = nullptr;
    size_t tuneK_cap = 0;
    // captured build (kx_graph_plan / kx_graph_launch)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_valid = false;
    int64_t graph_launches = 0;
    int graph_depth = 0;
    int64_t* d_gw = nullptr;              // device words of the captured build
    int64_t* h_gw = nullptr;              // pinned host copy of its statistics
    size_t gw_n = 0;
    kx::Task* d_groots = nullptr;
    uint8_t* d_gactive = nullptr;
    int64_t graph_st0 = 0;                // statistics block in d_gw
    cudaStream_t gstream = nullptr;       // capture and replay stream
    // per-stream profile of the last profiled build
    double prof_ms[kx::NSTREAM] = {};
    int64_t prof_n[kx::NSTREAM] = {};
    double prof_flops[kx::NSTREAM] = {};
    int32_t prof_launches[kx::NSTREAM] = {};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
    // split planning (kx_split_plan): sampled K shell blocks -> slot (dense
    // over shell pairs, -1 = not sampled) and their per-bin FP32 sums,
    // present only during the planning count; per-class error constants
    int32_t* plan_slot = nullptr;
    double* plan_acc = nullptr;
    float plan_lbin0 = 0.f;
    int plan_nbin = 0;
    float* d_cmax = nullptr;
    float* d_crms = nullptr;
    double graph_split = 0.0;             // split of the captured build (its plan may have chosen it)
    double graph_err_bound = 0.0, graph_err_est = 0.0;
    // per-row-leaf work of a kx_row_work count (null otherwise) and the
    // FLOPs of one quartet of every stream
    double* work_acc = nullptr;
    double* d_work = nullptr;
    size_t work_cap = 0;
    float* d_sflops = nullptr;
};

namespace kx {

// error helpers ---------------------------------------------------------------
int set_err(kx_ctx* c, int code, const std::string& msg);
int cuda_check(kx_ctx* c, cudaError_t e, const char* what);
#define KX_CUDA(c, call)                                   \
    do {                                                   \
        cudaError_t _e = (call);                           \
        if (_e != cudaSuccess) return kx::cuda_check(c, _e, #call); \
    } while (0)
#define KX_TRY(call)                 \
    do {                             \
        int _r = (call);             \
        if (_r != KX_OK) return _r;  \
    } while (0)

template <typename T>
int grow(kx_ctx* c, T** p, size_t* cap, size_t need) {
    if (need <= *cap && *p) return KX_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t n = need + need / 4 + 64;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return set_err(c, KX_ENOMEM, "device allocation of " + std::to_string(n * sizeof(T)) + " bytes failed");
    }
    *cap = n;
    return KX_OK;
}

// stage entry points (defined in the .cu files) ------------------------------
int order_atoms(kx_ctx* c);                                  // kx_setup.cu
int schwarz(kx_ctx* c, double tau_ovlp);                      // kx_setup.cu
int build_tree(kx_ctx* c, int leaf_max);                      // kx_setup.cu
int boys_table(kx_ctx* c);                                    // kx_setup.cu
// P/K addressing of the current build: ldp = ldk = 0 means packed per system
int set_frames(kx_ctx* c, int64_t ldp, int64_t ldk, bool packed);   // kx_setup.cu
int p_norms(kx_ctx* c, const double* P);                      // kx_setup.cu
// dw: also fill the double-word copies of the FP64 pair records
int pair_tables(kx_ctx* c, double tau, bool screen, bool dw);          // kx_setup.cu
int pair_tables_dev(kx_ctx* c, double tau, bool screen, bool dw);      // kx_setup.cu, capture-safe
int exclusive_scan(kx_ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_host);  // kx_traverse.cu
// K(mu,nu) = K(nu,mu) wherever the shell of mu comes after the shell of nu
// in tree order (the half a symmetric build leaves out)
int mirror_k(kx_ctx* c, double* K);                           // kx_traverse.cu
int traverse_and_evaluate(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o,
                          double* K, int64_t ldk, kx_stats* st);  // kx_traverse.cu
// what one driver call does: the whole build, the traversal alone (the leaf
// list is kept), or the ERI stage over an explicit device leaf list
// RUN_COUNT: traversal and the shell screen's count pass only (no records, no K)
enum { RUN_EXCHANGE = 0, RUN_TRAVERSE = 1, RUN_EVALUATE = 2, RUN_COUNT = 3 };
int drive(kx_ctx* c, int mode, const double* P, int64_t ldp, const kx_opts* o, double* K, int64_t ldk,
          kx_stats* st, const Task* list, int64_t nlist);
void drop_graph(kx_ctx* c);
// captured builds and the launch-shape autotuner (kx_traverse.cu); P and K packed
int graph_plan(kx_ctx* c, const double* P, const kx_opts* o, double* K, double headroom, kx_stats* st);
int graph_launch(kx_ctx* c, kx_stats* st);
// split threshold of a mixed build from the FP32 error model (kx_split.cu):
// fills st->split_used, fp32_err_estimate, fp32_err_bound
int split_plan(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double budget, kx_stats* st);
int autotune(kx_ctx* c, const double* P, const kx_opts* o, double* K, kx_stats* st, int* n_tuned);

// shell expansion + class kernels (kx_expand.cu, kx_eri_*.cu)
struct ClassCounts {
    int64_t n[NSTREAM];        // [precision][class]; precision 0 = FP64
};
// Shell-screen passes over a list of leaf quartets.  expand_count writes
// the number of kept quartets of every (stream, block) into bin[stream *
// blocks + block] (blocks = expand_blocks(n)); after an exclusive scan of
// bin, expand_write puts every record at its block's offset in its stream.
unsigned expand_blocks(const kx_ctx* c, int64_t n_leaves);
int expand_count(kx_ctx* c, const Task* leaves, int64_t n_leaves, double tau, double split,
                 int mixed, int shell_screen, int64_t* bin);
int expand_write(kx_ctx* c, const Task* leaves, int64_t n_leaves, double tau, double split,
                 int mixed, int shell_screen, int64_t* bin_off, Quartet* rec);
// capture-safe variants: the leaf count is the device word *dn (cap bounds
// it and fixes the grid, expand_blocks(cap))
int expand_count_dev(kx_ctx* c, const Task* leaves, int64_t cap, const int64_t* dn, double tau, double split,
                     int mixed, int shell_screen, int64_t* bin);
int expand_write_dev(kx_ctx* c, const Task* leaves, int64_t cap, const int64_t* dn, double tau, double split,
                     int mixed, int shell_screen, int64_t* bin_off, Quartet* rec);
int exclusive_scan_dev(kx_ctx* c, const int64_t* in, int64_t* out, int64_t n, const int64_t* dn, int64_t* grand);
size_t scan_scratch(int64_t n);

// ERI class kernels (kx_eri_impl.cuh).  Launch shapes: any multiple of 32
// threads up to ERI_MAX_THREADS; the grid strides over the records, so a
// persistent grid (a few blocks per SM) and one thread per record run the
// same code.
constexpr int ERI_THREADS = 128;       // default block size
constexpr int ERI_MAX_THREADS = 256;

// The records of one (class, precision) stream: rec[i] for i in [i0, i1),
// or, with range != nullptr, in [range[0], range[1]) read on the device.
// P is the FP64 P or its FP32 copy (same layout); both are addressed
// through the pair tables' row bases.
struct EriArgs {
    const Quartet* rec;
    int64_t i0, i1;
    const int64_t* range;
    const PairMeta* bmeta;
    const PairMeta* kmeta;
    const void* bra;
    const void* ket;
    const void* boys;
    const void* P;
    double* K;
    int64_t nab, ncd;
};
typedef void (*EriKernel)(EriArgs);
// a class kernel and the dynamic shared memory it needs per thread of a block
struct EriKern {
    EriKernel k;
    int smem_per_thread;
    int n_variants;       // kernels available for this stream (see eri_kernel)
};

EriKern eri_kernel(int cls, int prec, int variant);   // kx_expand.cu, over the nine below
// double-word kernels of the classes with la+lb+lc+ld <= DW_LMAX (else null)
EriKern eri_kernel_dw(int cls);                       // kx_expand.cu, over the nine below
EriKern eri_kernel_dw_ab00(int cls);
EriKern eri_kernel_dw_ab01(int cls);
EriKern eri_kernel_dw_ab02(int cls);
EriKern eri_kernel_dw_ab10(int cls);
EriKern eri_kernel_dw_ab11(int cls);
EriKern eri_kernel_dw_ab12(int cls);
EriKern eri_kernel_dw_ab20(int cls);
EriKern eri_kernel_dw_ab21(int cls);
EriKern eri_kernel_dw_ab22(int cls);
// the ket-pruned FP64 and FP32 kernels of a class with la+lb+lc+ld >= 7
EriKern eri_kernel_big64p(int cls);
EriKern eri_kernel_bigp(int cls);
EriKern eri_kernel_ab00(int cls, int prec, int variant);
EriKern eri_kernel_ab01(int cls, int prec, int variant);
EriKern eri_kernel_ab02(int cls, int prec, int variant);
EriKern eri_kernel_ab10(int cls, int prec, int variant);
EriKern eri_kernel_ab11(int cls, int prec, int variant);
EriKern eri_kernel_ab12(int cls, int prec, int variant);
EriKern eri_kernel_ab20(int cls, int prec, int variant);
EriKern eri_kernel_ab21(int cls, int prec, int variant);
EriKern eri_kernel_ab22(int cls, int prec, int variant);
double class_flops_ab00(int cls);
double class_flops_ab01(int cls);
double class_flops_ab02(int cls);
double class_flops_ab10(int cls);
double class_flops_ab11(int cls);
double class_flops_ab12(int cls);
double class_flops_ab20(int cls);
double class_flops_ab21(int cls);
double class_flops_ab22(int cls);
// arguments of stream (cls, prec) over rec[i0, i1) (or the device range)
EriArgs eri_args(kx_ctx* c, int cls, int prec, const Quartet* rec, int64_t i0, int64_t i1,
                 const int64_t* range, const double* P, double* K);
// launches the class kernel of stream (cls, prec) with the context's launch
// shape for that stream
int eri_launch(kx_ctx* c, int cls, int prec, const Quartet* rec, int64_t i0, int64_t i1, const int64_t* range,
               const double* P, double* K);
// threads per block a stream's kernel can use (its shared memory bounds it),
// and the dynamic shared memory of a launch of that many threads; raises the
// kernel's shared-memory limit once per context
int eri_fit_threads(const EriKern& k, int threads);
int eri_prepare(kx_ctx* c, int s, int variant, const EriKern& k);

// algorithmic FLOPs of one shell quartet of a class (the counter of the ERI kernels)
double class_flops(int cls);
// the part of it that does not depend on P: P-Q, rho, T and the prefactor,
// the Boys function (Taylor) with its scaling, and the Hermite recursion of
// R_tuv for t+u+v <= L (every class of total angular momentum L alike); the
// rest of class_flops is the contraction with P through the Hermite sets
inline double integral_flops(int L) {
    double f = 20;                            // P-Q, rho, T, prefactor
    f += 6 + (L + 1) * (2 * 6 + 1) + L;       // Boys (Taylor) and scaling
    for (int n = L - 1; n >= 0; --n)          // Hermite recursion
        for (int j = L - n; j >= 1; --j)
            for (int t = j; t >= 0; --t)
                for (int u = j - t; u >= 0; --u) {
                    const int v = j - t - u;
                    const int k = t > 0 ? t : (u > 0 ? u : v);
                    f += (k > 1) ? 3 : 1;
                }
    return f;
}
int peak_probe(int device, int precision, double* gflops);   // kx_setup.cu

}  // namespace kx
