// kx_traverse.cu -- the hextree traversal of Eq. 7 with the metric query of
// Eq. 8, run level-synchronously on the GPU, and the driver that feeds its
// surviving leaf quartets to the shell-quartet screen and the ERI kernels.
//
// Level k holds a frontier of tasks (A,B,C,D) of level-k nodes.  One pass
// evaluates, for every task, the bound of each of its children
//     beta = (||Q_{A'B'}||_F * ||P_{B'D'}||_F) * ||Q_{C'D'}||_F
// (IEEE products, no fused multiply-add) and records the survivors
// (beta > tau) as a 16-bit mask; an exclusive scan of the survivor counts
// gives every child its slot, and a second pass writes the next frontier.
// Children are written in the order (iA, iB, iC, iD), A most significant, so
// the frontier is deterministic.  A level-k node that is a leaf has itself
// as its only child, so leaves reached early ride along to the deepest
// level.  The last level is produced in chunks whose size bounds the memory
// of the leaf list and of the shell-quartet records made from it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "kx_traverse_impl.cuh"

namespace kx {

// ===========================================================================
// device-wide exclusive scan of int64
// ===========================================================================

constexpr int SCAN_T = 256;
constexpr int SCAN_I = 16;
constexpr int SCAN_TILE = SCAN_T * SCAN_I;

// n = *dn when dn is given (the grid then covers a capacity >= *dn)
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int64_t* __restrict__ in, int64_t n,
                                                       const int64_t* __restrict__ dn,
                                                       int64_t* __restrict__ tile_sum) {
    __shared__ int64_t sh[32];
    if (dn) n = min(n, *dn);
    const int64_t base = blockIdx.x * (int64_t)SCAN_TILE + threadIdx.x * (int64_t)SCAN_I;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k)
        if (base + k < n) s += in[base + k];
    int64_t total;
    block_excl_scan64(s, sh, &total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const int64_t* __restrict__ in, int64_t n,
                                                       const int64_t* __restrict__ dn,
                                                       const int64_t* __restrict__ tile_off,
                                                       int64_t* __restrict__ out, int64_t* __restrict__ grand) {
    __shared__ int64_t sh[32];
    if (dn) n = min(n, *dn);
    const int64_t base = blockIdx.x * (int64_t)SCAN_TILE + threadIdx.x * (int64_t)SCAN_I;
    int64_t v[SCAN_I];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int64_t total;
    int64_t off = block_excl_scan64(s, sh, &total) + (tile_off ? tile_off[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        if (base + k < n) out[base + k] = off;
        off += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) *grand = off;
}

static size_t scan_tmp_need(int64_t n) {
    size_t need = 4;
    while (n > SCAN_TILE) {
        int64_t t = (n + SCAN_TILE - 1) / SCAN_TILE;
        need += 2 * (size_t)t + 2;
        n = t;
    }
    return need;
}

// dn (device, may be null) bounds the outermost level; the tile grids are
// sized by the capacity n, entries beyond *dn count as zero
static int scan_rec(cudaStream_t st, const int64_t* in, int64_t* out, int64_t n, const int64_t* dn, int64_t* tmp,
                    int64_t* grand) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles <= 1) {
        k_scan_apply<<<1, SCAN_T, 0, st>>>(in, n, dn, nullptr, out, grand);
        return 1;
    }
    int64_t* tsum = tmp;
    int64_t* toff = tmp + tiles;
    int64_t* inner_grand = tmp + 2 * tiles;
    k_scan_tiles<<<(unsigned)tiles, SCAN_T, 0, st>>>(in, n, dn, tsum);
    int k = scan_rec(st, tsum, toff, tiles, nullptr, tmp + 2 * tiles + 2, inner_grand);
    k_scan_apply<<<(unsigned)tiles, SCAN_T, 0, st>>>(in, n, dn, toff, out, grand);
    return k + 2;
}

int exclusive_scan(kx_ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_host) {
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return KX_OK;
    }
    KX_TRY(grow(c, &c->d_scantmp, &c->scantmp_cap, scan_tmp_need(n) + 8));
    int64_t* grand = c->d_scantmp;
    c->launches += scan_rec(c->stream, in, out, n, nullptr, c->d_scantmp + 8, grand);
    if (total_host) {
        KX_CUDA(c, cudaMemcpyAsync(total_host, grand, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        KX_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return KX_OK;
}

// the same without any host read-back (capture-safe): the total goes to the
// device word *grand; the scratch must have been grown for capacity n
int exclusive_scan_dev(kx_ctx* c, const int64_t* in, int64_t* out, int64_t n, const int64_t* dn, int64_t* grand) {
    if (n <= 0) return KX_OK;
    if (c->scantmp_cap < scan_tmp_need(n) + 8) return set_err(c, KX_ECAPACITY, "scan scratch not reserved");
    c->launches += scan_rec(c->stream, in, out, n, dn, c->d_scantmp + 8, grand);
    return KX_OK;
}

size_t scan_scratch(int64_t n) { return scan_tmp_need(n) + 8; }

// ===========================================================================
// traversal kernels
// ===========================================================================

// bound of every child of every task at the next level; survivors as a mask.
// The next level's norms of the task's system sit at t0 + X * n + Y
// (block lseg_next[system]).
__global__ void k_expand_mask(const Task* __restrict__ front, int64_t n, const int32_t* __restrict__ child,
                              const int32_t* __restrict__ nchild, const int32_t* __restrict__ node_sys,
                              const Seg* __restrict__ lseg_next, const double* __restrict__ S,
                              const double* __restrict__ Pn, double tau, uint16_t* __restrict__ mask,
                              int64_t* __restrict__ cnt, const int64_t* __restrict__ dn, int sym,
                              const RowRange rows) {
    if (dn) n = min(n, *dn);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Task t = front[i];
        // symmetric build: only K blocks (A,C) with A <= C
        const Seg g = lseg_next[node_sys[t.a]];
        const unsigned m = task_child_mask(t, child, nchild, S, Pn, g.t0(), g.n, tau, sym && t.a == t.c, rows);
        mask[i] = (uint16_t)m;
        cnt[i] = __popc(m);
    }
}

// parents [p0, p1) write their surviving children at off - obase; with
// drange (device: p0, p1, obase) the range comes from the device
__global__ void k_expand_write(const Task* __restrict__ front, int64_t p0, int64_t p1,
                               const uint16_t* __restrict__ mask, const int64_t* __restrict__ off, int64_t obase,
                               const int32_t* __restrict__ child, Task* __restrict__ out,
                               const int64_t* __restrict__ drange) {
    if (drange) {
        p0 = drange[0];
        p1 = drange[1];
        obase = drange[2];
    }
    for (int64_t i = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p1;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned m = mask[i];
        if (!m) continue;
        write_children(front[i], m, child, out, off[i] - obase, INT64_MAX);
    }
}

// trees that are single leaves: the root task of every system, kept iff its
// bound exceeds tau, in system order (one thread: only for tiny systems)
__global__ void k_root_only(const Seg* __restrict__ lseg0, int nsys, const double* __restrict__ S,
                            const double* __restrict__ Pn, double tau, Task* __restrict__ out,
                            int64_t* __restrict__ n_out, int leaf0, int leaf1) {
    int64_t k = 0;
    for (int y = leaf0; y < leaf1; ++y) {
        const int64_t i = lseg0[y].off;   // the block of a one-node level: (y, y)
        const double beta = __dmul_rn(__dmul_rn(S[i], Pn[i]), S[i]);
        if (beta > tau) out[k++] = Task{(uint16_t)y, (uint16_t)y, (uint16_t)y, (uint16_t)y};
    }
    n_out[0] = k;
}

// chunk boundaries: b_j = first parent whose output offset is >= j * cap
__global__ void k_chunk_bounds(const int64_t* __restrict__ off, int64_t n, int64_t cap, int nch,
                               int64_t* __restrict__ bounds) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > nch) return;
    if (j == 0) { bounds[0] = 0; return; }
    if (j == nch) { bounds[j] = n; return; }
    int64_t target = (int64_t)j * cap, a = 0, b = n;
    while (a < b) {
        int64_t m = (a + b) >> 1;
        if (off[m] < target) a = m + 1; else b = m;
    }
    bounds[j] = a;
}

// K(mu,nu) = K(nu,mu) where the shell of mu follows the shell of nu in tree
// order: those entries were left out by a symmetric build; the ones read
// are never written here
__global__ void k_mirror(const Seg* __restrict__ fseg, int nsys, int64_t total, const MatFrame* __restrict__ mf,
                         const int32_t* __restrict__ ftpos, double* __restrict__ K) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int y = seg_find(fseg, nsys, e);
        const Seg g = fseg[y];
        const int64_t r = e - g.off;
        const int mu = g.base + (int)(r / g.n), nu = g.base + (int)(r % g.n);
        if (ftpos[mu] > ftpos[nu]) {
            const MatFrame f = mf[y];
            K[f.k0 + (int64_t)mu * f.ldk + nu] = K[f.k0 + (int64_t)nu * f.ldk + mu];
        }
    }
}

// FP32 copy of P in the same layout: n rows of n entries at stride ldp
// (a packed batch is one row of all its entries)
__global__ void k_to_f32(const double* __restrict__ P, int64_t ldp, int64_t rows, int64_t n,
                         float* __restrict__ P32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (i / n) * ldp + (i % n);
        P32[j] = __double2float_rn(P[j]);
    }
}

// double-word copy of P (hi = nearest float, lo = the rounded remainder)
__global__ void k_to_dw(const double* __restrict__ P, int64_t ldp, int64_t rows, int64_t n,
                        float2* __restrict__ Pdw) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows * n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (i / n) * ldp + (i % n);
        const double x = P[j];
        const float hi = __double2float_rn(x);
        Pdw[j] = make_float2(hi, __double2float_rn(x - (double)hi));
    }
}

// ===========================================================================
// driver
// ===========================================================================

int mirror_k(kx_ctx* c, double* K) {
    const int64_t total = c->sys_mat[c->n_sys];
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)c->n_sm * 32);
    k_mirror<<<g, 256, 0, c->stream>>>(c->d_fseg, c->n_sys, total, c->d_mframe, c->d_ftpos, K);
    c->launches++;
    return KX_OK;
}

void drop_graph(kx_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->graph_valid = false;
}


namespace {

struct Timer {
    kx_ctx* c;
    std::vector<std::pair<cudaEvent_t, int>> marks;   // event, stage that starts
    void mark(int stage) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, c->stream);
        marks.push_back({e, stage});
    }
    void finish(double* ms) {   // ms[stage] += elapsed until the next mark
        for (size_t i = 0; i + 1 < marks.size(); ++i) {
            float t = 0.f;
            cudaEventElapsedTime(&t, marks[i].first, marks[i + 1].first);
            if (marks[i].second >= 0) ms[marks[i].second] += t;
        }
        for (auto& m : marks) cudaEventDestroy(m.first);
        marks.clear();
    }
};

enum { ST_NORMS = 0, ST_TRAV = 1, ST_EXPAND = 2, ST_ERI = 3, ST_NONE = -1 };

struct Run {
    kx_ctx* c;
    const double* P;
    int64_t ldp;
    const kx_opts* o;
    double* K;
    int64_t ldk;
    kx_stats* st;
    Timer* tm;
    int64_t rec_limit;
    double eri_max_ms;
    bool count_only;
};

int process_leaves(Run& r, const Task* leaves, int64_t n);
int finish_run(kx_ctx* c, kx_stats* st, Timer& tm, int D);

// Launch-shape autotuner of one (precision, class) stream: times every
// candidate on (a prefix of) the stream's records, accumulating into a
// scratch K, and keeps the fastest.  Candidates: each kernel variant of the
// stream (the FP64 large classes have two), with 64, 128 and 256 threads per
// block (as far as its shared memory allows), each with one thread per
// record or a persistent grid of 1x or 2x the blocks that fit on an SM.
constexpr int64_t TUNE_MIN = 1 << 14;      // records needed to tune a stream
constexpr int64_t TUNE_MAX = 1 << 19;      // records timed per candidate
int tune_stream(kx_ctx* c, int s, const Quartet* rec, int64_t i0, int64_t i1, const double* P) {
    if (i1 - i0 < TUNE_MIN) return KX_OK;
    const int prec = s / NCLASS, cls = s % NCLASS;
    const int nvar = eri_kernel(cls, prec, 0).n_variants;
    const int64_t j1 = std::min(i1, i0 + TUNE_MAX);
    const EriArgs args = eri_args(c, cls, prec, rec, i0, j1, nullptr, P, c->d_tuneK);
    cudaEvent_t e0, e1;
    KX_CUDA(c, cudaEventCreate(&e0));
    KX_CUDA(c, cudaEventCreate(&e1));
    float best = 1e30f;
    int bt = ERI_THREADS, bb = 0, bv = 0;
    for (int variant = 0; variant < nvar; ++variant) {
    const EriKern kk = eri_kernel(cls, prec, variant);
    if (!kk.k) return set_err(c, KX_EINVAL, "bad class");
    KX_TRY(eri_prepare(c, s, variant, kk));
    EriKernel k = kk.k;
    for (int threads : {64, 128, 256}) {
        if (eri_fit_threads(kk, threads) != threads) continue;
        const size_t smem = (size_t)threads * kk.smem_per_thread;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem) != cudaSuccess || occ < 1) {
            (void)cudaGetLastError();
            continue;
        }
        for (int bpsm : {0, occ, 2 * occ}) {
            int64_t blocks = (j1 - i0 + threads - 1) / threads;
            if (bpsm > 0) blocks = std::min<int64_t>(blocks, (int64_t)bpsm * c->n_sm);
            float t = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, c->stream);
                k<<<(unsigned)blocks, threads, smem, c->stream>>>(args);
                cudaEventRecord(e1, c->stream);
                KX_CUDA(c, cudaEventSynchronize(e1));
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t += ms;   // the first launch warms the caches
            }
            if (t < best) {
                best = t;
                bt = threads;
                bb = bpsm;
                bv = variant;
            }
        }
    }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    KX_CUDA(c, cudaGetLastError());
    c->eri_threads[s] = bt;
    c->eri_bpsm[s] = bb;
    c->eri_variant[s] = bv;
    c->tuned[s] = true;
    return KX_OK;
}

// adds n shell quartets of stream s to the build's counters
void add_stream_stats(kx_stats* st, int s, int64_t n) {
    const double f = class_flops(s % NCLASS) * (double)n;
    st->n_shell_quartets += n;
    switch (s / NCLASS) {
        case 0: st->flops_fp64 += f; st->n_shell_quartets_fp64 += n; break;
        case 1: st->flops_fp32 += f; break;
        default: st->flops_dw += f; st->n_shell_quartets_dw += n; break;
    }
}

// shell screen, class binning and class kernels for one list of leaf quartets
int process_leaves(Run& r, const Task* leaves, int64_t n) {
    kx_ctx* c = r.c;
    if (n <= 0) return KX_OK;
    const int mixed = r.o->precision;
    const double split = mixed ? r.o->split_threshold : 0.0;
    r.tm->mark(ST_EXPAND);
    const unsigned nb = expand_blocks(c, n);
    const int64_t nbin = (int64_t)NSTREAM * nb;
    KX_TRY(grow(c, &c->d_bin, &c->bin_cap, (size_t)(2 * nbin)));
    int64_t* bin = c->d_bin;
    int64_t* binoff = c->d_bin + nbin;
    KX_TRY(expand_count(c, leaves, n, r.o->tau, split, mixed, r.o->shell_screen, bin));
    c->launches++;
    int64_t total = 0;
    KX_TRY(exclusive_scan(c, bin, binoff, nbin, &total));
    c->plan_max_rec = std::max(c->plan_max_rec, total);
    if (total > r.rec_limit && n > 1 && !r.count_only) {
        // too many records for one pass: pieces of about 0.9 rec_limit records
        // each (a piece that still overflows splits again)
        const int64_t m = std::min<int64_t>(n, std::max<int64_t>(2, (int64_t)(1.1 * (double)total / r.rec_limit) + 1));
        for (int64_t i = 0; i < m; ++i) {
            const int64_t i0 = n * i / m, i1 = n * (i + 1) / m;
            if (i1 > i0) KX_TRY(process_leaves(r, leaves + i0, i1 - i0));
        }
        return KX_OK;
    }
    if (total == 0) return KX_OK;
    // stream s starts at binoff[s * nb]
    int64_t off[NSTREAM + 1];
    KX_CUDA(c, cudaMemcpy2DAsync(off, sizeof(int64_t), binoff, sizeof(int64_t) * nb, sizeof(int64_t), NSTREAM,
                                 cudaMemcpyDeviceToHost, c->stream));
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    off[NSTREAM] = total;
    unsigned long long h[NSTREAM], endv[NSTREAM];
    for (int s = 0; s < NSTREAM; ++s) {
        h[s] = (unsigned long long)(off[s + 1] - off[s]);
        endv[s] = (unsigned long long)off[s + 1];
    }
    if (r.count_only) {
        for (int s = 0; s < NSTREAM; ++s) {
            add_stream_stats(r.st, s, (int64_t)h[s]);
            c->prof_n[s] += (int64_t)h[s];
        }
        r.st->n_chunks++;
        return KX_OK;
    }
    KX_TRY(grow(c, &c->d_rec, &c->rec_cap, (size_t)total));
    KX_CUDA(c, cudaMemcpyAsync(c->d_counters + CTR_END, endv, sizeof(endv), cudaMemcpyHostToDevice, c->stream));
    KX_TRY(expand_write(c, leaves, n, r.o->tau, split, mixed, r.o->shell_screen, binoff, c->d_rec));
    c->launches++;
    r.tm->mark(ST_ERI);
    for (int s = 0; s < NSTREAM; ++s) {
        if (!h[s]) continue;
        const int prec = s / NCLASS, cls = s % NCLASS;
        c->plan_active[s] = 1;
        if (c->tuning && !c->tuned[s]) KX_TRY(tune_stream(c, s, c->d_rec, off[s], off[s + 1], r.P));
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (r.o->profile) {
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            cudaEventRecord(e0, c->stream);
        }
        KX_TRY(eri_launch(c, cls, prec, c->d_rec, off[s], off[s + 1], nullptr, r.P, r.K));
        if (r.o->profile) {
            cudaEventRecord(e1, c->stream);
            c->prof_ev.push_back({s, {e0, e1}});
        }
        c->launches++;
        add_stream_stats(r.st, s, (int64_t)h[s]);
        c->prof_n[s] += (int64_t)h[s];
        c->prof_flops[s] += class_flops(cls) * (double)h[s];
        c->prof_launches[s] += 1;
    }
    r.st->n_chunks++;
    KX_CUDA(c, cudaGetLastError());
    return KX_OK;
}

int keep_leaves(kx_ctx* c, const Task* leaves, int64_t n) {
    if (n <= 0) return KX_OK;
    if (c->keep_n + n > c->keep_cap) {
        Task* nb = nullptr;
        size_t cap = (c->keep_n + n) * 2 + 64;
        KX_CUDA(c, cudaMalloc(&nb, sizeof(Task) * cap));
        if (c->keep_n) cudaMemcpyAsync(nb, c->d_keep, sizeof(Task) * c->keep_n, cudaMemcpyDeviceToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        cudaFree(c->d_keep);
        c->d_keep = nb;
        c->keep_cap = cap;
    }
    KX_CUDA(c, cudaMemcpyAsync(c->d_keep + c->keep_n, leaves, sizeof(Task) * n, cudaMemcpyDeviceToDevice,
                               c->stream));
    c->keep_n += n;
    return KX_OK;
}

}  // namespace

// The leaves [*l0, *l1) of the build's K row-block shard (every leaf when
// the options name none); KX_EINVAL for a range outside the leaves.
int row_leaves(kx_ctx* c, const kx_opts* o, int* l0, int* l1) {
    const int nl = c->levels[c->depth].n;
    if (o->row_leaf_lo == 0 && o->row_leaf_hi == 0) {
        *l0 = 0;
        *l1 = nl;
        return KX_OK;
    }
    if (o->row_leaf_lo < 0 || o->row_leaf_lo >= o->row_leaf_hi || o->row_leaf_hi > nl)
        return set_err(c, KX_EINVAL, "row_leaf_lo/row_leaf_hi must satisfy 0 <= lo < hi <= " + std::to_string(nl));
    *l0 = o->row_leaf_lo;
    *l1 = o->row_leaf_hi;
    return KX_OK;
}

// The shard's row filter for the children at `level` (no filter when the
// shard is every leaf)
RowRange row_range(const kx_ctx* c, const kx_opts* o, int level) {
    const int nl = c->levels[c->depth].n;
    if ((o->row_leaf_lo == 0 && o->row_leaf_hi == 0) || (o->row_leaf_lo == 0 && o->row_leaf_hi == nl))
        return RowRange{nullptr, nullptr, 0, 0};
    const int lv = c->levels[c->depth].off;
    return RowRange{c->d_node_lo + c->levels[level].off, c->d_node_hi + c->levels[level].off,
                    c->node_lo[lv + o->row_leaf_lo], c->node_hi[lv + o->row_leaf_hi - 1]};
}

int drive(kx_ctx* c, int mode, const double* P, int64_t ldp, const kx_opts* o, double* K, int64_t ldk,
          kx_stats* st, const Task* list, int64_t nlist) {
    const int D = c->depth;
    int rl0 = 0, rl1 = 0;
    KX_TRY(row_leaves(c, o, &rl0, &rl1));
    const bool evaluate = mode == RUN_EXCHANGE || mode == RUN_EVALUATE;
    // the leaf quartets go through the shell screen (count pass only for RUN_COUNT)
    const bool screen = evaluate || mode == RUN_COUNT;
    // an eager build may move the buffers a captured plan points to
    drop_graph(c);
    Timer tm{c, {}};
    Run r{c, P, ldp, o, K, ldk, st, &tm, 0, 0.0, mode == RUN_COUNT};
    // record budget per pass: the caller's, else 2^31 - 8192 records (16 GB;
    // the class kernels' record slots are 32-bit) or 40 % of the free device
    // memory, whichever is smaller
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const int64_t lim = std::min<int64_t>(((int64_t)1 << 31) - 8192, (int64_t)(0.4 * (double)fr / sizeof(Quartet)));
    r.rec_limit = o->chunk_records > 0 ? o->chunk_records : std::max<int64_t>(lim, 1 << 20);
    r.rec_limit = std::min<int64_t>(r.rec_limit, ((int64_t)1 << 31) - 8192);
    // leaf quartets per chunk: a pass's worth of records at the record rate
    // per leaf quartet of the previous build
    const int64_t lq_cap = std::max<int64_t>((int64_t)((double)r.rec_limit / std::max(4.0, c->rec_per_leaf)), 1 << 16);
    c->last_lq = lq_cap;

    c->launches = 0;
    c->plan_max_rec = 0;
    for (int s = 0; s < NSTREAM; ++s) {
        c->plan_active[s] = 0;
        c->prof_ms[s] = 0.0;
        c->prof_n[s] = 0;
        c->prof_flops[s] = 0.0;
        c->prof_launches[s] = 0;
    }
    for (auto& pe : c->prof_ev) {
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    c->prof_ev.clear();
    // ldp = ldk = 0: P and K are packed per system
    const bool packed = ldp == 0 && ldk == 0;
    KX_TRY(set_frames(c, ldp, ldk, packed));
    c->build_sym = o->symmetric;
    tm.mark(ST_NORMS);
    const int64_t mat_total = c->sys_mat[c->n_sys];
    if (evaluate) {
        if (packed)
            KX_CUDA(c, cudaMemsetAsync(K, 0, sizeof(double) * mat_total, c->stream));
        else
            KX_CUDA(c, cudaMemset2DAsync(K, sizeof(double) * ldk, 0, sizeof(double) * c->n_fn, c->n_fn, c->stream));
    }
    KX_TRY(p_norms(c, P));
    if (evaluate && o->precision != KX_FP64) {
        const int64_t rows = packed ? 1 : c->n_fn, cols = packed ? mat_total : c->n_fn, ld = packed ? 0 : ldp;
        KX_TRY(grow(c, &c->d_P32, &c->P32_cap, (size_t)((rows - 1) * ld + cols)));
        k_to_f32<<<1024, 256, 0, c->stream>>>(P, ld, rows, cols, c->d_P32);
        c->launches++;
        if (o->precision == KX_MIXED_DW) {
            KX_TRY(grow(c, &c->d_Pdw, &c->Pdw_cap, (size_t)((rows - 1) * ld + cols)));
            k_to_dw<<<1024, 256, 0, c->stream>>>(P, ld, rows, cols, c->d_Pdw);
            c->launches++;
        }
    }
    if (evaluate) KX_TRY(pair_tables(c, o->tau, o->shell_screen != 0, o->precision == KX_MIXED_DW));
    const bool keep = mode == RUN_TRAVERSE || (mode == RUN_EXCHANGE && o->keep_worklist);
    if (mode == RUN_EXCHANGE || mode == RUN_TRAVERSE) {
        c->keep_n = 0;
        c->keep_valid = false;
    }
    if (mode == RUN_EVALUATE) {
        // an explicit leaf-quartet list: the ERI stage in chunks of lq_cap
        st->n_leaf_quartets = nlist;
        for (int64_t i0 = 0; i0 < nlist; i0 += lq_cap)
            KX_TRY(process_leaves(r, list + i0, std::min<int64_t>(lq_cap, nlist - i0)));
        if (o->symmetric) KX_TRY(mirror_k(c, K));
        return finish_run(c, st, tm, D);
    }

    tm.mark(ST_TRAV);
    const double* S = c->d_nrm_s;
    const double* Pn = c->d_nrm_p;
    // level 0: the root task (Y, Y, Y, Y) of every system Y
    const int ny = c->n_sys;
    KX_TRY(grow(c, &c->d_front[0], &c->front_cap[0], (size_t)ny + 16));
    {
        std::vector<Task> roots(ny);
        for (int y = 0; y < ny; ++y) roots[y] = Task{(uint16_t)y, (uint16_t)y, (uint16_t)y, (uint16_t)y};
        KX_CUDA(c, cudaMemcpyAsync(c->d_front[0], roots.data(), sizeof(Task) * ny, cudaMemcpyHostToDevice,
                                   c->stream));
        KX_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    int64_t nfront = ny;
    int cur = 0;
    st->n_tasks[0] = ny;
    if (D == 0) {
        KX_TRY(grow(c, &c->d_scan, &c->scan_cap, 16));
        int64_t* d_n = c->d_scan;
        k_root_only<<<1, 1, 0, c->stream>>>(c->d_lseg, ny, S, Pn, o->tau, c->d_front[0], d_n, rl0, rl1);
        c->launches++;
        int64_t nk = 0;
        KX_CUDA(c, cudaMemcpyAsync(&nk, d_n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        KX_CUDA(c, cudaStreamSynchronize(c->stream));
        st->n_tasks[0] = nk;
        st->n_leaf_quartets = nk;
        if (keep) KX_TRY(keep_leaves(c, c->d_front[0], nk));
        if (screen) KX_TRY(process_leaves(r, c->d_front[0], nk));
    } else {
        for (int k = 0; k < D; ++k) {
            const int32_t* child = c->d_node_child + c->levels[k].off;
            const int32_t* nchild = c->d_node_nchild + c->levels[k].off;
            const int32_t* nsys = c->d_node_sys + c->levels[k].off;
            const Seg* lnext = c->d_lseg + (size_t)(k + 1) * ny;
            KX_TRY(grow(c, &c->d_mask, &c->mask_cap, (size_t)nfront));
            KX_TRY(grow(c, &c->d_scan, &c->scan_cap, (size_t)2 * nfront));
            int64_t* cnt = c->d_scan;
            int64_t* off = c->d_scan + nfront;
            unsigned g = (unsigned)std::min<int64_t>((nfront + 255) / 256, (int64_t)c->n_sm * 64);
            k_expand_mask<<<g, 256, 0, c->stream>>>(c->d_front[cur], nfront, child, nchild, nsys, lnext, S, Pn,
                                                    o->tau, c->d_mask, cnt, nullptr, o->symmetric,
                                                    row_range(c, o, k + 1));
            c->launches++;
            int64_t total = 0;
            KX_TRY(exclusive_scan(c, cnt, off, nfront, &total));
            st->n_tasks[k + 1] = total;
            if (k + 1 < D) {
                KX_TRY(grow(c, &c->d_front[1 - cur], &c->front_cap[1 - cur], (size_t)std::max<int64_t>(total, 1)));
                k_expand_write<<<g, 256, 0, c->stream>>>(c->d_front[cur], 0, nfront, c->d_mask, off, 0, child,
                                                         c->d_front[1 - cur], nullptr);
                c->launches++;
                cur = 1 - cur;
                nfront = total;
                if (total == 0) break;
                continue;
            }
            // last level: leaf quartets in chunks of at most lq_cap (+15)
            st->n_leaf_quartets = total;
            if (total == 0) break;
            const int nch = (int)((total + lq_cap - 1) / lq_cap);
            KX_TRY(grow(c, &c->d_front[1 - cur], &c->front_cap[1 - cur], (size_t)std::min<int64_t>(total, lq_cap + 16)));
            int64_t* d_bounds = nullptr;
            KX_CUDA(c, cudaMalloc(&d_bounds, sizeof(int64_t) * (nch + 1)));
            k_chunk_bounds<<<(nch + 1 + 127) / 128, 128, 0, c->stream>>>(off, nfront, lq_cap, nch, d_bounds);
            c->launches++;
            std::vector<int64_t> bounds(nch + 1);
            cudaMemcpyAsync(bounds.data(), d_bounds, sizeof(int64_t) * (nch + 1), cudaMemcpyDeviceToHost, c->stream);
            cudaError_t e = cudaStreamSynchronize(c->stream);
            cudaFree(d_bounds);
            if (e != cudaSuccess) return cuda_check(c, e, "chunk bounds");
            std::vector<int64_t> offh(1);
            for (int j = 0; j < nch; ++j) {
                const int64_t p0 = bounds[j], p1 = bounds[j + 1];
                if (p1 <= p0) continue;
                // output range of the chunk
                int64_t o0 = 0, o1 = 0;
                KX_CUDA(c, cudaMemcpyAsync(&o0, off + p0, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
                if (p1 < nfront)
                    KX_CUDA(c, cudaMemcpyAsync(&o1, off + p1, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
                KX_CUDA(c, cudaStreamSynchronize(c->stream));
                if (p1 >= nfront) o1 = total;
                tm.mark(ST_EXPAND);
                unsigned g2 = (unsigned)std::min<int64_t>((p1 - p0 + 255) / 256, (int64_t)c->n_sm * 64);
                k_expand_write<<<g2, 256, 0, c->stream>>>(c->d_front[cur], p0, p1, c->d_mask, off, o0, child,
                                                          c->d_front[1 - cur], nullptr);
                c->launches++;
                if (keep) KX_TRY(keep_leaves(c, c->d_front[1 - cur], o1 - o0));
                if (screen) KX_TRY(process_leaves(r, c->d_front[1 - cur], o1 - o0));
            }
        }
    }
    if (keep) c->keep_valid = true;
    if (evaluate && o->symmetric) KX_TRY(mirror_k(c, K));
    if (screen && st->n_leaf_quartets > 0 && st->n_shell_quartets > 0)
        c->rec_per_leaf = 1.25 * (double)st->n_shell_quartets / (double)st->n_leaf_quartets;
    return finish_run(c, st, tm, D);
}

namespace {

int finish_run(kx_ctx* c, kx_stats* st, Timer& tm, int D) {
    tm.mark(ST_NONE);
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    KX_CUDA(c, cudaGetLastError());
    double ms[4] = {0, 0, 0, 0};
    tm.finish(ms);
    st->ms_norms = ms[ST_NORMS];
    st->ms_traverse = ms[ST_TRAV];
    st->ms_expand = ms[ST_EXPAND];
    st->ms_eri = ms[ST_ERI];
    st->depth = D;
    double mx = 0.0;
    for (auto& pe : c->prof_ev) {
        float t = 0.f;
        cudaEventElapsedTime(&t, pe.second.first, pe.second.second);
        c->prof_ms[pe.first] += t;
        mx = std::max(mx, (double)t);
        cudaEventDestroy(pe.second.first);
        cudaEventDestroy(pe.second.second);
    }
    c->prof_ev.clear();
    st->ms_eri_kernel_max = mx;
    st->n_launches = (int32_t)c->launches;
    unsigned long long cand = 0, werr = 0;
    cudaMemcpy(&cand, c->d_counters + CTR_CAND, sizeof(cand), cudaMemcpyDeviceToHost);
    cudaMemcpy(&werr, c->d_counters + CTR_ERR, sizeof(werr), cudaMemcpyDeviceToHost);
    st->n_candidates = (int64_t)cand;
    if (werr) return set_err(c, KX_ECUDA, "shell-quartet count and write passes disagree");
    return KX_OK;
}

}  // namespace

int traverse_and_evaluate(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double* K, int64_t ldk,
                          kx_stats* st) {
    return drive(c, RUN_EXCHANGE, P, ldp, o, K, ldk, st, nullptr, 0);
}

// ===========================================================================
// captured builds: every launch sized from device words, one CUDA graph
// ===========================================================================
//
// A plan fixes, from an eager build of the same systems and options, the
// capacities of every buffer (frontiers, leaf chunks, shell-quartet
// records) with some headroom, and records the whole build -- P norms, pair
// tables, every traversal level, every leaf chunk's screen, binning and
// class-kernel launches -- into one CUDA graph.  No launch of the graph
// reads a size on the host: counts live in device words (layout below), the
// traversal and screen kernels stride over them with persistent grids, and
// the class kernels read their record ranges from the device.  A count that
// exceeds its capacity, or records of a class stream the plan did not
// launch, set an overflow word instead of writing out of bounds; the host
// checks it after the replay (KX_ECAPACITY: re-plan).  No kernel waits on
// another block, so no device-side wait exists that could time out.

namespace {

// device words of a captured build
struct GraphWords {
    int D, nch;
    int64_t n(int k) const { return k; }                    // level task counts [D + 1]
    int64_t t(int k) const { return 32 + k; }               // level totals (scan grands) [D + 1]
    int64_t wr(int k) const { return 64 + 3 * k; }          // write ranges of levels [D]
    int64_t ch(int j) const { return 160 + 4 * (int64_t)j; } // chunk: p0, p1, o0, n_leaf
    int64_t rg() const { return 160 + 4 * (int64_t)nch; }   // stream ranges [2 * NSTREAM]
    int64_t ne() const { return rg() + 2 * NSTREAM; }       // leaf count of the write pass
    int64_t bt() const { return ne() + 1; }                 // record total of a chunk
    int64_t st() const { return bt() + 1; }                 // statistics: records per stream [NSTREAM]
    int64_t lq() const { return st() + NSTREAM; }        // leaf quartets evaluated
    int64_t flag() const { return lq() + 1; }               // overflow
    int64_t size() const { return flag() + 3; }             // + two read-back slots
};

// next frontier size, or 0 (and the overflow word) when it exceeds cap;
// the write pass of the level covers its parents only when it fits
__global__ void k_level_check(const int64_t* __restrict__ total, const int64_t* __restrict__ n_parent,
                              int64_t cap, int64_t* __restrict__ n_next, int64_t* __restrict__ wr,
                              int64_t* __restrict__ flag) {
    const bool ok = *total <= cap;
    *n_next = ok ? *total : 0;
    wr[0] = 0;
    wr[1] = ok ? *n_parent : 0;
    wr[2] = 0;
    if (!ok) *flag = 1;
}

// chunk j of the last level: parents [p0, p1) whose children fill the
// leaf-quartet slots [j * lq, (j + 1) * lq) (rounded to whole parents)
__global__ void k_chunk_dev(const int64_t* __restrict__ off, const int64_t* __restrict__ n_parent,
                            const int64_t* __restrict__ total, int64_t lq, int j, int nch,
                            int64_t* __restrict__ ch, int64_t* __restrict__ flag) {
    const int64_t n = *n_parent, tot = *total;
    if (j == 0 && tot > (int64_t)nch * lq) *flag = 1;
    auto first_at = [&](int64_t target) {   // first parent with off >= target
        int64_t a = 0, b = n;
        while (a < b) {
            const int64_t m = (a + b) >> 1;
            if (off[m] < target) a = m + 1; else b = m;
        }
        return a;
    };
    const int64_t p0 = first_at((int64_t)j * lq);
    const int64_t p1 = (j + 1 == nch) ? n : first_at((int64_t)(j + 1) * lq);
    const int64_t o0 = p0 < n ? off[p0] : tot, o1 = p1 < n ? off[p1] : tot;
    const bool ok = tot <= (int64_t)nch * lq && o1 - o0 <= lq + 16;
    ch[0] = p0;
    ch[1] = ok ? p1 : p0;
    ch[2] = o0;
    ch[3] = ok ? o1 - o0 : 0;
    if (!ok) *flag = 1;
}

// record ranges of the chunk's class streams from the scanned bins; records
// beyond the capacity, or of a stream without a captured launch, void the
// chunk (the overflow word is set)
__global__ void k_stream_setup(const int64_t* __restrict__ binoff, int nb, const int64_t* __restrict__ total,
                               int64_t rec_cap, const uint8_t* __restrict__ active,
                               const int64_t* __restrict__ n_leaf, int64_t* __restrict__ ranges,
                               unsigned long long* __restrict__ end, int64_t* __restrict__ stats,
                               int64_t* __restrict__ n_eff, int64_t* __restrict__ lq_total,
                               int64_t* __restrict__ flag) {
    const int64_t tot = *total;
    bool ok = tot <= rec_cap;
    for (int s = threadIdx.x; s < NSTREAM; s += blockDim.x) {
        const int64_t a = binoff[(int64_t)s * nb], b = s + 1 < NSTREAM ? binoff[(int64_t)(s + 1) * nb] : tot;
        if (b > a && !active[s]) ok = false;
    }
    ok = __syncthreads_and(ok);
    for (int s = threadIdx.x; s < NSTREAM; s += blockDim.x) {
        const int64_t a = binoff[(int64_t)s * nb], b = s + 1 < NSTREAM ? binoff[(int64_t)(s + 1) * nb] : tot;
        ranges[2 * s] = ok ? a : 0;
        ranges[2 * s + 1] = ok ? b : 0;
        end[s] = ok ? (unsigned long long)b : 0ull;
        if (ok) stats[s] += b - a;
    }
    if (threadIdx.x == 0) {
        *n_eff = ok ? *n_leaf : 0;
        if (ok) *lq_total += *n_leaf;
        else *flag = 1;
    }
}

struct GraphCaps {
    int64_t fcap, mcap, lq, rec, nch;
};

// the screen, binning and class launches of one leaf list (capture-safe)
int chunk_dev(kx_ctx* c, const kx_opts* o, const GraphWords& W, const GraphCaps& cap, const Task* leaves,
              int64_t leaf_cap, const int64_t* dn, const double* P, double* K) {
    const int mixed = o->precision;
    const double split = mixed ? o->split_threshold : 0.0;
    const unsigned nb = expand_blocks(c, leaf_cap);
    const int64_t nbin = (int64_t)NSTREAM * nb;
    int64_t* bin = c->d_bin;
    int64_t* binoff = c->d_bin + nbin;
    int64_t* w = c->d_gw;
    KX_TRY(expand_count_dev(c, leaves, leaf_cap, dn, o->tau, split, mixed, o->shell_screen, bin));
    KX_TRY(exclusive_scan_dev(c, bin, binoff, nbin, nullptr, w + W.bt()));
    k_stream_setup<<<1, 256, 0, c->stream>>>(binoff, (int)nb, w + W.bt(), cap.rec, c->d_gactive, dn, w + W.rg(),
                                            c->d_counters + CTR_END, w + W.st(), w + W.ne(), w + W.lq(),
                                            w + W.flag());
    c->launches++;
    KX_TRY(expand_write_dev(c, leaves, leaf_cap, w + W.ne(), o->tau, split, mixed, o->shell_screen, binoff,
                            c->d_rec));
    for (int s = 0; s < NSTREAM; ++s) {
        if (!c->plan_active[s]) continue;
        KX_TRY(eri_launch(c, s % NCLASS, s / NCLASS, c->d_rec, 0, 0, w + W.rg() + 2 * s, P, K));
        c->launches++;
    }
    return KX_OK;
}

int capture_build(kx_ctx* c, const double* P, const kx_opts* o, double* K, const GraphWords& W,
                  const GraphCaps& cap) {
    const int D = c->depth, ny = c->n_sys;
    int64_t* w = c->d_gw;
    const int64_t mat_total = c->sys_mat[ny];
    c->build_sym = o->symmetric;
    // statistics and overflow words, device counters
    KX_CUDA(c, cudaMemsetAsync(w + W.t(0), 0, sizeof(int64_t) * 32, c->stream));
    KX_CUDA(c, cudaMemsetAsync(w + W.st(), 0, sizeof(int64_t) * (W.size() - W.st()), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_CAND, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_ERR, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(K, 0, sizeof(double) * mat_total, c->stream));
    KX_TRY(p_norms(c, P));
    if (o->precision != KX_FP64) {
        k_to_f32<<<1024, 256, 0, c->stream>>>(P, 0, 1, mat_total, c->d_P32);
        c->launches++;
    }
    if (o->precision == KX_MIXED_DW) {
        k_to_dw<<<1024, 256, 0, c->stream>>>(P, 0, 1, mat_total, c->d_Pdw);
        c->launches++;
    }
    KX_TRY(pair_tables_dev(c, o->tau, o->shell_screen != 0, o->precision == KX_MIXED_DW));
    const double* S = c->d_nrm_s;
    const double* Pn = c->d_nrm_p;
    if (D == 0) {
        int rl0 = 0, rl1 = 0;
        KX_TRY(row_leaves(c, o, &rl0, &rl1));
        k_root_only<<<1, 1, 0, c->stream>>>(c->d_lseg, ny, S, Pn, o->tau, c->d_front[0], w + W.t(0), rl0, rl1);
        c->launches++;
        KX_TRY(chunk_dev(c, o, W, cap, c->d_front[0], ny, w + W.t(0), P, K));
        if (o->symmetric) KX_TRY(mirror_k(c, K));
        return KX_OK;
    }
    const Task* front = c->d_groots;
    int cur = 0;
    const int64_t* dn = w + W.n(0);
    int64_t* cnt = c->d_scan;
    int64_t* off = c->d_scan + cap.mcap;
    const unsigned g = (unsigned)std::min<int64_t>((cap.mcap + 255) / 256, (int64_t)c->n_sm * 16);
    for (int k = 0; k < D; ++k) {
        const int32_t* child = c->d_node_child + c->levels[k].off;
        const int32_t* nchild = c->d_node_nchild + c->levels[k].off;
        const int32_t* nsys = c->d_node_sys + c->levels[k].off;
        const Seg* lnext = c->d_lseg + (size_t)(k + 1) * ny;
        k_expand_mask<<<g, 256, 0, c->stream>>>(front, cap.mcap, child, nchild, nsys, lnext, S, Pn, o->tau,
                                                c->d_mask, cnt, dn, o->symmetric, row_range(c, o, k + 1));
        c->launches++;
        KX_TRY(exclusive_scan_dev(c, cnt, off, cap.mcap, dn, w + W.t(k + 1)));
        if (k + 1 < D) {
            k_level_check<<<1, 1, 0, c->stream>>>(w + W.t(k + 1), dn, cap.fcap, w + W.n(k + 1), w + W.wr(k),
                                                  w + W.flag());
            k_expand_write<<<g, 256, 0, c->stream>>>(front, 0, 0, c->d_mask, off, 0, child, c->d_front[cur],
                                                     w + W.wr(k));
            c->launches += 2;
            front = c->d_front[cur];
            cur = 1 - cur;
            dn = w + W.n(k + 1);
            continue;
        }
        // last level, in chunks of cap.lq leaf quartets
        Task* leaves = c->d_front[cur];
        for (int j = 0; j < cap.nch; ++j) {
            k_chunk_dev<<<1, 1, 0, c->stream>>>(off, dn, w + W.t(D), cap.lq, j, (int)cap.nch, w + W.ch(j),
                                                w + W.flag());
            k_expand_write<<<g, 256, 0, c->stream>>>(front, 0, 0, c->d_mask, off, 0, child, leaves, w + W.ch(j));
            c->launches += 2;
            KX_TRY(chunk_dev(c, o, W, cap, leaves, cap.lq + 16, w + W.ch(j) + 3, P, K));
        }
    }
    if (o->symmetric) KX_TRY(mirror_k(c, K));
    return KX_OK;
}

}  // namespace

namespace {

// reserves every buffer of a plan at its capacity and records the graph
int capture_plan(kx_ctx* c, const double* P, const kx_opts* o, double* K, const GraphCaps& cap) {
    const int D = c->depth, ny = c->n_sys;
    GraphWords W{D, (int)cap.nch};
    const unsigned nb = expand_blocks(c, cap.lq + 16);
    const int64_t nbin = (int64_t)NSTREAM * nb;
    const int64_t fcap = std::max<int64_t>({cap.fcap, cap.lq + 16, (int64_t)ny + 16});
    KX_TRY(grow(c, &c->d_front[0], &c->front_cap[0], (size_t)fcap));
    KX_TRY(grow(c, &c->d_front[1], &c->front_cap[1], (size_t)fcap));
    KX_TRY(grow(c, &c->d_mask, &c->mask_cap, (size_t)cap.mcap));
    KX_TRY(grow(c, &c->d_scan, &c->scan_cap, (size_t)std::max<int64_t>(2 * cap.mcap, 2 * c->sp_total + 16)));
    KX_TRY(grow(c, &c->d_bin, &c->bin_cap, (size_t)(2 * nbin)));
    KX_TRY(grow(c, &c->d_rec, &c->rec_cap, (size_t)cap.rec));
    KX_TRY(grow(c, &c->d_scantmp, &c->scantmp_cap,
                scan_scratch(std::max<int64_t>({cap.mcap, nbin, c->sp_total}))));
    if (o->precision != KX_FP64) KX_TRY(grow(c, &c->d_P32, &c->P32_cap, (size_t)c->sys_mat[ny]));
    if (o->precision == KX_MIXED_DW) KX_TRY(grow(c, &c->d_Pdw, &c->Pdw_cap, (size_t)c->sys_mat[ny]));
    if (c->gw_n < (size_t)W.size()) {
        cudaFree(c->d_gw);
        cudaFreeHost(c->h_gw);
        c->d_gw = nullptr;
        c->h_gw = nullptr;
        c->gw_n = 0;
        KX_CUDA(c, cudaMalloc(&c->d_gw, sizeof(int64_t) * W.size()));
        KX_CUDA(c, cudaMallocHost(&c->h_gw, sizeof(int64_t) * W.size()));
        c->gw_n = (size_t)W.size();
    }
    if (!c->d_gactive) KX_CUDA(c, cudaMalloc(&c->d_gactive, NSTREAM));
    cudaFree(c->d_groots);
    c->d_groots = nullptr;
    KX_CUDA(c, cudaMalloc(&c->d_groots, sizeof(Task) * ny));
    {
        std::vector<Task> roots(ny);
        for (int y = 0; y < ny; ++y) roots[y] = Task{(uint16_t)y, (uint16_t)y, (uint16_t)y, (uint16_t)y};
        std::vector<int64_t> n0(32, 0);
        n0[0] = ny;
        KX_CUDA(c, cudaMemcpy(c->d_groots, roots.data(), sizeof(Task) * ny, cudaMemcpyHostToDevice));
        KX_CUDA(c, cudaMemcpy(c->d_gw, n0.data(), sizeof(int64_t) * 32, cudaMemcpyHostToDevice));
        KX_CUDA(c, cudaMemcpy(c->d_gactive, c->plan_active, NSTREAM, cudaMemcpyHostToDevice));
    }
    KX_TRY(set_frames(c, 0, 0, true));
    if (!c->gstream) KX_CUDA(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    // record on the capture stream (the legacy default stream cannot be captured)
    c->launches = 0;
    cudaStream_t saved = c->stream;
    c->stream = c->gstream;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        c->stream = saved;
        return cuda_check(c, e, "begin capture");
    }
    int r = capture_build(c, P, o, K, W, cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->stream, &g);
    c->stream = saved;
    if (r != KX_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
    }
    if (e != cudaSuccess) return cuda_check(c, e, "stream capture");
    c->graph = g;
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    if (e != cudaSuccess) {
        drop_graph(c);
        return cuda_check(c, e, "graph instantiation");
    }
    c->graph_launches = c->launches;
    c->graph_depth = D;
    c->graph_st0 = W.st();
    c->graph_valid = true;
    return KX_OK;
}

}  // namespace

int graph_plan(kx_ctx* c, const double* P, const kx_opts* o, double* K, double headroom, kx_stats* st) {
    // the eager build: K, and the sizes the plan needs
    kx_opts oe = *o;
    oe.keep_worklist = 0;
    oe.profile = 0;
    KX_TRY(drive(c, RUN_EXCHANGE, P, 0, &oe, K, 0, st, nullptr, 0));
    const int D = c->depth, ny = c->n_sys;
    const double m = 1.0 + headroom;
    int64_t maxlev = 0, maxpar = ny;
    for (int k = 1; k < D; ++k) maxlev = std::max<int64_t>(maxlev, st->n_tasks[k]);
    for (int k = 0; k < D; ++k) maxpar = std::max<int64_t>(maxpar, st->n_tasks[k]);
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    // records of one chunk: the class-kernel slots are 32-bit, and the
    // records should leave most of the memory to the rest
    const int64_t budget = std::min<int64_t>(((int64_t)1 << 31) - 8192, (int64_t)(0.4 * fr / sizeof(Quartet)));
    GraphCaps cap;
    cap.lq = c->last_lq;   // the eager build's chunks
    cap.fcap = (int64_t)(maxlev * m) + 64;
    cap.mcap = (int64_t)(maxpar * m) + 64;
    const double need = c->plan_max_rec * m + 4096;
    if (need <= (double)budget) {
        cap.rec = (int64_t)need;
    } else {
        // smaller chunks than the eager build's, sized from its densest chunk
        // with a margin for uneven chunks; the check replay below confirms
        cap.lq = std::max<int64_t>(1 << 16, (int64_t)(cap.lq * (double)budget / need * 0.8));
        cap.rec = budget;
    }
    // reserve every pair of nonzero Schwarz factor
    KX_TRY(pair_tables(c, 0.0, false, o->precision == KX_MIXED_DW));
    for (int attempt = 0; attempt < 4; ++attempt) {
        cap.nch = std::max<int64_t>(1, (int64_t)std::ceil(st->n_tasks[D] * m / (double)cap.lq));
        if (cap.nch > 4096) return set_err(c, KX_ECAPACITY, "too many leaf chunks for a captured build");
        KX_TRY(capture_plan(c, P, o, K, cap));
        // a replay on the planning P must fit its own plan
        kx_stats chk;
        const int r = graph_launch(c, &chk);
        if (r == KX_OK) return KX_OK;
        if (r != KX_ECAPACITY) return r;
        drop_graph(c);
        cap.lq = std::max<int64_t>(1 << 16, cap.lq / 2);
    }
    return set_err(c, KX_ECAPACITY, "no chunk size fits the records of a leaf chunk");
}

int graph_launch(kx_ctx* c, kx_stats* st) {
    if (!c->graph_valid) return set_err(c, KX_ESTATE, "no captured build (kx_graph_plan)");
    // statistics block: records per stream [NSTREAM], leaf quartets, overflow
    const int64_t nstat = NSTREAM + 2;
    const int64_t st0 = c->graph_st0;
    // the graph runs on the context's capture stream, ordered after and
    // before the work of the context's own stream
    cudaStream_t gs = c->gstream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    cudaStreamWaitEvent(gs, e0, 0);
    KX_CUDA(c, cudaGraphLaunch(c->gexec, gs));
    cudaEventRecord(e1, gs);
    cudaStreamWaitEvent(c->stream, e1, 0);
    KX_CUDA(c, cudaMemcpyAsync(c->h_gw, c->d_gw, sizeof(int64_t) * 64, cudaMemcpyDeviceToHost, gs));
    KX_CUDA(c, cudaMemcpyAsync(c->h_gw + st0, c->d_gw + st0, sizeof(int64_t) * nstat, cudaMemcpyDeviceToHost, gs));
    KX_CUDA(c, cudaMemcpyAsync(c->h_gw + st0 + nstat, c->d_counters + CTR_CAND, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, gs));
    KX_CUDA(c, cudaMemcpyAsync(c->h_gw + st0 + nstat + 1, c->d_counters + CTR_ERR, sizeof(int64_t),
                               cudaMemcpyDeviceToHost, gs));
    cudaError_t e = cudaStreamSynchronize(gs);
    const int64_t cand = c->h_gw[st0 + nstat], werr = c->h_gw[st0 + nstat + 1];
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_check(c, e, "graph launch");
    if (st) {
        std::memset(st, 0, sizeof(*st));
        const int D = c->graph_depth;
        for (int k = 0; k <= D && k < 32; ++k) st->n_tasks[k] = k == 0 ? c->h_gw[0] : c->h_gw[32 + k];
        st->depth = D;
        for (int s = 0; s < NSTREAM; ++s) add_stream_stats(st, s, c->h_gw[st0 + s]);
        st->n_leaf_quartets = c->h_gw[st0 + NSTREAM];
        st->n_candidates = (int64_t)cand;
        st->n_launches = (int32_t)c->graph_launches;
        st->ms_total = ms;
        st->split_used = c->graph_split;
        st->fp32_err_estimate = c->graph_err_est;
        st->fp32_err_bound = c->graph_err_bound;
    }
    if (c->h_gw[st0 + NSTREAM + 1]) return set_err(c, KX_ECAPACITY, "a count exceeded the captured plan: re-plan");
    if (werr) return set_err(c, KX_ECUDA, "shell-quartet count and write passes disagree");
    return KX_OK;
}

int autotune(kx_ctx* c, const double* P, const kx_opts* o, double* K, kx_stats* st, int* n_tuned) {
    KX_TRY(grow(c, &c->d_tuneK, &c->tuneK_cap, (size_t)c->sys_mat[c->n_sys]));
    for (int s = 0; s < NSTREAM; ++s) c->tuned[s] = false;
    c->tuning = true;
    int r = drive(c, RUN_EXCHANGE, P, 0, o, K, 0, st, nullptr, 0);
    c->tuning = false;
    int n = 0;
    for (int s = 0; s < NSTREAM; ++s) n += c->tuned[s];
    if (n_tuned) *n_tuned = n;
    return r;
}

}  // namespace kx
