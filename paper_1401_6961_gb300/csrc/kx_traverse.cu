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

#include "kx_internal.cuh"

namespace kx {

// ===========================================================================
// device-wide exclusive scan of int64
// ===========================================================================

constexpr int SCAN_T = 256;
constexpr int SCAN_I = 16;
constexpr int SCAN_TILE = SCAN_T * SCAN_I;

__device__ int64_t block_excl_scan64(int64_t v, int64_t* sh, int64_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int64_t ex = x - v + (w > 0 ? sh[w - 1] : 0);
    *total = sh[nw - 1];
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(const int64_t* __restrict__ in, int64_t n,
                                                       int64_t* __restrict__ tile_sum) {
    __shared__ int64_t sh[32];
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
                                                       const int64_t* __restrict__ tile_off,
                                                       int64_t* __restrict__ out, int64_t* __restrict__ grand) {
    __shared__ int64_t sh[32];
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

static int scan_rec(cudaStream_t st, const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, int64_t* grand) {
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles <= 1) {
        k_scan_apply<<<1, SCAN_T, 0, st>>>(in, n, nullptr, out, grand);
        return 1;
    }
    int64_t* tsum = tmp;
    int64_t* toff = tmp + tiles;
    int64_t* inner_grand = tmp + 2 * tiles;
    k_scan_tiles<<<(unsigned)tiles, SCAN_T, 0, st>>>(in, n, tsum);
    int k = scan_rec(st, tsum, toff, tiles, tmp + 2 * tiles + 2, inner_grand);
    k_scan_apply<<<(unsigned)tiles, SCAN_T, 0, st>>>(in, n, toff, out, grand);
    return k + 2;
}

int exclusive_scan(kx_ctx* c, const int64_t* in, int64_t* out, int64_t n, int64_t* total_host) {
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return KX_OK;
    }
    KX_TRY(grow(c, &c->d_scantmp, &c->scantmp_cap, scan_tmp_need(n) + 8));
    int64_t* grand = c->d_scantmp;
    c->launches += scan_rec(c->stream, in, out, n, c->d_scantmp + 8, grand);
    if (total_host) {
        KX_CUDA(c, cudaMemcpyAsync(total_host, grand, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        KX_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return KX_OK;
}

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
                              int64_t* __restrict__ cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Task t = front[i];
        const Seg g = lseg_next[node_sys[t.a]];
        const int64_t t0 = g.t0();
        const int nn = g.n;
        const int ca = child[t.a], na = nchild[t.a];
        const int cb = child[t.b], nb = nchild[t.b];
        const int cc = child[t.c], nc = nchild[t.c];
        const int cd = child[t.d], nd = nchild[t.d];
        unsigned m = 0;
        for (int ia = 0; ia < na; ++ia)
            for (int ib = 0; ib < nb; ++ib) {
                const double sab = S[t0 + (int64_t)(ca + ia) * nn + (cb + ib)];
                for (int id = 0; id < nd; ++id) {
                    const double x = __dmul_rn(sab, Pn[t0 + (int64_t)(cb + ib) * nn + (cd + id)]);
                    for (int ic = 0; ic < nc; ++ic) {
                        const double beta = __dmul_rn(x, S[t0 + (int64_t)(cc + ic) * nn + (cd + id)]);
                        if (beta > tau) m |= 1u << (((ia * 2 + ib) * 2 + ic) * 2 + id);
                    }
                }
            }
        mask[i] = (uint16_t)m;
        cnt[i] = __popc(m);
    }
}

__global__ void k_expand_write(const Task* __restrict__ front, int64_t p0, int64_t p1,
                               const uint16_t* __restrict__ mask, const int64_t* __restrict__ off, int64_t obase,
                               const int32_t* __restrict__ child, Task* __restrict__ out) {
    for (int64_t i = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p1;
         i += (int64_t)gridDim.x * blockDim.x) {
        unsigned m = mask[i];
        if (!m) continue;
        const Task t = front[i];
        int64_t pos = off[i] - obase;
        const int ca = child[t.a], cb = child[t.b], cc = child[t.c], cd = child[t.d];
        while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            out[pos++] = Task{(uint16_t)(ca + ((bit >> 3) & 1)), (uint16_t)(cb + ((bit >> 2) & 1)),
                              (uint16_t)(cc + ((bit >> 1) & 1)), (uint16_t)(cd + (bit & 1))};
        }
    }
}

// trees that are single leaves: the root task of every system, kept iff its
// bound exceeds tau, in system order (one thread: only for tiny systems)
__global__ void k_root_only(const Seg* __restrict__ lseg0, int nsys, const double* __restrict__ S,
                            const double* __restrict__ Pn, double tau, Task* __restrict__ out,
                            int64_t* __restrict__ n_out) {
    int64_t k = 0;
    for (int y = 0; y < nsys; ++y) {
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

// ===========================================================================
// driver
// ===========================================================================

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
};

int process_leaves(Run& r, const Task* leaves, int64_t n);
int finish_run(kx_ctx* c, kx_stats* st, Timer& tm, int D);

// shell screen, class binning and class kernels for one list of leaf quartets
int process_leaves(Run& r, const Task* leaves, int64_t n) {
    kx_ctx* c = r.c;
    if (n <= 0) return KX_OK;
    const int mixed = r.o->precision == KX_MIXED;
    const double split = mixed ? r.o->split_threshold : 0.0;
    r.tm->mark(ST_EXPAND);
    const unsigned nb = expand_blocks(n);
    const int64_t nbin = (int64_t)2 * NCLASS * nb;
    KX_TRY(grow(c, &c->d_bin, &c->bin_cap, (size_t)(2 * nbin)));
    int64_t* bin = c->d_bin;
    int64_t* binoff = c->d_bin + nbin;
    KX_TRY(expand_count(c, leaves, n, r.o->tau, split, mixed, r.o->shell_screen, bin));
    c->launches++;
    int64_t total = 0;
    KX_TRY(exclusive_scan(c, bin, binoff, nbin, &total));
    if (total > r.rec_limit && n > 1) {
        // too many records for one pass: halve the leaf list
        int64_t h0 = n / 2;
        KX_TRY(process_leaves(r, leaves, h0));
        return process_leaves(r, leaves + h0, n - h0);
    }
    if (total == 0) return KX_OK;
    // stream s starts at binoff[s * nb]
    int64_t off[2 * NCLASS + 1];
    KX_CUDA(c, cudaMemcpy2DAsync(off, sizeof(int64_t), binoff, sizeof(int64_t) * nb, sizeof(int64_t), 2 * NCLASS,
                                 cudaMemcpyDeviceToHost, c->stream));
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    off[2 * NCLASS] = total;
    unsigned long long h[2 * NCLASS], endv[2 * NCLASS];
    for (int s = 0; s < 2 * NCLASS; ++s) {
        h[s] = (unsigned long long)(off[s + 1] - off[s]);
        endv[s] = (unsigned long long)off[s + 1];
    }
    KX_TRY(grow(c, &c->d_rec, &c->rec_cap, (size_t)total));
    KX_CUDA(c, cudaMemcpyAsync(c->d_counters + CTR_END, endv, sizeof(endv), cudaMemcpyHostToDevice, c->stream));
    KX_TRY(expand_write(c, leaves, n, r.o->tau, split, mixed, r.o->shell_screen, binoff, c->d_rec));
    c->launches++;
    r.tm->mark(ST_ERI);
    for (int s = 0; s < 2 * NCLASS; ++s) {
        if (!h[s]) continue;
        const int prec = s / NCLASS, cls = s % NCLASS;
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
        const double f = class_flops(cls) * (double)h[s];
        if (prec == 0) r.st->flops_fp64 += f; else r.st->flops_fp32 += f;
        c->prof_n[s] += (int64_t)h[s];
        c->prof_flops[s] += f;
        c->prof_launches[s] += 1;
    }
    r.st->n_shell_quartets += total;
    for (int s = 0; s < NCLASS; ++s) r.st->n_shell_quartets_fp64 += (int64_t)h[s];
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

int drive(kx_ctx* c, int mode, const double* P, int64_t ldp, const kx_opts* o, double* K, int64_t ldk,
          kx_stats* st, const Task* list, int64_t nlist) {
    const int D = c->depth;
    const bool evaluate = mode != RUN_TRAVERSE;
    Timer tm{c, {}};
    Run r{c, P, ldp, o, K, ldk, st, &tm, 0, 0.0};
    // record budget per pass: the caller's, else 2^30 records (8 GB) or a
    // quarter of the free device memory, whichever is smaller
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    int64_t lim = (int64_t)std::min<size_t>((size_t)1 << 30, fr / 4 / sizeof(Quartet));
    r.rec_limit = o->chunk_records > 0 ? o->chunk_records : std::max<int64_t>(lim, 1 << 20);
    r.rec_limit = std::min<int64_t>(r.rec_limit, (int64_t)1 << 31);   // record slots are 32-bit in the binning
    const int64_t lq_cap = std::max<int64_t>(r.rec_limit / 48, 1 << 16);

    c->launches = 0;
    for (int s = 0; s < 2 * NCLASS; ++s) {
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
    tm.mark(ST_NORMS);
    const int64_t mat_total = c->sys_mat[c->n_sys];
    if (evaluate) {
        if (packed)
            KX_CUDA(c, cudaMemsetAsync(K, 0, sizeof(double) * mat_total, c->stream));
        else
            KX_CUDA(c, cudaMemset2DAsync(K, sizeof(double) * ldk, 0, sizeof(double) * c->n_fn, c->n_fn, c->stream));
    }
    KX_TRY(p_norms(c, P));
    if (evaluate && o->precision == KX_MIXED) {
        const int64_t rows = packed ? 1 : c->n_fn, cols = packed ? mat_total : c->n_fn, ld = packed ? 0 : ldp;
        KX_TRY(grow(c, &c->d_P32, &c->P32_cap, (size_t)((rows - 1) * ld + cols)));
        k_to_f32<<<1024, 256, 0, c->stream>>>(P, ld, rows, cols, c->d_P32);
        c->launches++;
    }
    if (evaluate) KX_TRY(pair_tables(c, o->tau, o->shell_screen != 0));
    const bool keep = mode == RUN_TRAVERSE || (mode == RUN_EXCHANGE && o->keep_worklist);
    if (mode != RUN_EVALUATE) {
        c->keep_n = 0;
        c->keep_valid = false;
    }
    if (mode == RUN_EVALUATE) {
        // an explicit leaf-quartet list: the ERI stage in chunks of lq_cap
        st->n_leaf_quartets = nlist;
        for (int64_t i0 = 0; i0 < nlist; i0 += lq_cap)
            KX_TRY(process_leaves(r, list + i0, std::min<int64_t>(lq_cap, nlist - i0)));
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
        k_root_only<<<1, 1, 0, c->stream>>>(c->d_lseg, ny, S, Pn, o->tau, c->d_front[0], d_n);
        c->launches++;
        int64_t nk = 0;
        KX_CUDA(c, cudaMemcpyAsync(&nk, d_n, sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        KX_CUDA(c, cudaStreamSynchronize(c->stream));
        st->n_tasks[0] = nk;
        st->n_leaf_quartets = nk;
        if (keep) KX_TRY(keep_leaves(c, c->d_front[0], nk));
        if (evaluate) KX_TRY(process_leaves(r, c->d_front[0], nk));
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
            unsigned g = (unsigned)std::min<int64_t>((nfront + 255) / 256, 152 * 64);
            k_expand_mask<<<g, 256, 0, c->stream>>>(c->d_front[cur], nfront, child, nchild, nsys, lnext, S, Pn,
                                                    o->tau, c->d_mask, cnt);
            c->launches++;
            int64_t total = 0;
            KX_TRY(exclusive_scan(c, cnt, off, nfront, &total));
            st->n_tasks[k + 1] = total;
            if (k + 1 < D) {
                KX_TRY(grow(c, &c->d_front[1 - cur], &c->front_cap[1 - cur], (size_t)std::max<int64_t>(total, 1)));
                k_expand_write<<<g, 256, 0, c->stream>>>(c->d_front[cur], 0, nfront, c->d_mask, off, 0, child,
                                                         c->d_front[1 - cur]);
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
                unsigned g2 = (unsigned)std::min<int64_t>((p1 - p0 + 255) / 256, 152 * 64);
                k_expand_write<<<g2, 256, 0, c->stream>>>(c->d_front[cur], p0, p1, c->d_mask, off, o0, child,
                                                          c->d_front[1 - cur]);
                c->launches++;
                if (keep) KX_TRY(keep_leaves(c, c->d_front[1 - cur], o1 - o0));
                if (evaluate) KX_TRY(process_leaves(r, c->d_front[1 - cur], o1 - o0));
            }
        }
    }
    if (keep) c->keep_valid = true;
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

}  // namespace kx
