// kx_expand.cu -- from surviving leaf quartets to shell-quartet records.
//
// A leaf quartet (A,B,C,D) holds |A||B||C||D| shell quartets.  With the
// shell screen on, each is kept iff the metric query of Eq. 8 applied to the
// single-shell blocks passes,
//     beta = (S_ab * ||P_bd||_F) * S_cd > tau,
// i.e. the recursion of Eq. 7 carried one level further, to single shells.
// The test first runs on log2 values in FP32 (sum of three logs against
// log2 tau); only quartets whose log sum lies within LOG_MARGIN of the
// threshold -- a band wider than every FP32 rounding error in that sum --
// are decided by the exact FP64 product.  The decision is therefore the
// FP64 decision, at FP32 cost.  The same test against the split threshold
// routes a kept quartet to the FP64 or the FP32 kernels in mixed mode.
//
// Records are binned by angular-momentum class and precision ("stream",
// 243 of them: FP64, FP32 and double word).  One warp handles one leaf quartet; lanes walk its shell
// quartets with d fastest, then b, c, a, so runs of equal (a,c) -- one K
// block -- stay adjacent in each stream.  A first pass counts the records of
// every (stream, block); after a scan of those counts a second pass writes
// each block's records from its offsets through shared-memory cursors, so no
// global atomic is involved and the blocks' ranges are fixed.
#include <algorithm>
#include <cmath>

#include "kx_internal.cuh"

namespace kx {

constexpr float LOG_MARGIN = 1e-3f;   // log2 units; FP32 error of the sum < 6e-4

struct ExpandArgs {
    const Task* leaves;
    int64_t n;
    const int64_t* dn;       // device count (n is then a capacity), may be null
    const int32_t* llo;
    const int32_t* lhi;
    const int32_t* tl;
    const int32_t* tsys;     // system of every tree position
    const Seg* sseg;         // shell-pair table block of every system
    const float* slog;
    const float* plog;
    const double* snorm;
    const double* pnorm;
    const int32_t* pairmap;
    double tau, split;
    float ltau, lsplit;
    int mixed;               // the build's precision (KX_FP64, KX_MIXED, KX_MIXED_DW)
    int screen;
    int sym;                 // symmetric build: inside a diagonal block (A == C) only a <= c
    // count pass only, may be null: work[A] += the algorithmic FLOPs of the
    // kept shell quartets of every leaf quartet with row leaf A (sflops[s]
    // = FLOPs of one quartet of stream s)
    double* work;
    const float* sflops;
    // statistics pass (split planning): for every FP32 quartet of a sampled
    // K shell block (blkslot[(a,c)] >= 0), in bin j = floor((log2 beta -
    // lbin0) * PLAN_BINS_PER_OCTAVE) clamped to [0, nbin):
    // acc[(slot * nbin + j) * 2] += cmax[cls]
    // beta and acc[... + 1] += (crms[cls] beta)^2
    const int32_t* blkslot;
    double* blkacc;
    const float* cmax;
    const float* crms;
    float lbin0;
    int nbin;
};

__device__ __forceinline__ void block_stats(const ExpandArgs& p, float x, int stream, int64_t t0, int ns, int a,
                                            int c) {
    if (stream < NCLASS || stream >= 2 * NCLASS) return;   // FP32 quartets only
    const int slot = __ldg(p.blkslot + t0 + (int64_t)a * ns + c);
    if (slot < 0) return;
    const int cls = stream - NCLASS;
    const int j = min(max((int)floorf((x - p.lbin0) * PLAN_BINS_PER_OCTAVE), 0), p.nbin - 1);
    const double beta = (double)exp2f(x);
    double* acc = p.blkacc + ((int64_t)slot * p.nbin + j) * 2;
    atomicAdd(acc, (double)__ldg(p.cmax + cls) * beta);
    const double r = (double)__ldg(p.crms + cls) * beta;
    atomicAdd(acc + 1, r * r);
}

__device__ __forceinline__ bool above(float x, float lthr, double thr, const double* __restrict__ snorm,
                                      const double* __restrict__ pnorm, int64_t ab, int64_t bd, int64_t cd) {
    if (x > lthr + LOG_MARGIN) return true;
    if (x < lthr - LOG_MARGIN) return false;
    return __dmul_rn(__dmul_rn(snorm[ab], pnorm[bd]), snorm[cd]) > thr;
}

constexpr int EXP_WARPS = 8;     // warps per block
constexpr int STAGE = 16;        // shells per leaf held in the shared tables

// q = x / n for x < 2^16 and 2 <= n < 2^16 by q = mulhi(x, m), m = floor(2^32/n) + 1:
// x*m/2^32 = x/n + x*e/2^32 with 0 < e < 1, and x/2^32 < 1/n keeps the floor
// exact; n = 1 is passed as m = 0 and returns x.
struct Div {
    unsigned m;
    __device__ explicit Div(int n) : m(n > 1 ? 0xffffffffu / (unsigned)n + 1u : 0u) {}
};
__device__ __forceinline__ unsigned fdiv(unsigned x, Div d) { return d.m ? __umulhi(x, d.m) : x; }

struct WarpTables {
    float sab[STAGE * STAGE];    // log2 S_ab, [ia][ib]
    float scd[STAGE * STAGE];    // log2 S_cd, [ic][id]
    float pbd[STAGE * STAGE];    // log2 ||P_bd||, [ib][id]
    float mb[STAGE];             // max over a of log2 S_ab, per b
    float md[STAGE];             // max over c of log2 S_cd, per d
    float ma[STAGE];             // max over b of log2 S_ab, per a
    float mc[STAGE];             // max over d of log2 S_cd, per c
    uint8_t cab[STAGE * STAGE];  // pair class la*3+lb
    uint8_t ccd[STAGE * STAGE];
    uint8_t kl[STAGE * STAGE];   // (b,d) pairs that can pass for some (a,c): ib*16+id
    uint8_t rl[STAGE * STAGE];   // rows (a,c) that can pass for some kept (b,d): ia*16+ic
};

// Decides one candidate and returns its stream (-1 = culled).  The pair
// tables hold every pair of a kept quartet (their filter is looser than the
// quartet test), so only the write pass reads the slots.  Without the shell
// screen a quartet is kept unless one of its pairs is empty (Eq. 4), which
// the -inf logs of zero Schwarz factors tell.
template <bool WRITE>
__device__ __forceinline__ int decide(const ExpandArgs& p, float x, float sab, float scd, int a, int b, int c,
                                      int d, int cls, int64_t t0, int ns, int32_t& pab, int32_t& pcd) {
    const int64_t ab = t0 + (int64_t)a * ns + b, bd = t0 + (int64_t)b * ns + d, cd = t0 + (int64_t)c * ns + d;
    const bool keep = p.screen ? above(x, p.ltau, p.tau, p.snorm, p.pnorm, ab, bd, cd)
                               : (sab > -INFINITY && scd > -INFINITY);
    if (!keep) return -1;
    if (WRITE) {
        pab = __ldg(p.pairmap + ab);
        pcd = __ldg(p.pairmap + cd);
    }
    // above the split: FP64, or double-word FP32 where the class has a
    // double-word kernel; at or below it: FP32
    int prec = 0;
    if (p.mixed) {
        if (!above(x, p.lsplit, p.split, p.snorm, p.pnorm, ab, bd, cd)) prec = 1;
        else if (p.mixed == KX_MIXED_DW && class_l(cls) <= DW_LMAX) prec = 2;
    }
    return prec * NCLASS + cls;
}

// One warp-aggregated shared-memory add per distinct stream of the lanes
// kept candidates.  Count pass: per-block totals.  Write pass: the block's
// cursor of that stream gives the slot of every lane's record.
template <bool WRITE>
__device__ __forceinline__ void emit(int stream, int32_t pab, int32_t pcd, int lane, unsigned int* scount,
                                     Quartet* __restrict__ rec, const unsigned long long* __restrict__ end,
                                     unsigned long long* __restrict__ err, const float* __restrict__ sflops,
                                     float& wsum) {
    if (!WRITE) {
        if (stream >= 0) {
            atomicAdd(&scount[stream], 1u);
            if (sflops) wsum += __ldg(sflops + stream);
        }
        return;
    }
    const unsigned keepmask = __ballot_sync(0xffffffffu, stream >= 0);
    if (stream < 0) return;
    const unsigned grp = __match_any_sync(keepmask, stream);
    const int leader = __ffs(grp) - 1;
    unsigned bas = 0;
    if (lane == leader) bas = atomicAdd(&scount[stream], (unsigned)__popc(grp));
    if (WRITE) {
        bas = __shfl_sync(grp, bas, leader);
        const unsigned long long slot = (unsigned long long)bas + __popc(grp & ((1u << lane) - 1u));
        // the count pass sized every (stream, block) range; never write past the stream
        if (slot < end[stream]) rec[slot] = Quartet{pab, pcd};
        else atomicAdd(err, 1ull);
    }
}

// MODE 0: count pass; 1: write pass; 2: count pass with the block
// statistics of split planning
template <int MODE>
__global__ void __launch_bounds__(EXP_WARPS * 32)
k_expand(ExpandArgs p, int64_t* __restrict__ bin, Quartet* __restrict__ rec, unsigned long long* __restrict__ cand,
         const unsigned long long* __restrict__ end, unsigned long long* __restrict__ err) {
    constexpr bool WRITE = MODE == 1;
    constexpr bool STATS = MODE == 2;
    // bin[s * gridDim.x + block]: count pass writes the block's count of
    // stream s, the write pass reads the scanned offset
    __shared__ unsigned int scount[NSTREAM];
    __shared__ WarpTables tabs[EXP_WARPS];
    for (int i = threadIdx.x; i < NSTREAM; i += blockDim.x)
        scount[i] = WRITE ? (unsigned)bin[(int64_t)i * gridDim.x + blockIdx.x] : 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    WarpTables& tb = tabs[threadIdx.x >> 5];
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long ncand = 0;
    const int64_t nq = p.dn ? min(p.n, *p.dn) : p.n;
    for (int64_t q = warp; q < nq; q += nwarp) {
        const Task t = p.leaves[q];
        float wsum = 0.f;   // FLOPs of this lane's kept candidates (row-work counts only)
        const int a0 = p.llo[t.a], na = p.lhi[t.a] - a0;
        const int b0 = p.llo[t.b], nb = p.lhi[t.b] - b0;
        const int c0 = p.llo[t.c], nc = p.lhi[t.c] - c0;
        const int d0 = p.llo[t.d], nd = p.lhi[t.d] - d0;
        const int total = na * nb * nc * nd;
        ncand += total;
        // the four leaves belong to one system: its shell-pair block
        const Seg sg = p.sseg[p.tsys[a0]];
        const int64_t t0 = sg.t0();
        const int ns = sg.n;
        const bool diag = p.sym && t.a == t.c;   // then a0 == c0
        const Div md(nd), mb(nb), mc(nc);
        if (na <= STAGE && nb <= STAGE && nc <= STAGE && nd <= STAGE && total <= 65536) {
            // stage the leaf quartet's log tables and pair classes
            __syncwarp();
            for (int k = lane; k < na * nb; k += 32) {
                const int ia = fdiv(k, mb), ib = k - ia * nb;
                const int a = a0 + ia, b = b0 + ib;
                tb.sab[ia * STAGE + ib] = __ldg(p.slog + t0 + (int64_t)a * ns + b);
                tb.cab[ia * STAGE + ib] = (uint8_t)(__ldg(p.tl + a) * 3 + __ldg(p.tl + b));
            }
            for (int k = lane; k < nc * nd; k += 32) {
                const int ic = fdiv(k, md), id = k - ic * nd;
                const int c = c0 + ic, d = d0 + id;
                tb.scd[ic * STAGE + id] = __ldg(p.slog + t0 + (int64_t)c * ns + d);
                tb.ccd[ic * STAGE + id] = (uint8_t)(__ldg(p.tl + c) * 3 + __ldg(p.tl + d));
            }
            for (int k = lane; k < nb * nd; k += 32) {
                const int ib = fdiv(k, md), id = k - ib * nd;
                tb.pbd[ib * STAGE + id] = __ldg(p.plog + t0 + (int64_t)(b0 + ib) * ns + d0 + id);
            }
            __syncwarp();
            // column maxima for the (b,d) pre-filter, row maxima for the
            // (a,c) pre-filter
            if (lane < nb) {
                float m = -INFINITY;
                for (int ia = 0; ia < na; ++ia) m = fmaxf(m, tb.sab[ia * STAGE + lane]);
                tb.mb[lane] = m;
            }
            if (lane < nd) {
                float m = -INFINITY;
                for (int ic = 0; ic < nc; ++ic) m = fmaxf(m, tb.scd[ic * STAGE + lane]);
                tb.md[lane] = m;
            }
            if (lane >= 16 && lane - 16 < na) {
                float m = -INFINITY;
                for (int ib = 0; ib < nb; ++ib) m = fmaxf(m, tb.sab[(lane - 16) * STAGE + ib]);
                tb.ma[lane - 16] = m;
            }
            if (lane >= 16 && lane - 16 < nc) {
                float m = -INFINITY;
                for (int id = 0; id < nd; ++id) m = fmaxf(m, tb.scd[(lane - 16) * STAGE + id]);
                tb.mc[lane - 16] = m;
            }
            __syncwarp();
            // (b,d) pairs that can pass for some (a,c), kept in (b,d) order:
            // log2 bound max_a S_ab + ||P_bd|| + max_c S_cd; the margin keeps it
            // conservative against the FP32 rounding of the sums
            int nk = 0;
            for (int k0 = 0; k0 < nb * nd; k0 += 32) {
                const int k = k0 + lane;
                bool ok = false;
                int ib = 0, id = 0;
                if (k < nb * nd) {
                    ib = fdiv(k, md);
                    id = k - ib * nd;
                    ok = !p.screen ||
                         (tb.mb[ib] + tb.pbd[ib * STAGE + id] + tb.md[id] >= p.ltau - 2.f * LOG_MARGIN);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                if (ok) tb.kl[nk + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)(ib * STAGE + id);
                nk += __popc(bal);
            }
            __syncwarp();
            if (nk == 0) continue;
            // rows (a,c) that can pass for some kept (b,d), in (a,c) order:
            // log2 bound max_b S_ab + max_kept ||P_bd|| + max_d S_cd, with the
            // same margin; in a symmetric diagonal block only a <= c
            float mp = -INFINITY;
            for (int k = lane; k < nk; k += 32) mp = fmaxf(mp, tb.pbd[(tb.kl[k] >> 4) * STAGE + (tb.kl[k] & 15)]);
            for (int d = 16; d > 0; d >>= 1) mp = fmaxf(mp, __shfl_xor_sync(0xffffffffu, mp, d));
            int nr = 0;
            for (int r0 = 0; r0 < na * nc; r0 += 32) {
                const int r = r0 + lane;
                bool ok = false;
                int ia = 0, ic = 0;
                if (r < na * nc) {
                    ia = fdiv(r, mc);
                    ic = r - ia * nc;
                    ok = !(diag && ia > ic) &&
                         (!p.screen || tb.ma[ia] + mp + tb.mc[ic] >= p.ltau - 2.f * LOG_MARGIN);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, ok);
                if (ok) tb.rl[nr + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)(ia * STAGE + ic);
                nr += __popc(bal);
            }
            __syncwarp();
            // sweep (row, k) over the two compacted lists, k fastest: one
            // flat index so every lane has work
            const int total2 = nr * nk;
            const Div dk(nk);
            for (int base = 0; base < total2; base += 32) {
                const unsigned idx = base + lane;
                int stream = -1;
                int32_t pab = -1, pcd = -1;
                if (idx < (unsigned)total2) {
                    const unsigned row = fdiv(idx, dk);
                    const int k = idx - row * nk;
                    const int ac = tb.rl[row];
                    const int ia = ac >> 4, ic = ac & 15;
                    const int bd = tb.kl[k];
                    const int ib = bd >> 4, id = bd & 15;
                    const float sab = tb.sab[ia * STAGE + ib], scd = tb.scd[ic * STAGE + id];
                    const float x = sab + tb.pbd[ib * STAGE + id] + scd;
                    const int cls = tb.cab[ia * STAGE + ib] * 9 + tb.ccd[ic * STAGE + id];
                    stream = decide<WRITE>(p, x, sab, scd, a0 + ia, b0 + ib, c0 + ic, d0 + id, cls, t0, ns, pab,
                                           pcd);
                    if (STATS) block_stats(p, x, stream, t0, ns, a0 + ia, c0 + ic);
                }
                emit<WRITE>(stream, pab, pcd, lane, scount, rec, end, err, p.sflops, wsum);
            }
        } else {
            // very large leaves: read the tables from global memory
            for (int base = 0; base < total; base += 32) {
                const int idx = base + lane;
                int stream = -1;
                int32_t pab = -1, pcd = -1;
                if (idx < total) {
                    int r = idx;
                    const int id = r % nd; r /= nd;
                    const int ib = r % nb; r /= nb;
                    const int ic = r % nc;
                    const int ia = r / nc;
                    const int a = a0 + ia, b = b0 + ib, c = c0 + ic, d = d0 + id;
                    const float sab = p.slog[t0 + (int64_t)a * ns + b], scd = p.slog[t0 + (int64_t)c * ns + d];
                    const float x = sab + p.plog[t0 + (int64_t)b * ns + d] + scd;
                    const int cls = ((p.tl[a] * 3 + p.tl[b]) * 3 + p.tl[c]) * 3 + p.tl[d];
                    if (!(diag && a > c)) {
                        stream = decide<WRITE>(p, x, sab, scd, a, b, c, d, cls, t0, ns, pab, pcd);
                        if (STATS) block_stats(p, x, stream, t0, ns, a, c);
                    }
                }
                emit<WRITE>(stream, pab, pcd, lane, scount, rec, end, err, p.sflops, wsum);
            }
        }
        if (!WRITE && p.work) {
            for (int d = 16; d > 0; d >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, d);
            if (lane == 0 && wsum > 0.f) atomicAdd(p.work + t.a, (double)wsum);
        }
    }
    if (!WRITE) {
        __syncthreads();
        for (int i = threadIdx.x; i < NSTREAM; i += blockDim.x)
            bin[(int64_t)i * gridDim.x + blockIdx.x] = scount[i];
        for (int d = 16; d > 0; d >>= 1) ncand += __shfl_xor_sync(0xffffffffu, ncand, d);
        if (lane == 0 && ncand) atomicAdd(cand, ncand / 32);
    }
}

static ExpandArgs make_args(kx_ctx* c, const Task* leaves, int64_t n, double tau, double split, int mixed,
                            int screen) {
    // symmetric builds: the flag of the build in progress
    const int sym = c->build_sym;
    ExpandArgs a;
    a.leaves = leaves;
    a.n = n;
    a.dn = nullptr;
    a.llo = c->d_leaf_lo;
    a.lhi = c->d_leaf_hi;
    a.tl = c->d_tl;
    a.tsys = c->d_tsys;
    a.sseg = c->d_sseg;
    a.slog = c->d_slog;
    a.plog = c->d_plog;
    a.snorm = c->d_snorm;
    a.pnorm = c->d_pnorm;
    a.pairmap = c->d_pairmap;
    a.tau = tau;
    a.split = split;
    a.ltau = tau > 0.0 ? (float)std::log2(tau) : -INFINITY;
    a.lsplit = split > 0.0 ? (float)std::log2(split) : -INFINITY;
    a.mixed = mixed;
    a.screen = screen;
    a.sym = sym;
    a.work = c->work_acc;
    a.sflops = c->d_sflops;
    a.blkslot = c->plan_slot;
    a.blkacc = c->plan_acc;
    a.cmax = c->d_cmax;
    a.crms = c->d_crms;
    a.lbin0 = c->plan_lbin0;
    a.nbin = c->plan_nbin;
    return a;
}

// one warp per leaf quartet, at most 16 blocks per SM (a persistent grid)
static unsigned expand_grid(const kx_ctx* c, int64_t n) {
    int64_t blocks = (n + EXP_WARPS - 1) / EXP_WARPS;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)c->n_sm * 16));
}

unsigned expand_blocks(const kx_ctx* c, int64_t n) { return expand_grid(c, n); }

int expand_count(kx_ctx* c, const Task* leaves, int64_t n, double tau, double split, int mixed, int shell_screen,
                 int64_t* bin) {
    if (n <= 0) return KX_OK;
    ExpandArgs a = make_args(c, leaves, n, tau, split, mixed, shell_screen);
    if (c->plan_slot)
        k_expand<2><<<expand_grid(c, n), EXP_WARPS * 32, 0, c->stream>>>(a, bin, nullptr, c->d_counters + CTR_CAND,
                                                                       nullptr, nullptr);
    else
        k_expand<0><<<expand_grid(c, n), EXP_WARPS * 32, 0, c->stream>>>(a, bin, nullptr, c->d_counters + CTR_CAND,
                                                                       nullptr, nullptr);
    return KX_OK;
}

int expand_write(kx_ctx* c, const Task* leaves, int64_t n, double tau, double split, int mixed, int shell_screen,
                 int64_t* bin_off, Quartet* rec) {
    if (n <= 0) return KX_OK;
    ExpandArgs a = make_args(c, leaves, n, tau, split, mixed, shell_screen);
    k_expand<1><<<expand_grid(c, n), EXP_WARPS * 32, 0, c->stream>>>(a, bin_off, rec, nullptr,
                                                                      c->d_counters + CTR_END,
                                                                      c->d_counters + CTR_ERR);
    return KX_OK;
}

int expand_count_dev(kx_ctx* c, const Task* leaves, int64_t cap, const int64_t* dn, double tau, double split,
                     int mixed, int shell_screen, int64_t* bin) {
    if (cap <= 0) return KX_OK;
    ExpandArgs a = make_args(c, leaves, cap, tau, split, mixed, shell_screen);
    a.dn = dn;
    k_expand<0><<<expand_grid(c, cap), EXP_WARPS * 32, 0, c->stream>>>(a, bin, nullptr, c->d_counters + CTR_CAND,
                                                                         nullptr, nullptr);
    c->launches++;
    return KX_OK;
}

int expand_write_dev(kx_ctx* c, const Task* leaves, int64_t cap, const int64_t* dn, double tau, double split,
                     int mixed, int shell_screen, int64_t* bin_off, Quartet* rec) {
    if (cap <= 0) return KX_OK;
    ExpandArgs a = make_args(c, leaves, cap, tau, split, mixed, shell_screen);
    a.dn = dn;
    k_expand<1><<<expand_grid(c, cap), EXP_WARPS * 32, 0, c->stream>>>(a, bin_off, rec, nullptr,
                                                                        c->d_counters + CTR_END,
                                                                        c->d_counters + CTR_ERR);
    c->launches++;
    return KX_OK;
}

// ---------------------------------------------------------------------------
// class dispatch
// ---------------------------------------------------------------------------

EriKern eri_kernel_dw(int cls) {
    switch (cls / 9) {
        case 0: return eri_kernel_dw_ab00(cls);
        case 1: return eri_kernel_dw_ab01(cls);
        case 2: return eri_kernel_dw_ab02(cls);
        case 3: return eri_kernel_dw_ab10(cls);
        case 4: return eri_kernel_dw_ab11(cls);
        case 5: return eri_kernel_dw_ab12(cls);
        case 6: return eri_kernel_dw_ab20(cls);
        case 7: return eri_kernel_dw_ab21(cls);
        case 8: return eri_kernel_dw_ab22(cls);
        default: return EriKern{nullptr, 0, 0};
    }
}

EriKern eri_kernel(int cls, int prec, int variant) {
    if (prec == 2) return eri_kernel_dw(cls);
    switch (cls / 9) {
        case 0: return eri_kernel_ab00(cls, prec, variant);
        case 1: return eri_kernel_ab01(cls, prec, variant);
        case 2: return eri_kernel_ab02(cls, prec, variant);
        case 3: return eri_kernel_ab10(cls, prec, variant);
        case 4: return eri_kernel_ab11(cls, prec, variant);
        case 5: return eri_kernel_ab12(cls, prec, variant);
        case 6: return eri_kernel_ab20(cls, prec, variant);
        case 7: return eri_kernel_ab21(cls, prec, variant);
        case 8: return eri_kernel_ab22(cls, prec, variant);
        default: return EriKern{nullptr, 0, 0};
    }
}

constexpr int SMEM_BLOCK_MAX = 227 * 1024;   // opt-in shared memory per block

int eri_fit_threads(const EriKern& k, int threads) {
    while (k.smem_per_thread > 0 && threads > 32 && threads * k.smem_per_thread > SMEM_BLOCK_MAX) threads /= 2;
    return threads;
}

int eri_prepare(kx_ctx* c, int s, int variant, const EriKern& k) {
    if (k.smem_per_thread > 0 && !c->eri_smem_set[s][variant % 3]) {
        KX_CUDA(c, cudaFuncSetAttribute((const void*)k.k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        SMEM_BLOCK_MAX));
        c->eri_smem_set[s][variant % 3] = true;
    }
    return KX_OK;
}

EriArgs eri_args(kx_ctx* c, int cls, int prec, const Quartet* rec, int64_t i0, int64_t i1, const int64_t* range,
                 const double* P, double* K) {
    const int pab = cls / 9, pcd = cls % 9;
    EriArgs a;
    a.rec = rec;
    a.i0 = i0;
    a.i1 = i1;
    a.range = range;
    a.bmeta = c->d_pairmeta[pab];
    a.kmeta = c->d_pairmeta[pcd];
    if (prec == 2) {
        a.bra = c->d_pairdw[pab];
        a.ket = c->d_pairdw[pcd];
        a.boys = c->d_boysdw;
        a.P = c->d_Pdw;
    } else {
        a.bra = prec == 0 ? (const void*)c->d_pair64[pab] : (const void*)c->d_pair32[pab];
        a.ket = prec == 0 ? (const void*)c->d_pair64[pcd] : (const void*)c->d_pair32[pcd];
        a.boys = prec == 0 ? (const void*)c->d_boys64 : (const void*)c->d_boys32;
        a.P = prec == 0 ? (const void*)P : (const void*)c->d_P32;
    }
    a.K = K;
    a.nab = c->n_pairs[pab];
    a.ncd = c->n_pairs[pcd];
    return a;
}

int eri_launch(kx_ctx* c, int cls, int prec, const Quartet* rec, int64_t i0, int64_t i1, const int64_t* range,
               const double* P, double* K) {
    if (!range && i1 <= i0) return KX_OK;
    const int s = prec * NCLASS + cls;
    const EriKern kk = eri_kernel(cls, prec, c->eri_variant[s]);
    if (!kk.k) return set_err(c, KX_EINVAL, "bad class");
    KX_TRY(eri_prepare(c, s, c->eri_variant[s], kk));
    const int threads = eri_fit_threads(kk, c->eri_threads[s]);
    const size_t smem = (size_t)threads * kk.smem_per_thread;
    int64_t blocks;
    if (range) {
        // device-side range (captured launches): always a persistent grid
        blocks = (int64_t)std::max(c->eri_bpsm[s], 4) * c->n_sm;
    } else {
        blocks = (i1 - i0 + threads - 1) / threads;
        if (c->eri_bpsm[s] > 0) blocks = std::min<int64_t>(blocks, (int64_t)c->eri_bpsm[s] * c->n_sm);
    }
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)1 << 30));
    kk.k<<<(unsigned)blocks, threads, smem, c->stream>>>(eri_args(c, cls, prec, rec, i0, i1, range, P, K));
    return KX_OK;
}

double class_flops(int cls) {
    switch (cls / 9) {
        case 0: return class_flops_ab00(cls);
        case 1: return class_flops_ab01(cls);
        case 2: return class_flops_ab02(cls);
        case 3: return class_flops_ab10(cls);
        case 4: return class_flops_ab11(cls);
        case 5: return class_flops_ab12(cls);
        case 6: return class_flops_ab20(cls);
        case 7: return class_flops_ab21(cls);
        case 8: return class_flops_ab22(cls);
        default: return 0.0;
    }
}

}  // namespace kx
