// kx_split.cu -- the split threshold of a mixed-precision build, chosen
// from an error model of the FP32 quartets (kx_split_plan).
//
// A shell quartet q = (a,b,c,d) evaluated in FP32 perturbs the K shell block
// (a,c) by at most c_max[cls] eps32 beta_q and, for independent roundings,
// by a root-mean-square c_rms[cls] eps32 beta_q, with beta_q = S_ab ||P_bd||
// S_cd its Eq. 8 bound and eps32 = 2^-24.  The constants are per
// angular-momentum class, measured on GB300 by evaluating single shell
// quartets (single-shell leaves, pairwise distinct K blocks) in FP32 and in
// FP64 and taking max|dK_block| / (eps32 beta) over 2,000-2,500 quartets
// per class of (H2O)16 in the medium basis, their bounds spread over ten
// decades (`python -m paper_1401_6961_gb300.calibrate` repeats the
// measurement and prints these tables).  c_max is 1.5 times the largest
// ratio seen (1.2 to 6.2 by class); c_rms the root-mean-square ratio (0.16
// to 0.76).
//
// For a candidate split s, the FP32 quartets of a K shell block (a,c) are
// its quartets with beta <= s, so its error is bounded by
//     B_ac(s) = eps32 sum_{q in (a,c), beta_q <= s} c_max beta_q
// and of root-mean-square size
//     E_ac(s) = eps32 sqrt(sum_{q in (a,c), beta_q <= s} (c_rms beta_q)^2).
// A statistics variant of the shell screen's count pass accumulates both
// sums in quarter-octave bins of log2 beta for a sample of K shell blocks:
// every diagonal block (a,a), every block (a, a+1) of neighbours in tree
// order, and 4 n_shell seeded random blocks.  The plan takes the largest
// split s = tau 2^(k/4) whose 5-sigma estimate 5 max_ac E_ac(s) over the sampled
// blocks fits the budget, and reports that estimate and max_ac B_ac(s).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kx_internal.cuh"

namespace kx {

namespace {

// per class ((la*3 + lb)*3 + lc)*3 + ld
const float CMAX[NCLASS] = {
    6.4f, 5.28f, 7.2f, 7.06f, 3.61f, 7.66f, 6.6f, 4.31f, 4.39f,
    5.28f, 4.68f, 2.85f, 3.5f, 4.06f, 3.8f, 6.55f, 3.13f, 2.68f,
    5.1f, 4.19f, 2.05f, 3.99f, 2.63f, 2.0f, 9.32f, 3.31f, 2.49f,
    8.28f, 5.53f, 4.27f, 4.95f, 5.32f, 4.0f, 8.5f, 5.56f, 4.11f,
    5.38f, 2.68f, 2.16f, 3.76f, 3.73f, 2.44f, 4.21f, 3.24f, 2.31f,
    3.96f, 2.18f, 2.2f, 3.74f, 2.94f, 2.04f, 5.45f, 2.38f, 3.53f,
    8.01f, 5.44f, 5.66f, 6.22f, 9.32f, 5.22f, 6.57f, 7.3f, 4.99f,
    4.1f, 4.7f, 2.84f, 4.39f, 3.99f, 3.03f, 6.09f, 2.7f, 1.77f,
    4.19f, 2.47f, 1.83f, 4.14f, 2.92f, 2.1f, 5.25f, 2.36f, 3.01f,
};
const float CRMS[NCLASS] = {
    0.654f, 0.399f, 0.395f, 0.681f, 0.402f, 0.372f, 0.762f, 0.434f, 0.441f,
    0.416f, 0.247f, 0.218f, 0.357f, 0.246f, 0.195f, 0.451f, 0.257f, 0.227f,
    0.358f, 0.221f, 0.175f, 0.32f, 0.209f, 0.158f, 0.397f, 0.216f, 0.192f,
    0.642f, 0.37f, 0.338f, 0.561f, 0.389f, 0.32f, 0.683f, 0.396f, 0.359f,
    0.414f, 0.232f, 0.211f, 0.384f, 0.239f, 0.2f, 0.424f, 0.248f, 0.241f,
    0.358f, 0.186f, 0.163f, 0.288f, 0.201f, 0.157f, 0.368f, 0.199f, 0.183f,
    0.732f, 0.439f, 0.404f, 0.639f, 0.447f, 0.336f, 0.763f, 0.441f, 0.41f,
    0.428f, 0.271f, 0.219f, 0.411f, 0.248f, 0.2f, 0.459f, 0.26f, 0.22f,
    0.366f, 0.21f, 0.189f, 0.379f, 0.224f, 0.178f, 0.406f, 0.221f, 0.207f,
};

constexpr double EPS32 = 5.9604644775390625e-08;   // 2^-24
constexpr double SIGMAS = 5.0;                     // the estimate is 5 root-mean-square sizes
constexpr double SPLIT_MAX = 1.0;                  // largest candidate split
constexpr double TAU_FLOOR = 1e-14;                // lowest bin edge when tau = 0

// 64-bit linear congruential generator (Knuth's MMIX constants): the
// seeded block sample
struct Lcg {
    uint64_t s;
    uint32_t next() {
        s = s * 6364136223846793005ull + 1442695040888963407ull;
        return (uint32_t)(s >> 33);
    }
};

}  // namespace

int split_plan(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double budget, kx_stats* st) {
    if (c->n_sys != 1) return set_err(c, KX_ENOTIMPL, "split planning takes single-system contexts");
    if (!(budget > 0.0) || !std::isfinite(budget)) return set_err(c, KX_EINVAL, "the error budget must be > 0");
    const int n = c->n_shell;
    const int sym = o->symmetric;
    // the sampled blocks (tree positions), each once
    std::vector<int32_t> slot((size_t)n * n, -1);
    std::vector<std::pair<int, int>> blocks;
    auto add = [&](int a, int b) {
        if (a < 0 || b < 0 || a >= n || b >= n) return;
        if (sym && a > b) std::swap(a, b);
        int32_t& s = slot[(size_t)a * n + b];
        if (s < 0) {
            s = (int32_t)blocks.size();
            blocks.push_back({a, b});
        }
    };
    for (int a = 0; a < n; ++a) add(a, a);
    for (int a = 0; a + 1 < n; ++a) add(a, a + 1);
    Lcg g{0x9e3779b97f4a7c15ull ^ (uint64_t)n};
    for (int k = 0; k < 4 * n; ++k) add((int)(g.next() % (uint32_t)n), (int)(g.next() % (uint32_t)n));
    const double t0 = std::max(o->tau, TAU_FLOOR);
    const int nbin = std::max(1, (int)std::ceil(std::log2(SPLIT_MAX / t0) * PLAN_BINS_PER_OCTAVE));
    const size_t nacc = blocks.size() * (size_t)nbin * 2;
    if (!c->d_cmax) {
        KX_CUDA(c, cudaMalloc(&c->d_cmax, sizeof(CMAX)));
        KX_CUDA(c, cudaMalloc(&c->d_crms, sizeof(CRMS)));
        KX_CUDA(c, cudaMemcpy(c->d_cmax, CMAX, sizeof(CMAX), cudaMemcpyHostToDevice));
        KX_CUDA(c, cudaMemcpy(c->d_crms, CRMS, sizeof(CRMS), cudaMemcpyHostToDevice));
    }
    int32_t* d_slot = nullptr;
    double* d_acc = nullptr;
    cudaError_t e = cudaMalloc(&d_slot, sizeof(int32_t) * slot.size());
    if (e == cudaSuccess) e = cudaMalloc(&d_acc, sizeof(double) * nacc);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_slot, slot.data(), sizeof(int32_t) * slot.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_acc, 0, sizeof(double) * nacc, c->stream);
    if (e != cudaSuccess) {
        cudaFree(d_slot);
        cudaFree(d_acc);
        return cuda_check(c, e, "split plan buffers");
    }
    // the count pass with every quartet up to SPLIT_MAX classed as FP32
    kx_opts o2 = *o;
    o2.precision = KX_MIXED;
    o2.split_threshold = SPLIT_MAX;
    o2.split_budget = 0.0;
    kx_stats s2;
    std::memset(&s2, 0, sizeof(s2));
    c->plan_slot = d_slot;
    c->plan_acc = d_acc;
    c->plan_lbin0 = (float)std::log2(t0);
    c->plan_nbin = nbin;
    int r = drive(c, RUN_COUNT, P, ldp, &o2, nullptr, 0, &s2, nullptr, 0);
    c->plan_slot = nullptr;
    c->plan_acc = nullptr;
    std::vector<double> acc(nacc);
    if (r == KX_OK) {
        e = cudaMemcpyAsync(acc.data(), d_acc, sizeof(double) * nacc, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) r = cuda_check(c, e, "split plan read-back");
    }
    cudaFree(d_slot);
    cudaFree(d_acc);
    if (r != KX_OK) return r;
    // bin j holds beta in [t0 2^(j/4), t0 2^((j+1)/4)) (the bottom bin
    // everything below); the FP32 quartets of split s_k = t0 2^(k/4) are
    // bins j < k
    std::vector<double> s1(blocks.size(), 0.0), sq(blocks.size(), 0.0);
    double best = 0.0, best_est = 0.0, best_bnd = 0.0;
    for (int k = 1; k <= nbin; ++k) {
        double m1 = 0.0, m2 = 0.0;
        for (size_t b = 0; b < blocks.size(); ++b) {
            s1[b] += acc[(b * nbin + (k - 1)) * 2];
            sq[b] += acc[(b * nbin + (k - 1)) * 2 + 1];
            m1 = std::max(m1, s1[b]);
            m2 = std::max(m2, sq[b]);
        }
        const double est = SIGMAS * EPS32 * std::sqrt(m2), bnd = EPS32 * m1;
        if (est > budget) break;
        best = t0 * std::exp2((double)k / PLAN_BINS_PER_OCTAVE);
        best_est = est;
        best_bnd = bnd;
    }
    st->split_used = best;
    st->fp32_err_estimate = best_est;
    st->fp32_err_bound = best_bnd;
    return KX_OK;
}

}  // namespace kx
