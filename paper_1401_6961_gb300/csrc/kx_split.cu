// kx_split.cu -- the split threshold of a mixed-precision build, chosen
// from an error model of the FP32 quartets (kx_split_plan).
//
// A shell quartet q = (a,b,c,d) evaluated in FP32 perturbs the K shell block
// (a,c) by at most c_max[cls] eps32 beta_q and, for independent roundings,
// by a root-mean-square c_rms[cls] eps32 beta_q, with beta_q = S_ab ||P_bd||
// S_cd its Eq. 8 bound and eps32 = 2^-24.  The constants are per
// angular-momentum class, measured on GB300 by evaluating single shell
// quartets (single-shell leaves, pairwise distinct K blocks) in FP32 and in
// FP64 and taking max|dK_block| / (eps32 beta) over about 2,000 quartets per
// class of a water cluster in the medium basis, their bounds spread over
// ten decades (paper_1401_6961_gb300/calibrate.py repeats the measurement).
// c_max is 1.5 times the largest ratio seen; c_rms the root-mean-square
// ratio.
//
// For a candidate split s, the FP32 quartets of a K shell block (a,c) are
// its quartets with beta <= s, so its error is bounded by
//     B_ac(s) = eps32 sum_{q in (a,c), beta_q <= s} c_max beta_q
// and of root-mean-square size
//     E_ac(s) = eps32 sqrt(sum_{q in (a,c), beta_q <= s} (c_rms beta_q)^2).
// A statistics variant of the shell screen's count pass accumulates both
// sums in bins of log2 beta for a sample of K shell blocks: every diagonal
// block (a,a), every block (a, a+1) of neighbours in tree order, and 4
// n_shell seeded random blocks.  The plan takes the largest split
// s = tau 2^k whose 5-sigma estimate 5 max_ac E_ac(s) over the sampled
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
    6.45f, 5.33f, 7.25f, 7.11f, 3.66f, 7.71f, 6.65f, 4.36f, 4.44f,
    5.33f, 4.73f, 2.9f, 3.55f, 4.11f, 3.85f, 6.6f, 3.18f, 2.73f,
    5.15f, 4.24f, 2.1f, 4.04f, 2.68f, 2.05f, 9.37f, 3.36f, 2.54f,
    8.33f, 5.58f, 4.32f, 5.0f, 5.37f, 4.05f, 8.55f, 5.61f, 4.16f,
    5.43f, 2.73f, 2.21f, 3.81f, 3.78f, 2.49f, 4.26f, 3.29f, 2.36f,
    4.01f, 2.23f, 2.25f, 3.79f, 2.99f, 2.09f, 5.5f, 2.43f, 3.58f,
    8.06f, 5.49f, 5.71f, 6.27f, 9.37f, 5.27f, 6.62f, 7.35f, 5.04f,
    4.15f, 4.75f, 2.89f, 4.44f, 4.04f, 3.08f, 6.14f, 2.75f, 1.82f,
    4.24f, 2.52f, 1.88f, 4.19f, 2.97f, 2.15f, 5.3f, 2.41f, 3.06f,
};
const float CRMS[NCLASS] = {
    1.03f, 0.705f, 0.702f, 1.14f, 0.605f, 0.582f, 1.19f, 0.71f, 0.727f,
    0.727f, 0.428f, 0.376f, 0.626f, 0.383f, 0.299f, 0.737f, 0.391f, 0.358f,
    0.596f, 0.36f, 0.297f, 0.513f, 0.328f, 0.249f, 0.651f, 0.346f, 0.325f,
    1.03f, 0.619f, 0.639f, 0.866f, 0.611f, 0.533f, 1.11f, 0.654f, 0.567f,
    0.634f, 0.358f, 0.336f, 0.614f, 0.36f, 0.315f, 0.657f, 0.39f, 0.352f,
    0.64f, 0.307f, 0.282f, 0.461f, 0.301f, 0.241f, 0.583f, 0.303f, 0.267f,
    1.16f, 0.755f, 0.677f, 0.944f, 0.646f, 0.529f, 1.14f, 0.662f, 0.625f,
    0.701f, 0.474f, 0.351f, 0.688f, 0.383f, 0.308f, 0.727f, 0.409f, 0.347f,
    0.538f, 0.326f, 0.316f, 0.636f, 0.319f, 0.261f, 0.622f, 0.312f, 0.313f,
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
    const int nbin = std::max(1, (int)std::ceil(std::log2(SPLIT_MAX / t0)));
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
    // bin j holds beta in [t0 2^j, t0 2^(j+1)) (the bottom bin everything
    // below); the FP32 quartets of split s_k = t0 2^k are bins j < k
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
        best = t0 * std::ldexp(1.0, k);
        best_est = est;
        best_bnd = bnd;
    }
    st->split_used = best;
    st->fp32_err_estimate = best_est;
    st->fp32_err_bound = best_bnd;
    return KX_OK;
}

}  // namespace kx
