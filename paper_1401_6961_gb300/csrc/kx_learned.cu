// kx_learned.cu -- learned culling of leaf quartets (the growth direction in
// which a small network tightens the Schwarz x ||P|| bound of Eq. 8).
//
// Pieces, all driven through the C ABI:
//   * kx_traverse: the traversal alone; the leaf quartets stay on the device;
//   * kx_leaf_features: ten descriptors of every kept leaf quartet;
//   * an MLP 10 -> 64 -> 64 -> 64 -> 1 (GELU) predicting log10 ||dK_AC||_F of
//     the leaf quartet: FP32 training kernels (forward, backward, Adam) and a
//     BF16-operand / FP32-accumulate inference kernel;
//   * kx_cull_kept: drops a kept leaf quartet whose exact bound is at most
//     10 tau when its predicted contribution, times the square root of the
//     number of such quartets sharing its K block, is below a per-block
//     budget (a quartet whose bound exceeds 10 tau is always kept);
//   * kx_evaluate_kept / kx_exchange_leaves: the ERI stage over the kept
//     list or over an explicit list; kx_block_norms: ||K_AC||_F per quartet,
//     which, for a list whose (A,C) are all distinct, is the exact
//     contribution norm of each quartet (the training targets).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "kx_internal.cuh"

namespace kx {

constexpr int NF = KX_NFEAT;          // 10 features
constexpr int NH = KX_MLP_HIDDEN;     // 64
// parameter layout: mu[NF], inv_sigma[NF], W1[NH][NF], b1[NH], W2[NH][NH], b2[NH],
// W3[NH][NH], b3[NH], W4[NH], b4
constexpr int P_MU = 0, P_IS = NF, P_W1 = 2 * NF, P_B1 = P_W1 + NH * NF, P_W2 = P_B1 + NH,
              P_B2 = P_W2 + NH * NH, P_W3 = P_B2 + NH, P_B3 = P_W3 + NH * NH, P_W4 = P_B3 + NH,
              P_B4 = P_W4 + NH, P_N = P_B4 + 1;
static_assert(P_N == KX_MLP_NPARAM, "parameter count");

// ---------------------------------------------------------------------------
// leaf descriptors and features
// ---------------------------------------------------------------------------

// per leaf: centroid of its shell centres, radius, max l, min exponent
__global__ void k_leaf_desc(int nl, const int32_t* __restrict__ llo, const int32_t* __restrict__ lhi,
                            const double* __restrict__ tctr, const int32_t* __restrict__ tl,
                            const double* __restrict__ talpha, float* __restrict__ desc) {
    int L = blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nl) return;
    double c[3] = {0, 0, 0};
    int lmax = 0;
    double amin = 1e300;
    const int n = lhi[L] - llo[L];
    for (int s = llo[L]; s < lhi[L]; ++s) {
        for (int x = 0; x < 3; ++x) c[x] += tctr[3 * s + x];
        lmax = max(lmax, tl[s]);
        amin = fmin(amin, talpha[s]);
    }
    for (int x = 0; x < 3; ++x) c[x] /= n;
    double r = 0.0;
    for (int s = llo[L]; s < lhi[L]; ++s) {
        double d2 = 0.0;
        for (int x = 0; x < 3; ++x) d2 += (tctr[3 * s + x] - c[x]) * (tctr[3 * s + x] - c[x]);
        r = fmax(r, sqrt(d2));
    }
    float* o = desc + 8 * L;
    o[0] = (float)c[0]; o[1] = (float)c[1]; o[2] = (float)c[2];
    o[3] = (float)r;
    o[4] = (float)lmax;
    o[5] = (float)log10(amin);
    o[6] = 0.f; o[7] = 0.f;
}

__device__ __forceinline__ float lg10(double x) { return x > 0.0 ? (float)log10(x) : -300.f; }

__device__ __forceinline__ float dist3(const float* a, const float* b) {
    const float dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return sqrtf(dx * dx + dy * dy + dz * dz);
}

// features of every leaf quartet (A,B,C,D) of the list:
//  0 log10 ||Q_AB||, 1 log10 ||Q_CD||, 2 log10 ||P_BD||, 3 log10 beta,
//  4 |c_A - c_C|, 5 |c_B - c_D|, 6 |(c_A+c_B)/2 - (c_C+c_D)/2| (bohr),
//  7 largest block radius, 8 largest l, 9 log10 smallest exponent
__global__ void k_features(const Task* __restrict__ w, int64_t n, int nl, const double* __restrict__ S,
                           const double* __restrict__ Pn, const float* __restrict__ desc, float* __restrict__ feat) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Task t = w[i];
        const double sab = S[(int64_t)t.a * nl + t.b], scd = S[(int64_t)t.c * nl + t.d];
        const double pbd = Pn[(int64_t)t.b * nl + t.d];
        const double beta = __dmul_rn(__dmul_rn(sab, pbd), scd);
        const float* dA = desc + 8 * t.a;
        const float* dB = desc + 8 * t.b;
        const float* dC = desc + 8 * t.c;
        const float* dD = desc + 8 * t.d;
        float cab[3], ccd[3];
        for (int x = 0; x < 3; ++x) {
            cab[x] = 0.5f * (dA[x] + dB[x]);
            ccd[x] = 0.5f * (dC[x] + dD[x]);
        }
        float* f = feat + i * NF;
        f[0] = lg10(sab);
        f[1] = lg10(scd);
        f[2] = lg10(pbd);
        f[3] = lg10(beta);
        f[4] = dist3(dA, dC);
        f[5] = dist3(dB, dD);
        f[6] = dist3(cab, ccd);
        f[7] = fmaxf(fmaxf(dA[3], dB[3]), fmaxf(dC[3], dD[3]));
        f[8] = fmaxf(fmaxf(dA[4], dB[4]), fmaxf(dC[4], dD[4]));
        f[9] = fminf(fminf(dA[5], dB[5]), fminf(dC[5], dD[5]));
    }
}

// ---------------------------------------------------------------------------
// culling with the safety rule, stable compaction of the kept list
// ---------------------------------------------------------------------------

__device__ __forceinline__ double leaf_beta(const Task& t, int nl, const double* __restrict__ S,
                                            const double* __restrict__ Pn) {
    return __dmul_rn(__dmul_rn(S[(int64_t)t.a * nl + t.b], Pn[(int64_t)t.b * nl + t.d]), S[(int64_t)t.c * nl + t.d]);
}

// number of cullable quartets (bound <= 10 tau) of every K block (A,C)
__global__ void k_cull_count(const Task* __restrict__ w, int64_t n, int nl, const double* __restrict__ S,
                             const double* __restrict__ Pn, double ten_tau, int* __restrict__ cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Task t = w[i];
        if (leaf_beta(t, nl, S, Pn) <= ten_tau) atomicAdd(cnt + (int64_t)t.a * nl + t.c, 1);
    }
}

// Culls quartet i iff its bound is at most 10 tau and its predicted
// contribution times the number m of cullable quartets of its K block is
// below the budget: the predicted sum of what any K block loses then stays
// below the budget whatever the signs of the dropped contributions.  (A
// root-sum-square rule, sqrt(m) in place of m, let (H2O)_256 lose 1.5e-8 at
// tau = 1e-8.)  A quartet whose exact bound exceeds 10 tau is never culled.
__global__ void k_cull_flags(const Task* __restrict__ w, int64_t n, int nl, const double* __restrict__ S,
                             const double* __restrict__ Pn, const float* __restrict__ pred, double ten_tau,
                             float log10_budget, const int* __restrict__ cnt, int64_t* __restrict__ keep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const Task t = w[i];
        bool cull = false;
        if (leaf_beta(t, nl, S, Pn) <= ten_tau) {
            const int m = cnt[(int64_t)t.a * nl + t.c];
            cull = pred[i] + log10f((float)m) < log10_budget;
        }
        keep[i] = cull ? 0 : 1;
    }
}

__global__ void k_compact(const Task* __restrict__ w, int64_t n, const int64_t* __restrict__ keep,
                          const int64_t* __restrict__ off, Task* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (keep[i]) out[off[i]] = w[i];
}

// ||K_AC||_F of every leaf quartet of a list (K in user order; the leaves'
// functions are gathered through the tree order)
__global__ void k_block_norms(const Task* __restrict__ w, int64_t n, const int32_t* __restrict__ llo,
                              const int32_t* __restrict__ lhi, const int32_t* __restrict__ tl,
                              const int32_t* __restrict__ tfoff, const double* __restrict__ K, int64_t ldk,
                              double* __restrict__ out) {
    const int64_t q = blockIdx.x;
    if (q >= n) return;
    const Task t = w[q];
    double s = 0.0;
    // shells of A x shells of C, spread over the block's threads
    const int na = lhi[t.a] - llo[t.a], nc = lhi[t.c] - llo[t.c];
    for (int k = threadIdx.x; k < na * nc; k += blockDim.x) {
        const int a = llo[t.a] + k / nc, c = llo[t.c] + k % nc;
        const int fa = tfoff[a], fc = tfoff[c], ma = ncart(tl[a]), mc = ncart(tl[c]);
        for (int i = 0; i < ma; ++i)
            for (int j = 0; j < mc; ++j) {
                const double v = K[(int64_t)(fa + i) * ldk + fc + j];
                s += v * v;
            }
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
        if ((int)threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sqrt(sh[0]);
}

// ---------------------------------------------------------------------------
// the MLP
// ---------------------------------------------------------------------------

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

constexpr int INF_T = 64;    // samples per inference block

// BF16 inference: weights and activations rounded to BF16, products
// accumulated in FP32, GELU in FP32.  Activations live in shared memory,
// feature-major so that thread t reads column t.
__global__ void __launch_bounds__(INF_T) k_mlp_infer(const float* __restrict__ prm, const float* __restrict__ feat,
                                                     int64_t n, float* __restrict__ pred) {
    __shared__ __nv_bfloat16 w1[NH * NF], w2[NH * NH], w3[NH * NH], w4[NH];
    __shared__ float b1[NH], b2[NH], b3[NH], mu[NF], is[NF];
    __shared__ __nv_bfloat16 act[2][NH][INF_T];
    for (int k = threadIdx.x; k < NH * NF; k += INF_T) w1[k] = __float2bfloat16(prm[P_W1 + k]);
    for (int k = threadIdx.x; k < NH * NH; k += INF_T) {
        w2[k] = __float2bfloat16(prm[P_W2 + k]);
        w3[k] = __float2bfloat16(prm[P_W3 + k]);
    }
    for (int k = threadIdx.x; k < NH; k += INF_T) {
        w4[k] = __float2bfloat16(prm[P_W4 + k]);
        b1[k] = prm[P_B1 + k];
        b2[k] = prm[P_B2 + k];
        b3[k] = prm[P_B3 + k];
    }
    if (threadIdx.x < NF) {
        mu[threadIdx.x] = prm[P_MU + threadIdx.x];
        is[threadIdx.x] = prm[P_IS + threadIdx.x];
    }
    __syncthreads();
    const float b4 = prm[P_B4];
    const int t = threadIdx.x;
    for (int64_t base = blockIdx.x * (int64_t)INF_T; base < n; base += (int64_t)gridDim.x * INF_T) {
        const int64_t i = base + t;
        __nv_bfloat16 x[NF];
        for (int f = 0; f < NF; ++f)
            x[f] = __float2bfloat16(i < n ? (feat[i * NF + f] - mu[f]) * is[f] : 0.f);
        for (int j = 0; j < NH; ++j) {
            float acc = b1[j];
#pragma unroll
            for (int f = 0; f < NF; ++f) acc = fmaf(__bfloat162float(w1[j * NF + f]), __bfloat162float(x[f]), acc);
            act[0][j][t] = __float2bfloat16(gelu(acc));
        }
        for (int j = 0; j < NH; ++j) {
            float acc = b2[j];
#pragma unroll 16
            for (int k = 0; k < NH; ++k)
                acc = fmaf(__bfloat162float(w2[j * NH + k]), __bfloat162float(act[0][k][t]), acc);
            act[1][j][t] = __float2bfloat16(gelu(acc));
        }
        for (int j = 0; j < NH; ++j) {
            float acc = b3[j];
#pragma unroll 16
            for (int k = 0; k < NH; ++k)
                acc = fmaf(__bfloat162float(w3[j * NH + k]), __bfloat162float(act[1][k][t]), acc);
            act[0][j][t] = __float2bfloat16(gelu(acc));
        }
        float y = b4;
#pragma unroll 16
        for (int k = 0; k < NH; ++k) y = fmaf(__bfloat162float(w4[k]), __bfloat162float(act[0][k][t]), y);
        if (i < n) pred[i] = y;
    }
}

constexpr int TR_S = 64;     // samples per training block
constexpr int TR_T = 256;    // threads per training block

struct TrainSmem {
    float a0[TR_S][NF];
    float z1[TR_S][NH], a1[TR_S][NH];
    float z2[TR_S][NH], a2[TR_S][NH];
    float z3[TR_S][NH], a3[TR_S][NH];
    float d[TR_S][NH], d2[TR_S][NH];
    float dy[TR_S];
};

// Z[s][j] = b[j] + sum_k A[s][k] W[j][k], then A' = gelu(Z); thread t owns
// output column j = t % NH for samples (t / NH) * 16 .. +16
template <int NIN>
__device__ __forceinline__ void dense_fwd(const float (*A)[NIN], const float* __restrict__ W,
                                          const float* __restrict__ b, float (*Z)[NH], float (*Aout)[NH], int ns) {
    const int j = threadIdx.x % NH, s0 = (threadIdx.x / NH) * (TR_S / (TR_T / NH));
    float w[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k) w[k] = W[j * NIN + k];
    const float bj = b[j];
    for (int s = s0; s < s0 + TR_S / (TR_T / NH); ++s) {
        float acc = bj;
#pragma unroll
        for (int k = 0; k < NIN; ++k) acc = fmaf(A[s][k], w[k], acc);
        Z[s][j] = acc;
        Aout[s][j] = s < ns ? gelu(acc) : 0.f;
    }
}

// Mean-squared-error loss 0.5 * mean (y - t)^2 and its gradient, summed
// into grad (atomics); the normalisation parameters get no gradient.
__global__ void __launch_bounds__(TR_T) k_mlp_grad(const float* __restrict__ prm, const float* __restrict__ feat,
                                                   const float* __restrict__ tgt, int64_t n, float inv_n,
                                                   float* __restrict__ grad, double* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TrainSmem& sm = *reinterpret_cast<TrainSmem*>(smraw);
    const int64_t s_base = blockIdx.x * (int64_t)TR_S;
    const int ns = (int)std::min<int64_t>(TR_S, n - s_base);
    const int t = threadIdx.x;
    for (int k = t; k < TR_S * NF; k += TR_T) {
        const int s = k / NF, f = k % NF;
        sm.a0[s][f] = s < ns ? (feat[(s_base + s) * NF + f] - prm[P_MU + f]) * prm[P_IS + f] : 0.f;
    }
    __syncthreads();
    dense_fwd<NF>(sm.a0, prm + P_W1, prm + P_B1, sm.z1, sm.a1, ns);
    __syncthreads();
    dense_fwd<NH>(sm.a1, prm + P_W2, prm + P_B2, sm.z2, sm.a2, ns);
    __syncthreads();
    dense_fwd<NH>(sm.a2, prm + P_W3, prm + P_B3, sm.z3, sm.a3, ns);
    __syncthreads();
    // output and loss
    if (t < TR_S) {
        float y = prm[P_B4];
        for (int k = 0; k < NH; ++k) y = fmaf(sm.a3[t][k], prm[P_W4 + k], y);
        float e = t < ns ? y - tgt[s_base + t] : 0.f;
        sm.dy[t] = e * inv_n;
        double l = 0.5 * (double)e * e * inv_n;
        for (int d = 16; d > 0; d >>= 1) l += __shfl_xor_sync(0xffffffffu, l, d);
        if ((t & 31) == 0) atomicAdd(loss, l);
    }
    __syncthreads();
    // layer 4: gW4[k] = sum_s dy[s] a3[s][k]; d[s][k] = dy[s] W4[k] gelu'(z3)
    if (t < NH) {
        float g = 0.f;
        for (int s = 0; s < ns; ++s) g = fmaf(sm.dy[s], sm.a3[s][t], g);
        atomicAdd(grad + P_W4 + t, g);
    }
    if (t == 0) {
        float g = 0.f;
        for (int s = 0; s < ns; ++s) g += sm.dy[s];
        atomicAdd(grad + P_B4, g);
    }
    for (int k = t; k < TR_S * NH; k += TR_T) {
        const int s = k / NH, j = k % NH;
        sm.d[s][j] = sm.dy[s] * prm[P_W4 + j] * gelu_d(sm.z3[s][j]);
    }
    __syncthreads();
    // hidden layers 3 and 2: gW = D^T A_prev, gb = sum D, D_prev = (D W) * gelu'(z_prev)
    const float* Wl[2] = {prm + P_W3, prm + P_W2};
    const int gW[2] = {P_W3, P_W2}, gB[2] = {P_B3, P_B2};
    float (*Aprev[2])[NH] = {sm.a2, sm.a1};
    float (*Zprev[2])[NH] = {sm.z2, sm.z1};
    float (*Din)[NH] = sm.d;
    float (*Dout)[NH] = sm.d2;
    for (int layer = 0; layer < 2; ++layer) {
        for (int k = t; k < NH * NH; k += TR_T) {
            const int j = k / NH, i = k % NH;
            float g = 0.f;
            for (int s = 0; s < ns; ++s) g = fmaf(Din[s][j], Aprev[layer][s][i], g);
            atomicAdd(grad + gW[layer] + k, g);
        }
        if (t < NH) {
            float g = 0.f;
            for (int s = 0; s < ns; ++s) g += Din[s][t];
            atomicAdd(grad + gB[layer] + t, g);
        }
        for (int k = t; k < TR_S * NH; k += TR_T) {
            const int s = k / NH, i = k % NH;
            float acc = 0.f;
            for (int j = 0; j < NH; ++j) acc = fmaf(Din[s][j], Wl[layer][j * NH + i], acc);
            Dout[s][i] = acc * gelu_d(Zprev[layer][s][i]);
        }
        __syncthreads();
        float (*tmp)[NH] = Din;
        Din = Dout;
        Dout = tmp;
    }
    // layer 1: gW1 = D^T a0, gb1 = sum D
    for (int k = t; k < NH * NF; k += TR_T) {
        const int j = k / NF, f = k % NF;
        float g = 0.f;
        for (int s = 0; s < ns; ++s) g = fmaf(Din[s][j], sm.a0[s][f], g);
        atomicAdd(grad + P_W1 + k, g);
    }
    if (t < NH) {
        float g = 0.f;
        for (int s = 0; s < ns; ++s) g += Din[s][t];
        atomicAdd(grad + P_B1 + t, g);
    }
}

__global__ void k_adam(float* __restrict__ prm, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 2 * NF || i >= P_N) return;   // the normalisation is not trained
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    prm[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

int leaf_desc(kx_ctx* c, float** out) {
    const int nl = c->levels[c->depth].n;
    KX_TRY(grow(c, &c->d_leafdesc, &c->leafdesc_cap, (size_t)8 * nl));
    k_leaf_desc<<<(nl + 127) / 128, 128, 0, c->stream>>>(nl, c->d_leaf_lo, c->d_leaf_hi, c->d_tctr, c->d_tl,
                                                         c->d_talpha, c->d_leafdesc);
    *out = c->d_leafdesc;
    return KX_OK;
}

}  // namespace kx

using namespace kx;

namespace {
struct Guard {
    int prev = -1;
    bool ok = true;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
        if (!ok) (void)cudaGetLastError();
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" {

int kx_traverse(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, int64_t* n_leaves) {
    if (c && c->n_sys != 1) return set_err(c, KX_ENOTIMPL, "single-system contexts only");
    if (!c) return KX_EINVAL;
    if (!P || !o || !n_leaves) return set_err(c, KX_EINVAL, "null argument");
    if (ldp < c->n_fn) return set_err(c, KX_EINVAL, "leading dimension smaller than n_fn");
    if (!std::isfinite(o->tau) || o->tau < 0.0) return set_err(c, KX_EINVAL, "tau must be >= 0");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    Guard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    kx_stats st;
    std::memset(&st, 0, sizeof(st));
    KX_TRY(drive(c, RUN_TRAVERSE, P, ldp, o, nullptr, 0, &st, nullptr, 0));
    c->kept_tau = o->tau;
    *n_leaves = (int64_t)c->keep_n;
    return KX_OK;
}

int kx_evaluate_kept(kx_ctx* c, const double* P, int64_t ldp, const kx_opts* o, double* K, int64_t ldk,
                     kx_stats* st) {
    if (c && c->n_sys != 1) return set_err(c, KX_ENOTIMPL, "single-system contexts only");
    if (!c) return KX_EINVAL;
    if (!P || !K || !o) return set_err(c, KX_EINVAL, "null argument");
    if (ldp < c->n_fn || ldk < c->n_fn) return set_err(c, KX_EINVAL, "leading dimension smaller than n_fn");
    if (o->precision < KX_FP64 || o->precision > KX_MIXED_DW) return set_err(c, KX_EINVAL, "bad precision");
    if (!c->keep_valid) return set_err(c, KX_ESTATE, "no kept leaf list (kx_traverse first)");
    Guard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    kx_stats local;
    kx_stats* s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_CAND, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_ERR, 0, sizeof(unsigned long long), c->stream));
    return drive(c, RUN_EVALUATE, P, ldp, o, K, ldk, s, c->d_keep, (int64_t)c->keep_n);
}

int kx_exchange_leaves(kx_ctx* c, const double* P, int64_t ldp, const int32_t* leaves, int64_t n, const kx_opts* o,
                       double* K, int64_t ldk, kx_stats* st) {
    if (c && c->n_sys != 1) return set_err(c, KX_ENOTIMPL, "single-system contexts only");
    if (!c) return KX_EINVAL;
    if (!P || !K || !o || (n > 0 && !leaves) || n < 0) return set_err(c, KX_EINVAL, "bad argument");
    if (ldp < c->n_fn || ldk < c->n_fn) return set_err(c, KX_EINVAL, "leading dimension smaller than n_fn");
    if (o->precision < KX_FP64 || o->precision > KX_MIXED_DW) return set_err(c, KX_EINVAL, "bad precision");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    const int nl = c->levels[c->depth].n;
    std::vector<Task> h(n);
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 4; ++k)
            if (leaves[4 * i + k] < 0 || leaves[4 * i + k] >= nl) return set_err(c, KX_EINVAL, "leaf out of range");
        h[i] = Task{(uint16_t)leaves[4 * i], (uint16_t)leaves[4 * i + 1], (uint16_t)leaves[4 * i + 2],
                    (uint16_t)leaves[4 * i + 3]};
    }
    Guard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    KX_TRY(grow(c, &c->d_list, &c->list_cap, (size_t)std::max<int64_t>(n, 1)));
    if (n > 0) KX_CUDA(c, cudaMemcpyAsync(c->d_list, h.data(), sizeof(Task) * n, cudaMemcpyHostToDevice, c->stream));
    kx_stats local;
    kx_stats* s = st ? st : &local;
    std::memset(s, 0, sizeof(*s));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_CAND, 0, sizeof(unsigned long long), c->stream));
    KX_CUDA(c, cudaMemsetAsync(c->d_counters + CTR_ERR, 0, sizeof(unsigned long long), c->stream));
    int r = drive(c, RUN_EVALUATE, P, ldp, o, K, ldk, s, c->d_list, n);
    if (r == KX_OK) KX_CUDA(c, cudaStreamSynchronize(c->stream));
    return r;
}

int kx_leaf_features(kx_ctx* c, float* feat, int64_t cap, int64_t* n) {
    if (c && c->n_sys != 1) return set_err(c, KX_ENOTIMPL, "single-system contexts only");
    if (!c) return KX_EINVAL;
    if (!n || cap < 0 || (cap > 0 && !feat)) return set_err(c, KX_EINVAL, "bad argument");
    if (!c->keep_valid || !c->have_pq) return set_err(c, KX_ESTATE, "no kept leaf list (kx_traverse first)");
    *n = (int64_t)c->keep_n;
    if ((int64_t)c->keep_n > cap) return set_err(c, KX_ECAPACITY, "feature buffer too small");
    Guard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    float* desc = nullptr;
    KX_TRY(leaf_desc(c, &desc));
    const int D = c->depth, nl = c->levels[D].n;
    if (c->keep_n > 0) {
        unsigned grid = (unsigned)std::min<size_t>((c->keep_n + 255) / 256, (size_t)c->n_sm * 32);
        k_features<<<grid, 256, 0, c->stream>>>(c->d_keep, (int64_t)c->keep_n, nl, c->d_nrm_s + c->pyr_off[D],
                                               c->d_nrm_p + c->pyr_off[D], desc, feat);
    }
    KX_CUDA(c, cudaGetLastError());
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    return KX_OK;
}

int kx_cull_kept(kx_ctx* c, const float* pred, double tau, double log10_budget, int64_t* n_kept) {
    if (c && c->n_sys != 1) return set_err(c, KX_ENOTIMPL, "single-system contexts only");
    if (!c) return KX_EINVAL;
    if (!n_kept || (!pred && c->keep_n > 0) || !std::isfinite(tau) || tau < 0.0 || std::isnan(log10_budget))
        return set_err(c, KX_EINVAL, "bad argument");
    if (!c->keep_valid || !c->have_pq) return set_err(c, KX_ESTATE, "no kept leaf list (kx_traverse first)");
    Guard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    const int64_t n = (int64_t)c->keep_n;
    const int D = c->depth, nl = c->levels[D].n;
    if (n == 0) {
        *n_kept = 0;
        return KX_OK;
    }
    KX_TRY(grow(c, &c->d_scan, &c->scan_cap, (size_t)2 * n + ((size_t)nl * nl + 1) / 2 + 1));
    KX_TRY(grow(c, &c->d_list, &c->list_cap, (size_t)n));
    int64_t* keep = c->d_scan;
    int64_t* off = c->d_scan + n;
    int* cnt = reinterpret_cast<int*>(c->d_scan + 2 * n);
    const double* S = c->d_nrm_s + c->pyr_off[D];
    const double* Pn = c->d_nrm_p + c->pyr_off[D];
    unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)c->n_sm * 32);
    KX_CUDA(c, cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)nl * nl, c->stream));
    k_cull_count<<<grid, 256, 0, c->stream>>>(c->d_keep, n, nl, S, Pn, 10.0 * tau, cnt);
    k_cull_flags<<<grid, 256, 0, c->stream>>>(c->d_keep, n, nl, S, Pn, pred, 10.0 * tau, (float)log10_budget, cnt,
                                            keep);
    int64_t total = 0;
    KX_TRY(exclusive_scan(c, keep, off, n, &total));
    k_compact<<<grid, 256, 0, c->stream>>>(c->d_keep, n, keep, off, c->d_list);
    KX_CUDA(c, cudaMemcpyAsync(c->d_keep, c->d_list, sizeof(Task) * total, cudaMemcpyDeviceToDevice, c->stream));
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    c->keep_n = (size_t)total;
    *n_kept = total;
    return KX_OK;
}

int kx_block_norms(kx_ctx* c, const double* K, int64_t ldk, const int32_t* leaves, int64_t n, double* norms) {
    if (c && c->n_sys != 1) return set_err(c, KX_ENOTIMPL, "single-system contexts only");
    if (!c) return KX_EINVAL;
    if (!K || ldk < c->n_fn || n < 0 || (n > 0 && (!leaves || !norms))) return set_err(c, KX_EINVAL, "bad argument");
    if (!c->have_tree) return set_err(c, KX_ESTATE, "kx_build_tree must come first");
    const int nl = c->levels[c->depth].n;
    std::vector<Task> h(n);
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 4; ++k)
            if (leaves[4 * i + k] < 0 || leaves[4 * i + k] >= nl) return set_err(c, KX_EINVAL, "leaf out of range");
        h[i] = Task{(uint16_t)leaves[4 * i], (uint16_t)leaves[4 * i + 1], (uint16_t)leaves[4 * i + 2],
                    (uint16_t)leaves[4 * i + 3]};
    }
    if (n == 0) return KX_OK;
    Guard g(c->device);
    if (!g.ok) return set_err(c, KX_ECUDA, "cudaSetDevice failed");
    KX_TRY(grow(c, &c->d_list, &c->list_cap, (size_t)n));
    double* d_out = nullptr;
    KX_CUDA(c, cudaMalloc(&d_out, sizeof(double) * n));
    cudaMemcpyAsync(c->d_list, h.data(), sizeof(Task) * n, cudaMemcpyHostToDevice, c->stream);
    k_block_norms<<<(unsigned)n, 256, 0, c->stream>>>(c->d_list, n, c->d_leaf_lo, c->d_leaf_hi, c->d_tl, c->d_tfoff,
                                                     K, ldk, d_out);
    cudaMemcpyAsync(norms, d_out, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_check(c, e, "kx_block_norms");
    return KX_OK;
}

int kx_mlp_infer_bf16(const float* params, const float* feat, int64_t n, float* pred, void* stream) {
    if (n < 0 || (n > 0 && (!params || !feat || !pred))) return KX_EINVAL;
    if (n == 0) return KX_OK;
    int dev = 0, n_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || n_sm < 1)
        return KX_ECUDA;
    unsigned grid = (unsigned)std::min<int64_t>((n + INF_T - 1) / INF_T, (int64_t)n_sm * 8);
    k_mlp_infer<<<grid, INF_T, 0, (cudaStream_t)stream>>>(params, feat, n, pred);
    if (cudaGetLastError() != cudaSuccess) return KX_ECUDA;
    return KX_OK;
}

int kx_mlp_loss_grad(const float* params, const float* feat, const float* target, int64_t n, float* grad,
                     double* loss, void* stream) {
    if (n <= 0 || !params || !feat || !target || !grad || !loss) return KX_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainSmem)) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            return KX_ECUDA;
        }
        attr = true;
    }
    double* d_loss = nullptr;
    if (cudaMalloc(&d_loss, sizeof(double)) != cudaSuccess) {
        (void)cudaGetLastError();
        return KX_ENOMEM;
    }
    cudaMemsetAsync(d_loss, 0, sizeof(double), st);
    cudaMemsetAsync(grad, 0, sizeof(float) * P_N, st);
    unsigned grid = (unsigned)((n + TR_S - 1) / TR_S);
    k_mlp_grad<<<grid, TR_T, sizeof(TrainSmem), st>>>(params, feat, target, n, 1.f / (float)n, grad, d_loss);
    cudaMemcpyAsync(loss, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaFree(d_loss);
    return e == cudaSuccess ? KX_OK : KX_ECUDA;
}

int kx_mlp_adam(float* params, const float* grad, float* m, float* v, float lr, int32_t step, void* stream) {
    if (!params || !grad || !m || !v || step < 1 || !(lr > 0.f)) return KX_EINVAL;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
    k_adam<<<(P_N + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? KX_OK : KX_ECUDA;
}

}  // extern "C"
