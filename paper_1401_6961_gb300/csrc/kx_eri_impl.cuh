// kx_eri_impl.cuh -- McMurchie-Davidson shell-quartet kernels, one
// instantiation per angular-momentum class (la,lb,lc,ld) and precision.
//
// One thread evaluates one surviving shell quartet (a,b,c,d) (the leaf
// contractions of Eq. 7 restricted to the quartets that pass Eq. 8) and
// contracts it straight into its K block,
//
//   K_{mu nu} += sum_{lam in b, sig in d} (mu lam|nu sig) P_{lam sig},
//   (mu lam|nu sig) = pref * sum_{h in bra} E^{ab}_{mu lam,h}
//                      sum_{h' in ket} (-1)^{|h'|} E^{cd}_{nu sig,h'} R_{h+h'},
//
// with Hermite indices h = (t,u,v).  R_{tuv} comes from the Boys function
// F_n(T), T = rho |P-Q|^2, by the usual Hermite recursion.  The contraction
// with P is folded into the Hermite-to-Cartesian transform, in whichever of
// two orders has the smaller middle (R-contraction) step:
//   order A (loop nu, lam):  T_{h'} = sum_sig E^{cd}_{nu sig,h'} P_{lam sig},
//                            U_h = sum_{h'} (-1)^{|h'|} R_{h+h'} T_{h'},
//                            K_{mu nu} += sum_h E^{ab}_{mu lam,h} U_h;
//   order B (loop mu, sig):  W_h = sum_lam E^{ab}_{mu lam,h} P_{lam sig},
//                            V_{h'} = sum_h R_{h+h'} W_h,
//                            K_{mu nu} += sum_{h'} (-1)^{|h'|} E^{cd}_{nu sig,h'} V_{h'}.
// Every loop is a compile-time loop, so all Hermite and Cartesian indices
// are constants and the intermediates live in registers.  Per-thread K
// partials are reduced across the warp over runs of equal (a,c) before the
// FP64 atomic add into K.
#pragma once

#include <utility>

#include "kx_dw.cuh"
#include "kx_internal.cuh"

namespace kx {

// ---------------------------------------------------------------------------
// compile-time loops
// ---------------------------------------------------------------------------

template <int N>
using ic = std::integral_constant<int, N>;

template <typename F, int... I>
__device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, I...>) {
    (f(ic<I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
    if constexpr (N > 0) sfor_impl(f, std::make_integer_sequence<int, N>{});
}
#define KX_CV(x) decltype(x)::value

__host__ __device__ constexpr int imax0(int x) { return x > 0 ? x : 0; }

// h = (t,u,v) is reached by some component pair whose first member has the
// fixed powers (x,y,z) and whose second member has total l2:
// sum of the excesses over (x,y,z) must not exceed l2.
__host__ __device__ constexpr bool reach(int t, int u, int v, int x, int y, int z, int l2) {
    return imax0(t - x) + imax0(u - y) + imax0(v - z) <= l2;
}

// ---------------------------------------------------------------------------
// precision traits
// ---------------------------------------------------------------------------

template <typename R>
struct Real;
template <>
struct Real<double> {
    __device__ static double sqrt_(double x) { return sqrt(x); }
    __device__ static double exp_(double x) { return exp(x); }
    __device__ static int rnd(double x) { return __double2int_rn(x); }
};
template <>
struct Real<float> {
    __device__ static float sqrt_(float x) { return sqrtf(x); }
    __device__ static float exp_(float x) { return expf(x); }
    __device__ static int rnd(float x) { return __float2int_rn(x); }
};
// Double-word FP32.  exp only enters the large-T Boys recursion as e^{-T}
// with T >= 40, where it is below 3e-10 of the term it corrects, so its
// FP32 value (relative error ~1e-7) is accurate far beyond double-word
// precision there.
template <>
struct Real<dw> {
    __device__ static dw sqrt_(dw x) { return dw_sqrt(x); }
    __device__ static dw exp_(dw x) { return dw(expf(x.hi), 0.f); }
    __device__ static int rnd(dw x) { return __float2int_rn(x.hi); }
};

// read-only loads of a value of the kernel's precision
__device__ __forceinline__ double ld_(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ld_(const float* p) { return __ldg(p); }
__device__ __forceinline__ dw ld_(const dw* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return dw(v.x, v.y);
}
__device__ __forceinline__ double shfl_up(unsigned mask, double v, int d) { return __shfl_up_sync(mask, v, d); }
__device__ __forceinline__ float shfl_up(unsigned mask, float v, int d) { return __shfl_up_sync(mask, v, d); }

// FP32 -> FP64 by bit manipulation (integer pipe), subnormals flushed.
__device__ __forceinline__ double f2d_bits(float f) {
    uint32_t u = __float_as_uint(f);
    uint32_t e = (u >> 23) & 0xffu;
    uint64_t s = (uint64_t)(u & 0x80000000u) << 32;
    if (e == 0) return __longlong_as_double((long long)s);
    uint64_t m = (uint64_t)(u & 0x7fffffu) << 29;
    uint64_t ee = (e == 0xffu) ? 0x7ffull : (uint64_t)(e + 896u);
    return __longlong_as_double((long long)(s | (ee << 52) | m));
}
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d_bits(x); }
__device__ __forceinline__ double to_f64(dw x) { return dw_to_f64(x); }

// ---------------------------------------------------------------------------
// Boys function and Hermite integrals
// ---------------------------------------------------------------------------

// G_n = pref (-2 rho)^n F_n(T), n = 0..L.
// T < BOYS_TMAX: seven-term Taylor series about the nearest grid point,
//   F_m(T_i + d) = sum_k (-d)^k / k! F_{m+k}(T_i).
// T >= BOYS_TMAX: F_0 = (1/2) sqrt(pi/T) (erfc(sqrt T) < 1e-18 there) and
//   the upward recursion F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T), stable for
//   2m+1 < 2T; in FP32 the e^{-T} term is below the rounding unit and the
//   scaled form G_{n+1} = -G_n (2n+1) / |P-Q|^2 avoids underflow.
template <int L, typename R>
__device__ __forceinline__ void boys_scaled(R* G, R T, R rho, R r2, R pref, const R* __restrict__ tab) {
    if (T < R(BOYS_TMAX)) {
        int ig = Real<R>::rnd(T * R(BOYS_DENS));
        R d = T - R(ig) * R(1.0 / BOYS_DENS);
        R md[6];
        sfor<6>([&](auto k_) {
            constexpr int k = KX_CV(k_);
            md[k] = -d * R(1.0 / (k + 1));
        });
        // the L+7 table values F_0..F_{L+6}(T_i) of the row
        R rv[L + 7];
        if constexpr (sizeof(R) == 4) {
            constexpr int NV = (L + 7 + 3) / 4;
            const float4* row4 = reinterpret_cast<const float4*>(tab + ig * BOYS32_ROW);
            sfor<NV>([&](auto v_) {
                constexpr int v = KX_CV(v_);
                const float4 q = __ldg(row4 + v);
                if constexpr (4 * v + 0 < L + 7) rv[4 * v + 0] = q.x;
                if constexpr (4 * v + 1 < L + 7) rv[4 * v + 1] = q.y;
                if constexpr (4 * v + 2 < L + 7) rv[4 * v + 2] = q.z;
                if constexpr (4 * v + 3 < L + 7) rv[4 * v + 3] = q.w;
            });
        } else {
            const R* row = tab + ig * (BOYS_M + 1);
            sfor<L + 7>([&](auto k_) { rv[KX_CV(k_)] = ld_(row + KX_CV(k_)); });
        }
        R s = pref;
        const R m2r = R(-2) * rho;
        sfor<L + 1>([&](auto m_) {
            constexpr int m = KX_CV(m_);
            R acc = rv[m + 6];
            sfor<6>([&](auto k_) {
                constexpr int k = 5 - KX_CV(k_);
                acc = rv[m + k] + acc * md[k];
            });
            G[m] = s * acc;
            if constexpr (m < L) s *= m2r;
        });
    } else {
        R f0 = R(0.5) * Real<R>::sqrt_(R(PI) / T);
        if constexpr (sizeof(R) == 8) {
            R e = Real<R>::exp_(-T);
            R inv2t = R(0.5) / T;
            R F = f0, s = pref;
            const R m2r = R(-2) * rho;
            sfor<L + 1>([&](auto m_) {
                constexpr int m = KX_CV(m_);
                G[m] = s * F;
                if constexpr (m < L) {
                    F = (R(2 * m + 1) * F - e) * inv2t;
                    s *= m2r;
                }
            });
        } else {
            R inv_r2 = R(1) / r2;
            R g = pref * f0;
            sfor<L + 1>([&](auto m_) {
                constexpr int m = KX_CV(m_);
                G[m] = g;
                if constexpr (m < L) g *= R(-(2 * m + 1)) * inv_r2;
            });
        }
    }
}

// R_{tuv} (n = 0) for t+u+v <= L, in place from the highest n down:
//   R^n_{t,u,v} = (t-1) R^{n+1}_{t-2,u,v} + X R^{n+1}_{t-1,u,v}  (t > 0),
// likewise in u (t = 0) and v (t = u = 0); R^n_{000} = G_n.
template <int L, typename R>
__device__ __forceinline__ void hermite_r(R* Rt, const R* G, R X, R Y, R Z) {
    Rt[0] = G[L];
    sfor<L>([&](auto k_) {
        constexpr int n = L - 1 - KX_CV(k_);
        sfor<L - n>([&](auto j_) {
            constexpr int j = L - n - KX_CV(j_);
            sfor<j + 1>([&](auto t_) {
                constexpr int t = KX_CV(t_);
                sfor<j - t + 1>([&](auto u_) {
                    constexpr int u = KX_CV(u_);
                    constexpr int v = j - t - u;
                    if constexpr (t > 0) {
                        R r = X * Rt[hidx(t - 1, u, v)];
                        if constexpr (t > 1) r += R(t - 1) * Rt[hidx(t - 2, u, v)];
                        Rt[hidx(t, u, v)] = r;
                    } else if constexpr (u > 0) {
                        R r = Y * Rt[hidx(t, u - 1, v)];
                        if constexpr (u > 1) r += R(u - 1) * Rt[hidx(t, u - 2, v)];
                        Rt[hidx(t, u, v)] = r;
                    } else {
                        R r = Z * Rt[hidx(t, u, v - 1)];
                        if constexpr (v > 1) r += R(v - 1) * Rt[hidx(t, u, v - 2)];
                        Rt[hidx(t, u, v)] = r;
                    }
                });
            });
        });
        Rt[0] = G[n];
    });
}

// ---------------------------------------------------------------------------
// pair data
// ---------------------------------------------------------------------------

// record stride of a pair class in the FP64 and FP32 tables
template <typename R>
__host__ __device__ constexpr int rec_stride(int la, int lb) {
    return sizeof(R) == 8 ? pair_stride(la, lb) : PAIR32_STRIDE;
}

// E^{ij}_t of one dimension (layout eidx(LA,LB,i,j,t)) by the recursions
//   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}
//   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1},
// unrolled; entries outside t <= i+j are zero.
template <int LA, int LB>
__device__ __forceinline__ void e_build(float* E, float xpa, float xpb, float inv2p) {
    sfor<etab(LA, LB)>([&](auto k_) { E[KX_CV(k_)] = 0.f; });
    E[eidx(LA, LB, 0, 0, 0)] = 1.f;
    sfor<LA + 1>([&](auto i_) {
        constexpr int i = KX_CV(i_);
        if constexpr (i > 0) {
            sfor<i + 1>([&](auto t_) {
                constexpr int t = KX_CV(t_);
                float v = 0.f;
                if constexpr (t <= i - 1) v = xpa * E[eidx(LA, LB, i - 1, 0, t)];
                if constexpr (t > 0) v += inv2p * E[eidx(LA, LB, i - 1, 0, t - 1)];
                if constexpr (t + 1 <= i - 1) v += float(t + 1) * E[eidx(LA, LB, i - 1, 0, t + 1)];
                E[eidx(LA, LB, i, 0, t)] = v;
            });
        }
        sfor<LB>([&](auto jj_) {
            constexpr int j = KX_CV(jj_) + 1;
            sfor<i + j + 1>([&](auto t_) {
                constexpr int t = KX_CV(t_);
                float v = 0.f;
                if constexpr (t <= i + j - 1) v = xpb * E[eidx(LA, LB, i, j - 1, t)];
                if constexpr (t > 0) v += inv2p * E[eidx(LA, LB, i, j - 1, t - 1)];
                if constexpr (t + 1 <= i + j - 1) v += float(t + 1) * E[eidx(LA, LB, i, j - 1, t + 1)];
                E[eidx(LA, LB, i, j, t)] = v;
            });
        });
    });
}

// Loads the bra and ket pairs of a quartet: exponent sums, prefactors,
// P - Q and the per-dimension E tables (E[x*etab + ...]).
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void load_pairs(const R* __restrict__ pb, const R* __restrict__ pk, R* eab, R* ecd, R& p,
                                           R& qq, R& kab, R& kcd, R& X, R& Y, R& Z) {
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    if constexpr (sizeof(R) == 8) {
        sfor<3 * EAB>([&](auto k_) { eab[KX_CV(k_)] = ld_(pb + 5 + KX_CV(k_)); });
        sfor<3 * ECD>([&](auto k_) { ecd[KX_CV(k_)] = ld_(pk + 5 + KX_CV(k_)); });
        p = ld_(pb);
        qq = ld_(pk);
        X = ld_(pb + 1) - ld_(pk + 1);
        Y = ld_(pb + 2) - ld_(pk + 2);
        Z = ld_(pb + 3) - ld_(pk + 3);
        kab = ld_(pb + 4);
        kcd = ld_(pk + 4);
    } else {
        const float4* b4 = reinterpret_cast<const float4*>(pb);
        const float4* k4 = reinterpret_cast<const float4*>(pk);
        float b[16], k[16];
        sfor<4>([&](auto v_) {
            constexpr int v = KX_CV(v_);
            const float4 x = __ldg(b4 + v), y = __ldg(k4 + v);
            b[4 * v] = x.x; b[4 * v + 1] = x.y; b[4 * v + 2] = x.z; b[4 * v + 3] = x.w;
            k[4 * v] = y.x; k[4 * v + 1] = y.y; k[4 * v + 2] = y.z; k[4 * v + 3] = y.w;
        });
        p = b[P32_P];
        qq = k[P32_P];
        kab = b[P32_KAB];
        kcd = k[P32_KAB];
        // (hi_P - hi_Q) is exact when P ~ Q; the lo parts restore the rest
        X = (b[P32_PHI] - k[P32_PHI]) + (b[P32_PLO] - k[P32_PLO]);
        Y = (b[P32_PHI + 1] - k[P32_PHI + 1]) + (b[P32_PLO + 1] - k[P32_PLO + 1]);
        Z = (b[P32_PHI + 2] - k[P32_PHI + 2]) + (b[P32_PLO + 2] - k[P32_PLO + 2]);
        sfor<3>([&](auto x_) {
            constexpr int x = KX_CV(x_);
            e_build<LA, LB>(eab + x * EAB, b[P32_PA + x], b[P32_PB + x], b[P32_INV2P]);
            e_build<LC, LD>(ecd + x * ECD, k[P32_PA + x], k[P32_PB + x], k[P32_INV2P]);
        });
    }
}

// ---------------------------------------------------------------------------
// contraction orders
// ---------------------------------------------------------------------------

// cost of the R-contraction step of each order (multiply-adds)
template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr int mid_cost(bool orderA) {
    int n = 0;
    if (orderA) {
        for (int nu = 0; nu < ncart(LC); ++nu)
            for (int lam = 0; lam < ncart(LB); ++lam) {
                int nh = 0, nh2 = 0;
                for (int t = 0; t <= LA + LB; ++t)
                    for (int u = 0; t + u <= LA + LB; ++u)
                        for (int v = 0; t + u + v <= LA + LB; ++v)
                            nh += reach(t, u, v, cart_x(LB, lam), cart_y(LB, lam), cart_z(LB, lam), LA);
                for (int t = 0; t <= LC + LD; ++t)
                    for (int u = 0; t + u <= LC + LD; ++u)
                        for (int v = 0; t + u + v <= LC + LD; ++v)
                            nh2 += reach(t, u, v, cart_x(LC, nu), cart_y(LC, nu), cart_z(LC, nu), LD);
                n += nh * nh2;
            }
    } else {
        for (int mu = 0; mu < ncart(LA); ++mu)
            for (int sig = 0; sig < ncart(LD); ++sig) {
                int nh = 0, nh2 = 0;
                for (int t = 0; t <= LA + LB; ++t)
                    for (int u = 0; t + u <= LA + LB; ++u)
                        for (int v = 0; t + u + v <= LA + LB; ++v)
                            nh += reach(t, u, v, cart_x(LA, mu), cart_y(LA, mu), cart_z(LA, mu), LB);
                for (int t = 0; t <= LC + LD; ++t)
                    for (int u = 0; t + u <= LC + LD; ++u)
                        for (int v = 0; t + u + v <= LC + LD; ++v)
                            nh2 += reach(t, u, v, cart_x(LD, sig), cart_y(LD, sig), cart_z(LD, sig), LC);
                n += nh * nh2;
            }
    }
    return n;
}

template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr bool use_order_a() {
    return mid_cost<LA, LB, LC, LD>(true) <= mid_cost<LA, LB, LC, LD>(false);
}

// order A: loop nu in c, lam in b
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void contract_a(R* kacc, const R* Rt, const R* eab, const R* ecd,
                                           const R* __restrict__ Pb, int ldp) {
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD;
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    sfor<NC>([&](auto inu_) {
        constexpr int inu = KX_CV(inu_);
        constexpr int nx = cart_x(LC, inu), ny = cart_y(LC, inu), nz = cart_z(LC, inu);
        sfor<NB>([&](auto ilam_) {
            constexpr int ilam = KX_CV(ilam_);
            constexpr int lx = cart_x(LB, ilam), ly = cart_y(LB, ilam), lz = cart_z(LB, ilam);
            const R* prow = Pb + ilam * ldp;
            // T_{h'} = sum_sig E^{cd}_{nu sig,h'} P_{lam sig}
            R Tv[nherm(LCD)];
            sfor<LCD + 1>([&](auto t_) {
                constexpr int t = KX_CV(t_);
                sfor<LCD + 1 - t>([&](auto u_) {
                    constexpr int u = KX_CV(u_);
                    sfor<LCD + 1 - t - u>([&](auto v_) {
                        constexpr int v = KX_CV(v_);
                        if constexpr (reach(t, u, v, nx, ny, nz, LD)) Tv[hidx(t, u, v)] = R(0);
                    });
                });
            });
            sfor<ND>([&](auto isig_) {
                constexpr int isig = KX_CV(isig_);
                constexpr int sx = cart_x(LD, isig), sy = cart_y(LD, isig), sz = cart_z(LD, isig);
                const R pv = ld_(prow + isig);
                sfor<nx + sx + 1>([&](auto t_) {
                    constexpr int t = KX_CV(t_);
                    sfor<ny + sy + 1>([&](auto u_) {
                        constexpr int u = KX_CV(u_);
                        const R exy = ecd[eidx(LC, LD, nx, sx, t)] * ecd[ECD + eidx(LC, LD, ny, sy, u)] * pv;
                        sfor<nz + sz + 1>([&](auto v_) {
                            constexpr int v = KX_CV(v_);
                            Tv[hidx(t, u, v)] += exy * ecd[2 * ECD + eidx(LC, LD, nz, sz, v)];
                        });
                    });
                });
            });
            // U_h = sum_{h'} (-1)^{|h'|} R_{h+h'} T_{h'}
            R Uv[nherm(LAB)];
            sfor<LAB + 1>([&](auto t_) {
                constexpr int t = KX_CV(t_);
                sfor<LAB + 1 - t>([&](auto u_) {
                    constexpr int u = KX_CV(u_);
                    sfor<LAB + 1 - t - u>([&](auto v_) {
                        constexpr int v = KX_CV(v_);
                        if constexpr (reach(t, u, v, lx, ly, lz, LA)) {
                            R s = R(0);
                            sfor<LCD + 1>([&](auto t2_) {
                                constexpr int t2 = KX_CV(t2_);
                                sfor<LCD + 1 - t2>([&](auto u2_) {
                                    constexpr int u2 = KX_CV(u2_);
                                    sfor<LCD + 1 - t2 - u2>([&](auto v2_) {
                                        constexpr int v2 = KX_CV(v2_);
                                        if constexpr (reach(t2, u2, v2, nx, ny, nz, LD)) {
                                            if constexpr ((t2 + u2 + v2) & 1)
                                                s -= Rt[hidx(t + t2, u + u2, v + v2)] * Tv[hidx(t2, u2, v2)];
                                            else
                                                s += Rt[hidx(t + t2, u + u2, v + v2)] * Tv[hidx(t2, u2, v2)];
                                        }
                                    });
                                });
                            });
                            Uv[hidx(t, u, v)] = s;
                        }
                    });
                });
            });
            // K_{mu nu} += sum_h E^{ab}_{mu lam,h} U_h
            sfor<NA>([&](auto imu_) {
                constexpr int imu = KX_CV(imu_);
                constexpr int mx = cart_x(LA, imu), my = cart_y(LA, imu), mz = cart_z(LA, imu);
                R s = R(0);
                sfor<mx + lx + 1>([&](auto t_) {
                    constexpr int t = KX_CV(t_);
                    sfor<my + ly + 1>([&](auto u_) {
                        constexpr int u = KX_CV(u_);
                        const R exy = eab[eidx(LA, LB, mx, lx, t)] * eab[EAB + eidx(LA, LB, my, ly, u)];
                        R sz_ = R(0);
                        sfor<mz + lz + 1>([&](auto v_) {
                            constexpr int v = KX_CV(v_);
                            sz_ += eab[2 * EAB + eidx(LA, LB, mz, lz, v)] * Uv[hidx(t, u, v)];
                        });
                        s += exy * sz_;
                    });
                });
                kacc[imu * NC + inu] += s;
            });
        });
    });
}

// order B: loop mu in a, sig in d
template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void contract_b(R* kacc, const R* Rt, const R* eab, const R* ecd,
                                           const R* __restrict__ Pb, int ldp) {
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD;
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    sfor<NA>([&](auto imu_) {
        constexpr int imu = KX_CV(imu_);
        constexpr int mx = cart_x(LA, imu), my = cart_y(LA, imu), mz = cart_z(LA, imu);
        sfor<ND>([&](auto isig_) {
            constexpr int isig = KX_CV(isig_);
            constexpr int sx = cart_x(LD, isig), sy = cart_y(LD, isig), sz = cart_z(LD, isig);
            // W_h = sum_lam E^{ab}_{mu lam,h} P_{lam sig}
            R Wv[nherm(LAB)];
            sfor<LAB + 1>([&](auto t_) {
                constexpr int t = KX_CV(t_);
                sfor<LAB + 1 - t>([&](auto u_) {
                    constexpr int u = KX_CV(u_);
                    sfor<LAB + 1 - t - u>([&](auto v_) {
                        constexpr int v = KX_CV(v_);
                        if constexpr (reach(t, u, v, mx, my, mz, LB)) Wv[hidx(t, u, v)] = R(0);
                    });
                });
            });
            sfor<NB>([&](auto ilam_) {
                constexpr int ilam = KX_CV(ilam_);
                constexpr int lx = cart_x(LB, ilam), ly = cart_y(LB, ilam), lz = cart_z(LB, ilam);
                const R pv = ld_(Pb + ilam * ldp + isig);
                sfor<mx + lx + 1>([&](auto t_) {
                    constexpr int t = KX_CV(t_);
                    sfor<my + ly + 1>([&](auto u_) {
                        constexpr int u = KX_CV(u_);
                        const R exy = eab[eidx(LA, LB, mx, lx, t)] * eab[EAB + eidx(LA, LB, my, ly, u)] * pv;
                        sfor<mz + lz + 1>([&](auto v_) {
                            constexpr int v = KX_CV(v_);
                            Wv[hidx(t, u, v)] += exy * eab[2 * EAB + eidx(LA, LB, mz, lz, v)];
                        });
                    });
                });
            });
            // V_{h'} = sum_h R_{h+h'} W_h
            R Vv[nherm(LCD)];
            sfor<LCD + 1>([&](auto t2_) {
                constexpr int t2 = KX_CV(t2_);
                sfor<LCD + 1 - t2>([&](auto u2_) {
                    constexpr int u2 = KX_CV(u2_);
                    sfor<LCD + 1 - t2 - u2>([&](auto v2_) {
                        constexpr int v2 = KX_CV(v2_);
                        if constexpr (reach(t2, u2, v2, sx, sy, sz, LC)) {
                            R s = R(0);
                            sfor<LAB + 1>([&](auto t_) {
                                constexpr int t = KX_CV(t_);
                                sfor<LAB + 1 - t>([&](auto u_) {
                                    constexpr int u = KX_CV(u_);
                                    sfor<LAB + 1 - t - u>([&](auto v_) {
                                        constexpr int v = KX_CV(v_);
                                        if constexpr (reach(t, u, v, mx, my, mz, LB))
                                            s += Rt[hidx(t + t2, u + u2, v + v2)] * Wv[hidx(t, u, v)];
                                    });
                                });
                            });
                            Vv[hidx(t2, u2, v2)] = s;
                        }
                    });
                });
            });
            // K_{mu nu} += sum_{h'} (-1)^{|h'|} E^{cd}_{nu sig,h'} V_{h'}
            sfor<NC>([&](auto inu_) {
                constexpr int inu = KX_CV(inu_);
                constexpr int nx = cart_x(LC, inu), ny = cart_y(LC, inu), nz = cart_z(LC, inu);
                R s = R(0);
                sfor<nx + sx + 1>([&](auto t_) {
                    constexpr int t = KX_CV(t_);
                    sfor<ny + sy + 1>([&](auto u_) {
                        constexpr int u = KX_CV(u_);
                        const R exy = ecd[eidx(LC, LD, nx, sx, t)] * ecd[ECD + eidx(LC, LD, ny, sy, u)];
                        R sz_ = R(0);
                        sfor<nz + sz + 1>([&](auto v_) {
                            constexpr int v = KX_CV(v_);
                            if constexpr ((t + u + v) & 1)
                                sz_ -= ecd[2 * ECD + eidx(LC, LD, nz, sz, v)] * Vv[hidx(t, u, v)];
                            else
                                sz_ += ecd[2 * ECD + eidx(LC, LD, nz, sz, v)] * Vv[hidx(t, u, v)];
                        });
                        s += exy * sz_;
                    });
                });
                kacc[imu * NC + inu] += s;
            });
        });
    });
}

// ---------------------------------------------------------------------------
// warp-level K reduction
// ---------------------------------------------------------------------------

// Sums the per-thread K partials over each run of lanes with the same
// (fa, fc) and lets the last lane of the run add the sums into K (FP64) at
// Kb, the address of K(fa, fc) (row stride ldk).
template <int NA, int NC, typename R>
__device__ __forceinline__ void flush_k(R* kacc, int fa, int fc, double* __restrict__ Kb, int ldk) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long key = fa < 0 ? -1ll : (((long long)fa << 32) | (unsigned)fc);
    const long long prev = __shfl_up_sync(full, key, 1);
    const bool head = (lane == 0) || (prev != key);
    const unsigned heads = __ballot_sync(full, head);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    const bool tail = (lane == 31) || ((heads >> (lane + 1)) & 1u);
    sfor<NA * NC>([&](auto e_) {
        constexpr int e = KX_CV(e_);
        R v = kacc[e];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            R o = shfl_up(full, v, d);
            if (lane - d >= start) v += o;
        }
        if (tail && key >= 0) atomicAdd(Kb + (e / NC) * ldk + e % NC, to_f64(v));
    });
}

// ---------------------------------------------------------------------------
// the class kernel
// ---------------------------------------------------------------------------

template <int LA, int LB, int LC, int LD, typename R>
__global__ void __launch_bounds__(ERI_MAX_THREADS) k_eri(EriArgs args) {
    constexpr int NA = ncart(LA), NC = ncart(LC);
    constexpr int L = LA + LB + LC + LD;
    constexpr int SAB = rec_stride<R>(LA, LB), SCD = rec_stride<R>(LC, LD);
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    const R* __restrict__ bra = (const R*)args.bra;
    const R* __restrict__ ket = (const R*)args.ket;
    const R* __restrict__ boys = (const R*)args.boys;
    const R* __restrict__ P = (const R*)args.P;
    const int64_t i0 = args.range ? args.range[0] : args.i0, i1 = args.range ? args.range[1] : args.i1;
    // block-uniform trip count: every warp takes part in every flush
    for (int64_t base = i0 + blockIdx.x * (int64_t)blockDim.x; base < i1; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        R kacc[NA * NC];
        sfor<NA * NC>([&](auto e_) { kacc[KX_CV(e_)] = R(0); });
        int fa = -1, fc = -1, ldk = 0;
        double* Kb = args.K;
        const Quartet q = i < i1 ? args.rec[i] : Quartet{-1, -1};
        // slots outside the pair tables (never produced by the expansion) are skipped
        if (q.ab >= 0 && q.ab < args.nab && q.cd >= 0 && q.cd < args.ncd) {
            const R* pb = bra + (int64_t)q.ab * SAB;
            const R* pk = ket + (int64_t)q.cd * SCD;
            const PairMeta mb = args.bmeta[q.ab], mk = args.kmeta[q.cd];
            fa = mb.fa;
            fc = mk.fa;
            ldk = mb.ldk;
            Kb = args.K + mb.krow_a + fc;
            R eab[3 * EAB], ecd[3 * ECD];
            R p, qq, kab, kcd, X, Y, Z;
            load_pairs<LA, LB, LC, LD, R>(pb, pk, eab, ecd, p, qq, kab, kcd, X, Y, Z);
            const R pq = p * qq, sum = p + qq;
            const R rho = pq / sum;
            const R r2 = X * X + Y * Y + Z * Z;
            const R T = rho * r2;
            const R pref = R(2.0 * 17.493418327624862) * kab * kcd / (pq * Real<R>::sqrt_(sum));
            R G[L + 1];
            boys_scaled<L, R>(G, T, rho, r2, pref, boys);
            R Rt[nherm(L)];
            hermite_r<L, R>(Rt, G, X, Y, Z);
            const R* Pb = P + mb.prow_b + mk.fb;
            if constexpr (use_order_a<LA, LB, LC, LD>())
                contract_a<LA, LB, LC, LD, R>(kacc, Rt, eab, ecd, Pb, mb.ldp);
            else
                contract_b<LA, LB, LC, LD, R>(kacc, Rt, eab, ecd, Pb, mb.ldp);
        }
        flush_k<NA, NC, R>(kacc, fa, fc, Kb, ldk);
    }
}

// ---------------------------------------------------------------------------
// rolled variant for the largest classes (L = la+lb+lc+ld >= ROLL_L)
// ---------------------------------------------------------------------------
//
// The same arithmetic as k_eri, with the Cartesian and Hermite loops kept as
// run-time loops and the intermediates in thread-local arrays.  Full
// unrolling of these classes yields tens of thousands of straight-line
// operations per thread, far past the register file; on GB300 the FP64
// kernels are bound by the FP64 pipe, so the loop overhead is hidden there.

constexpr int ROLL_L = 7;

template <int L, typename R>
__device__ __forceinline__ void hermite_r_rolled(R* Rt, const R* G, R X, R Y, R Z) {
    Rt[0] = G[L];
#pragma unroll 1
    for (int n = L - 1; n >= 0; --n) {
#pragma unroll 1
        for (int j = L - n; j >= 1; --j)
#pragma unroll 1
            for (int t = j; t >= 0; --t)
#pragma unroll 1
                for (int u = j - t; u >= 0; --u) {
                    const int v = j - t - u;
                    R r;
                    if (t > 0) {
                        r = X * Rt[hidx(t - 1, u, v)];
                        if (t > 1) r += R(t - 1) * Rt[hidx(t - 2, u, v)];
                    } else if (u > 0) {
                        r = Y * Rt[hidx(t, u - 1, v)];
                        if (u > 1) r += R(u - 1) * Rt[hidx(t, u - 2, v)];
                    } else {
                        r = Z * Rt[hidx(t, u, v - 1)];
                        if (v > 1) r += R(v - 1) * Rt[hidx(t, u, v - 2)];
                    }
                    Rt[hidx(t, u, v)] = r;
                }
        Rt[0] = G[n];
    }
}

template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void contract_a_rolled(R* kacc, const R* Rt, const R* eab, const R* ecd,
                                                  const R* __restrict__ Pb, int ldp) {
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD;
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
#pragma unroll 1
    for (int inu = 0; inu < NC; ++inu) {
        const int nx = cart_x(LC, inu), ny = cart_y(LC, inu), nz = cart_z(LC, inu);
#pragma unroll 1
        for (int ilam = 0; ilam < NB; ++ilam) {
            const int lx = cart_x(LB, ilam), ly = cart_y(LB, ilam), lz = cart_z(LB, ilam);
            const R* prow = Pb + ilam * ldp;
            R Tv[nherm(LCD)];
#pragma unroll 1
            for (int k = 0; k < nherm(LCD); ++k) Tv[k] = R(0);
#pragma unroll 1
            for (int isig = 0; isig < ND; ++isig) {
                const int sx = cart_x(LD, isig), sy = cart_y(LD, isig), sz = cart_z(LD, isig);
                const R pv = ld_(prow + isig);
#pragma unroll 1
                for (int t = 0; t <= nx + sx; ++t)
#pragma unroll 1
                    for (int u = 0; u <= ny + sy; ++u) {
                        const R exy = ecd[eidx(LC, LD, nx, sx, t)] * ecd[ECD + eidx(LC, LD, ny, sy, u)] * pv;
#pragma unroll 1
                        for (int v = 0; v <= nz + sz; ++v)
                            Tv[hidx(t, u, v)] += exy * ecd[2 * ECD + eidx(LC, LD, nz, sz, v)];
                    }
            }
            R Uv[nherm(LAB)];
#pragma unroll 1
            for (int t = 0; t <= LAB; ++t)
#pragma unroll 1
                for (int u = 0; t + u <= LAB; ++u)
#pragma unroll 1
                    for (int v = 0; t + u + v <= LAB; ++v) {
                        if (!reach(t, u, v, lx, ly, lz, LA)) continue;
                        R s = R(0);
#pragma unroll 1
                        for (int t2 = 0; t2 <= LCD; ++t2)
#pragma unroll 1
                            for (int u2 = 0; t2 + u2 <= LCD; ++u2)
#pragma unroll 1
                                for (int v2 = 0; t2 + u2 + v2 <= LCD; ++v2) {
                                    if (!reach(t2, u2, v2, nx, ny, nz, LD)) continue;
                                    const R term = Rt[hidx(t + t2, u + u2, v + v2)] * Tv[hidx(t2, u2, v2)];
                                    s = ((t2 + u2 + v2) & 1) ? s - term : s + term;
                                }
                        Uv[hidx(t, u, v)] = s;
                    }
#pragma unroll 1
            for (int imu = 0; imu < NA; ++imu) {
                const int mx = cart_x(LA, imu), my = cart_y(LA, imu), mz = cart_z(LA, imu);
                R s = R(0);
#pragma unroll 1
                for (int t = 0; t <= mx + lx; ++t)
#pragma unroll 1
                    for (int u = 0; u <= my + ly; ++u) {
                        const R exy = eab[eidx(LA, LB, mx, lx, t)] * eab[EAB + eidx(LA, LB, my, ly, u)];
                        R sz_ = R(0);
#pragma unroll 1
                        for (int v = 0; v <= mz + lz; ++v)
                            sz_ += eab[2 * EAB + eidx(LA, LB, mz, lz, v)] * Uv[hidx(t, u, v)];
                        s += exy * sz_;
                    }
                kacc[imu * NC + inu] += s;
            }
        }
    }
}

template <int LA, int LB, int LC, int LD, typename R>
__device__ __forceinline__ void contract_b_rolled(R* kacc, const R* Rt, const R* eab, const R* ecd,
                                                  const R* __restrict__ Pb, int ldp) {
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD;
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
#pragma unroll 1
    for (int imu = 0; imu < NA; ++imu) {
        const int mx = cart_x(LA, imu), my = cart_y(LA, imu), mz = cart_z(LA, imu);
#pragma unroll 1
        for (int isig = 0; isig < ND; ++isig) {
            const int sx = cart_x(LD, isig), sy = cart_y(LD, isig), sz = cart_z(LD, isig);
            R Wv[nherm(LAB)];
#pragma unroll 1
            for (int k = 0; k < nherm(LAB); ++k) Wv[k] = R(0);
#pragma unroll 1
            for (int ilam = 0; ilam < NB; ++ilam) {
                const int lx = cart_x(LB, ilam), ly = cart_y(LB, ilam), lz = cart_z(LB, ilam);
                const R pv = ld_(Pb + ilam * ldp + isig);
#pragma unroll 1
                for (int t = 0; t <= mx + lx; ++t)
#pragma unroll 1
                    for (int u = 0; u <= my + ly; ++u) {
                        const R exy = eab[eidx(LA, LB, mx, lx, t)] * eab[EAB + eidx(LA, LB, my, ly, u)] * pv;
#pragma unroll 1
                        for (int v = 0; v <= mz + lz; ++v)
                            Wv[hidx(t, u, v)] += exy * eab[2 * EAB + eidx(LA, LB, mz, lz, v)];
                    }
            }
            R Vv[nherm(LCD)];
#pragma unroll 1
            for (int t2 = 0; t2 <= LCD; ++t2)
#pragma unroll 1
                for (int u2 = 0; t2 + u2 <= LCD; ++u2)
#pragma unroll 1
                    for (int v2 = 0; t2 + u2 + v2 <= LCD; ++v2) {
                        if (!reach(t2, u2, v2, sx, sy, sz, LC)) continue;
                        R s = R(0);
#pragma unroll 1
                        for (int t = 0; t <= LAB; ++t)
#pragma unroll 1
                            for (int u = 0; t + u <= LAB; ++u)
#pragma unroll 1
                                for (int v = 0; t + u + v <= LAB; ++v)
                                    if (reach(t, u, v, mx, my, mz, LB))
                                        s += Rt[hidx(t + t2, u + u2, v + v2)] * Wv[hidx(t, u, v)];
                        Vv[hidx(t2, u2, v2)] = s;
                    }
#pragma unroll 1
            for (int inu = 0; inu < NC; ++inu) {
                const int nx = cart_x(LC, inu), ny = cart_y(LC, inu), nz = cart_z(LC, inu);
                R s = R(0);
#pragma unroll 1
                for (int t = 0; t <= nx + sx; ++t)
#pragma unroll 1
                    for (int u = 0; u <= ny + sy; ++u) {
                        const R exy = ecd[eidx(LC, LD, nx, sx, t)] * ecd[ECD + eidx(LC, LD, ny, sy, u)];
                        R sz_ = R(0);
#pragma unroll 1
                        for (int v = 0; v <= nz + sz; ++v) {
                            const R term = ecd[2 * ECD + eidx(LC, LD, nz, sz, v)] * Vv[hidx(t, u, v)];
                            sz_ = ((t + u + v) & 1) ? sz_ - term : sz_ + term;
                        }
                        s += exy * sz_;
                    }
                kacc[imu * NC + inu] += s;
            }
        }
    }
}

template <int LA, int LB, int LC, int LD, typename R>
__global__ void __launch_bounds__(ERI_MAX_THREADS) k_eri_rolled(EriArgs args) {
    constexpr int NA = ncart(LA), NC = ncart(LC);
    constexpr int L = LA + LB + LC + LD;
    constexpr int SAB = rec_stride<R>(LA, LB), SCD = rec_stride<R>(LC, LD);
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    const R* __restrict__ bra = (const R*)args.bra;
    const R* __restrict__ ket = (const R*)args.ket;
    const R* __restrict__ boys = (const R*)args.boys;
    const R* __restrict__ P = (const R*)args.P;
    const int64_t i0 = args.range ? args.range[0] : args.i0, i1 = args.range ? args.range[1] : args.i1;
    for (int64_t base = i0 + blockIdx.x * (int64_t)blockDim.x; base < i1; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        R kacc[NA * NC];
#pragma unroll
        for (int e = 0; e < NA * NC; ++e) kacc[e] = R(0);
        int fa = -1, fc = -1, ldk = 0;
        double* Kb = args.K;
        const Quartet q = i < i1 ? args.rec[i] : Quartet{-1, -1};
        // slots outside the pair tables (never produced by the expansion) are skipped
        if (q.ab >= 0 && q.ab < args.nab && q.cd >= 0 && q.cd < args.ncd) {
            const R* pb = bra + (int64_t)q.ab * SAB;
            const R* pk = ket + (int64_t)q.cd * SCD;
            const PairMeta mb = args.bmeta[q.ab], mk = args.kmeta[q.cd];
            fa = mb.fa;
            fc = mk.fa;
            ldk = mb.ldk;
            Kb = args.K + mb.krow_a + fc;
            R eab[3 * EAB], ecd[3 * ECD];
            R p, qq, kab, kcd, X, Y, Z;
            load_pairs<LA, LB, LC, LD, R>(pb, pk, eab, ecd, p, qq, kab, kcd, X, Y, Z);
            const R pq = p * qq, sum = p + qq;
            const R rho = pq / sum;
            const R r2 = X * X + Y * Y + Z * Z;
            const R T = rho * r2;
            const R pref = R(2.0 * 17.493418327624862) * kab * kcd / (pq * Real<R>::sqrt_(sum));
            R G[L + 1];
            boys_scaled<L, R>(G, T, rho, r2, pref, boys);
            R Rt[nherm(L)];
            hermite_r_rolled<L, R>(Rt, G, X, Y, Z);
            const R* Pb = P + mb.prow_b + mk.fb;
            if constexpr (use_order_a<LA, LB, LC, LD>())
                contract_a_rolled<LA, LB, LC, LD, R>(kacc, Rt, eab, ecd, Pb, mb.ldp);
            else
                contract_b_rolled<LA, LB, LC, LD, R>(kacc, Rt, eab, ecd, Pb, mb.ldp);
        }
        flush_k<NA, NC, R>(kacc, fa, fc, Kb, ldk);
    }
}

// ---------------------------------------------------------------------------
// FP32 kernel for the largest classes (L >= ROLL_L): full Hermite sets with
// compile-time indices, Cartesian loops at run time, R and E in shared memory
// ---------------------------------------------------------------------------
//
// The rolled kernel keeps T, U and R in thread-local arrays indexed at run
// time (local memory).  Here, per (nu, lam) of order A, T_{h'} and U_h run
// over the FULL Hermite sets of the ket and bra (no reach pruning), so every
// index is a compile-time constant and T, U live in registers; R_{h+h'} is
// read from the thread's slice of shared memory once per sum index
// s = h + h' and used for every (h, h') pair with that sum.  The E tables
// are in shared memory as well; the slices a given nu or lam needs are
// loaded into registers first.  The extra multiply-adds on zero E entries
// and unreachable Hermite indices cost less than the local-memory traffic
// they replace.  Shared memory: per thread nherm(L) + 3 etab(la,lb) +
// 3 etab(lc,ld) floats, interleaved across the block (entry j of thread t at
// j * blockDim + t) so that a warp's accesses fall in distinct banks.

template <int LA, int LB, int LC, int LD>
__host__ __device__ constexpr int big_slice() {
    return nherm(LA + LB + LC + LD) + 3 * etab(LA, LB) + 3 * etab(LC, LD);
}

template <int L>
__device__ __forceinline__ void hermite_r_shared(float* Rs, int st, const float* G, float X, float Y, float Z) {
    Rs[0] = G[L];
#pragma unroll 1
    for (int n = L - 1; n >= 0; --n) {
#pragma unroll 1
        for (int j = L - n; j >= 1; --j)
#pragma unroll 1
            for (int t = j; t >= 0; --t)
#pragma unroll 1
                for (int u = j - t; u >= 0; --u) {
                    const int v = j - t - u;
                    float r;
                    if (t > 0) {
                        r = X * Rs[hidx(t - 1, u, v) * st];
                        if (t > 1) r += float(t - 1) * Rs[hidx(t - 2, u, v) * st];
                    } else if (u > 0) {
                        r = Y * Rs[hidx(t, u - 1, v) * st];
                        if (u > 1) r += float(u - 1) * Rs[hidx(t, u - 2, v) * st];
                    } else {
                        r = Z * Rs[hidx(t, u, v - 1) * st];
                        if (v > 1) r += float(v - 1) * Rs[hidx(t, u, v - 2) * st];
                    }
                    Rs[hidx(t, u, v) * st] = r;
                }
        Rs[0] = G[n];
    }
}

template <int L>
__device__ __forceinline__ void hermite_r_shared64(double* Rs, int st, const double* G, double X, double Y,
                                                   double Z) {
    Rs[0] = G[L];
#pragma unroll 1
    for (int n = L - 1; n >= 0; --n) {
#pragma unroll 1
        for (int j = L - n; j >= 1; --j)
#pragma unroll 1
            for (int t = j; t >= 0; --t)
#pragma unroll 1
                for (int u = j - t; u >= 0; --u) {
                    const int v = j - t - u;
                    double r;
                    if (t > 0) {
                        r = X * Rs[hidx(t - 1, u, v) * st];
                        if (t > 1) r += double(t - 1) * Rs[hidx(t - 2, u, v) * st];
                    } else if (u > 0) {
                        r = Y * Rs[hidx(t, u - 1, v) * st];
                        if (u > 1) r += double(u - 1) * Rs[hidx(t, u - 2, v) * st];
                    } else {
                        r = Z * Rs[hidx(t, u, v - 1) * st];
                        if (v > 1) r += double(v - 1) * Rs[hidx(t, u, v - 2) * st];
                    }
                    Rs[hidx(t, u, v) * st] = r;
                }
        Rs[0] = G[n];
    }
}

template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(128) k_eri_big(EriArgs args) {
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
    constexpr int HAB = nherm(LAB), HCD = nherm(LCD), HL = nherm(L);
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    constexpr int SAB = PAIR32_STRIDE, SCD = PAIR32_STRIDE;
    extern __shared__ float big_sh[];
    const int st = blockDim.x;
    float* const Rs = big_sh + threadIdx.x;                 // R:  [HL]
    float* const Es_ab = Rs + HL * st;                     // E^ab: [3 * EAB]
    float* const Es_cd = Es_ab + 3 * EAB * st;             // E^cd: [3 * ECD]
    const float* __restrict__ bra = (const float*)args.bra;
    const float* __restrict__ ket = (const float*)args.ket;
    const float* __restrict__ boys = (const float*)args.boys;
    const float* __restrict__ P = (const float*)args.P;
    const int64_t i0 = args.range ? args.range[0] : args.i0, i1 = args.range ? args.range[1] : args.i1;
    for (int64_t base = i0 + blockIdx.x * (int64_t)blockDim.x; base < i1; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const Quartet q = i < i1 ? args.rec[i] : Quartet{-1, -1};
        const bool valid = q.ab >= 0 && q.ab < args.nab && q.cd >= 0 && q.cd < args.ncd;
        int fa = -1, fc = -1, ldk = 0, ldp = 0;
        double* Kb = args.K;
        const float* Pb = P;
        if (valid) {
            const float* pb = bra + (int64_t)q.ab * SAB;
            const float* pk = ket + (int64_t)q.cd * SCD;
            const PairMeta mb = args.bmeta[q.ab], mk = args.kmeta[q.cd];
            fa = mb.fa;
            fc = mk.fa;
            ldk = mb.ldk;
            ldp = mb.ldp;
            Kb = args.K + mb.krow_a + fc;
            Pb = P + mb.prow_b + mk.fb;
            // pair data, E tables into shared memory
            const float4* b4 = reinterpret_cast<const float4*>(pb);
            const float4* k4 = reinterpret_cast<const float4*>(pk);
            float b[16], k[16];
            sfor<4>([&](auto v_) {
                constexpr int v = KX_CV(v_);
                const float4 x = __ldg(b4 + v), y = __ldg(k4 + v);
                b[4 * v] = x.x; b[4 * v + 1] = x.y; b[4 * v + 2] = x.z; b[4 * v + 3] = x.w;
                k[4 * v] = y.x; k[4 * v + 1] = y.y; k[4 * v + 2] = y.z; k[4 * v + 3] = y.w;
            });
            const float X = (b[P32_PHI] - k[P32_PHI]) + (b[P32_PLO] - k[P32_PLO]);
            const float Y = (b[P32_PHI + 1] - k[P32_PHI + 1]) + (b[P32_PLO + 1] - k[P32_PLO + 1]);
            const float Z = (b[P32_PHI + 2] - k[P32_PHI + 2]) + (b[P32_PLO + 2] - k[P32_PLO + 2]);
            sfor<3>([&](auto x_) {
                constexpr int x = KX_CV(x_);
                float e1[EAB];
                e_build<LA, LB>(e1, b[P32_PA + x], b[P32_PB + x], b[P32_INV2P]);
                sfor<EAB>([&](auto j_) { Es_ab[(x * EAB + KX_CV(j_)) * st] = e1[KX_CV(j_)]; });
                float e2[ECD];
                e_build<LC, LD>(e2, k[P32_PA + x], k[P32_PB + x], k[P32_INV2P]);
                sfor<ECD>([&](auto j_) { Es_cd[(x * ECD + KX_CV(j_)) * st] = e2[KX_CV(j_)]; });
            });
            const float p = b[P32_P], qq = k[P32_P];
            const float pq = p * qq, sum = p + qq;
            const float rho = pq / sum;
            const float r2 = X * X + Y * Y + Z * Z;
            const float pref = float(2.0 * 17.493418327624862) * b[P32_KAB] * k[P32_KAB] / (pq * sqrtf(sum));
            float G[L + 1];
            boys_scaled<L, float>(G, rho * r2, rho, r2, pref, boys);
            hermite_r_shared<L>(Rs, st, G, X, Y, Z);
        }
#pragma unroll 1
        for (int inu = 0; inu < NC; ++inu) {
            float kacc[NA];
            sfor<NA>([&](auto e_) { kacc[KX_CV(e_)] = 0.f; });
            if (valid) {
                const int nx = cart_x(LC, inu), ny = cart_y(LC, inu), nz = cart_z(LC, inu);
                // E^cd_{nu sig, h'} factors of this nu: per dimension
                // E[n][s][t'] for s = 0..LD, t' = 0..LCD
                float exd[LD + 1][LCD + 1], eyd[LD + 1][LCD + 1], ezd[LD + 1][LCD + 1];
                sfor<LD + 1>([&](auto s_) {
                    constexpr int s = KX_CV(s_);
                    sfor<LCD + 1>([&](auto t_) {
                        constexpr int t = KX_CV(t_);
                        exd[s][t] = Es_cd[(0 * ECD + eidx(LC, LD, 0, s, t) + nx * (LD + 1) * (LCD + 1)) * st];
                        eyd[s][t] = Es_cd[(1 * ECD + eidx(LC, LD, 0, s, t) + ny * (LD + 1) * (LCD + 1)) * st];
                        ezd[s][t] = Es_cd[(2 * ECD + eidx(LC, LD, 0, s, t) + nz * (LD + 1) * (LCD + 1)) * st];
                    });
                });
#pragma unroll 1
                for (int ilam = 0; ilam < NB; ++ilam) {
                    const int lx = cart_x(LB, ilam), ly = cart_y(LB, ilam), lz = cart_z(LB, ilam);
                    // T_{h'} = sum_sig E^cd_{nu sig,h'} P_{lam sig}
                    float pv[ND];
                    sfor<ND>([&](auto g_) { pv[KX_CV(g_)] = __ldg(Pb + ilam * ldp + KX_CV(g_)); });
                    float T[HCD];
                    sfor<HCD>([&](auto h_) { T[KX_CV(h_)] = 0.f; });
                    sfor<ND>([&](auto g_) {
                        constexpr int g = KX_CV(g_);
                        constexpr int sx = cart_x(LD, g), sy = cart_y(LD, g), sz = cart_z(LD, g);
                        sfor<LCD + 1>([&](auto t_) {
                            constexpr int t = KX_CV(t_);
                            const float a1 = pv[g] * exd[sx][t];
                            sfor<LCD + 1 - t>([&](auto u_) {
                                constexpr int u = KX_CV(u_);
                                const float a2 = a1 * eyd[sy][u];
                                sfor<LCD + 1 - t - u>([&](auto v_) {
                                    constexpr int v = KX_CV(v_);
                                    T[hidx(t, u, v)] += a2 * ezd[sz][v];
                                });
                            });
                        });
                    });
                    // U_h = sum_{h'} (-1)^{|h'|} R_{h+h'} T_{h'}, R read once per s = h + h'
                    float U[HAB];
                    sfor<HAB>([&](auto h_) { U[KX_CV(h_)] = 0.f; });
                    sfor<L + 1>([&](auto ts_) {
                        constexpr int ts = KX_CV(ts_);
                        sfor<L + 1 - ts>([&](auto us_) {
                            constexpr int us = KX_CV(us_);
                            sfor<L + 1 - ts - us>([&](auto vs_) {
                                constexpr int vs = KX_CV(vs_);
                                const float r = Rs[hidx(ts, us, vs) * st];
                                sfor<(ts < LAB ? ts : LAB) + 1>([&](auto t_) {
                                    constexpr int t = KX_CV(t_);
                                    sfor<(us < LAB - t ? us : LAB - t) + 1>([&](auto u_) {
                                        constexpr int u = KX_CV(u_);
                                        sfor<(vs < LAB - t - u ? vs : LAB - t - u) + 1>([&](auto v_) {
                                            constexpr int v = KX_CV(v_);
                                            constexpr int t2 = ts - t, u2 = us - u, v2 = vs - v;
                                            if constexpr (t2 + u2 + v2 <= LCD) {
                                                if constexpr ((t2 + u2 + v2) & 1)
                                                    U[hidx(t, u, v)] -= r * T[hidx(t2, u2, v2)];
                                                else
                                                    U[hidx(t, u, v)] += r * T[hidx(t2, u2, v2)];
                                            }
                                        });
                                    });
                                });
                            });
                        });
                    });
                    // K_{mu nu} += sum_h E^ab_{mu lam,h} U_h, E^ab factors of this lam
                    float exa[LA + 1][LAB + 1], eya[LA + 1][LAB + 1], eza[LA + 1][LAB + 1];
                    sfor<LA + 1>([&](auto m_) {
                        constexpr int m = KX_CV(m_);
                        sfor<LAB + 1>([&](auto t_) {
                            constexpr int t = KX_CV(t_);
                            exa[m][t] = Es_ab[(0 * EAB + eidx(LA, LB, m, 0, t) + lx * (LAB + 1)) * st];
                            eya[m][t] = Es_ab[(1 * EAB + eidx(LA, LB, m, 0, t) + ly * (LAB + 1)) * st];
                            eza[m][t] = Es_ab[(2 * EAB + eidx(LA, LB, m, 0, t) + lz * (LAB + 1)) * st];
                        });
                    });
                    sfor<NA>([&](auto mu_) {
                        constexpr int mu = KX_CV(mu_);
                        constexpr int mx = cart_x(LA, mu), my = cart_y(LA, mu), mz = cart_z(LA, mu);
                        float sacc = 0.f;
                        sfor<LAB + 1>([&](auto t_) {
                            constexpr int t = KX_CV(t_);
                            sfor<LAB + 1 - t>([&](auto u_) {
                                constexpr int u = KX_CV(u_);
                                const float exy = exa[mx][t] * eya[my][u];
                                float sz_ = 0.f;
                                sfor<LAB + 1 - t - u>([&](auto v_) {
                                    constexpr int v = KX_CV(v_);
                                    sz_ += eza[mz][v] * U[hidx(t, u, v)];
                                });
                                sacc += exy * sz_;
                            });
                        });
                        kacc[mu] += sacc;
                    });
                }
            }
            // column nu of the K block: warp-segmented sums over equal (fa, fc)
            flush_k<NA, 1, float>(kacc, fa, fc, Kb + inu, ldk);
        }
    }
}

// FP64 variant for the largest classes: the same full-set (nu, lam) loop with
// T and U in registers and R in the thread's slice of shared memory
// (nherm(L) doubles, interleaved across the block); the E slices of each nu
// and lam are read from the FP64 pair record itself (L1-resident while the
// quartet is evaluated).  An alternative to the rolled kernel that the
// autotuner may pick per class.
template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(128) k_eri_big64(EriArgs args) {
    using R = double;
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
    constexpr int HAB = nherm(LAB), HCD = nherm(LCD);
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    constexpr int SAB = pair_stride(LA, LB), SCD = pair_stride(LC, LD);
    extern __shared__ double big_sh64[];
    const int st = blockDim.x;
    double* const Rs = big_sh64 + threadIdx.x;
    const R* __restrict__ bra = (const R*)args.bra;
    const R* __restrict__ ket = (const R*)args.ket;
    const R* __restrict__ boys = (const R*)args.boys;
    const R* __restrict__ P = (const R*)args.P;
    const int64_t i0 = args.range ? args.range[0] : args.i0, i1 = args.range ? args.range[1] : args.i1;
    for (int64_t base = i0 + blockIdx.x * (int64_t)blockDim.x; base < i1; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const Quartet q = i < i1 ? args.rec[i] : Quartet{-1, -1};
        const bool valid = q.ab >= 0 && q.ab < args.nab && q.cd >= 0 && q.cd < args.ncd;
        int fa = -1, fc = -1, ldk = 0, ldp = 0;
        double* Kb = args.K;
        const R* Pb = P;
        const R* Eab = bra;   // E tables of the two pair records (x, y, z blocks)
        const R* Ecd = ket;
        if (valid) {
            const R* pb = bra + (int64_t)q.ab * SAB;
            const R* pk = ket + (int64_t)q.cd * SCD;
            const PairMeta mb = args.bmeta[q.ab], mk = args.kmeta[q.cd];
            fa = mb.fa;
            fc = mk.fa;
            ldk = mb.ldk;
            ldp = mb.ldp;
            Kb = args.K + mb.krow_a + fc;
            Pb = P + mb.prow_b + mk.fb;
            Eab = pb + 5;
            Ecd = pk + 5;
            const R p = __ldg(pb), qq = __ldg(pk);
            const R X = __ldg(pb + 1) - __ldg(pk + 1), Y = __ldg(pb + 2) - __ldg(pk + 2),
                    Z = __ldg(pb + 3) - __ldg(pk + 3);
            const R pq = p * qq, sum = p + qq;
            const R rho = pq / sum;
            const R r2 = X * X + Y * Y + Z * Z;
            const R pref = R(2.0 * 17.493418327624862) * __ldg(pb + 4) * __ldg(pk + 4) / (pq * sqrt(sum));
            R G[L + 1];
            boys_scaled<L, R>(G, rho * r2, rho, r2, pref, boys);
            hermite_r_shared64<L>(Rs, st, G, X, Y, Z);
        }
#pragma unroll 1
        for (int inu = 0; inu < NC; ++inu) {
            R kacc[NA];
            sfor<NA>([&](auto e_) { kacc[KX_CV(e_)] = R(0); });
            if (valid) {
                const int nx = cart_x(LC, inu), ny = cart_y(LC, inu), nz = cart_z(LC, inu);
#pragma unroll 1
                for (int ilam = 0; ilam < NB; ++ilam) {
                    const int lx = cart_x(LB, ilam), ly = cart_y(LB, ilam), lz = cart_z(LB, ilam);
                    R T[HCD];
                    {
                        R exd[LD + 1][LCD + 1], eyd[LD + 1][LCD + 1], ezd[LD + 1][LCD + 1];
                        sfor<LD + 1>([&](auto s_) {
                            constexpr int s = KX_CV(s_);
                            sfor<LCD + 1>([&](auto t_) {
                                constexpr int t = KX_CV(t_);
                                exd[s][t] = __ldg(Ecd + 0 * ECD + eidx(LC, LD, 0, s, t) + nx * (LD + 1) * (LCD + 1));
                                eyd[s][t] = __ldg(Ecd + 1 * ECD + eidx(LC, LD, 0, s, t) + ny * (LD + 1) * (LCD + 1));
                                ezd[s][t] = __ldg(Ecd + 2 * ECD + eidx(LC, LD, 0, s, t) + nz * (LD + 1) * (LCD + 1));
                            });
                        });
                        R pv[ND];
                        sfor<ND>([&](auto g_) { pv[KX_CV(g_)] = __ldg(Pb + ilam * ldp + KX_CV(g_)); });
                        sfor<HCD>([&](auto h_) { T[KX_CV(h_)] = R(0); });
                        sfor<ND>([&](auto g_) {
                            constexpr int g = KX_CV(g_);
                            constexpr int sx = cart_x(LD, g), sy = cart_y(LD, g), sz = cart_z(LD, g);
                            sfor<LCD + 1>([&](auto t_) {
                                constexpr int t = KX_CV(t_);
                                const R a1 = pv[g] * exd[sx][t];
                                sfor<LCD + 1 - t>([&](auto u_) {
                                    constexpr int u = KX_CV(u_);
                                    const R a2 = a1 * eyd[sy][u];
                                    sfor<LCD + 1 - t - u>([&](auto v_) {
                                        constexpr int v = KX_CV(v_);
                                        T[hidx(t, u, v)] += a2 * ezd[sz][v];
                                    });
                                });
                            });
                        });
                    }
                    R U[HAB];
                    sfor<HAB>([&](auto h_) { U[KX_CV(h_)] = R(0); });
                    sfor<L + 1>([&](auto ts_) {
                        constexpr int ts = KX_CV(ts_);
                        sfor<L + 1 - ts>([&](auto us_) {
                            constexpr int us = KX_CV(us_);
                            sfor<L + 1 - ts - us>([&](auto vs_) {
                                constexpr int vs = KX_CV(vs_);
                                const R r = Rs[hidx(ts, us, vs) * st];
                                sfor<(ts < LAB ? ts : LAB) + 1>([&](auto t_) {
                                    constexpr int t = KX_CV(t_);
                                    sfor<(us < LAB - t ? us : LAB - t) + 1>([&](auto u_) {
                                        constexpr int u = KX_CV(u_);
                                        sfor<(vs < LAB - t - u ? vs : LAB - t - u) + 1>([&](auto v_) {
                                            constexpr int v = KX_CV(v_);
                                            constexpr int t2 = ts - t, u2 = us - u, v2 = vs - v;
                                            if constexpr (t2 + u2 + v2 <= LCD) {
                                                if constexpr ((t2 + u2 + v2) & 1)
                                                    U[hidx(t, u, v)] -= r * T[hidx(t2, u2, v2)];
                                                else
                                                    U[hidx(t, u, v)] += r * T[hidx(t2, u2, v2)];
                                            }
                                        });
                                    });
                                });
                            });
                        });
                    });
                    R exa[LA + 1][LAB + 1], eya[LA + 1][LAB + 1], eza[LA + 1][LAB + 1];
                    sfor<LA + 1>([&](auto m_) {
                        constexpr int m = KX_CV(m_);
                        sfor<LAB + 1>([&](auto t_) {
                            constexpr int t = KX_CV(t_);
                            exa[m][t] = __ldg(Eab + 0 * EAB + eidx(LA, LB, m, 0, t) + lx * (LAB + 1));
                            eya[m][t] = __ldg(Eab + 1 * EAB + eidx(LA, LB, m, 0, t) + ly * (LAB + 1));
                            eza[m][t] = __ldg(Eab + 2 * EAB + eidx(LA, LB, m, 0, t) + lz * (LAB + 1));
                        });
                    });
                    sfor<NA>([&](auto mu_) {
                        constexpr int mu = KX_CV(mu_);
                        constexpr int mx = cart_x(LA, mu), my = cart_y(LA, mu), mz = cart_z(LA, mu);
                        R sacc = R(0);
                        sfor<LAB + 1>([&](auto t_) {
                            constexpr int t = KX_CV(t_);
                            sfor<LAB + 1 - t>([&](auto u_) {
                                constexpr int u = KX_CV(u_);
                                const R exy = exa[mx][t] * eya[my][u];
                                R sz_ = R(0);
                                sfor<LAB + 1 - t - u>([&](auto v_) {
                                    constexpr int v = KX_CV(v_);
                                    sz_ += eza[mz][v] * U[hidx(t, u, v)];
                                });
                                sacc += exy * sz_;
                            });
                        });
                        kacc[mu] += sacc;
                    });
                }
            }
            flush_k<NA, 1, R>(kacc, fa, fc, Kb + inu, ldk);
        }
    }
}

// ---------------------------------------------------------------------------
// algorithmic FLOP count of one quartet (mirrors the loops above)
// ---------------------------------------------------------------------------

template <int LA, int LB, int LC, int LD>
double eri_flops() {
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
    double f = integral_flops(L);             // set-up, Boys, Hermite recursion
    auto nreach = [](int Lh, int x, int y, int z, int l2) {
        int n = 0;
        for (int t = 0; t <= Lh; ++t)
            for (int u = 0; t + u <= Lh; ++u)
                for (int v = 0; t + u + v <= Lh; ++v) n += reach(t, u, v, x, y, z, l2);
        return n;
    };
    if (use_order_a<LA, LB, LC, LD>()) {
        for (int nu = 0; nu < NC; ++nu)
            for (int lam = 0; lam < NB; ++lam) {
                int nx = cart_x(LC, nu), ny = cart_y(LC, nu), nz = cart_z(LC, nu);
                int lx = cart_x(LB, lam), ly = cart_y(LB, lam), lz = cart_z(LB, lam);
                for (int sig = 0; sig < ND; ++sig) {
                    int sx = cart_x(LD, sig), sy = cart_y(LD, sig), sz = cart_z(LD, sig);
                    f += (nx + sx + 1) * (ny + sy + 1) * (2 + 2 * (nz + sz + 1));
                }
                f += 2.0 * nreach(LAB, lx, ly, lz, LA) * nreach(LCD, nx, ny, nz, LD);
                for (int mu = 0; mu < NA; ++mu) {
                    int mx = cart_x(LA, mu), my = cart_y(LA, mu), mz = cart_z(LA, mu);
                    f += (mx + lx + 1) * (my + ly + 1) * (3 + 2 * (mz + lz + 1)) + 1;
                }
            }
    } else {
        for (int mu = 0; mu < NA; ++mu)
            for (int sig = 0; sig < ND; ++sig) {
                int mx = cart_x(LA, mu), my = cart_y(LA, mu), mz = cart_z(LA, mu);
                int sx = cart_x(LD, sig), sy = cart_y(LD, sig), sz = cart_z(LD, sig);
                for (int lam = 0; lam < NB; ++lam) {
                    int lx = cart_x(LB, lam), ly = cart_y(LB, lam), lz = cart_z(LB, lam);
                    f += (mx + lx + 1) * (my + ly + 1) * (2 + 2 * (mz + lz + 1));
                }
                f += 2.0 * nreach(LAB, mx, my, mz, LB) * nreach(LCD, sx, sy, sz, LC);
                for (int nu = 0; nu < NC; ++nu) {
                    int nx = cart_x(LC, nu), ny = cart_y(LC, nu), nz = cart_z(LC, nu);
                    f += (nx + sx + 1) * (ny + sy + 1) * (3 + 2 * (nz + sz + 1)) + 1;
                }
            }
    }
    return f;
}

// The kernel of a class and precision: unrolled below ROLL_L.  Above it
// the FP64 classes have three variants (0 the rolled kernel, 1 the
// shared-memory kernel with full Hermite sets, 2 the same with the ket set
// pruned per nu) and the FP32 classes two (0 the shared-memory kernel, 1 the
// same pruned per nu); the autotuner picks one per class.
template <int LA, int LB, int LC, int LD>
EriKern eri_kernel(int prec, int variant) {
    if constexpr (LA + LB + LC + LD < ROLL_L) {
        return {prec == 0 ? &k_eri<LA, LB, LC, LD, double> : &k_eri<LA, LB, LC, LD, float>, 0, 1};
    } else {
        if (prec == 1) {
            if (variant == 1) return eri_kernel_bigp(LA * 27 + LB * 9 + LC * 3 + LD);
            return {&k_eri_big<LA, LB, LC, LD>, (int)sizeof(float) * big_slice<LA, LB, LC, LD>(), 2};
        }
        if (variant == 1)
            return {&k_eri_big64<LA, LB, LC, LD>, (int)sizeof(double) * nherm(LA + LB + LC + LD), 3};
        if (variant == 2) return eri_kernel_big64p(LA * 27 + LB * 9 + LC * 3 + LD);
        return {&k_eri_rolled<LA, LB, LC, LD, double>, 0, 3};
    }
}

// dispatch over (lc, ld) for a fixed bra pair class (la, lb)
#define KX_ERI_CASE(LA_, LB_, LC_, LD_) \
    case LC_ * 3 + LD_: return eri_kernel<LA_, LB_, LC_, LD_>(prec, variant);
#define KX_ERI_DISPATCH(LA_, LB_)                                                                        \
    EriKern eri_kernel_ab##LA_##LB_(int cls, int prec, int variant) {                                    \
        switch (cls % 9) {                                                                               \
            KX_ERI_CASE(LA_, LB_, 0, 0) KX_ERI_CASE(LA_, LB_, 0, 1) KX_ERI_CASE(LA_, LB_, 0, 2)          \
            KX_ERI_CASE(LA_, LB_, 1, 0) KX_ERI_CASE(LA_, LB_, 1, 1) KX_ERI_CASE(LA_, LB_, 1, 2)          \
            KX_ERI_CASE(LA_, LB_, 2, 0) KX_ERI_CASE(LA_, LB_, 2, 1) KX_ERI_CASE(LA_, LB_, 2, 2)          \
            default: return EriKern{nullptr, 0, 0};                                                      \
        }                                                                                                \
    }                                                                                                    \
    double class_flops_ab##LA_##LB_(int cls) {                                                           \
        static const double f[9] = {eri_flops<LA_, LB_, 0, 0>(), eri_flops<LA_, LB_, 0, 1>(),             \
                                    eri_flops<LA_, LB_, 0, 2>(), eri_flops<LA_, LB_, 1, 0>(),             \
                                    eri_flops<LA_, LB_, 1, 1>(), eri_flops<LA_, LB_, 1, 2>(),             \
                                    eri_flops<LA_, LB_, 2, 0>(), eri_flops<LA_, LB_, 2, 1>(),             \
                                    eri_flops<LA_, LB_, 2, 2>()};                                         \
        return f[cls % 9];                                                                               \
    }

// Double-word FP32 kernels (kx_dw.cuh) of the classes with la+lb+lc+ld <=
// DW_LMAX; the larger classes have none (fully unrolled in double-word
// arithmetic they take minutes each to compile and spill heavily) and run
// their FP64 kernels instead.
template <int LA, int LB, int LC, int LD>
EriKern eri_kernel_dw() {
    static_assert(DW_LMAX < ROLL_L, "double-word kernels are the unrolled ones");
    if constexpr (LA + LB + LC + LD <= DW_LMAX) return {&k_eri<LA, LB, LC, LD, dw>, 0, 1};
    else return {nullptr, 0, 0};
}

#define KX_ERI_DW_CASE(LA_, LB_, LC_, LD_) \
    case LC_ * 3 + LD_: return eri_kernel_dw<LA_, LB_, LC_, LD_>();
#define KX_ERI_DISPATCH_DW(LA_, LB_)                                                                     \
    EriKern eri_kernel_dw_ab##LA_##LB_(int cls) {                                                        \
        switch (cls % 9) {                                                                               \
            KX_ERI_DW_CASE(LA_, LB_, 0, 0) KX_ERI_DW_CASE(LA_, LB_, 0, 1) KX_ERI_DW_CASE(LA_, LB_, 0, 2) \
            KX_ERI_DW_CASE(LA_, LB_, 1, 0) KX_ERI_DW_CASE(LA_, LB_, 1, 1) KX_ERI_DW_CASE(LA_, LB_, 1, 2) \
            KX_ERI_DW_CASE(LA_, LB_, 2, 0) KX_ERI_DW_CASE(LA_, LB_, 2, 1) KX_ERI_DW_CASE(LA_, LB_, 2, 2) \
            default: return EriKern{nullptr, 0, 0};                                                      \
        }                                                                                                \
    }

}  // namespace kx
