// kx_eri_big64p.cu -- the third FP64 kernel of the largest classes
// (la+lb+lc+ld >= 7), in a translation unit of its own so that its five
// instantiations compile in parallel with the per-bra-class units.
#include "kx_eri_impl.cuh"

namespace kx {

// FP64 variant 2 for the largest classes: the big64 scheme with the ket
// Cartesian index nu unrolled, so the ket Hermite set of every nu is pruned
// to the indices that some (nu, sig) reaches -- the union over sig of the
// boxes t' <= nx + sx, u' <= ny + sy, v' <= nz + sz -- in the T build and in
// the R-contraction step; lam stays a run-time loop with the full bra set.
// The extra code (one copy of the lam loop per nu) buys fewer FP64
// multiply-adds: the R contraction shrinks by the ket pruning ratio.
template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(128) k_eri_big64p(EriArgs args) {
    using R = double;
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
    constexpr int HAB = nherm(LAB), HCD = nherm(LCD);
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    constexpr int SAB = pair_stride(LA, LB), SCD = pair_stride(LC, LD);
    extern __shared__ double big_sh64p[];
    const int st = blockDim.x;
    double* const Rs = big_sh64p + threadIdx.x;
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
        const R* Eab = bra;
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
        sfor<NC>([&](auto nu_) {
            constexpr int inu = KX_CV(nu_);
            constexpr int nx = cart_x(LC, inu), ny = cart_y(LC, inu), nz = cart_z(LC, inu);
            R kacc[NA];
            sfor<NA>([&](auto e_) { kacc[KX_CV(e_)] = R(0); });
            if (valid) {
#pragma unroll 1
                for (int ilam = 0; ilam < NB; ++ilam) {
                    const int lx = cart_x(LB, ilam), ly = cart_y(LB, ilam), lz = cart_z(LB, ilam);
                    // T_{h'} over the reachable ket set of this nu
                    R T[HCD];
                    sfor<HCD>([&](auto h_) { T[KX_CV(h_)] = R(0); });
                    sfor<ND>([&](auto g_) {
                        constexpr int g = KX_CV(g_);
                        constexpr int sx = cart_x(LD, g), sy = cart_y(LD, g), sz = cart_z(LD, g);
                        const R pv = __ldg(Pb + ilam * ldp + g);
                        sfor<nx + sx + 1>([&](auto t_) {
                            constexpr int t = KX_CV(t_);
                            const R a1 = pv * __ldg(Ecd + 0 * ECD + eidx(LC, LD, nx, sx, t));
                            sfor<ny + sy + 1>([&](auto u_) {
                                constexpr int u = KX_CV(u_);
                                const R a2 = a1 * __ldg(Ecd + 1 * ECD + eidx(LC, LD, ny, sy, u));
                                sfor<nz + sz + 1>([&](auto v_) {
                                    constexpr int v = KX_CV(v_);
                                    T[hidx(t, u, v)] += a2 * __ldg(Ecd + 2 * ECD + eidx(LC, LD, nz, sz, v));
                                });
                            });
                        });
                    });
                    // U_h = sum_{h' reachable} (-1)^{|h'|} R_{h+h'} T_{h'}
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
                                            if constexpr (reach(t2, u2, v2, nx, ny, nz, LD)) {
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
                    // K_{mu nu} += sum_h E^ab_{mu lam,h} U_h
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
        });
    }
}

EriKern eri_kernel_big64p(int cls) {
    constexpr int SM = sizeof(double);
    switch (cls) {
        case 2 * 27 + 2 * 9 + 2 * 3 + 2: return {&k_eri_big64p<2, 2, 2, 2>, SM * nherm(8), 3};
        case 2 * 27 + 2 * 9 + 2 * 3 + 1: return {&k_eri_big64p<2, 2, 2, 1>, SM * nherm(7), 3};
        case 2 * 27 + 2 * 9 + 1 * 3 + 2: return {&k_eri_big64p<2, 2, 1, 2>, SM * nherm(7), 3};
        case 2 * 27 + 1 * 9 + 2 * 3 + 2: return {&k_eri_big64p<2, 1, 2, 2>, SM * nherm(7), 3};
        case 1 * 27 + 2 * 9 + 2 * 3 + 2: return {&k_eri_big64p<1, 2, 2, 2>, SM * nherm(7), 3};
        default: return EriKern{nullptr, 0, 0};
    }
}

}  // namespace kx
