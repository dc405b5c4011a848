// kx_eri_bigp.cu -- the second FP32 kernel of the largest classes
// (la+lb+lc+ld >= 7), in a translation unit of its own so that its five
// instantiations compile in parallel with the per-bra-class units.
#include "kx_eri_impl.cuh"

namespace kx {

// The FP32 shared-memory kernel (R and the E tables of both pairs in the
// thread's interleaved slice of shared memory) with the ket Cartesian index
// nu unrolled: the ket Hermite set of every nu is pruned to the indices
// some (nu, sig) reaches -- the union over sig of the boxes t' <= nx + sx,
// u' <= ny + sy, v' <= nz + sz -- in the T build and in the R contraction;
// lam stays a run-time loop over the full bra set.  The autotuner chooses
// between this kernel and the full-set one per class.
template <int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(128) k_eri_bigp(EriArgs args) {
    constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
    constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
    constexpr int HAB = nherm(LAB), HCD = nherm(LCD), HL = nherm(L);
    constexpr int EAB = etab(LA, LB), ECD = etab(LC, LD);
    constexpr int SAB = PAIR32_STRIDE, SCD = PAIR32_STRIDE;
    extern __shared__ float bigp_sh[];
    const int st = blockDim.x;
    float* const Rs = bigp_sh + threadIdx.x;               // R:  [HL]
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
        sfor<NC>([&](auto nu_) {
            constexpr int inu = KX_CV(nu_);
            constexpr int nx = cart_x(LC, inu), ny = cart_y(LC, inu), nz = cart_z(LC, inu);
            float kacc[NA];
            sfor<NA>([&](auto e_) { kacc[KX_CV(e_)] = 0.f; });
            if (valid) {
                // the nonzero E^cd_{nu sig, h'} factors of this nu, per dimension
                float exd[LD + 1][nx + LD + 1], eyd[LD + 1][ny + LD + 1], ezd[LD + 1][nz + LD + 1];
                sfor<LD + 1>([&](auto s_) {
                    constexpr int s = KX_CV(s_);
                    sfor<nx + s + 1>([&](auto t_) {
                        exd[s][KX_CV(t_)] = Es_cd[(0 * ECD + eidx(LC, LD, nx, s, KX_CV(t_))) * st];
                    });
                    sfor<ny + s + 1>([&](auto t_) {
                        eyd[s][KX_CV(t_)] = Es_cd[(1 * ECD + eidx(LC, LD, ny, s, KX_CV(t_))) * st];
                    });
                    sfor<nz + s + 1>([&](auto t_) {
                        ezd[s][KX_CV(t_)] = Es_cd[(2 * ECD + eidx(LC, LD, nz, s, KX_CV(t_))) * st];
                    });
                });
#pragma unroll 1
                for (int ilam = 0; ilam < NB; ++ilam) {
                    const int lx = cart_x(LB, ilam), ly = cart_y(LB, ilam), lz = cart_z(LB, ilam);
                    // T_{h'} = sum_sig E^cd_{nu sig,h'} P_{lam sig} over the reachable ket set
                    float T[HCD];
                    sfor<HCD>([&](auto h_) { T[KX_CV(h_)] = 0.f; });
                    sfor<ND>([&](auto g_) {
                        constexpr int g = KX_CV(g_);
                        constexpr int sx = cart_x(LD, g), sy = cart_y(LD, g), sz = cart_z(LD, g);
                        const float pv = __ldg(Pb + ilam * ldp + g);
                        sfor<nx + sx + 1>([&](auto t_) {
                            constexpr int t = KX_CV(t_);
                            const float a1 = pv * exd[sx][t];
                            sfor<ny + sy + 1>([&](auto u_) {
                                constexpr int u = KX_CV(u_);
                                const float a2 = a1 * eyd[sy][u];
                                sfor<nz + sz + 1>([&](auto v_) {
                                    constexpr int v = KX_CV(v_);
                                    T[hidx(t, u, v)] += a2 * ezd[sz][v];
                                });
                            });
                        });
                    });
                    // U_h = sum_{h' reachable} (-1)^{|h'|} R_{h+h'} T_{h'}
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
            flush_k<NA, 1, float>(kacc, fa, fc, Kb + inu, ldk);
        });
    }
}

EriKern eri_kernel_bigp(int cls) {
    switch (cls) {
        case 2 * 27 + 2 * 9 + 2 * 3 + 2:
            return {&k_eri_bigp<2, 2, 2, 2>, (int)sizeof(float) * big_slice<2, 2, 2, 2>(), 2};
        case 2 * 27 + 2 * 9 + 2 * 3 + 1:
            return {&k_eri_bigp<2, 2, 2, 1>, (int)sizeof(float) * big_slice<2, 2, 2, 1>(), 2};
        case 2 * 27 + 2 * 9 + 1 * 3 + 2:
            return {&k_eri_bigp<2, 2, 1, 2>, (int)sizeof(float) * big_slice<2, 2, 1, 2>(), 2};
        case 2 * 27 + 1 * 9 + 2 * 3 + 2:
            return {&k_eri_bigp<2, 1, 2, 2>, (int)sizeof(float) * big_slice<2, 1, 2, 2>(), 2};
        case 1 * 27 + 2 * 9 + 2 * 3 + 2:
            return {&k_eri_bigp<1, 2, 2, 2>, (int)sizeof(float) * big_slice<1, 2, 2, 2>(), 2};
        default: return EriKern{nullptr, 0, 0};
    }
}

}  // namespace kx
