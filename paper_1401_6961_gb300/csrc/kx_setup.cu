// kx_setup.cu -- geometry- and density-dependent set-up stages:
//   * Hilbert ordering of the atoms (locality ordering, Sec. "Exchange as
//     hextree traversal"),
//   * ragged bisection of the shell index space (Eq. 1),
//   * shell-pair Schwarz factors (the diagonal integrals of Eq. 8) with the
//     optional overlap prune of Eq. 4,
//   * the Frobenius-norm quadtrees (pyramids) of Eq. 2 for Q and P,
//   * the Boys-function table and the per-pair Hermite expansion tables used
//     by the McMurchie-Davidson kernels.
#include <math.h>

#include <algorithm>
#include <cstring>

#include "kx_dw.cuh"
#include "kx_internal.cuh"

namespace kx {

int set_err(kx_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

int cuda_check(kx_ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return set_err(c, e == cudaErrorMemoryAllocation ? KX_ENOMEM : KX_ECUDA, m);
}

// ===========================================================================
// Hilbert order
// ===========================================================================

// Key of a cell on a 2^bits grid per axis: Skilling's transpose form.  From
// the top bit down, the low bits of every axis are either inverted (axis bit
// set) or exchanged with axis 0 (bit clear); the axes are then Gray-coded
// and the key is read by interleaving their bits, axis 0 most significant.
__device__ uint64_t hilbert_key3(uint32_t x0, uint32_t x1, uint32_t x2, int bits) {
    uint32_t X[3] = {x0, x1, x2};
    for (uint32_t Q = 1u << (bits - 1); Q > 1; Q >>= 1) {
        uint32_t low = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= low;
            } else {
                uint32_t t = (X[0] ^ X[i]) & low;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t flip = 0;
    for (uint32_t Q = 1u << (bits - 1); Q > 1; Q >>= 1)
        if (X[2] & Q) flip ^= Q - 1;
    X[0] ^= flip;
    X[1] ^= flip;
    X[2] ^= flip;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b)
#pragma unroll
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

// One block per system: bounding box, keys, ranks of the system's atoms
// (atoms [ao[s], ao[s+1]); ranks count from ao[s]).
__global__ void k_atom_keys(const double* __restrict__ xyz, const int32_t* __restrict__ ao,
                            uint64_t* __restrict__ key, int32_t* __restrict__ rank) {
    __shared__ double s_lo[3], s_hi[3];
    const int a0 = ao[blockIdx.x], n = ao[blockIdx.x + 1] - a0;
    xyz += 3 * (int64_t)a0;
    key += a0;
    rank += a0;
    if (threadIdx.x < 3) {
        double lo = xyz[threadIdx.x], hi = xyz[threadIdx.x];
        for (int a = 1; a < n; ++a) {
            double v = xyz[3 * a + threadIdx.x];
            lo = fmin(lo, v);
            hi = fmax(hi, v);
        }
        s_lo[threadIdx.x] = lo;
        s_hi[threadIdx.x] = hi;
    }
    __syncthreads();
    double span = 0.0;
    for (int x = 0; x < 3; ++x) span = fmax(span, __dsub_rn(s_hi[x], s_lo[x]));
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        uint32_t q[3];
        for (int x = 0; x < 3; ++x) {
            int v = 0;
            if (span > 0.0) {
                // q = floor(((x - lo) / span) * 1023 + 0.5), each step rounded
                double t = __ddiv_rn(__dsub_rn(xyz[3 * a + x], s_lo[x]), span);
                double u = __dmul_rn(t, 1023.0);
                v = (int)floor(__dadd_rn(u, 0.5));
                v = v < 0 ? 0 : (v > 1023 ? 1023 : v);
            }
            q[x] = (uint32_t)v;
        }
        key[a] = hilbert_key3(q[0], q[1], q[2], 10);
    }
    __syncthreads();
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
        uint64_t ka = key[a];
        int r = 0;
        for (int b = 0; b < n; ++b) {
            uint64_t kb = key[b];
            r += (kb < ka) || (kb == ka && b < a);
        }
        rank[a] = a0 + r;
    }
}

// Tree position of every shell: atoms by rank, input order inside an atom,
// within the shell range [so[y], so[y+1]) of the shell's system y.
__global__ void k_shell_pos(const int32_t* __restrict__ shell_atom, const int32_t* __restrict__ rank,
                            const int32_t* __restrict__ so, int nsys, int ns, int32_t* __restrict__ perm) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= ns) return;
    int lo = 0, hi = nsys - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (so[m] <= s) lo = m; else hi = m - 1;
    }
    const int t0 = so[lo], t1 = so[lo + 1];
    int ra = rank[shell_atom[s]];
    int pos = t0;
    for (int t = t0; t < t1; ++t) {
        int rt = rank[shell_atom[t]];
        pos += (rt < ra) || (rt == ra && t < s);
    }
    perm[pos] = s;
}

int order_atoms(kx_ctx* c) {
    int n = c->n_atom, ns = c->n_shell, nsys = c->n_sys;
    double* d_xyz = nullptr;
    uint64_t* d_key = nullptr;
    int32_t *d_rank = nullptr, *d_sa = nullptr, *d_ao = nullptr, *d_so = nullptr;
    auto cleanup = [&]() {
        cudaFree(d_xyz); cudaFree(d_key); cudaFree(d_rank); cudaFree(d_sa); cudaFree(d_ao); cudaFree(d_so);
    };
    cudaError_t e = cudaMalloc(&d_xyz, sizeof(double) * 3 * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_key, sizeof(uint64_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_rank, sizeof(int32_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&d_sa, sizeof(int32_t) * ns);
    if (e == cudaSuccess) e = cudaMalloc(&d_ao, sizeof(int32_t) * (nsys + 1));
    if (e == cudaSuccess) e = cudaMalloc(&d_so, sizeof(int32_t) * (nsys + 1));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_perm, sizeof(int32_t) * ns);
    if (e != cudaSuccess) { cleanup(); return cuda_check(c, e, "order_atoms alloc"); }
    cudaMemcpyAsync(d_xyz, c->xyz.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_sa, c->shell_atom.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_ao, c->sys_atom.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_so, c->sys_shell.data(), sizeof(int32_t) * (nsys + 1), cudaMemcpyHostToDevice, c->stream);
    k_atom_keys<<<nsys, 1024, 0, c->stream>>>(d_xyz, d_ao, d_key, d_rank);
    k_shell_pos<<<(ns + 255) / 256, 256, 0, c->stream>>>(d_sa, d_rank, d_so, nsys, ns, c->d_perm);
    c->perm.resize(ns);
    cudaMemcpyAsync(c->perm.data(), c->d_perm, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, c->stream);
    e = cudaStreamSynchronize(c->stream);
    cleanup();
    if (e != cudaSuccess) return cuda_check(c, e, "order_atoms");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "order_atoms kernels");
    c->have_order = true;
    return KX_OK;
}

// ===========================================================================
// Hermite expansion coefficients (per dimension) and Hermite integrals
// ===========================================================================

// E^{ij}_t of the product of two 1D Gaussians with the Gaussian-product
// factor left out: E^{00}_0 = 1,
//   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1},
//   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}.
// Output layout E[eidx(la,lb,i,j,t)].
__device__ void hermite_e_1d(int la, int lb, double XPA, double XPB, double inv2p, double* E) {
    const int LT = la + lb + 1;
    #pragma unroll 1
    for (int k = 0; k < etab(la, lb); ++k) E[k] = 0.0;
    E[eidx(la, lb, 0, 0, 0)] = 1.0;
    #pragma unroll 1
    for (int i = 0; i <= la; ++i) {
        if (i > 0) {
            #pragma unroll 1
            for (int t = 0; t <= i; ++t) {
                double v = XPA * E[eidx(la, lb, i - 1, 0, t)];
                if (t > 0) v += inv2p * E[eidx(la, lb, i - 1, 0, t - 1)];
                if (t + 1 <= i - 1) v += (t + 1) * E[eidx(la, lb, i - 1, 0, t + 1)];
                E[eidx(la, lb, i, 0, t)] = v;
            }
        }
        #pragma unroll 1
        for (int j = 1; j <= lb; ++j)
            #pragma unroll 1
            for (int t = 0; t <= i + j && t < LT; ++t) {
                double v = XPB * E[eidx(la, lb, i, j - 1, t)];
                if (t > 0) v += inv2p * E[eidx(la, lb, i, j - 1, t - 1)];
                if (t + 1 <= i + j - 1) v += (t + 1) * E[eidx(la, lb, i, j - 1, t + 1)];
                E[eidx(la, lb, i, j, t)] = v;
            }
    }
}

// Hermite Coulomb integrals R_{tuv} (n = 0) for t+u+v <= L at P-Q = (X,Y,Z),
// from R^n_{000} = G_n (already scaled) by
//   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X R^{n+1}_{t,u,v}  (same in u, v),
// evaluated in place from the highest n down.  Generic L <= 8.
__device__ void hermite_r_generic(int L, const double* G, double X, double Y, double Z, double* R) {
    R[0] = G[L];
    #pragma unroll 1
    for (int n = L - 1; n >= 0; --n) {
        #pragma unroll 1
        for (int j = L - n; j >= 1; --j)
            #pragma unroll 1
            for (int t = j; t >= 0; --t)
                #pragma unroll 1
                for (int u = j - t; u >= 0; --u) {
                    int v = j - t - u;
                    double r;
                    if (t > 0) {
                        r = X * R[hidx(t - 1, u, v)];
                        if (t > 1) r += (t - 1) * R[hidx(t - 2, u, v)];
                    } else if (u > 0) {
                        r = Y * R[hidx(t, u - 1, v)];
                        if (u > 1) r += (u - 1) * R[hidx(t, u - 2, v)];
                    } else {
                        r = Z * R[hidx(t, u, v - 1)];
                        if (v > 1) r += (v - 1) * R[hidx(t, u, v - 2)];
                    }
                    R[hidx(t, u, v)] = r;
                }
        R[0] = G[n];
    }
}

__device__ double norm_prim(double a, int l) {
    double df = (l == 2) ? 3.0 : 1.0;
    return pow(2.0 * a / PI, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(df);
}

// ===========================================================================
// Schwarz factors (Eq. 8) and the overlap prune (Eq. 4)
// ===========================================================================

// One thread per unordered pair a <= b (tree positions).  (ab|ab) has
// P = Q, so T = 0, F_n(0) = 1/(2n+1), and R depends on rho = p/2 only.
__global__ void k_schwarz(const Seg* __restrict__ seg, int nseg, int64_t npair, const int32_t* __restrict__ tl,
                          const double* __restrict__ tctr, const double* __restrict__ talpha, double tau_ovlp,
                          double* __restrict__ s2, double* __restrict__ snorm, float* __restrict__ slog) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= npair) return;
    const Seg sg = seg[seg_find(seg, nseg, idx)];
    const int a = sg.base + (int)((idx - sg.off) / sg.n), b = sg.base + (int)((idx - sg.off) % sg.n);
    if (a > b) return;
    int la = tl[a], lb = tl[b];
    double A[3] = {tctr[3 * a], tctr[3 * a + 1], tctr[3 * a + 2]};
    double B[3] = {tctr[3 * b], tctr[3 * b + 1], tctr[3 * b + 2]};
    double al = talpha[a], be = talpha[b];
    double p = al + be, inv2p = 0.5 / p;
    double AB2 = 0.0;
    double E[3][45];
    #pragma unroll 1
    for (int x = 0; x < 3; ++x) {
        double Px = (al * A[x] + be * B[x]) / p;
        AB2 += (A[x] - B[x]) * (A[x] - B[x]);
        hermite_e_1d(la, lb, Px - A[x], Px - B[x], inv2p, E[x]);
    }
    double Kab = exp(-al * be / p * AB2);
    double na = norm_prim(al, la), nb = norm_prim(be, lb);
    int pruned = 0;
    if (tau_ovlp > 0.0) {
        // (phi_mu, phi_nu) = N_a N_b K_ab (pi/p)^{3/2} E^x_0 E^y_0 E^z_0
        double s0 = na * nb * Kab * pow(PI / p, 1.5);
        double mx = 0.0;
        #pragma unroll 1
        for (int i = 0; i < ncart(la); ++i)
            #pragma unroll 1
            for (int j = 0; j < ncart(lb); ++j) {
                double v = s0 * E[0][eidx(la, lb, cart_x(la, i), cart_x(lb, j), 0)] *
                           E[1][eidx(la, lb, cart_y(la, i), cart_y(lb, j), 0)] *
                           E[2][eidx(la, lb, cart_z(la, i), cart_z(lb, j), 0)];
                mx = fmax(mx, fabs(v));
            }
        pruned = mx < tau_ovlp;
    }
    double total = 0.0;
    if (!pruned) {
        const int L = 2 * (la + lb);
        double rho = 0.5 * p;
        double pref = 2.0 * pow(PI, 2.5) / (p * p * sqrt(2.0 * p)) * Kab * Kab * na * na * nb * nb;
        double G[9];
        double s = pref;
        #pragma unroll 1
        for (int n = 0; n <= L; ++n) {
            G[n] = s / (2 * n + 1);
            s *= -2.0 * rho;
        }
        double R[165];
        hermite_r_generic(L, G, 0.0, 0.0, 0.0, R);
        // (mu lam|mu lam) = sum_{h,h'} E_h (-1)^{|h'|} E_h' R_{h+h'}
        #pragma unroll 1
        for (int i = 0; i < ncart(la); ++i)
            #pragma unroll 1
            for (int j = 0; j < ncart(lb); ++j) {
                int ix = cart_x(la, i), iy = cart_y(la, i), iz = cart_z(la, i);
                int jx = cart_x(lb, j), jy = cart_y(lb, j), jz = cart_z(lb, j);
                double acc = 0.0;
                #pragma unroll 1
                for (int t = 0; t <= ix + jx; ++t)
                    #pragma unroll 1
                    for (int u = 0; u <= iy + jy; ++u)
                        #pragma unroll 1
                        for (int v = 0; v <= iz + jz; ++v) {
                            double eh = E[0][eidx(la, lb, ix, jx, t)] * E[1][eidx(la, lb, iy, jy, u)] *
                                        E[2][eidx(la, lb, iz, jz, v)];
                            double inner = 0.0;
                            #pragma unroll 1
                            for (int t2 = 0; t2 <= ix + jx; ++t2)
                                #pragma unroll 1
                                for (int u2 = 0; u2 <= iy + jy; ++u2)
                                    #pragma unroll 1
                                    for (int v2 = 0; v2 <= iz + jz; ++v2) {
                                        double e2 = E[0][eidx(la, lb, ix, jx, t2)] * E[1][eidx(la, lb, iy, jy, u2)] *
                                                    E[2][eidx(la, lb, iz, jz, v2)];
                                        double r = R[hidx(t + t2, u + u2, v + v2)];
                                        inner += ((t2 + u2 + v2) & 1) ? -e2 * r : e2 * r;
                                    }
                            acc += eh * inner;
                        }
                total += acc;
            }
    }
    double nrm = sqrt(total);
    float lg = total > 0.0 ? (float)log2(nrm) : -INFINITY;
    int64_t i1 = idx, i2 = sg.t0() + (int64_t)b * sg.n + a;
    s2[i1] = total; s2[i2] = total;
    snorm[i1] = nrm; snorm[i2] = nrm;
    slog[i1] = lg; slog[i2] = lg;
}

// basis in tree order
__global__ void k_tree_basis(int ns, const int32_t* __restrict__ perm, const int32_t* __restrict__ l,
                             const double* __restrict__ ctr, const double* __restrict__ alpha,
                             const int32_t* __restrict__ foff, int32_t* __restrict__ tl,
                             double* __restrict__ tctr, double* __restrict__ talpha,
                             int32_t* __restrict__ tfoff) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    int s = perm[i];
    tl[i] = l[s];
    talpha[i] = alpha[s];
    tfoff[i] = foff[s];
    for (int x = 0; x < 3; ++x) tctr[3 * i + x] = ctr[3 * s + x];
}

int schwarz(kx_ctx* c, double tau_ovlp) {
    int ns = c->n_shell;
    int64_t n2 = c->sp_total;
    // upload the basis in user order, gather it into tree order
    std::vector<double> ctr(3 * (size_t)ns);
    std::vector<int32_t> foff(ns);
    for (int s = 0; s < ns; ++s) {
        for (int x = 0; x < 3; ++x) ctr[3 * s + x] = c->xyz[3 * c->shell_atom[s] + x];
        foff[s] = (int32_t)c->fn_off[s];
    }
    int32_t *d_l = nullptr, *d_foff = nullptr;
    double *d_ctr = nullptr, *d_alpha = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](void** p, size_t b) { if (e == cudaSuccess) e = cudaMalloc(p, b); };
    if (!c->d_tl) {
        A((void**)&c->d_tl, sizeof(int32_t) * ns);
        A((void**)&c->d_tctr, sizeof(double) * 3 * ns);
        A((void**)&c->d_talpha, sizeof(double) * ns);
        A((void**)&c->d_tfoff, sizeof(int32_t) * ns);
        A((void**)&c->d_s2, sizeof(double) * n2);
        A((void**)&c->d_snorm, sizeof(double) * n2);
        A((void**)&c->d_slog, sizeof(float) * n2);
    }
    A((void**)&d_l, sizeof(int32_t) * ns);
    A((void**)&d_foff, sizeof(int32_t) * ns);
    A((void**)&d_ctr, sizeof(double) * 3 * ns);
    A((void**)&d_alpha, sizeof(double) * ns);
    if (e != cudaSuccess) {
        cudaFree(d_l); cudaFree(d_foff); cudaFree(d_ctr); cudaFree(d_alpha);
        return cuda_check(c, e, "schwarz alloc");
    }
    cudaMemcpyAsync(d_l, c->shell_l.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_foff, foff.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_ctr, ctr.data(), sizeof(double) * 3 * ns, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(d_alpha, c->shell_alpha.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, c->stream);
    k_tree_basis<<<(ns + 255) / 256, 256, 0, c->stream>>>(ns, c->d_perm, d_l, d_ctr, d_alpha, d_foff, c->d_tl,
                                                          c->d_tctr, c->d_talpha, c->d_tfoff);
    k_schwarz<<<(unsigned)((n2 + 127) / 128), 128, 0, c->stream>>>(c->d_sseg, c->n_sys, n2, c->d_tl, c->d_tctr,
                                                                 c->d_talpha, tau_ovlp, c->d_s2, c->d_snorm,
                                                                 c->d_slog);
    e = cudaStreamSynchronize(c->stream);
    cudaFree(d_l); cudaFree(d_foff); cudaFree(d_ctr); cudaFree(d_alpha);
    if (e != cudaSuccess) return cuda_check(c, e, "schwarz");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "schwarz kernels");
    c->have_schwarz = true;
    return KX_OK;
}

// ===========================================================================
// ragged bisection (Eq. 1), one block, level by level
// ===========================================================================

constexpr int TREE_THREADS = 1024;

// Block-wide exclusive scan of per-thread values (shared scratch of
// TREE_THREADS ints); returns the exclusive prefix, *total gets the sum.
__device__ int block_excl_scan(int v, int* sh, int* total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int d = 1; d < 32; d <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int excl = x - v + (w > 0 ? sh[w - 1] : 0);
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return excl;
}

// Nodes of level k occupy [off_k, off_k + n_k) of the flat arrays.  A node
// is a leaf when it holds at most leaf_max functions or a single shell; a
// leaf is carried to the next level unchanged (one child).  A non-leaf is
// split at the shell boundary s in (lo, hi) minimising
// |2 pre[s] - pre[lo] - pre[hi]|, the lower s on a tie.
__global__ void __launch_bounds__(TREE_THREADS)
k_build_tree(int ns, const int32_t* __restrict__ tl, const int32_t* __restrict__ roots, int nroot, int leaf_max,
             int max_nodes, int32_t* __restrict__ pre, int32_t* __restrict__ lo, int32_t* __restrict__ hi,
             int32_t* __restrict__ child, int32_t* __restrict__ nchild, int32_t* __restrict__ level_n,
             int32_t* __restrict__ status) {
    __shared__ int sh[32];
    __shared__ int s_n, s_off, s_done;
    // function-count prefix sums (sequential, once per geometry); level 0
    // holds one root per system, [roots[i], roots[i+1])
    if (threadIdx.x == 0) {
        pre[0] = 0;
        for (int s = 0; s < ns; ++s) pre[s + 1] = pre[s] + ncart(tl[s]);
        s_n = nroot;
        s_off = 0;
        s_done = 0;
        status[0] = 0;
    }
    for (int i = threadIdx.x; i < nroot; i += blockDim.x) {
        lo[i] = roots[i];
        hi[i] = roots[i + 1];
    }
    __syncthreads();
    int level = 0;
    while (true) {
        int n = s_n, off = s_off;
        if (threadIdx.x == 0) level_n[level] = n;
        // each thread handles a contiguous run of nodes
        int per = (n + blockDim.x - 1) / blockDim.x;
        int b0 = min(n, (int)threadIdx.x * per), b1 = min(n, b0 + per);
        int mine = 0, nonleaf = 0;
        for (int i = b0; i < b1; ++i) {
            int l0 = lo[off + i], h0 = hi[off + i];
            int leaf = (pre[h0] - pre[l0] <= leaf_max) || (h0 - l0 == 1);
            nchild[off + i] = leaf ? 1 : 2;
            mine += leaf ? 1 : 2;
            nonleaf |= !leaf;
        }
        int total;
        int base = block_excl_scan(mine, sh, &total);
        int any = __syncthreads_or(nonleaf);
        if (!any) break;                       // every node is a leaf: deepest level
        if (off + n + total > max_nodes || level + 1 >= MAX_LEVELS) {
            if (threadIdx.x == 0) status[0] = 1;
            break;
        }
        int noff = off + n;
        int pos = base;
        for (int i = b0; i < b1; ++i) {
            int l0 = lo[off + i], h0 = hi[off + i];
            child[off + i] = pos;
            if (nchild[off + i] == 1) {
                lo[noff + pos] = l0;
                hi[noff + pos] = h0;
                pos += 1;
            } else {
                int target = pre[l0] + pre[h0];
                // first s in (l0, h0) with 2 pre[s] >= target
                int a = l0 + 1, b = h0 - 1, s1 = h0;
                while (a <= b) {
                    int m = (a + b) >> 1;
                    if (2 * pre[m] >= target) { s1 = m; b = m - 1; } else { a = m + 1; }
                }
                int best;
                if (s1 >= h0) best = h0 - 1;
                else if (s1 - 1 > l0 && (target - 2 * pre[s1 - 1]) <= (2 * pre[s1] - target)) best = s1 - 1;
                else best = s1;
                lo[noff + pos] = l0;
                hi[noff + pos] = best;
                lo[noff + pos + 1] = best;
                hi[noff + pos + 1] = h0;
                pos += 2;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_off = noff;
            s_n = total;
        }
        __syncthreads();
        ++level;
    }
    if (threadIdx.x == 0) status[1] = level;
}

// ---------------------------------------------------------------------------
// norm pyramids (Eq. 2): squared Frobenius norms per level, bottom-up
// ---------------------------------------------------------------------------

// Deepest level: sum over the shells of the two leaves, a outer, b inner.
// Flat index e over the level's block-diagonal table (blocks lseg, one per
// system, offsets absolute); the shell table block of the same system.
__global__ void k_pyr_leaves(int64_t e0, int64_t e1, const Seg* __restrict__ lseg, const Seg* __restrict__ sseg,
                             int nsys, const int32_t* __restrict__ llo, const int32_t* __restrict__ lhi,
                             const double* __restrict__ sq_shell, double* __restrict__ sq,
                             double* __restrict__ nrm) {
    int64_t i = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= e1) return;
    const int y = seg_find(lseg, nsys, i);
    const Seg lg = lseg[y], sg = sseg[y];
    const int X = lg.base + (int)((i - lg.off) / lg.n), Y = lg.base + (int)((i - lg.off) % lg.n);
    const int64_t t0 = sg.t0();
    double s = 0.0;
    for (int a = llo[X]; a < lhi[X]; ++a)
        for (int b = llo[Y]; b < lhi[Y]; ++b) s = __dadd_rn(s, sq_shell[t0 + (int64_t)a * sg.n + b]);
    sq[i] = s;
    nrm[i] = sqrt(s);
}

// level k from level k+1: children pairs in order (0,0),(0,1),(1,0),(1,1)
__global__ void k_pyr_up(int64_t e0, int64_t e1, const Seg* __restrict__ lseg, const Seg* __restrict__ lseg_next,
                         int nsys, const int32_t* __restrict__ child, const int32_t* __restrict__ nchild,
                         const double* sq_all, double* sq, double* __restrict__ nrm) {
    int64_t i = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= e1) return;
    const int y = seg_find(lseg, nsys, i);
    const Seg lg = lseg[y], ng = lseg_next[y];
    const int X = lg.base + (int)((i - lg.off) / lg.n), Y = lg.base + (int)((i - lg.off) % lg.n);
    const int64_t t0 = ng.t0();
    int cx = child[X], cy = child[Y], nx = nchild[X], ny = nchild[Y];
    double s = 0.0;
    for (int ii = 0; ii < nx; ++ii)
        for (int jj = 0; jj < ny; ++jj) s = __dadd_rn(s, sq_all[t0 + (int64_t)(cx + ii) * ng.n + (cy + jj)]);
    sq[i] = s;
    nrm[i] = sqrt(s);
}

static int build_pyramid(kx_ctx* c, const double* sq_shell, double* sq, double* nrm) {
    const int D = c->depth, ny = c->n_sys;
    {
        const int64_t e0 = c->pyr_off[D], e1 = c->pyr_off[D + 1];
        k_pyr_leaves<<<(unsigned)((e1 - e0 + 255) / 256), 256, 0, c->stream>>>(
            e0, e1, c->d_lseg + (size_t)D * ny, c->d_sseg, ny, c->d_leaf_lo, c->d_leaf_hi, sq_shell, sq, nrm);
    }
    c->launches += 1 + D;
    for (int k = D - 1; k >= 0; --k) {
        const int64_t e0 = c->pyr_off[k], e1 = c->pyr_off[k + 1];
        k_pyr_up<<<(unsigned)((e1 - e0 + 255) / 256), 256, 0, c->stream>>>(
            e0, e1, c->d_lseg + (size_t)k * ny, c->d_lseg + (size_t)(k + 1) * ny, ny,
            c->d_node_child + c->levels[k].off, c->d_node_nchild + c->levels[k].off, sq, sq, nrm);
    }
    return KX_OK;
}

int build_tree(kx_ctx* c, int leaf_max) {
    int ns = c->n_shell;
    int max_nodes = MAX_LEVELS * ns + 1;
    int32_t *d_pre = nullptr, *d_lo = nullptr, *d_hi = nullptr, *d_child = nullptr, *d_nchild = nullptr,
            *d_leveln = nullptr, *d_status = nullptr;
    cudaError_t e = cudaSuccess;
    auto A = [&](int32_t** p, size_t n) { if (e == cudaSuccess) e = cudaMalloc(p, sizeof(int32_t) * n); };
    A(&d_pre, ns + 1); A(&d_lo, max_nodes); A(&d_hi, max_nodes); A(&d_child, max_nodes);
    A(&d_nchild, max_nodes); A(&d_leveln, MAX_LEVELS); A(&d_status, 2);
    auto cleanup = [&]() {
        cudaFree(d_pre); cudaFree(d_lo); cudaFree(d_hi); cudaFree(d_child); cudaFree(d_nchild);
        cudaFree(d_leveln); cudaFree(d_status);
    };
    if (e != cudaSuccess) { cleanup(); return cuda_check(c, e, "build_tree alloc"); }
    int32_t* d_roots = nullptr;
    e = cudaMalloc(&d_roots, sizeof(int32_t) * (c->n_sys + 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_roots, c->sys_shell.data(), sizeof(int32_t) * (c->n_sys + 1), cudaMemcpyHostToDevice,
                            c->stream);
    if (e != cudaSuccess) { cudaFree(d_roots); cleanup(); return cuda_check(c, e, "build_tree alloc"); }
    k_build_tree<<<1, TREE_THREADS, 0, c->stream>>>(ns, c->d_tl, d_roots, c->n_sys, leaf_max, max_nodes, d_pre, d_lo,
                                                    d_hi, d_child, d_nchild, d_leveln, d_status);
    int32_t status[2] = {0, 0};
    std::vector<int32_t> leveln(MAX_LEVELS, 0);
    cudaMemcpyAsync(status, d_status, sizeof(status), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(leveln.data(), d_leveln, sizeof(int32_t) * MAX_LEVELS, cudaMemcpyDeviceToHost, c->stream);
    e = cudaStreamSynchronize(c->stream);
    cudaFree(d_roots);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { cleanup(); return cuda_check(c, e, "build_tree"); }
    if (status[0] != 0) {
        cleanup();
        return set_err(c, KX_ECAPACITY, "bisection deeper than the supported 32 levels");
    }
    int D = status[1];
    c->depth = D;
    c->leaf_max = leaf_max;
    c->levels.assign(D + 1, LevelInfo{0, 0});
    int off = 0;
    for (int k = 0; k <= D; ++k) {
        c->levels[k].n = leveln[k];
        c->levels[k].off = off;
        off += leveln[k];
    }
    int total = off;
    c->node_lo.resize(total); c->node_hi.resize(total); c->node_child.resize(total); c->node_nchild.resize(total);
    cudaMemcpy(c->node_lo.data(), d_lo, sizeof(int32_t) * total, cudaMemcpyDeviceToHost);
    cudaMemcpy(c->node_hi.data(), d_hi, sizeof(int32_t) * total, cudaMemcpyDeviceToHost);
    cudaMemcpy(c->node_child.data(), d_child, sizeof(int32_t) * total, cudaMemcpyDeviceToHost);
    cudaMemcpy(c->node_nchild.data(), d_nchild, sizeof(int32_t) * total, cudaMemcpyDeviceToHost);
    cleanup();
    // keep compact device copies
    cudaFree(c->d_node_lo); cudaFree(c->d_node_hi); cudaFree(c->d_node_child); cudaFree(c->d_node_nchild);
    cudaFree(c->d_leaf_lo); cudaFree(c->d_leaf_hi);
    c->d_node_lo = c->d_node_hi = c->d_node_child = c->d_node_nchild = c->d_leaf_lo = c->d_leaf_hi = nullptr;
    int nl = c->levels[D].n;
    e = cudaSuccess;
    A(&c->d_node_lo, total); A(&c->d_node_hi, total); A(&c->d_node_child, total); A(&c->d_node_nchild, total);
    A(&c->d_leaf_lo, nl); A(&c->d_leaf_hi, nl);
    if (e != cudaSuccess) return cuda_check(c, e, "build_tree alloc");
    cudaMemcpyAsync(c->d_node_lo, c->node_lo.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_node_hi, c->node_hi.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_node_child, c->node_child.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_node_nchild, c->node_nchild.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice,
                    c->stream);
    cudaMemcpyAsync(c->d_leaf_lo, c->node_lo.data() + c->levels[D].off, sizeof(int32_t) * nl, cudaMemcpyHostToDevice,
                    c->stream);
    cudaMemcpyAsync(c->d_leaf_hi, c->node_hi.data() + c->levels[D].off, sizeof(int32_t) * nl, cudaMemcpyHostToDevice,
                    c->stream);
    // per-level blocks: the nodes of a level are system-major (level 0 holds
    // the roots in system order and children follow their parents)
    const int ny = c->n_sys;
    std::vector<int32_t> node_sys(total);
    c->lseg.assign((size_t)(D + 1) * ny, Seg{0, 0, 0});
    c->pyr_off.assign(D + 2, 0);
    for (int k = 0; k <= D; ++k) {
        if (c->levels[k].n > 65535) return set_err(c, KX_ECAPACITY, "more than 65535 nodes in one tree level");
        int y = 0;
        for (int X = 0; X < c->levels[k].n; ++X) {
            const int lo = c->node_lo[c->levels[k].off + X];
            while (y + 1 < ny && c->sys_shell[y + 1] <= lo) ++y;
            node_sys[c->levels[k].off + X] = y;
            Seg& g = c->lseg[(size_t)k * ny + y];
            if (g.n == 0) g.base = X;
            g.n++;
        }
        int64_t off = c->pyr_off[k];
        for (int y2 = 0; y2 < ny; ++y2) {
            Seg& g = c->lseg[(size_t)k * ny + y2];
            if (g.n == 0) return set_err(c, KX_ECUDA, "tree level without a node of some system");
            g.off = off;
            off += (int64_t)g.n * g.n;
        }
        c->pyr_off[k + 1] = off;
    }
    cudaFree(c->d_lseg); cudaFree(c->d_node_sys);
    c->d_lseg = nullptr; c->d_node_sys = nullptr;
    e = cudaMalloc(&c->d_lseg, sizeof(Seg) * c->lseg.size());
    if (e == cudaSuccess) e = cudaMalloc(&c->d_node_sys, sizeof(int32_t) * total);
    if (e != cudaSuccess) return cuda_check(c, e, "build_tree alloc");
    cudaMemcpyAsync(c->d_lseg, c->lseg.data(), sizeof(Seg) * c->lseg.size(), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_node_sys, node_sys.data(), sizeof(int32_t) * total, cudaMemcpyHostToDevice, c->stream);
    // pyramid storage
    int64_t pyr = c->pyr_off[D + 1];
    cudaFree(c->d_sq_s); cudaFree(c->d_sq_p); cudaFree(c->d_nrm_s); cudaFree(c->d_nrm_p);
    c->d_sq_s = c->d_sq_p = c->d_nrm_s = c->d_nrm_p = nullptr;
    auto AD = [&](double** p) { if (e == cudaSuccess) e = cudaMalloc(p, sizeof(double) * pyr); };
    AD(&c->d_sq_s); AD(&c->d_sq_p); AD(&c->d_nrm_s); AD(&c->d_nrm_p);
    if (e != cudaSuccess) return cuda_check(c, e, "pyramid alloc");
    KX_TRY(build_pyramid(c, c->d_s2, c->d_sq_s, c->d_nrm_s));
    e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(c, e, "schwarz pyramid");
    c->have_tree = true;
    c->have_pq = false;
    return KX_OK;
}

// ===========================================================================
// P shell-block norms and their pyramid
// ===========================================================================

__global__ void k_p_shell(const Seg* __restrict__ seg, int nseg, int64_t n2, const int32_t* __restrict__ tl,
                          const int32_t* __restrict__ tfoff, const MatFrame* __restrict__ mf,
                          const double* __restrict__ P, double* __restrict__ pq, double* __restrict__ pn,
                          float* __restrict__ plog) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const int y = seg_find(seg, nseg, i);
    const Seg sg = seg[y];
    const int b = sg.base + (int)((i - sg.off) / sg.n), d = sg.base + (int)((i - sg.off) % sg.n);
    const MatFrame f = mf[y];
    int fb = tfoff[b], fd = tfoff[d], nb = ncart(tl[b]), nd = ncart(tl[d]);
    double s = 0.0;
    for (int x = 0; x < nb; ++x)
        for (int z = 0; z < nd; ++z) {
            double v = P[f.p0 + (int64_t)(fb + x) * f.ldp + fd + z];
            s = __dadd_rn(s, __dmul_rn(v, v));
        }
    pq[i] = s;
    double r = sqrt(s);
    pn[i] = r;
    plog[i] = s > 0.0 ? (float)log2(r) : -INFINITY;
}

int set_frames(kx_ctx* c, int64_t ldp, int64_t ldk, bool packed) {
    const int ny = c->n_sys;
    std::vector<MatFrame> f(ny);
    for (int y = 0; y < ny; ++y) {
        if (packed) {
            const int64_t n = c->sys_fn[y + 1] - c->sys_fn[y], f0 = c->sys_fn[y];
            // X(mu,nu) = X[mat_y + (mu - f0) * n + (nu - f0)]
            f[y].p0 = f[y].k0 = c->sys_mat[y] - f0 * (n + 1);
            f[y].ldp = f[y].ldk = (int32_t)n;
        } else {
            f[y].p0 = f[y].k0 = 0;
            f[y].ldp = (int32_t)ldp;
            f[y].ldk = (int32_t)ldk;
        }
    }
    if (!c->d_mframe) KX_CUDA(c, cudaMalloc(&c->d_mframe, sizeof(MatFrame) * ny));
    KX_CUDA(c, cudaMemcpyAsync(c->d_mframe, f.data(), sizeof(MatFrame) * ny, cudaMemcpyHostToDevice, c->stream));
    KX_CUDA(c, cudaStreamSynchronize(c->stream));
    c->packed = packed;
    return KX_OK;
}

int p_norms(kx_ctx* c, const double* P) {
    int64_t n2 = c->sp_total;
    cudaError_t e = cudaSuccess;
    if (!c->d_pq) {
        e = cudaMalloc(&c->d_pq, sizeof(double) * n2);
        if (e == cudaSuccess) e = cudaMalloc(&c->d_pnorm, sizeof(double) * n2);
        if (e == cudaSuccess) e = cudaMalloc(&c->d_plog, sizeof(float) * n2);
        if (e != cudaSuccess) return cuda_check(c, e, "p_norms alloc");
    }
    k_p_shell<<<(unsigned)((n2 + 255) / 256), 256, 0, c->stream>>>(c->d_sseg, c->n_sys, n2, c->d_tl, c->d_tfoff,
                                                                  c->d_mframe, P, c->d_pq, c->d_pnorm, c->d_plog);
    c->launches++;
    KX_TRY(build_pyramid(c, c->d_pq, c->d_sq_p, c->d_nrm_p));
    c->have_pq = true;
    return KX_OK;
}

// ===========================================================================
// Boys table
// ===========================================================================

// F_m(T_i), T_i = i / BOYS_DENS, m = 0..BOYS_M: the top order from its
// positive-term series e^{-T} sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)),
// the rest by downward recursion F_{m-1} = (2T F_m + e^{-T}) / (2m-1).
__global__ void k_boys_table(double* __restrict__ t64, float* __restrict__ t32, float2* __restrict__ tdw, int npts) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npts) return;
    double T = (double)i / BOYS_DENS;
    const int M = BOYS_M;
    double term = 1.0 / (2 * M + 1), sum = term;
    #pragma unroll 1
    for (int k = 1; k < 4000; ++k) {
        term *= 2.0 * T / (2 * M + 2 * k + 1);
        sum += term;
        if (term < 1e-19 * sum) break;
    }
    double e = exp(-T);
    double F[BOYS_M + 1];
    F[M] = e * sum;
    #pragma unroll 1
    for (int m = M; m > 0; --m) F[m - 1] = (2.0 * T * F[m] + e) / (2 * m - 1);
    #pragma unroll 1
    for (int m = 0; m <= M; ++m) {
        t64[(int64_t)i * (BOYS_M + 1) + m] = F[m];
        t32[(int64_t)i * BOYS32_ROW + m] = (float)F[m];
        const float hi = (float)F[m];
        tdw[(int64_t)i * (BOYS_M + 1) + m] = make_float2(hi, (float)(F[m] - (double)hi));
    }
    for (int m = M + 1; m < BOYS32_ROW; ++m) t32[(int64_t)i * BOYS32_ROW + m] = 0.f;
}

int boys_table(kx_ctx* c) {
    int npts = BOYS_NPTS;
    cudaError_t e = cudaMalloc(&c->d_boys64, sizeof(double) * npts * (BOYS_M + 1));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_boys32, sizeof(float) * npts * BOYS32_ROW);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_boysdw, sizeof(float2) * npts * (BOYS_M + 1));
    if (e != cudaSuccess) return cuda_check(c, e, "boys alloc");
    k_boys_table<<<(npts + 127) / 128, 128, 0, c->stream>>>(c->d_boys64, c->d_boys32, c->d_boysdw, npts);
    return KX_OK;
}

// ===========================================================================
// pair tables for the ERI kernels
// ===========================================================================

// significant(a,b): the pair can appear in a surviving shell quartet.  With
// the shell screen on, S_ab * Pmax * Smax <= tau implies every quartet
// through (a,b) is culled; the test is made against tau * (1 - 2^-40) so
// that the different rounding order of the quartet bound can never keep a
// quartet whose pair was dropped.  Pairs emptied by Eq. 4 (s2 = 0) never
// take part.
__global__ void k_pair_flags(const Seg* __restrict__ seg, int nseg, int64_t n2, const int32_t* __restrict__ tl,
                             const double* __restrict__ snorm, const double* __restrict__ s2, double tau,
                             const unsigned long long* __restrict__ mx, int screen, int cls,
                             int64_t* __restrict__ flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n2) return;
    // maxima of S and of the P shell-block norms (bit patterns, see k_max_reduce)
    const double smax = __longlong_as_double((long long)mx[0]), pmax = __longlong_as_double((long long)mx[1]);
    int a, b;
    seg_pair(seg, nseg, i, a, b);
    int ok = (tl[a] * 3 + tl[b] == cls) && s2[i] > 0.0;
    if (ok && screen) ok = __dmul_rn(__dmul_rn(snorm[i], pmax), smax) > tau * (1.0 - 0x1p-40);
    flag[i] = ok;
}

__global__ void k_pair_fill(const Seg* __restrict__ seg, int nseg, int64_t n2, int cls,
                            const int32_t* __restrict__ tl, const double* __restrict__ tctr,
                            const double* __restrict__ talpha, const int32_t* __restrict__ tfoff,
                            const MatFrame* __restrict__ mf, const int64_t* __restrict__ flag,
                            const int64_t* __restrict__ slot, int32_t* __restrict__ pairmap,
                            PairMeta* __restrict__ meta, double* __restrict__ d64, float* __restrict__ d32,
                            float2* __restrict__ ddw) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n2) return;
    const int y = seg_find(seg, nseg, i);
    const Seg sg = seg[y];
    const int a = sg.base + (int)((i - sg.off) / sg.n), b = sg.base + (int)((i - sg.off) % sg.n);
    if (tl[a] * 3 + tl[b] != cls) return;
    if (!flag[i]) {
        pairmap[i] = -1;
        return;
    }
    int64_t s = slot[i];
    pairmap[i] = (int32_t)s;
    int la = tl[a], lb = tl[b];
    const MatFrame f = mf[y];
    meta[s] = PairMeta{f.p0 + (int64_t)tfoff[b] * f.ldp, f.k0 + (int64_t)tfoff[a] * f.ldk, tfoff[a], tfoff[b],
                       f.ldp, f.ldk};
    double al = talpha[a], be = talpha[b], p = al + be;
    double A[3] = {tctr[3 * a], tctr[3 * a + 1], tctr[3 * a + 2]};
    double B[3] = {tctr[3 * b], tctr[3 * b + 1], tctr[3 * b + 2]};
    const int stride = pair_stride(la, lb), et = etab(la, lb);
    double* o = d64 + s * stride;
    float* o32 = d32 + s * PAIR32_STRIDE;
    double AB2 = 0.0;
    double E[45];
    o[0] = p;
    o32[P32_P] = (float)p;
    o32[P32_INV2P] = (float)(0.5 / p);
    for (int x = 0; x < 3; ++x) {
        double Px = (al * A[x] + be * B[x]) / p;
        o[1 + x] = Px;
        const float hi = (float)Px;
        o32[P32_PHI + x] = hi;
        o32[P32_PLO + x] = (float)(Px - (double)hi);
        o32[P32_PA + x] = (float)(Px - A[x]);
        o32[P32_PB + x] = (float)(Px - B[x]);
        AB2 += (A[x] - B[x]) * (A[x] - B[x]);
        hermite_e_1d(la, lb, Px - A[x], Px - B[x], 0.5 / p, E);
        for (int k = 0; k < et; ++k) o[5 + x * et + k] = E[k];
    }
    o[4] = norm_prim(al, la) * norm_prim(be, lb) * exp(-al * be / p * AB2);
    o32[P32_KAB] = (float)o[4];
    o32[15] = 0.f;
    if (stride > 5 + 3 * et) o[stride - 1] = 0.0;
    // the same record as double words (hi = nearest float, lo = remainder)
    if (ddw) {
        float2* od = ddw + s * stride;
        for (int k = 0; k < stride; ++k) {
            const double x = o[k];
            const float hi = (float)x;
            od[k] = make_float2(hi, (float)(x - (double)hi));
        }
    }
}

__global__ void k_max_reduce(const double* __restrict__ x, int64_t n, unsigned long long* __restrict__ out) {
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmax(m, x[i]);
    for (int d = 16; d > 0; d >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, d));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

static void pair_maxima(kx_ctx* c) {
    const int64_t n2 = c->sp_total;
    unsigned long long* d_mx = c->d_counters;   // two slots
    cudaMemsetAsync(d_mx, 0, 2 * sizeof(unsigned long long), c->stream);
    k_max_reduce<<<1024, 256, 0, c->stream>>>(c->d_snorm, n2, d_mx);
    k_max_reduce<<<1024, 256, 0, c->stream>>>(c->d_pnorm, n2, d_mx + 1);
    c->launches += 2;
}

// the double-word pair records of class cls, at the capacity of the FP64 table
static int reserve_pairdw(kx_ctx* c, int cls) {
    if (c->pairdw_cap[cls] >= c->pair_cap[cls] && c->d_pairdw[cls]) return KX_OK;
    cudaFree(c->d_pairdw[cls]);
    c->d_pairdw[cls] = nullptr;
    c->pairdw_cap[cls] = 0;
    const int stride = pair_stride(cls / 3, cls % 3);
    KX_CUDA(c, cudaMalloc(&c->d_pairdw[cls], sizeof(float2) * stride * std::max<int64_t>(c->pair_cap[cls], 1)));
    c->pairdw_cap[cls] = c->pair_cap[cls];
    return KX_OK;
}

int pair_tables(kx_ctx* c, double tau, bool screen, bool dw) {
    int64_t n2 = c->sp_total;
    pair_maxima(c);
    if (!c->d_pairmap) KX_CUDA(c, cudaMalloc(&c->d_pairmap, sizeof(int32_t) * n2));
    KX_TRY(grow(c, &c->d_scan, &c->scan_cap, (size_t)2 * n2 + 16));
    int64_t* flag = c->d_scan;
    int64_t* slot = c->d_scan + n2;
    unsigned g = (unsigned)((n2 + 255) / 256);
    for (int cls = 0; cls < NPAIRCLASS; ++cls) {
        int la = cls / 3, lb = cls % 3;
        k_pair_flags<<<g, 256, 0, c->stream>>>(c->d_sseg, c->n_sys, n2, c->d_tl, c->d_snorm, c->d_s2, tau,
                                               c->d_counters, screen ? 1 : 0, cls, flag);
        int64_t total = 0;
        KX_TRY(exclusive_scan(c, flag, slot, n2, &total));
        c->n_pairs[cls] = total;
        size_t need = (size_t)std::max<int64_t>(total, 1);
        if ((size_t)c->pair_cap[cls] < need) {
            cudaFree(c->d_pair64[cls]); cudaFree(c->d_pair32[cls]); cudaFree(c->d_pairmeta[cls]);
            c->d_pair64[cls] = nullptr; c->d_pair32[cls] = nullptr; c->d_pairmeta[cls] = nullptr;
            size_t cap = need + need / 8 + 16;
            int stride = pair_stride(la, lb);
            cudaError_t e = cudaMalloc(&c->d_pair64[cls], sizeof(double) * stride * cap);
            if (e == cudaSuccess) e = cudaMalloc(&c->d_pair32[cls], sizeof(float) * PAIR32_STRIDE * cap);
            if (e == cudaSuccess) e = cudaMalloc(&c->d_pairmeta[cls], sizeof(PairMeta) * cap);
            if (e != cudaSuccess) {
                c->pair_cap[cls] = 0;
                return cuda_check(c, e, "pair table alloc");
            }
            c->pair_cap[cls] = (int64_t)cap;
        }
        if (dw) KX_TRY(reserve_pairdw(c, cls));
        k_pair_fill<<<g, 256, 0, c->stream>>>(c->d_sseg, c->n_sys, n2, cls, c->d_tl, c->d_tctr, c->d_talpha,
                                              c->d_tfoff, c->d_mframe, flag, slot, c->d_pairmap, c->d_pairmeta[cls],
                                              c->d_pair64[cls], c->d_pair32[cls], dw ? c->d_pairdw[cls] : nullptr);
        c->launches += 2;
    }
    return KX_OK;
}

// Capture-safe: no host read-back.  The tables must already hold every pair
// of nonzero Schwarz factor (pair_tables(c, 0, false) reserves that); the
// slot bound of the class kernels is then the capacity.
int pair_tables_dev(kx_ctx* c, double tau, bool screen, bool dw) {
    int64_t n2 = c->sp_total;
    if (!c->d_pairmap || c->scan_cap < (size_t)2 * n2 + 16)
        return set_err(c, KX_ESTATE, "pair tables not reserved");
    pair_maxima(c);
    int64_t* flag = c->d_scan;
    int64_t* slot = c->d_scan + n2;
    unsigned g = (unsigned)((n2 + 255) / 256);
    for (int cls = 0; cls < NPAIRCLASS; ++cls) {
        k_pair_flags<<<g, 256, 0, c->stream>>>(c->d_sseg, c->n_sys, n2, c->d_tl, c->d_snorm, c->d_s2, tau,
                                               c->d_counters, screen ? 1 : 0, cls, flag);
        KX_TRY(exclusive_scan_dev(c, flag, slot, n2, nullptr, (int64_t*)(c->d_counters + 2)));
        c->n_pairs[cls] = c->pair_cap[cls];
        if (dw && (c->pairdw_cap[cls] < c->pair_cap[cls] || !c->d_pairdw[cls]))
            return set_err(c, KX_ESTATE, "double-word pair tables not reserved");
        k_pair_fill<<<g, 256, 0, c->stream>>>(c->d_sseg, c->n_sys, n2, cls, c->d_tl, c->d_tctr, c->d_talpha,
                                              c->d_tfoff, c->d_mframe, flag, slot, c->d_pairmap, c->d_pairmeta[cls],
                                              c->d_pair64[cls], c->d_pair32[cls], dw ? c->d_pairdw[cls] : nullptr);
        c->launches += 2;
    }
    return KX_OK;
}

// ===========================================================================
// FMA throughput probe
// ===========================================================================

// Eight independent multiply-add chains per thread; x <- x*a + b converges
// to b/(1-a), so the values stay finite for any iteration count.
template <typename R>
__global__ void __launch_bounds__(256) k_fma_probe(R* __restrict__ out, int iters, R a, R b) {
    R x0 = R(threadIdx.x) * R(1e-3), x1 = x0 + R(1), x2 = x0 + R(2), x3 = x0 + R(3);
    R x4 = x0 + R(4), x5 = x0 + R(5), x6 = x0 + R(6), x7 = x0 + R(7);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

// FP64 tensor-core (DMMA) chains: mma.sync m8n8k4 with FP64 operands, four
// independent accumulator tiles per warp; each instruction is 8*8*4
// multiply-adds of the warp.  a and b stay fixed, so the accumulators grow
// linearly and stay finite.
__global__ void __launch_bounds__(256) k_dmma_probe(double* __restrict__ out, int iters, double a, double b) {
    double c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = 0.0;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                         : "+d"(c[2 * k]), "+d"(c[2 * k + 1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += c[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Double-word FP32 multiply-add chains (kx_dw.cuh), eight independent
// chains per thread; x <- x * a + b converges, so the values stay finite.
// Counted as 2 FLOPs per double-word multiply-add (the FP64-equivalent
// rate of the double-word kernels).
__global__ void __launch_bounds__(256) k_dw_probe(float2* __restrict__ out, int iters, float ah, float al,
                                                  float bh, float bl) {
    const dw a(ah, al), b(bh, bl);
    dw x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = dw((float)(threadIdx.x + k) * 1e-3f, 0.f);
#pragma unroll 2
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = dw_fma(x[k], a, b);
    }
    dw s = x[0];
#pragma unroll
    for (int k = 1; k < 8; ++k) s = dw_add(s, x[k]);
    out[blockIdx.x * blockDim.x + threadIdx.x] = make_float2(s.hi, s.lo);
}

int peak_probe(int device, int precision, double* gflops) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        (void)cudaGetLastError();
        return KX_ECUDA;
    }
    const int blocks = prop.multiProcessorCount * 8, threads = 256;
    const int iters = precision == KX_FP64 ? 1 << 12
                      : precision == KX_PROBE_FP64_MMA ? 1 << 10
                      : precision == KX_PROBE_DW ? 1 << 14 : 1 << 17;
    void* out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) {
        (void)cudaGetLastError();
        return KX_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 6; ++rep) {
        cudaEventRecord(e0);
        if (precision == KX_FP64)
            k_fma_probe<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-6);
        else if (precision == KX_PROBE_FP64_MMA)
            k_dmma_probe<<<blocks, threads>>>((double*)out, iters, 1e-3, 1e-3);
        else if (precision == KX_PROBE_DW)
            k_dw_probe<<<blocks, threads>>>((float2*)out, iters, 0.9999f, 1e-11f, 1e-4f, 3e-12f);
        else
            k_fma_probe<float><<<blocks, threads>>>((float*)out, iters, 0.9999f, 1e-4f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        // FMA probes: 8 chains of one FMA per thread; DMMA: 4 instructions of
        // 256 multiply-adds per warp, i.e. 32 per thread
        const double per_thread = precision == KX_PROBE_FP64_MMA ? 4.0 * 256.0 / 32.0 : 8.0;
        const double flops = 2.0 * per_thread * iters * (double)blocks * threads;
        if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e9);
    }
    cudaError_t e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return KX_ECUDA;
    *gflops = best;
    return KX_OK;
}

}  // namespace kx
