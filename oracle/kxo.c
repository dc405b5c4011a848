/*
 * kxo.c -- plain FP64 CPU oracle for the screened exchange build.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test-suite, the smoke check and
 * the benchmark's CPU-baseline leg, never by the library.  Nothing here is
 * blocked, fused or reordered beyond what each definition states, so it can
 * be checked against the paper and the textbook recurrences by eye.
 *
 * What each part follows:
 *   kxo_boys             F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt: its
 *                        positive-term series for T < 30 with downward
 *                        recursion, and F_0 = (1/2) sqrt(pi/T) erf(sqrt T)
 *                        with upward recursion for T >= 30.
 *   kxo_eri              Obara-Saika vertical recursion (J. Chem. Phys. 84,
 *                        3963 (1986)) plus the Head-Gordon-Pople horizontal
 *                        recursion (J. Chem. Phys. 89, 5777 (1988)); the
 *                        paper's integral engine is the latter (Sec.
 *                        "Implementation and results").
 *   kxo_exchange_direct  the paper's Eq. 6 summed over every function.
 *   kxo_schwarz_sq       the diagonal integrals entering Eq. 8.
 *   kxo_overlap          the overlap test of Eq. 4.
 *   kxo_hilbert_*        the Hilbert-curve ordering of Sec. "Exchange as
 *                        hextree traversal" (Skilling, AIP Conf. Proc. 707,
 *                        381 (2004), transpose form, 3 axes x 10 bits).
 *   kxo_tree_build       the ragged bisection of Eq. 1.
 *   kxo_traverse         the recursion of Eq. 7 with the metric query of
 *                        Eq. 8, depth first.
 *   kxo_exchange_worklist the leaf contractions of Eq. 7 (and Eq. 6) over
 *                        the surviving leaf quartets.
 */
#include "kxo.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KXO_PI 3.14159265358979323846
#define LMAX 2
#define LPAIR (2 * LMAX)          /* 4  */
#define LQUART (4 * LMAX)         /* 8  */
#define NTRIP 35                  /* Cartesian triples with total <= 4 */

int kxo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Boys function                                                            */
/* ------------------------------------------------------------------------ */

void kxo_boys(int mmax, double T, double* F) {
    double e = exp(-T);
    if (T < 30.0) {
        /* F_m(T) = e^{-T} sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) */
        double term = 1.0 / (2 * mmax + 1);
        double sum = term;
        for (int k = 1; k < 2000; ++k) {
            term *= 2.0 * T / (2 * mmax + 2 * k + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        F[mmax] = e * sum;
        /* F_{m-1} = (2T F_m + e^{-T}) / (2m - 1) */
        for (int m = mmax; m > 0; --m) F[m - 1] = (2.0 * T * F[m] + e) / (2 * m - 1);
    } else {
        F[0] = 0.5 * sqrt(KXO_PI / T) * erf(sqrt(T));
        /* F_{m+1} = ((2m+1) F_m - e^{-T}) / (2T) */
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0 * T);
    }
}

/* ------------------------------------------------------------------------ */
/* Cartesian components                                                     */
/* ------------------------------------------------------------------------ */

static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* idx-th component of angular momentum l, x power descending then y. */
static void cart(int l, int idx, int c[3]) {
    int n = 0;
    for (int i = l; i >= 0; --i)
        for (int j = l - i; j >= 0; --j) {
            if (n == idx) { c[0] = i; c[1] = j; c[2] = l - i - j; return; }
            ++n;
        }
}

static double norm_prim(double a, int l) {
    double df = (l == 2) ? 3.0 : 1.0;                /* (2l-1)!! for l <= 2 */
    return pow(2.0 * a / KXO_PI, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(df);
}

/* compact index of a Cartesian triple with total <= 4 */
static int trip_index[LPAIR + 1][LPAIR + 1][LPAIR + 1];
static int trip_list[NTRIP][3];
static int trip_ready = 0;

static void trip_init(void) {
    if (trip_ready) return;
    int n = 0;
    for (int L = 0; L <= LPAIR; ++L)
        for (int k = 0; k < ncart(L); ++k) {
            int c[3];
            cart(L, k, c);
            trip_index[c[0]][c[1]][c[2]] = n;
            trip_list[n][0] = c[0]; trip_list[n][1] = c[1]; trip_list[n][2] = c[2];
            ++n;
        }
    trip_ready = 1;
}

static int tidx(const int c[3]) { return trip_index[c[0]][c[1]][c[2]]; }
static int ttot(const int c[3]) { return c[0] + c[1] + c[2]; }
static int first_dir(const int c[3]) { return c[0] > 0 ? 0 : (c[1] > 0 ? 1 : 2); }

/* ------------------------------------------------------------------------ */
/* Obara-Saika / Head-Gordon-Pople ERIs                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    double v[LQUART + 1][NTRIP][NTRIP];   /* [e 0 | f 0]^(m) */
    double AB[3], CD[3];
} vrr_t;

/* (a b | f 0) from the m = 0 table by (a, b+1_i| = (a+1_i, b| + AB_i (a b| */
static double hrr_bra(const vrr_t* V, const int a[3], const int b[3], int f) {
    if (ttot(b) == 0) return V->v[0][tidx(a)][f];
    int i = first_dir(b);
    int a1[3] = {a[0], a[1], a[2]}, b1[3] = {b[0], b[1], b[2]};
    a1[i] += 1;
    b1[i] -= 1;
    return hrr_bra(V, a1, b1, f) + V->AB[i] * hrr_bra(V, a, b1, f);
}

/* (a b | c d) by |c, d+1_i) = |c+1_i, d) + CD_i |c d) */
static double hrr_ket(const vrr_t* V, const int a[3], const int b[3], const int c[3], const int d[3]) {
    if (ttot(d) == 0) return hrr_bra(V, a, b, tidx(c));
    int i = first_dir(d);
    int c1[3] = {c[0], c[1], c[2]}, d1[3] = {d[0], d[1], d[2]};
    c1[i] += 1;
    d1[i] -= 1;
    return hrr_ket(V, a, b, c1, d1) + V->CD[i] * hrr_ket(V, a, b, c, d1);
}

void kxo_eri(const double* A, double aa, int la, const double* B, double bb, int lb,
             const double* C, double cc, int lc, const double* D, double dd, int ld,
             double* out) {
    trip_init();
    vrr_t* V = (vrr_t*)malloc(sizeof(vrr_t));
    double p = aa + bb, q = cc + dd;
    double P[3], Q[3], W[3], AB2 = 0.0, CD2 = 0.0, PQ2 = 0.0;
    for (int i = 0; i < 3; ++i) {
        P[i] = (aa * A[i] + bb * B[i]) / p;
        Q[i] = (cc * C[i] + dd * D[i]) / q;
        V->AB[i] = A[i] - B[i];
        V->CD[i] = C[i] - D[i];
        AB2 += V->AB[i] * V->AB[i];
        CD2 += V->CD[i] * V->CD[i];
    }
    for (int i = 0; i < 3; ++i) {
        PQ2 += (P[i] - Q[i]) * (P[i] - Q[i]);
        W[i] = (p * P[i] + q * Q[i]) / (p + q);
    }
    double rho = p * q / (p + q);
    double T = rho * PQ2;
    int Lab = la + lb, Lcd = lc + ld, L = Lab + Lcd;
    double F[LQUART + 1];
    kxo_boys(L, T, F);
    double pref = 2.0 * pow(KXO_PI, 2.5) / (p * q * sqrt(p + q))
                  * exp(-aa * bb / p * AB2) * exp(-cc * dd / q * CD2);

    /* [0 0|0 0]^(m) */
    for (int m = 0; m <= L; ++m) V->v[m][0][0] = pref * F[m];

    /* electron 1: [e+1_i 0|0 0]^(m) */
    for (int e = 1; e < NTRIP; ++e) {
        const int* et = trip_list[e];
        int ne = ttot(et);
        if (ne > Lab) break;
        int i = first_dir(et);
        int em[3] = {et[0], et[1], et[2]};
        em[i] -= 1;
        int iem = tidx(em);
        for (int m = 0; m <= L - ne; ++m) {
            double v = (P[i] - A[i]) * V->v[m][iem][0] + (W[i] - P[i]) * V->v[m + 1][iem][0];
            if (em[i] > 0) {
                int emm[3] = {em[0], em[1], em[2]};
                emm[i] -= 1;
                int iemm = tidx(emm);
                v += em[i] / (2.0 * p) * (V->v[m][iemm][0] - rho / p * V->v[m + 1][iemm][0]);
            }
            V->v[m][e][0] = v;
        }
    }

    /* electron 2: [e 0|f+1_i 0]^(m) */
    for (int f = 1; f < NTRIP; ++f) {
        const int* ft = trip_list[f];
        int nf = ttot(ft);
        if (nf > Lcd) break;
        int i = first_dir(ft);
        int fm[3] = {ft[0], ft[1], ft[2]};
        fm[i] -= 1;
        int ifm = tidx(fm);
        for (int e = 0; e < NTRIP; ++e) {
            const int* et = trip_list[e];
            int ne = ttot(et);
            if (ne > Lab) break;
            for (int m = 0; m <= L - ne - nf; ++m) {
                double v = (Q[i] - C[i]) * V->v[m][e][ifm] + (W[i] - Q[i]) * V->v[m + 1][e][ifm];
                if (fm[i] > 0) {
                    int fmm[3] = {fm[0], fm[1], fm[2]};
                    fmm[i] -= 1;
                    int ifmm = tidx(fmm);
                    v += fm[i] / (2.0 * q) * (V->v[m][e][ifmm] - rho / q * V->v[m + 1][e][ifmm]);
                }
                if (et[i] > 0) {
                    int e1[3] = {et[0], et[1], et[2]};
                    e1[i] -= 1;
                    v += et[i] / (2.0 * (p + q)) * V->v[m + 1][tidx(e1)][ifm];
                }
                V->v[m][e][f] = v;
            }
        }
    }

    double nrm = norm_prim(aa, la) * norm_prim(bb, lb) * norm_prim(cc, lc) * norm_prim(dd, ld);
    int na = ncart(la), nb = ncart(lb), nc = ncart(lc), nd = ncart(ld);
    for (int i = 0; i < na; ++i) {
        int ca[3];
        cart(la, i, ca);
        for (int j = 0; j < nb; ++j) {
            int cb[3];
            cart(lb, j, cb);
            for (int k = 0; k < nc; ++k) {
                int cc3[3];
                cart(lc, k, cc3);
                for (int l = 0; l < nd; ++l) {
                    int cd3[3];
                    cart(ld, l, cd3);
                    out[((i * nb + j) * nc + k) * nd + l] = nrm * hrr_ket(V, ca, cb, cc3, cd3);
                }
            }
        }
    }
    free(V);
}

/* ------------------------------------------------------------------------ */
/* overlap (Eq. 4)                                                          */
/* ------------------------------------------------------------------------ */

/* 1D Obara-Saika overlap S_ij, i <= la, j <= lb */
static void overlap1d(double XPA, double XPB, double p, double s00, int la, int lb,
                      double S[LMAX + 1][LMAX + 1]) {
    S[0][0] = s00;
    for (int i = 0; i <= la; ++i)
        for (int j = 0; j <= lb; ++j) {
            if (i == 0 && j == 0) continue;
            double v;
            if (i > 0) {
                v = XPA * S[i - 1][j];
                if (i > 1) v += (i - 1) / (2.0 * p) * S[i - 2][j];
                if (j > 0) v += j / (2.0 * p) * S[i - 1][j - 1];
            } else {
                v = XPB * S[i][j - 1];
                if (j > 1) v += (j - 1) / (2.0 * p) * S[i][j - 2];
            }
            S[i][j] = v;
        }
}

void kxo_overlap(const double* A, double a, int la, const double* B, double b, int lb,
                 double* out) {
    double p = a + b, mu = a * b / p;
    double S[3][LMAX + 1][LMAX + 1];
    for (int x = 0; x < 3; ++x) {
        double Px = (a * A[x] + b * B[x]) / p;
        double X = A[x] - B[x];
        overlap1d(Px - A[x], Px - B[x], p, sqrt(KXO_PI / p) * exp(-mu * X * X), la, lb, S[x]);
    }
    double nrm = norm_prim(a, la) * norm_prim(b, lb);
    for (int i = 0; i < ncart(la); ++i) {
        int ca[3];
        cart(la, i, ca);
        for (int j = 0; j < ncart(lb); ++j) {
            int cb[3];
            cart(lb, j, cb);
            out[i * ncart(lb) + j] =
                nrm * S[0][ca[0]][cb[0]] * S[1][ca[1]][cb[1]] * S[2][ca[2]][cb[2]];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* basis helpers                                                            */
/* ------------------------------------------------------------------------ */

static int64_t* fn_offsets(const kxo_basis* bs) {
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (bs->n_shell + 1));
    off[0] = 0;
    for (int s = 0; s < bs->n_shell; ++s) off[s + 1] = off[s] + ncart(bs->l[s]);
    return off;
}

static void shell_eri(const kxo_basis* bs, int a, int b, int c, int d, double* out) {
    kxo_eri(bs->center + 3 * a, bs->alpha[a], bs->l[a], bs->center + 3 * b, bs->alpha[b], bs->l[b],
            bs->center + 3 * c, bs->alpha[c], bs->l[c], bs->center + 3 * d, bs->alpha[d], bs->l[d],
            out);
}

/* K_{mu nu} += sum_{lam in b, sig in d} (mu lam|nu sig) P_{lam sig} */
static void contract(const kxo_basis* bs, const int64_t* off, int64_t N, int a, int b, int c, int d,
                     const double* eri, const double* Pm, double* K) {
    int na = ncart(bs->l[a]), nb = ncart(bs->l[b]), nc = ncart(bs->l[c]), nd = ncart(bs->l[d]);
    for (int i = 0; i < na; ++i)
        for (int k = 0; k < nc; ++k) {
            double acc = 0.0;
            for (int j = 0; j < nb; ++j)
                for (int l = 0; l < nd; ++l)
                    acc += eri[((i * nb + j) * nc + k) * nd + l] * Pm[(off[b] + j) * N + off[d] + l];
            K[(off[a] + i) * N + off[c] + k] += acc;
        }
}

void kxo_exchange_direct(const kxo_basis* bs, const double* Pm, double* K) {
    int64_t* off = fn_offsets(bs);
    int64_t N = off[bs->n_shell];
    int ns = bs->n_shell;
    memset(K, 0, sizeof(double) * N * N);
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < ns; ++a) {
        double* buf = (double*)malloc(sizeof(double) * 1296);
        for (int c = 0; c < ns; ++c)
            for (int b = 0; b < ns; ++b)
                for (int d = 0; d < ns; ++d) {
                    shell_eri(bs, a, b, c, d, buf);
                    contract(bs, off, N, a, b, c, d, buf, Pm, K);
                }
        free(buf);
    }
    free(off);
}

void kxo_schwarz_sq(const kxo_basis* bs, double tau_ovlp, double* s2) {
    int ns = bs->n_shell;
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < ns; ++a) {
        double* buf = (double*)malloc(sizeof(double) * 1296);
        double ov[36];
        for (int b = 0; b < ns; ++b) {
            int na = ncart(bs->l[a]), nb = ncart(bs->l[b]);
            int pruned = 0;
            if (tau_ovlp > 0.0) {
                kxo_overlap(bs->center + 3 * a, bs->alpha[a], bs->l[a],
                            bs->center + 3 * b, bs->alpha[b], bs->l[b], ov);
                pruned = 1;
                for (int k = 0; k < na * nb; ++k)
                    if (fabs(ov[k]) >= tau_ovlp) pruned = 0;
            }
            double s = 0.0;
            if (!pruned) {
                shell_eri(bs, a, b, a, b, buf);
                for (int i = 0; i < na; ++i)
                    for (int j = 0; j < nb; ++j) s += buf[((i * nb + j) * na + i) * nb + j];
            }
            s2[(int64_t)a * ns + b] = s;
        }
        free(buf);
    }
}

void kxo_pblock_sq(const kxo_basis* bs, const double* Pm, double* out) {
    int64_t* off = fn_offsets(bs);
    int64_t N = off[bs->n_shell];
    int ns = bs->n_shell;
    for (int b = 0; b < ns; ++b)
        for (int d = 0; d < ns; ++d) {
            double s = 0.0;
            for (int64_t i = off[b]; i < off[b + 1]; ++i)
                for (int64_t j = off[d]; j < off[d + 1]; ++j) s += Pm[i * N + j] * Pm[i * N + j];
            out[(int64_t)b * ns + d] = s;
        }
    free(off);
}

/* ------------------------------------------------------------------------ */
/* Hilbert order                                                            */
/* ------------------------------------------------------------------------ */

/* Skilling's method: turn the axes into the "transposed" Hilbert index by
 * undoing the per-level inversions/exchanges from the top bit down, Gray
 * code the result, then read the key by interleaving bits across axes
 * (axis 0 most significant inside each level). */
void kxo_key_of_cell(const int32_t* q3, int bits, int64_t* key) {
    uint32_t X[3] = {(uint32_t)q3[0], (uint32_t)q3[1], (uint32_t)q3[2]};
    uint32_t top = 1u << (bits - 1);
    for (uint32_t Q = top; Q > 1; Q >>= 1) {
        uint32_t low = Q - 1;
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
    for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = top; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    int64_t k = 0;
    for (int bit = bits - 1; bit >= 0; --bit)
        for (int i = 0; i < 3; ++i) k = (k << 1) | ((X[i] >> bit) & 1u);
    *key = k;
}

/* Atom centres quantised on a 1024^3 grid over the cubic bounding box:
 * q = floor(((x - lo) / span) * 1023 + 0.5). */
void kxo_hilbert_keys(int n_atom, const double* xyz, int64_t* key) {
    double lo[3], hi[3];
    for (int x = 0; x < 3; ++x) { lo[x] = xyz[x]; hi[x] = xyz[x]; }
    for (int a = 0; a < n_atom; ++a)
        for (int x = 0; x < 3; ++x) {
            if (xyz[3 * a + x] < lo[x]) lo[x] = xyz[3 * a + x];
            if (xyz[3 * a + x] > hi[x]) hi[x] = xyz[3 * a + x];
        }
    double span = 0.0;
    for (int x = 0; x < 3; ++x)
        if (hi[x] - lo[x] > span) span = hi[x] - lo[x];
    for (int a = 0; a < n_atom; ++a) {
        int32_t q[3];
        for (int x = 0; x < 3; ++x) {
            if (span > 0.0) {
                double t = (xyz[3 * a + x] - lo[x]) / span;
                double u = t * 1023.0;
                q[x] = (int32_t)floor(u + 0.5);
                if (q[x] < 0) q[x] = 0;
                if (q[x] > 1023) q[x] = 1023;
            } else {
                q[x] = 0;
            }
        }
        kxo_key_of_cell(q, 10, &key[a]);
    }
}

void kxo_shell_order(int n_atom, const double* xyz, int n_shell, const int32_t* shell_atom,
                     int32_t* perm) {
    int64_t* key = (int64_t*)malloc(sizeof(int64_t) * n_atom);
    kxo_hilbert_keys(n_atom, xyz, key);
    /* atom rank: by (key, input index) -- a plain insertion sort */
    int* order = (int*)malloc(sizeof(int) * n_atom);
    for (int i = 0; i < n_atom; ++i) order[i] = i;
    for (int i = 1; i < n_atom; ++i) {
        int v = order[i], j = i - 1;
        while (j >= 0 && (key[order[j]] > key[v] || (key[order[j]] == key[v] && order[j] > v))) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = v;
    }
    /* shells atom-major in that order, input order inside an atom */
    int n = 0;
    for (int r = 0; r < n_atom; ++r)
        for (int s = 0; s < n_shell; ++s)
            if (shell_atom[s] == order[r]) perm[n++] = s;
    free(order);
    free(key);
}

/* ------------------------------------------------------------------------ */
/* ragged bisection (Eq. 1)                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
    const int64_t* pre;
    int leaf_max;
    int n;
    int32_t *lo, *hi, *c0, *c1, *dep;
} tree_builder;

static int tree_rec(tree_builder* tb, int lo, int hi, int depth) {
    int id = tb->n++;
    tb->lo[id] = lo;
    tb->hi[id] = hi;
    tb->dep[id] = depth;
    int64_t nfn = tb->pre[hi] - tb->pre[lo];
    if (nfn <= tb->leaf_max || hi - lo == 1) {
        tb->c0[id] = -1;
        tb->c1[id] = -1;
        return id;
    }
    /* the shell boundary s in (lo, hi) nearest the function-count midpoint,
     * the lower one on a tie: minimise |2 pre[s] - pre[lo] - pre[hi]| */
    int best = lo + 1;
    int64_t bestd = -1;
    for (int s = lo + 1; s < hi; ++s) {
        int64_t dlt = 2 * tb->pre[s] - tb->pre[lo] - tb->pre[hi];
        if (dlt < 0) dlt = -dlt;
        if (bestd < 0 || dlt < bestd) { bestd = dlt; best = s; }
    }
    int c0 = tree_rec(tb, lo, best, depth + 1);
    int c1 = tree_rec(tb, best, hi, depth + 1);
    tb->c0[id] = c0;
    tb->c1[id] = c1;
    return id;
}

int kxo_tree_build(int n_shell, const int32_t* nfn_tree, int leaf_max, int32_t* lo, int32_t* hi,
                   int32_t* child0, int32_t* child1, int32_t* depth) {
    if (n_shell <= 0) return 0;
    int64_t* pre = (int64_t*)malloc(sizeof(int64_t) * (n_shell + 1));
    pre[0] = 0;
    for (int s = 0; s < n_shell; ++s) pre[s + 1] = pre[s] + nfn_tree[s];
    tree_builder tb = {pre, leaf_max, 0, lo, hi, child0, child1, depth};
    tree_rec(&tb, 0, n_shell, 0);
    free(pre);
    return tb.n;
}

/* ------------------------------------------------------------------------ */
/* block norms and the traversal (Eqs. 7, 8)                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    const kxo_basis* bs;
    const double* P;
    const int32_t* perm;
    const int32_t *lo, *hi, *c0, *c1;
    int n_node;
    const double* s2;
    int64_t* off;           /* user function offsets */
    int64_t N;
    double* sq_s;           /* memo: squared ||Q_AB||_F, -1 = unknown */
    double* sq_p;           /* memo: squared ||P_BD||_F */
    int* leaf_ord;          /* node -> leaf ordinal or -1 */
    char* row_mark;         /* tree position -> row selected */
    int n_rows;
    double tau;
    int32_t* out;
    int64_t cap, n_out;
} trav_t;

/* ||Q_AB||_F^2 = sum_{a in A} sum_{b in B} sum_{mu in a, lam in b} (mu lam|mu lam) */
static double node_sq_s(trav_t* t, int A, int B) {
    double* m = &t->sq_s[(int64_t)A * t->n_node + B];
    if (*m >= 0.0) return *m;
    double s = 0.0;
    int ns = t->bs->n_shell;
    for (int a = t->lo[A]; a < t->hi[A]; ++a)
        for (int b = t->lo[B]; b < t->hi[B]; ++b) s += t->s2[(int64_t)t->perm[a] * ns + t->perm[b]];
    *m = s;
    return s;
}

/* ||P_BD||_F^2 = sum over the functions of the block, tree order */
static double node_sq_p(trav_t* t, int B, int D) {
    double* m = &t->sq_p[(int64_t)B * t->n_node + D];
    if (*m >= 0.0) return *m;
    double s = 0.0;
    for (int b = t->lo[B]; b < t->hi[B]; ++b) {
        int ub = t->perm[b];
        for (int64_t i = t->off[ub]; i < t->off[ub + 1]; ++i)
            for (int d = t->lo[D]; d < t->hi[D]; ++d) {
                int ud = t->perm[d];
                for (int64_t j = t->off[ud]; j < t->off[ud + 1]; ++j) {
                    double v = t->P[i * t->N + j];
                    s += v * v;
                }
            }
    }
    *m = s;
    return s;
}

/* Eq. 8: (||Q_AB|| * ||P_BD||) * ||Q_CD||, no fused multiply-add */
static double task_bound(trav_t* t, int A, int B, int C, int D) {
    double x = sqrt(node_sq_s(t, A, B));
    double y = sqrt(node_sq_p(t, B, D));
    double z = sqrt(node_sq_s(t, C, D));
    volatile double xy = x * y;
    return xy * z;
}

static int node_has_row(trav_t* t, int A) {
    if (t->n_rows == 0) return 1;
    for (int a = t->lo[A]; a < t->hi[A]; ++a)
        if (t->row_mark[a]) return 1;
    return 0;
}

/* One task of Eq. 7: cull by Eq. 8, else recurse into every combination of
 * the children of the non-leaf indices (a leaf stands for itself). */
static void visit(trav_t* t, int A, int B, int C, int D) {
    if (!node_has_row(t, A)) return;
    double beta = task_bound(t, A, B, C, D);
    if (!(beta > t->tau)) return;
    int isleaf[4] = {t->c0[A] < 0, t->c0[B] < 0, t->c0[C] < 0, t->c0[D] < 0};
    if (isleaf[0] && isleaf[1] && isleaf[2] && isleaf[3]) {
        if (t->n_out < t->cap) {
            int32_t* o = t->out + 4 * t->n_out;
            o[0] = t->leaf_ord[A];
            o[1] = t->leaf_ord[B];
            o[2] = t->leaf_ord[C];
            o[3] = t->leaf_ord[D];
        }
        t->n_out++;
        return;
    }
    int kidsA[2], kidsB[2], kidsC[2], kidsD[2];
    int nA = isleaf[0] ? 1 : 2, nB = isleaf[1] ? 1 : 2, nC = isleaf[2] ? 1 : 2, nD = isleaf[3] ? 1 : 2;
    kidsA[0] = isleaf[0] ? A : t->c0[A]; kidsA[1] = t->c1[A];
    kidsB[0] = isleaf[1] ? B : t->c0[B]; kidsB[1] = t->c1[B];
    kidsC[0] = isleaf[2] ? C : t->c0[C]; kidsC[1] = t->c1[C];
    kidsD[0] = isleaf[3] ? D : t->c0[D]; kidsD[1] = t->c1[D];
    for (int i = 0; i < nA; ++i)
        for (int j = 0; j < nB; ++j)
            for (int k = 0; k < nC; ++k)
                for (int l = 0; l < nD; ++l) visit(t, kidsA[i], kidsB[j], kidsC[k], kidsD[l]);
}

static int trav_init(trav_t* t, const kxo_basis* bs, const double* P, const int32_t* perm, int n_node,
                     const int32_t* lo, const int32_t* hi, const int32_t* c0, const int32_t* c1,
                     const double* s2, double tau, const int32_t* row_shell, int n_rows) {
    memset(t, 0, sizeof(*t));
    t->bs = bs; t->P = P; t->perm = perm; t->lo = lo; t->hi = hi; t->c0 = c0; t->c1 = c1;
    t->n_node = n_node; t->s2 = s2; t->tau = tau;
    t->off = fn_offsets(bs);
    t->N = t->off[bs->n_shell];
    size_t nn = (size_t)n_node * n_node;
    t->sq_s = (double*)malloc(sizeof(double) * nn);
    t->sq_p = (double*)malloc(sizeof(double) * nn);
    t->leaf_ord = (int*)malloc(sizeof(int) * n_node);
    t->row_mark = (char*)calloc(bs->n_shell, 1);
    if (!t->sq_s || !t->sq_p || !t->leaf_ord || !t->row_mark) return -1;
    for (size_t i = 0; i < nn; ++i) { t->sq_s[i] = -1.0; t->sq_p[i] = -1.0; }
    /* leaf ordinals left to right = by ascending lo */
    int nl = 0;
    for (int s = 0; s < bs->n_shell; ++s)
        for (int v = 0; v < n_node; ++v)
            if (c0[v] < 0 && lo[v] == s) t->leaf_ord[v] = nl++;
    for (int v = 0; v < n_node; ++v)
        if (c0[v] >= 0) t->leaf_ord[v] = -1;
    t->n_rows = n_rows;
    if (n_rows > 0) {
        for (int r = 0; r < n_rows; ++r)
            for (int s = 0; s < bs->n_shell; ++s)
                if (perm[s] == row_shell[r]) t->row_mark[s] = 1;
    }
    return 0;
}

static void trav_free(trav_t* t) {
    free(t->off); free(t->sq_s); free(t->sq_p); free(t->leaf_ord); free(t->row_mark);
}

int64_t kxo_traverse(const kxo_basis* bs, const double* P, const int32_t* perm, int n_node,
                     const int32_t* lo, const int32_t* hi, const int32_t* child0, const int32_t* child1,
                     const double* s2, double tau, const int32_t* row_shell, int n_rows, int32_t* out,
                     int64_t cap) {
    trav_t t;
    if (trav_init(&t, bs, P, perm, n_node, lo, hi, child0, child1, s2, tau, row_shell, n_rows)) {
        trav_free(&t);
        return -1;
    }
    t.out = out;
    t.cap = cap;
    visit(&t, 0, 0, 0, 0);
    int64_t n = t.n_out;
    trav_free(&t);
    return n;
}

int64_t kxo_leaf_bruteforce(const kxo_basis* bs, const double* P, const int32_t* perm, int n_node,
                            const int32_t* lo, const int32_t* hi, const int32_t* child0,
                            const double* s2, double tau, int32_t* out, int64_t cap,
                            double* beta_out) {
    trav_t t;
    if (trav_init(&t, bs, P, perm, n_node, lo, hi, child0, child0, s2, tau, NULL, 0)) {
        trav_free(&t);
        return -1;
    }
    int nl = 0;
    int* leaf_node = (int*)malloc(sizeof(int) * n_node);
    for (int v = 0; v < n_node; ++v)
        if (child0[v] < 0) leaf_node[t.leaf_ord[v]] = v, ++nl;
    int64_t n = 0;
    for (int A = 0; A < nl; ++A)
        for (int B = 0; B < nl; ++B)
            for (int C = 0; C < nl; ++C)
                for (int D = 0; D < nl; ++D) {
                    double beta = task_bound(&t, leaf_node[A], leaf_node[B], leaf_node[C], leaf_node[D]);
                    if (beta > tau) {
                        if (n < cap) {
                            out[4 * n] = A; out[4 * n + 1] = B; out[4 * n + 2] = C; out[4 * n + 3] = D;
                            if (beta_out) beta_out[n] = beta;
                        }
                        ++n;
                    }
                }
    free(leaf_node);
    trav_free(&t);
    return n;
}

/* ------------------------------------------------------------------------ */
/* leaf contractions                                                        */
/* ------------------------------------------------------------------------ */

static int cmp_first(const void* x, const void* y) {
    const int64_t* a = (const int64_t*)x;
    const int64_t* b = (const int64_t*)y;
    return (a[0] > b[0]) - (a[0] < b[0]);
}

int64_t kxo_exchange_worklist(const kxo_basis* bs, const double* Pm, const int32_t* perm, int n_node,
                              const int32_t* lo, const int32_t* hi, const int32_t* child0,
                              const double* s2, double tau, int shell_screen, const int32_t* work,
                              int64_t n_work, const int32_t* row_shell, int n_rows, double* K) {
    int64_t* off = fn_offsets(bs);
    int64_t N = off[bs->n_shell];
    int ns = bs->n_shell;
    memset(K, 0, sizeof(double) * N * N);
    /* leaf ordinal -> node */
    int nl = 0;
    int* leaf_node = (int*)malloc(sizeof(int) * n_node);
    for (int s = 0; s < ns; ++s)
        for (int v = 0; v < n_node; ++v)
            if (child0[v] < 0 && lo[v] == s) leaf_node[nl++] = v;
    char* row_mark = (char*)calloc(ns, 1);
    for (int r = 0; r < n_rows; ++r) row_mark[row_shell[r]] = 1;
    /* ||P_bd||_F per shell pair (user order) */
    double* pq = (double*)malloc(sizeof(double) * (size_t)ns * ns);
    kxo_pblock_sq(bs, Pm, pq);
    /* group the worklist by (A, C): one thread owns the K block of a group */
    int64_t* idx = (int64_t*)malloc(sizeof(int64_t) * 2 * (n_work > 0 ? n_work : 1));
    for (int64_t w = 0; w < n_work; ++w) {
        idx[2 * w] = (int64_t)work[4 * w] * nl + work[4 * w + 2];
        idx[2 * w + 1] = w;
    }
    qsort(idx, n_work, 2 * sizeof(int64_t), cmp_first);
    int64_t n_grp = 0;
    int64_t* grp = (int64_t*)malloc(sizeof(int64_t) * (n_work + 1));
    for (int64_t w = 0; w < n_work; ++w)
        if (w == 0 || idx[2 * w] != idx[2 * w - 2]) grp[n_grp++] = w;
    grp[n_grp] = n_work;
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total)
    for (int64_t g = 0; g < n_grp; ++g) {
        double* buf = (double*)malloc(sizeof(double) * 1296);
        for (int64_t s = grp[g]; s < grp[g + 1]; ++s) {
            const int32_t* q = work + 4 * idx[2 * s + 1];
            int nA = leaf_node[q[0]], nB = leaf_node[q[1]], nC = leaf_node[q[2]], nD = leaf_node[q[3]];
            for (int ta = lo[nA]; ta < hi[nA]; ++ta) {
                int a = perm[ta];
                if (n_rows > 0 && !row_mark[a]) continue;
                for (int tc = lo[nC]; tc < hi[nC]; ++tc) {
                    int c = perm[tc];
                    for (int tb = lo[nB]; tb < hi[nB]; ++tb) {
                        int b = perm[tb];
                        for (int td = lo[nD]; td < hi[nD]; ++td) {
                            int d = perm[td];
                            if (shell_screen) {
                                /* Eq. 8 applied to the single-shell blocks */
                                double x = sqrt(s2[(int64_t)a * ns + b]);
                                double y = sqrt(pq[(int64_t)b * ns + d]);
                                double z = sqrt(s2[(int64_t)c * ns + d]);
                                volatile double xy = x * y;
                                double beta = xy * z;
                                if (!(beta > tau)) continue;
                            }
                            shell_eri(bs, a, b, c, d, buf);
                            contract(bs, off, N, a, b, c, d, buf, Pm, K);
                            total += 1;
                        }
                    }
                }
            }
        }
        free(buf);
    }
    free(grp); free(idx); free(pq); free(row_mark); free(leaf_node); free(off);
    return total;
}
