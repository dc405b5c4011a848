/*
 * kxo.h -- plain FP64 CPU oracle for the screened Fock exchange build of
 * Challacombe & Bock, "An N-Body Solution to the Problem of Fock Exchange".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no source
 * with the CUDA library (no headers, helpers, tables or constants).
 *
 * Conventions (shared by contract with the CUDA library, restated here):
 *   - uncontracted Cartesian Gaussian shells, one primitive each, l <= 2;
 *   - components ordered with the x power descending (p: x,y,z;
 *     d: xx,xy,xz,yy,yz,zz);
 *   - every component of a shell carries
 *     N(a,l) = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!);
 *   - K_{mu nu} = sum_{lambda sigma} (mu lambda|nu sigma) P_{lambda sigma}
 *     (the paper's Eq. 6 without its -1/2, indices renamed);
 *   - all matrices dense, row-major, in user function order.
 */
#ifndef KXO_H
#define KXO_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n_shell;
    const double* center;  /* [n_shell*3] shell centres, bohr */
    const int32_t* l;      /* [n_shell] angular momentum 0..2 */
    const double* alpha;   /* [n_shell] exponent, bohr^-2 */
} kxo_basis;

/* Boys function F_m(T), m = 0..mmax (mmax <= 16). */
void kxo_boys(int mmax, double T, double* F);

/* Normalised primitive shell-quartet ERI block (ab|cd), layout
 * out[((i*nb + j)*nc + k)*nd + l]. */
void kxo_eri(const double* A, double a, int la, const double* B, double b, int lb,
             const double* C, double c, int lc, const double* D, double d, int ld,
             double* out);

/* Normalised overlap block (a|b), out[i*nb + j]. */
void kxo_overlap(const double* A, double a, int la, const double* B, double b, int lb,
                 double* out);

/* Unscreened exchange by its definition (every shell quartet). */
void kxo_exchange_direct(const kxo_basis* bs, const double* P, double* K);

/* Shell-pair squared Schwarz norms s2[a*n+b] = sum_{mu in a, lam in b}
 * (mu lam|mu lam); pairs whose every overlap is below tau_ovlp (Eq. 4)
 * get 0 when tau_ovlp > 0. */
void kxo_schwarz_sq(const kxo_basis* bs, double tau_ovlp, double* s2);

/* Shell-block squared Frobenius norms of P: out[b*n+d]. */
void kxo_pblock_sq(const kxo_basis* bs, const double* P, double* out);

/* Hilbert key (10 bits per axis, 30-bit key) of every atom, and the
 * resulting shell order perm[tree position] = user shell index. */
void kxo_hilbert_keys(int n_atom, const double* xyz, int64_t* key);
void kxo_key_of_cell(const int32_t* q3, int bits, int64_t* key);
void kxo_shell_order(int n_atom, const double* xyz, int n_shell,
                     const int32_t* shell_atom, int32_t* perm);

/* Ragged bisection of tree-ordered shells (Eq. 1).  Arrays of capacity
 * 2*n_shell; returns the node count.  child0/child1 = -1 for a leaf. */
int kxo_tree_build(int n_shell, const int32_t* nfn_tree, int leaf_max,
                   int32_t* lo, int32_t* hi, int32_t* child0, int32_t* child1,
                   int32_t* depth);

/* The traversal of Eq. 7 with the metric query of Eq. 8.  Node norms are
 * the Frobenius norms of the blocks, each computed from its definition.
 * Emits leaf quartets (A,B,C,D) as leaf ordinals (left-to-right).  Only
 * tasks whose A holds one of row_shell (user indices) are visited when
 * n_rows > 0.  Returns the number found (entries beyond cap not written),
 * or -1 on error. */
int64_t kxo_traverse(const kxo_basis* bs, const double* P, const int32_t* perm,
                     int n_node, const int32_t* lo, const int32_t* hi,
                     const int32_t* child0, const int32_t* child1,
                     const double* s2, double tau,
                     const int32_t* row_shell, int n_rows,
                     int32_t* out, int64_t cap);

/* Every leaf quartet whose own leaf bound exceeds tau (brute force). */
int64_t kxo_leaf_bruteforce(const kxo_basis* bs, const double* P, const int32_t* perm,
                            int n_node, const int32_t* lo, const int32_t* hi,
                            const int32_t* child0, const double* s2, double tau,
                            int32_t* out, int64_t cap, double* beta_out);

/* Exchange restricted to a leaf-quartet worklist, with the optional
 * shell-level metric query.  K rows outside row_shell (when n_rows > 0)
 * are left zero.  Returns the number of shell quartets evaluated. */
int64_t kxo_exchange_worklist(const kxo_basis* bs, const double* P, const int32_t* perm,
                              int n_node, const int32_t* lo, const int32_t* hi,
                              const int32_t* child0, const double* s2, double tau,
                              int shell_screen, const int32_t* work, int64_t n_work,
                              const int32_t* row_shell, int n_rows, double* K);

int kxo_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
