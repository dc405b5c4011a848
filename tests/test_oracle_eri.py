"""Pins of the oracle's electron-repulsion and overlap integrals.

The oracle uses Obara-Saika / Head-Gordon-Pople recurrences.  Independent of
them, the tests use:

* the (ss|ss) closed form
  (ss|ss) = 2 pi^{5/2} / (p q sqrt(p+q)) K_AB K_CD F_0(rho |P-Q|^2);
* the centre-derivative identities of unnormalised Cartesian Gaussians,
  x_A g = (1/2a) dg/dA_x and x_A^2 g = (1/4a^2) (d^2 g/dA_x^2 + 2a g),
  applied analytically (sympy, with dF_n/dT = -F_{n+1}) to that closed form,
  which gives every class up to (dd|dd) without any recurrence;
* the 8-fold permutational symmetry of (mu lam|nu sig) and the
  Cauchy-Schwarz inequality;
* closed-form overlaps and the unit self-overlap of x^l components.
"""
import math

import numpy as np
import pytest

import oracle

sp = pytest.importorskip("sympy")
mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 30

NC = (1, 3, 6)


def comps(l):
    out = []
    for i in range(l, -1, -1):
        for j in range(l - i, -1, -1):
            out.append((i, j, l - i - j))
    return out


def norm(a, l):
    return (2 * a / math.pi) ** 0.75 * (4 * a) ** (l / 2) / math.sqrt(3.0 if l == 2 else 1.0)


# ---------------------------------------------------------------------------
# closed form
# ---------------------------------------------------------------------------

def boys0(T):
    return 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))


def ssss_closed(A, a, B, b, C, c, D, d):
    A, B, C, D = map(np.asarray, (A, B, C, D))
    p, q = a + b, c + d
    P = (a * A + b * B) / p
    Q = (c * C + d * D) / q
    rho = p * q / (p + q)
    KAB = math.exp(-a * b / p * np.sum((A - B) ** 2))
    KCD = math.exp(-c * d / q * np.sum((C - D) ** 2))
    T = rho * np.sum((P - Q) ** 2)
    return 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * KAB * KCD * boys0(T)


def test_ssss_closed_form():
    rng = np.random.default_rng(11)
    for _ in range(200):
        ctr = rng.uniform(-3, 3, size=(4, 3))
        ex = np.exp(rng.uniform(math.log(0.05), math.log(20.0), size=4))
        got = oracle.eri(ctr[0], ex[0], 0, ctr[1], ex[1], 0, ctr[2], ex[2], 0, ctr[3], ex[3], 0)
        ref = ssss_closed(ctr[0], ex[0], ctr[1], ex[1], ctr[2], ex[2], ctr[3], ex[3])
        ref *= norm(ex[0], 0) * norm(ex[1], 0) * norm(ex[2], 0) * norm(ex[3], 0)
        assert got[0, 0, 0, 0] == pytest.approx(ref, rel=1e-13, abs=1e-300)


def test_ssss_same_centre():
    # all four on one centre: T = 0, F_0 = 1
    A = np.array([0.3, -0.2, 0.5])
    got = oracle.eri(A, 1.0, 0, A, 1.0, 0, A, 1.0, 0, A, 1.0, 0)[0, 0, 0, 0]
    ref = 2 * math.pi ** 2.5 / (4 * math.sqrt(4.0)) * norm(1.0, 0) ** 4
    assert got == pytest.approx(ref, rel=1e-15)


# ---------------------------------------------------------------------------
# centre derivatives of the closed form (sympy)
# ---------------------------------------------------------------------------

class _Boys(sp.Function):
    nargs = 2

    def fdiff(self, argindex=2):
        n, T = self.args
        return -_Boys(n + 1, T)


def _boys_mp(n, T):
    n = int(n)
    if T == 0:
        return mpmath.mpf(1) / (2 * n + 1)
    return mpmath.gammainc(n + mpmath.mpf(1) / 2, 0, T) / (2 * T ** (n + mpmath.mpf(1) / 2))


_X = sp.symbols("ax ay az bx by bz cx cy cz dx dy dz")
_CTR = (_X[0:3], _X[3:6], _X[6:9], _X[9:12])


def _closed_sym(ex):
    al, be, ga, de = ex
    A, B, C, D = _CTR
    p, q = al + be, ga + de
    rho = p * q / (p + q)
    P = [(al * A[i] + be * B[i]) / p for i in range(3)]
    Q = [(ga * C[i] + de * D[i]) / q for i in range(3)]
    AB2 = sum((A[i] - B[i]) ** 2 for i in range(3))
    CD2 = sum((C[i] - D[i]) ** 2 for i in range(3))
    T = rho * sum((P[i] - Q[i]) ** 2 for i in range(3))
    return (2 * sp.pi ** sp.Rational(5, 2) / (p * q * sp.sqrt(p + q))
            * sp.exp(-al * be / p * AB2) * sp.exp(-ga * de / q * CD2) * _Boys(0, T))


def _apply(expr, ctr, zeta, comp):
    for x, k in enumerate(comp):
        v = ctr[x]
        if k == 1:
            expr = sp.diff(expr, v) / (2 * zeta)
        elif k == 2:
            expr = (sp.diff(expr, v, 2) + 2 * zeta * expr) / (4 * zeta ** 2)
    return expr


def _derivative_value(ex_r, coords_r, cmp4):
    e = _closed_sym(ex_r)
    for ci in range(4):
        e = _apply(e, _CTR[ci], ex_r[ci], cmp4[ci])
    e = e.subs({_X[i]: coords_r[i] for i in range(12)})
    f = sp.lambdify([], e, modules=[{"_Boys": _boys_mp}, "mpmath"])
    return float(f())


# (class, component indices to check; None = all)
DERIV_CASES = [
    ((1, 0, 0, 0), None), ((0, 1, 0, 0), None), ((0, 0, 1, 0), None), ((0, 0, 0, 1), None),
    ((2, 0, 0, 0), None), ((0, 0, 0, 2), None),
    ((1, 1, 0, 0), None), ((1, 0, 1, 0), None), ((0, 1, 0, 1), None),
    ((2, 1, 0, 0), [(0, 0, 0, 0), (1, 2, 0, 0), (5, 1, 0, 0)]),
    ((2, 0, 2, 0), [(0, 0, 0, 0), (1, 0, 4, 0), (3, 0, 5, 0)]),
    ((1, 1, 1, 1), [(0, 0, 0, 0), (0, 1, 2, 1), (2, 2, 2, 2)]),
    ((0, 2, 1, 2), [(0, 1, 0, 1), (0, 4, 2, 3)]),
    ((2, 1, 1, 2), [(1, 2, 0, 5)]),
    ((2, 2, 2, 2), [(1, 5, 0, 4)]),
]


@pytest.mark.parametrize("cls,picks", DERIV_CASES, ids=[str(c[0]) for c in DERIV_CASES])
def test_eri_centre_derivatives(cls, picks):
    rng = np.random.default_rng(sum(x * 3 ** i for i, x in enumerate(cls)) + 5)
    coords = np.round(rng.uniform(-1.5, 1.5, size=12), 3)
    ex = np.round(np.exp(rng.uniform(math.log(0.2), math.log(3.0), size=4)), 3)
    ex_r = [sp.Rational(str(x)) for x in ex]
    coords_r = [sp.Rational(str(x)) for x in coords]
    la, lb, lc, ld = cls
    got = oracle.eri(coords[0:3], ex[0], la, coords[3:6], ex[1], lb,
                     coords[6:9], ex[2], lc, coords[9:12], ex[3], ld)
    nrm = norm(ex[0], la) * norm(ex[1], lb) * norm(ex[2], lc) * norm(ex[3], ld)
    if picks is None:
        picks = [(i, j, k, l) for i in range(NC[la]) for j in range(NC[lb])
                 for k in range(NC[lc]) for l in range(NC[ld])]
    cl = [comps(la), comps(lb), comps(lc), comps(ld)]
    for (i, j, k, l) in picks:
        ref = _derivative_value(ex_r, coords_r, (cl[0][i], cl[1][j], cl[2][k], cl[3][l]))
        assert got[i, j, k, l] / nrm == pytest.approx(ref, rel=1e-11, abs=1e-14), (i, j, k, l)


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

def _random_quartet(rng, ls=None):
    ctr = rng.uniform(-2, 2, size=(4, 3))
    ex = np.exp(rng.uniform(math.log(0.1), math.log(6.0), size=4))
    if ls is None:
        ls = rng.integers(0, 3, size=4)
    return ctr, ex, [int(x) for x in ls]


def test_eri_eightfold_symmetry():
    rng = np.random.default_rng(3)
    for _ in range(40):
        ctr, ex, ls = _random_quartet(rng)
        s = [(ctr[i], ex[i], ls[i]) for i in range(4)]

        def E(a, b, c, d):
            return oracle.eri(*s[a], *s[b], *s[c], *s[d])
        base = E(0, 1, 2, 3)
        np.testing.assert_allclose(E(1, 0, 2, 3), base.transpose(1, 0, 2, 3), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(E(0, 1, 3, 2), base.transpose(0, 1, 3, 2), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(E(1, 0, 3, 2), base.transpose(1, 0, 3, 2), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(E(2, 3, 0, 1), base.transpose(2, 3, 0, 1), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(E(3, 2, 0, 1), base.transpose(3, 2, 0, 1), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(E(2, 3, 1, 0), base.transpose(2, 3, 1, 0), rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(E(3, 2, 1, 0), base.transpose(3, 2, 1, 0), rtol=1e-12, atol=1e-15)


def test_eri_cauchy_schwarz():
    rng = np.random.default_rng(4)
    for _ in range(60):
        ctr, ex, ls = _random_quartet(rng)
        s = [(ctr[i], ex[i], ls[i]) for i in range(4)]
        v = oracle.eri(*s[0], *s[1], *s[2], *s[3])
        ab = oracle.eri(*s[0], *s[1], *s[0], *s[1])
        cd = oracle.eri(*s[2], *s[3], *s[2], *s[3])
        na, nb, nc, nd = v.shape
        dab = np.array([[ab[i, j, i, j] for j in range(nb)] for i in range(na)])
        dcd = np.array([[cd[k, l, k, l] for l in range(nd)] for k in range(nc)])
        assert np.all(dab >= 0) and np.all(dcd >= 0)
        bound = np.sqrt(dab)[:, :, None, None] * np.sqrt(dcd)[None, None, :, :]
        assert np.all(np.abs(v) <= bound * (1 + 1e-12) + 1e-300)


def test_eri_far_apart_decay():
    # two distant, well separated charge distributions: (ss|ss) -> 1/R
    A = np.zeros(3)
    C = np.array([0.0, 0.0, 40.0])
    a = 5.0
    got = oracle.eri(A, a, 0, A, a, 0, C, a, 0, C, a, 0)[0, 0, 0, 0]
    # each normalised s^2 distribution carries charge <s|s> = 1
    assert got == pytest.approx(1.0 / 40.0, rel=1e-12)


# ---------------------------------------------------------------------------
# overlap (Eq. 4)
# ---------------------------------------------------------------------------

def test_overlap_self_normalisation():
    A = np.array([0.1, 0.2, 0.3])
    for l in range(3):
        for a in (0.15, 1.0, 7.3):
            S = oracle.overlap(A, a, l, A, a, l)
            expect = [1.0 if max(c) == l else 1.0 / 3.0 for c in comps(l)]
            np.testing.assert_allclose(np.diag(S), expect, rtol=1e-13)


def test_overlap_ss_closed_form_and_derivative():
    rng = np.random.default_rng(9)
    for _ in range(20):
        A, B = rng.uniform(-2, 2, size=(2, 3))
        a, b = np.exp(rng.uniform(-2, 2, size=2))
        p = a + b
        ss = (math.pi / p) ** 1.5 * math.exp(-a * b / p * np.sum((A - B) ** 2))
        got = oracle.overlap(A, a, 0, B, b, 0)[0, 0] / (norm(a, 0) * norm(b, 0))
        assert got == pytest.approx(ss, rel=1e-13)
        # (p_x|s) = (1/2a) d/dA_x (s|s) = (1/2a) * (-2 a b/p (A_x - B_x)) (s|s)
        got_p = oracle.overlap(A, a, 1, B, b, 0)[:, 0] / (norm(a, 1) * norm(b, 0))
        ref_p = -(b / p) * (A - B) * ss
        np.testing.assert_allclose(got_p, ref_p, rtol=1e-12, atol=1e-300)
