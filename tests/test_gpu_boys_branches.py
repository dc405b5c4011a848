"""Every angular-momentum class at chosen values of the Boys argument.

The class kernels evaluate F_m(T) from a Taylor table for T < 40 and from
F_0 = (1/2) sqrt(pi/T) with upward recursion above (the FP32 kernels in the
scaled form G_{n+1} = -G_n (2n+1) / |P-Q|^2).  Random systems may never put
every class on both sides of that switch, so these systems do: shells a, b
sit on one atom and c, d on another at distance R = sqrt(T / rho), rho =
pq / (p + q), so that T = rho |P - Q|^2 takes each listed value exactly
(T = 0: all four shells on one atom).  P is zero outside the (b, d) block,
so the K block (a, c) holds exactly one shell quartet of the class,
contracted with P (Eq. 6), and is compared with the oracle's Obara-Saika
integrals (oracle.eri) contracted the same way; the whole K is compared
with the oracle's direct exchange.

Tolerances: FP64, the contract's absolute 1e-10.  Forced FP32 (split above
every bound): 16 eps32 beta with beta = S_ab ||P_bd||_F S_cd, the Eq. 8
bound of the quartet; single FP32 quartets measured on GB300 stay below
6.2 eps32 beta in every class.  Double-word FP32 (KX_MIXED_DW with split 0:
every class with la+lb+lc+ld <= 5 in double words, the rest in FP64): the
FP64 bar, 1e-10.
"""
import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
EPS32 = 2.0 ** -24
T_VALUES = (0.0, 1e-8, 30.0, 39.9, 40.1, 200.0, 1e4)
ALPHA = (0.9, 0.35, 1.3, 0.6)   # a, b, c, d (bohr^-2)


@pytest.fixture(scope="module")
def kx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1401_6961_gb300 import build
    build.build()
    import paper_1401_6961_gb300 as kx
    kx.load()
    return kx


def quartet_system(la, lb, lc, ld, T):
    """Four shells (a, b on atom X at the origin; c, d on atom Y) placed so
    that the Boys argument of the quartet (ab|cd) is T."""
    aa, ab, ac, ad = ALPHA
    p, q = aa + ab, ac + ad
    rho = p * q / (p + q)
    R = np.sqrt(T / rho)
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    if T == 0.0:
        xyz = np.zeros((1, 3))
        atom = np.array([0, 0, 0, 0], dtype=np.int32)
    else:
        xyz = np.stack([np.zeros(3), R * u])
        atom = np.array([0, 0, 1, 1], dtype=np.int32)
    syms = ["X"] * len(xyz)
    s = wl.System(name=f"q{la}{lb}{lc}{ld}", symbols=syms, xyz=xyz, shell_atom=atom,
                  shell_l=np.array([la, lb, lc, ld], dtype=np.int32), shell_alpha=np.array(ALPHA))
    return s


def run_case(kx, T, precision):
    import torch
    rng = np.random.default_rng(int(T * 10) + 7)
    worst = 0.0
    for cls in range(81):
        la, lb, lc, ld = cls // 27, (cls // 9) % 3, (cls // 3) % 3, cls % 3
        s = quartet_system(la, lb, lc, ld, T)
        off = s.shell_offset
        P = np.zeros((s.n_fn, s.n_fn))
        P[off[1]:off[2], off[3]:off[4]] = rng.standard_normal((off[2] - off[1], off[4] - off[3]))
        ex = kx.Exchange(s, leaf_max=1)
        opts = dict(tau=0.0, symmetric=0)
        if precision == "fp32":
            opts.update(precision=kx.KX_MIXED, split_threshold=1e300)
        elif precision == "dw":
            opts.update(precision=kx.KX_MIXED_DW, split_threshold=0.0)
        K = ex(torch.from_numpy(P).cuda(), **opts).cpu().numpy()
        if precision == "fp32":
            assert ex.stats.n_shell_quartets_fp64 == 0
        elif precision == "dw":
            # the quartet of the class itself runs in double words when L <= 5,
            # in FP64 above; nothing runs in FP32 at split 0
            if la + lb + lc + ld <= 5:
                assert ex.stats.n_shell_quartets_dw >= 1
            else:
                assert ex.stats.n_shell_quartets_fp64 >= 1
            assert ex.stats.n_shell_quartets == ex.stats.n_shell_quartets_dw + ex.stats.n_shell_quartets_fp64
        ex.close()
        ctr = s.xyz[s.shell_atom]
        v = oracle.eri(ctr[0], ALPHA[0], la, ctr[1], ALPHA[1], lb, ctr[2], ALPHA[2], lc, ctr[3], ALPHA[3], ld)
        Pbd = P[off[1]:off[2], off[3]:off[4]]
        ref = np.einsum("ijkl,jl->ik", v, Pbd)
        got = K[off[0]:off[1], off[2]:off[3]]
        err = np.abs(got - ref).max()
        K0 = oracle.exchange_direct(s, P)
        err_all = np.abs(K - K0).max()
        if precision in ("fp64", "dw"):
            assert err <= TOL64 and err_all <= TOL64, (cls, T, err, err_all)
            worst = max(worst, err)
        else:
            s2 = oracle.schwarz_sq(s)
            beta = np.sqrt(s2[0, 1]) * np.linalg.norm(Pbd) * np.sqrt(s2[2, 3])
            assert err <= 16 * EPS32 * beta, (cls, T, err, beta, err / (EPS32 * beta))
            assert err_all <= 1e-8 + 16 * EPS32 * np.abs(K0).max() * 4, (cls, T, err_all)
            worst = max(worst, err / (EPS32 * beta))
    return worst


@pytest.mark.parametrize("T", T_VALUES)
def test_every_class_at_boys_argument_fp64(kx, T):
    run_case(kx, T, "fp64")


@pytest.mark.parametrize("T", T_VALUES)
def test_every_class_at_boys_argument_fp32(kx, T):
    worst = run_case(kx, T, "fp32")
    print(f"T = {T:g}: largest FP32 error {worst:.2f} eps32 beta")


@pytest.mark.parametrize("T", T_VALUES)
def test_every_class_at_boys_argument_double_word(kx, T):
    worst = run_case(kx, T, "dw")
    print(f"T = {T:g}: largest double-word error {worst:.2e}")
