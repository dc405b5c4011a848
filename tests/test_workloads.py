"""The seeded input recipe: the synthetic stand-ins for the paper's water
droplets, alkanes and densities have the geometry, sizes and structure the
recipe states, and the same seed gives the same bytes."""
import math

import numpy as np
import pytest

import workloads as wl

ANG = 1.0 / wl.BOHR_PER_ANGSTROM


def _waters(sys_):
    xyz = sys_.xyz * ANG
    assert sys_.symbols == ["O", "H", "H"] * (sys_.n_atom // 3)
    return xyz[0::3], xyz[1::3], xyz[2::3]


def _check_monomers(sys_):
    o, h1, h2 = _waters(sys_)
    d1 = np.linalg.norm(h1 - o, axis=1)
    d2 = np.linalg.norm(h2 - o, axis=1)
    np.testing.assert_allclose(d1, wl.OH_BOND, atol=1e-12)
    np.testing.assert_allclose(d2, wl.OH_BOND, atol=1e-12)
    cosang = ((h1 - o) * (h2 - o)).sum(1) / (d1 * d2)
    np.testing.assert_allclose(np.degrees(np.arccos(cosang)), wl.HOH_ANGLE, atol=1e-9)


def _min_oo(sys_):
    o, _, _ = _waters(sys_)
    d = np.linalg.norm(o[:, None] - o[None], axis=-1)
    d[np.diag_indices_from(d)] = np.inf
    return d.min()


def test_water4_square_and_sizes():
    s = wl.water4(1)
    _check_monomers(s)
    o, _, _ = _waters(s)
    sides = [np.linalg.norm(o[i] - o[(i + 1) % 4]) for i in range(4)]
    np.testing.assert_allclose(sides, 2.8, atol=1e-12)
    assert (s.n_atom, s.n_shell, s.n_fn) == (12, 36, 52)


@pytest.mark.parametrize("n,basis,n_fn,n_shell", [(64, "medium", 1984, 1024), (16, "medium", 496, 256),
                                                  (128, "small", 1664, 1152)])
def test_water_cluster_density_and_spacing(n, basis, n_fn, n_shell):
    s = wl.water_cluster(n, 7, basis)
    _check_monomers(s)
    assert (s.n_fn, s.n_shell) == (n_fn, n_shell)
    # 1 g/cm^3: the cube that holds n waters
    side = wl.water_box_side(n)
    assert side == pytest.approx((n * 18.015 / 6.02214076e23) ** (1 / 3) * 1e8, rel=1e-12)
    o, _, _ = _waters(s)
    assert o.min() >= -0.3 - 1e-12 and o.max() <= side + 0.3 + 1e-12
    assert _min_oo(s) >= 2.5


def test_benchmark_and_sweep_members_keep_the_oo_floor():
    assert _min_oo(wl.water64(2)) >= 2.5
    for n in (64, 128, 256):
        assert _min_oo(wl.water_sweep(n, "small")) >= 2.5


def test_alkane_bonds_and_counts():
    """Bond lengths, backbone angles and counts."""
    for n in (3, 6, 14, 40):
        s = wl.alkane(n, 6000 + n)
        xyz = s.xyz * ANG
        c = xyz[:n]
        h = xyz[n:]
        assert s.symbols == ["C"] * n + ["H"] * (2 * n + 2)
        np.testing.assert_allclose(np.linalg.norm(c[1:] - c[:-1], axis=1), wl.CC_BOND, atol=1e-9)
        # hydrogens follow their carbons: three on each end, two on the others
        parent = [0] * 3 + [i for i in range(1, n - 1) for _ in range(2)] + [n - 1] * 3
        np.testing.assert_allclose(np.linalg.norm(h - c[parent], axis=1), wl.CH_BOND, atol=1e-9)
        # backbone angles are tetrahedral
        for i in range(1, n - 1):
            u, v = c[i - 1] - c[i], c[i + 1] - c[i]
            ang = math.degrees(math.acos(u @ v / (np.linalg.norm(u) * np.linalg.norm(v))))
            assert ang == pytest.approx(wl.TETRAHEDRAL, abs=1e-6)
        # small basis: C carries the O shells (9 functions), H 2 s shells
        assert s.n_fn == 9 * n + 2 * (2 * n + 2)


def test_alkanes_are_self_avoiding():
    """No clashes in the chains of the learned-culling evaluation: carbons
    three or more bonds apart are at least 2.4 Angstrom apart, every other
    pair of atoms that is not bonded at least 1.5 Angstrom (a brute-force
    check over all pairs, independent of the generator's own test)."""
    for n in (10, 14, 20, 40, 80):
        s = wl.alkane(n, 6000 + n)
        xyz = s.xyz * ANG
        carbon = [i for i in range(n)] + [0] * 3 + [i for i in range(1, n - 1) for _ in range(2)] + [n - 1] * 3
        is_c = np.array([q == "C" for q in s.symbols])
        d = np.linalg.norm(xyz[:, None] - xyz[None], axis=-1)
        for i in range(s.n_atom):
            for j in range(i + 1, s.n_atom):
                if is_c[i] and is_c[j]:
                    sep = abs(carbon[i] - carbon[j])
                    if sep == 1:
                        continue
                    assert d[i, j] >= (2.4 if sep >= 3 else 1.5) - 1e-12, (n, i, j, d[i, j])
                elif is_c[i] != is_c[j] and carbon[i] == carbon[j]:
                    continue
                else:
                    assert d[i, j] >= 1.5 - 1e-12, (n, i, j, d[i, j])


def test_density_is_symmetric_and_decays():
    s = wl.water_cluster(16, 16, "small")
    P = wl.density(s, 1016)
    assert P.shape == (s.n_fn, s.n_fn)
    np.testing.assert_array_equal(P, P.T)
    fa = s.function_atom()
    r = s.xyz[fa] * ANG
    d = np.linalg.norm(r[:, None] - r[None], axis=-1)
    z = P / np.exp(-d / 2.0)
    iu = np.triu_indices(s.n_fn)
    # the undamped factors are standard normal draws
    assert abs(z[iu].mean()) < 0.05 and abs(z[iu].std() - 1.0) < 0.05


def test_same_seed_same_bytes():
    a, b = wl.water_cluster(32, 5, "medium"), wl.water_cluster(32, 5, "medium")
    np.testing.assert_array_equal(a.xyz, b.xyz)
    np.testing.assert_array_equal(wl.density(a, 9), wl.density(b, 9))
    assert not np.array_equal(wl.density(a, 9), wl.density(a, 10))


def test_batch_recipe():
    systems, dens = wl.batch_workload()
    assert len(systems) == len(dens) == 256
    nw = np.array([s.n_atom // 3 for s in systems])
    assert nw.min() >= 4 and nw.max() <= 48
    assert sum(s.n_fn for s in systems) == 87360
    assert all(d.shape == (s.n_fn, s.n_fn) for s, d in zip(systems, dens))
    assert sum(d.size for d in dens) * 8 == 296980320
