"""Seeded synthetic workloads for the screened exchange build.

This module only *generates inputs*: molecular geometries, uncontracted
Gaussian shell lists and model density matrices.  It holds none of the
method's arithmetic (no integrals, norms, trees or screening), so both the
CUDA path and the CPU oracle can consume the very same bytes.

The paper's own runs (Sec. "Implementation and results") use SCF-converged
B3LYP/6-31G** densities of water droplets (H2O)_n.  Those densities, the
basis data and the program that made them are not available here, so these
generators stand in for them:

* water clusters at 1 g/cm^3 (the paper's droplets are at STP conditions),
  random molecular orientations, Hilbert-curve ordering is applied later by
  the library itself;
* uncontracted even-tempered basis sets (one primitive per shell, Cartesian
  d);
* a symmetric model density with exponential decay,
  P_{ls} = z_{ls} * exp(-|R_l - R_s| / 2 Angstrom), z ~ N(0, 1), which has the
  "decay without sparsification" structure the paper requires (end of Sec.
  "Exchange as hextree traversal").

Units: geometries are generated in Angstrom and returned in bohr
(1 Angstrom = 1/0.529177210903 bohr); exponents are in bohr^-2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Sequence, Tuple

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
AVOGADRO = 6.02214076e23
WATER_MASS = 18.015          # g/mol
OH_BOND = 0.9572             # Angstrom
HOH_ANGLE = 104.52           # degrees
CC_BOND = 1.54
CH_BOND = 1.09
TETRAHEDRAL = 109.4712206    # degrees

# Cartesian component counts per angular momentum (Cartesian d: 6).
NCART = (1, 3, 6)

# ----------------------------------------------------------------------------
# basis sets: element -> list of (l, alpha) in the per-atom shell order
# ----------------------------------------------------------------------------


def _even_tempered(alpha0: float, ratio: float, n: int) -> List[float]:
    return [alpha0 * ratio ** k for k in range(n)]


BASIS_SETS: Dict[str, Dict[str, List[Tuple[int, float]]]] = {
    # (H2O)_4 basis: O 3 s (0.3*4^k) + 2 p (0.5*4^k); H 2 s (0.2*5^k)
    # -> 13 functions per water.
    "small": {
        "O": [(0, a) for a in _even_tempered(0.3, 4.0, 3)]
        + [(1, a) for a in _even_tempered(0.5, 4.0, 2)],
        "H": [(0, a) for a in _even_tempered(0.2, 5.0, 2)],
        "C": [(0, a) for a in _even_tempered(0.3, 4.0, 3)]
        + [(1, a) for a in _even_tempered(0.5, 4.0, 2)],
    },
    # (H2O)_64 basis: alpha_k = 0.15 * 3.5^k per l; O 4 s + 3 p + 1 d;
    # H 3 s + 1 p -> 31 functions per water.
    "medium": {
        "O": [(0, a) for a in _even_tempered(0.15, 3.5, 4)]
        + [(1, a) for a in _even_tempered(0.15, 3.5, 3)]
        + [(2, a) for a in _even_tempered(0.15, 3.5, 1)],
        "H": [(0, a) for a in _even_tempered(0.15, 3.5, 3)]
        + [(1, a) for a in _even_tempered(0.15, 3.5, 1)],
        "C": [(0, a) for a in _even_tempered(0.15, 3.5, 4)]
        + [(1, a) for a in _even_tempered(0.15, 3.5, 3)]
        + [(2, a) for a in _even_tempered(0.15, 3.5, 1)],
    },
}


@dataclasses.dataclass
class System:
    """A molecule plus its uncontracted shell list (user order).

    Shells are atom-major in atom input order, and within an atom in the
    basis-set order above.  Functions follow shells; inside a shell the
    Cartesian components are ordered with the x power descending
    (p: x, y, z; d: xx, xy, xz, yy, yz, zz).
    """

    name: str
    symbols: List[str]
    xyz: np.ndarray            # (n_atom, 3) bohr
    shell_atom: np.ndarray     # (n_shell,) int32
    shell_l: np.ndarray        # (n_shell,) int32
    shell_alpha: np.ndarray    # (n_shell,) float64, bohr^-2

    @property
    def n_atom(self) -> int:
        return len(self.symbols)

    @property
    def n_shell(self) -> int:
        return int(self.shell_l.shape[0])

    @property
    def shell_nfn(self) -> np.ndarray:
        return np.array([NCART[l] for l in self.shell_l], dtype=np.int32)

    @property
    def shell_offset(self) -> np.ndarray:
        off = np.zeros(self.n_shell + 1, dtype=np.int64)
        np.cumsum(self.shell_nfn, out=off[1:])
        return off

    @property
    def n_fn(self) -> int:
        return int(self.shell_nfn.sum())

    def function_atom(self) -> np.ndarray:
        return np.repeat(self.shell_atom, self.shell_nfn).astype(np.int64)


def build_system(name: str, symbols: Sequence[str], xyz_ang: np.ndarray,
                 basis: str) -> System:
    table = BASIS_SETS[basis]
    sa, sl, sx = [], [], []
    for i, s in enumerate(symbols):
        for (l, a) in table[s]:
            sa.append(i)
            sl.append(l)
            sx.append(a)
    return System(
        name=name,
        symbols=list(symbols),
        xyz=np.ascontiguousarray(np.asarray(xyz_ang, dtype=np.float64) * BOHR_PER_ANGSTROM),
        shell_atom=np.asarray(sa, dtype=np.int32),
        shell_l=np.asarray(sl, dtype=np.int32),
        shell_alpha=np.asarray(sx, dtype=np.float64),
    )


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _water_monomer() -> np.ndarray:
    """O at the origin, H atoms in the xy plane (Angstrom)."""
    half = math.radians(HOH_ANGLE) / 2.0
    h1 = OH_BOND * np.array([math.cos(half), math.sin(half), 0.0])
    h2 = OH_BOND * np.array([math.cos(half), -math.sin(half), 0.0])
    return np.stack([np.zeros(3), h1, h2])


def _place_waters(o_sites: np.ndarray, rng: np.random.Generator) -> Tuple[List[str], np.ndarray]:
    mono = _water_monomer()
    syms: List[str] = []
    xyz: List[np.ndarray] = []
    for o in o_sites:
        rot = _random_rotation(rng)
        w = mono @ rot.T + o
        syms += ["O", "H", "H"]
        xyz.append(w)
    return syms, np.concatenate(xyz, axis=0)


def water_box_side(n: int, density_g_cm3: float = 1.0) -> float:
    """Cube side (Angstrom) holding n waters at the given density."""
    vol_cm3 = n * WATER_MASS / AVOGADRO / density_g_cm3
    return vol_cm3 ** (1.0 / 3.0) * 1e8


def water_cluster_sites(n: int, rng: np.random.Generator, jitter: float = 0.3,
                        min_oo: float = 2.5) -> np.ndarray:
    """O positions of n waters in a cube at 1 g/cm^3.

    Sites are the points of an m^3 grid (m = ceil(n^(1/3)), spacing L/m);
    when n < m^3 a seeded subset of n sites is used.  Each O is displaced by
    a uniform jitter in [-jitter, jitter]^3 Angstrom, redrawn until every
    O-O distance is at least ``min_oo``.  No periodic images (the paper's
    droplets are finite clusters).
    """
    side = water_box_side(n)
    m = int(math.ceil(round(n ** (1.0 / 3.0), 9)))
    while m ** 3 < n:
        m += 1
    h = side / m
    grid = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)],
                    dtype=np.float64)
    if len(grid) > n:
        pick = np.sort(rng.choice(len(grid), size=n, replace=False))
        grid = grid[pick]
    base = (grid + 0.5) * h
    out = np.empty_like(base)
    for i in range(n):
        for _ in range(1000):
            cand = base[i] + rng.uniform(-jitter, jitter, size=3)
            if i == 0 or np.min(np.linalg.norm(out[:i] - cand, axis=1)) >= min_oo:
                break
        out[i] = cand
    return out


def water_square4(rng: np.random.Generator, side: float = 2.8) -> np.ndarray:
    """Four O atoms on a square of the given side (O-O ~ 2.8 Angstrom)."""
    return np.array([[0, 0, 0], [side, 0, 0], [side, side, 0], [0, side, 0]],
                    dtype=np.float64)


def water4(seed: int = 1) -> System:
    """(H2O)_4 with random orientations and the small basis (52 functions)."""
    rng = np.random.default_rng(seed)
    syms, xyz = _place_waters(water_square4(rng), rng)
    return build_system("(H2O)4", syms, xyz, "small")


def water_cluster(n: int, seed: int, basis: str = "medium") -> System:
    """(H2O)_n at 1 g/cm^3 in a seeded cube."""
    rng = np.random.default_rng(seed)
    sites = water_cluster_sites(n, rng)
    syms, xyz = _place_waters(sites, rng)
    return build_system(f"(H2O){n}", syms, xyz, basis)


def water64(seed: int = 2) -> System:
    """(H2O)_64 with the medium basis (1984 functions, 1024 shells)."""
    return water_cluster(64, seed, "medium")


def water_sweep(n: int, basis: str = "medium") -> System:
    """Scaling sweep member (H2O)_n, n in {64, 128, 256, 512}; seed 4000+n."""
    return water_cluster(n, 4000 + n, basis)


def water_batch(count: int = 256, seed_base: int = 3, lo: int = 4, hi: int = 48) -> List[System]:
    """Independent clusters of uneven size (n ~ U{lo..hi}), small basis."""
    rng = np.random.default_rng(seed_base)
    sizes = rng.integers(lo, hi + 1, size=count)
    return [water_cluster(int(n), seed_base * 100000 + i, "small") for i, n in enumerate(sizes)]


def batch_workload(count: int = 256, seed_base: int = 3, lo: int = 4, hi: int = 48
                   ) -> Tuple[List[System], List[np.ndarray]]:
    """The batched workload: ``water_batch`` clusters, each with its own
    density (cluster i of seed base s: seed s * 100000 + i + 1000)."""
    systems = water_batch(count, seed_base, lo, hi)
    dens = [density(x, seed_base * 100000 + i + 1000) for i, x in enumerate(systems)]
    return systems, dens


def _place_nerf(a: np.ndarray, b: np.ndarray, c: np.ndarray, bond: float,
                angle_deg: float, torsion_deg: float) -> np.ndarray:
    """Atom d bonded to c with angle b-c-d and torsion a-b-c-d."""
    ang = math.radians(angle_deg)
    tor = math.radians(torsion_deg)
    bc = c - b
    bc /= np.linalg.norm(bc)
    n = np.cross(b - a, bc)
    n /= np.linalg.norm(n)
    m = np.cross(n, bc)
    d2 = np.array([-bond * math.cos(ang), bond * math.sin(ang) * math.cos(tor),
                   bond * math.sin(ang) * math.sin(tor)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * n


ALKANE_MIN_CC = 2.4      # Angstrom: carbons three or more bonds apart
ALKANE_MIN_NONBONDED = 1.5   # Angstrom: every other pair of atoms not bonded
ALKANE_TRIES = 40        # torsion draws per carbon before stepping back one carbon


def _alkane_hydrogens(c: List[np.ndarray], i: int) -> List[np.ndarray]:
    """Hydrogen positions of carbon i of the chain c (its neighbours placed)."""
    n = len(c)
    nb = [j for j in (i - 1, i + 1) if 0 <= j < n]
    if len(nb) == 2:
        u = (c[i] - c[nb[0]]) + (c[i] - c[nb[1]])
        u /= np.linalg.norm(u)
        w = np.cross(c[nb[0]] - c[i], c[nb[1]] - c[i])
        w /= np.linalg.norm(w)
        half = math.radians(TETRAHEDRAL) / 2.0
        return [c[i] + CH_BOND * (math.cos(half) * u + sgn * math.sin(half) * w) for sgn in (1.0, -1.0)]
    j = nb[0]
    # a reference atom for the torsion: the next carbon along, or a fixed
    # off-axis point for ethane-like ends
    k = [q for q in (j - 1, j + 1) if 0 <= q < n and q != i]
    ref = c[k[0]] if k else c[j] + np.array([0.0, 1.0, 0.0])
    return [_place_nerf(ref, c[j], c[i], CH_BOND, TETRAHEDRAL, tor) for tor in (60.0, 180.0, 300.0)]


def _clashes(new: List[Tuple[np.ndarray, str, int]], old: List[Tuple[np.ndarray, str, int]]) -> bool:
    """True if an atom of `new` sits too close to an atom of `new` or `old`.

    Atoms are (position, element, carbon index: the carbon itself or the one
    a hydrogen is bonded to).  Bonded pairs (C-C of neighbouring carbons, C-H
    of a hydrogen and its carbon) are exempt; carbons three or more bonds
    apart must be ALKANE_MIN_CC apart, every other pair ALKANE_MIN_NONBONDED.
    """
    pool = old + new
    for ia, (x, ex, cx) in enumerate(new):
        for jb, (y, ey, cy) in enumerate(pool):
            if jb >= len(old) and jb - len(old) <= ia:
                continue   # each pair of new atoms once, never an atom with itself
            if ex == "C" and ey == "C":
                if abs(cx - cy) <= 1:
                    continue
                lim = ALKANE_MIN_CC if abs(cx - cy) >= 3 else ALKANE_MIN_NONBONDED
            elif ex != ey and cx == cy:
                continue   # C-H bond
            else:
                lim = ALKANE_MIN_NONBONDED
            if float(np.linalg.norm(x - y)) < lim:
                return True
    return False


def alkane(n_carbon: int, seed: int, basis: str = "small") -> System:
    """Linear alkane C_nH_{2n+2} with seeded torsions, free of clashes.

    C-C 1.54, C-H 1.09 Angstrom, tetrahedral angles; backbone torsions are
    drawn from {60, 180, 300} degrees plus a uniform +-15 degree jitter.  The
    chain is self-avoiding: a torsion is drawn again when the carbon it
    places, or the hydrogens it completes, would come closer than 2.4
    Angstrom to a carbon three or more bonds away or 1.5 Angstrom to any
    other atom it is not bonded to, and after ALKANE_TRIES draws the previous
    carbon is drawn again.  Atoms: the carbons in chain order, then the
    hydrogens carbon by carbon.  Carbon uses the oxygen shell set of the
    chosen basis.
    """
    if n_carbon < 3:
        raise ValueError("alkane needs at least three carbons")
    rng = np.random.default_rng(seed)
    ang = math.radians(TETRAHEDRAL)
    c = [np.array([0.0, 0.0, 0.0]), np.array([CC_BOND, 0.0, 0.0]),
         np.array([CC_BOND, 0.0, 0.0]) + CC_BOND * np.array([-math.cos(ang), math.sin(ang), 0.0])]
    # atoms placed by each step: step 2 = the first three carbons and the
    # hydrogens of carbons 0 and 1; step i >= 3 = carbon i and the hydrogens
    # of carbon i-1 (and of carbon i itself when it ends the chain)
    steps: List[List[Tuple[np.ndarray, str, int]]] = []
    first = [(c[k], "C", k) for k in range(3)]
    first += [(h, "H", k) for k in ((0, 1, 2) if n_carbon == 3 else (0, 1)) for h in _alkane_hydrogens(c, k)]
    if _clashes(first, []):
        raise RuntimeError("alkane: clash in the first three carbons")
    steps.append(first)
    tries = [0] * (n_carbon + 1)
    i = 3
    draws = 0
    while i < n_carbon:
        draws += 1
        if draws > 200000:
            raise RuntimeError(f"alkane: no self-avoiding chain of {n_carbon} carbons found (seed {seed})")
        if tries[i] >= ALKANE_TRIES:
            # step back: the previous carbon is drawn again
            tries[i] = 0
            if i == 3:
                raise RuntimeError(f"alkane: no self-avoiding chain of {n_carbon} carbons found (seed {seed})")
            steps.pop()
            c.pop()
            i -= 1
            continue
        tries[i] += 1
        tor = float(rng.choice([60.0, 180.0, 300.0]) + rng.uniform(-15.0, 15.0))
        ci = _place_nerf(c[i - 3], c[i - 2], c[i - 1], CC_BOND, TETRAHEDRAL, tor)
        trial = c + [ci]
        new = [(ci, "C", i)] + [(h, "H", i - 1) for h in _alkane_hydrogens(trial, i - 1)]
        if i == n_carbon - 1:
            new += [(h, "H", i) for h in _alkane_hydrogens(trial, i)]
        old = [a for st in steps for a in st]
        if _clashes(new, old):
            continue
        c.append(ci)
        steps.append(new)
        i += 1
        if i < n_carbon:
            tries[i] = 0
    atoms = [a for st in steps for a in st]
    carbons = sorted((a for a in atoms if a[1] == "C"), key=lambda a: a[2])
    hydrogens = sorted((a for a in atoms if a[1] == "H"), key=lambda a: a[2])   # stable: placement order
    syms = ["C"] * n_carbon + ["H"] * len(hydrogens)
    xyz = np.stack([a[0] for a in carbons] + [a[0] for a in hydrogens])
    return build_system(f"C{n_carbon}H{2 * n_carbon + 2}", syms, xyz, basis)


# ----------------------------------------------------------------------------
# model density matrix
# ----------------------------------------------------------------------------


def density(sys_: System, seed: int, decay_ang: float = 2.0) -> np.ndarray:
    """Symmetric model density P_{ls} = z_{ls} exp(-|R_l - R_s| / decay).

    z ~ N(0,1) is drawn for the upper triangle (diagonal included) in
    row-major order and mirrored; R is the centre of the function's atom and
    the distance is taken in Angstrom.  Rows and columns follow the user
    function order of ``sys_``.
    """
    rng = np.random.default_rng(seed)
    n = sys_.n_fn
    fa = sys_.function_atom()
    r = sys_.xyz[fa] / BOHR_PER_ANGSTROM
    d = np.sqrt(((r[:, None, :] - r[None, :, :]) ** 2).sum(-1))
    z = rng.standard_normal((n, n))
    z = np.triu(z)
    z = z + np.triu(z, 1).T
    return np.ascontiguousarray(z * np.exp(-d / decay_ang))


# ----------------------------------------------------------------------------
# random shells for integral tests
# ----------------------------------------------------------------------------


def random_shells(n: int, seed: int, lmax: int = 2, box: float = 3.0,
                  alpha_range: Tuple[float, float] = (0.1, 8.0)) -> System:
    """n shells on n distinct random atoms (bohr box), random l and alpha."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(-box, box, size=(n, 3)) / BOHR_PER_ANGSTROM
    l = rng.integers(0, lmax + 1, size=n).astype(np.int32)
    a = np.exp(rng.uniform(math.log(alpha_range[0]), math.log(alpha_range[1]), size=n))
    sys_ = System(name=f"random{n}", symbols=["X"] * n,
                  xyz=np.ascontiguousarray(xyz * BOHR_PER_ANGSTROM),
                  shell_atom=np.arange(n, dtype=np.int32), shell_l=l, shell_alpha=a)
    return sys_


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

# tau values used with each named workload
WORKLOADS = {
    "water4": dict(make=lambda: water4(1), p_seed=1001, taus=(0.0, 1e-10)),
    "water64": dict(make=lambda: water64(2), p_seed=1002, taus=(1e-10,)),
    # a smaller cluster with the same basis and density generator
    "water16": dict(make=lambda: water_cluster(16, 16, "medium"), p_seed=1016, taus=(1e-10,)),
}


def workload(name: str) -> Tuple[System, np.ndarray]:
    """(system, density) for a named workload."""
    if name in WORKLOADS:
        w = WORKLOADS[name]
        s = w["make"]()
        return s, density(s, w["p_seed"])
    if name.startswith("water_sweep"):
        n = int(name[len("water_sweep"):])
        s = water_sweep(n)
        return s, density(s, 5000 + n)
    if name.startswith("alkane"):
        n = int(name[len("alkane"):])
        s = alkane(n, 6000 + n)
        return s, density(s, 7000 + n)
    raise KeyError(name)
