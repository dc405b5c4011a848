"""Host analysis of the symmetry cases (paper_1401_6961_gb300.symmetry) and
the integral/contraction FLOP split of the library's counter
(kx_class_flops); no GPU."""
import itertools

import numpy as np
import pytest


@pytest.fixture(scope="module")
def kx():
    import paper_1401_6961_gb300 as kx
    try:
        kx.load()
    except (OSError, ImportError) as e:
        pytest.skip(f"library not built: {e}")
    return kx


def _brute(work):
    from paper_1401_6961_gb300.symmetry import _images
    kept = {tuple(int(x) for x in q) for q in work}
    seen, full, coinc, sparse = set(), 0, 0, 0
    for q in kept:
        imgs = frozenset(_images(q))
        if imgs in seen:
            continue
        seen.add(imgs)
        k = len(imgs & kept)
        if k < len(imgs):
            sparse += 1
        elif len(imgs) == 8:
            full += 1
        else:
            coinc += 1
    return len(seen), full, coinc, sparse


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_occurrence_counts_match_brute_force(seed):
    from paper_1401_6961_gb300 import symmetry
    rng = np.random.default_rng(seed)
    allq = np.array(list(itertools.product(range(4), repeat=4)))
    work = allq[rng.random(len(allq)) < 0.7]
    c = symmetry.occurrence_counts(work)
    blocks, full, coinc, sparse = _brute(work)
    assert (c["blocks"], c["full"], c["coincident"], c["sparse"]) == (blocks, full, coinc, sparse)
    assert c["quartets"] == len(work)


def test_every_quartet_kept_has_no_sparse_blocks():
    from paper_1401_6961_gb300 import symmetry
    allq = np.array(list(itertools.product(range(5), repeat=4)))
    c = symmetry.occurrence_counts(allq)
    assert c["sparse"] == 0
    # canonical blocks of 5 leaves: unordered pairs of unordered pairs
    pairs = 5 * 6 // 2
    assert c["blocks"] == pairs * (pairs + 1) // 2
    assert c["quartets"] == 5 ** 4


def test_class_flop_split(kx):
    # L = 0: set-up 20 and Boys 6 + 13 + 0, no Hermite recursion
    t, i = kx.kx_class_flops(0)
    assert i == 39.0 and t > i
    # L = 1: Boys 6 + 26 + 1 and three first-order Hermite terms
    t, i = kx.kx_class_flops(1)
    assert i == 20 + 33 + 3
    for cls in range(81):
        t, i = kx.kx_class_flops(cls)
        L = cls // 27 + (cls // 9) % 3 + (cls // 3) % 3 + cls % 3
        assert 0 < i < t
        assert i == kx.kx_class_flops([c for c in range(81) if
                                       c // 27 + (c // 9) % 3 + (c // 3) % 3 + c % 3 == L][0])[1]
    with pytest.raises(kx.KxError):
        kx.kx_class_flops(81)
