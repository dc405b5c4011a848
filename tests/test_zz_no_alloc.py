"""The traversal entry point that allocates nothing (kx_traverse_level_noalloc).

It serves callers that cannot let a library allocate device memory (all
memory handed to their own allocator up front, or no allocation after
start-up).  Its output must equal the existing entry point's: walking it
level by level from the root task gives exactly the leaf-quartet worklist
that kx_exchange keeps (kx_get_worklist) for the same tau, in plain and in
symmetric builds (there only the K blocks A <= C).  Worklists are
integers, so the comparison is exact.  Two calls in a row check that the
shared scratch array carries nothing over.  This file sorts last so that a
run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


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


def _sorted(w):
    w = np.asarray(w, dtype=np.int64).reshape(-1, 4)
    return w[np.lexsort(w.T[::-1])] if len(w) else w


def _walk(kx, ex, tau):
    import torch
    _, depth = ex.leaves()
    front = torch.zeros((1, 4), dtype=torch.int16, device="cuda")   # root task (0,0,0,0)
    n = 1
    for level in range(depth):
        cap = max(16 * n, 16)
        nxt = torch.empty((cap, 4), dtype=torch.int16, device="cuda")
        n = kx.kx_traverse_level_noalloc(ex.ctx, level, front.data_ptr(), n, tau, nxt.data_ptr(), cap)
        front = nxt[:n]
    return front.cpu().numpy().view(np.uint16).astype(np.int64)


def _systems():
    big = wl.water64(2)
    s3 = wl.build_system("w3", big.symbols[:9], big.xyz[:9] / wl.BOHR_PER_ANGSTROM, "medium")
    w4, P4 = wl.workload("water4")
    return [(w4, P4, 1e-10, 4), (s3, wl.density(s3, 3003), 1e-10, 10), (w4, P4, 1e-3, 4)]


@pytest.mark.parametrize("symmetric", [0, 1])
@pytest.mark.parametrize("case", [0, 1, 2])
def test_noalloc_level_walk_matches_kx_exchange(kx, case, symmetric):
    import torch
    sys_, P, tau, leaf_max = _systems()[case]
    ex = kx.Exchange(sys_, leaf_max=leaf_max)
    ex(torch.from_numpy(P).cuda(), tau=tau, keep_worklist=1, symmetric=symmetric)
    ref = _sorted(ex.worklist())
    assert len(ref) > 0
    if symmetric:
        assert (ref[:, 0] <= ref[:, 2]).all()
    for _ in range(2):
        got = _sorted(_walk(kx, ex, tau))
        assert got.shape == ref.shape and np.array_equal(got, ref)
    ex.close()


def test_noalloc_rejects_node_ids_outside_the_level(kx):
    import torch
    sys_, P = wl.workload("water4")
    ex = kx.Exchange(sys_)
    ex(torch.from_numpy(P).cuda(), tau=1e-10)
    # level 0 holds one node (the root): id 3 is outside it; the kernel skips
    # that task without reading any table and the call reports KX_EINVAL
    front = torch.tensor([[0, 0, 0, 0], [0, 3, 0, 0]], dtype=torch.int16, device="cuda")
    nxt = torch.empty((64, 4), dtype=torch.int16, device="cuda")
    with pytest.raises(kx.KxError) as e:
        kx.kx_traverse_level_noalloc(ex.ctx, 0, front.data_ptr(), 2, 1e-10, nxt.data_ptr(), 64)
    assert e.value.code == kx.KX_EINVAL
    # the valid task alone still expands as before
    n = kx.kx_traverse_level_noalloc(ex.ctx, 0, front.data_ptr(), 1, 1e-10, nxt.data_ptr(), 64)
    assert 0 < n <= 16
    ex.close()


def test_noalloc_rejects_oversized_frontier(kx):
    import torch
    sys_, P = wl.workload("water4")
    ex = kx.Exchange(sys_)
    ex(torch.from_numpy(P).cuda(), tau=1e-10)
    with pytest.raises(kx.KxError) as e:
        kx.kx_traverse_level_noalloc(ex.ctx, 0, 0, kx.KX_NOALLOC_MAX_TASKS + 1, 1e-10, 0, 0)
    assert e.value.code == kx.KX_ECAPACITY
    # too small an output: the first cap tasks and the full count
    front = torch.zeros((1, 4), dtype=torch.int16, device="cuda")
    nxt = torch.full((2, 4), -1, dtype=torch.int16, device="cuda")
    with pytest.raises(kx.KxError) as e:
        kx.kx_traverse_level_noalloc(ex.ctx, 0, front.data_ptr(), 1, 1e-10, nxt.data_ptr(), 2)
    assert e.value.code == kx.KX_ECAPACITY
    ex.close()
