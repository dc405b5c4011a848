"""The C-ABI library without a GPU: it loads, exports every entry point
declared in include/kx.h, and rejects bad calls before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1401_6961_gb300 import build
    build.build()
    import paper_1401_6961_gb300 as kx
    return kx.load()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "kx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kx_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("kx_create", "kx_build_schwarz", "kx_build_tree", "kx_exchange", "kx_exchange_host",
              "kx_get_worklist", "kx_get_norms", "kx_last_error", "kx_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import paper_1401_6961_gb300 as kx
    names = declared_entry_points()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(kx.EXPORTS) == names


def test_default_opts(lib):
    import paper_1401_6961_gb300 as kx
    o = kx.kx_default_opts()
    assert o.tau == 1e-10 and o.precision == kx.KX_FP64 and o.shell_screen == 1
    assert o.keep_worklist == 0 and o.chunk_records == 0 and o.symmetric == 0


def test_struct_layouts_match_header(lib):
    import paper_1401_6961_gb300 as kx
    assert ctypes.sizeof(kx.kx_opts) == 64
    assert ctypes.sizeof(kx.kx_basis) == 40
    # 5 counters + 32 levels + 4 ints + 12 doubles
    assert ctypes.sizeof(kx.kx_stats) == 8 * 5 + 8 * 32 + 4 * 4 + 8 * 12


def test_create_rejects_bad_basis_without_gpu(lib):
    import paper_1401_6961_gb300 as kx
    xyz = np.zeros((1, 3))
    good = dict(xyz=xyz, shell_atom=[0], shell_l=[0], shell_alpha=[1.0])
    bad = [dict(good, shell_l=[3]), dict(good, shell_alpha=[-1.0]), dict(good, shell_atom=[1]),
           dict(good, shell_alpha=[float("nan")]), dict(good, xyz=np.array([[np.inf, 0, 0]]))]
    for b in bad:
        with pytest.raises(kx.KxError) as e:
            kx.kx_create(**b)
        assert e.value.code == kx.KX_EINVAL


def test_null_context_calls(lib):
    import paper_1401_6961_gb300 as kx
    assert lib.kx_build_schwarz(None, 0.0) == kx.KX_EINVAL
    assert lib.kx_build_tree(None, 10, None) == kx.KX_EINVAL
    assert lib.kx_count(None, None, 0, None, None) == kx.KX_EINVAL
    assert lib.kx_n_functions(None) == -1
    assert lib.kx_last_error(None) == b"null context"
    lib.kx_destroy(None)


def test_no_gpu_reports_cuda_error(lib):
    import torch
    import paper_1401_6961_gb300 as kx
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(kx.KxError) as e:
        kx.kx_create(np.zeros((1, 3)), [0], [0], [1.0])
    assert e.value.code == kx.KX_ECUDA


C_PROGRAM = r"""
#include "kx.h"
#include <stdio.h>
int main(void) {
    kx_opts o;
    kx_stats st;
    kx_default_opts(&o);
    if (kx_count(NULL, NULL, 0, &o, &st) != KX_EINVAL) return 1;
    if (kx_exchange(NULL, NULL, 0, &o, NULL, 0, NULL) != KX_EINVAL) return 2;
    if (kx_n_functions(NULL) != -1) return 3;
    printf("%s\n", kx_last_error(NULL));
    kx_destroy(NULL);
    {
        /* host-only shard plan: the tie at the middle leaf goes to the lower boundary */
        const double w[5] = {1.0, 1.0, 4.0, 1.0, 1.0};
        int32_t b[3];
        if (kx_shard_bounds(w, 5, 2, b) != KX_OK || b[0] != 0 || b[1] != 2 || b[2] != 5) return 4;
    }
    printf("%d %d %d\n", (int)sizeof(kx_opts), (int)sizeof(kx_stats), (int)sizeof(kx_basis));
    return 0;
}
"""


def test_header_is_plain_c_and_links(lib, tmp_path):
    """The boundary is usable from C: the header compiles as strict C11 and a
    C program links against libkx.so and calls it (null-context checks only:
    no device work)."""
    import shutil
    import subprocess
    import paper_1401_6961_gb300 as kx
    from paper_1401_6961_gb300 import _binding
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_kx.c"
    src.write_text(C_PROGRAM)
    libdir = os.path.dirname(_binding.library_path())
    exe = tmp_path / "use_kx"
    r = subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I",
                        os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lkx",
                        f"-Wl,-rpath,{libdir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.returncode
    lines = r.stdout.strip().splitlines()
    assert lines[0] == "null context"
    # the C compiler's struct sizes are the binding's
    assert [int(x) for x in lines[1].split()] == [ctypes.sizeof(kx.kx_opts), ctypes.sizeof(kx.kx_stats),
                                                  ctypes.sizeof(kx.kx_basis)]
