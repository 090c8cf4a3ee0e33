"""The C-ABI library builds, loads and exports every function the header
declares; argument checks answer without touching a GPU."""
import ctypes
import re

import numpy as np
import pytest


@pytest.fixture(scope="module")
def S():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_08849_gb300 import sfem
    return sfem


def test_exports_every_header_function(S):
    names = S.header_functions()
    assert "sfem_mesh_setup" in names and "sfem_solve" in names
    # the allocation-free apply is declared and exported like the others
    assert "sfem_apply_noalloc" in names and hasattr(S.lib, "sfem_apply_noalloc")
    for n in names:
        assert hasattr(S.lib, n), n


def test_status_strings_and_version(S):
    assert S.lib.sfem_version() == 1
    for code in range(0, -8, -1):
        assert S.sfem_strerror(code) != "unknown status"
    assert S.sfem_strerror(-99) == "unknown status"


def test_argument_checks_without_gpu(S):
    h = ctypes.c_void_p()
    xyz = np.zeros((4, 3))
    tets = np.array([[0, 1, 2, 3]], np.int32)
    # NULL out pointer
    assert S.lib.sfem_mesh_setup(None, xyz.ctypes.data, 4, tets.ctypes.data, 1, 1.0, 0.3,
                                 None, None, 0, None, None, 0, None, None) == S.SFEM_EINVAL
    # bad material and sizes are rejected before any device work
    for E, nu, nn, nt in ((-1.0, 0.3, 4, 1), (1.0, 0.5, 4, 1), (1.0, 0.3, 3, 1), (1.0, 0.3, 4, 0)):
        st = S.lib.sfem_mesh_setup(ctypes.byref(h), xyz.ctypes.data, nn, tets.ctypes.data, nt, E, nu,
                                   None, None, 0, None, None, 0, None, None)
        assert st == S.SFEM_EINVAL
        assert h.value is None
    # null handles
    assert S.lib.sfem_apply(None, None, None, 0, 1) == S.SFEM_EINVAL
    assert S.lib.sfem_apply_noalloc(None, None, None) == S.SFEM_EINVAL
    assert S.lib.sfem_tile_info(None, None, 1) == S.SFEM_EINVAL
    assert S.lib.sfem_assemble(None, None) == S.SFEM_EINVAL
    assert S.lib.sfem_solve(None, None, None, None, None) == S.SFEM_EINVAL
    # the tensor-core GEMM checks sizes, pointers and leading dimensions first
    assert S.lib.sfem_gemm_f32(0, 1, 1, None, 1, 0, None, 1, 0, None, 1, None) == S.SFEM_EINVAL
    buf = ctypes.c_void_p(16)  # never dereferenced: the checks fail first
    assert S.lib.sfem_gemm_f32(4, 4, 8, buf, 4, 0, buf, 4, 0, buf, 4, None) == S.SFEM_EINVAL  # lda < K
    assert S.lib.sfem_gemm_f32(4, 4, 8, buf, 8, 0, buf, 4, 0, buf, 3, None) == S.SFEM_EINVAL  # ldc < N
    S.lib.sfem_destroy(None)
    assert re.search(r"\w", S.lib.sfem_last_error().decode())


def test_struct_layouts_match_header(S, tmp_path):
    """ctypes mirrors of the ABI structs have the sizes and field offsets a C
    compiler gives the declarations in include/sfem.h."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [S.sfem_opts, S.sfem_mesh_info, S.sfem_csr, S.sfem_solve_opts, S.sfem_solve_info,
               S.sfem_batch_opts, S.sfem_batch_stats, S.sfem_learned_opts,
               S.sfem_coarse_opts]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sfem.h"', "int main(void){"]
    for st in structs:
        n = st.__name__
        lines.append(f'printf("{n} %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n}.{f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    inc = os.path.join(os.path.dirname(S.HEADER))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I" + inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for st in structs:
        n = st.__name__
        assert int(got[n]) == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert int(got[f"{n}.{f}"]) == getattr(st, f).offset, (n, f)
