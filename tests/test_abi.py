"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/g3bfs.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import subprocess

import pytest

import paper_2012_10026_gb300 as g3


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(g3.LIB_PATH):
        from paper_2012_10026_gb300 import build
        build.build()
    return g3.lib()


def test_exports_every_declared_symbol(L):
    declared = g3.declared_symbols()
    assert "g3_bfs" in declared and "g3_build_csr" in declared and "g3_rcm_relabel" in declared
    out = subprocess.run(["nm", "-D", "--defined-only", g3.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    for s in declared:
        assert hasattr(L, s)


def test_status_strings_and_version(L):
    assert L.g3_status_str(0) == b"ok"
    assert L.g3_status_str(1) == b"invalid argument"
    assert L.g3_status_str(99) == b"unknown status"
    assert b"sm_103a" in L.g3_version()


def test_default_options(L):
    o = g3.opts()
    assert (o.controller, o.alpha, o.beta, o.t1, o.t2, o.t3) == (0, 14, 24, 32, 1024, 32768)
    assert o.bu_reverse == 1 and o.timing == 0 and not o.mlp_params


def test_bad_arguments_rejected_on_host(L):
    out = ctypes.c_void_p(123)
    assert L.g3_build_csr(None, None, 10, 5, None, ctypes.byref(out)) == g3.G3_EINVAL
    assert out.value is None
    assert L.g3_build_csr(None, None, 0, 0, None, ctypes.byref(out)) == g3.G3_EINVAL
    assert L.g3_build_csr(None, None, -1, 4, None, ctypes.byref(out)) == g3.G3_EINVAL
    assert L.g3_build_csr(None, None, 0, 4, None, None) == g3.G3_EINVAL
    assert L.g3_rcm_relabel(None, None) == g3.G3_EINVAL
    assert L.g3_bfs(None, 0, None, None, None, None, 0, None, None) == g3.G3_EINVAL
    assert L.g3_get_perm(None, None, None, None) == g3.G3_EINVAL
    assert L.g3_get_csr(None, None, None, None) == g3.G3_EINVAL
    info = g3.g3_graph_info()
    assert L.g3_graph_info_get(None, ctypes.byref(info)) == g3.G3_EINVAL
    assert b"NULL" in L.g3_last_error_detail() or b"null" in L.g3_last_error_detail()
    L.g3_graph_free(None)  # no-op


def test_struct_layouts_match_header(tmp_path):
    # the C compiler's layout of each struct in include/g3bfs.h must equal the
    # binding's ctypes layout, field by field
    structs = [g3.g3_graph_info, g3.g3_bfs_opts, g3.g3_level_stats, g3.g3_msbfs_opts,
               g3.g3_msbfs_stats, g3.g3_batch_opts, g3.g3_tune_entry]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "g3bfs.h"', 'int main(void){']
    for S in structs:
        lines.append(f'printf("{S.__name__} %zu\\n", sizeof({S.__name__}));')
        for name, _ in S._fields_:
            lines.append(f'printf("{S.__name__}.{name} %zu\\n", offsetof({S.__name__}, {name}));')
    lines.append('return 0;}')
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(g3.__file__)), "include")
    subprocess.run(["gcc", "-I", inc, str(c), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for S in structs:
        assert int(got[S.__name__]) == ctypes.sizeof(S), S.__name__
        for name, _ in S._fields_:
            assert int(got[f"{S.__name__}.{name}"]) == getattr(S, name).offset, (S.__name__, name)


def test_product_does_not_import_oracle():
    import sys
    pkg_dir = os.path.dirname(g3.__file__)
    for root, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
