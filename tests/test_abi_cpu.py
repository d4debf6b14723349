"""The C-ABI library builds, loads and exports every symbol include/hisq.h declares.

No GPU needed: only calls that fail argument validation before touching CUDA
are made.
"""
import ctypes
import os
import re

import pytest

from conftest import ROOT, lib_built

HEADER = os.path.join(ROOT, "include", "hisq.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hisq_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = lib_built()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hisq_gauge_load", "hisq_dslash", "hisq_dslash_ex", "hisq_cg_solve",
                 "hisq_link_compress", "hisq_link_reconstruct", "hisq_mdagm"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in hisq.h but not exported"


def test_binding_covers_every_declared_symbol():
    import paper_1411_4439_gb300.hisq as B
    assert sorted(B.EXPORTED) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(B, name))


def test_version_and_defaults_without_gpu(lib):
    import paper_1411_4439_gb300 as H
    assert H.hisq_version() >= 10000
    p = H.hisq_cg_default_params()
    assert (p.maxiter, p.reliable_every, p.inner_prec, p.even_odd) == (100000, 50, H.HISQ_F32, 1)
    assert abs(p.reliable_delta - 0.1) < 1e-15


@pytest.mark.parametrize("L", [(4, 4, 4, 5), (2, 4, 4, 4), (4, 4, 4, 0)])
def test_bad_extents_rejected_before_cuda(L):
    import numpy as np
    import paper_1411_4439_gb300 as H
    U = np.zeros((4, 4, 4, 4, 4, 3, 3), dtype=np.complex128)
    with pytest.raises(H.HisqError) as e:
        H.hisq_gauge_load(L, U, U)
    assert e.value.status == H.hisq.HISQ_EINVAL
    assert "extent" in str(e.value)


def test_bad_modes_rejected(lib):
    import numpy as np
    import paper_1411_4439_gb300 as H
    U = np.zeros((4, 4, 4, 4, 4, 3, 3), dtype=np.complex128)
    for kw in (dict(recon_N=12), dict(recon_U=8), dict(prec=7),
               dict(prec=H.HISQ_F64, recon_N=14)):
        with pytest.raises(H.HisqError) as e:
            H.hisq_gauge_load((4, 4, 4, 4), U, U, **kw)
        assert e.value.status == H.hisq.HISQ_EINVAL


def test_null_handle_rejected(lib):
    assert lib.hisq_gauge_free(None) == 0
    f = lib.hisq_dslash
    f.restype = ctypes.c_int
    assert f(None, None, None, 1, 0, 1, None) == 1   # HISQ_EINVAL


def test_binding_constants_match_the_header():
    """Every HISQ_* enumerator of the header has the same value in the binding."""
    import paper_1411_4439_gb300.hisq as B
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    pairs = re.findall(r"\b(HISQ_[A-Z0-9_]+)\s*=\s*(\d+)", text)
    assert len(pairs) >= 25
    for name, value in pairs:
        assert getattr(B, name) == int(value), name


def test_new_entry_points_reject_bad_arguments_before_cuda(lib):
    """Tuned load, bundle tuner, autotuner, batched solve and mapping calls
    validate their arguments before any CUDA call."""
    import paper_1411_4439_gb300.hisq as B
    L = (ctypes.c_int * 4)(4, 4, 4, 4)
    h = ctypes.c_void_p()
    f = lib.hisq_gauge_load_tuned
    f.restype = ctypes.c_int
    assert f(L, None, None, 0, B.HISQ_F32, 0, ctypes.c_double(1e-10), None, ctypes.byref(h)) == B.HISQ_EINVAL
    assert f(L, None, None, 0, 7, 4, ctypes.c_double(1e-10), None, ctypes.byref(h)) == B.HISQ_EINVAL
    assert f(L, None, None, 0, B.HISQ_F32, 4, ctypes.c_double(1e-10), None, None) == B.HISQ_EINVAL
    f = lib.hisq_autotune_bundle
    f.restype = ctypes.c_int
    assert f(None, 8, B.HISQ_F32, B.HISQ_AOS, 5, None, None) == B.HISQ_EINVAL
    f = lib.hisq_autotune_dslash
    f.restype = ctypes.c_int
    assert f(None, 8, B.HISQ_F32, B.HISQ_AOS, 5, None, None, None, None) == B.HISQ_EINVAL
    f = lib.hisq_cg_solve_batched
    f.restype = ctypes.c_int
    assert f(None, 1, None, None, None) == B.HISQ_EINVAL
    probs = (B.hisq_cg_problem * 1)()
    assert f(probs, 0, None, None, None) == B.HISQ_EINVAL
    assert f(probs, 65, None, None, None) == B.HISQ_EINVAL
    assert f(probs, 1, None, None, None) == B.HISQ_EINVAL       # NULL handle in the problem
    f = lib.hisq_set_dslash_mapping
    f.restype = ctypes.c_int
    assert f(None, 4, 2, B.HISQ_MAP_PIPELINED2) == B.HISQ_EINVAL
    err = lib.hisq_last_error
    err.restype = ctypes.c_char_p
    assert b"NULL handle" in err()


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structures have the size and field offsets a C compiler
    gives the header's structures (compiled here with the host compiler)."""
    import shutil
    import subprocess

    from paper_1411_4439_gb300 import hisq as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"hisq_cg_params": B.hisq_cg_params, "hisq_cg_stats": B.hisq_cg_stats,
               "hisq_cg_problem": B.hisq_cg_problem}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "hisq.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
