"""C-ABI library: builds for sm_103a, loads, exports every declared entry point, and reports
argument errors as statuses (no GPU needed for any of these)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1812_11626_gb300 import gksl
    return gksl


def _declared():
    hdr = open(os.path.join(ROOT, "include", "gksl.h")).read()
    return sorted(set(re.findall(r"\b(gksl_[a-z0-9_]+)\s*\(", hdr)))


def test_every_declared_symbol_is_exported(G):
    syms = subprocess.run(["nm", "-D", "--defined-only", G.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in syms.splitlines() if line.strip()}
    missing = [d for d in _declared() if d not in exported]
    assert not missing, missing
    assert set(_declared()) == set(G.EXPORTED)


def test_library_is_sm103a(G):
    out = subprocess.run(["cuobjdump", "--list-elf", G.LIB_PATH], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_argument_errors_are_statuses(G):
    import ctypes
    lib = G._lib
    n = ctypes.c_longlong()
    assert lib.gksl_structure_count(1, 0, ctypes.byref(n)) == G.GKSL_ERR_ARG
    assert lib.gksl_structure_count(5, 7, ctypes.byref(n)) == G.GKSL_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.gksl_create(1, 0, None, ctypes.byref(out)) == G.GKSL_ERR_ARG
    assert lib.gksl_set_drive(None, 0.0, 0.0, 1.0) == G.GKSL_ERR_ARG
    assert lib.gksl_batch_reset(None) == G.GKSL_ERR_ARG


def test_create_without_device_fails_cleanly(G):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(G.GkslError) as e:
        G.gksl_create(4, 0)
    assert e.value.status == G.GKSL_ERR_CUDA


def test_flag_constants_match_header(G):
    """Every GKSL_* constant that both the header and the binding define has the same value."""
    hdr = open(os.path.join(ROOT, "include", "gksl.h")).read()
    defs = {k: int(v) for k, v in re.findall(r"#define\s+(GKSL_[A-Z0-9_]+)\s+(\d+)u?\b", hdr)}
    assert "GKSL_ASM_WIDE_COLUMNS" in defs
    shared = [k for k in defs if hasattr(G, k)]
    assert len(shared) >= 6
    for k in shared:
        assert getattr(G, k) == defs[k], k


def test_info_struct_layout_matches_header(G, tmp_path):
    """The binding's gksl_info has the size and field offsets that a C compiler gives the
    header's struct (compiled here with gcc)."""
    import ctypes
    fields = [f for f, _ in G.gksl_info._fields_]
    src = tmp_path / "info.c"
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gksl.h"', "int main(void) {",
             '  printf("size %zu\\n", sizeof(gksl_info));']
    lines += [f'  printf("{f} %zu\\n", offsetof(gksl_info, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "info"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(G.gksl_info)
    for f in fields:
        assert int(out[f]) == getattr(G.gksl_info, f).offset, f


def test_noalloc_arguments_rejected_before_any_call(G):
    """The allocation-free entry point: the binding rejects host tensors and wrong dtypes before it
    calls the library, and the library itself rejects an oversized D or a null A0 with
    GKSL_ERR_ARG before it touches the GPU."""
    import ctypes

    import torch
    D = 3
    rp = torch.tensor([0, 1, 2, 3], dtype=torch.int32)
    col = torch.tensor([0, 1, 2], dtype=torch.int32)
    val = torch.ones(3, dtype=torch.float64)
    v = torch.zeros(D, dtype=torch.float64)
    for args in ((D, rp, col, val, None, None, None, None, v),
                 (D, rp.long(), col, val, None, None, None, None, v)):
        with pytest.raises(G.GkslError) as e:
            G.gksl_propagate_csr_noalloc(*args, 0.0, 1e-3, 1, 0.0, 0.0, 1.0)
        assert e.value.status == G.GKSL_ERR_ARG
    f = G._lib.gksl_propagate_csr_noalloc
    one = ctypes.c_void_p(8)   # never dereferenced: both calls return before any CUDA call
    assert f(G.GKSL_NOALLOC_MAX_D + 1, one, one, one, None, None, None, None, one, 0.0, 1e-3, 1, 0.0, 0.0, 1.0,
             None) == G.GKSL_ERR_ARG
    assert f(D, None, None, None, None, None, None, None, one, 0.0, 1e-3, 1, 0.0, 0.0, 1.0, None) == G.GKSL_ERR_ARG
