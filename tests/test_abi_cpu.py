"""C-ABI library: builds for sm_103a, loads, exports every declared symbol (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2012_03119_gb300 as gss
from paper_2012_03119_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(gss_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return gss.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), f"{n} declared but not exported"


def test_binding_covers_every_symbol():
    assert set(declared_functions()) <= set(gss.SIGNATURES)


def test_exports_are_c_symbols(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gss_\w+)", out))
    assert set(declared_functions()) <= exported


def test_build_targets_sm_103a_only():
    """The library is compiled for sm_103a alone: one -gencode, no PTX for other targets.
    (On a GPU, every -m gpu test launching a kernel shows that this code runs there.)"""
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_entry_points(lib):
    assert gss.gss_strerror(-4) == "GSS_E_OVERFLOW"
    assert gss.gss_strerror(0) == "GSS_OK"
    cfg = gss.gss_config_init()
    assert cfg.report_capacity == 1 << 22 and cfg.max_assignments == 1024 and cfg.mode == 0 and cfg.layout == 1
    assert lib.gss_config_init(None) == gss.GSS_E_INVAL
    assert lib.gss_destroy(None) == 0
    assert lib.gss_last_error(None) == b"no context"


def test_create_argument_checks(lib):
    out = ctypes.c_void_p()
    assert lib.gss_create(None, 10, None) == gss.GSS_E_INVAL
    assert lib.gss_create(ctypes.byref(out), 0, None) == gss.GSS_E_INVAL
    cfg = gss.gss_config_init()
    cfg.max_assignments = gss.GSS_MAX_ASSIGNMENTS + 1
    assert lib.gss_create(ctypes.byref(out), 10, ctypes.byref(cfg)) == gss.GSS_E_INVAL


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = ctypes.c_void_p()
    assert lib.gss_create(ctypes.byref(out), 10, None) == gss.GSS_E_CUDA
    assert not out.value


def test_expand_reports_host_helper():
    import numpy as np
    rec = np.zeros(2, gss.REPORT_DTYPE)
    rec[0] = (5, 1, 0b101)
    rec[1] = (2, 0, 1 << 31)
    assert gss.expand_reports(rec).tolist() == [[2, 31], [5, 32], [5, 34]]


def test_binding_structs_match_the_header(tmp_path):
    """Every public struct of include/gss.h has the size and field offsets that the ctypes
    binding declares (compiled with the host C compiler; no device needed)."""
    structs = [gss.gss_config, gss.gss_stats, gss.gss_batch_info, gss.gss_server_config, gss.gss_request_info,
               gss.gss_server_stats]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gss.h"', "int main(void) {"]
    for st in structs:
        n = st.__name__
        lines.append(f'  printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines.append('  printf("gss_report size %zu\\n", sizeof(gss_report));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        n = st.__name__
        assert got[(n, "size")] == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert got[(n, f)] == getattr(st, f).offset, (n, f)
    assert got[("gss_report", "size")] == gss.REPORT_DTYPE.itemsize == 12
