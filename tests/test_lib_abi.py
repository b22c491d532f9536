"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/seg4d.h with the struct layouts the binding assumes.
No compute call is made here (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2111_11866_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "seg4d.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(seg4d_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 14, names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(_lib.SIGNATURES), set(names) - set(_lib.SIGNATURES)


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sizes.c"
    src.write_text('#include "seg4d.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   "int main(void){printf(\"%zu %zu %zu %zu %zu %zu\\n\", sizeof(seg4d_params),"
                   " sizeof(seg4d_seed), sizeof(seg4d_info), sizeof(seg4d_dims),"
                   " offsetof(seg4d_info, sweeps_total), offsetof(seg4d_params, max_iters));"
                   "printf(\"%zu %zu\\n\", offsetof(seg4d_params, tol_inf), offsetof(seg4d_info, res_inf));"
                   "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = [int(x) for x in out]
    want = [C.sizeof(_lib.CParams), C.sizeof(_lib.CSeed), C.sizeof(_lib.CInfo),
            C.sizeof(_lib.CDims), _lib.CInfo.sweeps_total.offset, _lib.CParams.max_iters.offset,
            _lib.CParams.tol_inf.offset, _lib.CInfo.res_inf.offset]
    assert got == want


def test_default_params_and_device_bytes(lib):
    p = _lib.Params.defaults()
    assert p.h == (0.01, 0.01, 0.01, 0.01) and p.tau == 0.01 and p.eps == 1.0
    assert p.delta == 0.5 and p.vartheta == 0.5 and p.lambda_th == 0.87 and p.R_init == 12.0
    assert abs(p.sigma_t - 0.01**2 / 8) < 1e-20
    nb = _lib.Seg4D.device_bytes((128, 128, 64, 32))
    # 72 bytes per voxel of grid state (G once per face) plus 48 of the FP32
    # solve's arrays (scaled weights by both ends), and a small side table of
    # boundary-face G
    assert 115 * 33554432 < nb < 125 * 33554432
    # the lean handle: 64 bytes per voxel
    nl = _lib.Seg4D.device_bytes((128, 128, 64, 32), lean=True)
    assert 60 * 33554432 < nl < 68 * 33554432
    assert _lib.Seg4D.device_bytes((0, 1, 1, 1)) == 0


def test_host_tensors_are_used_in_place():
    """CPU tensors (pinned ones included) are passed by pointer as host memory,
    so reads land in the caller's tensor; numpy arrays likewise."""
    import numpy as np
    import torch
    t = torch.zeros(2, 3, 4, 5)
    p, dev, keep = _lib._ptr(t, 120)
    assert dev == 0 and keep is t and p.value == t.data_ptr()
    a = np.zeros((2, 3, 4, 5), np.float32)
    p, dev, keep = _lib._ptr(a, 120)
    assert dev == 0 and keep is a
    with pytest.raises(TypeError):
        _lib._ptr(torch.zeros(120, dtype=torch.float64), 120)
