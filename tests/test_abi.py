"""C-ABI checks that need no GPU: the library loads, exports every function
include/gbconv.h declares, and validates arguments on the host (documented
status codes, nothing launched)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2207_00257_gb300 import _build, binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    _build.build()
    B.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "gbconv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_symbols_exported():
    names = header_functions()
    assert "conv2d_fwd" in names and "conv2d_grouped" in names
    out = subprocess.run(["nm", "-D", "--defined-only", B.lib_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if " T " in line)
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert sorted(B.EXPORTS) == names
    for n in names:
        assert hasattr(B.lib(), n)


def test_status_strings_and_version():
    for s in range(7):
        assert B.status_string(s).startswith("GBCONV_")
    assert B.status_string(99) == "GBCONV_UNKNOWN_STATUS"
    assert B.gbconv_version() == 10000


SHAPES = [
    (1, 3, 32, 32, 16, 3, 3, 1, 1, 1), (32, 256, 56, 56, 64, 1, 1, 1, 0, 1),
    (32, 128, 56, 56, 128, 3, 3, 2, 1, 1), (2, 8, 7, 9, 8, 5, 3, (2, 1), (2, 0), (1, 3)),
    (1, 16, 112, 112, 16, 7, 7, 2, 3, 1), (4, 8, 6, 6, 8, 3, 3, 1, 0, 2),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_output_dims_match_oracle(shape):
    N, C, H, W, K, R, S, st, pd, dl = shape
    prob = B.problem(N, C, H, W, K, R, S, st, pd, dl)
    s, P, Q = B.gbconv_output_dims(prob)
    assert s == B.GBCONV_OK
    p = oracle.Conv(N, C, H, W, K, R, S, st, pd, dl)
    assert (P, Q) == (p.P, p.Q)


def test_invalid_problems_rejected():
    bad = [
        dict(N=-1), dict(C=0), dict(H=0), dict(K=0), dict(R=0), dict(stride=(0, 1)),
        dict(dil=(1, 0)), dict(pad=(-1, 0)), dict(R=9, H=4),  # P < 1
        dict(in_dtype=7), dict(layout=5), dict(flags=8),
    ]
    for kw in bad:
        base = dict(N=2, C=8, H=8, W=8, K=8, R=3, S=3, stride=1, pad=1, dil=1)
        base.update(kw)
        extra = {k: base.pop(k) for k in ("in_dtype", "layout", "flags") if k in base}
        prob = B.problem(base["N"], base["C"], base["H"], base["W"], base["K"], base["R"],
                         base["S"], base["stride"], base["pad"], base["dil"], **extra)
        s, _, _ = B.gbconv_output_dims(prob)
        assert s == B.GBCONV_ERR_INVALID_ARG, kw
        assert B.conv2d_fwd(prob, 16, 32, 0, 0, 0, 48, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG, kw


def test_null_pointers_rejected_before_launch():
    prob = B.problem(2, 8, 8, 8, 8, 3, 3, 1, 1, 1)
    assert B.conv2d_fwd(prob, 0, 16, 0, 0, 0, 32, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG
    assert B.conv2d_fwd(prob, 16, 0, 0, 0, 0, 32, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG
    assert B.conv2d_fwd(prob, 16, 32, 0, 0, 0, 0, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG
    pb = B.problem(2, 8, 8, 8, 8, 3, 3, 1, 1, 1, flags=B.GBCONV_FLAG_BIAS)
    assert B.conv2d_fwd(pb, 16, 32, 0, 0, 0, 48, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG  # no bias
    assert B.conv2d_fwd(prob, 16, 32, 0, 0, 0, 16, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG  # alias
    assert B.conv2d_dgrad(prob, 0, 16, 32, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG
    assert B.conv2d_wgrad(prob, 16, 32, 0, 0, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG
    assert B.gbconv_quantize_e4m3(0, B.GBCONV_F32, 1, 16, 32, 48, 0) == B.GBCONV_ERR_INVALID_ARG
    assert B.gbconv_quantize_e4m3(16, B.GBCONV_E4M3, 1, 16, 32, 48, 0) == B.GBCONV_ERR_UNSUPPORTED
    assert B.conv2d_grouped(-1, [], [], [], None, [], 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG
    assert B.conv2d_grouped(0, [], [], [], None, [], 0, 0, 0) == B.GBCONV_OK


def test_tensor_core_alignment_rules():
    # BF16 NHWC needs C % 8 == 0 and K % 8 == 0, and 16-byte aligned pointers
    p = B.problem(2, 12, 8, 8, 8, 3, 3, 1, 1, 1, B.GBCONV_BF16, B.GBCONV_BF16)
    assert B.conv2d_fwd(p, 4096, 8192, 0, 0, 0, 12288, 0, 0, 0) == B.GBCONV_ERR_ALIGNMENT
    p = B.problem(2, 16, 8, 8, 8, 3, 3, 1, 1, 1, B.GBCONV_BF16, B.GBCONV_BF16)
    assert B.conv2d_fwd(p, 4098, 8192, 0, 0, 0, 12288, 0, 0, 0) == B.GBCONV_ERR_ALIGNMENT
    # E4M3 needs C % 16 and both scales
    p = B.problem(2, 8, 8, 8, 8, 3, 3, 1, 1, 1, B.GBCONV_E4M3, B.GBCONV_BF16)
    assert B.conv2d_fwd(p, 4096, 8192, 0, 64, 128, 12288, 0, 0, 0) == B.GBCONV_ERR_ALIGNMENT
    p = B.problem(2, 16, 8, 8, 8, 3, 3, 1, 1, 1, B.GBCONV_E4M3, B.GBCONV_BF16)
    assert B.conv2d_fwd(p, 4096, 8192, 0, 0, 0, 12288, 0, 0, 0) == B.GBCONV_ERR_INVALID_ARG


def test_unsupported_combinations():
    # BF16 NCHW forward needs its layout-transform workspace; its gradients and
    # F32 -> BF16 are not offered
    p = B.problem(2, 16, 8, 8, 8, 3, 3, 1, 1, 1, B.GBCONV_BF16, B.GBCONV_BF16, B.GBCONV_NCHW)
    assert B.conv2d_fwd(p, 4096, 8192, 0, 0, 0, 12288, 0, 0, 0) == B.GBCONV_ERR_WORKSPACE
    s, n = B.gbconv_workspace_size(B.GBCONV_OP_FWD, p)
    assert s == B.GBCONV_OK and n == 4096 + 2304 + 2048  # x, w, y, each rounded to 256 B
    p = B.problem(2, 16, 8, 8, 8, 3, 3, 1, 1, 1, B.GBCONV_F32, B.GBCONV_BF16)
    assert B.conv2d_fwd(p, 4096, 8192, 0, 0, 0, 12288, 0, 0, 0) == B.GBCONV_ERR_UNSUPPORTED
    # E4M3 output is never produced
    p = B.problem(2, 16, 8, 8, 8, 3, 3, 1, 1, 1, B.GBCONV_E4M3, B.GBCONV_E4M3)
    assert B.conv2d_fwd(p, 4096, 8192, 0, 64, 128, 12288, 0, 0, 0) == B.GBCONV_ERR_UNSUPPORTED
    p = B.problem(2, 16, 8, 8, 8, 3, 3, 1, 1, 1, B.GBCONV_E4M3, B.GBCONV_BF16)
    assert B.conv2d_dgrad(p, 4096, 8192, 12288, 0, 0, 0) == B.GBCONV_ERR_UNSUPPORTED


def test_workspace_sizes():
    # forward needs none; dgrad on the tensor-core path holds the rotated filter
    p = B.problem(32, 128, 56, 56, 128, 3, 3, 1, 1, 1)
    assert B.gbconv_workspace_size(B.GBCONV_OP_FWD, p) == (B.GBCONV_OK, 0)
    s, n = B.gbconv_workspace_size(B.GBCONV_OP_DGRAD, p)
    assert s == B.GBCONV_OK and n == (128 * 9 * 128 * 2 + 255) // 256 * 256
    # stride 2 (BF16 NHWC): sub-pixel phases hold the transposed filter
    p2 = B.problem(32, 128, 56, 56, 128, 3, 3, 2, 1, 1)
    assert B.gbconv_workspace_size(B.GBCONV_OP_DGRAD, p2) == (B.GBCONV_OK, n)
    # FP32 NCHW runs on the CUDA-core kernel: no workspace
    p3 = B.problem(2, 8, 16, 16, 8, 3, 3, 2, 1, 1, B.GBCONV_F32, B.GBCONV_F32, B.GBCONV_NCHW)
    assert B.gbconv_workspace_size(B.GBCONV_OP_DGRAD, p3) == (B.GBCONV_OK, 0)
    s, n = B.gbconv_workspace_size(B.GBCONV_OP_WGRAD, p)
    s2, cfg = B.gbconv_get_config(B.GBCONV_OP_WGRAD, p)
    assert s == s2 == B.GBCONV_OK and cfg.split_k >= 1
    assert n >= (cfg.split_k * 128 * 128 * 9 + 128 * 128) * 4
    # too small a workspace is refused before anything runs
    assert B.conv2d_wgrad(p, 4096, 8192, 12288, 0, 16384, n - 256, 0) == B.GBCONV_ERR_WORKSPACE
    assert B.conv2d_dgrad(p, 4096, 8192, 12288, 16384, 16, 0) == B.GBCONV_ERR_WORKSPACE


def test_config_table_roundtrip(tmp_path):
    p = B.problem(8, 64, 28, 28, 128, 3, 3, 1, 1, 1)
    s, c0 = B.gbconv_get_config(B.GBCONV_OP_FWD, p)
    assert s == B.GBCONV_OK and c0.block_n in (32, 64, 128, 256) and c0.stages >= 2
    assert B.gbconv_set_config(B.GBCONV_OP_FWD, p, B.gbconv_config_t(64, 5, 1, 1)) == B.GBCONV_OK
    s, c1 = B.gbconv_get_config(B.GBCONV_OP_FWD, p)
    assert (c1.block_n, c1.stages, c1.raster) == (64, 5, 1)
    assert B.gbconv_set_config(B.GBCONV_OP_FWD, p, B.gbconv_config_t(48, 0, 0, 0)) == \
        B.GBCONV_ERR_INVALID_ARG
    path = str(tmp_path / "tune.json")
    assert B.gbconv_tune_cache_save(path) == B.GBCONV_OK
    B.gbconv_shutdown()
    s, c2 = B.gbconv_get_config(B.GBCONV_OP_FWD, p)
    assert (c2.block_n, c2.stages) == (c0.block_n, c0.stages)
    assert B.gbconv_tune_cache_load(path) == B.GBCONV_OK
    s, c3 = B.gbconv_get_config(B.GBCONV_OP_FWD, p)
    assert (c3.block_n, c3.stages, c3.raster) == (64, 5, 1)
    import json
    json.load(open(path))  # the file is valid JSON
    B.gbconv_shutdown()


def test_debug_controls():
    assert B.gbconv_debug_set(B.GBCONV_DEBUG_WAIT_LIMIT_NS, -5) == B.GBCONV_ERR_INVALID_ARG
    assert B.gbconv_debug_set(99, 0) == B.GBCONV_ERR_INVALID_ARG
    assert B.gbconv_debug_set(B.GBCONV_DEBUG_WAIT_LIMIT_NS, 0) == B.GBCONV_OK
    assert B.gbconv_debug_set(B.GBCONV_DEBUG_SKIP_LOADS, 0) == B.GBCONV_OK


def test_product_path_does_not_import_oracle():
    """The CUDA path and the oracle share no code: nothing in the package
    imports, links or opens anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_2207_00257_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "liboracle" not in text and "oracle.c" not in text, f
                assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", text), f
