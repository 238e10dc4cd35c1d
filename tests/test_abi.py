"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and exports
every entry point include/fgfrft.h declares; host-side argument checks need no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2602_20870_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fgfrft.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fgfrft_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["fgfrft_precompute", "fgfrft_assemble", "fgfrft_apply", "fgfrft_grad"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    from paper_2602_20870_gb300 import fgfrft
    assert sorted(fgfrft.SIGNATURES) == declared_functions()


def test_plan_bytes_layout(lib):
    f = lib.fgfrft_plan_bytes
    f.restype = ctypes.c_size_t
    f.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int]
    # status area + (2L+2) blocks of N*N padded to 32 entries, 8 bytes each
    N, L = 64, 16
    assert f(N, L, 1) == 256 + (2 * L + 2) * N * N * 8
    # split planes: 4 planes of N rows x round_up(N, 8), each padded to 128 entries, 2 bytes
    N = 65
    Np = 72
    plane = -(-(N * Np) // 128) * 128
    c64 = -(-((2 * L + 2) * (-(-(N * N) // 32) * 32) * 8) // 256) * 256
    assert f(N, L, 3) == 256 + c64 + -(-((2 * L + 2) * 4 * plane * 2) // 256) * 256
    # entry-major copy: 4 planes x Kp (2L+2 rounded up to 8) chunk columns x N*N entries
    # (padded to 128), 2 bytes
    Kp = -(-(2 * L + 2) // 8) * 8
    entry = -(-(4 * Kp * (-(-(N * N) // 128) * 128) * 2) // 256) * 256
    assert f(N, L, 7) == 256 + c64 + -(-((2 * L + 2) * 4 * plane * 2) // 256) * 256 + entry
    # half stack: M_0..M_L and P, L + 2 blocks of two FP32 planes of 64 x 64 tiles
    nt = -(-N // 64)
    assert f(N, L, 8) == 256 + -(-((L + 2) * 2 * nt * nt * 4096 * 4) // 256) * 256
    assert f(0, L, 1) == 0 and f(N, -1, 1) == 0 and f(N, L, 0) == 0 and f(N, L, 16) == 0 and f(N, L, 4) == 0


def test_strerror_and_version(lib):
    lib.fgfrft_strerror.restype = ctypes.c_char_p
    for code in range(8):
        assert lib.fgfrft_strerror(code).startswith(b"FGFRFT_")
    assert b"unknown" in lib.fgfrft_strerror(99)
    assert lib.fgfrft_version() >= 100


def test_host_argument_checks_without_gpu(lib):
    """Calls with invalid arguments return before touching the device."""
    from paper_2602_20870_gb300 import fgfrft as FG
    L = FG.load()
    h = ctypes.c_void_p()
    assert L.fgfrft_precompute(None, 64, 4, 1, None, 0, 0.0, None, None, 0, None, 0, None,
                               ctypes.byref(h)) == FG.ERR_INVALID_ARG
    # neg1_tol outside {0} U [1e-6, 0.5] is refused before anything else is looked at
    buf = ctypes.create_string_buffer(1 << 16)
    base = (ctypes.addressof(buf) + 255) // 256 * 256
    for tol in (-1.0, 1e-7, 0.6, float("nan")):
        assert L.fgfrft_precompute(ctypes.c_void_p(base), 4, 1, 1, None, 0, tol, None, ctypes.c_void_p(base),
                                   1 << 12, ctypes.c_void_p(base), 1 << 12, None, ctypes.byref(h)) == FG.ERR_INVALID_ARG
    # plan_info on no plan
    assert L.fgfrft_plan_info(None, None, None, None, None, None, None, None, None) == FG.ERR_INVALID_ARG
    assert L.fgfrft_apply(None, None, 1, 0, None, None, 0, None, 0, None) == FG.ERR_INVALID_ARG
    assert L.fgfrft_grad(None, None, 1, 0, None, None, None, None, None, None, 0, None, 0, None) == FG.ERR_INVALID_ARG
    assert L.fgfrft_assemble(None, None, 1, 0, None, None, 0, None) == FG.ERR_INVALID_ARG
    assert L.fgfrft_plan_destroy(None) == FG.ERR_INVALID_ARG


def test_binding_rejects_mismatched_tensors_before_the_call():
    """The binding checks dtype, contiguity, shape, size and device of the tensors it
    passes as raw pointers (a short or misread buffer would be accessed on the GPU)."""
    import pytest
    import torch
    from paper_2602_20870_gb300 import fgfrft as FG
    G = torch.zeros((3, 8), dtype=torch.complex64)
    D = torch.zeros((3, 8), dtype=torch.complex64)
    out = torch.zeros(3, dtype=torch.float32)
    cases = [
        (G.to(torch.complex128), D, out, "G must be torch.complex64"),
        (G, D.to(torch.complex128), out, "D must be torch.complex64"),
        (G, torch.zeros((3, 16), dtype=torch.complex64)[:, ::2], out, "D must be contiguous"),
        (G, torch.zeros((4, 8), dtype=torch.complex64), out, "D has shape"),
        (G, D, torch.zeros(2, dtype=torch.float32), "out has 2 elements"),
        (G, D, out.to(torch.float64), "out must be torch.float32"),
        (G, D, out, "G must be on a CUDA device"),
    ]
    for g, d, o, msg in cases:
        with pytest.raises(ValueError, match=msg):
            FG.grad_alpha_noalloc(g, d, o)
    with pytest.raises(ValueError, match="must be a"):
        FG.grad_alpha_noalloc(G[0], D, out)
