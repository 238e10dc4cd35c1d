"""Thin Python binding of libfgfrft (ctypes).

Argument marshalling only: every step of the transform runs in the library's
CUDA kernels.  PyTorch provides device memory and the current CUDA stream.
The library must have been built (``paper_2602_20870_gb300.build.build()``);
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from .build import LIB

# enum values mirrored from include/fgfrft.h
OK = 0
ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_NOT_UNITARY, ERR_AMBIGUOUS_SPECTRUM = 1, 2, 3, 4
ERR_NO_MEMORY, ERR_CUDA, ERR_TIMEOUT = 5, 6, 7
STORE_C64, STORE_SPLIT_F16, STORE_ENTRY_F16, STORE_HALF = 1, 2, 4, 8
ADJOINT, SHARED_ALPHA = 1, 2
REAL_SIGNALS, REAL_OUTPUT = 0x100, 0x200
PATH_PLAIN, PATH_ASSEMBLED, PATH_STACKED, PATH_STACKED_FP32 = 0x10, 0x20, 0x40, 0x80
OP_ASSEMBLE, OP_APPLY, OP_GRAD = 1, 2, 3

PATHS = {"auto": 0, "plain": PATH_PLAIN, "assembled": PATH_ASSEMBLED, "stacked": PATH_STACKED,
         "stacked_fp32": PATH_STACKED_FP32}

# exported entry points and their ctypes signatures
_vp, _i64, _i32, _sz, _dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
SIGNATURES = {
    "fgfrft_strerror": (ctypes.c_char_p, [_i32]),
    "fgfrft_version": (_i32, []),
    "fgfrft_plan_bytes": (_sz, [_i64, _i32, _i32]),
    "fgfrft_precompute_work_bytes": (_sz, [_i64]),
    "fgfrft_precompute": (_i32, [_vp, _i64, _i32, _i32, _vp, _i64, _dp, _vp, _vp, _sz, _vp, _sz, _vp,
                                 ctypes.POINTER(_vp)]),
    "fgfrft_plan_info": (_i32, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                                ctypes.POINTER(_i32), ctypes.POINTER(_dp), ctypes.POINTER(_i32),
                                ctypes.POINTER(_sz), ctypes.POINTER(_dp)]),
    "fgfrft_plan_block": (_vp, [_vp, _i32, _i32, ctypes.POINTER(_i64)]),
    "fgfrft_plan_status": (_i32, [_vp, _vp]),
    "fgfrft_plan_destroy": (_i32, [_vp]),
    "fgfrft_plan_real": (_i32, [_vp]),
    "fgfrft_plan_pair": (_i32, [_vp]),
    "fgfrft_work_bytes": (_sz, [_vp, _i32, _vp, _i64, _i32, _i32]),
    "fgfrft_assemble": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp, _sz, _vp]),
    "fgfrft_apply": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp, _i32, _vp, _sz, _vp]),
    "fgfrft_grad": (_i32, [_vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _sz, _vp]),
    "fgfrft_timing_enable": (_i32, [_i32]),
    "fgfrft_timing_reset": (_i32, []),
    "fgfrft_timing_read": (_i32, [_i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_dp)]),
    "fgfrft_grad_alpha_noalloc": (_i32, [_vp, _vp, _i64, _i64, _vp, _vp]),
    "fgfrft_check_wait_timeout": (_i32, [_vp, _vp]),
}

NOALLOC_MAX_PARTIALS = 65536


def _require(t, name: str, dtype, shape=None, min_numel=None):
    """Raise ValueError unless ``t`` is a contiguous tensor of ``dtype`` (and, when given, of
    ``shape``, with at least ``min_numel`` elements): the C calls take raw pointers and
    sizes, so a mismatch here would be misread on the device."""
    if not torch.is_tensor(t):
        raise ValueError(f"{name} must be a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if min_numel is not None and t.numel() < min_numel:
        raise ValueError(f"{name} has {t.numel()} elements, at least {min_numel} needed")


def _require_cuda(tensors: dict, device=None):
    """Raise ValueError unless every tensor is on one CUDA device (``device`` if given)."""
    for name, t in tensors.items():
        if t.device.type != "cuda":
            raise ValueError(f"{name} must be on a CUDA device, not {t.device}")
        want = device if device is not None else next(iter(tensors.values())).device
        if t.device != want:
            raise ValueError(f"{name} is on {t.device}, expected {want}")


def grad_alpha_noalloc(G: torch.Tensor, D: torch.Tensor, out: torch.Tensor, stream=None):
    """Re <G_j, D_j> per signal row into ``out`` (float32, B) with no device allocation:
    the library's fixed scratch holds the partial sums (see fgfrft_grad_alpha_noalloc).
    G and D: contiguous complex64 (B, N) on one CUDA device; out: contiguous float32 with
    at least B elements on the same device."""
    if not torch.is_tensor(G) or G.dim() != 2:
        raise ValueError("G must be a (B, N) tensor")
    B, N = G.shape
    _require(G, "G", torch.complex64)
    _require(D, "D", torch.complex64, shape=(B, N))
    _require(out, "out", torch.float32, min_numel=B)
    _require_cuda({"G": G, "D": D, "out": out})
    rc = _lib().fgfrft_grad_alpha_noalloc(_ptr(G), _ptr(D), B, N, _ptr(out), ctypes.c_void_p(_stream(stream)))
    _check(rc, "fgfrft_grad_alpha_noalloc")
    return out

# kernel classes (enum fgfrft_kernel_class)
KERNEL_CLASSES = ["coeffs", "assemble_single", "assemble_multi", "split_signals", "tc_gemm", "simt_gemm",
                  "grad_reduce", "offline"]


def timing_enable(on: bool = True):
    _check(_lib().fgfrft_timing_enable(1 if on else 0), "fgfrft_timing_enable")


def timing_reset():
    _check(_lib().fgfrft_timing_reset(), "fgfrft_timing_reset")


def timing_read() -> dict:
    """{class: (launches, timed_calls, total_ms)} for every kernel class (synchronises)."""
    out = {}
    for i, name in enumerate(KERNEL_CLASSES):
        n, t, ms = _i64(), _i64(), _dp()
        _check(_lib().fgfrft_timing_read(i, ctypes.byref(n), ctypes.byref(t), ctypes.byref(ms)), "fgfrft_timing_read")
        out[name] = (n.value, t.value, ms.value)
    return out


class FGFRFTError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {_lib().fgfrft_strerror(code).decode()} (status {code})")


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB):
            raise ImportError(f"libfgfrft.so is not built ({LIB}); run paper_2602_20870_gb300.build.build()")
        lib = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def load():
    """Load libfgfrft.so (raises ImportError if it is not built)."""
    return _lib()


def _check(rc: int, where: str):
    if rc != OK:
        raise FGFRFTError(rc, where)


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _alpha_array(alpha, count=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
    if count is not None and a.size == 1 and count > 1:
        a = np.full(count, float(a[0]))
    return a


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """Offline part of Algorithm 1 on the GPU, and the online calls on its stack.

    ``F`` is an N x N unitary matrix (numpy or torch, converted to complex128 on
    the device).  The plan's device memory is a torch uint8 tensor owned here.
    ``neg1_tol``: 0 classifies the lambda = -1 eigenvalues adaptively, a value in
    [1e-5, 0.5] counts |lambda + 1| below it as -1 (see fgfrft_precompute).
    ``keep_projector``: keep the FP64 projector (complex128 N x N, before rounding) in
    ``self.P64``.  ``self.min_gap`` = (lower, upper) bound of min |lambda + 1| over
    the complement.
    """

    def __init__(self, F, L_max: int, storage: int = STORE_C64 | STORE_SPLIT_F16 | STORE_ENTRY_F16, W=None,
                 device="cuda", stream=None, neg1_tol: float = 0.0, keep_projector: bool = False):
        lib = _lib()
        Ft = torch.as_tensor(np.asarray(F) if not torch.is_tensor(F) else F)
        Ft = Ft.to(device=device, dtype=torch.complex128).contiguous()
        N = Ft.shape[0]
        if Ft.shape != (N, N):
            raise ValueError("F must be square")
        self.N, self.L_max, self.storage, self.device = int(N), int(L_max), int(storage), torch.device(device)
        nbytes = lib.fgfrft_plan_bytes(N, L_max, storage)
        if nbytes == 0:
            raise FGFRFTError(ERR_INVALID_ARG, "fgfrft_plan_bytes")
        self.mem = torch.empty(nbytes, dtype=torch.uint8, device=device)
        wbytes = lib.fgfrft_precompute_work_bytes(N)
        work = torch.empty(wbytes, dtype=torch.uint8, device=device)
        Wt = None
        r = 0
        if W is not None:
            Wt = torch.as_tensor(np.asarray(W) if not torch.is_tensor(W) else W).to(
                device=device, dtype=torch.complex128).contiguous()
            r = Wt.shape[1] if Wt.ndim == 2 else 0
        self.P64 = torch.empty((N, N), dtype=torch.complex128, device=device) if keep_projector else None
        h = ctypes.c_void_p()
        rc = lib.fgfrft_precompute(_ptr(Ft), N, L_max, storage, _ptr(Wt), r, float(neg1_tol), _ptr(self.P64),
                                   _ptr(self.mem), nbytes, _ptr(work), wbytes, ctypes.c_void_p(_stream(stream)),
                                   ctypes.byref(h))
        _check(rc, "fgfrft_precompute")
        self._h = h
        del work
        n64, lm, st, rn, sq, pb = _i64(), _i32(), _i32(), _i32(), _i32(), _sz()
        res = _dp()
        gap = (_dp * 2)()
        _check(lib.fgfrft_plan_info(h, ctypes.byref(n64), ctypes.byref(lm), ctypes.byref(st), ctypes.byref(rn),
                                    ctypes.byref(res), ctypes.byref(sq), ctypes.byref(pb), gap), "fgfrft_plan_info")
        self.r_neg1, self.proj_residual, self.squarings, self.plan_bytes = rn.value, res.value, sq.value, pb.value
        self.min_gap = (gap[0], gap[1])
        self.real = lib.fgfrft_plan_real(h) == 1
        # the fused multi-order assembly reads the pair stack (real F without -1 eigenvalue)
        self.pair = lib.fgfrft_plan_pair(h) == 1
        # one work buffer per CUDA stream: calls on different streams never share scratch
        self._works = {}

    # ---------------------------------------------------------------- helpers
    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib().fgfrft_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream_of(self, stream):
        """(key, stream object) of the stream a call runs on; key 0 off CUDA (host tests)."""
        if self.device.type != "cuda":
            return 0, None
        st = stream if stream is not None else torch.cuda.current_stream(self.device)
        return st.cuda_stream, st

    def _with_work(self, op: int, alpha: np.ndarray, count: int, L: int, flags: int, call, stream=None) -> int:
        """call(w) -> status with the stream's cached work buffer; the buffer is sized (a host
        pass over the orders in fgfrft_work_bytes) only when the stream has none yet or the
        call reports it too small, which it does before enqueuing anything."""
        key, _ = self._stream_of(stream)
        w = self._works.get(key)
        if w is not None:
            rc = call(w)
            if rc != ERR_INVALID_ARG:
                return rc
            need = _lib().fgfrft_work_bytes(self._h, op, alpha.ctypes.data_as(ctypes.c_void_p), count, L, flags)
            if need == 0 or need <= w.numel():
                return rc  # an argument error, not the buffer size
        return call(self.work_tensor(op, alpha, count, L, flags, stream))

    def work_tensor(self, op: int, alpha: np.ndarray, count: int, L: int, flags: int, stream=None) -> torch.Tensor:
        """The work buffer of the stream (allocated on that stream, so the caching allocator
        hands its memory to nothing else while the stream's kernels may still use it)."""
        n = _lib().fgfrft_work_bytes(self._h, op, alpha.ctypes.data_as(ctypes.c_void_p), count, L, flags)
        if n == 0:
            # invalid request: the call itself reports the precise status before using the buffer
            n = 256
        key, st = self._stream_of(stream)
        w = self._works.get(key)
        if w is None or w.numel() < n:
            if st is not None:
                with torch.cuda.stream(st):
                    w = torch.empty(n, dtype=torch.uint8, device=self.device)
            else:
                w = torch.empty(n, dtype=torch.uint8, device=self.device)
            self._works[key] = w
        return w

    def block(self, l: int, storage: int = STORE_C64) -> torch.Tensor:
        """Stored block M_l (l in -L_max..L_max) or P (l = L_max + 1) as a device tensor view."""
        stride = _i64()
        ptr = _lib().fgfrft_plan_block(self._h, storage, l, ctypes.byref(stride))
        if not ptr:
            raise FGFRFTError(ERR_INVALID_ARG, "fgfrft_plan_block")
        base = self.mem.data_ptr()
        off = ptr - base
        if storage == STORE_HALF:
            # two FP32 planes of 64 x 64 tiles; element (r, c) of a tile at r * 64 + (c ^ (r & 31))
            nt = (self.N + 63) // 64
            planes = self.mem[off:off + stride.value * 4].view(torch.float32).view(2, nt, nt, 64, 64)
            r = torch.arange(64, device=planes.device)
            idx = (r[None, :] ^ (r[:, None] & 31)).expand(2, nt, nt, 64, 64)
            tiles = torch.gather(planes, 4, idx)
            full = tiles.permute(0, 1, 3, 2, 4).reshape(2, nt * 64, nt * 64)[:, :self.N, :self.N]
            return torch.complex(full[0], full[1])
        if storage == STORE_C64:
            nbytes = self.N * self.N * 8
            return self.mem[off:off + nbytes].view(torch.complex64).view(self.N, self.N)
        Np = (self.N + 7) // 8 * 8
        pe = stride.value // 4
        planes = self.mem[off:off + stride.value * 2].view(torch.float16).view(4, pe)
        return planes[:, : self.N * Np].reshape(4, self.N, Np)[:, :, : self.N]

    def check_wait_timeout(self, stream=None):
        """Run the bounded-wait failure path once (fgfrft_check_wait_timeout); the next
        ``status()`` reports FGFRFT_ERR_TIMEOUT."""
        _check(_lib().fgfrft_check_wait_timeout(self._h, ctypes.c_void_p(_stream(stream))),
               "fgfrft_check_wait_timeout")

    def status(self, stream=None):
        _check(_lib().fgfrft_plan_status(self._h, ctypes.c_void_p(_stream(stream))), "fgfrft_plan_status")

    # ---------------------------------------------------------------- online
    def assemble(self, alpha, L: int | None = None, out: torch.Tensor | None = None, stream=None):
        """Q_L^{alpha_a} for each order (Def. 1), complex64 (A, N, N)."""
        L = self.L_max if L is None else int(L)
        a = _alpha_array(alpha)
        A = a.size
        if out is None:
            out = torch.empty((A, self.N, self.N), dtype=torch.complex64, device=self.device)
        rc = self._with_work(OP_ASSEMBLE, a, A, L, 0, lambda w: _lib().fgfrft_assemble(
            self._h, a.ctypes.data_as(ctypes.c_void_p), A, L, _ptr(out), _ptr(w), w.numel(),
            ctypes.c_void_p(_stream(stream))), stream)
        _check(rc, "fgfrft_assemble")
        return out

    def apply(self, alpha, X: torch.Tensor, L: int | None = None, adjoint: bool = False, path: str = "auto",
              out: torch.Tensor | None = None, stream=None, real_io: bool = False, real_output: bool = False):
        """Y[j] = Q_L^{alpha_j} X[j] (Def. 2), X of shape (B, N), one signal per row.

        A CPU ``X`` is copied to the device and the result copied back (end to end).
        ``real_io``: X is passed as real float32 signals (half the bytes of complex64; the
        tensor-core paths read it directly); ``real_output`` (with ``real_io``): Y is
        real float32, for a real F without a -1 eigenvalue (Q is then real)."""
        L = self.L_max if L is None else int(L)
        host = X.device.type == "cpu"
        xdt = torch.float32 if real_io else torch.complex64
        Xd = X.to(self.device, dtype=xdt, non_blocking=True).contiguous() if host or X.dtype != xdt \
            else X.contiguous()
        B = Xd.shape[0]
        a = _alpha_array(alpha, B)
        flags = PATHS[path] | (ADJOINT if adjoint else 0) | (REAL_SIGNALS if real_io else 0) | \
            (REAL_OUTPUT if real_io and real_output else 0)
        ydt = torch.float32 if (real_io and real_output) else torch.complex64
        Y = torch.empty(Xd.shape, dtype=ydt, device=self.device) if (out is None or host) else out
        rc = self._with_work(OP_APPLY, a, B, L, flags, lambda w: _lib().fgfrft_apply(
            self._h, a.ctypes.data_as(ctypes.c_void_p), B, L, _ptr(Xd), _ptr(Y), flags, _ptr(w), w.numel(),
            ctypes.c_void_p(_stream(stream))), stream)
        _check(rc, "fgfrft_apply")
        if host:
            dst = out if out is not None else torch.empty(Y.shape, dtype=Y.dtype, pin_memory=True)
            dst.copy_(Y, non_blocking=True)
            return dst
        return Y

    def forward_dual(self, alpha, X: torch.Tensor, L: int | None = None, path: str = "auto", stream=None):
        """(Y, dY/dalpha) from one pass over the stored powers (Prop. 3)."""
        L = self.L_max if L is None else int(L)
        X = X.contiguous()
        if X.dim() != 2 or X.shape[1] != self.N:
            raise ValueError(f"X must be (B, {self.N})")
        _require(X, "X", torch.complex64)
        _require_cuda({"X": X})
        B = X.shape[0]
        a = _alpha_array(alpha, B)
        flags = PATHS[path]
        Y = torch.empty_like(X)
        D = torch.empty_like(X)
        rc = self._with_work(OP_GRAD, a, B, L, flags, lambda w: _lib().fgfrft_grad(
            self._h, a.ctypes.data_as(ctypes.c_void_p), B, L, _ptr(X), _ptr(Y), _ptr(D), None, None, None, flags,
            _ptr(w), w.numel(), ctypes.c_void_p(_stream(stream))), stream)
        _check(rc, "fgfrft_grad(forward)")
        return Y, D

    def backward(self, alpha, G: torch.Tensor, D: torch.Tensor | None, L: int | None = None,
                 need_x: bool = True, path: str = "auto", stream=None, shared: bool = False):
        """(Q^H G, Re <G, D> per column) (Props. 2-3 and the chain rule).  ``shared``: one
        order for every column; the library then returns the one gradient of that order
        (the sum over the columns) as a 1-element tensor."""
        L = self.L_max if L is None else int(L)
        G = G.contiguous()
        if G.dim() != 2 or G.shape[1] != self.N:
            raise ValueError(f"G must be (B, {self.N})")
        B = G.shape[0]
        _require(G, "G", torch.complex64)
        if D is not None:
            _require(D, "D", torch.complex64, shape=(B, self.N))
        _require_cuda({"G": G, "D": D} if D is not None else {"G": G})
        a = _alpha_array(alpha, B)
        if shared:
            a = a[:1]
        flags = PATHS[path] | (SHARED_ALPHA if shared else 0)
        gX = torch.empty_like(G) if need_x else None
        ga = torch.empty(1 if shared else B, dtype=torch.float32, device=G.device) if D is not None else None
        rc = self._with_work(OP_GRAD, a, B, L, flags, lambda w: _lib().fgfrft_grad(
            self._h, a.ctypes.data_as(ctypes.c_void_p), B, L, None, None, _ptr(D), _ptr(G), _ptr(gX), _ptr(ga),
            flags, _ptr(w), w.numel(), ctypes.c_void_p(_stream(stream))), stream)
        _check(rc, "fgfrft_grad(backward)")
        return gX, ga


class Pipeline:
    """Streams host batches through ``Plan.apply``: the copy of batch k+1 to the device,
    the transform of batch k and the copy of batch k-1 back to the host run on three
    CUDA streams at once, with two device buffers per side.  ``submit`` returns at once;
    ``wait`` blocks until every submitted batch is back in its host buffer.  ``real_io`` /
    ``real_output`` as in ``Plan.apply`` (real float32 host buffers)."""

    def __init__(self, plan: Plan, shape, L: int | None = None, path: str = "auto", real_io: bool = False,
                 real_output: bool = False):
        self.plan, self.L, self.path = plan, plan.L_max if L is None else int(L), path
        self.real_io, self.real_output = real_io, real_io and real_output
        dev = plan.device
        self.s_in, self.s_run, self.s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        xdt = torch.float32 if real_io else torch.complex64
        ydt = torch.float32 if self.real_output else torch.complex64
        self.X = [torch.empty(shape, dtype=xdt, device=dev) for _ in range(2)]
        self.Y = [torch.empty(shape, dtype=ydt, device=dev) for _ in range(2)]
        self.ev_in = [torch.cuda.Event() for _ in range(2)]
        self.ev_run = [torch.cuda.Event() for _ in range(2)]
        self.ev_out = [torch.cuda.Event() for _ in range(2)]
        self.k = 0

    def submit(self, alpha, Xh: torch.Tensor, Yh: torch.Tensor):
        """Enqueue Yh = Q X for pinned host tensors Xh, Yh."""
        b = self.k % 2
        if self.k >= 2:
            self.s_in.wait_event(self.ev_run[b])    # X[b] no longer read by batch k-2
            self.s_run.wait_event(self.ev_out[b])   # Y[b] already copied out
        with torch.cuda.stream(self.s_in):
            self.X[b].copy_(Xh, non_blocking=True)
            self.ev_in[b].record(self.s_in)
        self.s_run.wait_event(self.ev_in[b])
        with torch.cuda.stream(self.s_run):
            self.plan.apply(alpha, self.X[b], self.L, path=self.path, out=self.Y[b], stream=self.s_run,
                            real_io=self.real_io, real_output=self.real_output)
            self.ev_run[b].record(self.s_run)
        self.s_out.wait_event(self.ev_run[b])
        with torch.cuda.stream(self.s_out):
            Yh.copy_(self.Y[b], non_blocking=True)
            self.ev_out[b].record(self.s_out)
        self.k += 1

    def wait(self):
        self.s_out.synchronize()


class FGFRFTFunction(torch.autograd.Function):
    """Y = Q_L^{alpha} X with a hand-written backward (Props. 2-3).

    alpha: float64 tensor of shape (B,) (one order per signal row of X) or (1,);
    X: complex64 (B, N) on the plan's device.  The forward computes Y and dY/dalpha
    in one pass; the backward returns Q^H G and Re <G, dY/dalpha>."""

    @staticmethod
    def forward(ctx, alpha: torch.Tensor, X: torch.Tensor, plan: Plan, L: int, path: str = "auto"):
        B = X.shape[0]
        a = alpha.detach().to("cpu", torch.float64).numpy()
        Y, D = plan.forward_dual(a, X, L, path)
        ctx.plan, ctx.L, ctx.path, ctx.a = plan, L, path, a
        ctx.alpha_device, ctx.alpha_dtype = alpha.device, alpha.dtype
        ctx.shared = alpha.numel() == 1 and B > 1
        ctx.alpha_shape = alpha.shape
        ctx.save_for_backward(D)
        return Y

    @staticmethod
    def backward(ctx, G):
        (D,) = ctx.saved_tensors
        need_x = ctx.needs_input_grad[1]
        # a shared order: the library sums the per-column gradients into one value
        gX, ga = ctx.plan.backward(ctx.a, G.to(torch.complex64).contiguous(), D, ctx.L, need_x, ctx.path,
                                   shared=ctx.shared)
        galpha = None
        if ctx.needs_input_grad[0]:
            galpha = ga.to(device=ctx.alpha_device, dtype=ctx.alpha_dtype).reshape(ctx.alpha_shape)
        return galpha, gX, None, None, None


def fgfrft(alpha: torch.Tensor, X: torch.Tensor, plan: Plan, L: int | None = None, path: str = "auto"):
    """Differentiable FGFRFT: Q_L^{alpha} X (autograd through alpha and X)."""
    return FGFRFTFunction.apply(alpha, X, plan, plan.L_max if L is None else int(L), path)
