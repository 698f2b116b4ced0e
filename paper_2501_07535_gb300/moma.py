"""Thin ctypes binding of libmoma.so (include/moma.h), same names as the C ABI.

Argument marshalling only: every step of the arithmetic runs in the library's CUDA
kernels.  PyTorch supplies device memory (tensors are passed by data pointer) and
streams.  If the shared library is missing the import of this module still works, but
the first call raises: there is no CPU fallback.

Vectors are torch tensors on the GPU with dtype int32 or uint32 holding the raw 32-bit
limbs, shape (L, n) limb-major (limb 0 least significant), or (count, L, n) for the
batched transforms.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import inputs

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmoma.so")

STATUS = {0: "MOMA_OK", 1: "MOMA_ERR_INVALID_ARG", 2: "MOMA_ERR_MODULUS", 3: "MOMA_ERR_SIZE",
          4: "MOMA_ERR_ALIGN", 5: "MOMA_ERR_OOM", 6: "MOMA_ERR_CUDA", 7: "MOMA_ERR_TIMEOUT",
          8: "MOMA_ERR_BUDGET", 9: "MOMA_ERR_UNSUPPORTED"}
MOMA_OK = 0


class MomaError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


_lib = None

_P = ctypes.c_void_p
_SZ = ctypes.c_size_t
_SIGS = {
    "moma_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "moma_ctx_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "moma_ctx_create_full": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "moma_ctx_is_full": (ctypes.c_int, [_P]),
    "moma_ctx_destroy": (None, [_P]),
    "moma_ctx_limbs": (ctypes.c_int, [_P]),
    "moma_ctx_device_bytes": (ctypes.c_size_t, [_P]),
    "moma_ctx_root": (ctypes.c_int, [_P, _SZ, _P]),
    "moma_ctx_sync_status": (ctypes.c_int, [_P]),
    "moma_ctx_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "moma_ctx_inject_missing_copy": (ctypes.c_int, [_P]),
    "moma_vec_addmod": (ctypes.c_int, [_P, _SZ, _P, _P, _P, _P]),
    "moma_vec_submod": (ctypes.c_int, [_P, _SZ, _P, _P, _P, _P]),
    "moma_vec_mulmod": (ctypes.c_int, [_P, _SZ, _P, _P, _P, _P]),
    "moma_vec_axpymod": (ctypes.c_int, [_P, _SZ, _P, _P, _P, _P, _P]),
    "moma_ntt_fwd": (ctypes.c_int, [_P, _SZ, _P, _P, _P]),
    "moma_ntt_inv": (ctypes.c_int, [_P, _SZ, _P, _P, _P]),
    "moma_ntt_fwd_many": (ctypes.c_int, [_P, _SZ, _SZ, _P, _P, _P]),
    "moma_ntt_inv_many": (ctypes.c_int, [_P, _SZ, _SZ, _P, _P, _P]),
    "moma_polymul": (ctypes.c_int, [_P, _SZ, _P, _P, _P, _P]),
    "moma_probe_imad": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "moma_ctx_set_config": (ctypes.c_int, [_P, ctypes.c_int, _SZ, _P]),
    "moma_ctx_get_config": (ctypes.c_int, [_P, ctypes.c_int, _SZ, _P]),
    "moma_autotune": (ctypes.c_int, [_P, ctypes.c_int, _SZ, _SZ, _P, _P, ctypes.POINTER(ctypes.c_double)]),
    "moma_ntt_fwd_noalloc": (ctypes.c_int, [_P, _SZ, _P, _P, _P]),
    "moma_word_probe": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _SZ, _P, _P, _P, _P]),
    "moma_ntt_fwd_negacyclic": (ctypes.c_int, [_P, _SZ, _SZ, _P, _P, _P]),
    "moma_ntt_inv_negacyclic": (ctypes.c_int, [_P, _SZ, _SZ, _P, _P, _P]),
    "moma_polymul_negacyclic": (ctypes.c_int, [_P, _SZ, _P, _P, _P, _P]),
    "moma_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "moma_batch_run": (ctypes.c_int, [_P, _P]),
    "moma_batch_sync_status": (ctypes.c_int, [_P]),
    "moma_batch_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "moma_batch_inject_missing_dependency": (ctypes.c_int, [_P]),
    "moma_batch_destroy": (None, [_P]),
    "moma_batch_submit": (ctypes.c_int, [_P, ctypes.c_int, _P]),
}

OPS = {"ntt_fwd": 0, "ntt_inv": 1, "polymul": 2, "add": 3, "sub": 4, "mul": 5, "axpy": 6}


class moma_job(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("ctx", _P), ("n", _SZ), ("a", _P), ("b", _P), ("out", _P), ("alpha", _P)]


class moma_config(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_int), ("tile_log", ctypes.c_int), ("max_logr", ctypes.c_int),
                ("vec_width", ctypes.c_int), ("cta_threads", ctypes.c_int), ("tight_regs", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib() -> ctypes.CDLL:
    """Load libmoma.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2501_07535_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(code: int, what: str):
    if code != MOMA_OK:
        raise MomaError(code, what)


_current_stream = None  # () -> raw handle of torch's current stream on the current device


def _current_stream_handle() -> int:
    """torch's current stream as a raw handle.  The public route (torch.cuda.current_stream())
    costs about 12 us per call on the GPU machine's host cores, a share of a small transform call,
    so the two C entry points behind it are used directly when this torch has them."""
    global _current_stream
    if _current_stream is None:
        import torch
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        dev = getattr(torch._C, "_cuda_getDevice", None)
        if raw is not None and dev is not None:
            _current_stream = lambda: raw(dev())  # noqa: E731
        else:
            _current_stream = lambda: torch.cuda.current_stream().cuda_stream  # noqa: E731
    return _current_stream()


def _stream_handle(stream) -> int | None:
    if stream is None:
        return _current_stream_handle()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise TypeError("expected int32/uint32 limbs")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _limbs_array(x: int, L: int):
    arr = (ctypes.c_uint32 * L)(*inputs.int_to_limbs(x, L))
    return arr


# ----------------------------------------------------------------- C-ABI names

def moma_status_string(code: int) -> str:
    return lib().moma_status_string(code).decode()


def moma_ctx_create(q: int, bits: int) -> int:
    L = bits // 32
    h = _P()
    qa = _limbs_array(q, L)
    _check(lib().moma_ctx_create(ctypes.cast(qa, _P), bits, ctypes.byref(h)), "moma_ctx_create")
    return h.value


def moma_ctx_create_full(q: int, bits: int) -> int:
    """Context for a full-width modulus (Montgomery reduction)."""
    L = bits // 32
    h = _P()
    qa = _limbs_array(q, L)
    _check(lib().moma_ctx_create_full(ctypes.cast(qa, _P), bits, ctypes.byref(h)), "moma_ctx_create_full")
    return h.value


def moma_ctx_is_full(ctx: int) -> int:
    return lib().moma_ctx_is_full(ctx)


def moma_ctx_destroy(ctx: int):
    lib().moma_ctx_destroy(ctx)


def moma_ctx_limbs(ctx: int) -> int:
    return lib().moma_ctx_limbs(ctx)


def moma_ctx_device_bytes(ctx: int) -> int:
    return lib().moma_ctx_device_bytes(ctx)


def moma_ctx_root(ctx: int, n: int) -> int:
    L = moma_ctx_limbs(ctx)
    out = (ctypes.c_uint32 * L)()
    _check(lib().moma_ctx_root(ctx, n, ctypes.cast(out, _P)), "moma_ctx_root")
    return inputs.limbs_to_int(list(out))


def moma_ctx_sync_status(ctx: int) -> int:
    return lib().moma_ctx_sync_status(ctx)


def moma_ctx_set_wait_limit(ctx: int, ns: int):
    _check(lib().moma_ctx_set_wait_limit(ctx, ns), "moma_ctx_set_wait_limit")


def moma_ctx_inject_missing_copy(ctx: int):
    _check(lib().moma_ctx_inject_missing_copy(ctx), "moma_ctx_inject_missing_copy")


def moma_vec_addmod(ctx, n, a, b, c, stream=None):
    _check(lib().moma_vec_addmod(ctx, n, _ptr(a), _ptr(b), _ptr(c), _stream_handle(stream)), "moma_vec_addmod")


def moma_vec_submod(ctx, n, a, b, c, stream=None):
    _check(lib().moma_vec_submod(ctx, n, _ptr(a), _ptr(b), _ptr(c), _stream_handle(stream)), "moma_vec_submod")


def moma_vec_mulmod(ctx, n, a, b, c, stream=None):
    _check(lib().moma_vec_mulmod(ctx, n, _ptr(a), _ptr(b), _ptr(c), _stream_handle(stream)), "moma_vec_mulmod")


def moma_vec_axpymod(ctx, n, alpha: int, x, y, out, stream=None):
    al = _limbs_array(alpha, moma_ctx_limbs(ctx))
    _check(lib().moma_vec_axpymod(ctx, n, ctypes.cast(al, _P), _ptr(x), _ptr(y), _ptr(out),
                                  _stream_handle(stream)), "moma_vec_axpymod")


def moma_ntt_fwd(ctx, n, x, y, stream=None):
    _check(lib().moma_ntt_fwd(ctx, n, _ptr(x), _ptr(y), _stream_handle(stream)), "moma_ntt_fwd")


def moma_ntt_inv(ctx, n, x, y, stream=None):
    _check(lib().moma_ntt_inv(ctx, n, _ptr(x), _ptr(y), _stream_handle(stream)), "moma_ntt_inv")


def moma_ntt_fwd_many(ctx, n, count, x, y, stream=None):
    _check(lib().moma_ntt_fwd_many(ctx, n, count, _ptr(x), _ptr(y), _stream_handle(stream)), "moma_ntt_fwd_many")


def moma_ntt_inv_many(ctx, n, count, x, y, stream=None):
    _check(lib().moma_ntt_inv_many(ctx, n, count, _ptr(x), _ptr(y), _stream_handle(stream)), "moma_ntt_inv_many")


def moma_ntt_fwd_noalloc(ctx, n, x, y, stream=None):
    """Forward NTT without device allocation (scratch in a fixed array of the library).

    For callers that may not allocate device memory at call time.  n*L <= 2^20; call
    moma_ntt_fwd once for this context and n first (it builds the twiddle tables)."""
    _check(lib().moma_ntt_fwd_noalloc(ctx, n, _ptr(x), _ptr(y), _stream_handle(stream)), "moma_ntt_fwd_noalloc")


def moma_polymul(ctx, n, a, b, c, stream=None):
    _check(lib().moma_polymul(ctx, n, _ptr(a), _ptr(b), _ptr(c), _stream_handle(stream)), "moma_polymul")


def moma_ntt_fwd_negacyclic(ctx, n, x, y, count=1, stream=None):
    """Forward transform over Z_q[x]/(x^n + 1): y[k] = x evaluated at psi^(2k+1)."""
    _check(lib().moma_ntt_fwd_negacyclic(ctx, n, count, _ptr(x), _ptr(y), _stream_handle(stream)),
           "moma_ntt_fwd_negacyclic")


def moma_ntt_inv_negacyclic(ctx, n, x, y, count=1, stream=None):
    _check(lib().moma_ntt_inv_negacyclic(ctx, n, count, _ptr(x), _ptr(y), _stream_handle(stream)),
           "moma_ntt_inv_negacyclic")


def moma_polymul_negacyclic(ctx, n, a, b, c, stream=None):
    """c = a * b mod (x^n + 1, q)."""
    _check(lib().moma_polymul_negacyclic(ctx, n, _ptr(a), _ptr(b), _ptr(c), _stream_handle(stream)),
           "moma_polymul_negacyclic")


WORD_OPS = {"add": 0, "sub": 1, "mul": 2, "mul_hi": 3, "barrett": 4, "fixed": 5, "mont": 6, "barrett_full": 7}


def moma_word_probe(ctx, op, engine, n, a, b, out, stream=None):
    """Raw outputs of one word-level block (op a name of WORD_OPS or its code); out: (2L+1) x n."""
    code = WORD_OPS[op] if isinstance(op, str) else int(op)
    _check(lib().moma_word_probe(ctx, code, engine, n, _ptr(a), _ptr(b), _ptr(out), _stream_handle(stream)),
           "moma_word_probe")


def moma_probe_imad(variant: int, blocks: int, threads: int, iters: int):
    ms = ctypes.c_double()
    cnt = ctypes.c_double()
    _check(lib().moma_probe_imad(variant, blocks, threads, iters, ctypes.byref(ms), ctypes.byref(cnt)),
           "moma_probe_imad")
    return ms.value, cnt.value


def _op(op) -> int:
    return OPS[op] if isinstance(op, str) else int(op)


def moma_ctx_set_config(ctx, op, n, engine=0, tile_log=0, max_logr=0, vec_width=0, cta_threads=0, tight_regs=0):
    cfg = moma_config(engine, tile_log, max_logr, vec_width, cta_threads, tight_regs)
    _check(lib().moma_ctx_set_config(ctx, _op(op), n, ctypes.byref(cfg)), "moma_ctx_set_config")


def moma_ctx_get_config(ctx, op, n) -> dict:
    cfg = moma_config()
    _check(lib().moma_ctx_get_config(ctx, _op(op), n, ctypes.byref(cfg)), "moma_ctx_get_config")
    return cfg.as_dict()


def moma_autotune(ctx, op, n, count=1, stream=None):
    """Time every candidate schedule of `op` at size n; the context keeps the fastest."""
    cfg = moma_config()
    us = ctypes.c_double()
    _check(lib().moma_autotune(ctx, _op(op), n, count, _stream_handle(stream), ctypes.byref(cfg),
                               ctypes.byref(us)), "moma_autotune")
    return cfg.as_dict(), us.value


def _jobs_array(jobs):
    """jobs: list of dicts {op, ctx, n, a, b, out, alpha}; tensors or raw pointers."""
    arr = (moma_job * len(jobs))()
    keep = []
    for i, j in enumerate(jobs):
        def p(x):
            if x is None:
                return None
            return x if isinstance(x, int) else _ptr(x)
        alpha = None
        if j.get("alpha") is not None:
            al = _limbs_array(j["alpha"], moma_ctx_limbs(j["ctx"]))
            keep.append(al)
            alpha = ctypes.cast(al, _P)
        arr[i] = moma_job(_op(j["op"]), j["ctx"], j["n"], p(j["a"]), p(j.get("b")), p(j["out"]), alpha)
    return arr, keep


def moma_batch_create(jobs) -> int:
    arr, keep = _jobs_array(jobs)
    h = _P()
    _check(lib().moma_batch_create(ctypes.cast(arr, _P), len(jobs), ctypes.byref(h)), "moma_batch_create")
    return h.value


def moma_batch_run(batch, stream=None):
    _check(lib().moma_batch_run(batch, _stream_handle(stream)), "moma_batch_run")


def moma_batch_sync_status(batch) -> int:
    return lib().moma_batch_sync_status(batch)


def moma_batch_set_wait_limit(batch, polls: int):
    _check(lib().moma_batch_set_wait_limit(batch, polls), "moma_batch_set_wait_limit")


def moma_batch_inject_missing_dependency(batch):
    _check(lib().moma_batch_inject_missing_dependency(batch), "moma_batch_inject_missing_dependency")


def moma_batch_destroy(batch):
    lib().moma_batch_destroy(batch)


def moma_batch_submit(jobs, stream=None) -> int:
    arr, keep = _jobs_array(jobs)
    return lib().moma_batch_submit(ctypes.cast(arr, _P), len(jobs), _stream_handle(stream))


# ----------------------------------------------------------------- conveniences

def to_device(arr: np.ndarray, device="cuda"):
    """uint32 numpy array -> int32 CUDA tensor with the same bits."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint32).view(np.int32)).to(device)


def to_host(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


class Context:
    """Owns one moma_ctx (one modulus)."""

    def __init__(self, q: int, bits: int):
        self.q = q
        self.bits = bits
        self.L = bits // 32
        self.handle = moma_ctx_create(q, bits)

    def close(self):
        if self.handle:
            moma_ctx_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def root(self, n: int) -> int:
        return moma_ctx_root(self.handle, n)

    def sync_status(self) -> int:
        return moma_ctx_sync_status(self.handle)

    def _out(self, like, out):
        import torch
        return torch.empty_like(like) if out is None else out

    def addmod(self, a, b, out=None, stream=None):
        out = self._out(a, out)
        moma_vec_addmod(self.handle, a.shape[-1], a, b, out, stream)
        return out

    def submod(self, a, b, out=None, stream=None):
        out = self._out(a, out)
        moma_vec_submod(self.handle, a.shape[-1], a, b, out, stream)
        return out

    def mulmod(self, a, b, out=None, stream=None):
        out = self._out(a, out)
        moma_vec_mulmod(self.handle, a.shape[-1], a, b, out, stream)
        return out

    def axpy(self, alpha: int, x, y, out=None, stream=None):
        out = self._out(x, out)
        moma_vec_axpymod(self.handle, x.shape[-1], alpha, x, y, out, stream)
        return out

    def ntt(self, x, out=None, inverse=False, stream=None):
        out = self._out(x, out)
        n = x.shape[-1]
        if x.dim() == 3:
            (moma_ntt_inv_many if inverse else moma_ntt_fwd_many)(self.handle, n, x.shape[0], x, out, stream)
        else:
            (moma_ntt_inv if inverse else moma_ntt_fwd)(self.handle, n, x, out, stream)
        return out

    def intt(self, x, out=None, stream=None):
        return self.ntt(x, out, inverse=True, stream=stream)

    def polymul(self, a, b, out=None, stream=None):
        out = self._out(a, out)
        moma_polymul(self.handle, a.shape[-1], a, b, out, stream)
        return out
