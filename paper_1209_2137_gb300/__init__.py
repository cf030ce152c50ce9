"""icx: GPU decoding of SIMD-BP128 / SIMD-FastPFOR streams (Lemire & Boytsov,
"Decoding billions of integers per second through vectorization").

A thin ctypes binding over the C ABI of ``libicx.so`` (declared in
``include/icx.h``).  It only marshals arguments: every step of decoding and
encoding runs in the library's CUDA kernels.  PyTorch supplies device memory
and streams.  If the compiled library is missing, every call raises
``IcxError`` -- there is no CPU fallback.

Integer arrays are ``torch.uint32`` tensors (bit patterns of the paper's
unsigned 32-bit integers); streams are ``torch.uint8``; indexes
``torch.uint64``.  All device tensors must be contiguous and 16-byte aligned.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG_DIR, "libicx.so")

OK, EINVAL, EALIGN, ECORRUPT, ENOSPC, ECUDA, ETIMEOUT = range(7)
STATUS_NAMES = {0: "ICX_OK", 1: "ICX_EINVAL", 2: "ICX_EALIGN", 3: "ICX_ECORRUPT", 4: "ICX_ENOSPC",
                5: "ICX_ECUDA", 6: "ICX_ETIMEOUT"}
DELTA_NONE, DELTA_1, DELTA_4 = 0, 1, 4
FMT_PAPER, FMT_W32 = 0, 1

_lock = threading.Lock()
_lib = None


class IcxError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}")
        self.code = code


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libicx.so for sm_103a (nvcc; no GPU needed)."""
    from . import builder as _b
    return _b.build(force=force, verbose=verbose)


def lib():
    """The loaded C library; raises IcxError if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise IcxError(ECUDA, f"CUDA library not built ({LIB_PATH} missing); "
                                      "run paper_1209_2137_gb300.build()")
            L = ctypes.CDLL(LIB_PATH)
            sz, vp, i = ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int
            sig = {
                "icx_bp128_index_len": ([sz], sz),
                "icx_fastpfor_index_len": ([sz], sz),
                "icx_bp128_max_bytes": ([sz, i], sz),
                "icx_fastpfor_max_bytes": ([sz], sz),
                "icx_workspace_bytes": ([sz], sz),
                "icx_encode_workspace_bytes": ([sz], sz),
                "icx_workspace_init": ([vp, sz, vp], i),
                "icx_status_read": ([vp, vp, ctypes.POINTER(ctypes.c_int)], i),
                "bp128_index": ([vp, sz, sz, i, vp, vp, sz, vp], i),
                "fastpfor_index": ([vp, sz, sz, vp, vp, sz, vp], i),
                "bp128_decode": ([vp, sz, vp, sz, i, i, vp, vp, sz, vp], i),
                "fastpfor_decode": ([vp, sz, vp, sz, i, vp, vp, sz, vp], i),
                "delta_decode": ([vp, vp, sz, i, vp, sz, vp], i),
                "delta_encode": ([vp, vp, sz, i, vp], i),
                "bp128_encode": ([vp, sz, i, i, vp, sz, vp, vp, vp, sz, vp], i),
                "fastpfor_encode": ([vp, sz, i, vp, sz, vp, vp, vp, sz, vp], i),
                "icx_version": ([], ctypes.c_char_p),
                "icx_set_tuning": ([ctypes.c_char_p, i], i),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes, fn.restype = args, res
            _lib = L
    return _lib


EXPORTED = ("icx_bp128_index_len", "icx_fastpfor_index_len", "icx_bp128_max_bytes", "icx_fastpfor_max_bytes",
            "icx_workspace_bytes", "icx_encode_workspace_bytes", "icx_workspace_init", "icx_status_read",
            "bp128_index", "fastpfor_index", "bp128_decode", "fastpfor_decode", "delta_decode", "delta_encode",
            "bp128_encode", "fastpfor_encode", "icx_version", "icx_set_tuning")


def _check(code: int, what: str):
    if code != OK:
        raise IcxError(code, what)


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype, what):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise IcxError(EINVAL, f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise IcxError(EINVAL, f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise IcxError(EINVAL, f"{what} must be contiguous")
    return t


# -- sizes -------------------------------------------------------------------

def bp128_index_len(n: int) -> int:
    return lib().icx_bp128_index_len(n)


def fastpfor_index_len(n: int) -> int:
    return lib().icx_fastpfor_index_len(n)


def bp128_max_bytes(n: int, fmt: int = FMT_PAPER) -> int:
    return lib().icx_bp128_max_bytes(n, fmt)


def fastpfor_max_bytes(n: int) -> int:
    return lib().icx_fastpfor_max_bytes(n)


def workspace_bytes(n: int) -> int:
    return lib().icx_workspace_bytes(n)


def encode_workspace_bytes(n: int) -> int:
    return lib().icx_encode_workspace_bytes(n)


class Workspace:
    """Device workspace of a decode (look-back tile states + status word).

    Initialised once on creation; it resets itself after every launch.  One
    workspace serves one stream at a time."""

    def __init__(self, n: int, device=None, stream=None, encode: bool = False):
        import torch
        self.n = n
        self.bytes = encode_workspace_bytes(n) if encode else workspace_bytes(n)
        self.tensor = torch.empty(self.bytes, dtype=torch.uint8, device=device or "cuda")
        _check(lib().icx_workspace_init(_ptr(self.tensor), self.bytes, _stream(stream)), "icx_workspace_init")

    def ptr(self):
        return _ptr(self.tensor)

    def status(self, stream=None) -> int:
        """Synchronises the stream, returns and clears the status word."""
        out = ctypes.c_int(0)
        _check(lib().icx_status_read(self.ptr(), _stream(stream), ctypes.byref(out)), "icx_status_read")
        return out.value

    def raise_status(self, what="decode", stream=None):
        st = self.status(stream)
        if st != OK:
            raise IcxError(st, what)


def _ws(ws, n, stream):
    if ws is None:
        ws = Workspace(n, stream=stream)
    return ws


# -- index -------------------------------------------------------------------

def bp128_index(data, n: int, fmt: int = FMT_PAPER, index=None, workspace=None, stream=None):
    import torch
    _dev(data, torch.uint8, "data")
    if index is None:
        index = torch.empty(bp128_index_len(n), dtype=torch.uint64, device=data.device)
    ws = _ws(workspace, n, stream)
    _check(lib().bp128_index(_ptr(data), data.numel(), n, fmt, _ptr(index), ws.ptr(), ws.bytes, _stream(stream)),
           "bp128_index")
    return index


def fastpfor_index(data, n: int, index=None, workspace=None, stream=None):
    import torch
    _dev(data, torch.uint8, "data")
    if index is None:
        index = torch.empty(fastpfor_index_len(n), dtype=torch.uint64, device=data.device)
    ws = _ws(workspace, n, stream)
    _check(lib().fastpfor_index(_ptr(data), data.numel(), n, _ptr(index), ws.ptr(), ws.bytes, _stream(stream)),
           "fastpfor_index")
    return index


# -- decode ------------------------------------------------------------------

def bp128_decode(data, n: int, delta: int = DELTA_1, fmt: int = FMT_PAPER, index=None, out=None,
                 workspace=None, stream=None, in_bytes=None):
    """Decodes n integers (Sec. 6.2 metablocks + Sec. 3 prefix sum)."""
    import torch
    _dev(data, torch.uint8, "data")
    if out is None:
        out = torch.empty(n, dtype=torch.uint32, device=data.device)
    _dev(out, torch.uint32, "out")
    ws = _ws(workspace, n, stream)
    nbytes = data.numel() if in_bytes is None else in_bytes
    _check(lib().bp128_decode(_ptr(data), nbytes, _ptr(out), n, delta, fmt, _ptr(index), ws.ptr(), ws.bytes,
                              _stream(stream)), "bp128_decode")
    return out


def fastpfor_decode(data, n: int, delta: int = DELTA_1, index=None, out=None, workspace=None, stream=None,
                    in_bytes=None):
    """Decodes n integers (Sec. 5 pages with exception patching + Sec. 3)."""
    import torch
    _dev(data, torch.uint8, "data")
    if out is None:
        out = torch.empty(n, dtype=torch.uint32, device=data.device)
    _dev(out, torch.uint32, "out")
    ws = _ws(workspace, n, stream)
    nbytes = data.numel() if in_bytes is None else in_bytes
    _check(lib().fastpfor_decode(_ptr(data), nbytes, _ptr(out), n, delta, _ptr(index), ws.ptr(), ws.bytes,
                                 _stream(stream)), "fastpfor_decode")
    return out


def delta_decode(d, delta: int = DELTA_1, out=None, workspace=None, stream=None):
    """Prefix sum with stride 1 or 4 (Sec. 3); out may be d (in place)."""
    import torch
    _dev(d, torch.uint32, "d")
    if out is None:
        out = torch.empty_like(d)
    ws = _ws(workspace, d.numel(), stream)
    _check(lib().delta_decode(_ptr(d), _ptr(out), d.numel(), delta, ws.ptr(), ws.bytes, _stream(stream)),
           "delta_decode")
    return out


# -- encode ------------------------------------------------------------------

def delta_encode(x, delta: int = DELTA_1, out=None, stream=None):
    import torch
    _dev(x, torch.uint32, "x")
    if out is None:
        out = torch.empty_like(x)
    _check(lib().delta_encode(_ptr(x), _ptr(out), x.numel(), delta, _stream(stream)), "delta_encode")
    return out


class Encoded:
    """A stream produced on the GPU: bytes (trimmed), its index and n."""

    def __init__(self, data, index, n, codec, delta, fmt=FMT_PAPER):
        self.data, self.index, self.n = data, index, n
        self.codec, self.delta, self.fmt = codec, delta, fmt

    @property
    def nbytes(self) -> int:
        return self.data.numel()


def _encode(codec, x, delta, fmt, stream):
    import torch
    _dev(x, torch.uint32, "x")
    n = x.numel()
    if codec == "bp128":
        cap, ilen = bp128_max_bytes(n, fmt), bp128_index_len(n)
    else:
        cap, ilen = fastpfor_max_bytes(n), fastpfor_index_len(n)
    buf = torch.empty(cap, dtype=torch.uint8, device=x.device)
    index = torch.empty(ilen, dtype=torch.uint64, device=x.device)
    total = torch.zeros(1, dtype=torch.uint64, device=x.device)
    ews = Workspace(n, stream=stream, encode=True)
    s = _stream(stream)
    if codec == "bp128":
        code = lib().bp128_encode(_ptr(x), n, delta, fmt, _ptr(buf), cap, _ptr(index), _ptr(total), ews.ptr(),
                                  ews.bytes, s)
    else:
        code = lib().fastpfor_encode(_ptr(x), n, delta, _ptr(buf), cap, _ptr(index), _ptr(total), ews.ptr(),
                                     ews.bytes, s)
    _check(code, f"{codec}_encode")
    ews.raise_status(f"{codec}_encode", stream)
    nbytes = int(total.cpu().view(torch.int64).item())
    data = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=x.device)[:nbytes]
    data.copy_(buf[:nbytes])
    return Encoded(data, index, n, codec, delta, fmt)


def bp128_encode(x, delta: int = DELTA_1, fmt: int = FMT_PAPER, stream=None) -> Encoded:
    """Encodes on the GPU (widths = bit length of each block's largest delta)."""
    return _encode("bp128", x, delta, fmt, stream)


def fastpfor_encode(x, delta: int = DELTA_1, stream=None) -> Encoded:
    return _encode("fastpfor", x, delta, FMT_PAPER, stream)


def decode(enc: Encoded, out=None, workspace=None, stream=None):
    if enc.codec == "bp128":
        return bp128_decode(enc.data, enc.n, enc.delta, enc.fmt, enc.index, out, workspace, stream)
    return fastpfor_decode(enc.data, enc.n, enc.delta, enc.index, out, workspace, stream)


def set_tuning(key: str, value: int) -> None:
    """Launch parameter of the decoders, e.g. ("bp128.warps_per_cta", 4)."""
    _check(lib().icx_set_tuning(key.encode(), int(value)), f"icx_set_tuning({key})")


def version() -> str:
    return lib().icx_version().decode()
