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
FMT_PAPER, FMT_W32, FMT_BP32 = 0, 1, 2
FMT_SCALAR = 2  # the SIMD-FastPFOR calls: the paper's scalar FastPFOR
FMT_SIMPLE8B = 3  # the SIMD-FastPFOR calls: the paper's SimplePFOR
CODEC_BP128, CODEC_FASTPFOR = 0, 1

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
                "icx_workspace_set_wait_limit": ([vp, sz, ctypes.c_uint, vp], i),
                "icx_workspace_layout": ([sz, sz, ctypes.POINTER(sz)], i),
                "bp128_index": ([vp, sz, sz, i, vp, vp, sz, vp], i),
                "fastpfor_index": ([vp, sz, sz, i, vp, vp, sz, vp], i),
                "bp128_decode": ([vp, sz, vp, sz, i, i, vp, vp, sz, vp], i),
                "fastpfor_decode": ([vp, sz, vp, sz, i, i, vp, vp, sz, vp], i),
                "bp128_intersect": ([vp, sz, sz, i, i, vp, vp, sz, vp, vp, vp, sz, vp], i),
                "sorted_intersect": ([vp, sz, vp, sz, vp, vp, vp], i),
                "delta_decode": ([vp, vp, sz, i, vp, sz, vp], i),
                "delta_encode": ([vp, vp, sz, i, vp], i),
                "bp128_encode": ([vp, sz, i, i, vp, sz, vp, vp, vp, sz, vp], i),
                "fastpfor_encode": ([vp, sz, i, i, vp, sz, vp, vp, vp, sz, vp], i),
                "icx_version": ([], ctypes.c_char_p),
                "icx_set_tuning": ([ctypes.c_char_p, i], i),
                "icx_plan_create": ([vp, sz, vp, ctypes.POINTER(vp)], i),
                "icx_plan_error_list": ([], ctypes.c_longlong),
                "icx_plan_launch": ([vp, vp], i),
                "icx_plan_launch_per_list": ([vp, vp], i),
                "icx_plan_status": ([vp, vp, ctypes.POINTER(ctypes.c_int)], i),
                "icx_plan_tuning": ([vp, vp], i),
                "icx_plan_destroy": ([vp], None),
                "icx_server_create": ([vp, sz, sz, i, i, ctypes.POINTER(vp)], i),
                "icx_server_run": ([vp, sz, vp, vp, vp, vp, vp, vp, vp], i),
                "icx_server_destroy": ([vp], None),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes, fn.restype = args, res
            _lib = L
    return _lib


EXPORTED = ("icx_bp128_index_len", "icx_fastpfor_index_len", "icx_bp128_max_bytes", "icx_fastpfor_max_bytes",
            "icx_workspace_bytes", "icx_encode_workspace_bytes", "icx_workspace_init", "icx_status_read",
            "icx_workspace_set_wait_limit", "icx_workspace_layout",
            "bp128_index", "fastpfor_index", "bp128_decode", "fastpfor_decode", "bp128_intersect",
            "sorted_intersect", "delta_decode", "delta_encode",
            "bp128_encode", "fastpfor_encode", "icx_version", "icx_set_tuning", "icx_plan_create",
            "icx_plan_error_list", "icx_plan_launch", "icx_plan_launch_per_list", "icx_plan_status", "icx_plan_tuning",
            "icx_plan_destroy", "icx_server_create", "icx_server_run", "icx_server_destroy")


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

    def set_wait_limit(self, usec: int, stream=None):
        """Limit of the decoders' device waits on this workspace (0 = default)."""
        _check(lib().icx_workspace_set_wait_limit(self.ptr(), self.bytes, int(usec), _stream(stream)),
               "icx_workspace_set_wait_limit")

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


def fastpfor_index(data, n: int, index=None, workspace=None, stream=None, fmt: int = FMT_PAPER):
    import torch
    _dev(data, torch.uint8, "data")
    if index is None:
        index = torch.empty(fastpfor_index_len(n), dtype=torch.uint64, device=data.device)
    ws = _ws(workspace, n, stream)
    _check(lib().fastpfor_index(_ptr(data), data.numel(), n, fmt, _ptr(index), ws.ptr(), ws.bytes,
                                _stream(stream)), "fastpfor_index")
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
                    in_bytes=None, fmt: int = FMT_PAPER):
    """Decodes n integers (Sec. 5 pages with exception patching + Sec. 3);
    fmt FMT_PAPER = SIMD-FastPFOR, FMT_SCALAR = the scalar FastPFOR."""
    import torch
    _dev(data, torch.uint8, "data")
    if out is None:
        out = torch.empty(n, dtype=torch.uint32, device=data.device)
    _dev(out, torch.uint32, "out")
    ws = _ws(workspace, n, stream)
    nbytes = data.numel() if in_bytes is None else in_bytes
    _check(lib().fastpfor_decode(_ptr(data), nbytes, _ptr(out), n, delta, fmt, _ptr(index), ws.ptr(), ws.bytes,
                                 _stream(stream)), "fastpfor_decode")
    return out


def _member_out(b, bits, count):
    import torch
    _dev(b, torch.uint32, "b")
    if bits is None:
        bits = torch.empty((b.numel() + 31) // 32, dtype=torch.uint32, device=b.device)
    if count is None:
        count = torch.empty(1, dtype=torch.uint64, device=b.device)
    _dev(bits, torch.uint32, "bits")
    _dev(count, torch.uint64, "count")
    return bits, count


def bp128_intersect(data, n: int, b, delta: int = DELTA_1, fmt: int = FMT_PAPER, index=None, bits=None,
                    count=None, workspace=None, stream=None, in_bytes=None):
    """Membership of the sorted query list b in the sorted list the stream
    decodes to, decoded and consumed in one pass (Sec. 7).  Returns (bits,
    count): bit j of the uint32 words `bits` set iff b[j] is in the list;
    count (a one-element uint64 tensor on the device) the number of set bits."""
    import torch
    _dev(data, torch.uint8, "data")
    bits, count = _member_out(b, bits, count)
    ws = _ws(workspace, n, stream)
    nbytes = data.numel() if in_bytes is None else in_bytes
    _check(lib().bp128_intersect(_ptr(data), nbytes, n, delta, fmt, _ptr(index), _ptr(b), b.numel(), _ptr(bits),
                                 _ptr(count), ws.ptr(), ws.bytes, _stream(stream)), "bp128_intersect")
    return bits, count


def sorted_intersect(a, b, bits=None, count=None, stream=None):
    """The same consumer over the decoded sorted list a (the unfused path)."""
    import torch
    _dev(a, torch.uint32, "a")
    bits, count = _member_out(b, bits, count)
    _check(lib().sorted_intersect(_ptr(a), a.numel(), _ptr(b), b.numel(), _ptr(bits), _ptr(count),
                                  _stream(stream)), "sorted_intersect")
    return bits, count


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
        code = lib().fastpfor_encode(_ptr(x), n, delta, fmt, _ptr(buf), cap, _ptr(index), _ptr(total),
                                     ews.ptr(), ews.bytes, s)
    _check(code, f"{codec}_encode")
    ews.raise_status(f"{codec}_encode", stream)
    nbytes = int(total.cpu().view(torch.int64).item())
    data = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=x.device)[:nbytes]
    data.copy_(buf[:nbytes])
    return Encoded(data, index, n, codec, delta, fmt)


def bp128_encode(x, delta: int = DELTA_1, fmt: int = FMT_PAPER, stream=None) -> Encoded:
    """Encodes on the GPU (widths = bit length of each block's largest delta)."""
    return _encode("bp128", x, delta, fmt, stream)


def fastpfor_encode(x, delta: int = DELTA_1, stream=None, fmt: int = FMT_PAPER) -> Encoded:
    return _encode("fastpfor", x, delta, fmt, stream)


def decode(enc: Encoded, out=None, workspace=None, stream=None):
    if enc.codec == "bp128":
        return bp128_decode(enc.data, enc.n, enc.delta, enc.fmt, enc.index, out, workspace, stream)
    return fastpfor_decode(enc.data, enc.n, enc.delta, enc.index, out, workspace, stream, fmt=enc.fmt)


def set_tuning(key: str, value: int) -> None:
    """Launch parameter of the decoders, e.g. ("bp128.warps_per_cta", 4)."""
    _check(lib().icx_set_tuning(key.encode(), int(value)), f"icx_set_tuning({key})")


def version() -> str:
    return lib().icx_version().decode()


# -- batched decoding ----------------------------------------------------------

class ListDesc(ctypes.Structure):
    """icx_list_desc: one list of a batch."""
    _fields_ = [("d_in", ctypes.c_void_p), ("in_bytes", ctypes.c_size_t), ("d_out", ctypes.c_void_p),
                ("n", ctypes.c_size_t), ("d_index", ctypes.c_void_p), ("codec", ctypes.c_int),
                ("delta", ctypes.c_int), ("fmt", ctypes.c_int)]


class Tuning(ctypes.Structure):
    """icx_tuning: warps_per_cta 4/8 (0 = tune), order 0/1/2 (-1 = tune),
    l2_prefetch 1/0 (-1 = tune), cache_path (None: $ICX_TUNE_CACHE)."""
    _fields_ = [("warps_per_cta", ctypes.c_int), ("order", ctypes.c_int), ("l2_prefetch", ctypes.c_int),
                ("cache_path", ctypes.c_char_p)]


class Plan:
    """A batch of lists decoded by one CUDA graph launch (icx_plan_*).

    ``descs`` is a sequence of ListDesc; the device buffers they point to must
    outlive the plan.  ``tuning`` is a Tuning, a dict of its fields, or None
    (tune everything)."""

    def __init__(self, descs, tuning=None):
        arr = (ListDesc * len(descs))(*descs)
        if isinstance(tuning, dict):
            path = tuning.get("cache_path")
            tuning = Tuning(tuning.get("warps_per_cta", 0), tuning.get("order", -1), tuning.get("l2_prefetch", -1),
                            path.encode() if isinstance(path, str) else path)
        self._keep = (arr, tuning)
        handle = ctypes.c_void_p()
        code = lib().icx_plan_create(ctypes.cast(arr, ctypes.c_void_p), len(descs),
                                     ctypes.cast(ctypes.pointer(tuning), ctypes.c_void_p) if tuning else None,
                                     ctypes.byref(handle))
        if code != OK:
            bad = lib().icx_plan_error_list()
            raise IcxError(code, "icx_plan_create" + (f" (list {bad})" if bad >= 0 else ""))
        self._h = handle

    def launch(self, stream=None):
        _check(lib().icx_plan_launch(self._h, _stream(stream)), "icx_plan_launch")

    def launch_per_list(self, stream=None):
        _check(lib().icx_plan_launch_per_list(self._h, _stream(stream)), "icx_plan_launch_per_list")

    def status(self, stream=None) -> int:
        st = ctypes.c_int(0)
        _check(lib().icx_plan_status(self._h, _stream(stream), ctypes.byref(st)), "icx_plan_status")
        return st.value

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().icx_plan_tuning(self._h, ctypes.cast(ctypes.pointer(t), ctypes.c_void_p)), "icx_plan_tuning")
        return {"warps_per_cta": t.warps_per_cta, "order": t.order, "l2_prefetch": t.l2_prefetch}

    def close(self):
        if getattr(self, "_h", None):
            lib().icx_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ListPool:
    """Many lists encoded on the GPU into one pooled buffer, one encoder call
    per list and no host synchronisation until all are issued.

    ``values`` (a host uint32 array) holds the lists back to back, list i at
    values[offsets[i]:offsets[i+1]]; codecs, deltas, fmts give each list's
    format.  The values are uploaded with every list starting on a 16-byte
    boundary (``x``, list i at x[x_off[i]:x_off[i]+n[i]]).  After
    construction: data (uint8 pool), index (uint64 pool), and per list
    in_off, in_bytes, index_off (host integers)."""

    def __init__(self, values, offsets, codecs, deltas, fmts=None, device="cuda", stream=None):
        import numpy as np
        import torch
        L = len(offsets) - 1
        fmts = np.zeros(L, dtype=np.int64) if fmts is None else np.asarray(fmts)
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.n = np.diff(self.offsets)
        self.codecs, self.deltas, self.fmts = np.asarray(codecs), np.asarray(deltas), fmts
        padded = (self.n + 3) // 4 * 4
        self.x_off = np.zeros(L, dtype=np.int64)
        np.cumsum(padded[:-1], out=self.x_off[1:])
        host = np.zeros(int(padded.sum()) + 4, dtype=np.uint32)
        dst = np.repeat(self.x_off - self.offsets[:-1], self.n) + np.arange(int(self.offsets[-1]), dtype=np.int64)
        host[dst] = np.asarray(values, dtype=np.uint32)[:int(self.offsets[-1])]
        self.x = torch.from_numpy(host.view(np.int32)).to(device).view(torch.uint32)
        # positions of ``x`` that belong to no list (alignment padding)
        pad = padded - self.n
        pad_pos = np.repeat(self.x_off + self.n, pad) + (np.arange(int(pad.sum())) -
                                                        np.repeat(np.cumsum(pad) - pad, pad))
        self.padding = torch.from_numpy(np.concatenate([pad_pos, [host.size - 4 + k for k in range(4)]])
                                        .astype(np.int64)).to(device)
        cap = np.zeros(L, dtype=np.int64)
        ilen = np.zeros(L, dtype=np.int64)
        for i in range(L):
            n = int(self.n[i])
            if self.codecs[i] == CODEC_BP128:
                cap[i], ilen[i] = bp128_max_bytes(n, int(fmts[i])), bp128_index_len(n)
            else:
                cap[i], ilen[i] = fastpfor_max_bytes(n), fastpfor_index_len(n)
        cap = (cap + 15) // 16 * 16
        ilen = (ilen + 1) // 2 * 2
        self.in_off = np.zeros(L, dtype=np.int64)
        self.index_off = np.zeros(L, dtype=np.int64)
        np.cumsum(cap[:-1], out=self.in_off[1:])
        np.cumsum(ilen[:-1], out=self.index_off[1:])
        dev = self.x.device
        self.data = torch.empty(int(cap.sum()) + 16, dtype=torch.uint8, device=dev)
        self.index = torch.empty(int(ilen.sum()) + 2, dtype=torch.uint64, device=dev)
        totals = torch.zeros(L, dtype=torch.uint64, device=dev)
        nmax = int(self.n.max()) if L else 1
        ews = Workspace(max(nmax, 1), device=dev, stream=stream, encode=True)
        s = _stream(stream)
        base_v, base_d, base_i, base_t = self.x.data_ptr(), self.data.data_ptr(), self.index.data_ptr(), \
            totals.data_ptr()
        F = lib()
        for i in range(L):
            n = int(self.n[i])
            args = (ctypes.c_void_p(base_v + 4 * int(self.x_off[i])), n)
            outp = ctypes.c_void_p(base_d + int(self.in_off[i]))
            idxp = ctypes.c_void_p(base_i + 8 * int(self.index_off[i]))
            totp = ctypes.c_void_p(base_t + 8 * i)
            if self.codecs[i] == CODEC_BP128:
                code = F.bp128_encode(*args, int(self.deltas[i]), int(fmts[i]), outp, int(cap[i]), idxp, totp,
                                      ews.ptr(), ews.bytes, s)
            else:
                code = F.fastpfor_encode(*args, int(self.deltas[i]), FMT_PAPER, outp, int(cap[i]), idxp, totp,
                                         ews.ptr(), ews.bytes, s)
            _check(code, f"encode list {i}")
        ews.raise_status("pooled encode", stream)
        self.in_bytes = totals.cpu().numpy().view(np.int64).copy()
        self.cap = cap

    @property
    def nbytes(self) -> int:
        return int(self.in_bytes.sum())

    def output_offsets(self):
        """Per list the first element of its output in a pooled uint32 tensor
        laid out like ``x`` (16-byte aligned starts), and the pool length."""
        return self.x_off, int(self.x.numel())

    def descs(self, out, out_off, with_index=True):
        """ListDesc per list, decoding into out[out_off[i]:out_off[i]+n[i]]."""
        bd, bi, bo = self.data.data_ptr(), self.index.data_ptr(), out.data_ptr()
        res = []
        for i in range(len(self.n)):
            res.append(ListDesc(bd + int(self.in_off[i]), int(self.in_bytes[i]), bo + 4 * int(out_off[i]),
                                int(self.n[i]), (bi + 8 * int(self.index_off[i])) if with_index else None,
                                int(self.codecs[i]), int(self.deltas[i]), int(self.fmts[i])))
        return res


# -- serving loop -----------------------------------------------------------------

class ServerStats(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("ints", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("max_batch", ctypes.c_uint64), ("max_queue", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("wall_s", ctypes.c_double), ("queue_s", ctypes.c_double), ("service_s", ctypes.c_double),
                ("gpu_s", ctypes.c_double)]


class Server:
    """The serving loop (icx_server_*) over a resident pool of lists.

    ``descs``: ListDesc per pool list (d_out ignored); the buffers they point
    to must outlive the server."""

    def __init__(self, descs, budget_bytes: int = 16 << 30, streams: int = 2, warps_per_cta: int = 8):
        arr = (ListDesc * len(descs))(*descs)
        self._keep = arr
        handle = ctypes.c_void_p()
        code = lib().icx_server_create(ctypes.cast(arr, ctypes.c_void_p), len(descs), budget_bytes, streams,
                                       warps_per_cta, ctypes.byref(handle))
        if code != OK:
            bad = lib().icx_plan_error_list()
            raise IcxError(code, "icx_server_create" + (f" (list {bad})" if bad >= 0 else ""))
        self._h = handle

    def run(self, arrival_ns, req_offsets, list_ids, results=False):
        """Serves the schedule; returns (latency_ns per request, stats dict,
        results or None).  With results=True every request's lists come back
        decoded, back to back (a list of numpy arrays, one per request)."""
        import numpy as np
        arrival = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
        offs = np.ascontiguousarray(req_offsets, dtype=np.uint64)
        ids = np.ascontiguousarray(list_ids, dtype=np.uint32)
        nreq = arrival.size
        lat = np.zeros(nreq, dtype=np.uint64)
        stats = ServerStats()
        res = res_off = None
        if results:
            n = np.array([d.n for d in self._keep], dtype=np.uint64)
            per = np.array([int(n[ids[offs[r]:offs[r + 1]]].sum()) for r in range(nreq)], dtype=np.uint64)
            res_off = np.zeros(nreq, dtype=np.uint64)
            np.cumsum(per[:-1], out=res_off[1:])
            res = np.zeros(int(per.sum()) + 1, dtype=np.uint32)
        vp = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
        _check(lib().icx_server_run(self._h, nreq, vp(arrival), vp(offs), vp(ids), vp(lat), vp(res), vp(res_off),
                                    ctypes.cast(ctypes.pointer(stats), ctypes.c_void_p)), "icx_server_run")
        st = {f: getattr(stats, f) for f, _ in ServerStats._fields_}
        out = None
        if results:
            out = [res[int(res_off[r]):int(res_off[r]) + int(per[r])] for r in range(nreq)]
        return lat, st, out

    def close(self):
        if getattr(self, "_h", None):
            lib().icx_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

