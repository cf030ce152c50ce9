"""Scalar CPU oracle for the SIMD-BP128 / SIMD-FastPFOR decoding path.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import this package.  The product library
(``paper_1209_2137_gb300``) never loads it and shares no code with it.

This module compiles ``icx_oracle.c`` (plain C11, bit-by-bit routines written
from the paper's definitions) into ``liboracle.so`` beside it and exposes the
entry points on numpy arrays.  Section numbers refer to Lemire & Boytsov,
"Decoding billions of integers per second through vectorization".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "icx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PAPER = 0
W32 = 1


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (no GPU involved)."""
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "icx_oracle.h")))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            sz, u8p, u32p, u64p = ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
            i = ctypes.c_int
            lib.orc_bitlen.argtypes, lib.orc_bitlen.restype = [ctypes.c_uint32], i
            lib.orc_packed_bytes.argtypes, lib.orc_packed_bytes.restype = [sz, i, i], sz
            lib.orc_pack.argtypes, lib.orc_pack.restype = [u32p, sz, i, i, u8p], None
            lib.orc_unpack.argtypes, lib.orc_unpack.restype = [u8p, sz, i, i, u32p], None
            lib.orc_delta_encode.argtypes, lib.orc_delta_encode.restype = [u32p, sz, i, u32p], None
            lib.orc_delta_decode.argtypes, lib.orc_delta_decode.restype = [u32p, sz, i, u32p], None
            lib.orc_vbyte_encode.argtypes, lib.orc_vbyte_encode.restype = [u32p, sz, u8p], sz
            lib.orc_vbyte_decode.argtypes, lib.orc_vbyte_decode.restype = [u8p, sz, sz, u32p], sz
            for name in ("bp128", "fastpfor"):
                getattr(lib, f"orc_{name}_max_bytes").argtypes = [sz]
                getattr(lib, f"orc_{name}_max_bytes").restype = sz
                getattr(lib, f"orc_{name}_index_len").argtypes = [sz]
                getattr(lib, f"orc_{name}_index_len").restype = sz
            lib.orc_bp128_encode.argtypes, lib.orc_bp128_encode.restype = [u32p, sz, i, i, u8p], sz
            lib.orc_bp128_decode.argtypes, lib.orc_bp128_decode.restype = [u8p, sz, sz, i, i, u32p], i
            lib.orc_bp128_index.argtypes, lib.orc_bp128_index.restype = [u8p, sz, sz, i, u64p], i
            lib.orc_fastpfor_choose.argtypes = [u32p, sz, ctypes.POINTER(i), ctypes.POINTER(i),
                                                ctypes.POINTER(i), u64p]
            lib.orc_fastpfor_choose.restype = None
            lib.orc_fastpfor_block_record.argtypes = [u32p, sz, u8p, u32p, ctypes.POINTER(sz)]
            lib.orc_fastpfor_block_record.restype = sz
            lib.orc_fastpfor_encode.argtypes, lib.orc_fastpfor_encode.restype = [u32p, sz, i, u8p], sz
            lib.orc_fastpfor_decode.argtypes, lib.orc_fastpfor_decode.restype = [u8p, sz, sz, i, u32p], i
            lib.orc_fastpfor_index.argtypes, lib.orc_fastpfor_index.restype = [u8p, sz, sz, u64p], i
            lib.orc_fastpfor_encode_layout.argtypes = [u32p, sz, i, i, u8p]
            lib.orc_fastpfor_encode_layout.restype = sz
            lib.orc_fastpfor_decode_layout.argtypes = [u8p, sz, sz, i, i, u32p]
            lib.orc_fastpfor_decode_layout.restype = i
            lib.orc_fastpfor_index_layout.argtypes = [u8p, sz, sz, i, u64p]
            lib.orc_fastpfor_index_layout.restype = i
            lib.orc_member_bits.argtypes, lib.orc_member_bits.restype = [u32p, sz, u32p, sz, u32p, u64p], None
            lib.orc_bp32_max_bytes.argtypes, lib.orc_bp32_max_bytes.restype = [sz], sz
            lib.orc_simple8b_encode.argtypes, lib.orc_simple8b_encode.restype = [u32p, sz, u64p], sz
            lib.orc_simple8b_decode.argtypes, lib.orc_simple8b_decode.restype = [u64p, sz, sz, u32p], i
            lib.orc_simplepfor_max_bytes.argtypes, lib.orc_simplepfor_max_bytes.restype = [sz], sz
            lib.orc_simplepfor_encode.argtypes, lib.orc_simplepfor_encode.restype = [u32p, sz, i, u8p], sz
            lib.orc_simplepfor_decode.argtypes, lib.orc_simplepfor_decode.restype = [u8p, sz, sz, i, u32p], i
            lib.orc_simplepfor_index.argtypes, lib.orc_simplepfor_index.restype = [u8p, sz, sz, u64p], i
            lib.orc_bp32_encode.argtypes, lib.orc_bp32_encode.restype = [u32p, sz, i, u8p], sz
            lib.orc_bp32_decode.argtypes, lib.orc_bp32_decode.restype = [u8p, sz, sz, i, u32p], i
            lib.orc_bp32_index.argtypes, lib.orc_bp32_index.restype = [u8p, sz, sz, u64p], i
            _lib = lib
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


class CorruptStream(ValueError):
    """The oracle found a stream that does not follow the format."""


# -- Sec. 2 / Sec. 4 ---------------------------------------------------------

def bitlen(x: int) -> int:
    return _load().orc_bitlen(ctypes.c_uint32(int(x)))


def pack(values, lanes: int, b: int) -> np.ndarray:
    """Sec. 4: LSB-first packing over `lanes` interleaved 32-bit lanes."""
    v = _u32(values)
    lib = _load()
    out = np.zeros(lib.orc_packed_bytes(v.size, lanes, b), dtype=np.uint8)
    lib.orc_pack(_ptr(v), v.size, lanes, b, _ptr(out))
    return out


def unpack(data, count: int, lanes: int, b: int) -> np.ndarray:
    d = _u8(data)
    lib = _load()
    assert d.size >= lib.orc_packed_bytes(count, lanes, b)
    out = np.zeros(count, dtype=np.uint32)
    lib.orc_unpack(_ptr(d), count, lanes, b, _ptr(out))
    return out


# -- Sec. 3 ------------------------------------------------------------------

def delta_encode(x, stride: int) -> np.ndarray:
    v = _u32(x)
    out = np.zeros_like(v)
    _load().orc_delta_encode(_ptr(v), v.size, stride, _ptr(out))
    return out


def delta_decode(d, stride: int) -> np.ndarray:
    v = _u32(d)
    out = np.zeros_like(v)
    _load().orc_delta_decode(_ptr(v), v.size, stride, _ptr(out))
    return out


# -- Sec. 2.4 ----------------------------------------------------------------

def vbyte_encode(values) -> np.ndarray:
    v = _u32(values)
    out = np.zeros(5 * v.size + 1, dtype=np.uint8)
    n = _load().orc_vbyte_encode(_ptr(v), v.size, _ptr(out))
    return out[:n].copy()


def vbyte_decode(data, count: int) -> np.ndarray:
    d = _u8(data)
    out = np.zeros(count, dtype=np.uint32)
    used = _load().orc_vbyte_decode(_ptr(d), d.size, count, _ptr(out))
    if used == ctypes.c_size_t(-1).value:
        raise CorruptStream("variable byte stream truncated or overlong")
    return out


# -- Sec. 6.2: SIMD-BP128 ----------------------------------------------------

def bp128_encode(x, delta: int, layout: int = PAPER) -> np.ndarray:
    v = _u32(x)
    lib = _load()
    out = np.zeros(lib.orc_bp128_max_bytes(v.size), dtype=np.uint8)
    n = lib.orc_bp128_encode(_ptr(v), v.size, delta, layout, _ptr(out))
    return out[:n].copy()


def bp128_decode(data, n: int, delta: int, layout: int = PAPER) -> np.ndarray:
    d = _u8(data)
    out = np.zeros(n, dtype=np.uint32)
    rc = _load().orc_bp128_decode(_ptr(d), d.size, n, delta, layout, _ptr(out))
    if rc != 0:
        raise CorruptStream(f"bp128 stream corrupt (rc={rc})")
    return out


def bp128_index(data, n: int, layout: int = PAPER) -> np.ndarray:
    d = _u8(data)
    lib = _load()
    out = np.zeros(lib.orc_bp128_index_len(n), dtype=np.uint64)
    rc = lib.orc_bp128_index(_ptr(d), d.size, n, layout, _ptr(out))
    if rc != 0:
        raise CorruptStream(f"bp128 stream corrupt (rc={rc})")
    return out


# -- Sec. 6.2: BP32 ----------------------------------------------------------

def bp32_encode(x, delta: int) -> np.ndarray:
    v = _u32(x)
    lib = _load()
    out = np.zeros(lib.orc_bp32_max_bytes(v.size), dtype=np.uint8)
    n = lib.orc_bp32_encode(_ptr(v), v.size, delta, _ptr(out))
    return out[:n].copy()


def bp32_decode(data, n: int, delta: int) -> np.ndarray:
    d = _u8(data)
    out = np.zeros(n, dtype=np.uint32)
    rc = _load().orc_bp32_decode(_ptr(d), d.size, n, delta, _ptr(out))
    if rc != 0:
        raise CorruptStream(f"bp32 stream corrupt (rc={rc})")
    return out


def bp32_index(data, n: int) -> np.ndarray:
    d = _u8(data)
    lib = _load()
    out = np.zeros(lib.orc_bp128_index_len(n), dtype=np.uint64)
    rc = lib.orc_bp32_index(_ptr(d), d.size, n, _ptr(out))
    if rc != 0:
        raise CorruptStream(f"bp32 stream corrupt (rc={rc})")
    return out


# -- Sec. 5: (SIMD-)FastPFOR -------------------------------------------------

def fastpfor_choose(values):
    """Returns (b, maxbits, c, costs[0..maxbits]) for one block."""
    v = _u32(values)
    b, mb, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    costs = np.zeros(33, dtype=np.uint64)
    _load().orc_fastpfor_choose(_ptr(v), v.size, ctypes.byref(b), ctypes.byref(mb),
                                ctypes.byref(c), _ptr(costs))
    return b.value, mb.value, c.value, costs[: mb.value + 1].copy()


def fastpfor_block_record(values):
    """Returns (record bytes, exception high parts) for one block."""
    v = _u32(values)
    assert v.size <= 256
    rec = np.zeros(3 + v.size, dtype=np.uint8)
    high = np.zeros(max(1, v.size), dtype=np.uint32)
    nh = ctypes.c_size_t()
    r = _load().orc_fastpfor_block_record(_ptr(v), v.size, _ptr(rec), _ptr(high), ctypes.byref(nh))
    return rec[:r].copy(), high[: nh.value].copy()


def fastpfor_encode(x, delta: int, layout: int = PAPER) -> np.ndarray:
    """SIMD-FastPFOR (layout PAPER) or the scalar FastPFOR (layout SCALAR)."""
    v = _u32(x)
    lib = _load()
    out = np.zeros(lib.orc_fastpfor_max_bytes(v.size), dtype=np.uint8)
    n = lib.orc_fastpfor_encode_layout(_ptr(v), v.size, delta, layout, _ptr(out))
    return out[:n].copy()


def fastpfor_decode(data, n: int, delta: int, layout: int = PAPER) -> np.ndarray:
    d = _u8(data)
    out = np.zeros(n, dtype=np.uint32)
    rc = _load().orc_fastpfor_decode_layout(_ptr(d), d.size, n, delta, layout, _ptr(out))
    if rc != 0:
        raise CorruptStream(f"fastpfor stream corrupt (rc={rc})")
    return out


def fastpfor_index(data, n: int, layout: int = PAPER) -> np.ndarray:
    d = _u8(data)
    lib = _load()
    out = np.zeros(lib.orc_fastpfor_index_len(n), dtype=np.uint64)
    rc = lib.orc_fastpfor_index_layout(_ptr(d), d.size, n, layout, _ptr(out))
    if rc != 0:
        raise CorruptStream(f"fastpfor stream corrupt (rc={rc})")
    return out


# -- Sec. 2 / Sec. 5: Simple-8b and SimplePFOR --------------------------------

def simple8b_encode(values) -> np.ndarray:
    v = _u32(values)
    words = np.zeros(max(1, v.size), dtype=np.uint64)
    w = _load().orc_simple8b_encode(_ptr(v), v.size, _ptr(words))
    return words[:w].copy()


def simple8b_decode(words, count: int) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint64)
    out = np.zeros(max(1, count), dtype=np.uint32)
    rc = _load().orc_simple8b_decode(_ptr(w), w.size, count, _ptr(out))
    if rc != 0:
        raise CorruptStream("simple-8b words do not hold the given count")
    return out[:count].copy()


def simplepfor_encode(x, delta: int) -> np.ndarray:
    v = _u32(x)
    lib = _load()
    out = np.zeros(lib.orc_simplepfor_max_bytes(v.size), dtype=np.uint8)
    n = lib.orc_simplepfor_encode(_ptr(v), v.size, delta, _ptr(out))
    return out[:n].copy()


def simplepfor_decode(data, n: int, delta: int) -> np.ndarray:
    d = _u8(data)
    out = np.zeros(n, dtype=np.uint32)
    rc = _load().orc_simplepfor_decode(_ptr(d), d.size, n, delta, _ptr(out))
    if rc != 0:
        raise CorruptStream(f"simplepfor stream corrupt (rc={rc})")
    return out


def simplepfor_index(data, n: int) -> np.ndarray:
    d = _u8(data)
    lib = _load()
    out = np.zeros(lib.orc_fastpfor_index_len(n), dtype=np.uint64)
    rc = lib.orc_simplepfor_index(_ptr(d), d.size, n, _ptr(out))
    if rc != 0:
        raise CorruptStream(f"simplepfor stream corrupt (rc={rc})")
    return out


BP32 = 2  # layout value of the BP32 format in the SIMD-BP128 calls
SCALAR = 2  # the same value: scalar 32-integer packing (BP32 / FastPFOR)


def encode(codec: str, x, delta: int, layout: int = PAPER) -> np.ndarray:
    if codec == "bp128":
        return bp32_encode(x, delta) if layout == BP32 else bp128_encode(x, delta, layout)
    if codec == "fastpfor":
        return fastpfor_encode(x, delta, layout)
    if codec == "simplepfor":
        return simplepfor_encode(x, delta)
    raise ValueError(codec)


def decode(codec: str, data, n: int, delta: int, layout: int = PAPER) -> np.ndarray:
    if codec == "bp128":
        return bp32_decode(data, n, delta) if layout == BP32 else bp128_decode(data, n, delta, layout)
    if codec == "fastpfor":
        return fastpfor_decode(data, n, delta, layout)
    if codec == "simplepfor":
        return simplepfor_decode(data, n, delta)
    raise ValueError(codec)


def index(codec: str, data, n: int, layout: int = PAPER) -> np.ndarray:
    if codec == "bp128":
        return bp32_index(data, n) if layout == BP32 else bp128_index(data, n, layout)
    if codec == "fastpfor":
        return fastpfor_index(data, n, layout)
    if codec == "simplepfor":
        return simplepfor_index(data, n)
    raise ValueError(codec)


# -- Sec. 7: decoding fused into a consumer (sorted-list membership) ---------

def member_bits(a, b):
    """Membership of the sorted query list b in the sorted list a, by merging
    the two: returns (bits, count), bit j of the uint32 words `bits` (bit j%32
    of word j//32) set iff b[j] occurs in a; count = number of set bits."""
    va, vb = _u32(a), _u32(b)
    bits = np.zeros(max(1, (vb.size + 31) // 32), dtype=np.uint32)
    cnt = np.zeros(1, dtype=np.uint64)
    _load().orc_member_bits(_ptr(va), va.size, _ptr(vb), vb.size, _ptr(bits), _ptr(cnt))
    return bits[: (vb.size + 31) // 32].copy(), int(cnt[0])
