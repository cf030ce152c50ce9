"""The oracle decoder on every host core, for the CPU baseline.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the benchmark's
CPU-baseline leg and the tests call it; the product library never does.

A coded stream is a sequence of independent units (SIMD-BP128, W32 and BP32:
metablocks of 2048 integers; SIMD-FastPFOR and SimplePFOR: pages of 65536),
located by the stream's index, then the Variable Byte tail (Sec. 2.4).  The
units of a contiguous range, with the tail when the range is the last one,
are themselves a valid stream of the same format, so each thread hands its
range's bytes to the plain single-thread oracle routine unchanged.  With
differential coding each range then decodes from a zero prefix, and one
pass adds the carry: the last integer before the range (stride 1), or the
last four (stride 4, residue by residue, since a range starts at a multiple
of four) -- Sec. 3.  That add is the only arithmetic here.  The oracle
routines release the interpreter lock while they run (ctypes calls), so the
threads decode in parallel.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

from . import decode, index

UNIT_INTS = {"bp128": 2048, "fastpfor": 65536, "simplepfor": 65536}


def host_cores() -> int:
    """Cores this process may run on (the affinity mask, else the CPU count)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def split_ranges(units: int, parts: int):
    """`parts` contiguous unit ranges of nearly equal size covering [0, units)."""
    parts = max(1, min(parts, units))
    edges = [units * i // parts for i in range(parts + 1)]
    return [(edges[i], edges[i + 1]) for i in range(parts) if edges[i + 1] > edges[i]]


def decode_parallel(codec: str, data, n: int, delta: int, layout: int = 0, threads: int | None = None,
                    pool: cf.ThreadPoolExecutor | None = None, idx=None) -> np.ndarray:
    """Decodes the same integers as ``oracle.decode(codec, data, n, delta, layout)``
    with the stream's unit ranges on `threads` threads."""
    data = np.ascontiguousarray(data, dtype=np.uint8)
    threads = threads or host_cores()
    unit = UNIT_INTS[codec]
    units = (n // 128 + unit // 128 - 1) // (unit // 128)  # full and partial units
    if threads <= 1 or units <= 1:
        return decode(codec, data, n, delta, layout)
    if idx is None:
        idx = index(codec, data, n, layout)
    ranges = split_ranges(units, threads)

    def one(rng):
        u0, u1 = rng
        last = u1 == units
        lo, hi = int(idx[u0]), (data.size if last else int(idx[u1]))
        count = (n if last else u1 * unit) - u0 * unit
        return decode(codec, data[lo:hi], count, delta, layout)

    own = pool is None
    ex = pool or cf.ThreadPoolExecutor(max_workers=len(ranges))
    try:
        parts = list(ex.map(one, ranges))
        # carry into each range: the decoded values just before it (the
        # previous range's last values, which are its own zero-prefix values
        # plus its carry); then every range adds its carry, in parallel
        carries = [None]
        for r in range(1, len(parts)):
            prev, c0 = parts[r - 1], carries[r - 1]
            if delta == 1:
                c = prev[-1:].copy()
            elif delta == 4:
                c = prev[-4:].copy()
            else:
                c = None
            if c is not None and c0 is not None:
                c += c0
            carries.append(c)
        offs = np.cumsum([0] + [p.size for p in parts])
        out = np.empty(n, dtype=np.uint32)

        def place(r):
            part, c = parts[r], carries[r]
            if c is not None and delta == 1:
                part += c[0]
            elif c is not None:
                m = part.size // 4 * 4
                part[:m].reshape(-1, 4)[:] += c
                part[m:] += c[: part.size - m]
            out[offs[r]:offs[r + 1]] = part

        list(ex.map(place, range(len(parts))))
    finally:
        if own:
            ex.shutdown()
    assert offs[-1] == n
    return out
