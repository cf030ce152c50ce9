"""The all-cores CPU baseline harness: the oracle decoder run on unit ranges
of a stream on several threads, with the differential carry added per range,
decodes exactly what the single-thread oracle decodes (every codec, layout
and stride; ranges of one and several units; partial last units and tails)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import parallel
from paper_1209_2137_gb300 import workloads as W

CASES = [("bp128", oracle.PAPER), ("bp128", oracle.W32), ("bp128", oracle.BP32), ("fastpfor", oracle.PAPER),
         ("fastpfor", oracle.SCALAR), ("simplepfor", oracle.PAPER)]


@pytest.mark.parametrize("codec,layout", CASES)
@pytest.mark.parametrize("delta", [0, 1, 4])
def test_parallel_decode_equals_single_thread(codec, layout, delta):
    unit = parallel.UNIT_INTS[codec]
    x = W.uniform_sorted(3 * unit + 5 * 128 + 77, 30, 71) if delta else W.exception_heavy(3 * unit + 5 * 128 + 77, 72)
    for n in (unit - 1, unit, 2 * unit + 3, x.size):
        enc = oracle.encode(codec, x[:n], delta, layout)
        want = oracle.decode(codec, enc, n, delta, layout)
        for threads in (1, 2, 3, 7):
            got = parallel.decode_parallel(codec, enc, n, delta, layout, threads=threads)
            assert np.array_equal(got, want), (n, threads)


def test_ranges_cover_every_unit():
    for units in (1, 2, 5, 64, 1000):
        for parts in (1, 3, 16, 2000):
            r = parallel.split_ranges(units, parts)
            assert r[0][0] == 0 and r[-1][1] == units
            assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
            assert all(a < b for a, b in r)
    assert parallel.host_cores() >= 1
