"""GPU checks of the serving loop (icx_server_*): every request's result is
the same decoded alone and in a busy mix (continuous batching over several
streams, admission waits under a small budget), and equals the oracle's
decode of its lists."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402

from tests.test_gpu_batch import Batch, make_batch  # noqa: E402


def requests(nlists, nreq, seed):
    z = W.splitmix64(seed, 0, 9 * nreq)
    k = 2 + (z[:nreq] % np.uint64(7)).astype(np.int64)
    offs = np.zeros(nreq + 1, dtype=np.int64)
    np.cumsum(k, out=offs[1:])
    ids = (z[nreq:nreq + offs[-1]] % np.uint64(nlists)).astype(np.uint32)
    return offs, ids


@pytest.fixture(scope="module")
def pool():
    return Batch(*make_batch(120, seed=21))


def expected(pool, offs, ids, r):
    parts = [pool.want[int(i)] for i in ids[offs[r]:offs[r + 1]]]
    return np.concatenate(parts) if parts else np.zeros(0, np.uint32)


def test_serve_alone_equals_mix(pool):
    nreq = 200
    offs, ids = requests(len(pool.xs), nreq, 5)
    # in the mix: everything arrives at once, so batches fill up and overlap
    sv = icx.Server(pool.descs(), budget_bytes=64 << 20, streams=3)
    lat, st, mix = sv.run(np.zeros(nreq, np.uint64), offs, ids, results=True)
    assert st["requests"] == nreq and st["batches"] < nreq and st["max_batch"] > 1
    for r in range(nreq):
        assert np.array_equal(mix[r], expected(pool, offs, ids, r)), r
    # alone: one request per run
    for r in range(0, nreq, 7):
        lat1, st1, alone = sv.run(np.zeros(1, np.uint64), offs[r:r + 2] - offs[r], ids[offs[r]:offs[r + 1]],
                                  results=True)
        assert st1["batches"] == 1 and np.array_equal(alone[0], mix[r]), r
    sv.close()


def test_serve_small_budget_waits_for_buffers(pool):
    nreq = 120
    offs, ids = requests(len(pool.xs), nreq, 9)
    biggest = max(sum((pool.xs[int(i)].size * 4 + 15) // 16 * 16 for i in ids[offs[r]:offs[r + 1]])
                  for r in range(nreq))
    budget = (biggest + 255) // 256 * 256 + 4096  # about one request at a time
    sv = icx.Server(pool.descs(), budget_bytes=budget, streams=2, warps_per_cta=4)
    lat, st, res = sv.run(np.arange(nreq, dtype=np.uint64) * 1000, offs, ids, results=True)
    assert st["requests"] == nreq and st["peak_bytes"] <= budget and st["max_queue"] >= 1
    for r in range(nreq):
        assert np.array_equal(res[r], expected(pool, offs, ids, r)), r
    assert (lat > 0).all()
    # a request larger than the whole budget is refused up front
    big = int(np.argmax([x.size for x in pool.xs]))
    sv2 = icx.Server(pool.descs(), budget_bytes=1024, streams=2)
    with pytest.raises(icx.IcxError) as e:
        sv2.run(np.zeros(1, np.uint64), np.array([0, 1]), np.array([big], np.uint32))
    assert e.value.code == icx.ENOSPC
    sv.close()
    sv2.close()


def test_serve_poisson_schedule(pool):
    # open loop at 20k requests/s: latencies measured from the scheduled arrivals
    nreq = 400
    offs, ids = requests(len(pool.xs), nreq, 13)
    z = W.splitmix64(17, 0, nreq)
    u = ((z >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
    arrival = np.cumsum(-np.log(u) / 20000.0 * 1e9).astype(np.uint64)
    sv = icx.Server(pool.descs(), budget_bytes=256 << 20, streams=2)
    lat, st, res = sv.run(arrival, offs, ids, results=False)
    assert st["requests"] == nreq
    assert st["ints"] == sum(int(pool.xs[int(i)].size) for i in ids)
    assert np.percentile(lat, 50) < 50e6  # well under 50 ms
    sv.close()
