"""GPU parity of batched decoding (icx_plan_*): every list of a mixed batch
(both codecs, every delta, both SIMD-BP128 layouts, lengths across the unit,
page and tail boundaries) decodes bit for bit to the oracle's decode of the
same bytes, under every tuning, through the per-list baseline too, and
across repeated launches."""
from __future__ import annotations

import json

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402

LENGTHS = [0, 1, 5, 127, 128, 129, 2047, 2048, 2049, 2175, 2176, 4099, 20000, 65535, 65536, 65537, 140003]


def make_batch(nlists=240, seed=7):
    z = W.splitmix64(seed, 0, 4 * nlists)
    lens = [LENGTHS[int(v % len(LENGTHS))] for v in z[:nlists]]
    codecs = [int(v & 1) for v in z[nlists:2 * nlists] >> np.uint64(20)]
    deltas = [(0, 1, 4)[int(v % 3)] for v in z[2 * nlists:3 * nlists]]
    fmts = [int(v & 1) if c == icx.CODEC_BP128 else 0 for v, c in zip(z[3 * nlists:] >> np.uint64(30), codecs)]
    xs = []
    for i, n in enumerate(lens):
        if deltas[i] == 0:
            xs.append(W.random_small(n, seed * 1000 + i) if n else np.zeros(0, np.uint32))
        else:
            xs.append(W.uniform_sorted(n, 24, seed * 1000 + i) if n else np.zeros(0, np.uint32))
    return xs, codecs, deltas, fmts


class Batch:
    """Oracle-encoded lists uploaded into one pool (16-byte aligned starts)."""

    def __init__(self, xs, codecs, deltas, fmts, corrupt=None):
        self.xs, self.codecs, self.deltas, self.fmts = xs, codecs, deltas, fmts
        names = ["bp128" if c == icx.CODEC_BP128 else "fastpfor" for c in codecs]
        self.enc = [oracle.encode(nm, x, d, f) if x.size else np.zeros(0, np.uint8)
                    for nm, x, d, f in zip(names, xs, deltas, fmts)]
        self.idx = [oracle.index(nm, e, x.size, f) for nm, e, x, f in zip(names, self.enc, xs, fmts)]
        self.want = [oracle.decode(nm, e, x.size, d, f) for nm, e, x, d, f in zip(names, self.enc, xs, deltas, fmts)]
        if corrupt is not None:
            e = self.enc[corrupt].copy()
            e[0] = 0xFF  # width byte of block 0 (SIMD-BP128) / header word (SIMD-FastPFOR)
            self.enc[corrupt] = e
        off, pos = [], 0
        for e in self.enc:
            off.append(pos)
            pos += (e.size + 15) // 16 * 16
        blob = np.zeros(pos + 16, np.uint8)
        for o, e in zip(off, self.enc):
            blob[o:o + e.size] = e
        ioff, ipos = [], 0
        for ix in self.idx:
            ioff.append(ipos)
            ipos += (ix.size + 1) // 2 * 2
        iblob = np.zeros(ipos + 2, np.uint64)
        for o, ix in zip(ioff, self.idx):
            iblob[o:o + ix.size] = ix
        self.data = torch.from_numpy(blob).cuda()
        self.index = torch.from_numpy(iblob.view(np.int64)).cuda()
        self.in_off, self.index_off = off, ioff
        self.out_off, tot = [], 0
        for x in xs:
            self.out_off.append(tot)
            tot += (x.size + 3) // 4 * 4
        self.out = torch.full((tot + 4,), 0x5A5A5A5A, dtype=torch.int64).to(torch.int32).cuda().view(torch.uint32)

    def descs(self, null_index=()):
        bd, bi, bo = self.data.data_ptr(), self.index.data_ptr(), self.out.data_ptr()
        return [icx.ListDesc(bd + self.in_off[i], int(self.enc[i].size), bo + 4 * self.out_off[i], int(x.size),
                             None if i in null_index else bi + 8 * self.index_off[i], self.codecs[i], self.deltas[i],
                             self.fmts[i]) for i, x in enumerate(self.xs)]

    def check(self, skip=()):
        got = self.out.cpu().numpy().view(np.uint32)
        for i, w in enumerate(self.want):
            if i in skip:
                continue
            g = got[self.out_off[i]:self.out_off[i] + w.size]
            assert np.array_equal(g, w), (i, self.codecs[i], self.deltas[i], self.fmts[i], w.size,
                                          int(np.argmax(g != w)) if w.size else -1)

    def clear(self):
        self.out.view(torch.int32).fill_(0x5A5A5A5A)


@pytest.fixture(scope="module")
def batch():
    return Batch(*make_batch())


def test_batch_matches_oracle_every_tuning(batch):
    for W_ in (4, 8):
        for order in (0, 1, 2):
            for l2 in (0, 1):
                batch.clear()
                plan = icx.Plan(batch.descs(), {"warps_per_cta": W_, "order": order, "l2_prefetch": l2})
                assert plan.tuning() == {"warps_per_cta": W_, "order": order, "l2_prefetch": l2}
                plan.launch()
                assert plan.status() == icx.OK
                batch.check()
                plan.close()


def test_batch_repeated_launches_and_per_list_baseline(batch):
    plan = icx.Plan(batch.descs(), {"warps_per_cta": 8, "order": 1, "l2_prefetch": 1})
    for _ in range(3):
        batch.clear()
        plan.launch()
        assert plan.status() == icx.OK
        batch.check()
    for _ in range(2):
        batch.clear()
        plan.launch_per_list()
        assert plan.status() == icx.OK
        batch.check()
    plan.close()


def test_batch_null_index_for_single_unit_lists(batch):
    null = {i for i, x in enumerate(batch.xs)
            if (batch.codecs[i] == icx.CODEC_BP128 and x.size < 17 * 128)
            or (batch.codecs[i] == icx.CODEC_FASTPFOR and x.size < 513 * 128)}
    assert len(null) > 20
    batch.clear()
    plan = icx.Plan(batch.descs(null), {"warps_per_cta": 4, "order": 0, "l2_prefetch": 0})
    plan.launch()
    assert plan.status() == icx.OK
    batch.check()
    plan.close()


def test_batch_autotune_and_cache(batch, tmp_path):
    path = tmp_path / "tune.json"
    batch.clear()
    plan = icx.Plan(batch.descs(), {"warps_per_cta": 0, "order": -1, "l2_prefetch": -1, "cache_path": str(path)})
    chosen = plan.tuning()
    plan.launch()
    assert plan.status() == icx.OK
    batch.check()
    plan.close()
    cache = json.loads(path.read_text())
    assert len(cache) == 1
    (key, val), = cache.items()
    assert key.startswith(f"lists={len(batch.xs)};")
    assert val == [chosen["warps_per_cta"], chosen["order"], chosen["l2_prefetch"]]
    plan2 = icx.Plan(batch.descs(), {"warps_per_cta": 0, "order": -1, "l2_prefetch": -1, "cache_path": str(path)})
    assert plan2.tuning() == chosen
    plan2.close()


def test_batch_corrupt_list_reports_error():
    xs, codecs, deltas, fmts = make_batch(40, seed=11)
    victim = next(i for i, x in enumerate(xs) if codecs[i] == icx.CODEC_BP128 and x.size >= 4096)
    b = Batch(xs, codecs, deltas, fmts, corrupt=victim)
    plan = icx.Plan(b.descs(), {"warps_per_cta": 8, "order": 0, "l2_prefetch": 1})
    plan.launch()
    assert plan.status() == icx.ECORRUPT
    plan.close()


def test_batch_posting_lists_pooled_gpu_encoder():
    # a small instance of the posting-list workload, encoded by the GPU
    # encoders into one pool; decoded lists equal the generated values
    L, offsets, values, bp = W.posting_lists(nlists=2048, total=1 << 21)
    codecs = np.where(bp, icx.CODEC_BP128, icx.CODEC_FASTPFOR)
    deltas = np.where(bp, icx.DELTA_4, icx.DELTA_1)
    pool = icx.ListPool(values, offsets, codecs, deltas)
    for i in range(0, 2048, 97):  # GPU bytes equal the oracle's
        x = values[offsets[i]:offsets[i + 1]]
        want = oracle.encode("bp128" if bp[i] else "fastpfor", x, int(deltas[i]))
        got = pool.data[int(pool.in_off[i]):int(pool.in_off[i]) + int(pool.in_bytes[i])].cpu().numpy()
        assert np.array_equal(got, want), i
    out_off, total = pool.output_offsets()
    out = torch.zeros(total, dtype=torch.int32, device="cuda").view(torch.uint32)
    plan = icx.Plan(pool.descs(out, out_off), {"warps_per_cta": 8, "order": 1, "l2_prefetch": 1})
    plan.launch()
    assert plan.status() == icx.OK
    assert torch.equal(out, pool.x)  # padding included: both zero
    got = out.cpu().numpy().view(np.uint32)
    for i in range(0, 2048, 31):
        n = int(L[i])
        assert np.array_equal(got[out_off[i]:out_off[i] + n], values[offsets[i]:offsets[i + 1]]), i
    plan.close()
