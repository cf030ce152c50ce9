"""One workspace shared by decodes of different codecs, layouts, strides and
lengths, in turn and many times over (so the launch epoch advances): every
decode must stay exact.  The decoders keep epoch-tagged words (look-back
states, block sums) and plain records (page parse, prepare kernel) in
separate regions for every length the workspace serves."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402


def test_mixed_decodes_on_one_workspace():
    big = 9 * 65536 + 4096 * 3 + 77
    xs = {n: W.uniform_sorted(n, 28, 90 + i) for i, n in enumerate((big, 65536 * 2 + 129, 4096 * 7 + 5, 3000))}
    jobs = []
    for n, x in xs.items():
        xt = torch.from_numpy(x).cuda()
        for codec, delta, fmt in (("bp128", 4, 0), ("bp128", 1, 0), ("bp128", 1, 1), ("bp128", 0, 0),
                                  ("fastpfor", 4, 0), ("fastpfor", 1, 0), ("fastpfor", 0, 0)):
            enc = icx.bp128_encode(xt, delta, fmt) if codec == "bp128" else icx.fastpfor_encode(xt, delta)
            jobs.append((enc, xt))
    ws = icx.Workspace(big)
    out = torch.empty(big, dtype=torch.uint32, device="cuda")
    rng = np.random.default_rng(7)
    for rnd in range(6):
        for j in rng.permutation(len(jobs)):
            enc, xt = jobs[j]
            o = out[: enc.n]
            o.fill_(0xDEADBEEF)
            icx.decode(enc, out=o, workspace=ws)
            assert ws.status() == icx.OK
            assert torch.equal(o, xt), (rnd, enc.codec, enc.delta, enc.fmt, enc.n)
