"""The timeout path of the bounded device waits (failure detection without a
GPU fault): a decode whose first tasks are never taken leaves the waits on
their published sums to run out; the kernel ends normally with ICX_ETIMEOUT
in the status word, resets its workspace, and the next decode on the same
workspace is correct."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1209_2137_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1209_2137_gb300 as icx  # noqa: E402


@pytest.mark.parametrize("delta", [icx.DELTA_1, icx.DELTA_4])
def test_waits_run_out_then_workspace_recovers(delta):
    n = 16 * 4096 + 777  # 16 pairs of metablocks and a tail: a few tasks per warp
    x = W.uniform_sorted(n, 30, 81)
    enc = icx.bp128_encode(torch.from_numpy(x).cuda(), delta)
    ws = icx.Workspace(n)
    out = torch.zeros(n, dtype=torch.uint32, device="cuda")
    # a short limit, and the task counter moved past the first tasks (the
    # sums of the first pairs are then never published)
    ws.set_wait_limit(200)
    ws.tensor[:4].view(torch.int32).fill_(12)
    icx.decode(enc, out=out, workspace=ws)
    assert ws.status() == icx.ETIMEOUT
    # the launch reset its counters: the same workspace decodes correctly
    ws.set_wait_limit(0)
    out.zero_()
    icx.decode(enc, out=out, workspace=ws)
    assert ws.status() == icx.OK
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.bp128_decode(enc.data.cpu().numpy(), n, delta))
