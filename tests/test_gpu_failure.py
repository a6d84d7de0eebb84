"""Failure detection without a fault: a device-side wait that runs out reports
GB_ERR_TIMEOUT through the queue, the kernel ends normally, and the same queue
and context keep working."""
import numpy as np
import pytest

from oracle import cgemm
from synth import generators as g

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_queue_stays_usable():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    q = gb.Queue(gb.Device(0), torch.cuda.current_stream())
    st = gb.load().gb_selftest_wait_timeout(q.handle, 20000)   # 20 ms limit
    assert st == 0
    with pytest.raises(gb.GbError, match="GB_ERR_TIMEOUT"):
        q.wait()
    q.wait()   # the status was cleared
    A = g.matrix("int8", 64, 64, 5, 0)
    B = g.matrix("int8", 64, 64, 5, 1)
    dC = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    gb.dgemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), dC, queue=q)
    q.wait()
    assert np.array_equal(dC.cpu().numpy(), cgemm.dgemm(1.0, A, B))


def test_selftest_rejects_bad_limits():
    import torch
    import paper_1602_08477_gb300 as gb
    q = gb.Queue(gb.Device(0), torch.cuda.current_stream())
    assert gb.load().gb_selftest_wait_timeout(q.handle, 0) == 1
    assert gb.load().gb_selftest_wait_timeout(None, 10) == 1
