"""GPU: pitched buffers, explicit copies and a DGEMM that uses nothing but the
C ABI for memory, streams and compute (no PyTorch tensors)."""
import numpy as np
import pytest

from oracle import cgemm, exact
from synth import generators as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import paper_1602_08477_gb300 as gb
    gb.build()
    return gb


@pytest.fixture(scope="module")
def dev(gb):
    return gb.Device(0)


def host_from(gb, a):
    h = gb.Buffer(a.shape, None)
    h.numpy()[...] = a
    return h


def test_round_trip_keeps_every_byte_and_uses_the_pitch(gb, dev):
    a = g.matrix("hard", 100, 77, 31, 0)
    h = host_from(gb, a)
    assert h.pitch_bytes == 624  # 616 B rounded up to 16
    d = gb.Buffer((100, 77), dev)
    assert d.pitch_bytes >= 77 * 8 and d.pitch_bytes % 8 == 0
    q = gb.OwnedQueue(dev)
    gb.copy(q, d, h)
    back = gb.Buffer((100, 77), None)
    gb.copy(q, back, d)
    q.wait()
    assert np.array_equal(back.numpy(), a)  # bit-exact, incl. signs and subnormals


def test_sub_block_and_3d_copies(gb, dev):
    q = gb.OwnedQueue(dev, blocking=True)
    a = g.matrix("uniform", 3 * 20, 33, 32, 0).reshape(3, 20, 33)
    h = host_from(gb, a)
    d = gb.Buffer((3, 20, 33), dev)
    gb.copy(q, d, h)
    out = gb.Buffer((3, 20, 33), None)
    out.numpy()[...] = -7.0
    gb.copy(q, out, d, extents=(2, 9, 5))  # per-plane copies
    got = out.numpy()
    assert np.array_equal(got[:2, :9, :5], a[:2, :9, :5])
    assert np.all(got[2] == -7.0) and np.all(got[:, 9:] == -7.0) and np.all(got[:, :, 5:] == -7.0)
    gb.copy(q, out, d)  # whole planes: one strided copy
    assert np.array_equal(out.numpy(), a)
    v = host_from(gb, np.arange(10.0))
    dv = gb.Buffer((10,), dev)
    gb.copy(q, dv, v)
    ov = gb.Buffer((10,), None)
    gb.copy(q, ov, dv, extents=(4,))
    assert np.array_equal(ov.numpy()[:4], np.arange(4.0))


@pytest.mark.parametrize("precision,kernel", [("native", "auto"), ("native", "dfma"),
                                              ("emulated", "auto")])
def test_dgemm_over_pitched_buffers(gb, dev, precision, kernel):
    m, n, k = 150, 97, 203
    A = g.matrix("uniform", m, k, 33, 0)
    B = g.matrix("uniform", k, n, 33, 1)
    C0 = g.matrix("uniform", m, n, 33, 2)
    q = gb.OwnedQueue(dev)
    dA, dB, dC = gb.Buffer((m, k), dev), gb.Buffer((k, n), dev), gb.Buffer((m, n), dev)
    assert dA.ld > k  # really pitched
    for d, h in ((dA, A), (dB, B), (dC, C0)):
        gb.copy(q, d, host_from(gb, h))
    ws = None
    if precision == "emulated":
        ws = gb.Buffer((gb.workspace_size("emulated", 12, m, n, k),), dev, dtype=np.uint8)
    gb.dgemm_buffers(q, dA, dB, dC, 0.75, -0.5, kernel=kernel, precision=precision, slices=12,
                     workspace=ws)
    out = gb.Buffer((m, n), None)
    gb.copy(q, out, dC)
    q.wait()
    got = out.numpy().copy()
    ref = cgemm.dgemm(0.75, A, B, -0.5, C0.copy())
    bound = exact.error_bound(k, 0.75, cgemm.dgemm(1.0, np.abs(A), np.abs(B)), -0.5, C0)
    assert np.all(np.abs(got - ref) <= 2 * bound)
