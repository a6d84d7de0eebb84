"""Stored expected values (tests/golden/, written by make_golden.py from the oracle).

CPU: the fixtures agree with the oracle and with exact arithmetic recomputed now
(a change to the oracle's arithmetic that moves a bit fails here).  GPU: every
kernel reproduces the integer fixture bit for bit and stays within the FP64
bound of the exact dyadic fixture.
"""
import hashlib
import os
import sys
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_golden as mg  # noqa: E402

from oracle import cgemm, exact  # noqa: E402


def _read(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def int_fixture():
    rows = _read("dgemm_int_n256.txt")
    sha = next(r[1] for r in rows if r[0] == "sha256")
    total = Fraction(next(r[1] for r in rows if r[0] == "sum"))
    entries = [(int(r[1]), int(r[2]), float(r[3])) for r in rows if r[0] == "entry"]
    return sha, total, entries


def dyadic_fixture():
    Cs = np.empty((mg.DY_M, mg.DY_N), dtype=object)
    for r in _read("dgemm_dyadic_5x7x3.txt"):
        Cs[int(r[1]), int(r[2])] = Fraction(r[3])
    return Cs


def _sha(C):
    return hashlib.sha256(np.ascontiguousarray(C, dtype="<f8").tobytes()).hexdigest()


def test_int_fixture_matches_the_oracle():
    sha, total, entries = int_fixture()
    C, exact_C = mg.int_case()
    assert np.array_equal(C, exact_C)
    assert _sha(C) == sha
    assert sum(Fraction(float(v)) for v in C.ravel()) == total
    assert len(entries) == 64 and all(C[i, j] == v for i, j, v in entries)


def test_dyadic_fixture_matches_exact_arithmetic_and_bounds_the_oracle():
    Cs = dyadic_fixture()
    again = mg.dyadic_case()
    assert all(Cs[i, j] == again[i][j] for i in range(mg.DY_M) for j in range(mg.DY_N))
    A, B, C0 = mg.dyadic_inputs()
    got = cgemm.dgemm(mg.DY_ALPHA, A, B, mg.DY_BETA, C0.copy())
    bound = exact.error_bound(mg.DY_K, mg.DY_ALPHA, cgemm.dgemm(1.0, np.abs(A), np.abs(B)),
                              mg.DY_BETA, C0)
    err = np.array([[abs(Fraction(float(got[i, j])) - Cs[i, j]) for j in range(mg.DY_N)]
                    for i in range(mg.DY_M)], dtype=object)
    assert all(err[i, j] <= Fraction(float(bound[i, j]))
               for i in range(mg.DY_M) for j in range(mg.DY_N))


KERNELS = [("native", "auto"), ("native", "naive"), ("native", "tiled"), ("native", "dfma"),
           ("native", "dmma"), ("emulated", 2), ("emulated", 11)]


def _gpu_gemm(gb, A, B, C0, alpha, beta, precision, kernel):
    import torch
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.from_numpy(C0.copy()).cuda()
    if precision == "native":
        gb.dgemm(dA, dB, dC, alpha, beta, kernel=kernel)
    else:
        gb.dgemm(dA, dB, dC, alpha, beta, precision="emulated", slices=kernel)
    torch.cuda.synchronize()
    return dC.cpu().numpy()


@pytest.mark.gpu
@pytest.mark.parametrize("precision,kernel", KERNELS)
def test_gpu_reproduces_the_integer_fixture_bit_for_bit(precision, kernel):
    import paper_1602_08477_gb300 as gb
    gb.build()
    sha, total, entries = int_fixture()
    A, B, C0 = mg.int_inputs()
    got = _gpu_gemm(gb, A, B, C0, mg.INT_ALPHA, mg.INT_BETA, precision, kernel)
    assert all(got[i, j] == v for i, j, v in entries)
    assert _sha(got) == sha


@pytest.mark.gpu
@pytest.mark.parametrize("precision,kernel", [pk for pk in KERNELS if pk != ("emulated", 2)])
def test_gpu_within_the_bound_of_the_exact_dyadic_fixture(precision, kernel):
    # (two slices carry 9 bits: FP64 accuracy needs the tuned count, here 11; the
    # integer fixture above fits in the first slice, so there s = 2 is exact)
    import paper_1602_08477_gb300 as gb
    gb.build()
    Cs = dyadic_fixture()
    A, B, C0 = mg.dyadic_inputs()
    got = _gpu_gemm(gb, A, B, C0, mg.DY_ALPHA, mg.DY_BETA, precision, kernel)
    bound = exact.error_bound(mg.DY_K, mg.DY_ALPHA, cgemm.dgemm(1.0, np.abs(A), np.abs(B)),
                              mg.DY_BETA, C0)
    for i in range(mg.DY_M):
        for j in range(mg.DY_N):
            assert abs(Fraction(float(got[i, j])) - Cs[i, j]) <= Fraction(float(bound[i, j]))
