"""Error of the emulated FP64 GEMM against the FP64 contract, per slice count, at
the full sizes of the emulated workload (n = 4096, 8192; uniform[-1, 1] and the
16-decade hard set), on sampled rows against the double-double reference.

Asserts what the slice-count tuning relies on: the error falls with s; s = 10
(the emulated benchmark's setting) is at or below native DGEMM's own error
(rho_emu <= rho_native, rho = max error / FP64 bound) on uniform inputs, s = 11
on the hard set, and both are within the FP64 bound.
Writes the table as JSON to the path in the environment variable
GB_ACCURACY_TABLE when it is set.
"""
import json
import os

import numpy as np
import pytest

from oracle import cgemm, exact
from synth import generators as g

pytestmark = pytest.mark.gpu



def test_error_vs_slices_at_full_size():
    import torch
    import paper_1602_08477_gb300 as gb
    gb.build()
    table = []
    for n in (4096, 8192):
        for kind, off in (("uniform", 2), ("hard", 3)):
            seed = g.BASE_SEED + off
            A_h = g.matrix(kind, n, n, seed, g.STREAM_A)
            B_h = g.matrix(kind, n, n, seed, g.STREAM_B)
            A, B = torch.from_numpy(A_h).cuda(), torch.from_numpy(B_h).cuda()
            C = torch.empty((n, n), dtype=torch.float64, device="cuda")
            sel = np.random.default_rng(n + off).choice(n, 6, replace=False)
            hi, lo = cgemm.dgemm_dd_rows(A_h, B_h, sel)
            bound = exact.error_bound(n, 1.0,
                                      cgemm.dgemm_rows(sel, 1.0, np.abs(A_h), np.abs(B_h)))
            gb.dgemm(A, B, C, kernel="auto")
            torch.cuda.synchronize()
            rho_native = float(np.max(np.abs(exact.residual(C.cpu().numpy()[sel], 1.0, hi, lo))
                                      / bound))
            for s in range(8, 15):
                gb.dgemm(A, B, C, precision="emulated", slices=s)
                torch.cuda.synchronize()
                res = exact.residual(C.cpu().numpy()[sel], 1.0, hi, lo)
                rho = float(np.max(np.abs(res) / bound))
                table.append(dict(n=n, kind=kind, slices=s, rho=rho, rho_native=rho_native))
            del A, B, C
            torch.cuda.empty_cache()
    out = os.environ.get("GB_ACCURACY_TABLE")
    if out:
        with open(out, "w") as f:
            json.dump(table, f, indent=1)

    def rho(n, kind, s):
        return next(r["rho"] for r in table if r["n"] == n and r["kind"] == kind and r["slices"] == s)

    for n in (4096, 8192):
        for kind in ("uniform", "hard"):
            assert rho(n, kind, 14) < rho(n, kind, 8)
        for kind, s in (("uniform", 10), ("hard", 11)):
            native = next(r["rho_native"] for r in table if r["n"] == n and r["kind"] == kind)
            assert native < 1.0
            assert rho(n, kind, s) <= native
