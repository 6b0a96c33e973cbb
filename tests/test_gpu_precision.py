"""Storage precision on the lid-driven cavity: shifted FP16 / BF16 storage with
FP32 arithmetic against FP32 and FP64 storage and against the FP64 oracle.

Case: 64^3 cavity, lid 0.05 along x on +y, tau 0.55, 5000 steps from rest
(the reduced-size oracle comparison of the 384^3 precision workload).  The
errors of rho and u (max and RMS over all cells) are asserted against stated
bounds; LBM_REPORT_DIR=<dir> also writes them as JSON.

Bounds (max |u - u_oracle| with |u| <= 0.05 at the lid; rho and u leave the
library as float32, so every row carries that output rounding, 2^-24 on
rho ~ 1 and about 2e-9 on u):
- FP64 storage: 4e-9 on u (the float32 output), and 1e-12 on the PDFs read
  back in FP64;
- FP32: 5e-6 (1e-4 of the lid speed);
- shifted FP16, scale 256 and scale 1: 1e-4 (0.2% of the lid speed);
- BF16: 2e-3 (4% of the lid speed; 8 mantissa bits).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1007_1388_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, TAU, STEPS, LID = 64, 0.55, 5000, 0.05


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1388_gb300 import build

    build.build()
    import paper_1007_1388_gb300 as L

    L.use_torch_allocator()
    oracle.build()
    return L


@pytest.fixture(scope="module")
def ref():
    p = oracle.Problem(dims=(N,) * 3, tau=TAU, wall_u=(LID, 0, 0), **W.cavity_bc())
    oracle.set_threads(os.cpu_count() or 1)
    try:
        f = oracle.run(p, oracle.zeros(p), STEPS)
    finally:
        oracle.set_threads(1)
    rho, u = oracle.macroscopic(p, f)
    return rho.reshape(-1), u.reshape(-1), f


CASES = [("f64", 3, 1.0, 4e-9), ("f32", 0, 1.0, 5e-6), ("f16s_scale256", 1, 256.0, 1e-4),
         ("bf16s", 2, 1.0, 2e-3), ("f16s_scale1", 1, 1.0, 1e-4)]


def _errors(rho, u, rr, ur):
    du, dr = u - ur, rho - rr
    return {"u_max": float(np.abs(du).max()), "u_rms": float(np.sqrt(np.mean(du * du))),
            "rho_max": float(np.abs(dr).max()), "rho_rms": float(np.sqrt(np.mean(dr * dr)))}


def test_cavity64_storage_precision_vs_oracle(L, ref):
    rr, ur, fr = ref
    report = {"case": f"{N}^3 cavity, lid {LID}, tau {TAU}, {STEPS} steps, vs FP64 oracle",
              "u_max_ref": float(np.abs(ur).max())}
    bad = []
    for name, storage, scale, tol in CASES:
        p = L.make_params(wall_u=(LID, 0, 0), storage=storage, storage_scale=scale,
                          **W.cavity_bc())
        ctx = L.lbm_create((N,) * 3, (N,) * 3, TAU, None, p)
        L.lbm_step(ctx, STEPS)
        rho, u = L.lbm_macroscopic(ctx)
        if storage == 3:
            df = np.abs(L.lbm_get_pdfs(ctx).reshape(fr.shape) - fr).max()
            report["f64_pdf_max"] = float(df)
            if not df <= 1e-12:
                bad.append(("f64 pdfs", float(df), 1e-12))
        ctx.destroy()
        e = _errors(rho.astype(np.float64), u.astype(np.float64), rr, ur)
        e["bound_u_max"] = tol
        report[name] = e
        print(name, e)
        if tol is not None and not e["u_max"] <= tol:
            bad.append((name, e["u_max"], tol))
    out = os.environ.get("LBM_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_cavity64.json"), "w") as fh:
            json.dump(report, fh, indent=1)
    assert not bad, bad
