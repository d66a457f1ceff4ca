"""Accuracy study of the 128^3 drop over 5000 steps (the D3Q19 drop workload at
its smallest size, full step count) for every storage mode against the FP64
oracle: mass-equivalent radius, Laplace pressure jump P_in - P_out and peak
spurious speed max|u_phys|.  The oracle takes about ten minutes on 16 cores, so
the study runs only when LBM_STUDY=1 is set:

    LBM_STUDY=1 python -m pytest tests/test_gpu_study_cfg2.py -s -q

Bar: 1e-3 for FP32 and 1 % for the rest-offset 16-bit storage; the
reference-offset storage is printed for the record.
"""
import os

import numpy as np
import pytest

from paper_1112_5547_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(os.environ.get("LBM_STUDY") != "1", reason="set LBM_STUDY=1 (ten-minute oracle)")]

G0 = 2.4 / 1.04
L, STEPS = 128, 5000


def _obs(rhoA, p, u, R0):
    r = inputs.radial_distance(rhoA.shape, (L / 2.0,) * 3)
    rin = rhoA[r < R0 / 4].mean()
    rout = rhoA[r > R0 + 8].mean()
    R = (3 * (rhoA - rout).sum() / (rin - rout) / (4 * np.pi)) ** (1 / 3)
    dP = p[r < R / 4].mean() - p[r > R + 8].mean()
    return np.array([R, dP, np.sqrt((u ** 2).sum(-1)).max()])


def test_cfg2_128_storage_modes(oracle_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5547_gb300 import build, lbm_sc
    build.build()
    R0 = L / 4
    f = inputs.drop((L, L, L), R0, seed=2)
    o = oracle_mod.OracleSC(1, (L, L, L), 1.0, 1.0, G0).init(*f).step(STEPS)
    a, b, u, p = o.moments()
    ref = _obs(a, p, u, R0)
    print("oracle R %.5f dP %.6e umax %.6e" % tuple(ref))
    rows = {}
    for prec, refrho in (("f32", 0), ("bf16_rest", 0), ("f16_rest", 0), ("bf16", 1), ("f16", 1)):
        lat = lbm_sc.Lattice(1, (L, L, L), 1.0, 1.0, G0, prec, *((1.0, 0.04) if refrho else (0.0, 0.0))).init(*f)
        lat.step(STEPS)
        rA, rB, uu, pp = (t.double().cpu().numpy() for t in lat.moments())
        err = np.abs(_obs(rA, pp, uu, R0) / ref - 1)
        rows[prec] = err
        print("%-10s R %.2e dP %.2e umax %.2e" % ((prec,) + tuple(err)))
        del lat
        torch.cuda.empty_cache()
    assert np.all(rows["f32"] < 1e-3)
    assert np.all(rows["bf16_rest"] < 1e-2)
    assert np.all(rows["f16_rest"] < 1e-2)
