"""Failure detection without a fault: every mbarrier wait of the TMA-fed
kernels is bounded.  A test hook (lbm_sc_set_wait_probe) makes the first CTA
wait on a barrier that nothing arrives on; its wait runs out after a few tries,
the CTA raises the error word, drains its own copies (with the full bound) and
returns.  The host then reads LBM_ERR_TIMEOUT, and the same handle, the hook
off and its fields re-initialised, steps on to the oracle's result: the GPU and
the context are unaffected."""
import numpy as np
import pytest

from paper_1112_5547_gb300 import inputs

pytestmark = pytest.mark.gpu

G0 = 2.4 / 1.04


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5547_gb300 import build, lbm_sc
    build.build()
    return lbm_sc


@pytest.mark.parametrize("precision,tile,tol", [("f32", 34, 1e-5), ("bf16_rest", 35, 2e-3)])
def test_expired_wait_reports_timeout_and_the_gpu_stays_usable(sc, oracle_mod, precision, tile, tol):
    shape = (12, 12, 64)  # (nz, ny, nx): two 64x6 tiles in y
    f = inputs.drop(shape, 5, seed=13)
    lat = sc.Lattice(sc.LBM_D3Q19, shape, 1.0, 1.0, G0, precision).init(*f)
    lat.set_tuning(tile, 0)
    assert lat.tuning()[0] == tile
    assert sc.lbm_sc_error_word(lat.handle) == 0
    sc.lbm_sc_set_wait_probe(lat.handle, 64)
    lat.step(1)
    st, _ = sc.lbm_sc_diagnostics(lat.handle, check=False)
    assert st == sc.LBM_ERR_TIMEOUT
    assert sc.lbm_sc_error_word(lat.handle) == 1  # expired, and every copy in flight landed before the CTA left
    with pytest.raises(sc.LbmError):
        sc.lbm_sc_set_wait_probe(lat.handle, -1)
    sc.lbm_sc_set_wait_probe(lat.handle, 0)
    lat.init(*f)
    assert sc.lbm_sc_error_word(lat.handle) == 0
    lat.step(20)
    d = lat.diagnostics()
    assert d["status"] == sc.LBM_OK
    g = [t.double().cpu().numpy() for t in lat.moments()]
    o = oracle_mod.OracleSC(1, shape, 1.0, 1.0, G0).init(*f).step(20).moments()
    for a, b in ((g[0], o[0]), (g[1], o[1])):
        assert np.abs(a - b).max() / np.abs(b).max() < tol
