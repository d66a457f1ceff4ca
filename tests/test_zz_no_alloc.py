"""lbm_sc_diagnostics_noalloc -- the diagnostics for callers that cannot
allocate device memory -- agrees with lbm_sc_diagnostics on two calls in a
row.  Kept in a file of its own, collected last."""
import ctypes

import numpy as np
import pytest

from paper_1112_5547_gb300 import inputs

pytestmark = pytest.mark.gpu

G0 = 2.4 / 1.04
SUMS = ("mass_A", "mass_B", "kinetic_energy", "in_count", "in_rho_A", "in_p", "out_count", "out_rho_A", "out_p")


@pytest.fixture(scope="module")
def sc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5547_gb300 import build, lbm_sc
    build.build()
    return lbm_sc


def _from_device(dev):
    raw = dev.cpu().numpy().tobytes()
    import paper_1112_5547_gb300.lbm_sc as m
    d = m.lbm_sc_diag.from_buffer_copy(raw)
    return d.as_dict()


@pytest.mark.parametrize("lattice,shape,precision", [(1, (24, 40, 70), "f32"), (0, (96, 130), "f64"),
                                                     (1, (24, 40, 70), "bf16"), (1, (24, 40, 70), "bf16_rest")])
def test_noalloc_diagnostics_match_handle_diagnostics(sc, lattice, shape, precision):
    """Also on 16-bit storage (reference- and rest-offset), whose buffers carry the
    two FP32 density planes of the rest-offset mode after the populations: the
    static-scratch variant must read them at the handle's own layout."""
    import torch
    f = inputs.drop(shape, min(shape) / 4.0, seed=21)
    ref_rho = (1.0, 0.04) if precision == "bf16" else (0.0, 0.0)
    lat = sc.Lattice(lattice, shape, 1.0, 0.8, G0, precision, *ref_rho).init(*f).step(15)
    centre = tuple(n / 2.0 for n in reversed(shape))
    win = sc.Window(centre, 3.0, min(shape) / 2.5)
    ref = lat.diagnostics(win)
    eb, q, px, py, gx, gy, pop = sc.lbm_sc_layout(lat.handle)
    out = torch.zeros(ctypes.sizeof(sc.lbm_sc_diag) // 8, dtype=torch.float64, device="cuda")
    for call in range(2):  # two calls in a row share the static scratch
        out.fill_(-7.0)
        sc.lbm_sc_diagnostics_noalloc(lat.params, pop, win.to_c(), out.data_ptr(), lat.stream.cuda_stream)
        torch.cuda.synchronize()
        got = _from_device(out)
        for k in SUMS:
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-12), (call, k)
        np.testing.assert_allclose(got["momentum"], ref["momentum"], rtol=0, atol=1e-10)
        for k in ("max_speed", "min_rho_A", "min_rho_B", "nonfinite", "droplet_nodes"):
            assert got[k] == ref[k], (call, k)


def test_noalloc_rejects_a_lattice_too_large_for_the_static_scratch(sc):
    import torch
    p = sc.make_params(sc.LBM_D2Q9, (4200, 1024), 1.0, 1.0, 1.0, "f32")  # 4.3M nodes > 16384 tiles of 32 x 8
    out = torch.zeros(ctypes.sizeof(sc.lbm_sc_diag) // 8, dtype=torch.float64, device="cuda")
    with pytest.raises(sc.LbmError) as e:
        sc.lbm_sc_diagnostics_noalloc(p, 1 << 20, None, out.data_ptr(), 0)
    assert e.value.status == sc.LBM_ERR_INVALID_ARG
