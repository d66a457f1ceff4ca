"""Host-side logic of the server: the seeded Poisson request stream and the
footprint used for admission (no GPU needed)."""
import numpy as np


def test_poisson_stream_is_seeded_and_in_range():
    from paper_1112_5547_gb300 import inputs, lbm_sc, serving
    a = serving.poisson_requests(400, rate=50.0, seed=7)
    b = serving.poisson_requests(400, rate=50.0, seed=7)
    assert [(r.shape, r.G, r.arrival) for r in a] == [(r.shape, r.G, r.arrival) for r in b]
    t = np.array([r.arrival for r in a])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.25 / 50.0  # mean inter-arrival 1/rate
    d3 = [r for r in a if r.lattice == lbm_sc.LBM_D3Q19]
    assert 0.35 < len(d3) / len(a) < 0.65
    for r in a:
        L = r.shape[0]
        assert 2.2 <= r.G * inputs.RHO_TOT <= 2.8
        assert 0.6 <= r.tau_A <= 1.5 and 0.6 <= r.tau_B <= 1.5
        assert L / 8 <= r.R <= L / 3
        assert all(0 <= c < L for c in r.centre)
        assert len(r.centre) == len(r.shape)


def test_footprint_is_the_workspace_and_the_batch_share():
    """A request's footprint is its workspace plus a bound on its share of the batch
    workspace, and that bound covers lbm_sc_batch_workspace_bytes for every batch
    tile the request's lattice takes, FP32 and rest-offset storage alike (handles
    are host-only: no GPU needed)."""
    from paper_1112_5547_gb300 import lbm_sc, serving
    r = serving.poisson_requests(1, seed=1, d3_fraction=1.0, sizes3=(192,))[0]
    p = lbm_sc.make_params(r.lattice, r.shape, r.tau_A, r.tau_B, r.G, "f32")
    assert serving.Server.footprint(r) == lbm_sc.lbm_sc_workspace_bytes(p) + serving.Server.batch_share(r)
    # the largest D3Q19 request: two FP32 buffers of 2 x 19 values per node
    assert serving.Server.footprint(r) >= 2 * 2 * 19 * 4 * 192 ** 3
    reqs = [q for prec in ("f32", "bf16_rest", "f16_rest")
            for q in serving.poisson_requests(12, seed=2, sizes2=(64, 1024), sizes3=(32, 40, 192), precision=prec)]
    for req in reqs:
        q = lbm_sc.make_params(req.lattice, req.shape, req.tau_A, req.tau_B, req.G, req.precision)
        h = lbm_sc.lbm_sc_create(q, 256 * 1024, lbm_sc.lbm_sc_workspace_bytes(q), 0)
        try:
            for tile in range(len(lbm_sc.BATCH_TILES)):
                for zc in (0, 1, 16):
                    ws = lbm_sc.lbm_sc_batch_workspace_bytes([h], tile, zc)
                    # one lattice's batch: its share plus the queue counters and the alignment slack
                    assert ws <= serving.Server.batch_share(req) + 1024, (req.shape, tile, zc, ws)
        finally:
            lbm_sc.lbm_sc_destroy(h)


def test_ragged_batch_specs_seeded_and_in_range():
    """The ragged-batch recipe: seeded, sizes from the set, G rho_tot, tau and R in range."""
    from paper_1112_5547_gb300 import inputs
    a = inputs.ragged_drop_specs()
    b = inputs.ragged_drop_specs()
    assert [(s["shape"], s["G"], s["R"], s["centre"]) for s in a] == [(s["shape"], s["G"], s["R"], s["centre"]) for s in b]
    assert len(a) == 64
    assert {s["shape"][0] for s in a} <= {32, 48, 64, 96, 128}
    for s in a:
        L = s["shape"][0]
        assert s["shape"] == (L, L, L)
        assert 2.2 <= s["G"] * inputs.RHO_TOT <= 2.8
        assert 0.6 <= s["tau_A"] <= 1.5 and 0.6 <= s["tau_B"] <= 1.5
        assert L / 8 <= s["R"] <= L / 3
    rA, rB = inputs.spec_fields(a[0])
    assert rA.shape == a[0]["shape"] and abs((rA + rB).mean() - inputs.RHO_TOT) < 1e-3


def test_interface_requests():
    """interface_fraction mixes flat-interface relaxations into the stream (a slab
    of half-width R across x), and 0 leaves the drops-only stream untouched."""
    from paper_1112_5547_gb300 import serving
    a = serving.poisson_requests(30, 50.0, 4)
    b = serving.poisson_requests(30, 50.0, 4, interface_fraction=0.0)
    assert [(r.shape, r.R, r.arrival, r.kind) for r in a] == [(r.shape, r.R, r.arrival, r.kind) for r in b]
    c = serving.poisson_requests(40, 50.0, 4, interface_fraction=0.5)
    kinds = [r.kind for r in c]
    assert 5 < kinds.count("interface") < 35
    r = next(q for q in c if q.kind == "interface")
    rA, rB = r.fields()
    assert rA.shape == r.shape
    L = r.shape[-1]
    x = np.arange(L)
    d = np.abs((x - r.centre[0] + L / 2) % L - L / 2)  # periodic distance to the slab centre
    prof = rA.reshape(-1, L).mean(0)
    assert prof[d < r.R - 4].min() > 0.9 and prof[d > r.R + 4].max() < 0.1
    assert serving.Server.footprint(r) > 0


def test_check_flags_non_positive_densities_and_non_finite_values():
    """check_of reads max|u_phys| and the instability rule from one diagnostics
    row: a species density that is zero or negative somewhere, or a non-finite
    value, marks the request unstable (the server retires it at that check)."""
    import ctypes

    import numpy as np

    from paper_1112_5547_gb300 import lbm_sc, serving

    def row(**kw):
        d = lbm_sc.lbm_sc_diag()
        d.min_rho_A, d.min_rho_B, d.max_speed = 0.04, 0.04, 0.02
        for k, v in kw.items():
            setattr(d, k, v)
        buf = np.frombuffer(bytes(d), dtype=np.float64)
        assert buf.size == serving.DIAG_DOUBLES == ctypes.sizeof(lbm_sc.lbm_sc_diag) // 8
        return buf

    assert serving.check_of(row()) == (0.02, False)
    assert serving.max_speed_of(row(max_speed=0.5)) == 0.5
    assert serving.check_of(row(min_rho_A=-1e-4))[1]
    assert serving.check_of(row(min_rho_B=0.0))[1]
    assert serving.check_of(row(nonfinite=3.0))[1]
    assert serving.check_of(row(min_rho_A=float("nan")))[1]
