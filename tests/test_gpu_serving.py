"""Continuous-batching server: every request's result (density field and step
count) is the same served in a mix as solved alone, requests that arrive while
others run are admitted as memory frees up, and the HBM budget is respected."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_5547_gb300 import build, serving
    build.build()
    return serving


def _small_requests(sv, n=8, seed=3):
    return sv.poisson_requests(n, rate=200.0, seed=seed, sizes2=(64, 96), sizes3=(32, 40))


def test_served_equals_alone(sv):
    reqs = _small_requests(sv)
    srv = sv.Server(hbm_budget=80e9, chunk=100, check_every=500, max_steps=1500, keep_fields=True)
    res, st = srv.run(reqs)
    assert len(res) == len(reqs)
    assert st.max_resident >= 2  # requests overlapped on the device
    for r in reqs:
        alone, _ = sv.solve_alone(r, chunk=100, check_every=500, max_steps=1500, keep_fields=True)
        got = res[r.rid]
        assert got.steps == alone.steps and got.converged == alone.converged
        assert np.array_equal(got.rhoA, alone.rhoA), r.rid
    assert st.p99_s >= st.p50_s > 0


def test_drops_and_interfaces_served_equal_alone(sv):
    """A stream with flat-interface relaxations among the drops: each result is
    the same served in the mix as solved alone."""
    reqs = sv.poisson_requests(8, rate=200.0, seed=11, sizes2=(64, 96), sizes3=(32, 40), interface_fraction=0.5)
    assert {r.kind for r in reqs} == {"drop", "interface"}
    srv = sv.Server(hbm_budget=80e9, chunk=100, check_every=500, max_steps=1500, keep_fields=True)
    res, st = srv.run(reqs)
    assert st.max_resident >= 2
    for r in reqs:
        alone, _ = sv.solve_alone(r, chunk=100, check_every=500, max_steps=1500, keep_fields=True)
        assert res[r.rid].steps == alone.steps and np.array_equal(res[r.rid].rhoA, alone.rhoA), r.rid


def test_mixed_storage_precisions_served_equal_alone(sv):
    """Requests that store their populations in FP32, bf16 rest-offset or fp16
    rest-offset words arrive in one stream: the server steps each lattice kind
    and storage precision as its own batch, and each result (field and step
    count) is the same served in the mix as solved alone."""
    import dataclasses
    precs = ("f32", "bf16_rest", "f16_rest")
    reqs = [dataclasses.replace(r, precision=precs[r.rid % 3]) for r in _small_requests(sv, n=9, seed=21)]
    assert {r.precision for r in reqs} == set(precs)
    srv = sv.Server(hbm_budget=80e9, chunk=100, check_every=500, max_steps=1500, keep_fields=True)
    res, st = srv.run(reqs)
    assert len(res) == len(reqs) and st.max_resident >= 2
    for r in reqs:
        alone, _ = sv.solve_alone(r, chunk=100, check_every=500, max_steps=1500, keep_fields=True)
        assert res[r.rid].steps == alone.steps and np.array_equal(res[r.rid].rhoA, alone.rhoA), (r.rid, r.precision)


def test_admission_respects_budget(sv):
    """A budget that holds only two of these lattices: at most two are resident,
    the rest wait, and every request still finishes with its own result."""
    reqs = sv.poisson_requests(5, rate=1000.0, seed=5, d3_fraction=1.0, sizes3=(40,))
    fp = sv.Server.footprint(reqs[0])
    srv = sv.Server(hbm_budget=sv.Server.RESERVE_BYTES + 2.5 * fp, chunk=100, check_every=500, max_steps=1000,
                    keep_fields=True)
    res, st = srv.run(reqs)
    assert st.max_resident == 2
    assert [r.rid for r in res] == list(range(5))
    for r in reqs[:2]:
        alone, _ = sv.solve_alone(r, chunk=100, check_every=500, max_steps=1000, keep_fields=True)
        assert np.array_equal(res[r.rid].rhoA, alone.rhoA)


def test_active_node_cap(sv):
    """With a cap on resident nodes, no more than the cap is resident (beyond a
    single over-sized request), and results are unchanged."""
    reqs = sv.poisson_requests(6, rate=1000.0, seed=6, d3_fraction=1.0, sizes3=(32,))
    srv = sv.Server(chunk=100, check_every=500, max_steps=1000, keep_fields=True, max_active_nodes=2 * 32 ** 3)
    res, st = srv.run(reqs)
    assert st.max_resident == 2
    for r in reqs[:2]:
        alone, _ = sv.solve_alone(r, chunk=100, check_every=500, max_steps=1000, keep_fields=True)
        assert np.array_equal(res[r.rid].rhoA, alone.rhoA)


def test_diagnostics_check_of_65_slots_stays_in_its_rows(sv):
    """One check of 65 due slots writes exactly one lbm_sc_diag per row: a guard
    placed right after the last row is untouched, and each row's max|u_phys|
    equals the handle diagnostics of that lattice."""
    import torch
    from paper_1112_5547_gb300 import inputs, lbm_sc
    srv = sv.Server(chunk=100, check_every=500)
    w = sv.DIAG_DOUBLES
    assert w * 8 == __import__("ctypes").sizeof(lbm_sc.lbm_sc_diag)
    n = 65
    guard = 12345.678
    buf = torch.full((n * w + 64,), guard, dtype=torch.float64, device="cuda")
    srv._diag = buf[:n * w].view(n, w)

    class _S:
        pass

    slots = []
    with torch.cuda.stream(srv.stream):
        for k in range(n):
            sh = (24, 24 + (k % 3) * 8)
            s = _S()
            s.lat = lbm_sc.Lattice(lbm_sc.LBM_D2Q9, sh, 1.0, 1.0, 2.4 / 1.04, "f32", stream=srv.stream).init(
                *inputs.drop(sh, 5, seed=k, dtype=np.float32))
            s.lat.step(3)
            slots.append(s)
        got = srv._check(slots)
        srv.stream.synchronize()
    assert np.all(buf[n * w:].cpu().numpy() == guard)
    for s, (u, unstable) in zip(slots, got):
        assert u == s.lat.diagnostics()["max_speed"] and not unstable
        s.lat.close()
