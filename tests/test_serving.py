"""Request loop with continuous batching (emg_server_*): admission by slots and memory,
overlapping solves, and results that are bitwise the same alone and in the mix."""
import numpy as np
import pytest

from workloads import SolveRequest, ogrid, request_stream


# ---------------------------------------------------------------- host only (no GPU)

def test_request_stream_is_seeded_and_follows_its_recipe():
    a = request_stream()
    b = request_stream()
    assert a == b and len(a) == 64 and a[0].arrival == 0.0
    assert all(x.arrival <= y.arrival for x, y in zip(a, a[1:]))
    big = request_stream(n=4000, seed=7)
    gaps = np.diff([r.arrival for r in big])
    assert abs(gaps.mean() - 0.25) < 0.02            # Poisson arrivals at 4 per second
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.1  # exponential gaps: cv = 1
    grids = {(r.n_theta, r.n_r) for r in big}
    assert grids == {(32, 16), (64, 32), (128, 64), (256, 128)}
    assert {r.p for r in big} == {1, 2, 3, 4}
    ma = np.array([r.mach for r in big])
    assert ma.min() >= 0.1 and ma.max() <= 0.5 and abs(ma.mean() - 0.3) < 0.01


def test_estimate_is_host_only_and_orders_the_forms():
    from paper_1807_01151_gb300 import estimate_device_bytes
    m = ogrid(16, 8)
    b = [estimate_device_bytes(m, p_max=p) for p in range(5)]
    assert all(x < y for x, y in zip(b, b[1:]))
    # FP32 blocks halve the block bytes but add FP32 copies of the tables: smaller from p = 3
    for p in (3, 4):
        assert estimate_device_bytes(m, p_max=p, prec=1) < estimate_device_bytes(m, p_max=p, prec=0)
    # the p = 4 FP64 blocks alone: E (75^2) doubles
    assert b[4] > 16 * 8 * 75 * 75 * 8


def test_server_rejects_a_request_larger_than_its_budget_without_a_gpu():
    from paper_1807_01151_gb300 import Server
    srv = Server(max_active=2, mem_budget=1000, max_cycles=10)
    rid = srv.submit(ogrid(8, 4), p_max=1)
    assert srv.step() == (0, 0)
    res = srv.results()
    assert len(res) == 1 and res[0]["id"] == rid and res[0]["status_name"] == "EMG_ERR_OOM"
    assert res[0]["cycles"] == 0 and res[0]["t_done"] >= res[0]["t_submit"]
    srv.close()


def test_cancel_of_a_queued_request_needs_no_gpu():
    from paper_1807_01151_gb300 import EmgError, Server
    srv = Server(max_active=1, mem_budget=1 << 40, max_cycles=10)
    a = srv.submit(ogrid(8, 4), p_max=1)
    b = srv.submit(ogrid(8, 4), p_max=2)
    srv.cancel(b)
    res = srv.results()
    assert [(r["id"], r["status_name"], r["cycles"]) for r in res] == [(b, "EMG_CANCELLED", 0)]
    with pytest.raises(EmgError):
        srv.cancel(b)              # already finished
    with pytest.raises(EmgError):
        srv.cancel(12345)          # unknown
    srv.cancel(a)
    assert [r["status_name"] for r in srv.results()] == ["EMG_CANCELLED"]
    srv.close()


# ---------------------------------------------------------------- GPU

MIX = [  # (grid, p, Ma, prec): subcritical cases that converge to 1e-10 in both forms
    ((16, 8), 1, 0.2, 0),
    ((32, 16), 2, 0.3, 1),
    ((16, 8), 3, 0.3, 1),
    ((24, 12), 2, 0.2, 0),
]


def _alone(grid, p, ma, prec):
    from paper_1807_01151_gb300 import Solver
    s = Solver(ogrid(*grid), p_max=p, mach=ma, prec=prec)
    rep = s.solve_steady(drop=1e-10, max_cycles=2000)
    U = s.get_state()
    s.close()
    return U, rep["cycles"]


def _serve(reqs, max_active, mem_budget=0, max_cycles=2000):
    from paper_1807_01151_gb300 import Server
    srv = Server(max_active=max_active, mem_budget=mem_budget, max_cycles=max_cycles, keep_state=True)
    ids = [srv.submit(ogrid(*g), p_max=p, mach=ma, prec=prec) for g, p, ma, prec in reqs]
    res, peak = {}, 0
    while len(res) < len(ids):
        a, q = srv.step()
        peak = max(peak, a)
        for r in srv.results():
            res[r["id"]] = r
    states = {i: srv.take_state(i) for i in ids if res[i]["status"] == 0}
    srv.close()
    return ids, res, states, peak


@pytest.mark.gpu
def test_estimate_equals_the_context_footprint():
    from paper_1807_01151_gb300 import Solver, estimate_device_bytes
    from workloads import cubed_sphere_shell
    for mesh, p, prec in [(ogrid(16, 8), 2, 0), (ogrid(16, 8), 3, 1), (cubed_sphere_shell(2, 2), 2, 1)]:
        s = Solver(mesh, p_max=p, prec=prec)
        assert s.device_bytes == estimate_device_bytes(mesh, p_max=p, prec=prec)
        s.close()


@pytest.mark.gpu
def test_results_are_bitwise_the_same_alone_and_in_the_mix():
    alone = [_alone(*r) for r in MIX]
    for slots in (4, 2):   # all at once; and half of them queued until slots free up
        ids, res, states, peak = _serve(MIX, max_active=slots)
        assert peak == min(slots, len(MIX))
        for k, i in enumerate(ids):
            assert res[i]["status"] == 0, res[i]
            assert res[i]["cycles"] == alone[k][1]
            assert res[i]["res_final"] <= 1e-10 * res[i]["res0"]
            np.testing.assert_array_equal(states[i], alone[k][0])


@pytest.mark.gpu
def test_admission_waits_for_memory_and_rejects_what_never_fits():
    from paper_1807_01151_gb300 import estimate_device_bytes
    reqs = [((16, 8), 2, 0.3, 0), ((16, 8), 2, 0.35, 0), ((64, 32), 4, 0.3, 0)]
    est = [estimate_device_bytes(ogrid(*g), p_max=p, prec=prec) for g, p, ma, prec in reqs]
    budget = est[0] + est[1] - 1                       # the two small ones cannot run together
    assert est[2] > budget
    ids, res, states, peak = _serve(reqs, max_active=3, mem_budget=budget)
    assert peak == 1
    a, b, c = (res[i] for i in ids)
    assert a["status"] == 0 and b["status"] == 0
    assert b["t_admit"] >= a["t_done"]                 # admitted once the first one's memory was free
    assert c["status_name"] == "EMG_ERR_OOM" and c["cycles"] == 0


@pytest.mark.gpu
def test_cycle_limit_ends_one_solve_without_disturbing_the_others():
    reqs = [((16, 8), 2, 0.3, 0), ((16, 8), 1, 0.3, 0)]
    ids, res, states, peak = _serve(reqs, max_active=2, max_cycles=5)
    for i in ids:
        assert res[i]["status_name"] == "EMG_ERR_NOT_CONVERGED" and res[i]["cycles"] == 5


@pytest.mark.gpu
def test_stream_driver_serves_arrivals_and_reports_latency():
    from paper_1807_01151_gb300 import serving
    reqs = [SolveRequest(0.05 * k, g[0], g[1], p, ma) for k, (g, p, ma, _) in enumerate(MIX * 2)]
    out, summ, states = serving.serve_stream(reqs, lambda r: ogrid(r.n_theta, r.n_r), max_active=4,
                                             keep_state=True)
    assert summ["converged"] == len(reqs) and summ["peak_active"] >= 2
    assert 0.0 < summ["p50_s"] <= summ["p99_s"] <= summ["makespan_s"] + 1e-9
    for k in range(len(MIX)):      # the same request twice in one stream: the same result
        np.testing.assert_array_equal(states[k], states[k + len(MIX)])


@pytest.mark.gpu
def test_stall_detection_ends_a_solve_that_stops_improving():
    from paper_1807_01151_gb300 import Server
    srv = Server(max_active=1, drop=1e-30, max_cycles=2000, stall_cycles=20)   # a drop no solve reaches
    rid = srv.submit(ogrid(16, 8), p_max=1, mach=0.3)
    res = []
    while not res:
        srv.step()
        res = srv.results()
    srv.close()
    r = res[0]
    assert r["id"] == rid and r["status_name"] == "EMG_ERR_NOT_CONVERGED"
    assert 20 < r["cycles"] < 2000 and r["res_final"] < 1e-9 * r["res0"]


@pytest.mark.gpu
def test_cancel_of_an_active_request_leaves_the_others_intact():
    from paper_1807_01151_gb300 import Server
    U_alone, cycles_alone = _alone(*MIX[0])
    srv = Server(max_active=2, max_cycles=2000, keep_state=True)
    keep = srv.submit(ogrid(*MIX[0][0]), p_max=MIX[0][1], mach=MIX[0][2], prec=MIX[0][3])
    gone = srv.submit(ogrid(64, 32), p_max=3, mach=0.3, prec=1)
    res = {}
    cancelled = False
    while len(res) < 2:
        a, q = srv.step()
        if not cancelled and a == 2:
            srv.cancel(gone)
            cancelled = True
        for r in srv.results():
            res[r["id"]] = r
    assert res[gone]["status_name"] == "EMG_CANCELLED"
    assert res[keep]["status"] == 0 and res[keep]["cycles"] == cycles_alone
    np.testing.assert_array_equal(srv.take_state(keep), U_alone)
    srv.close()


@pytest.mark.gpu
def test_served_golden_request_ends_at_the_oracle_steady_state():
    """The golden case (32x16 O-grid, p = 2, Ma 0.3; tests/golden, written from oracle/ alone)
    served among other solves, in the FP64 and the FP32-block form, ends at the oracle's steady
    state to 1e-9 (the fixed point R = 0 does not depend on the preconditioner or the mix)."""
    import os
    from tests.helpers import rel_err
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "cyl32x16_p2_steady.npz"))
    reqs = [((32, 16), 2, 0.3, 0), ((16, 8), 3, 0.3, 1), ((32, 16), 2, 0.3, 1), ((24, 12), 2, 0.2, 0)]
    ids, res, states, _ = _serve(reqs, max_active=3)
    for k in (0, 2):
        r = res[ids[k]]
        assert r["status"] == 0 and r["res_final"] <= 1e-10 * r["res0"], r
        assert rel_err(states[ids[k]], g["u"]) < 1e-9, (k, rel_err(states[ids[k]], g["u"]))
