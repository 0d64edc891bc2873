"""Serving loop (skr_server_*, skr_submit, skr_poll) through the C ABI."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import assembly  # noqa: E402
from workloads import darcy2d_sequence, darcy3d_sequence  # noqa: E402


@pytest.fixture(scope="module")
def skr():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__ as g
    g.build()
    import paper_2401_09516_gb300 as m
    return m


def _opts(skr, **kw):
    base = dict(m=30, k=8, tol=1e-8, precond="jacobi", precision="mixed")
    base.update(kw)
    return skr.skr_options_default(**base)


def _direct(loga):
    A, b = (assembly.darcy3d(loga) if loga.ndim == 3 else assembly.darcy2d(loga))
    return A, b, spla.spsolve(A.tocsc(), b)


def _mix():
    reqs = []
    for side, seed in ((32, 1), (48, 2)):
        for loga in darcy2d_sequence(side, 4, 0.2, seed=seed):
            reqs.append(loga)
    for loga in darcy3d_sequence(10, 3, 0.3, seed=3):
        reqs.append(loga)
    order = np.random.default_rng(7).permutation(len(reqs))
    return [reqs[i] for i in order]


def _system(skr, loga):
    return skr.darcy3d(loga) if loga.ndim == 3 else skr.darcy2d(loga)


def test_mixed_stream_matches_direct_solves(skr):
    reqs = _mix()
    with skr.Server(_opts(skr)) as srv:
        tickets = [srv.submit(_system(skr, l)) for l in reqs]
        outs = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0
    assert st["chains"] >= 3          # one per grid shape at least
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for loga, (x, res) in zip(reqs, outs):
        A, b, xd = _direct(loga)
        assert res["flag"] == 0, res
        assert np.linalg.norm(b - A @ x) <= 1.01e-8 * np.linalg.norm(b)
        assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)


def test_same_result_alone_and_in_the_mix(skr):
    reqs = _mix()
    probe = reqs[len(reqs) // 2]
    with skr.Server(_opts(skr)) as srv:
        x_alone, r_alone = srv.wait(srv.submit(_system(skr, probe)))
    with skr.Server(_opts(skr)) as srv:
        tickets = [srv.submit(_system(skr, l)) for l in reqs[: len(reqs) // 2]]
        tp = srv.submit(_system(skr, probe))
        tickets += [srv.submit(_system(skr, l)) for l in reqs[len(reqs) // 2 + 1:]]
        x_mix, r_mix = srv.wait(tp)
        for t in tickets:
            srv.wait(t)
    assert r_alone["flag"] == 0 and r_mix["flag"] == 0
    # both solves meet the same tolerance; they may differ only by it
    err = np.linalg.norm(x_alone - x_mix) / np.linalg.norm(x_alone)
    assert err <= 2e-6, err


def test_budget_admission_serialises_and_rejects_oversize(skr):
    L = darcy2d_sequence(40, 5, 0.2, seed=11)
    with skr.Server(_opts(skr), hbm_budget=0, max_chains=1) as srv:
        ts = [srv.submit(skr.darcy2d(l)) for l in L]
        outs = [srv.wait(t) for t in ts]
        st = srv.stats()
    assert st["chains"] == 1 and st["completed"] == 5
    # requests served on one chain reuse its recycle space
    assert outs[-1][1]["k_final"] > 0
    for loga, (x, res) in zip(L, outs):
        A, b, xd = _direct(loga)
        assert res["flag"] == 0
        assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
    with skr.Server(_opts(skr), hbm_budget=1 << 16) as srv:
        with pytest.raises(skr.SkrError) as e:
            srv.submit(skr.darcy2d(L[0]))
        assert e.value.status == skr._native.SKR_ERR_OOM


def test_unknown_ticket_and_routing_key(skr):
    L = darcy2d_sequence(24, 3, 0.2, seed=12)
    with skr.Server(_opts(skr)) as srv:
        with pytest.raises(skr.SkrError):
            skr.skr_poll(srv.handle, 12345, 10)
        t = srv.submit(skr.darcy2d(L[0]), key=np.array([0.0, 1.0]))
        x, res = srv.wait(t)
        assert res["flag"] == 0
        with pytest.raises(skr.SkrError):
            skr.skr_poll(srv.handle, t, x.size)     # a ticket is forgotten once collected


def test_warm_start_carries_the_previous_solution_of_a_chain(skr):
    loga = darcy2d_sequence(24, 1, 0.2, seed=9)[0]
    with skr.Server(_opts(skr, precision="fp64", warm_start=1), max_chains=1) as srv:
        x1, r1 = srv.wait(srv.submit(_system(skr, loga)))
        x2, r2 = srv.wait(srv.submit(_system(skr, loga)))
    assert r1["flag"] == 0 and r2["flag"] == 0
    assert r1["steps"] > 0 and r2["steps"] == 0, (r1, r2)
    np.testing.assert_array_equal(x2, x1)


@pytest.mark.parametrize("pc,blocks", [("bjacobi", 12), ("ssor", 1)])
def test_colour_sweep_preconditioners_in_the_serving_loop(skr, pc, blocks):
    reqs = _mix()
    with skr.Server(_opts(skr, precond=pc, pc_blocks=blocks)) as srv:
        outs = [srv.wait(t) for t in [srv.submit(_system(skr, l)) for l in reqs]]
    for loga, (x, res) in zip(reqs, outs):
        A, b, xd = _direct(loga)
        assert res["flag"] == 0, res
        assert np.linalg.norm(b - A @ x) <= 1.01e-8 * np.linalg.norm(b)
        assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)


def _interleaved_two_shapes():
    a = darcy2d_sequence(24, 3, 0.2, seed=21)
    b = darcy2d_sequence(32, 3, 0.2, seed=22)
    return [a[0], b[0], a[1], b[1], a[2], b[2]]


def _check_all_solved(reqs, outs):
    for loga, (x, res) in zip(reqs, outs):
        A, b, xd = _direct(loga)
        assert res["flag"] == 0, res
        assert np.linalg.norm(b - A @ x) <= 1.01e-8 * np.linalg.norm(b)
        assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)


def test_one_chain_serves_two_interleaved_shapes_by_eviction(skr):
    # max_chains = 1: every request of the other shape evicts the idle chain
    reqs = _interleaved_two_shapes()
    with skr.Server(_opts(skr), max_chains=1) as srv:
        tickets = [srv.submit(skr.darcy2d(l)) for l in reqs]
        outs = [srv.wait(t, timeout=120.0) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0
    assert st["chains"] == 1 and st["evicted"] >= 1
    _check_all_solved(reqs, outs)


def test_budget_of_one_chain_serves_two_shapes(skr):
    # a device-memory budget that holds one chain of the larger shape only
    reqs = _interleaved_two_shapes()
    with skr.Server(_opts(skr), max_chains=1) as probe:
        probe.wait(probe.submit(skr.darcy2d(reqs[1])))
        one = probe.stats()["hbm_bytes"]
    with skr.Server(_opts(skr), hbm_budget=int(one * 1.5)) as srv:
        tickets = [srv.submit(skr.darcy2d(l)) for l in reqs]
        outs = [srv.wait(t, timeout=120.0) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["hbm_bytes"] <= one * 1.5
    assert st["evicted"] >= 1
    _check_all_solved(reqs, outs)


def test_requests_beyond_the_sms_wait_and_all_complete(skr):
    # 3D requests of 8-CTA clusters: more than fit on the GPU at once are
    # queued by the server, not launched into the hardware queue, and all finish
    L = darcy3d_sequence(40, 24, 0.3, seed=23)
    with skr.Server(_opts(skr, cluster_size=8), max_chains=64) as srv:
        tickets = [srv.submit(skr.darcy3d(l)) for l in L]
        outs = [srv.wait(t, timeout=300.0) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(L)
    for loga, (x, res) in zip(L[:3], outs[:3]):
        A, b, xd = _direct(loga)
        assert res["flag"] == 0, res
        assert np.linalg.norm(x - xd) <= 1e-6 * np.linalg.norm(xd)
