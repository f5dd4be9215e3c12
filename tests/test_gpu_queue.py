"""Request queue with continuous batching: correctness in the mix, admission, cancellation, faults.

Faults are made on the host (an injected allocation failure, a source that is
not finite, a wait that times out on the host); nothing here faults the GPU.
"""
import os

import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field, unpack_field
from tests._lattice import rel_max_err, volume

pytestmark = pytest.mark.gpu

LATTICES = [(4, 4, 4, 4), (8, 8, 8, 8), (4, 6, 8, 10), (8, 8, 8, 16)]
_gauges = {}
_context = []


def _ctx():
    """One context for the module: the cached gauges below use its tuning cache."""
    if not _context:
        _context.append(wd.Context(0))
    return _context[0]


def _gauge(ctx, dims):
    key = dims
    if key not in _gauges:
        U = synth.gauge(dims, seed=1000 + volume(dims) % 983)
        _gauges[key] = (U, wd.Gauge(ctx, dims, U))
    return _gauges[key]


def _request(ctx, k, dims=None, tol=None, prec=wd.F16, seed=5001):
    rng = np.random.default_rng(seed + k)
    dims = dims or LATTICES[k % len(LATTICES)]
    U, g = _gauge(ctx, dims)
    mass = float(np.exp(rng.uniform(np.log(0.02), np.log(0.5))))
    tol = tol or float([1e-8, 1e-10, 1e-12][k % 3])
    b = synth.even_spinor(dims, seed=3300 + k)
    p = dict(gauge=g, mass=mass, tol=tol, inner_prec=prec, delta=0.1,
             b=pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, b), x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64))
    return p, (dims, U, mass, b)


def _true_rel(ctx, host, x_field):
    dims, U, mass, b = host
    x = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, x_field)
    return float(np.linalg.norm(b - oracle.mdagm(dims, U, mass, x)) / np.linalg.norm(b)), x


def test_queue_results_and_same_alone_as_in_mix():
    ctx = _ctx()
    q = wd.Queue(ctx, hbm_budget_bytes=8 << 30, max_slots=6)
    reqs = [_request(ctx, k) for k in range(12)]
    tickets = [q.submit(p) for p, _ in reqs]
    res = [q.wait(t, timeout_ms=120000) for t in tickets]
    mixed_x = []
    for (p, host), r in zip(reqs, res):
        assert r["status"] == 0, r
        rel, x = _true_rel(ctx, host, p["x"])
        assert rel <= p["tol"], (rel, p["tol"])
        assert r["t_submit"] <= r["t_admit"] <= r["t_start"] <= r["t_finish"]
        mixed_x.append(x)
    st = q.stats()
    assert st["completed"] == 12 and st["mean_running"] > 1.0
    q.close()
    # every request alone in a fresh one-slot queue gives the same bits: a request's
    # kernels and reductions do not depend on what else the queue runs
    for k in range(len(reqs)):
        p, host = reqs[k]
        alone = dict(p)
        alone["x"] = wd.alloc_field(host[0], wd.SITES_EVEN, wd.F64)
        q1 = wd.Queue(ctx, hbm_budget_bytes=8 << 30, max_slots=1)
        r = q1.wait(q1.submit(alone), timeout_ms=60000)
        q1.close()
        assert r["status"] == 0
        assert r["cg_iters"] == res[k]["cg_iters"], (k, r, res[k])
        _, xa = _true_rel(ctx, host, alone["x"])
        assert np.array_equal(mixed_x[k], xa), (k, rel_max_err(mixed_x[k], xa))


def test_requests_join_while_others_run():
    """Continuous batching: a request submitted while another runs is admitted before it ends."""
    ctx = _ctx()
    q = wd.Queue(ctx, hbm_budget_bytes=8 << 30, max_slots=4)
    small = [_request(ctx, k, dims=(4, 4, 4, 4), tol=1e-8)[0] for k in range(1, 4)]
    big, _ = _request(ctx, 0, dims=(16, 16, 16, 32), tol=1e-12)
    big["mass"] = 0.02
    t_big = q.submit(big)
    import time
    t_end = time.time() + 30
    while time.time() < t_end:
        st = q.stats()
        if st["running"] > 0 or st["completed"] > 0:
            break
        time.sleep(0.0005)
    ts = [q.submit(p) for p in small]
    rb = q.wait(t_big, timeout_ms=60000)
    rs = [q.wait(t, timeout_ms=60000) for t in ts]
    assert rb["status"] == 0 and all(r["status"] == 0 for r in rs)
    assert any(r["t_admit"] < rb["t_finish"] for r in rs)
    q.close()


def test_admission_respects_hbm_budget():
    ctx = _ctx()
    reqs = [_request(ctx, k, dims=(8, 8, 8, 8), tol=1e-10) for k in range(4)]
    # a budget of 1.5 request workspaces admits one request at a time
    one = wd.solve_workspace_bytes((8, 8, 8, 8), wd.F16)
    q = wd.Queue(ctx, hbm_budget_bytes=int(one * 1.5), max_slots=8)
    ts = [q.submit(p) for p, _ in reqs]
    res = [q.wait(t, timeout_ms=60000) for t in ts]
    st = q.stats()
    q.close()
    assert all(r["status"] == 0 for r in res)
    assert st["mean_running"] <= 1.0 + 1e-9
    assert st["admission_stalls"] > 0


def test_request_larger_than_budget_is_refused():
    ctx = _ctx()
    q = wd.Queue(ctx, hbm_budget_bytes=1 << 20, max_slots=2)
    p, _ = _request(ctx, 0, dims=(8, 8, 8, 8))
    with pytest.raises(wd.WdError) as e:
        q.submit(p)
    assert e.value.status == wd.WD_ENOMEM
    q.close()


def test_cancel_wait_timeout_and_poisoned_request():
    ctx = _ctx()
    q = wd.Queue(ctx, hbm_budget_bytes=8 << 30, max_slots=1)
    # a solve long enough (tens of ms) to still run while the others are submitted
    first, _ = _request(ctx, 0, dims=(16, 16, 16, 32), tol=1e-12)
    first["mass"] = 0.02
    later_reqs = [_request(ctx, k, dims=(4, 4, 4, 4))[0] for k in range(1, 4)]
    t0 = q.submit(first)
    with pytest.raises(wd.WdError) as e:
        q.wait(t0, timeout_ms=0)                           # host-side wait gives up; the request goes on
    assert e.value.status == wd.WD_ETIMEOUT
    later = [q.submit(r) for r in later_reqs]
    q.cancel(later[1])                                     # still waiting (one slot, busy): cancelled at once
    poisoned, _ = _request(ctx, 7, dims=(4, 4, 4, 4))
    nan = np.full((volume((4, 4, 4, 4)), 4, 3), np.nan, np.complex128)
    poisoned["b"] = pack_field(ctx, (4, 4, 4, 4), wd.SITES_EVEN, wd.F64, nan)
    tp = q.submit(poisoned)
    assert q.wait(t0, timeout_ms=60000)["status"] == 0
    assert q.wait(later[1], timeout_ms=60000)["status"] == wd.WD_ECANCELLED
    assert q.wait(later[0], timeout_ms=60000)["status"] == 0
    assert q.wait(later[2], timeout_ms=60000)["status"] == 0
    assert q.wait(tp, timeout_ms=60000)["status"] == wd.WD_EINVAL
    q.close()


def test_injected_allocation_failure(monkeypatch):
    ctx = _ctx()
    monkeypatch.setenv("WD_FAULT", "alloc:2")
    q = wd.Queue(ctx, hbm_budget_bytes=8 << 30, max_slots=1)
    reqs = [_request(ctx, k, dims=(4, 4, 4, 4), tol=1e-10) for k in range(4)]
    ts = [q.submit(p) for p, _ in reqs]
    res = [q.wait(t, timeout_ms=60000) for t in ts]
    q.close()
    assert [r["status"] for r in res] == [0, wd.WD_ENOMEM, 0, 0]
    assert _true_rel(ctx, reqs[2][1], reqs[2][0]["x"])[0] <= 1e-10


@pytest.mark.parametrize("prec", [wd.F16, wd.BF16])
def test_hard_solves_with_small_delta(prec):
    """Small mass, tight tolerance and delta = 0.01 (few reliable updates): every solve converges,
    with its true residual checked by the oracle."""
    ctx = _ctx()
    q = wd.Queue(ctx, hbm_budget_bytes=8 << 30, max_slots=8)
    reqs = []
    for k in range(6):
        p, host = _request(ctx, 20 + k, dims=[(8, 8, 8, 16), (8, 8, 8, 8), (4, 6, 8, 10)][k % 3], tol=1e-12, prec=prec)
        p["mass"] = 0.02
        p["delta"] = 0.01
        reqs.append((p, (host[0], host[1], 0.02, host[3])))
    ts = [q.submit(p) for p, _ in reqs]
    res = [q.wait(t, timeout_ms=120000) for t in ts]
    q.close()
    for (p, host), r in zip(reqs, res):
        assert r["status"] == 0, r
        assert _true_rel(ctx, host, p["x"])[0] <= 1e-12


def test_requests_on_one_gauge_share_group_launches():
    """Requests on the same gauge, inner precision and links iterate in one group: each
    launch of the group's loop serves several of them (mean group size > 1), and every
    result still meets its tolerance by the oracle."""
    ctx = _ctx()
    q = wd.Queue(ctx, hbm_budget_bytes=8 << 30, max_slots=8)
    reqs = [_request(ctx, k, dims=(8, 8, 8, 8), tol=1e-10) for k in range(8)]
    tickets = [q.submit(p) for p, _ in reqs]
    res = [q.wait(t, timeout_ms=120000) for t in tickets]
    st = q.stats()
    q.close()
    for (p, host), r in zip(reqs, res):
        assert r["status"] == 0, r
        assert _true_rel(ctx, host, p["x"])[0] <= p["tol"]
    assert st["group_launches"] > 0
    assert st["mean_group_size"] > 1.5, st


def test_results_taken_while_the_scheduler_runs():
    """Many short requests whose results are taken (wait and poll) as soon as each
    finishes, while new ones are submitted and others still run: a request finished in
    the scheduler's current pass stays valid until the scheduler has dropped it, so a
    result taken at that moment neither frees memory the scheduler still reads nor lets
    a new request reuse it.  Every request completes.  The fields of a request stay
    alive until its result is taken (the caller owns them)."""
    ctx = _ctx()
    q = wd.Queue(ctx, hbm_budget_bytes=8 << 30, max_slots=8)
    dims = (4, 4, 4, 4)
    U, g = _gauge(ctx, dims)
    b = pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, synth.even_spinor(dims, seed=3900))
    live = {}   # ticket -> request (keeps its x alive until the result is taken)
    order, statuses = [], []
    try:
        for k in range(240):
            p = dict(gauge=g, mass=0.1 + 0.001 * (k % 50), tol=1e-8, inner_prec=wd.F16, delta=0.1, b=b,
                     x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64))
            t = q.submit(p)
            live[t] = p
            order.append(t)
            if len(order) > 4:
                t = order.pop(0)
                r = q.poll(t) if k % 2 else None
                if r is None:
                    r = q.wait(t, timeout_ms=60000)
                statuses.append(r["status"])
                del live[t]
        for t in order:
            statuses.append(q.wait(t, timeout_ms=60000)["status"])
            del live[t]
        st = q.stats()
    finally:
        q.close()
    assert statuses == [0] * 240, statuses
    assert st["completed"] == 240, st
