"""Batched solves of uneven volumes: sequential, CUDA-graph and persistent-kernel modes.

Each solve is judged by its true residual computed with the oracle operator on
the GPU solution, and every solve's result in the mix must equal, bit for bit,
the same solve run alone: a solve's kernels and reductions do not depend on
the other solves of the batch (the persistent kernel's reductions use fixed
256-site chunks, whatever group of blocks a solve gets).
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field, unpack_field
from tests._lattice import rel_max_err, volume

pytestmark = pytest.mark.gpu

LATTICES = [(4, 4, 4, 4), (8, 8, 8, 8), (4, 6, 8, 10)]


def _problems(ctx, n, seed=4001, tol=1e-10):
    rng = np.random.default_rng(seed)
    probs, host = [], []
    gauges = {}
    for k in range(n):
        dims = LATTICES[k % len(LATTICES)]
        if dims not in gauges:
            U = synth.gauge(dims, seed=1000 + volume(dims) % 977)
            gauges[dims] = (U, wd.Gauge(ctx, dims, U))
        U, g = gauges[dims]
        mass = float(rng.uniform(0.05, 0.5))
        b = synth.even_spinor(dims, seed=3100 + k)
        probs.append(dict(gauge=g, mass=mass, tol=tol, b=pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, b),
                          x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64), inner_prec=wd.F32, delta=0.1))
        host.append((dims, U, mass, b))
    return probs, host


def _true_rel(ctx, host, x_field):
    dims, U, mass, b = host
    x = unpack_field(ctx, dims, wd.SITES_EVEN, wd.F64, x_field)
    r = b - oracle.mdagm(dims, U, mass, x)
    return float(np.linalg.norm(r) / np.linalg.norm(b)), x


@pytest.mark.parametrize("mode", [wd.BATCH_SEQUENTIAL, wd.BATCH_GRAPH, wd.BATCH_PERSISTENT])
def test_batch_converges_and_matches_alone(mode):
    ctx = wd.Context(0)
    probs, host = _problems(ctx, 7)
    stats = wd.cg_solve_batch(ctx, probs, mode=mode)
    xs_mix = []
    for k, st in enumerate(stats):
        assert st["status"] == 0, (k, st)
        assert st["true_rel_resid"] <= 1e-10, (k, st)
        rel, x = _true_rel(ctx, host[k], probs[k]["x"])
        assert rel <= 1e-10, (k, rel)
        xs_mix.append(x)
    # every solve alone (a batch of one) gives the same bits
    for k in range(len(probs)):
        one = [dict(probs[k])]
        one[0]["x"] = wd.alloc_field(host[k][0], wd.SITES_EVEN, wd.F64)
        st = wd.cg_solve_batch(ctx, one, mode=mode)[0]
        assert st["status"] == 0
        assert st["iters"] == stats[k]["iters"], (k, st, stats[k])
        _, x_alone = _true_rel(ctx, host[k], one[0]["x"])
        assert np.array_equal(xs_mix[k], x_alone), (k, rel_max_err(xs_mix[k], x_alone))


@pytest.mark.parametrize("mode,prec", [(wd.BATCH_GRAPH, wd.F16), (wd.BATCH_PERSISTENT, wd.F16),
                                       (wd.BATCH_PERSISTENT, wd.BF16)])
def test_batch_16bit_inner(mode, prec):
    """FP16 / BF16 storage of the iterated residual, direction and operator intermediates
    (FP32 arithmetic, FP32 solution increment, FP64 reliable updates)."""
    ctx = wd.Context(0)
    probs, host = _problems(ctx, 4, seed=4002)
    for p in probs:
        p["inner_prec"] = prec
    stats = wd.cg_solve_batch(ctx, probs, mode=mode)
    for k, st in enumerate(stats):
        assert st["status"] == 0 and st["true_rel_resid"] <= 1e-10
        assert _true_rel(ctx, host[k], probs[k]["x"])[0] <= 1e-10


def test_persistent_rejects_unsupported_options():
    ctx = wd.Context(0)
    probs, _ = _problems(ctx, 1)
    probs[0]["inner_prec"] = wd.F64
    with pytest.raises(wd.WdError) as e:
        wd.cg_solve_batch(ctx, probs, mode=wd.BATCH_PERSISTENT)
    assert e.value.status == wd.WD_EINVAL
    # one launch runs one inner precision
    probs, _ = _problems(ctx, 2)
    probs[1]["inner_prec"] = wd.F16
    with pytest.raises(wd.WdError) as e:
        wd.cg_solve_batch(ctx, probs, mode=wd.BATCH_PERSISTENT)
    assert e.value.status == wd.WD_EINVAL


def test_persistent_barrier_timeout_reports_etimeout(monkeypatch):
    """A group barrier whose last participant never arrives (injected on the host: each group
    waits for one block more than it has) gives up after its bounded wait, the kernel returns,
    the call reports WD_ETIMEOUT and the context keeps working."""
    ctx = wd.Context(0)
    probs, host = _problems(ctx, 2, seed=4003)
    monkeypatch.setenv("WD_FAULT", "barrier_missing")
    monkeypatch.setenv("WD_BARRIER_TIMEOUT_S", "0.2")
    stats = wd.cg_solve_batch(ctx, probs, mode=wd.BATCH_PERSISTENT, check=False)
    assert stats[0]["batch_status"] == wd.WD_ETIMEOUT
    assert all(s["status"] == wd.WD_ETIMEOUT for s in stats)
    monkeypatch.delenv("WD_FAULT")
    stats = wd.cg_solve_batch(ctx, probs, mode=wd.BATCH_PERSISTENT)
    assert all(s["status"] == 0 for s in stats)
    assert _true_rel(ctx, host[0], probs[0]["x"])[0] <= 1e-10
