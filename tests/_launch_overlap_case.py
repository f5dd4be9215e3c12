"""A fixed sequence of operator, BLAS and solver calls whose results (raw device bytes) are
saved to an .npz file.  tests/test_gpu_launch_overlap.py runs it once with programmatic
dependent launch (the default) and once with WD_PDL=0 and requires identical bytes.

Usage: python -m tests._launch_overlap_case <out.npz>
"""
import sys

import numpy as np
import torch

import paper_1901_07294_gb300 as wd
import synth
from tests._gpu import pack_field

L16 = (16, 16, 16, 16)
L8 = (8, 8, 8, 8)


def _bytes(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().copy()


def main(path):
    ctx = wd.Context(0)
    out = {}
    U = synth.gauge(L16, seed=1040)
    g = wd.Gauge(ctx, L16, U)
    psi = synth.spinor(L16, seed=4040)

    # chains of operator applications, each reading the output of the one before
    for prec in (wd.F64, wd.F32, wd.F16, wd.BF16, wd.DF):
        a = pack_field(ctx, L16, wd.SITES_FULL, prec, psi)
        b = wd.alloc_field(L16, wd.SITES_FULL, prec)
        for _ in range(6):
            wd.dslash_apply(ctx, g, b, a, 0.1, prec=prec)
            a, b = b, a
        out[f"dslash_chain_p{prec}"] = _bytes(a)
        e = pack_field(ctx, L16, wd.SITES_EVEN, prec, psi)
        e2 = wd.alloc_field(L16, wd.SITES_EVEN, prec)
        o = wd.alloc_field(L16, wd.SITES_ODD, prec)
        for _ in range(3):
            wd.dslash_eo_apply(ctx, g, o, e, None, 1, 0.0, 0.25, prec=prec)
            wd.dslash_eo_apply(ctx, g, e2, o, e, 0, 1.5, -0.25, dagger=True, prec=prec)
            e, e2 = e2, e
        out[f"eo_chain_p{prec}"] = _bytes(e)

    # BLAS chain: each reduction reads the field the update before it wrote
    x = pack_field(ctx, L16, wd.SITES_FULL, wd.F32, psi)
    y = pack_field(ctx, L16, wd.SITES_FULL, wd.F32, synth.spinor(L16, seed=4041))
    r = torch.zeros(16, dtype=torch.float64, device="cuda")
    for k in range(4):
        wd.axpby(ctx, L16, wd.SITES_FULL, wd.F32, 0.5 + k, x, -0.25, y)
        wd.norm2(ctx, L16, wd.SITES_FULL, wd.F32, y, r[4 * k:4 * k + 1])
        wd.dot(ctx, L16, wd.SITES_FULL, wd.F32, x, y, r[4 * k + 2:4 * k + 4])
    out["blas_chain_y"] = _bytes(y)
    out["blas_chain_r"] = _bytes(r)

    # solvers: host-driven and graph-driven mixed CG, FP64 CG, BiCGStab
    b8 = synth.even_spinor(L8, seed=4050)
    g8 = wd.Gauge(ctx, L8, synth.gauge(L8, seed=1041))
    fb = pack_field(ctx, L8, wd.SITES_EVEN, wd.F64, b8)
    runs = [("cg_f64", dict(inner_prec=wd.F64)),
            ("cg_f16", dict(inner_prec=wd.F16)),
            ("cg_f16_df", dict(inner_prec=wd.F16, outer_prec=wd.DF)),
            ("cg_f16_graph", dict(inner_prec=wd.F16, use_graph=True)),
            ("cg_f16_graph_df", dict(inner_prec=wd.F16, use_graph=True, outer_prec=wd.DF))]
    for name, kw in runs:
        fx = wd.alloc_field(L8, wd.SITES_EVEN, wd.F64)
        st = wd.cg_solve(ctx, g8, 0.1, fx, fb, tol=1e-10, **kw)
        out[name] = _bytes(fx)
        out[name + "_iters"] = np.array([st["iters"]])
    fx = wd.alloc_field(L8, wd.SITES_EVEN, wd.F64)
    wd.bicgstab_solve(ctx, g8, 0.1, fx, fb, tol=1e-10, inner_prec=wd.F16)
    out["bicgstab_f16"] = _bytes(fx)

    # a graph-mode batch (request groups on two gauges)
    probs = []
    for k in range(4):
        dims, gg = (L8, g8) if k % 2 else (L16, g)
        bk = pack_field(ctx, dims, wd.SITES_EVEN, wd.F64, synth.even_spinor(dims, seed=4060 + k))
        probs.append(dict(gauge=gg, mass=0.1 + 0.05 * k, tol=1e-10, b=bk, x=wd.alloc_field(dims, wd.SITES_EVEN, wd.F64),
                          inner_prec=wd.F16, outer_prec=wd.DF if k < 2 else wd.F64))
    wd.cg_solve_batch(ctx, probs, mode=wd.BATCH_GRAPH)
    for k, p in enumerate(probs):
        out[f"batch_graph_{k}"] = _bytes(p["x"])

    # the serving queue
    q = wd.Queue(ctx, 4 << 30, 4)
    tickets = []
    for k in range(3):
        bk = pack_field(ctx, L8, wd.SITES_EVEN, wd.F64, synth.even_spinor(L8, seed=4070 + k))
        p = dict(gauge=g8, mass=0.12 + 0.03 * k, tol=1e-10, b=bk, x=wd.alloc_field(L8, wd.SITES_EVEN, wd.F64),
                 inner_prec=wd.F16)
        tickets.append((q.submit(p), p))
    for k, (t, p) in enumerate(tickets):
        assert q.wait(t, timeout_ms=60000)["status"] == 0
        out[f"queue_{k}"] = _bytes(p["x"])
    q.close()

    # the operator over two slabs with a halo exchange
    dd = wd.DomainDecomposition(ctx, L16, 2, U)
    ld = dd.local_dims()
    full = psi.reshape(L16[3], -1, 4, 3)
    ins, outs = [], []
    for k in range(2):
        part = full[k * ld[3]:(k + 1) * ld[3]].reshape(-1, 4, 3)
        ins.append(pack_field(ctx, ld, wd.SITES_FULL, wd.F32, part))
        outs.append(wd.alloc_field(ld, wd.SITES_FULL, wd.F32))
    dd.dslash(outs, ins, 0.1, prec=wd.F32, halo_prec=wd.F16)
    for k in range(2):
        out[f"dd_{k}"] = _bytes(outs[k])
    dd.close()

    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
