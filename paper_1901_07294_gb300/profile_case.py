"""Runs one operator case a few times, for profiling (e.g. under ncu).

    python -m paper_1901_07294_gb300.profile_case --op eo --prec f32 --dims 32,32,32,32 --nrhs 12 \
        --launches 4 [--threads 128 --variant 3]
    python -m paper_1901_07294_gb300.profile_case --op cg --prec f16 --dims 24,24,24,48 --launches 1
    python -m paper_1901_07294_gb300.profile_case --op stream --kind 1 --n 16777216 --launches 3
    python -m paper_1901_07294_gb300.profile_case --op dd --nsub 4 --halo f16 --launches 3
    python -m paper_1901_07294_gb300.profile_case --op solve --prec f16 --dims 24,24,24,48 --launches 1

Inputs are the seeded synthetic gauge field and source of the benchmark.  With
--threads/--variant the launch shape is pinned; otherwise the library default
is used (no tuning, so few launches precede the profiled ones).  --op cg runs
`launches` mixed-precision CG solves (inner precision --prec, reliable updates,
delta 0.01, tol 1e-10, mass 0.1) on an even Gaussian source; --graph drives
them with CUDA graphs.  --op stream runs `launches` element-wise products of
kind --kind (wd_stream_mul) on --n elements of N(0,1) arrays.  --op dd applies
the operator `launches` times to the lattice split into --nsub slabs (field
precision --prec, halos --halo).  --op solve runs `launches` full-system solves
D x = b by BiCGStab (inner precision --prec, delta 0.01, tol 1e-10, mass 0.1).
"""
from __future__ import annotations

import argparse
import os
import sys


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["full", "eo", "cg", "stream", "dd", "solve"], default="full")
    ap.add_argument("--nsub", type=int, default=2)
    ap.add_argument("--halo", choices=["f64", "f32", "f16"], default="f32")
    ap.add_argument("--kind", type=int, default=1)
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--prec", choices=["f64", "f32", "f16", "bf16"], default="f32")
    ap.add_argument("--recon", type=int, default=18)
    ap.add_argument("--dims", default="32,32,32,32")
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--launches", type=int, default=4)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--variant", type=int, default=-1)
    ap.add_argument("--graph", action="store_true")
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np
    import torch

    import paper_1901_07294_gb300 as wd
    import synth

    prec = {"f64": wd.F64, "f32": wd.F32, "f16": wd.F16, "bf16": wd.BF16}[a.prec]
    dims = tuple(int(t) for t in a.dims.split(","))
    ctx = wd.Context(0)
    if a.op == "stream":
        gen = torch.Generator(device="cuda").manual_seed(6001)
        x, y, z = (torch.randn(2 * a.n, dtype=torch.float64, device="cuda", generator=gen) for _ in range(3))
        for _ in range(a.launches):
            wd.stream_mul(ctx, a.kind, a.n, x, y, z)
        torch.cuda.synchronize()
        print(f"profile_case: stream kind={a.kind} n={a.n} launches={a.launches} ok")
        return 0
    if a.op == "dd":
        hp = {"f64": wd.F64, "f32": wd.F32, "f16": wd.F16}[a.halo]
        dd = wd.DomainDecomposition(ctx, dims, a.nsub, synth.gauge(dims, seed=1001))
        ld = dd.local_dims()
        vloc = int(np.prod(ld))
        aos = torch.from_numpy(synth.spinor(dims, seed=2001).view(np.float64).reshape(-1).copy()).cuda()
        ins, outs = [], []
        for k in range(a.nsub):
            f = wd.alloc_field(ld, wd.SITES_FULL, prec)
            wd.pack(ctx, ld, wd.SITES_FULL, prec, aos[k * vloc * 24:(k + 1) * vloc * 24], f)
            ins.append(f)
            outs.append(wd.alloc_field(ld, wd.SITES_FULL, prec))
        for _ in range(a.launches):
            dd.dslash(outs, ins, 0.1, prec=prec, recon=a.recon, halo_prec=hp)
        torch.cuda.synchronize()
        print(f"profile_case: dd {a.prec} halo {a.halo} {a.dims} nsub={a.nsub} launches={a.launches} ok")
        return 0
    g = wd.Gauge(ctx, dims, synth.gauge(dims, seed=1001))
    if a.op == "solve":
        b = synth.spinor(dims, seed=3201)
        fb = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
        wd.pack(ctx, dims, wd.SITES_FULL, wd.F64, torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
        fx = wd.alloc_field(dims, wd.SITES_FULL, wd.F64)
        for _ in range(a.launches):
            st = wd.wilson_solve(ctx, g, 0.1, fx, fb, tol=1e-10, solver=wd.SOLVER_BICGSTAB, inner_prec=prec,
                                 inner_recon=a.recon, reliable=True, delta=0.01)
        torch.cuda.synchronize()
        print(f"profile_case: solve bicgstab {a.prec} {a.dims} solves={a.launches} iters={st['iters']} "
              f"updates={st['reliable_updates']} seconds={st['seconds']:.4f} ok")
        return 0
    if a.op == "cg":
        b = synth.even_spinor(dims, seed=3001)
        fb = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
        wd.pack(ctx, dims, wd.SITES_EVEN, wd.F64, torch.from_numpy(b.view(np.float64).reshape(-1).copy()).cuda(), fb)
        fx = wd.alloc_field(dims, wd.SITES_EVEN, wd.F64)
        for _ in range(a.launches):
            st = wd.cg_solve(ctx, g, 0.1, fx, fb, tol=1e-10, inner_prec=prec, inner_recon=a.recon, reliable=True,
                             delta=0.01, use_graph=a.graph)
        torch.cuda.synchronize()
        print(f"profile_case: cg {a.prec} r{a.recon} {a.dims} solves={a.launches} iters={st['iters']} "
              f"updates={st['reliable_updates']} seconds={st['seconds']:.4f} ok")
        return 0
    g.prepare(prec, a.recon)
    full = a.op == "full"
    if a.threads and a.variant >= 0:
        wd.tune_set_dslash(ctx, g, prec, a.recon, full, False, a.nrhs, a.threads, a.variant)
    aos = torch.from_numpy(synth.spinor(dims, seed=2001).view(np.float64).reshape(-1).copy()).cuda()
    one = wd.alloc_field(dims, wd.SITES_FULL, prec)
    wd.pack(ctx, dims, wd.SITES_FULL, prec, aos, one)
    if full:
        fin = one.repeat(a.nrhs)
        fout = wd.alloc_field(dims, wd.SITES_FULL, prec, a.nrhs)
    else:
        half = wd.field_bytes(dims, wd.SITES_ODD, prec)
        fin = one[half:].repeat(a.nrhs)
        fout = wd.alloc_field(dims, wd.SITES_EVEN, prec, a.nrhs)
    for _ in range(a.launches):
        if full:
            wd.dslash_apply(ctx, g, fout, fin, 0.1, nrhs=a.nrhs, prec=prec, recon=a.recon)
        else:
            wd.dslash_eo_apply(ctx, g, fout, fin, None, wd.EVEN, 0.0, 1.0, nrhs=a.nrhs, prec=prec, recon=a.recon)
    torch.cuda.synchronize()
    print(f"profile_case: {a.op} {a.prec} r{a.recon} {a.dims} nrhs={a.nrhs} launches={a.launches} ok")
    return 0


if __name__ == "__main__":
    sys.exit(main())
