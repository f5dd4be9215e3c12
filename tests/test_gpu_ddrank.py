"""One slab per process (wd_slab + ddrank.SlabOperator), through the C ABI on the GPU.

Several slabs run in this process with the in-process transport, which copies
each send buffer into the neighbour's receive buffer: the same gather,
interior and boundary kernels and the same ordering of streams as one rank per
GPU with NCCL, whose send/recv would deliver the same bytes.  The assembled
result is the global operator D by definition (oracle), and it equals the
single-process decomposition (wd_dd) bit for bit, which runs the same kernels.
"""
import numpy as np
import pytest

import oracle
import paper_1901_07294_gb300 as wd
import synth
from paper_1901_07294_gb300 import ddrank
from tests._gpu import TOL, check_dslash, pack_field, unpack_field
from tests._lattice import volume

pytestmark = pytest.mark.gpu

DIMS = (4, 6, 4, 8)
MASS = 0.1


@pytest.fixture(scope="module")
def ctx():
    return wd.Context(0)


def _ranks(ctx, dims, U, psi, nsub, prec, recon, halo_prec, t_sign=1, applies=1):
    import torch
    lt = dims[3] // nsub
    ld = (dims[0], dims[1], dims[2], lt)
    vloc = volume(ld)
    tr = ddrank.LocalTransport(nsub)
    ops, slabs = [], []
    for k in range(nsub):
        sl = wd.Slab(ctx, dims, nsub, k, U[k * vloc:(k + 1) * vloc])
        assert sl.local_dims() == ld
        if t_sign != 1:
            sl.set_boundary(t_sign)
        slabs.append(sl)
        ops.append(ddrank.SlabOperator(ddrank.CudaSlabOps(sl, prec, recon, halo_prec), tr, k))
    ins = [pack_field(ctx, ld, wd.SITES_FULL, prec, psi[k * vloc:(k + 1) * vloc]) for k in range(nsub)]
    outs = [wd.alloc_field(ld, wd.SITES_FULL, prec) for _ in range(nsub)]
    for _ in range(applies):
        for k in range(nsub):
            ops[k].post(ins[k])
        for k in range(nsub):
            ops[k].complete(outs[k], ins[k], MASS)
    torch.cuda.synchronize()
    got = np.concatenate([unpack_field(ctx, ld, wd.SITES_FULL, prec, o) for o in outs])
    raw = [o.clone() for o in outs]
    for sl in slabs:
        sl.close()
    return got, raw


@pytest.mark.parametrize("nsub", [1, 2, 4])
@pytest.mark.parametrize("prec", [wd.F64, wd.F32, wd.F16])
@pytest.mark.parametrize("recon", [18, 12])
def test_slab_ranks_match_global_operator(ctx, nsub, prec, recon):
    U = synth.gauge(DIMS, seed=1701)
    psi = synth.spinor(DIMS, seed=3701)
    hp = wd.F64 if prec == wd.F64 else wd.F32
    got, _ = _ranks(ctx, DIMS, U, psi, nsub, prec, recon, hp)
    check_dslash(got, oracle.dirac(DIMS, U, psi, MASS), prec, DIMS, U, psi, recon,
                 lambda u, p: oracle.dirac(DIMS, u, p, MASS), out_roundings=2)


@pytest.mark.parametrize("prec,halo_prec", [(wd.F32, wd.F16), (wd.F64, wd.F64), (wd.F16, wd.F16)])
def test_slab_ranks_equal_single_process_decomposition(ctx, prec, halo_prec):
    """Same kernels, same order per slab: the bytes of every slab's output agree with wd_dd,
    also after repeated applications (buffers reused)."""
    import torch
    U = synth.gauge(DIMS, seed=1702)
    psi = synth.spinor(DIMS, seed=3702)
    nsub = 2
    _, raw = _ranks(ctx, DIMS, U, psi, nsub, prec, 18, halo_prec, applies=3)
    dd = wd.DomainDecomposition(ctx, DIMS, nsub, U)
    ld = dd.local_dims()
    vloc = volume(ld)
    ins = [pack_field(ctx, ld, wd.SITES_FULL, prec, psi[k * vloc:(k + 1) * vloc]) for k in range(nsub)]
    outs = [wd.alloc_field(ld, wd.SITES_FULL, prec) for _ in range(nsub)]
    dd.dslash(outs, ins, MASS, prec=prec, recon=18, halo_prec=halo_prec)
    torch.cuda.synchronize()
    dd.close()
    for k in range(nsub):
        assert torch.equal(raw[k], outs[k]), k


def test_slab_ranks_antiperiodic(ctx):
    U = synth.gauge(DIMS, seed=1703)
    psi = synth.spinor(DIMS, seed=3703)
    got, _ = _ranks(ctx, DIMS, U, psi, 4, wd.F64, 18, wd.F64, t_sign=-1)
    ref = oracle.dirac(DIMS, oracle.antiperiodic_links(DIMS, U), psi, MASS)
    err = float(np.max(np.abs((got - ref).view(np.float64))) / np.max(np.abs(ref.view(np.float64))))
    assert err < TOL[wd.F64], err


def test_slab_rejects_bad_arguments(ctx):
    U = synth.gauge(DIMS, seed=1704)
    with pytest.raises(wd.WdError):
        wd.Slab(ctx, DIMS, 3, 0, U)          # 3 does not divide L_t = 8
    with pytest.raises(wd.WdError):
        wd.Slab(ctx, DIMS, 2, 2, U)          # slab index out of range
    with pytest.raises(wd.WdError):
        wd.Slab(ctx, DIMS, 8, 0, U)          # local L_t = 1
