"""One slab per process: the host logic of ddrank.SlabOperator over two gloo ranks on CPU.

No GPU here, so the three kernel steps are stood in for by numpy on the host
(test code only): the interior pass is the oracle's D on the slab with the t
links of the last local slice set to zero (no hop crosses the slab boundary),
the faces are (1 - gamma_t) psi at local t = 0 (sent down) and
U_t^dagger (1 + gamma_t) psi at local t = T-1 (sent up), and the boundary pass
adds -1/2 U_t h at t = T-1 and -1/2 w at t = 0.  What is tested is what the
ranks do on the host: which face goes to which neighbour, the matching of the
two messages between the same pair of ranks, the sign on the faces that cross
the global antiperiodic boundary, and the reuse of the buffers over repeated
applications.  The slabs assembled must equal the oracle's global D.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

DIMS = (4, 4, 2, 8)
MASS = 0.2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class NumpySlabOps:
    """Host stand-ins for wd_slab_gather / wd_slab_interior / wd_slab_boundary (test only)."""

    def __init__(self, dims, nsub, k, U_slab, t_sign):
        import torch
        import oracle
        self.oracle = oracle
        self.ld = (dims[0], dims[1], dims[2], dims[3] // nsub)
        self.nf = dims[0] * dims[1] * dims[2]
        self.U = U_slab
        self.Uopen = U_slab.copy()
        self.Uopen[(self.ld[3] - 1) * self.nf:, 3] = 0.0
        self.g = oracle.gamma(3)
        self.neg_f = t_sign < 0 and k == 0
        self.neg_b = t_sign < 0 and k == nsub - 1
        n = self.nf * 12 * 2
        self.send_fwd, self.send_bwd, self.recv_fwd, self.recv_bwd = (
            torch.zeros(n, dtype=torch.float64) for _ in range(4))

    @staticmethod
    def _set(t, a):
        t.copy_(__import__("torch").from_numpy(np.ascontiguousarray(a).view(np.float64).reshape(-1)))

    @staticmethod
    def _get(t, nf):
        return t.numpy().view(np.complex128).reshape(nf, 4, 3)

    def gather(self, inp):
        psi, nf, T = inp, self.nf, self.ld[3]
        one = np.eye(4)
        h = np.einsum("ab,sbc->sac", one - self.g, psi[:nf])
        hb = np.einsum("ab,sbc->sac", one + self.g, psi[(T - 1) * nf:])
        w = np.einsum("sdc,sad->sac", self.U[(T - 1) * nf:, 3].conj(), hb)   # U^dagger acting on colour
        self._set(self.send_fwd, -h if self.neg_f else h)
        self._set(self.send_bwd, -w if self.neg_b else w)

    def exchange_scope(self):
        import contextlib
        return contextlib.nullcontext()

    def interior(self, out, inp, mass):
        out[:] = self.oracle.dirac(self.ld, self.Uopen, inp, mass)

    def join(self):
        pass

    def boundary(self, out):
        nf, T = self.nf, self.ld[3]
        h = self._get(self.recv_fwd, nf)
        w = self._get(self.recv_bwd, nf)
        out[(T - 1) * nf:] += -0.5 * np.einsum("scd,sad->sac", self.U[(T - 1) * nf:, 3], h)
        out[:nf] += -0.5 * w


def _rank_main(rank, world, port, t_sign, out):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import synth
    from paper_1901_07294_gb300 import ddrank
    U = synth.gauge(DIMS, seed=1801)
    psi = synth.spinor(DIMS, seed=3801)
    vloc = int(np.prod(DIMS)) // world
    ops = NumpySlabOps(DIMS, world, rank, U[rank * vloc:(rank + 1) * vloc], t_sign)
    op = ddrank.SlabOperator(ops, ddrank.DistTransport(), rank)
    res = np.zeros((vloc, 4, 3), dtype=np.complex128)
    for _ in range(2):   # buffers are reused
        op.apply(res, psi[rank * vloc:(rank + 1) * vloc], MASS)
    out[rank] = res.copy()
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,t_sign", [(2, 1), (2, -1), (4, 1)])
def test_slab_ranks_over_gloo_assemble_global_operator(world, t_sign):
    import oracle
    import synth
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, t_sign, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert p.exitcode == 0
        got = np.concatenate([out[r] for r in range(world)])
    U = synth.gauge(DIMS, seed=1801)
    psi = synth.spinor(DIMS, seed=3801)
    if t_sign < 0:
        U = oracle.antiperiodic_links(DIMS, U)
    ref = oracle.dirac(DIMS, U, psi, MASS)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    assert err < 1e-14, err
