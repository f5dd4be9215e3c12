"""One slab per process: the host logic of a decomposed operator application.

Sec. II-A parallelises the hopping term by giving each process one
sub-lattice, which exchanges its boundary with its neighbours; Sec. V keeps
16-bit floats for compressing that exchanged data.  Here the lattice is split
along t into one slab per rank.  One application of D on a rank:

    side stream: gather the two faces of the input into send buffers
                 (wd_slab_gather), then hand them to the transport, which
                 delivers send_fwd to rank k-1 and send_bwd to rank k+1 and
                 receives recv_fwd from k+1 and recv_bwd from k-1 into this
                 rank's own buffers (NCCL send/recv: no peer loads);
    caller's stream, meanwhile: the interior pass (wd_slab_interior);
    caller's stream, after both: the boundary pass (wd_slab_boundary).

The steps run on the GPU in the library's kernels; this module only orders
them and moves the face buffers.  `SlabOperator` takes the three steps from
an `ops` object (`CudaSlabOps` for the library) and the exchange from a
transport: `DistTransport` (torch.distributed point-to-point: NCCL between
GPUs, gloo between CPU processes) or `LocalTransport` (every slab in this
process, the exchange a copy into each neighbour's buffer).
"""
from __future__ import annotations

TAG_FWD, TAG_BWD = 11, 12   # message tags (used by transports that match on them)


class SlabOperator:
    """D applied to this process's slab, with the faces exchanged through `transport`.

    `ops` provides: send_fwd, send_bwd, recv_fwd, recv_bwd (face buffers), gather(inp),
    exchange_scope() (a context in which the exchange is issued), interior(out, inp, mass),
    join() (the caller waits for the gather and exchange) and boundary(out)."""

    def __init__(self, ops, transport, index: int):
        self.ops = ops
        self.transport = transport
        self.index = int(index)
        self._pending = None
        transport.register(self)

    def post(self, inp) -> None:
        """Gathers this slab's faces and starts sending them (non-blocking)."""
        self.ops.gather(inp)
        with self.ops.exchange_scope():
            self._pending = self.transport.start(self)

    def complete(self, out, inp, mass: float) -> None:
        """Interior pass while the faces travel, then the received halos."""
        self.ops.interior(out, inp, mass)
        with self.ops.exchange_scope():
            self.transport.finish(self, self._pending)
        self._pending = None
        self.ops.join()
        self.ops.boundary(out)

    def apply(self, out, inp, mass: float) -> None:
        self.post(inp)
        self.complete(out, inp, mass)


class DistTransport:
    """Faces between processes with torch.distributed point-to-point operations, rank r of
    the group holding slab r.  On NCCL they run on the current CUDA stream (the ops' side
    stream) and write into the receivers' own device buffers."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def register(self, op) -> None:
        if op.index != self.rank:
            raise ValueError(f"slab {op.index} on rank {self.rank}: one slab per rank, slab index = rank")

    def _peer(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    def start(self, op):
        o = op.ops
        if self.size == 1:   # a single slab is its own neighbour
            return None
        lower, upper = self._peer((self.rank - 1) % self.size), self._peer((self.rank + 1) % self.size)
        d = self.dist
        ops = [d.P2POp(d.isend, o.send_fwd, lower, self.group, TAG_FWD),
               d.P2POp(d.irecv, o.recv_fwd, upper, self.group, TAG_FWD),
               d.P2POp(d.isend, o.send_bwd, upper, self.group, TAG_BWD),
               d.P2POp(d.irecv, o.recv_bwd, lower, self.group, TAG_BWD)]
        return d.batch_isend_irecv(ops)

    def finish(self, op, pending) -> None:
        if pending is None:
            op.ops.recv_fwd.copy_(op.ops.send_fwd)
            op.ops.recv_bwd.copy_(op.ops.send_bwd)
            return
        for w in pending:
            w.wait()


class LocalTransport:
    """Every slab in this process: receiving is a copy from the neighbour's send buffer.
    Post all slabs before completing any."""

    def __init__(self, nsub: int):
        self.ops = [None] * int(nsub)

    def register(self, op) -> None:
        self.ops[op.index] = op

    def start(self, op):
        return None

    def finish(self, op, pending) -> None:
        n = len(self.ops)
        up, lo = self.ops[(op.index + 1) % n].ops, self.ops[(op.index - 1) % n].ops
        up.join_into(op.ops)
        lo.join_into(op.ops)
        op.ops.recv_fwd.copy_(up.send_fwd)
        op.ops.recv_bwd.copy_(lo.send_bwd)


class CudaSlabOps:
    """The library's kernels for one `Slab`: face buffers in device memory (uint8 tensors of
    wd_slab_face_bytes each), the gather and the exchange on a side stream."""

    def __init__(self, slab, prec: int, recon: int, halo_prec: int):
        import torch
        self.slab, self.prec, self.recon, self.halo_prec = slab, int(prec), int(recon), int(halo_prec)
        nb = slab.face_bytes(self.halo_prec)
        self.send_fwd, self.send_bwd, self.recv_fwd, self.recv_bwd = (
            torch.empty(nb, dtype=torch.uint8, device="cuda") for _ in range(4))
        self.side = torch.cuda.Stream()

    def gather(self, inp) -> None:
        import torch
        self.side.wait_stream(torch.cuda.current_stream())
        self.slab.gather(inp, self.send_fwd, self.send_bwd, self.prec, self.recon, self.halo_prec, stream=self.side)

    def exchange_scope(self):
        import torch
        return torch.cuda.stream(self.side)

    def join_into(self, other) -> None:
        """`other`'s side stream waits for this slab's gather (in-process exchange)."""
        other.side.wait_stream(self.side)

    def interior(self, out, inp, mass: float) -> None:
        self.slab.interior(out, inp, mass, self.prec, self.recon)

    def join(self) -> None:
        import torch
        torch.cuda.current_stream().wait_stream(self.side)

    def boundary(self, out) -> None:
        self.slab.boundary(out, self.recv_fwd, self.recv_bwd, self.prec, self.recon, self.halo_prec)
