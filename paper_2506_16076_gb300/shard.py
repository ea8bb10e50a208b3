"""Transports for sharded execution (fc_shard): how ranks exchange what the library packs.

A sharded context calls its transport once per projection (interpolated fringe values),
once per viscosity evaluation (window sums of the cross-patch blending) and once per time
step (the minimum of eq. CFL), always in the same order on every rank: the communication
step of Algorithm 1. Two transports:

  DistComm   torch.distributed: an all-to-all with the library's splits and an all-reduce
             (MIN); NCCL for device tensors, one process per GPU.
  LocalComm  ranks that share one process and one device, one host thread per rank
             (in-process emulation of a multi-GPU run; the waiting is on the host, never in
             a kernel).

Marshalling only: the packing, the interpolation and every other step run in the library.
"""
import threading

import torch

from . import fcsdnn

partition = fcsdnn.partition


class DistComm:
    """The exchanges as torch.distributed collectives of the default (or given) group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group

    def exchange(self, send, send_counts, recv, recv_counts):
        self.dist.all_to_all_single(recv, send, list(recv_counts), list(send_counts), group=self.group)

    def allmin(self, send, recv):
        t = send.clone()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        recv.copy_(t)


class LocalHub:
    """Meeting point of the LocalComm ranks of one process."""

    def __init__(self, nranks, timeout=120.0):
        self.n = nranks
        self.barrier = threading.Barrier(nranks, timeout=timeout)
        self.slots = [None] * nranks


class LocalComm:
    """Rank `rank` of an in-process group: each exchange publishes this rank's send buffer,
    waits for the others, copies the blocks owed to it on the current stream, and waits
    again so that no send buffer is reused before every rank has read it."""

    def __init__(self, hub, rank):
        self.hub, self.rank = hub, rank

    def exchange(self, send, send_counts, recv, recv_counts):
        h, r = self.hub, self.rank
        torch.cuda.current_stream().synchronize()  # the packed values are complete
        h.slots[r] = (send, list(send_counts))
        h.barrier.wait()
        off = 0
        for q in range(h.n):
            if recv_counts[q]:
                s_q, c_q = h.slots[q]
                start = sum(c_q[:r])
                if c_q[r] != recv_counts[q]:
                    raise RuntimeError(f"rank {q} sends {c_q[r]} values to rank {r}, which expects {recv_counts[q]}")
                recv[off:off + recv_counts[q]].copy_(s_q[start:start + c_q[r]])
            off += recv_counts[q]
        torch.cuda.current_stream().synchronize()
        h.barrier.wait()

    def allmin(self, send, recv):
        h, r = self.hub, self.rank
        torch.cuda.current_stream().synchronize()
        h.slots[r] = send.clone()
        h.barrier.wait()
        m = h.slots[0]
        for q in range(1, h.n):
            m = torch.minimum(m, h.slots[q])
        recv.copy_(m)
        torch.cuda.current_stream().synchronize()
        h.barrier.wait()
