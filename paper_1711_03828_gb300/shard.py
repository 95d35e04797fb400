"""Chain sharding over ranks: the one exchange of an SCMF cycle.

The paper distributes whole molecules over the ranks (Sec. 3.1.1): every rank
moves its own molecules against the same quasi-instantaneous fields, and the
only communication of a cycle is the sum over ranks of the occupation numbers
n_t(c), after which every rank computes the fields itself.  Here each rank
holds one shard (a ``System`` whose description carries ``chain_offset`` and
``n_chains_total``, see ``soma_shard_sweep`` in ``include/soma.h``), and this
module drives it:

    shard.shard_sweep(buf)      # MC step of the rank's chains, their counts -> buf
    allreduce(buf)              # sum over ranks, in place (NCCL or gloo)
    shard.shard_fields(buf)     # fields from the summed counts

``buf`` is one int32 tensor of grid cells on the device the exchange runs on;
the packed A | B<<16 counts add exactly as 32-bit integers (two's complement
wrap-around is the unsigned sum) while every global count stays below 2^16.
The driver only marshals calls: the counts, the sweep and the fields are the
library's kernels.  Any object with the three ``shard_*`` calls can be driven,
which is how the exchange is tested on CPU ranks.
"""
from __future__ import annotations

import dataclasses


def shard_range(n_chains_total: int, world: int, rank: int):
    """(chain_offset, n_chains) of rank's contiguous share of the chains;
    the first n_chains_total % world ranks take one chain more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    q, r = divmod(int(n_chains_total), int(world))
    return rank * q + min(rank, r), q + (1 if rank < r else 0)


def shard_desc(desc, world: int, rank: int):
    """The description of rank's shard of the whole system ``desc``."""
    if desc.n_chains_total:
        raise ValueError("desc already describes a shard")
    off, cnt = shard_range(desc.n_chains, world, rank)
    if cnt < 1:
        raise ValueError(f"{desc.n_chains} chains cannot be shared by {world} ranks")
    return dataclasses.replace(desc, n_chains=cnt, chain_offset=off, n_chains_total=desc.n_chains)


class ShardedRun:
    """One rank's side of the sharded SCMF cycle.

    system: the rank's shard (``System`` or any object with ``shard_counts``,
    ``shard_sweep`` and ``shard_fields`` taking the count buffer); cells: grid
    cells; device: where the count buffer lives (the device of the exchange);
    allreduce: sums the buffer over the ranks in place (default:
    ``torch.distributed.all_reduce`` on the default group).  When the system
    runs on a CUDA stream of its own (``stream_handle()``), torch's current
    stream waits for it before the collective and it waits for torch's stream
    after, so the exchange is ordered after the count copy and before the
    field update whichever stream the caller uses.
    """

    def __init__(self, system, cells: int, device="cpu", allreduce=None):
        import torch
        self.system = system
        self.buf = torch.zeros(int(cells), dtype=torch.int32, device=device)
        if allreduce is None:
            import torch.distributed as dist

            def allreduce(t):
                dist.all_reduce(t, op=dist.ReduceOp.SUM)
        self.allreduce = allreduce
        self.cycles = 0
        self._ext = None
        handle = getattr(system, "stream_handle", None)
        if self.buf.is_cuda and handle is not None and handle():
            self._ext = torch.cuda.ExternalStream(int(handle()), device=self.buf.device)

    def _exchange(self):
        if self._ext is None:
            self.allreduce(self.buf)
            return
        import torch
        cur = torch.cuda.current_stream(self.buf.device)
        cur.wait_stream(self._ext)
        self.allreduce(self.buf)
        self._ext.wait_stream(cur)

    def start(self):
        """Fields of the whole system from the shards' current positions."""
        self.system.shard_counts(self.buf)
        self._exchange()
        self.system.shard_fields(self.buf)

    def cycle(self, n: int = 1):
        """n SCMF cycles, each with its one exchange of counts."""
        for _ in range(int(n)):
            self.system.shard_sweep(self.buf)
            self._exchange()
            self.system.shard_fields(self.buf)
            self.cycles += 1
