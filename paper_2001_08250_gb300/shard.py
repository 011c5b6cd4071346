"""Row-sharded PIR server over torch.distributed ranks: the scale-out that
Section 9.4 proposes (one server's database spread over several machines,
each holding a portion of it), one rank per GPU.

Each rank holds the rows ``talekpir.shard_plan`` gives it as a shard db
(``tpir_db_create_shard``).  A read runs the shard's partial reply on the
rank's GPU from the full-length request rows every rank receives; one
exchange then XOR-reduces the partials.  Collectives have no XOR reduction,
so the exchange is an all-gather of the partial replies (B x row_bytes per
rank) followed by the library's combine kernel (``tpir_xor_combine``).  The
reply is on every rank after the exchange.

Argument marshalling and the collective call only: the reads and the combine
run in the library's kernels.
"""

from __future__ import annotations

import torch
import torch.distributed as dist

from . import talekpir


def _device_combine(parts, out, stream=None) -> None:
    if not out.is_cuda:
        raise RuntimeError("the XOR exchange combines on the GPU; pass `combine` for CPU tensors")
    talekpir.xor_combine(parts, out.numel() * out.element_size(), out, stream)


def xor_exchange(partial: torch.Tensor, group=None, combine=None, out=None) -> torch.Tensor:
    """XOR of every rank's `partial` (same shape and dtype on all ranks), on
    every rank: all-gather, then `combine(parts, out)` (default: the library's
    combine kernel on the current stream)."""
    world = dist.get_world_size(group)
    parts = [torch.empty_like(partial) for _ in range(world)]
    dist.all_gather(parts, partial.contiguous(), group=group)
    if out is None:
        out = torch.empty_like(partial)
    if combine is None:
        _device_combine(parts, out, torch.cuda.current_stream().cuda_stream)
    else:
        combine(parts, out)
    return out


class ShardedServer:
    """This rank's row shard of an n_total-bucket table and its exchange."""

    def __init__(self, n_total: int, d: int, msg_bytes: int, group=None):
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.n_total, self.d, self.msg_bytes = int(n_total), int(d), int(msg_bytes)
        self.row_bytes = self.d * self.msg_bytes
        self.words64 = (self.n_total + 63) // 64
        self.row_begin, self.rows = talekpir.shard_plan(self.n_total, self.world)[self.rank]
        # a rank left without rows (more ranks than request words) adds zeros
        self.db = (talekpir.DB(self.rows, d, msg_bytes, shard=(self.n_total, self.row_begin))
                   if self.rows else None)

    def load(self, table_rows) -> None:
        """Load this shard's rows (uint8 [rows, row_bytes] host array, e.g. a
        snapshot of a writer's table sliced to [row_begin, row_begin + rows))."""
        if self.db is not None:
            self.db.load(table_rows)

    def read_partial_async(self, d_req, B: int, d_out, stream=None, d_seeds=None) -> None:
        """Partial replies of this shard into d_out (device, B x row_bytes)."""
        if self.db is None:
            d_out.zero_()
        elif d_seeds is not None:
            self.db.read_batch_masked_async(d_req, B, d_seeds, d_out, stream)
        else:
            self.db.read_batch_async(d_req, B, d_out, stream)

    def read(self, d_req, B: int, d_seeds=None, mask_rank: int = 0) -> torch.Tensor:
        """Full replies (device, B x row_bytes) on every rank: the partials of
        all shards XOR-reduced.  With d_seeds the replies are masked once, by
        the shard on rank `mask_rank`."""
        stream = torch.cuda.current_stream()
        partial = torch.empty((B, self.row_bytes), dtype=torch.uint8, device=d_req.device)
        self.read_partial_async(d_req, B, partial, stream.cuda_stream,
                                d_seeds if self.rank == mask_rank else None)
        if self.db is None and d_seeds is not None and self.rank == mask_rank:
            talekpir.mask_generate(d_seeds, B, self.row_bytes, partial, stream.cuda_stream)
        return xor_exchange(partial, self.group)

    def close(self) -> None:
        if self.db is not None:
            self.db.close()
            self.db = None
