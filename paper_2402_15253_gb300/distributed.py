"""Multi-rank driver of partitioned HistoCore.

Each rank holds one partition (a contiguous vertex range; on a GPU,
``paper_2402_15253_gb300.Partition``) and the ranks run Alg. 6 in lock-step
rounds (the synchronous model of Sec. IV-B): every rank runs SumHisto over its
own V_cnt, the ranks all-gather their change records (vertex, old, new) and
the smallest new estimate, and every rank pulls the UpdateHisto edits of all
records into its own rows. The computation ends in the first round in which
no rank has a record. The only communication is that exchange, through
``torch.distributed`` (NCCL for device tensors, gloo for host tensors).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def partition_bounds(n: int, parts: int) -> list[tuple[int, int]]:
    """Equal contiguous vertex ranges [lo, hi) of n vertices over `parts`."""
    return [(n * q // parts, n * (q + 1) // parts) for q in range(parts)]


def exchange(records: torch.Tensor, ymin: int, group=None) -> tuple[torch.Tensor, int]:
    """All-gathers every rank's records (int32, 3 per record, on the tensor's
    own device) in rank order and the smallest ymin; returns (all records,
    global ymin)."""
    dev = records.device
    world = dist.get_world_size(group)
    cnt = torch.tensor([records.numel()], dtype=torch.int64, device=dev)
    cnts = [torch.zeros_like(cnt) for _ in range(world)]
    dist.all_gather(cnts, cnt, group=group)
    sizes = [int(c.item()) for c in cnts]
    width = max(sizes) if sizes else 0
    if width == 0:
        gy = torch.tensor([ymin], dtype=torch.int64, device=dev)
        dist.all_reduce(gy, op=dist.ReduceOp.MIN, group=group)
        return torch.empty(0, dtype=torch.int32, device=dev), int(gy.item())
    padded = torch.zeros(width, dtype=torch.int32, device=dev)
    padded[:records.numel()] = records
    parts = [torch.zeros_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    gy = torch.tensor([ymin], dtype=torch.int64, device=dev)
    dist.all_reduce(gy, op=dist.ReduceOp.MIN, group=group)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)]), int(gy.item())


def run(partition, group=None, max_rounds: int | None = None) -> int:
    """Runs the rounds of partitioned HistoCore on this rank's `partition`
    (an object with sum() -> (records, ymin) and apply(records, ymin)); all
    ranks call it together. Returns the number of rounds."""
    rounds = 0
    while True:
        recs, ymin = partition.sum()
        all_recs, gymin = exchange(recs, ymin, group)
        if all_recs.numel() == 0:
            return rounds
        partition.apply(all_recs, gymin)
        rounds += 1
        if max_rounds is not None and rounds > max_rounds:
            raise RuntimeError("partitioned HistoCore did not converge")
