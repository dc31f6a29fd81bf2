"""The exchange protocol of partitioned HistoCore across ranks, on the CPU.

Two gloo ranks each hold one vertex range and run the product's driver
(paper_2402_15253_gb300.distributed.run), which all-gathers the change
records of every round. The per-rank work is a plain CPU stand-in written
here from Alg. 6 (SumHisto over the own V_cnt; UpdateHisto pulled into the
own rows), so the test checks the driver and the exchange, not the kernels:
the gathered coreness must equal the oracle's and the rounds those of the
oracle's sequential Alg. 6.
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

INT32_MAX = 2 ** 31 - 1


class CpuPartition:
    """Rows [lo, hi) of a CSR graph: estimates and histograms (slot s counts
    neighbours with estimate s below the own estimate, the own slot counts
    those at or above it)."""

    def __init__(self, rp, ci, lo, hi):
        self.rp, self.ci, self.lo, self.hi = rp, ci, lo, hi
        deg = np.diff(rp)
        self.est = [int(deg[v]) for v in range(lo, hi)]
        self.hist = []
        for v in range(lo, hi):
            h = [0] * (int(deg[v]) + 1)
            for w in ci[rp[v]:rp[v + 1]]:
                h[min(int(deg[w]), int(deg[v]))] += 1
            self.hist.append(h)
        self.vcnt = [i for i, v in enumerate(range(lo, hi))
                     if deg[v] >= 1 and self.hist[i][deg[v]] < deg[v]]

    def sum(self):
        recs = []
        for i in self.vcnt:
            K = self.est[i]
            s, k = 0, K
            while k >= 1:
                s += self.hist[i][k]
                if s >= k:
                    break
                k -= 1
            self.est[i] = k
            self.hist[i][k] = s
            recs += [self.lo + i, K, k]
        ymin = min(recs[2::3]) if recs else INT32_MAX
        return torch.tensor(recs, dtype=torch.int32), ymin

    def apply(self, records, ymin):
        r = records.view(-1, 3).tolist()
        changed = {v: (x, y) for v, x, y in r}
        nxt = []
        for i, v in enumerate(range(self.lo, self.hi)):
            K = self.est[i]
            if K <= ymin:
                continue
            fell = False
            for w in self.ci[self.rp[v]:self.rp[v + 1]]:
                c = changed.get(int(w))
                if c is None or K <= c[1]:
                    continue
                x, y = c
                self.hist[i][y] += 1
                self.hist[i][min(x, K)] -= 1
                fell |= x >= K
            if fell and self.hist[i][K] < K:
                nxt.append(i)
        self.vcnt = nxt
        return len(nxt)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _graphs():
    import graphgen as gg
    from conftest import load_g1
    n, edges, _ = load_g1()
    return [gg.from_edge_list(edges, n), gg.rmat_graph(9, 8, 81), gg.grid_graph(13, 17),
            gg.chung_lu_graph(600, 82, clique=12), gg.from_edge_list([(0, 1)], 5)]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2402_15253_gb300 import distributed as pd
    res = []
    for g in _graphs():
        rp, ci = g.numpy()
        lo, hi = pd.partition_bounds(g.n, world)[rank]
        part = CpuPartition(rp, ci, lo, hi)
        rounds = pd.run(part)
        est = torch.tensor(part.est, dtype=torch.int32)
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, torch.tensor([est.numel()], dtype=torch.int64))
        width = max(int(s) for s in sizes)
        padded = torch.zeros(max(width, 1), dtype=torch.int32)
        padded[:est.numel()] = est
        allp = [torch.zeros_like(padded) for _ in range(world)]
        dist.all_gather(allp, padded)
        core = torch.cat([p[:int(s)] for p, s in zip(allp, sizes)]).tolist()
        res.append((core, rounds))
    out[rank] = res
    dist.destroy_process_group()


def test_two_gloo_ranks_match_the_oracle():
    import oracle
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        assert out[0] == out[1]
        for g, (core, rounds) in zip(_graphs(), out[0]):
            rp, ci = g.numpy()
            assert core == oracle.bz_coreness(rp, ci).tolist()
            assert rounds == oracle.histocore(rp, ci)[1]["rounds"]


def test_partition_bounds_cover_every_vertex():
    from paper_2402_15253_gb300.distributed import partition_bounds
    for n, p in ((10, 3), (7, 7), (3, 5), (1000, 4), (0, 2)):
        b = partition_bounds(n, p)
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(b[i][1] == b[i + 1][0] for i in range(len(b) - 1))
