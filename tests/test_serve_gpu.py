"""The request server (continuous batching): every request's result is the
same in the mix as alone, and equals the oracle's."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pico():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_15253_gb300 as p
    torch.cuda.set_device(0)
    return p


def make_requests(count, seed, nmax=40000):
    graphs = [gg.spec_graph(s) for s in gg.batch_specs(count - 2, seed, nmin=20, nmax=nmax)]
    graphs.insert(3, gg.from_edge_list([], 5))            # no edges
    graphs.append(gg.rmat_graph(16, 16, seed))            # one large outlier
    reqs = []
    for g in graphs:
        rp = g.row_ptr.to(torch.int32).pin_memory()
        ci = g.col_idx.pin_memory() if g.arcs else torch.zeros(1, dtype=torch.int32).pin_memory()
        out = torch.full((max(g.n, 1),), -1, dtype=torch.int32).pin_memory()
        reqs.append((g, rp, ci, out))
    return reqs


def serve(pico, reqs, algo, budget, streams=4, max_batch=64, single=0, spacing_ns=20000):
    srv = pico.pico_server_create(budget, algo, streams, max_batch, single)
    assert srv
    t0 = pico.pico_clock_ns()
    tickets = []
    for i, (g, rp, ci, out) in enumerate(reqs):
        t = pico.pico_server_submit(srv, rp, ci, g.n, g.arcs, out, t0 + i * spacing_ns)
        assert t >= 0
        tickets.append(t)
    assert pico.pico_server_drain(srv) == 0
    tk = torch.zeros(len(reqs), dtype=torch.int64)
    dn = torch.zeros(len(reqs), dtype=torch.int64)
    dv = torch.zeros(len(reqs), dtype=torch.int64)
    k = pico.pico_server_poll_device(srv, tk, dn, dv, len(reqs))
    assert k == len(reqs)
    assert sorted(tk.tolist()) == tickets
    assert (dn >= t0).all()
    # each request's device time (its micro-batch's copies and launch) is
    # positive and fits between its arrival and its completion (1 ms of
    # slack between the event clock and the host clock)
    arrival = t0 + tk * spacing_ns
    assert (dv > 0).all() and (dv <= dn - arrival + 1_000_000).all()
    assert pico.pico_server_destroy(srv) == 0
    return [out[:g.n].clone().numpy() for g, _, _, out in reqs]


@pytest.mark.parametrize("algo", [0, 1])
def test_results_same_alone_and_in_the_mix(pico, algo):
    reqs = make_requests(120, 91)
    mixed = serve(pico, reqs, algo, budget=8 << 30)
    for (g, rp, ci, out), got in zip(reqs, mixed):
        want = oracle.bz_coreness(g.row_ptr.numpy(), g.col_idx.numpy())
        assert np.array_equal(got, want)
    # the same requests, each alone (sequential plain path), give the same bytes
    alone = serve(pico, reqs, algo, budget=8 << 30, streams=1, max_batch=1, single=1,
                  spacing_ns=0)
    for a, b in zip(alone, mixed):
        assert np.array_equal(a, b)


def test_tight_budget_admits_as_memory_frees(pico):
    reqs = make_requests(40, 92, nmax=20000)
    sizes = [pico.pico_workspace_bytes_batched(1, g.n, g.arcs, 0) + 16 * (g.n + g.arcs + 64)
             for g, _, _, _ in reqs]
    budget = max(sizes) * 2        # only a few requests fit on the device at once
    got = serve(pico, reqs, 0, budget=budget, streams=3, max_batch=8, spacing_ns=0)
    for (g, _, _, _), x in zip(reqs, got):
        assert np.array_equal(x, oracle.bz_coreness(g.row_ptr.numpy(), g.col_idx.numpy()))


def test_request_larger_than_budget_is_rejected(pico):
    g = gg.rmat_graph(14, 16, 93)
    rp = g.row_ptr.pin_memory()
    ci = g.col_idx.pin_memory()
    out = torch.zeros(g.n, dtype=torch.int32).pin_memory()
    srv = pico.pico_server_create(1 << 20, 0, 2, 8, 0)
    assert pico.pico_server_submit(srv, rp, ci, g.n, g.arcs, out, 0) == pico.PICO_ERR_OOM
    assert pico.pico_server_destroy(srv) == 0


def test_served_workload_mix_with_scale20_outliers(pico):
    """The served workload's shape: request graphs from the batch size
    distribution (100..200,000 vertices, half ER, half R-MAT) with R-MAT scale
    20 outliers (about 16.6 M arcs each) among them, Poisson arrivals, a
    40 GB admission budget; every result must be the oracle's."""
    import math
    specs = gg.batch_specs(60, 94)
    graphs = [gg.spec_graph(s) for s in specs]
    for i, pos in enumerate((7, 23, 41)):
        graphs.insert(pos, gg.rmat_graph(20, 16, gg.SEED_BASE + 50 + i))
    reqs = []
    for g in graphs:
        rp = g.row_ptr.to(torch.int32).pin_memory()
        ci = g.col_idx.pin_memory() if g.arcs else torch.zeros(1, dtype=torch.int32).pin_memory()
        out = torch.full((max(g.n, 1),), -1, dtype=torch.int32).pin_memory()
        reqs.append((g, rp, ci, out))
    srv = pico.pico_server_create(40 << 30, 0, 4, 512, 0)
    assert srv
    t0 = pico.pico_clock_ns() + 1_000_000
    t = 0.0
    for i, (g, rp, ci, out) in enumerate(reqs):
        t += -math.log(1.0 - gg.unit_int(94, 7, i)) / 4000.0   # about 4,000 requests/s
        assert pico.pico_server_submit(srv, rp, ci, g.n, g.arcs, out, t0 + int(t * 1e9)) >= 0
    assert pico.pico_server_drain(srv) == 0
    assert pico.pico_server_destroy(srv) == 0
    for g, _, _, out in reqs:
        want = oracle.bz_coreness(g.row_ptr.numpy(), g.col_idx.numpy())
        assert np.array_equal(out[:g.n].numpy(), want)
