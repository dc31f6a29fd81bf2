"""The parallel CPU comparison of the benchmark (cpu_peel) against the
oracle: random graphs of each family and closed forms."""
import numpy as np
import pytest

import cpu_peel
import graphgen as gg
import oracle


@pytest.mark.parametrize("make", [lambda: gg.rmat_graph(14, 16, 81),
                                  lambda: gg.er_graph(20000, 120000, 82),
                                  lambda: gg.chung_lu_graph(1 << 14, 83, clique=120),
                                  lambda: gg.grid_graph(60, 70),
                                  lambda: gg.complete_graph(40),
                                  lambda: gg.path_graph(1000),
                                  lambda: gg.star_graph(500)])
def test_matches_the_oracle(make):
    g = make()
    rp, ci = g.numpy()
    assert np.array_equal(cpu_peel.coreness(rp, ci), oracle.bz_coreness(rp, ci))


def test_isolated_and_empty():
    g = gg.from_edge_list([(0, 1)], 5)
    rp, ci = g.numpy()
    assert cpu_peel.coreness(rp, ci).tolist() == [1, 1, 0, 0, 0]
    assert cpu_peel.threads() >= 1
