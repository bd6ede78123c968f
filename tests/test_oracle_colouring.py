"""Pin the oracle's greedy colouring (the update order generalising the bipartite halves of
SI section 3 to non-bipartite graphs) by brute force on small graphs."""
import numpy as np
import pytest

import oracle
import sg_inputs


def brute_greedy(row_ptr, col):
    n = len(row_ptr) - 1
    colour = [-1] * n
    for i in range(n):
        used = {colour[j] for j in col[row_ptr[i]:row_ptr[i + 1]] if colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return np.array(colour, dtype=np.int32)


@pytest.mark.parametrize("n,c,seed", [(2, 1.0, 1), (50, 3.0, 2), (500, 4.0, 3), (2000, 8.0, 4)])
def test_greedy_colouring_matches_brute_force(n, c, seed):
    rp, col, _ = sg_inputs.poisson_graph(n, c, seed)
    colour, nc = oracle.greedy_colour(rp, col)
    want = brute_greedy(rp, col)
    assert np.array_equal(colour, want)
    assert nc == want.max() + 1
    # a proper colouring: no edge joins two vertices of the same colour
    src = np.repeat(np.arange(n), np.diff(rp))
    assert not np.any(colour[src] == colour[col])
    assert nc <= np.diff(rp).max() + 1


def test_bipartite_graph_gets_two_colours_on_even_cycle():
    n = 10
    ei = np.arange(n)
    ej = (ei + 1) % n
    rp, col, _ = sg_inputs.csr_from_edges(n, ei, ej)
    colour, nc = oracle.greedy_colour(rp, col)
    assert nc == 2 and np.array_equal(colour, np.arange(n) % 2)
