"""Pin the oracle's colouring (the update order generalising the bipartite halves of SI
section 3 to non-bipartite graphs): greedy in vertex order, then one recolouring pass, each by
brute force on small graphs, with the properties that hold for any graph."""
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


def brute_recolour(row_ptr, col, colour):
    n = len(row_ptr) - 1
    fresh = [-1] * n
    for i in sorted(range(n), key=lambda i: (-int(colour[i]), i)):
        used = {fresh[j] for j in col[row_ptr[i]:row_ptr[i + 1]] if fresh[j] >= 0}
        c = 0
        while c in used:
            c += 1
        fresh[i] = c
    return np.array(fresh, dtype=np.int32)


@pytest.mark.parametrize("n,c,seed", [(2, 1.0, 1), (50, 3.0, 2), (500, 4.0, 3), (2000, 8.0, 4),
                                      (20000, 4.0, 5)])
def test_recolouring_matches_brute_force_and_never_adds_a_colour(n, c, seed):
    rp, col, _ = sg_inputs.poisson_graph(n, c, seed)
    first, nc1 = oracle.greedy_colour(rp, col)
    colour, nc = oracle.recolour(rp, col, first)
    want = brute_recolour(rp, col, first)
    assert np.array_equal(colour, want)
    assert nc == want.max() + 1 <= nc1
    src = np.repeat(np.arange(n), np.diff(rp))
    assert not np.any(colour[src] == colour[col])
    both, ncb = oracle.vb_colouring(rp, col)
    assert np.array_equal(both, colour) and ncb == nc


def test_recolouring_removes_the_thin_last_classes():
    """A Poisson c = 4 graph: the greedy pass ends in classes of a handful of vertices, which
    the recolouring pass folds into the others."""
    rp, col, _ = sg_inputs.poisson_graph(200000, 4.0, 7)
    first, nc1 = oracle.greedy_colour(rp, col)
    colour, nc = oracle.recolour(rp, col, first)
    assert nc < nc1
    assert np.bincount(colour).min() > np.bincount(first).min()


def test_recolouring_keeps_the_two_halves_of_a_bipartite_graph():
    """The even cycle: the two halves swap (the old class 1 is coloured first)."""
    n = 10
    ei = np.arange(n)
    ej = (ei + 1) % n
    rp, col, _ = sg_inputs.csr_from_edges(n, ei, ej)
    colour, nc = oracle.vb_colouring(rp, col)
    assert nc == 2 and np.array_equal(colour, 1 - np.arange(n) % 2)
