"""The paper's own graph ensembles as input data: random regular graphs of degree z, plain and
bipartite (halves [0, N/2) and [N/2, N)).  Checks the structure the dynamics relies on: every
degree is z, the graph is simple, a bipartite graph only has edges across the halves, and
greedy colouring in vertex order splits a bipartite graph into exactly its two halves (the
paper's half-sweep update order, SI section 3)."""
import numpy as np
import pytest

import oracle
import sg_inputs


def _edges(rp, col):
    n = rp.size - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    return src, col.astype(np.int64)


@pytest.mark.parametrize("bipartite", [False, True])
@pytest.mark.parametrize("n,z", [(64, 3 * 2), (1000, 4), (4096, 4), (2 ** 14, 4)])
def test_regular_graph_structure(n, z, bipartite):
    if bipartite and z >= n // 2:
        pytest.skip("degree too large")
    rp, col, eid = sg_inputs.random_regular_graph(n, z, 11, bipartite=bipartite)
    assert np.all(np.diff(rp) == z)
    src, dst = _edges(rp, col)
    assert np.all(src != dst)
    keys = src * n + dst
    assert np.unique(keys).size == keys.size                      # no multi-edges
    rev = np.sort(dst * n + src)
    assert np.array_equal(np.sort(keys), rev)                     # symmetric
    assert eid.max() + 1 == n * z // 2                            # one id per undirected edge
    if bipartite:
        assert np.all((src < n // 2) != (dst < n // 2))           # edges only across halves


def test_bipartite_graph_colours_into_its_halves():
    n = 4096
    rp, col, _ = sg_inputs.random_regular_graph(n, 4, 5, bipartite=True)
    colour, nc = oracle.greedy_colour(rp, col)
    assert nc == 2
    assert np.all(colour[: n // 2] == 0) and np.all(colour[n // 2:] == 1)


def test_plain_regular_graph_is_not_bipartite_and_needs_more_colours():
    rp, col, _ = sg_inputs.random_regular_graph(4096, 4, 5)
    _, nc = oracle.greedy_colour(rp, col)
    assert nc >= 3


def test_generator_is_seeded():
    a = sg_inputs.random_regular_graph(2000, 4, 9, bipartite=True)
    b = sg_inputs.random_regular_graph(2000, 4, 9, bipartite=True)
    c = sg_inputs.random_regular_graph(2000, 4, 10, bipartite=True)
    assert np.array_equal(a[1], b[1]) and not np.array_equal(a[1], c[1])


def test_tritone_windows_follow_the_lumping_formula():
    """SI section 1: times T = t + t_w with equal floor(ln(T/4) / (0.5 ln 2)) form one lump;
    {4, 5} is the first lump (its mean time is 4.5)."""
    import math
    b = sg_inputs.tritone_windows(5000)
    assert list(b[:3]) == [4, 6, 8]
    for m in range(len(b) - 1):
        for T in range(int(b[m]), int(b[m + 1])):
            assert math.floor(math.log(T / 4) / (0.5 * math.log(2.0))) == m


def test_geometric_windows_have_ratio_two_to_the_quarter():
    b = sg_inputs.geometric_windows(64, 10 ** 6)
    assert b[0] == 64 and b[-1] > 10 ** 6
    assert np.all(np.diff(b) > 0)
    r = b[8:] / b[:-8]  # two octaves later: ratio 4 up to rounding
    assert np.all(np.abs(r - 4.0) < 4.0 * 2.0 / b[:-8] + 1e-12)
