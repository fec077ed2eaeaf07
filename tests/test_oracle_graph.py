"""Pins for the oracle's mesh, CRS graph, ElemGraph and boundary mask.

The graph is defined (Fig. 2, Algorithm 2 NodeIndex/ElemGraph) as: row I holds
every node that shares a cell with I.  The oracle builds it from the union of
cell node lists; these tests check it against an independent characterisation
(|i-i'|, |j-j'|, |k-k'| <= 1) and the closed forms that follow from it.
"""
import itertools

import numpy as np
import pytest

import oracle as O


def node(N, i, j, k):
    return i + (N + 1) * (j + (N + 1) * k)


@pytest.mark.parametrize("N", [1, 2, 3, 5])
def test_graph_matches_box_neighbourhood(N):
    row_map, col = O.graph(N)
    n = (N + 1) ** 3
    assert len(row_map) == n + 1 and row_map[0] == 0
    for k, j, i in itertools.product(range(N + 1), repeat=3):
        I = node(N, i, j, k)
        expect = sorted(node(N, i + a, j + b, k + c)
                        for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)
                        if 0 <= i + a <= N and 0 <= j + b <= N and 0 <= k + c <= N)
        got = col[row_map[I]:row_map[I + 1]].tolist()
        assert got == expect, (N, I)


@pytest.mark.parametrize("N", [1, 2, 4, 7, 8, 16])
def test_graph_closed_form_counts(N):
    row_map, col = O.graph(N)
    assert row_map[-1] == (3 * N + 1) ** 3 == len(col)
    lens = np.diff(row_map)
    f = np.array([2 if t in (0, N) else 3 for t in range(N + 1)])
    expect = (f[None, None, :] * f[None, :, None] * f[:, None, None]).reshape(-1)
    assert np.array_equal(lens, expect)
    # strictly ascending within each row
    for I in range(0, (N + 1) ** 3, max(1, (N + 1) ** 3 // 97)):
        r = col[row_map[I]:row_map[I + 1]]
        assert np.all(np.diff(r) > 0)


def test_graph_sizes_of_the_workloads():
    # 8^3 and 16^3 built in full; the others by the closed form checked above
    for N, n, nnz in [(8, 729, 15625), (16, 4913, 117649)]:
        row_map, col = O.graph(N)
        assert len(row_map) - 1 == n and len(col) == nnz


def test_graph_structurally_symmetric():
    N = 4
    row_map, col = O.graph(N)
    pairs = set()
    for I in range(len(row_map) - 1):
        for J in col[row_map[I]:row_map[I + 1]]:
            pairs.add((I, int(J)))
    assert all((J, I) in pairs for (I, J) in pairs)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_node_index_and_elem_graph(N):
    ni = O.node_index(N)
    for ck, cj, ci in itertools.product(range(N), repeat=3):
        c = ci + N * (cj + N * ck)
        for l in range(8):
            assert ni[c, l] == node(N, ci + (l & 1), cj + ((l >> 1) & 1), ck + ((l >> 2) & 1))
    row_map, col = O.graph(N)
    eg = O.elem_graph(N, row_map, col).reshape(N ** 3, 8, 8)
    for c in range(N ** 3):
        for a in range(8):
            I = ni[c, a]
            for b in range(8):
                e = eg[c, a, b]
                assert row_map[I] <= e < row_map[I + 1]
                assert col[e] == ni[c, b]


@pytest.mark.parametrize("N", [1, 2, 6])
def test_bmask(N):
    bm = O.bmask(N)
    assert bm.sum() == (N + 1) ** 3 - max(N - 1, 0) ** 3
    for k, j, i in itertools.product(range(N + 1), repeat=3):
        on = min(i, j, k) == 0 or max(i, j, k) == N
        assert bm[node(N, i, j, k)] == int(on)
