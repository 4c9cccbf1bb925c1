"""GPU parity of the multi-source BFS (Alg. 3): levels are integers and must
match the oracle bit for bit; the number of products must equal the
oracle's (1 + the largest level)."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

from paper_2408_11988_gb300 import DeviceCSR
from paper_2408_11988_gb300.msbfs import msbfs


# d up to 256 runs the bitmap pull form (1, 2, 4 or 8 words per row), d above
# it the list form
@pytest.mark.parametrize("scale,ef,d", [(10, 8, 128), (12, 16, 128), (9, 4, 40), (8, 2, 1), (10, 8, 200),
                                        (9, 8, 300), (10, 6, 64), (9, 8, 33), (11, 16, 256)])
def test_msbfs_matches_oracle(scale, ef, d):
    A = synth.rmat(scale, ef, 60 + scale, symmetrize=True)
    src = synth.sources(A, d, 61)
    r = msbfs(DeviceCSR.from_host(A, with_values=False), torch.as_tensor(src))
    lev, prods, fnnz = oracle.msbfs(A, src)
    np.testing.assert_array_equal(r.levels.cpu().numpy(), lev)
    assert r.products == prods
    np.testing.assert_array_equal(np.array(r.frontier_nnz), fnnz)


def test_msbfs_directed_pulls_over_rows():
    # on a directed graph the pull over A's rows follows A^T: compare with the
    # oracle's Alg. 3, which uses the same product
    A = synth.rmat(10, 8, 62)
    src = synth.sources(A, 64, 63)
    r = msbfs(DeviceCSR.from_host(A, with_values=False), torch.as_tensor(src))
    lev, prods, _ = oracle.msbfs(A, src)
    np.testing.assert_array_equal(r.levels.cpu().numpy(), lev)
    assert r.products == prods


def test_msbfs_full_size_all_sources():
    # the multi-source BFS workload at full size: R-MAT scale 20, edge factor
    # 16, symmetrised, 128 sources; every source column against a queue BFS
    A, src = synth.msbfs_graph()
    r = msbfs(DeviceCSR.from_host(A, with_values=False), torch.as_tensor(src))
    lev = r.levels.cpu().numpy()
    for s in range(len(src)):
        ref = oracle.bfs_levels(A, int(src[s]))
        np.testing.assert_array_equal(lev[:, s], ref, err_msg=f"source {s}")
    maxlev = int(lev.max())
    assert r.products == maxlev + 1
    assert r.frontier_nnz[-1] == 0 and sum(r.frontier_nnz) == int((lev >= 0).sum())


@pytest.mark.parametrize("scale,ef,d", [(10, 8, 128), (9, 4, 40), (8, 2, 1), (10, 8, 200), (10, 6, 64),
                                        (11, 16, 256)])
def test_msbfs_parents_match_oracle(scale, ef, d):
    # the BFS-tree variant, (sel2nd, min): parents are integers, bit-exact
    A = synth.rmat(scale, ef, 70 + scale, symmetrize=True)
    src = synth.sources(A, d, 71)
    r = msbfs(DeviceCSR.from_host(A, with_values=False), torch.as_tensor(src), parents=True)
    lev, par, prods, fnnz = oracle.msbfs_parents(A, src)
    np.testing.assert_array_equal(r.levels.cpu().numpy(), lev)
    np.testing.assert_array_equal(r.parents.cpu().numpy(), par)
    assert r.products == prods


def test_msbfs_parents_directed_and_hubs():
    # directed graph (pull over A's rows) with a hub row taken by a whole block
    A = synth.rmat(11, 24, 72)
    src = synth.sources(A, 96, 73)
    r = msbfs(DeviceCSR.from_host(A, with_values=False), torch.as_tensor(src), parents=True)
    lev, par, prods, _ = oracle.msbfs_parents(A, src)
    np.testing.assert_array_equal(r.levels.cpu().numpy(), lev)
    np.testing.assert_array_equal(r.parents.cpu().numpy(), par)


def _first_closer_neighbour(rp, col, ref, n):
    """For every vertex v with ref[v] > 0, its smallest neighbour u with
    ref[u] == ref[v] - 1 (rows of A are sorted, so the first such entry);
    -1 elsewhere."""
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    lv = ref[rows]
    ok = (lv > 0) & (ref[col] == lv - 1)
    idx = np.flatnonzero(ok)
    out = np.full(n, -1, dtype=np.int64)
    if idx.size:
        r = rows[idx]
        first = np.concatenate([[0], np.flatnonzero(np.diff(r)) + 1])
        out[r[first]] = col[idx[first]]
    return out


def test_msbfs_parents_full_size_all_sources():
    # full-size workload, all 128 sources: levels against a queue BFS, and
    # every reached vertex's parent is its smallest neighbour one level closer
    # (the (sel2nd, min) BFS tree); sources are their own parents
    A, src = synth.msbfs_graph()
    r = msbfs(DeviceCSR.from_host(A, with_values=False), torch.as_tensor(src), parents=True)
    lev = r.levels.cpu().numpy()
    par = r.parents.cpu().numpy()
    rp, col = A.rowptr, A.col
    for s in range(len(src)):
        ref = oracle.bfs_levels(A, int(src[s]))
        np.testing.assert_array_equal(lev[:, s], ref, err_msg=f"source {s}")
        want = _first_closer_neighbour(rp, col, ref, A.nrows)
        want[int(src[s])] = int(src[s])
        np.testing.assert_array_equal(par[:, s], want, err_msg=f"parents of source {s}")
