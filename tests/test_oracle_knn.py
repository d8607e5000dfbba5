"""Pins for the oracle's exact kNN graph and ground truth (Alg. 3 line 1 builds the kNN
graph; Sec. 5.2 scores against brute-force ground truth).

The pins are independent of the oracle's own code: scipy's pairwise distance routine with
numpy's lexicographic sort, integer data whose distances are exact, duplicates and the
self-exclusion rule.
"""
import numpy as np
import pytest
from scipy.spatial.distance import cdist

import oracle
from paper_1907_06146_gb300 import synth


def _lib_knn(base, queries, k, exclude_self):
    d2 = cdist(queries.astype(np.float64), base.astype(np.float64), "sqeuclidean")
    n = base.shape[0]
    ids = np.empty((queries.shape[0], k), np.int64)
    vals = np.empty((queries.shape[0], k))
    for r in range(queries.shape[0]):
        row = d2[r].copy()
        cand = np.arange(n)
        if exclude_self:
            cand = cand[cand != r]
            row = row[cand]
        order = np.lexsort((cand, row))  # primary key: distance, then id
        ids[r] = cand[order[:k]]
        vals[r] = row[order[:k]]
    return ids, vals


@pytest.mark.parametrize("n,d,k,seed", [(300, 7, 10, 1), (257, 32, 20, 2), (64, 3, 63, 3)])
def test_knn_rows_matches_library_float(n, d, k, seed):
    base = synth.uniform_points(n, d, seed)
    ids, d2 = oracle.knn_rows(base, k)
    ref_ids, ref_d2 = _lib_knn(base, base, k, exclude_self=True)
    np.testing.assert_array_equal(ids, ref_ids)
    np.testing.assert_allclose(d2, ref_d2, rtol=1e-12, atol=0)


def test_knn_rows_integer_ties_exact():
    # integers 0..3 in 4-D: many exactly equal distances, so the id tie-break decides
    base = synth.uniform_points(400, 4, 11, integer=True, hi=3)
    ids, d2 = oracle.knn_rows(base, 30)
    ref_ids, ref_d2 = _lib_knn(base, base, 30, exclude_self=True)
    np.testing.assert_array_equal(ids, ref_ids)
    np.testing.assert_array_equal(d2, ref_d2)


def test_knn_duplicates_and_self():
    base = synth.uniform_points(50, 5, 4)
    base[7] = base[3]
    base[12] = base[3]
    ids, d2 = oracle.knn_rows(base, 5)
    # row 3: its two duplicates first, at distance exactly 0, in id order; never itself
    assert ids[3, 0] == 7 and ids[3, 1] == 12
    assert d2[3, 0] == 0.0 and d2[3, 1] == 0.0
    assert ids[7, 0] == 3 and ids[7, 1] == 12
    for i in range(50):
        assert i not in ids[i]


def test_knn_rows_subset_equals_full():
    base = synth.uniform_points(200, 6, 5)
    full_ids, full_d2 = oracle.knn_rows(base, 8)
    rows = np.array([5, 0, 199, 42])
    ids, d2 = oracle.knn_rows(base, 8, rows=rows)
    np.testing.assert_array_equal(ids, full_ids[rows])
    np.testing.assert_array_equal(d2, full_d2[rows])


def test_knn_rejects_k_too_large():
    base = synth.uniform_points(10, 2, 6)
    with pytest.raises(ValueError):
        oracle.knn_rows(base, 10)


def test_knn_queries_matches_library():
    base = synth.uniform_points(500, 16, 7)
    q = synth.uniform_points(40, 16, 8)
    ids, d2 = oracle.knn_queries(base, q, 10)
    ref_ids, ref_d2 = _lib_knn(base, q, 10, exclude_self=False)
    np.testing.assert_array_equal(ids, ref_ids)
    np.testing.assert_allclose(d2, ref_d2, rtol=1e-12)


def test_knn_small_workload_sample():
    w = synth.small(n=2000, nq=10)
    rows = np.arange(0, 2000, 97)
    ids, _ = oracle.knn_rows(w.base, w.K, rows=rows)
    d2 = cdist(w.base[rows].astype(np.float64), w.base.astype(np.float64), "sqeuclidean")
    for r, i in enumerate(rows):
        d2[r, i] = np.inf
        order = np.lexsort((np.arange(2000), d2[r]))
        np.testing.assert_array_equal(ids[r], order[:w.K])


def test_recall_definition():
    truth = np.array([[1, 2, 3, 4], [5, 6, 7, 8]])
    found = np.array([[4, 3, 9, 1], [0, 0, 0, 5]])
    # |R n G| / |G| per query (Sec. 5.2), averaged: (3 + 1) / 8
    assert oracle.recall_at(found, truth, k=4) == pytest.approx(0.5)
