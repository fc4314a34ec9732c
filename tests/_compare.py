"""Comparison of batched search results (GPU vs oracle, or two GPU entry
points).

Distances: within 1e-5 relative (the fp32 contract).  Ids: equal rank by rank
except where two candidates' distances are within that tolerance of each
other (several answers are then correct); a swapped-in id must itself have
the distance the reference reports at that rank, pass the query's filter and
not repeat.  The number of results found must match exactly.
"""
import numpy as np

RTOL = 1e-5


def _close(a, b):
    return abs(a - b) <= RTOL * max(abs(a), abs(b)) + 1e-30


def assert_search_equal(ids, dist, ref_ids, ref_dist, X=None, Q=None, A=None, Qb=None,
                        exact=False, metric=0):
    ids, dist = np.asarray(ids), np.asarray(dist)
    ref_ids, ref_dist = np.asarray(ref_ids), np.asarray(ref_dist)
    assert ids.shape == ref_ids.shape
    if exact:
        np.testing.assert_array_equal(ids, ref_ids)
        np.testing.assert_array_equal(dist, ref_dist)
        return
    np.testing.assert_array_equal(ids >= 0, ref_ids >= 0)
    fin = np.isfinite(ref_dist)
    np.testing.assert_array_equal(np.isfinite(dist), fin)
    np.testing.assert_allclose(dist[fin], ref_dist[fin], rtol=RTOL, atol=0)
    for q in range(ids.shape[0]):
        got = ids[q][ids[q] >= 0]
        assert len(set(got.tolist())) == len(got), "duplicate id"
        for r in np.nonzero(ids[q] != ref_ids[q])[0]:
            i = int(ids[q, r])
            assert X is not None, "ids differ and no data to check near-ties"
            x, y = X[i].astype(np.float64), Q[q].astype(np.float64)
            di = float(((x - y) ** 2).sum()) if metric == 0 else float((x * y).sum())
            assert _close(di, float(ref_dist[q, r])), (q, r, i, di, ref_dist[q, r])
            if A is not None:
                b = Qb[q]
                assert np.all((b < 0) | (A[i] == b)), "swapped-in id violates the filter"
