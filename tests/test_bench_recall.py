"""The benchmark's recall (bench.recall_at_k, a numpy restatement of the
paper's RecallK@K with the tie-aware reading) against the oracle's recall on
random cases: duplicated and missing ids, padding, ties at the k-th
distance, queries with fewer than k valid points, both metrics."""
import importlib.util
import os

import numpy as np

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_recall", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_recall_matches_the_oracle():
    b = _bench()
    rng = np.random.default_rng(12)
    for metric in (0, 1):
        for trial in range(40):
            N, d, nq, k = 60, 4, 25, 10
            X = rng.integers(0, 4, (N, d)).astype(np.float32)  # small ints: many ties
            Q = rng.integers(0, 4, (nq, d)).astype(np.float32)
            cnt = rng.integers(0, 3 * k, nq)
            gt = np.full((nq, k), -1, dtype=np.int64)
            g64 = np.zeros((nq, k))
            ids = np.full((nq, k), -1, dtype=np.int64)
            for q in range(nq):
                valid = rng.choice(N, min(cnt[q], N), replace=False)
                dv = b.exact_dist(X[valid], Q[q], metric)
                order = np.lexsort((valid, dv if metric == 0 else -dv))[:k]
                gt[q, :len(order)] = valid[order]
                g64[q, :len(order)] = dv[order]
                n_ret = rng.integers(0, k + 1)
                ids[q, :n_ret] = rng.choice(valid if len(valid) and rng.random() < 0.7 else
                                            np.arange(N), n_ret)
            got = b.recall_at_k(ids, gt, g64, cnt, k, X, Q, metric)
            want = O.recall(ids, gt, g64, cnt, k, X=X, Q=Q, metric=metric)
            assert np.isclose(got[0], want[0]) and np.isclose(got[1], want[1]), (got, want[:2])
