"""Disjunctive constraints on the GPU (caps_search_batch_or, Sec. 5.3)
against the oracle's search_or, element by element.  Byte-valued rows make
every distance an exact integer, so the fp32 and the bf16 tensor-core forms
must both equal the oracle bit for bit."""
import numpy as np
import pytest

import oracle as O
from workloads import make_dense_workload

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2308_15014_gb300 import build
    build.build()


import paper_2308_15014_gb300 as caps  # noqa: E402


def _w(seed, d=64, nq=150, vocab=(5, 7, 11)):
    return make_dense_workload(name="or", N=12000, d=d, ncomp=16, center=("uniform", 128.0),
                               sigma=16.0, vocab=list(vocab), zipf_s=1.0, nq=nq, cmin=1,
                               cmax=len(vocab), B=24, h=7, iters=4, m=5, k=10, seed=seed,
                               integer=True)


def _lists(w, rng):
    out = []
    for q in range(w.nq):
        row = []
        for f, V in enumerate(w.vocab):
            b = int(w.Qb[q, f])
            if b >= 0:
                row.append(sorted(set([b] + rng.choice(V, rng.integers(0, 3), replace=False).tolist())))
            elif rng.random() < 0.15:
                row.append(sorted(rng.choice(V, 2, replace=False).tolist()))
            else:
                row.append([])
        out.append(row)
    out[0] = [[], [], []]               # no constraint at all
    out[1] = [[0, 1, 2, 3, 4], [], [10, 99]]  # a value outside the vocabulary
    return out


@pytest.mark.parametrize("prec,k,m", [(0, 10, 5), (1, 10, 5), (1, 7, 24), (0, 33, 3)])
def test_or_search_equals_oracle(prec, k, m):
    w = _w(300 + k + m)
    ix = caps.Index.build(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.A).cuda(), w.vocab,
                          w.B, h=w.h, iters=w.iters, init_idx=w.init_idx, prec=prec)
    lists = _lists(w, np.random.default_rng(k))
    ids, dist = ix.search_or(torch.from_numpy(w.Q).cuda(), lists, k, m)
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, C=ix.export(caps.ARR_CENTROIDS))
    oids, odist = O.search_or(w.X, O.Attrs.of(w), oi, w.Q, O.OrCons.of_lists(lists), k, m)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_array_equal(dist.cpu().numpy(), odist)
    # host buffers in and out give the same
    hids, hdist = ix.search_or(w.Q, lists, k, m)
    np.testing.assert_array_equal(hids, oids)
    ix.close()


def test_single_values_equal_search_batch():
    w = _w(351)
    ix = caps.Index.build(w.X, w.A, w.vocab, w.B, h=w.h, iters=w.iters, init_idx=w.init_idx,
                          prec=caps.BF16)
    lists = [[[int(b)] if b >= 0 else [] for b in w.Qb[q]] for q in range(w.nq)]
    ids, dist = ix.search_or(w.Q, lists, w.k, w.m)
    rids, rdist = ix.search(w.Q, w.Qb, w.k, w.m)
    np.testing.assert_array_equal(ids, rids)
    np.testing.assert_array_equal(dist, rdist)
    ix.close()


def test_or_rejects_too_many_combinations():
    w = _w(352, nq=3)
    ix = caps.Index.build(w.X, w.A, w.vocab, w.B, h=w.h, iters=2, init_idx=w.init_idx)
    lists = [[list(range(5)), list(range(7)), list(range(8))]] + [[[], [], []]] * 2  # 280 > 256
    with pytest.raises(caps.CapsError) as e:
        ix.search_or(w.Q, lists, 10, 4)
    assert e.value.code == caps.CAPS_EINVAL
    ix.close()
