"""Dynamic insertion on the GPU (caps_insert) against the oracle's insert:
after each batch the index arrays (partitions, tags, blocks, layout) equal
the oracle's bit for bit and searches equal the oracle's Alg. 2 on the grown
index (byte-valued rows: exact distances on every path).  A plan made before
an insertion refuses to run; an insertion that runs out of device memory
leaves the index as it was."""
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


def _w(seed, N=9000):
    return make_dense_workload(name="ins", N=N, d=64, ncomp=16, center=("uniform", 128.0),
                               sigma=16.0, vocab=[5, 9, 13], zipf_s=1.0, nq=160, cmin=1, cmax=3,
                               B=20, h=7, iters=4, m=5, k=10, seed=seed, integer=True)


def _init(w, n0):
    """k-means seed points among the first n0 rows (the built part)."""
    return (np.arange(w.B, dtype=np.int64) * (n0 // w.B)).astype(np.int64)


def _check(gi, oi, w, n, probe_in=None):
    np.testing.assert_array_equal(gi.export(caps.ARR_BIN), oi.bin)
    np.testing.assert_array_equal(gi.export(caps.ARR_TAGS), oi.tags)
    np.testing.assert_array_equal(gi.export(caps.ARR_KEY), oi.key)
    np.testing.assert_array_equal(gi.export(caps.ARR_PERM), oi.perm)
    np.testing.assert_array_equal(gi.export(caps.ARR_OFFSETS), oi.offsets)
    ids, dist = gi.search(w.Q, w.Qb, w.k, w.m)
    at = O.Attrs(A=w.A[:n], vocab=w.vocab)
    oids, odist, _, _ = O.search(w.X[:n], at, oi, w.Q, O.Cons(Qb=w.Qb), w.k, w.m,
                                 probe_in=probe_in)
    np.testing.assert_array_equal(ids, oids)
    np.testing.assert_array_equal(dist, odist)


@pytest.mark.parametrize("prec", [0, 1])
def test_insert_kmeans_equals_oracle(prec):
    w = _w(500 + prec)
    n0, n1 = 6000, 7500
    gi = caps.Index.build(w.X[:n0], w.A[:n0], w.vocab, w.B, h=w.h, iters=w.iters,
                          init_idx=_init(w, n0), prec=prec)
    oi = O.build(w.X[:n0], O.Attrs(A=w.A[:n0], vocab=w.vocab), w.B, w.h, 0, _init(w, n0),
                 C=gi.export(caps.ARR_CENTROIDS))
    _check(gi, oi, w, n0)
    for lo, hi in ((n0, n1), (n1, w.N)):
        gi.insert(torch.from_numpy(w.X[lo:hi]).cuda(), torch.from_numpy(w.A[lo:hi]).cuda())
        assert gi.info.N == hi
        oi = O.insert(oi, w.X[:hi], O.Attrs(A=w.A[:hi], vocab=w.vocab), hi - lo)
        _check(gi, oi, w, hi)
    gi.close()


def test_insert_learned_partitioner_equals_oracle():
    w = _w(510)
    n0 = 6000
    gi = caps.Index.build(w.X[:n0], w.A[:n0], w.vocab, w.B, h=w.h, iters=w.iters,
                          init_idx=_init(w, n0), prec=caps.BF16, part=caps.MLP, mlp_hidden=64,
                          mlp_epochs=2, mlp_samples=2000, mlp_batch=500, mlp_lr=1e-3, seed=5)
    H, d, B = gi.info.mlp_hidden, w.d, w.B
    Wf = gi.export(caps.ARR_MLP)
    net = O.MLP(Wf[:H * d].reshape(H, d), Wf[H * d:H * d + H],
                Wf[H * d + H:H * d + H + B * H].reshape(B, H), Wf[H * d + H + B * H:])
    oi = O.build(w.X[:n0], O.Attrs(A=w.A[:n0], vocab=w.vocab), w.B, w.h, 0, _init(w, n0),
                 bins=gi.export(caps.ARR_BIN))
    gi.insert(w.X[n0:], w.A[n0:])
    oi = O.insert(oi, w.X, O.Attrs.of(w), w.N - n0, bins_new=O.mlp_assign32(w.X[n0:], net))
    _check(gi, oi, w, w.N, probe_in=O.probe_logits(w.Q, net, w.m))
    gi.close()


def test_plan_made_before_an_insertion_refuses_to_run():
    w = _w(520)
    n0 = 7000
    gi = caps.Index.build(w.X[:n0], w.A[:n0], w.vocab, w.B, h=w.h, iters=2,
                          init_idx=_init(w, n0), prec=caps.BF16)
    Q, Qb = torch.from_numpy(w.Q).cuda(), torch.from_numpy(w.Qb).cuda()
    plan = gi.plan(Q, Qb, w.k, w.m, autotune=False)
    gi.insert(w.X[n0:], w.A[n0:])
    ids = torch.empty((w.nq, w.k), dtype=torch.int64, device="cuda")
    dist = torch.empty((w.nq, w.k), dtype=torch.float32, device="cuda")
    with pytest.raises(caps.CapsError) as e:
        plan.search(Q, Qb, out_ids=ids, out_dist=dist)
    assert e.value.code == caps.CAPS_EINVAL
    plan.close()
    plan = gi.plan(Q, Qb, w.k, w.m, autotune=False)
    plan.search(Q, Qb, out_ids=ids, out_dist=dist)
    torch.cuda.synchronize()
    rids, _ = gi.search(w.Q, w.Qb, w.k, w.m)
    np.testing.assert_array_equal(ids.cpu().numpy(), rids)
    plan.close()
    gi.close()


@pytest.mark.parametrize("fail_at", [1, 4, 9])
def test_insert_out_of_memory_leaves_the_index(fail_at):
    w = _w(530)
    n0 = 7000
    gi = caps.Index.build(w.X[:n0], w.A[:n0], w.vocab, w.B, h=w.h, iters=2,
                          init_idx=_init(w, n0), prec=caps.BF16)
    before = gi.search(w.Q, w.Qb, w.k, w.m)
    caps.inject_alloc_failure(fail_at)
    with pytest.raises(caps.CapsError) as e:
        gi.insert(w.X[n0:], w.A[n0:])
    caps.inject_alloc_failure(0)
    assert e.value.code == caps.CAPS_ENOMEM
    assert gi.info.N == n0
    after = gi.search(w.Q, w.Qb, w.k, w.m)
    np.testing.assert_array_equal(after[0], before[0])
    np.testing.assert_array_equal(after[1], before[1])
    gi.close()
