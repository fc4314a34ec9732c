"""Tuned, graph-captured query plans (caps_plan_*): one persistent scan launch
per batch inside one CUDA graph, launch shape chosen by the autotuner.

The plan must return exactly what caps_search_batch returns for the same
batch (the graph replays the same kernels), and the byte-valued bf16 case
must still equal the CPU oracle bit for bit.  The autotuner itself checks
that all four launch shapes (256 or 128 rows per tile x 128 or 64 probes per
work item) agree to the bit on the tuning batch, so a successful plan
creation covers every shape, the penalty form (block selection and filter
folded into the MMA) against the per-pair filter included.
"""
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


def wl(seed, N=20_000, d=128, B=16, h=7, nq=700, integer=True):
    return make_dense_workload(
        name="plan", N=N, d=d, ncomp=12, center=("uniform", 128.0) if integer else ("normal", 2.0),
        sigma=16.0 if integer else 1.0, vocab=[5, 7, 11], zipf_s=1.0, nq=nq, cmin=1, cmax=3,
        B=B, h=h, iters=5, m=4, k=10, seed=seed, integer=integer)


def gpu_index(w, prec):
    return caps.Index.build(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.A).cuda(), w.vocab,
                            w.B, h=w.h, iters=w.iters, metric=w.metric, init_idx=w.init_idx,
                            prec=prec)


def test_plan_bf16_autotuned_equals_direct_and_oracle():
    # 700 queries x 6 probes over 16 partitions: several 128-probe (and more
    # 64-probe) items per partition, partitions of ~1,250 rows (several tiles)
    w = wl(901)
    gi = gpu_index(w, caps.BF16)
    Q = torch.from_numpy(w.Q).cuda()
    Qb = torch.from_numpy(w.Qb).cuda()
    k, m = 10, 6
    plan = gi.plan(Q, Qb, k, m, autotune=True)
    inf = plan.info
    assert inf["nq"] == w.nq and inf["k"] == k and inf["m"] == m
    # filter per pair in the epilogue (256 or 128 rows per tile) or folded
    # into the MMA (128 rows), x 128 or 64 probes per item; the vocabularies
    # 5/7/11 (10 packed bits) and 8 blocks fit the one-hot code chunk
    assert {(c["tile_n"], c["item_cap"], c["pen"]) for c in inf["candidates"]} == {
        (256, 128, 0), (128, 128, 0), (256, 64, 0), (128, 64, 0), (128, 128, 1), (128, 64, 1)}
    assert all(c["ms"] > 0 for c in inf["candidates"])
    assert (inf["tile_n"], inf["item_cap"], inf["pen"]) in {
        (c["tile_n"], c["item_cap"], c["pen"]) for c in inf["candidates"]}
    assert inf["graph_nodes"] > 5
    d_ids, d_dist = gi.search(Q, Qb, k, m)
    for _ in range(3):  # replays are repeatable
        p_ids, p_dist = plan.search(Q, Qb)
        torch.cuda.synchronize()
        assert torch.equal(p_ids, d_ids)
        assert torch.equal(p_dist, d_dist)
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, w.iters, w.init_idx, w.metric)
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons.of(w), k, m)
    np.testing.assert_array_equal(p_ids.cpu().numpy(), oids)
    np.testing.assert_array_equal(p_dist.cpu().numpy(), odist)
    gi.status()
    plan.close()


def test_plan_host_buffers_and_short_batch():
    w = wl(902, nq=400)
    gi = gpu_index(w, caps.BF16)
    plan = gi.plan(w.Q, w.Qb, 10, 5, autotune=False)
    assert plan.info["candidates"] == [] and plan.info["pen"] == 1 and plan.info["tile_n"] == 128
    ids, dist = plan.search(w.Q, w.Qb)  # numpy in, numpy out
    r_ids, r_dist = gi.search(w.Q, w.Qb, 10, 5)
    np.testing.assert_array_equal(ids, r_ids)
    np.testing.assert_array_equal(dist, r_dist)
    # a shorter batch: its rows are answered, the plan's other rows ignored
    q2, b2 = np.ascontiguousarray(w.Q[::-1][:150]), np.ascontiguousarray(w.Qb[::-1][:150])
    ids2, dist2 = plan.search(q2, b2)
    r2_ids, r2_dist = gi.search(q2, b2, 10, 5)
    np.testing.assert_array_equal(ids2, r2_ids)
    np.testing.assert_array_equal(dist2, r2_dist)
    with pytest.raises(caps.CapsError):
        plan.search(np.zeros((401, w.X.shape[1]), np.float32), np.zeros((401, 3), np.int32))
    plan.close()


def test_plan_fp32_index_has_nothing_to_tune():
    w = wl(903, nq=300, integer=False)
    gi = gpu_index(w, caps.FP32)
    Q = torch.from_numpy(w.Q).cuda()
    Qb = torch.from_numpy(w.Qb).cuda()
    plan = gi.plan(Q, Qb, 10, 4, autotune=True)
    assert plan.info["candidates"] == [] and plan.info["tile_n"] == 0
    p_ids, p_dist = plan.search(Q, Qb)
    d_ids, d_dist = gi.search(Q, Qb, 10, 4)
    torch.cuda.synchronize()
    assert torch.equal(p_ids, d_ids) and torch.equal(p_dist, d_dist)
    plan.close()


def test_plan_rejects_bad_arguments():
    w = wl(904, N=4000, nq=50)
    gi = gpu_index(w, caps.BF16)
    with pytest.raises(caps.CapsError):
        gi.plan(w.Q, w.Qb, 0, 4)
    with pytest.raises(caps.CapsError):
        gi.plan(w.Q, w.Qb, 10, w.B + 1)
    with pytest.raises(caps.CapsError):
        gi.plan(w.Q[:0], w.Qb[:0], 10, 4)
