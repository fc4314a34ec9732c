"""GPU path vs the CPU oracle, element by element, through the C ABI.

Integer outputs of the build and of the probe/selection steps (assignment,
tags, blocks, layout, probes, selections) must match bit for bit: both sides
take those decisions on the same fp32 value (coordinates in order, one fused
multiply-add each).  The batch scan sums each distance in a different order
(lane partials, then pairwise), so its distances are compared within 1e-5
relative and its ids rank by rank up to near-ties; on byte-valued data every
partial sum is an exact integer and results must be identical.
"""
import numpy as np
import pytest

import oracle as O
from _compare import assert_search_equal
from workloads import config_small, make_dense_workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2308_15014_gb300 import build
    build.build()


import paper_2308_15014_gb300 as caps  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def tiny(seed, N=1000, d=33, ncomp=6, vocab=(3, 5, 9), nq=37, B=7, h=5, integer=False,
         metric=0, normalize=False, cmax=3):
    return make_dense_workload(
        name="tiny", N=N, d=d, ncomp=ncomp,
        center=("uniform", 128.0) if integer else ("normal", 2.0),
        sigma=16.0 if integer else 1.0, vocab=list(vocab), zipf_s=1.0, nq=nq, cmin=1,
        cmax=min(cmax, len(vocab)), B=B, h=h, iters=6, m=3, k=10, seed=seed,
        integer=integer, metric=metric, normalize=normalize)


def oracle_index(w, h=None, C=None, iters=None):
    return O.build(w.X, O.Attrs.of(w), w.B, w.h if h is None else h,
                   w.iters if iters is None else iters, w.init_idx, w.metric, C=C)


def gpu_index(w, h=None, C=None, iters=None, on_device=True):
    X = dev(w.X) if on_device else w.X
    A = dev(w.A) if on_device else w.A
    return caps.Index.build(X, A, w.vocab, w.B, h=w.h if h is None else h,
                            iters=w.iters if iters is None else iters, metric=w.metric,
                            init_idx=w.init_idx, centroids=C)


def assert_index_equal(gi, oi):
    np.testing.assert_array_equal(gi.export(caps.ARR_CENTROIDS), oi.C)
    np.testing.assert_array_equal(gi.export(caps.ARR_BIN), oi.bin)
    np.testing.assert_array_equal(gi.export(caps.ARR_TAGS), oi.tags)
    np.testing.assert_array_equal(gi.export(caps.ARR_KEY), oi.key)
    np.testing.assert_array_equal(gi.export(caps.ARR_PERM), oi.perm)
    np.testing.assert_array_equal(gi.export(caps.ARR_OFFSETS), oi.offsets)


# ------------------------------------------------------ a2: assignment ----

@pytest.mark.parametrize("N,d,B,metric,kind", [
    (10_000, 32, 16, 0, "small"),
    (1000, 33, 70, 0, "float"),      # ragged: N, d, B off every tile size
    (777, 8, 5, 1, "float"),         # inner product
    (5000, 4, 40, 0, "ties"),        # tiny integers: many exact ties
    (63, 128, 1, 0, "float"),        # fewer rows than one tile, one centroid
    (4100, 130, 129, 1, "float"),
])
def test_assign_bit_exact(N, d, B, metric, kind):
    rng = np.random.default_rng(N + d + B)
    if kind == "small":
        X = config_small().X
    elif kind == "ties":
        X = rng.integers(0, 3, (N, d)).astype(np.float32)
    else:
        X = rng.standard_normal((N, d)).astype(np.float32)
    C = X[rng.choice(N, B, replace=False)].copy()
    if kind == "ties":
        C[: B // 2] = C[B // 2: 2 * (B // 2)]  # duplicate centroids: ties
    want = O.assign(X, C, metric)
    got = caps.assign(dev(X), dev(C), metric, out=torch.empty(N, dtype=torch.int32, device="cuda"))
    np.testing.assert_array_equal(got.cpu().numpy(), want)
    got_h = caps.assign(X, C, metric)  # host buffers through the same entry point
    np.testing.assert_array_equal(got_h, want)


# ------------------------------------------- a1-a4: the whole index build ----

def test_build_small_config_bit_exact():
    w = config_small()
    assert_index_equal(gpu_index(w), oracle_index(w))


@pytest.mark.parametrize("h", [0, 1, 4, 15, 63])
def test_build_tree_heights(h):
    w = tiny(3 + h, h=h)
    assert_index_equal(gpu_index(w), oracle_index(w))


def test_build_integer_data_ip_and_host_buffers():
    w = tiny(11, integer=True, d=16, N=3000, B=20, h=7)
    assert_index_equal(gpu_index(w, on_device=False), oracle_index(w))
    wi = tiny(12, normalize=True, metric=1, d=24, N=2000, B=9, h=3)
    assert_index_equal(gpu_index(wi), oracle_index(wi))


def test_build_fixed_centroids_and_zero_iterations():
    w = tiny(21, N=2500, B=11, h=6)
    oi = oracle_index(w)
    assert_index_equal(gpu_index(w, C=oi.C), O.build(w.X, O.Attrs.of(w), w.B, w.h, 0,
                                                      w.init_idx, C=oi.C))
    assert_index_equal(gpu_index(w, iters=0), oracle_index(w, iters=0))


def test_build_empty_partitions_and_single_partition():
    # duplicate seed points leave partitions empty; B = 1 puts every point
    # into one partition
    w = tiny(31, N=500, B=6, h=4)
    w.X[w.init_idx[1]] = w.X[w.init_idx[0]]
    assert_index_equal(gpu_index(w), oracle_index(w))
    w1 = tiny(32, N=400, B=1, h=9)
    assert_index_equal(gpu_index(w1), oracle_index(w1))


# --------------------------------------------------- a5, a6: probe, select ----

@pytest.mark.parametrize("m", [1, 4, 16])
def test_probe_and_select_bit_exact(m):
    w = config_small()
    oi = oracle_index(w)
    gi = gpu_index(w)
    P = gi.probe(w.Q, m)
    np.testing.assert_array_equal(P, O.probe(w.Q, oi.C, m))
    Pd = gi.probe(dev(w.Q), m, out=torch.empty((w.nq, m), dtype=torch.int32, device="cuda"))
    np.testing.assert_array_equal(Pd.cpu().numpy(), P)
    S = gi.select(P, w.Qb)
    np.testing.assert_array_equal(S, O.select(oi.tags, w.h, O.Attrs.of(w), P, O.Cons.of(w)))


def test_select_exhaustive_constraints_tiny_vocab():
    w = tiny(41, N=600, vocab=(3, 3, 2), B=4, h=5)
    oi = oracle_index(w)
    gi = gpu_index(w)
    import itertools
    allb = np.array(list(itertools.product(*[range(-1, V) for V in (3, 3, 2)])), np.int32)
    P = np.tile(np.arange(w.B, dtype=np.int32), (len(allb), 1))
    np.testing.assert_array_equal(gi.select(P, allb),
                                  O.select(oi.tags, w.h, O.Attrs.of(w), P, O.Cons(Qb=allb)))


# ------------------------------------------------- a7: masked scan + top-k ----

def _oracle_search(w, oi, k, m, Qb=None):
    Qb = w.Qb if Qb is None else Qb
    return O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons(Qb=Qb), k, m)


def _check_valid(w, ids, Qb):
    for q in range(ids.shape[0]):
        for i in ids[q][ids[q] >= 0]:
            b = Qb[q]
            assert np.all((b < 0) | (w.A[i] == b)), "returned id violates the filter"


@pytest.mark.parametrize("k,m", [(10, 4), (1, 2), (33, 5), (100, 16), (128, 16)])
def test_search_small_config(k, m):
    w = config_small()
    oi = oracle_index(w)
    gi = gpu_index(w)
    ids, dist = gi.search(dev(w.Q), dev(w.Qb), k, m)
    ids, dist = ids.cpu().numpy(), dist.cpu().numpy()
    oids, odist, _, _ = _oracle_search(w, oi, k, m)
    assert_search_equal(ids, dist, oids, odist, X=w.X, Q=w.Q, A=w.A, Qb=w.Qb)
    _check_valid(w, ids, w.Qb)


@pytest.mark.parametrize("d,k,m", [(128, 10, 5), (96, 7, 3), (256, 40, 9), (64, 128, 20),
                                   (33, 10, 5)])
def test_search_byte_data_exact(d, k, m):
    # byte-valued data: every partial sum is an exact integer, so any
    # summation order gives the oracle's distances and ids exactly.  d = 33
    # takes the query-major scan, the others the partition-major one.
    w = tiny(60 + d, N=6000, d=d, B=24, h=9, integer=True, nq=67, vocab=(5, 7, 11))
    oi = oracle_index(w)
    gi = gpu_index(w)
    ids, dist = gi.search(dev(w.Q), dev(w.Qb), k, m)
    oids, odist, _, _ = _oracle_search(w, oi, k, m)
    assert_search_equal(ids.cpu().numpy(), dist.cpu().numpy(), oids, odist, exact=True)


def test_search_many_probes_per_partition_and_hub_partitions():
    # more than 32 probes of one partition -> several work items per
    # partition; skewed partition sizes from a few dominant components
    w = make_dense_workload(name="hub", N=20_000, d=32, ncomp=3, center=("uniform", 128.0),
                            sigma=16.0, vocab=[4, 6, 8], zipf_s=1.0, nq=300, cmin=1, cmax=3,
                            B=12, h=6, iters=5, m=4, k=10, seed=71, integer=True)
    oi = oracle_index(w)
    gi = gpu_index(w)
    ids, dist = gi.search(w.Q, w.Qb, 10, 6)
    oids, odist, _, _ = _oracle_search(w, oi, 10, 6)
    assert_search_equal(ids, dist, oids, odist, exact=True)


def test_search_host_buffers_equal_device_buffers():
    w = config_small()
    gi = gpu_index(w, on_device=False)
    ih, dh = gi.search(w.Q, w.Qb, 10, 4)
    idv, ddv = gi.search(dev(w.Q), dev(w.Qb), 10, 4)
    np.testing.assert_array_equal(ih, idv.cpu().numpy())
    np.testing.assert_array_equal(dh, ddv.cpu().numpy())


def test_search_probe_all_is_exact_filtered_knn():
    # m = B: every valid point is visited -> exact filtered kNN (Def. 2)
    w = tiny(51, N=3000, d=16, B=9, h=6, integer=True, nq=41)
    gi = gpu_index(w)
    ids, dist = gi.search(w.Q, w.Qb, 10, w.B)
    gt, g32, _, cnt = O.bruteforce(w.X, O.Attrs.of(w), w.Q, O.Cons.of(w), 10, order64=False)
    np.testing.assert_array_equal(ids, gt)
    np.testing.assert_array_equal(dist, g32)


def test_search_h0_and_unconstrained():
    w = tiny(52, N=2000, d=32, B=8, h=0, nq=30)
    oi = oracle_index(w)
    gi = gpu_index(w)
    for Qb in (w.Qb, np.full_like(w.Qb, -1)):
        ids, dist = gi.search(w.Q, Qb, 10, 3)
        oids, odist, _, _ = _oracle_search(w, oi, 10, 3, Qb)
        assert_search_equal(ids, dist, oids, odist, X=w.X, Q=w.Q, A=w.A, Qb=Qb)


def test_search_inner_product():
    w = tiny(53, N=2000, d=64, B=8, h=5, nq=30, metric=1, normalize=True)
    oi = oracle_index(w)
    gi = gpu_index(w)
    ids, dist = gi.search(w.Q, w.Qb, 10, 3)
    oids, odist, _, _ = _oracle_search(w, oi, 10, 3)
    assert_search_equal(ids, dist, oids, odist, X=w.X, Q=w.Q, A=w.A, Qb=w.Qb, metric=1)
    assert np.all(np.diff(dist, axis=1)[np.isfinite(dist[:, 1:])] <= 0)


def test_search_padding_dead_values_and_empty_batch():
    w = tiny(54, N=500, B=5, h=4, nq=9)
    gi = gpu_index(w)
    Qb = w.Qb.copy()
    Qb[0] = [0, 0, 0]            # possibly rare: may need padding
    Qb[1, 2] = w.vocab[2]        # value outside the vocabulary: no point can match
    Qb[2, 0] = 10_000
    ids, dist = gi.search(w.Q, Qb, 50, 2)
    oi = oracle_index(w)
    oids, odist, _, _ = _oracle_search(w, oi, 50, 2, Qb)
    assert_search_equal(ids, dist, oids, odist, X=w.X, Q=w.Q, A=w.A, Qb=Qb)
    assert (ids[1] == -1).all() and np.isinf(dist[1]).all()
    assert (ids[2] == -1).all()
    e_ids, e_dist = gi.search(w.Q[:0], Qb[:0], 10, 2)
    assert e_ids.shape == (0, 10)


def test_search_rejects_bad_arguments():
    w = tiny(55, N=300, B=4, h=2, nq=3)
    gi = gpu_index(w)
    for k, m in ((0, 1), (129, 1), (10, 0), (10, 5)):
        with pytest.raises(caps.CapsError) as e:
            gi.search(w.Q, w.Qb, k, m)
        assert e.value.code == caps.CAPS_EINVAL
    with pytest.raises(caps.CapsError):
        gi.search(w.Q, w.Qb[:, :2].copy(), 10, 1)  # wrong field count
    bad = w.A.copy()
    bad[3, 1] = w.vocab[1]
    with pytest.raises(caps.CapsError) as e:
        caps.Index.build(w.X, bad, w.vocab, w.B, h=2, iters=1, init_idx=w.init_idx)
    assert e.value.code == caps.CAPS_EINVAL
    with pytest.raises(caps.CapsError):
        caps.Index.build(w.X, w.A, w.vocab, w.B, h=2, iters=1,
                         init_idx=np.array([0, 0, 1, 2]))  # repeated seed


def test_recall_rises_with_probes_and_reaches_one():
    w = config_small()
    gi = gpu_index(w)
    gt, _, g64, cnt = O.bruteforce(w.X, O.Attrs.of(w), w.Q, O.Cons.of(w), 10)
    rec = []
    for m in (1, 4, 16):
        ids, _ = gi.search(w.Q, w.Qb, 10, m)
        rec.append(O.recall(ids, gt, g64, cnt, 10, X=w.X, Q=w.Q)[1])
    assert rec[0] <= rec[1] <= rec[2] and rec[2] == 1.0


@pytest.mark.parametrize("m", [33, 100, 150, 200])
def test_probe_wide_m_both_selection_kernels(m):
    # m <= 128 takes the warp running-top-m kernel, m > 128 the bitonic one
    w = tiny(81, N=4000, d=16, B=200, h=3, integer=True, nq=25)
    oi = oracle_index(w, iters=2)
    gi = gpu_index(w, iters=2)
    np.testing.assert_array_equal(gi.probe(w.Q, m), O.probe(w.Q, oi.C, m))
