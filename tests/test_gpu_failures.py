"""Failure detection without a GPU fault: the library's error paths are
driven from the host and each one must leave the library usable.

Out of device memory: the allocation gate fails the n-th device allocation
as cudaMalloc would on a full device (the allocator is not called).  Each
entry point that allocates -- index build, batched query (its stream-ordered
scratch), query plan -- must then return CAPS_ENOMEM and release what it
took, and the very next call on the same index must answer exactly as the
oracle does.
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


def _w():
    # byte-valued rows: every distance is an exact integer, results are
    # the oracle's bit for bit whatever the summation order
    return make_dense_workload(name="fail", N=6000, d=64, ncomp=10, center=("uniform", 128.0),
                               sigma=16.0, vocab=[4, 8, 16], zipf_s=1.0, nq=200, cmin=1, cmax=3,
                               B=16, h=7, iters=3, m=4, k=10, seed=404, integer=True)


def _build(w, prec):
    return caps.Index.build(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.A).cuda(), w.vocab,
                            w.B, h=w.h, iters=w.iters, init_idx=w.init_idx, prec=prec)


def _oracle(w, ix):
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, C=ix.export(caps.ARR_CENTROIDS))
    return O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons(Qb=w.Qb), w.k, w.m)[:2]


@pytest.mark.parametrize("prec", [0, 1])
def test_build_out_of_memory_then_build(prec):
    w = _w()
    for n in (1, 3, 7):
        caps.inject_alloc_failure(n)
        with pytest.raises(caps.CapsError) as e:
            _build(w, prec)
        assert e.value.code == caps.CAPS_ENOMEM
    caps.inject_alloc_failure(0)
    ix = _build(w, prec)
    ids, dist = ix.search(torch.from_numpy(w.Q).cuda(), torch.from_numpy(w.Qb).cuda(), w.k, w.m)
    oids, odist = _oracle(w, ix)
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_array_equal(dist.cpu().numpy(), odist)
    ix.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_search_out_of_memory_then_exact(prec):
    w = _w()
    ix = _build(w, prec)
    Q, Qb = torch.from_numpy(w.Q).cuda(), torch.from_numpy(w.Qb).cuda()
    oids, odist = _oracle(w, ix)
    for n in (1, 2, 5):
        caps.inject_alloc_failure(n)
        with pytest.raises(caps.CapsError) as e:
            ix.search(Q, Qb, w.k, w.m)
        assert e.value.code == caps.CAPS_ENOMEM
        caps.inject_alloc_failure(0)
        ids, dist = ix.search(Q, Qb, w.k, w.m)
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)
        np.testing.assert_array_equal(dist.cpu().numpy(), odist)
    # a plan whose buffers cannot be allocated, then one that can
    caps.inject_alloc_failure(1)
    with pytest.raises(caps.CapsError) as e:
        ix.plan(Q, Qb, w.k, w.m, autotune=False)
    assert e.value.code == caps.CAPS_ENOMEM
    caps.inject_alloc_failure(0)
    plan = ix.plan(Q, Qb, w.k, w.m, autotune=False)
    ids = torch.empty((w.nq, w.k), dtype=torch.int64, device="cuda")
    dist = torch.empty((w.nq, w.k), dtype=torch.float32, device="cuda")
    plan.search(Q, Qb, out_ids=ids, out_dist=dist)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(ids.cpu().numpy(), oids)
    np.testing.assert_array_equal(dist.cpu().numpy(), odist)
    plan.close()
    ix.close()


def test_alloc_count_moves_with_allocations():
    n0 = caps.alloc_count()
    w = _w()
    ix = _build(w, 0)
    assert caps.alloc_count() > n0
    ix.close()


@pytest.mark.parametrize("pen_bits_fit", [True, False])
def test_scan_bounded_wait_expires_then_exact(pen_bits_fit):
    """A wait that nothing completes: the tensor-core scan's producer is told
    (test hook) to issue no copy and no MMA for work item 0, so the
    epilogue's bounded wait for that item's first tile runs out (2 ms here);
    the kernel stops with nothing in flight and the search reports
    CAPS_ETIMEOUT.  The next search on the same index answers exactly.
    Queries without constraints select every block, so item 0 has tiles.
    pen_bits_fit False: 7 fields of vocab 100 (49 packed bits) leave no room
    for the penalty chunk, so the per-pair filter form of the scan runs."""
    vocab = [4, 8, 16] if pen_bits_fit else [100] * 7
    w = make_dense_workload(name="stall", N=6000, d=64, ncomp=10, center=("uniform", 128.0),
                            sigma=16.0, vocab=vocab, zipf_s=1.0, nq=200, cmin=1, cmax=3,
                            B=16, h=7, iters=3, m=4, k=10, seed=405, integer=True)
    ix = _build(w, caps.BF16)
    Q = torch.from_numpy(w.Q).cuda()
    free = np.full_like(w.Qb, -1)
    Qb = torch.from_numpy(free).cuda()
    oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, C=ix.export(caps.ARR_CENTROIDS))
    oids, odist, _, _ = O.search(w.X, O.Attrs.of(w), oi, w.Q, O.Cons(Qb=free), w.k, w.m)
    ids = torch.empty((w.nq, w.k), dtype=torch.int64, device="cuda")
    dist = torch.empty((w.nq, w.k), dtype=torch.float32, device="cuda")
    caps.scan_stall_hook(0, 2_000_000)
    try:
        ix.search(Q, Qb, w.k, w.m, out_ids=ids, out_dist=dist)  # device outputs: enqueued only
        with pytest.raises(caps.CapsError) as e:
            ix.status()
        assert e.value.code == caps.CAPS_ETIMEOUT
    finally:
        caps.scan_stall_hook(-1)
    ix.status()  # reported once, then clear
    for _ in range(2):
        ix.search(Q, Qb, w.k, w.m, out_ids=ids, out_dist=dist)
        ix.status()
        np.testing.assert_array_equal(ids.cpu().numpy(), oids)
        np.testing.assert_array_equal(dist.cpu().numpy(), odist)
    ix.close()
