"""caps_search_batch_noalloc, the batched query for callers that cannot
allocate device memory (memory reserved up front by another framework, a
serving loop that must not wait on the allocator, rules that forbid
allocator calls after start-up).  Its intermediates live in a fixed device
array inside the library instead of coming from an allocator.

The test calls it through the C ABI twice in a row -- the second call runs on
the array the first one left behind -- and checks both results against
caps_search_batch, with the same tolerance as the other GPU tests: distances
within 1e-5 relative, ids equal up to near-ties (the two entry points may sum
a distance in a different order).
This file sorts last so that a run stopping at the first failure has already
run every other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from _compare import assert_search_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def caps():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2308_15014_gb300 import build
    build.build()
    import paper_2308_15014_gb300 as c
    return c


def _workload(B, nq, d=32):
    from workloads import make_dense_workload
    return make_dense_workload(name="noalloc", N=30_000, d=d, ncomp=40, center=("normal", 2.0),
                               sigma=1.0, vocab=[6, 10, 20], zipf_s=1.0, nq=nq, cmin=1, cmax=3,
                               B=B, h=7, iters=4, m=8, k=10, seed=123)


@pytest.mark.parametrize("B,nq,k,m", [(16, 300, 10, 4), (2048, 5000, 20, 16)])
def test_noalloc_matches_search_batch_on_two_calls(caps, B, nq, k, m):
    # B = 2048 with 5,000 queries needs several passes over the 16 MiB array
    w = _workload(B, nq)
    ix = caps.Index.build(torch.from_numpy(w.X).cuda(), torch.from_numpy(w.A).cuda(), w.vocab,
                          w.B, h=w.h, iters=w.iters, init_idx=w.init_idx)
    Q = torch.from_numpy(w.Q).cuda()
    Qb = torch.from_numpy(w.Qb).cuda()
    ref_ids, ref_dist = ix.search(Q, Qb, k, m)
    for call in range(2):
        ids = torch.full((nq, k), -7, dtype=torch.int64, device="cuda")
        dist = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        n0 = caps.alloc_count()
        ix.search_noalloc(Q, Qb, k, m, ids, dist)
        torch.cuda.synchronize()
        # the property the entry point exists for: no device allocation
        assert caps.alloc_count() == n0, f"call {call} allocated device memory"
        assert_search_equal(ids.cpu().numpy(), dist.cpu().numpy(), ref_ids.cpu().numpy(),
                            ref_dist.cpu().numpy(), X=w.X, Q=w.Q, A=w.A, Qb=w.Qb)
    ix.close()


def test_noalloc_on_a_bf16_index_runs_the_exact_fp32_scan(caps):
    # a BF16 index keeps its fp32 rows; the no-allocation call scans those,
    # so it answers like caps_search_batch on an fp32 index of the same
    # partitions (k-means does not depend on the scan precision)
    nq, k, m = 400, 10, 6
    w = _workload(32, nq, d=64)
    X, A = torch.from_numpy(w.X).cuda(), torch.from_numpy(w.A).cuda()
    ix16 = caps.Index.build(X, A, w.vocab, w.B, h=w.h, iters=w.iters, init_idx=w.init_idx,
                            prec=caps.BF16)
    ix32 = caps.Index.build(X, A, w.vocab, w.B, h=w.h, iters=w.iters, init_idx=w.init_idx)
    Q = torch.from_numpy(w.Q).cuda()
    Qb = torch.from_numpy(w.Qb).cuda()
    ref_ids, ref_dist = ix32.search(Q, Qb, k, m)
    for _ in range(2):
        ids = torch.full((nq, k), -7, dtype=torch.int64, device="cuda")
        dist = torch.full((nq, k), -7.0, dtype=torch.float32, device="cuda")
        ix16.search_noalloc(Q, Qb, k, m, ids, dist)
        torch.cuda.synchronize()
        assert_search_equal(ids.cpu().numpy(), dist.cpu().numpy(), ref_ids.cpu().numpy(),
                            ref_dist.cpu().numpy(), X=w.X, Q=w.Q, A=w.A, Qb=w.Qb)
    ix16.close()
    ix32.close()


def test_noalloc_rejects_host_buffers(caps):
    w = _workload(16, 10)
    ix = caps.Index.build(w.X, w.A, w.vocab, w.B, h=w.h, iters=2, init_idx=w.init_idx)
    ids = torch.empty((10, 5), dtype=torch.int64, device="cuda")
    dist = torch.empty((10, 5), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError, match="CUDA"):
        ix.search_noalloc(torch.from_numpy(w.Q), torch.from_numpy(w.Qb), 5, 2, ids, dist)
    # the library refuses host memory on its own as well (the C ABI's check)
    from paper_2308_15014_gb300 import lib, _dense_attrs, _ptr
    import ctypes as ct
    Qh = np.ascontiguousarray(w.Q[:10])
    at, keep = _dense_attrs(torch.from_numpy(w.Qb[:10]).cuda())
    rc = lib().caps_search_batch_noalloc(ix._h, _ptr(Qh), 10, ct.byref(at), 5, 2, _ptr(ids),
                                         _ptr(dist), None)
    assert rc == caps.CAPS_EINVAL
    ix.close()
