"""The probe set screened on the tensor cores against the CPU oracle's top-m.

Alg. 2 probes the m partitions with the best fp32 scores, ties to the lower
partition.  For m <= 64 the GPU bounds every partition's score by a split-bf16
tensor-core product, puts partitions whose interval lies above the m-th
largest upper bound straight into the set, and re-scores exactly (same
fixed-order fp32 chain as the oracle) only those whose interval straddles the
boundary.  The set must therefore equal the oracle's exactly, exact ties at
the m-th score included, for L2 and IP centroids and for the learned
partitioner's logits.  caps_search_batch uses the same routine, so these are
also the probe sets of every batched search with m <= 64.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2308_15014_gb300 import build
    build.build()


import paper_2308_15014_gb300 as caps  # noqa: E402


def centroid_index(X, C, metric):
    N = X.shape[0]
    A = (np.arange(N) % 4).astype(np.int32).reshape(N, 1)
    return caps.Index.build(X, A, [4], C.shape[0], h=3, iters=0, metric=metric, centroids=C)


def assert_same_sets(P, R, B):
    assert P.shape == R.shape
    assert ((P >= 0) & (P < B)).all()
    Ps = np.sort(P, axis=1)
    assert (np.diff(Ps, axis=1) > 0).all(), "a partition appears twice in one probe set"
    np.testing.assert_array_equal(Ps, np.sort(R, axis=1))


def gaussian_case(seed, N, d, B, nq, scale=1.0):
    rng = np.random.default_rng(seed)
    X = (scale * rng.standard_normal((N, d))).astype(np.float32)
    C = np.ascontiguousarray(X[rng.choice(N, B, replace=False)]
                             + (0.1 * scale * rng.standard_normal((B, d))).astype(np.float32))
    Q = (scale * rng.standard_normal((nq, d))).astype(np.float32)
    return X, C, Q


@pytest.mark.parametrize("metric", [caps.L2, caps.IP])
@pytest.mark.parametrize("m", [1, 13, 40, 64])
def test_centroid_probe_set_equals_oracle(metric, m):
    # 700 queries: five full 128-query tiles and a ragged one; B = 300: one
    # full 256-partition tile and a ragged one
    X, C, Q = gaussian_case(300 + m + 7 * metric, N=3000, d=128, B=300, nq=700)
    gi = centroid_index(X, C, metric)
    assert_same_sets(gi.probe_set(Q, m), O.probe(Q, C, m, metric), 300)


@pytest.mark.parametrize("d", [13, 100])
def test_probe_set_ragged_width(d):
    # width not a multiple of 64 (zero padding of the split operands) and, for
    # d = 13, not a multiple of 4 (unaligned feature rows)
    X, C, Q = gaussian_case(310 + d, N=2000, d=d, B=96, nq=300)
    gi = centroid_index(X, C, caps.L2)
    for m in (1, 17, 64):
        assert_same_sets(gi.probe_set(Q, m), O.probe(Q, C, m), 96)


def test_probe_set_large_magnitude():
    # scores around 1e9: the error intervals scale with the norms
    X, C, Q = gaussian_case(320, N=2000, d=128, B=256, nq=400, scale=3000.0)
    for metric in (caps.L2, caps.IP):
        gi = centroid_index(X, C, metric)
        assert_same_sets(gi.probe_set(Q, 40), O.probe(Q, C, 40, metric), 256)


@pytest.mark.parametrize("metric", [caps.L2, caps.IP])
def test_probe_set_exact_ties_go_to_lower_partition(metric):
    # every centroid twice, small-integer coordinates, queries from the same
    # grid: exact ties at the m-th score everywhere, and the oracle's rule
    # (lower partition first) decides which duplicates are in the set
    rng = np.random.default_rng(330 + metric)
    d, B = 16, 128
    base = rng.integers(0, 3, (B // 2, d)).astype(np.float32)
    C = np.ascontiguousarray(np.concatenate([base, base])[rng.permutation(B)])
    X = rng.integers(0, 3, (1500, d)).astype(np.float32)
    Q = rng.integers(0, 3, (500, d)).astype(np.float32)
    gi = centroid_index(X, C, metric)
    for m in (1, 5, 31, 64):
        assert_same_sets(gi.probe_set(Q, m), O.probe(Q, C, m, metric), B)


def test_probe_set_all_scores_equal():
    # identical centroids: every interval straddles the boundary, the list of
    # uncertain partitions overflows and every partition is re-scored; the
    # lowest m partitions win the tie
    rng = np.random.default_rng(340)
    d, B = 32, 512
    C = np.ascontiguousarray(np.repeat(rng.standard_normal((1, d)).astype(np.float32), B, 0))
    X = rng.standard_normal((1000, d)).astype(np.float32)
    Q = rng.standard_normal((200, d)).astype(np.float32)
    gi = centroid_index(X, C, caps.L2)
    for m in (1, 40, 64):
        P = gi.probe_set(Q, m)
        assert_same_sets(P, np.tile(np.arange(m, dtype=np.int32), (200, 1)), B)


def test_probe_set_m_equals_b_and_beyond_screen():
    X, C, Q = gaussian_case(350, N=1500, d=32, B=48, nq=300)
    gi = centroid_index(X, C, caps.L2)
    assert_same_sets(gi.probe_set(Q, 48), O.probe(Q, C, 48), 48)  # every partition
    X, C, Q = gaussian_case(351, N=3000, d=32, B=200, nq=300)
    gi = centroid_index(X, C, caps.L2)
    # m > 64 takes the plain exact top-m: same set, best first
    np.testing.assert_array_equal(gi.probe_set(Q, 80), O.probe(Q, C, 80))
    with pytest.raises(caps.CapsError):
        gi.probe_set(Q, 201)


def rand_net(rng, d, H, B, scale):
    return O.MLP((scale * rng.standard_normal((H, d))).astype(np.float32),
                 (0.1 * rng.standard_normal(H)).astype(np.float32),
                 (scale * rng.standard_normal((B, H))).astype(np.float32),
                 (0.1 * rng.standard_normal(B)).astype(np.float32))


@pytest.mark.parametrize("H,B", [(512, 1024), (72, 200)])
def test_learned_probe_set_equals_oracle(H, B):
    # the logits of a 128 -> H -> B network (the bench's shape, and a ragged
    # one): hidden units from the fixed-order forward pass, then screened
    rng = np.random.default_rng(360 + H)
    N, d, nq = 3000, 128, 600
    X = rng.standard_normal((N, d)).astype(np.float32)
    Q = rng.standard_normal((nq, d)).astype(np.float32)
    net = rand_net(rng, d, H, B, scale=0.1)
    A = (np.arange(N) % 4).astype(np.int32).reshape(N, 1)
    S = 64
    samp = rng.choice(N, S, replace=False)
    gi = caps.Index.build(X, A, [4], B, h=3, iters=0, part=caps.MLP, mlp_hidden=H,
                          mlp_epochs=0, mlp_init=caps.mlp_flat(net.W1, net.b1, net.W2, net.b2),
                          mlp_samples=S, mlp_sample_idx=samp,
                          mlp_sample_cons=A[samp].astype(np.int32))
    for m in (1, 20, 64):
        assert_same_sets(gi.probe_set(Q, m), O.probe_logits(Q, net, m), B)
