"""Pins for the oracle's learned partitioner (Sec. 5.2): gradients against
central finite differences, closed forms of the loss and of Adam's first
step, and the fp32 fixed-order argmax against the fp64 forward."""
import numpy as np

import oracle as O


def _net(rng, d, H, B, scale=0.3):
    return O.MLP(scale * rng.standard_normal((H, d)), 0.1 * rng.standard_normal(H),
                 scale * rng.standard_normal((B, H)), 0.1 * rng.standard_normal(B))


def test_loss_closed_forms():
    rng = np.random.default_rng(1)
    d, H, B = 3, 4, 5
    X = rng.standard_normal((6, d)).astype(np.float32)
    zero = O.MLP(np.zeros((H, d)), np.zeros(H), np.zeros((B, H)), np.zeros(B))
    Y = np.eye(B, dtype=np.float32)[rng.integers(0, B, 6)]
    loss, g = O.mlp_loss_grad(X, Y, zero)
    # all logits equal: p = 1/B, loss = log B; dL/db2 = mean(p - y)
    assert abs(loss - np.log(B)) < 1e-12
    np.testing.assert_allclose(g.b2, (1.0 / B - Y.astype(np.float64)).mean(0), atol=1e-12)
    np.testing.assert_array_equal(g.W1, 0.0)  # relu(0) = 0 blocks the first layer


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    d, H, B, n = 5, 7, 6, 9
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = rng.random((n, B)).astype(np.float32)
    Y /= Y.sum(1, keepdims=True)
    net = _net(rng, d, H, B)
    loss, g = O.mlp_loss_grad(X, Y, net)
    eps = 1e-6
    for name in ("W1", "b1", "W2", "b2"):
        P = getattr(net, name)
        G = getattr(g, name)
        for idx in list(np.ndindex(P.shape))[:: max(1, P.size // 12)]:
            old = P[idx]
            P[idx] = old + eps
            lp, _ = O.mlp_loss_grad(X, Y, net)
            P[idx] = old - eps
            lm, _ = O.mlp_loss_grad(X, Y, net)
            P[idx] = old
            num = (lp - lm) / (2 * eps)
            assert abs(num - G[idx]) <= 1e-6 * max(1.0, abs(num)), (name, idx, num, G[idx])


def test_adam_first_step_is_lr_times_sign():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    m = np.zeros(3)
    v = np.zeros(3)
    O.adam(w, g, m, v, lr=0.01, t=1, eps=1e-12)
    # bias-corrected first moment g and second moment g^2 -> step lr*sign(g)
    np.testing.assert_allclose(w, [1.0 - 0.01, -2.0 + 0.01, 0.5 - 0.01], rtol=1e-9)


def test_fp32_assign_matches_fp64_argmax_when_separated():
    rng = np.random.default_rng(3)
    d, H, B = 8, 16, 10
    X = rng.standard_normal((200, d)).astype(np.float32)
    net = _net(rng, d, H, B, scale=1.0)
    Z, _ = O.mlp_forward64(X, net)
    srt = np.sort(Z, 1)
    clear = (srt[:, -1] - srt[:, -2]) > 1e-3
    got = O.mlp_assign32(X, net)
    np.testing.assert_array_equal(got[clear], Z.argmax(1)[clear])
    Z32 = O.mlp_logits32(X, net)
    np.testing.assert_allclose(Z32, Z, rtol=1e-4, atol=1e-4)


def test_training_reduces_loss_and_labels_are_distributions():
    from workloads import make_dense_workload
    w = make_dense_workload(name="mlp", N=1500, d=8, ncomp=5, center=("normal", 3.0), sigma=1.0,
                            vocab=[3, 4], zipf_s=1.0, nq=5, cmin=1, cmax=2, B=5, h=2, iters=5, m=2,
                            k=5, seed=9)
    at = O.Attrs.of(w)
    C, bins = O.kmeans(w.X, w.B, w.iters, w.init_idx)
    rng = np.random.default_rng(4)
    samples = rng.choice(w.N, 120, replace=False)
    cons = np.where(rng.random((120, 2)) < 0.5, w.A[samples], -1).astype(np.int32)
    Y = O.mlp_labels(w.X, at, bins, samples, cons, w.B, k=5)
    np.testing.assert_allclose(Y.sum(1), 1.0, rtol=1e-6)
    # a sample's neighbours share its constraint: check one label by hand
    s0 = int(samples[0])
    ok = np.all((cons[0] < 0) | (w.A == cons[0]), axis=1)
    ok[s0] = False
    cand = np.nonzero(ok)[0]
    dd = ((w.X[cand].astype(np.float64) - w.X[s0]) ** 2).sum(1)
    nb = cand[np.lexsort((cand, dd))[:5]]
    want = np.bincount(bins[nb], minlength=w.B) / len(nb)
    np.testing.assert_allclose(Y[0], want, rtol=1e-6)
    net = _net(np.random.default_rng(5), 8, 16, w.B, scale=0.3)
    _, losses = O.mlp_train(w.X[samples], Y, net, epochs=30, batch=40, lr=1e-2)
    assert losses[-1] < 0.7 * losses[0]


def _bias_only_net(d, H, b2, rng):
    """W1 = 0 and b1 = 0 make every hidden unit relu(0) = 0, so each row's
    logits are b2 whatever x is and no gradient reaches W1, b1 or W2."""
    B = len(b2)
    return O.MLP(np.zeros((H, d)), np.zeros(H), rng.standard_normal((B, H)),
                 np.asarray(b2, np.float64))


def test_train_minibatches_cover_every_row_in_order():
    """mlp_train's loss list, checked against the closed form of the
    cross-entropy with constant logits: with lr = 0 nothing moves, so step s
    reports mean over its rows r of sum_c Y[r,c] (logsumexp(b2) - b2[c]).
    n = 5, batch = 2: three minibatches per epoch ([0,1], [2,3], [4]), the
    last one partial; the second epoch follows a given permutation.  A
    dropped tail batch, a padded one, or minibatches cut from the rows in
    storage order instead of the epoch's order all change the list."""
    rng = np.random.default_rng(31)
    d, H = 3, 4
    b2 = np.array([0.0, 1.0, 2.5, -1.0])
    net = _bias_only_net(d, H, b2, rng)
    n, batch = 5, 2
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = rng.random((n, len(b2))).astype(np.float32)
    Y /= Y.sum(1, keepdims=True)
    order = [np.arange(n), np.array([3, 0, 4, 1, 2])]
    _, losses = O.mlp_train(X, Y, net, epochs=2, batch=batch, lr=0.0, order=order)
    lse = np.log(np.exp(b2).sum())
    Y64 = Y.astype(np.float64)
    row_ce = lse * Y64.sum(1) - Y64 @ b2
    want = []
    for e in range(2):
        for b0 in range(0, n, batch):
            want.append(row_ce[order[e][b0:b0 + batch]].mean())
    assert len(losses) == 6
    np.testing.assert_allclose(losses, want, rtol=1e-12, atol=1e-12)


def test_train_adam_step_counter_runs_across_epochs():
    """Adam with a constant gradient g moves every step by exactly
    lr * g / (|g| + eps): the bias-corrected moments are g and g^2 only when
    the step counter t equals the number of steps taken so far.  A softmax
    saturated far from its one-hot target (b2 = (0, 100, 0), every label on
    class 0) has d loss / d b2 = p - y = (-1, +1, ~e^-100) on every row of
    every minibatch, so after T steps b2[0] = T * lr / (1 + eps) and
    b2[1] = 100 - T * lr / (1 + eps).  n = 5 rows in batches of 2 for 2
    epochs is T = 6 steps; a counter restarted each epoch would make the
    fourth step about 1.72 lr, a dropped partial batch would give T = 4."""
    rng = np.random.default_rng(32)
    d, H = 2, 3
    net = _bias_only_net(d, H, [0.0, 100.0, 0.0], rng)
    n, batch, lr, eps = 5, 2, 0.01, 1e-8
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = np.zeros((n, 3), np.float32)
    Y[:, 0] = 1.0
    w, losses = O.mlp_train(X, Y, net, epochs=2, batch=batch, lr=lr)
    T = 6
    assert len(losses) == T
    step = lr / (1.0 + eps)
    assert abs(w.b2[0] - T * step) < 1e-12
    assert abs(w.b2[1] - (100.0 - T * step)) < 1e-12
    assert abs(w.b2[2]) < 1e-12
    np.testing.assert_array_equal(w.W1, 0.0)
    np.testing.assert_array_equal(w.b1, 0.0)
    np.testing.assert_array_equal(w.W2, net.W2)


def test_balanced_assign_hand_worked():
    """Three partitions, candidates best first; loads start at zero.
    p0 (2,0): both empty, the first -> 2 (loads 0,0,1); p1 (2,1): 1 has less
    -> 1 (0,1,1); p2 (2,1): tie at 1 -> the first, 2 (0,1,2); p3 (0,2): 0
    -> 0 (1,1,2); p4 (2,0,1): 0 and 1 tie at 1, 0 comes first among them ->
    0 (2,1,2); p5 (1,2,0): 1 (2,2,2)."""
    top = [[2, 0, -1], [2, 1, -1], [2, 1, -1], [0, 2, -1], [2, 0, 1], [1, 2, 0]]
    # rows of R = 3 (the -1 entries are never chosen: rows 0-3 list 2 real
    # candidates and a third equal to their first)
    top = np.array([[r[0], r[1], r[2] if r[2] >= 0 else r[0]] for r in top], np.int32)
    np.testing.assert_array_equal(O.balanced_assign(top, 3), [2, 1, 2, 0, 0, 1])
    # with loads already in place: partition 2 full, partition 1 next
    np.testing.assert_array_equal(O.balanced_assign(top[:2], 3, load0=[5, 0, 9]), [0, 1])


def test_balanced_assign_special_cases():
    rng = np.random.default_rng(33)
    n, B = 997, 13
    scores = rng.standard_normal((n, B))
    top = np.argsort(-scores, axis=1, kind="stable").astype(np.int32)
    # R = 1: the best partition of every point
    np.testing.assert_array_equal(O.balanced_assign(top[:, :1], B), top[:, 0])
    # R = B: every partition is a candidate, so the loads end within one
    bins = O.balanced_assign(top, B)
    load = np.bincount(bins, minlength=B)
    assert load.max() - load.min() <= 1
    # every point lands in one of its candidates, and a larger R never
    # leaves a larger largest load on this input
    for R in (2, 4):
        b = O.balanced_assign(top[:, :R], B)
        assert all(b[i] in top[i, :R] for i in range(n))
    assert np.bincount(O.balanced_assign(top[:, :4], B), minlength=B).max() <= \
        np.bincount(top[:, 0], minlength=B).max()


def _bf16_by_bits(v32):
    """fp32 -> bf16 by the bit pattern: add 0x7fff plus the lowest kept bit
    to the 32-bit word and clear the low 16 bits (round to nearest, ties to
    even), an independent way to the same rounding."""
    u = np.asarray(v32, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_rounding_matches_the_bit_rule():
    rng = np.random.default_rng(50)
    v = (rng.standard_normal(4000) * np.exp2(rng.integers(-20, 20, 4000))).astype(np.float32)
    # exact halfway cases between neighbouring bf16 values: ties go to even
    half = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 3 * (1 + 2.0 ** -8),
                     1 + 2.0 ** -8 + 2.0 ** -20], np.float32)
    v = np.concatenate([v, half, np.float32([0.0, 1.0, -2.5, 65504.0])])
    np.testing.assert_array_equal(O.round_bf16(v), _bf16_by_bits(v))
    assert O.round_bf16([1 + 2.0 ** -8])[0] == 1.0
    assert O.round_bf16([1 + 3 * 2.0 ** -8])[0] == 1 + 2.0 ** -6


def _dyadic_net(rng, d, H, B):
    """Weights on a coarse dyadic grid: every product and sum of the forward
    pass below is exact in bf16 and fp64 alike."""
    q = lambda shape, s: (rng.integers(-4, 5, shape) * s).astype(np.float64)
    return O.MLP(q((H, d), 0.125), q(H, 0.125), q((B, H), 0.0625), q(B, 0.25))


def test_bf16_step_equals_fp64_forward_when_operands_are_representable():
    # x in {-2..2}/2, weights on 1/8 and 1/16 grids: h and z are exact, so the
    # loss and the bias gradient of the output layer (unrounded dz) are the
    # fp64 step's, bit for bit; the other gradients use bf16(dz) and differ
    rng = np.random.default_rng(51)
    d, H, B, n = 5, 6, 7, 9
    net = _dyadic_net(rng, d, H, B)
    X = (rng.integers(-2, 3, (n, d)) * 0.5).astype(np.float32)
    Y = np.eye(B, dtype=np.float32)[rng.integers(0, B, n)]
    l64, g64 = O.mlp_loss_grad(X, Y, net)
    l16, g16 = O.mlp_loss_grad(X, Y, net, bf16=True)
    assert l16 == l64
    np.testing.assert_array_equal(g16.b2, g64.b2)


def test_bf16_step_exact_when_dz_is_representable():
    # W2 = 0, b2 = 0 and B = 4: p = 1/4 for every row, one-hot labels and
    # n = 2 give dz in {1/8, -3/8} (exact in bf16); h is exact (dyadic x and
    # W1), so gW2 = dz^T h equals the fp64 step's, and dh = W2^T dz = 0
    rng = np.random.default_rng(52)
    d, H, B, n = 3, 5, 4, 2
    net = _dyadic_net(rng, d, H, B)
    net.W2[:] = 0.0
    net.b2[:] = 0.0
    X = (rng.integers(-2, 3, (n, d)) * 0.5).astype(np.float32)
    Y = np.eye(B, dtype=np.float32)[[1, 3]]
    l64, g64 = O.mlp_loss_grad(X, Y, net)
    l16, g16 = O.mlp_loss_grad(X, Y, net, bf16=True)
    assert l16 == l64 == np.log(4.0)
    np.testing.assert_array_equal(g16.W2, g64.W2)
    assert np.abs(g64.W2).max() > 0
    np.testing.assert_array_equal(g16.W1, 0.0)
    np.testing.assert_array_equal(g16.b1, 0.0)


def test_bf16_step_within_the_rounding_error_of_fp64():
    # every product operand carries a relative error of at most 2^-9, and a
    # gradient entry goes through at most four such roundings on each path
    # (x, W1 -> h -> bf16(h); z -> dz -> bf16(dz); W2; bf16(dh)): about 1 %
    # first-order per term; in norm over a whole gradient the bf16 step stays
    # within 3 % of the fp64 one, while a transposed operand, a wrong sign or
    # a dropped term lands at O(100 %)
    rng = np.random.default_rng(53)
    d, H, B, n = 16, 24, 11, 64
    net = _net(rng, d, H, B, scale=0.5)
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = rng.random((n, B)).astype(np.float32)
    Y /= Y.sum(1, keepdims=True)
    l64, g64 = O.mlp_loss_grad(X, Y, net)
    l16, g16 = O.mlp_loss_grad(X, Y, net, bf16=True)
    assert abs(l16 - l64) <= 0.01 * abs(l64)
    for name in ("W1", "b1", "W2", "b2"):
        a, b = getattr(g16, name), getattr(g64, name)
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert 0.0 < rel < 0.03, (name, rel)


def test_bf16_training_on_a_bias_only_net_is_the_fp64_training():
    # W1 = 0, b1 = 0: every hidden unit is relu(0) = 0, so bf16(h) = 0, the
    # W2 gradient and dh vanish and only the unrounded bias gradient moves;
    # the bf16 training's trajectory is then the fp64 one exactly
    rng = np.random.default_rng(54)
    d, H = 3, 4
    net = _bias_only_net(d, H, [0.0, 1.0, 2.5, -1.0], rng)
    X = rng.standard_normal((5, d)).astype(np.float32)
    Y = rng.random((5, 4)).astype(np.float32)
    Y /= Y.sum(1, keepdims=True)
    w64, l64 = O.mlp_train(X, Y, net, epochs=2, batch=2, lr=0.05)
    w16, l16 = O.mlp_train(X, Y, net, epochs=2, batch=2, lr=0.05, bf16=True)
    assert l16 == l64
    for a, b in ((w16.W1, w64.W1), (w16.b1, w64.b1), (w16.W2, w64.W2), (w16.b2, w64.b2)):
        np.testing.assert_array_equal(a, b)
    assert np.abs(w64.b2 - net.b2).max() > 0.05


def test_bf16_step_rounds_the_backward_operands():
    # one row, W1 = 0 and b1 = e_u: h = e_u exactly, so z = bf16(W2)[:, u] + b2
    # (the loss is the fp64 loss of the net with W2 rounded), the W2 gradient's
    # column u is bf16(dz) while the b2 gradient is dz itself, and with a
    # one-hot x = e_j the W1 gradient's column j is bf16(dh) while the b1
    # gradient is dh itself
    rng = np.random.default_rng(55)
    d, H, B, u, j = 4, 6, 9, 2, 1
    net = O.MLP(np.zeros((H, d)), np.zeros(H), rng.standard_normal((B, H)), rng.standard_normal(B))
    net.b1[u] = 1.0
    X = np.zeros((1, d), np.float32)
    X[0, j] = 1.0
    Y = rng.random((1, B)).astype(np.float32)
    Y /= Y.sum()
    l16, g16 = O.mlp_loss_grad(X, Y, net, bf16=True)
    rounded = O.MLP(net.W1, net.b1, O.round_bf16(net.W2), net.b2)
    l64, _ = O.mlp_loss_grad(X, Y, rounded)
    assert l16 == l64
    assert (O.round_bf16(g16.b2) != g16.b2).any()  # dz unrounded in the bias gradient
    np.testing.assert_array_equal(g16.W2[:, u], O.round_bf16(g16.b2))
    np.testing.assert_array_equal(np.delete(g16.W2, u, axis=1), 0.0)
    assert O.round_bf16(g16.b1)[u] != g16.b1[u]
    np.testing.assert_array_equal(g16.W1[:, j], O.round_bf16(g16.b1))
    np.testing.assert_array_equal(np.delete(g16.W1, j, axis=1), 0.0)
    np.testing.assert_array_equal(np.delete(g16.b1, u), 0.0)


def test_bf16_step_rounds_the_inputs_and_activations():
    # one row x in [1, 2), W1 = I, b1 = 2^-12 (below half a bf16 step of 1):
    # h = bf16(x) + 2^-12 and bf16(h) = bf16(x).  With W2, b2 on a dyadic
    # grid the bf16 step's loss is the fp64 loss of the rounded row with
    # b1 = 0 (not that of the row itself); the W2 gradient is
    # bf16(dz) bf16(x)^T and the W1 gradient bf16(dh) bf16(x)^T, with dz and
    # dh the (unrounded) bias gradients
    rng = np.random.default_rng(56)
    d = H = 6
    B = 5
    net = _dyadic_net(rng, d, H, B)
    net.W1[:] = np.eye(H)
    net.b1[:] = 2.0 ** -12
    X = (1.0 + rng.random((1, d))).astype(np.float32)
    Xr = O.round_bf16(X)
    assert (Xr != X).all()
    Y = np.eye(B, dtype=np.float32)[[3]]
    l16, g16 = O.mlp_loss_grad(X, Y, net, bf16=True)
    plain = O.MLP(net.W1, np.zeros(H), net.W2, net.b2)
    lr_, _ = O.mlp_loss_grad(Xr.astype(np.float32), Y, plain)
    lx, _ = O.mlp_loss_grad(X, Y, plain)
    assert l16 == lr_ and l16 != lx
    np.testing.assert_array_equal(g16.W2, np.outer(O.round_bf16(g16.b2), Xr[0]))
    np.testing.assert_array_equal(g16.W1, np.outer(O.round_bf16(g16.b1), Xr[0]))


def test_bf16_step_only_sees_the_rounded_rows_and_weights():
    # rounding is idempotent: the bf16 step of a net and rows equals, bit for
    # bit, the bf16 step of the same net with W1 and W2 rounded beforehand
    # and of the rounded rows -- and differs from the fp64 step.  A product
    # operand left unrounded makes the two disagree.
    rng = np.random.default_rng(57)
    d, H, B, n = 6, 9, 7, 12
    net = _net(rng, d, H, B, scale=0.7)
    X = rng.standard_normal((n, d)).astype(np.float32)
    Y = rng.random((n, B)).astype(np.float32)
    Y /= Y.sum(1, keepdims=True)
    l16, g16 = O.mlp_loss_grad(X, Y, net, bf16=True)
    pre = O.MLP(O.round_bf16(net.W1), net.b1, O.round_bf16(net.W2), net.b2)
    lp, gp = O.mlp_loss_grad(O.round_bf16(X).astype(np.float32), Y, pre, bf16=True)
    assert l16 == lp
    for name in ("W1", "b1", "W2", "b2"):
        np.testing.assert_array_equal(getattr(g16, name), getattr(gp, name))
    for name in ("W1", "W2"):  # the pre-rounding did change the weights
        assert (getattr(pre, name) != getattr(net, name)).any()
    l64, _ = O.mlp_loss_grad(X, Y, net)
    assert l16 != l64
