"""Seeded synthetic workloads for CAPS (arXiv 2308.15014).

The paper evaluates on SIFT/Glove/GIST/... with attributes generated at
random (Sec. 6, "Datasets"): L=3 categorical fields per point, skewed value
frequencies (power law, Sec. 6.2), queries carrying a variable number of AND
constraints (Sec. 6.1, "absence fraction").  None of those datasets is used
here; these generators stand in for them by shape and distribution only.

Everything returned is plain numpy.  Nothing here computes a distance, a
partition, an attribute-frequency tree or a search result.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Workload:
    """One filtered-search problem instance (Def. 1-2 of the paper).

    Dense attributes: ``A`` is ``[N, L]`` int32 with ``0 <= A[:, f] < vocab[f]``;
    query constraints ``Qb`` are ``[nq, L]`` int32 with -1 meaning the field is
    unconstrained (variable constraints, Sec. 6.1).

    Sparse attributes: ``sp_off``/``sp_lab`` hold each point's sorted label set
    in CSR form; ``q_off``/``q_lab`` hold each query's required labels (the
    query filter is "every required label is present").
    """

    name: str
    X: np.ndarray                      # [N, d] float32
    Q: np.ndarray                      # [nq, d] float32
    metric: int                        # 0 = L2, 1 = inner product
    B: int                             # first-level partitions
    h: int                             # attribute-frequency-tree height
    iters: int                         # k-means iterations
    m: int                             # partitions probed per query
    k: int                             # neighbours returned
    init_idx: np.ndarray               # [B] int64, k-means seed points
    A: Optional[np.ndarray] = None     # [N, L] int32 (dense)
    vocab: Optional[np.ndarray] = None  # [L] int32 (dense)
    Qb: Optional[np.ndarray] = None    # [nq, L] int32 (dense, -1 = any)
    sp_off: Optional[np.ndarray] = None  # [N+1] int64 (sparse)
    sp_lab: Optional[np.ndarray] = None  # [nnz] int32 (sparse, sorted per point)
    sp_vocab: int = 0
    q_off: Optional[np.ndarray] = None   # [nq+1] int64 (sparse)
    q_lab: Optional[np.ndarray] = None   # [nnzq] int32
    selectivity: Optional[np.ndarray] = None  # [nq] |D_C| / N
    recipe: str = ""

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def d(self) -> int:
        return int(self.X.shape[1])

    @property
    def nq(self) -> int:
        return int(self.Q.shape[0])

    @property
    def dense(self) -> bool:
        return self.A is not None


def zipf_probs(V: int, s: float) -> np.ndarray:
    """Bounded Zipf law P(v) proportional to (v+1)^-s for v = 0..V-1."""
    p = (np.arange(V, dtype=np.float64) + 1.0) ** (-float(s))
    return p / p.sum()


def _mixture(rng, n, centers, sigma):
    comp = rng.integers(0, centers.shape[0], size=n)
    X = centers[comp].astype(np.float64)
    X += sigma * rng.standard_normal((n, centers.shape[1]))
    return X


def _dense_attrs(rng, n, vocab, s):
    A = np.empty((n, len(vocab)), dtype=np.int32)
    for f, V in enumerate(vocab):
        A[:, f] = rng.choice(V, size=n, p=zipf_probs(V, s))
    return A


class _DenseCounter:
    """|D_C| for dense conjunctive constraints, via per-field-subset counts."""

    def __init__(self, A: np.ndarray, vocab):
        self.A = A.astype(np.int64)
        self.radix = np.array(vocab, dtype=np.int64)
        self.cache = {}

    def count(self, b: np.ndarray) -> int:
        fields = tuple(int(f) for f in np.nonzero(b >= 0)[0])
        if not fields:
            return self.A.shape[0]
        if fields not in self.cache:
            key = np.zeros(self.A.shape[0], dtype=np.int64)
            for f in fields:
                key = key * self.radix[f] + self.A[:, f]
            u, c = np.unique(key, return_counts=True)
            self.cache[fields] = (u, c)
        u, c = self.cache[fields]
        kq = 0
        for f in fields:
            kq = kq * int(self.radix[f]) + int(b[f])
        i = np.searchsorted(u, kq)
        return int(c[i]) if i < len(u) and u[i] == kq else 0


def _dense_constraints(rng, A, vocab, nq, cmin, cmax, sel_range):
    """Each query copies 1..L fields' values from a random data point, so its
    filter is never empty; optionally rejection-sampled into a selectivity
    range."""
    N, L = A.shape
    counter = _DenseCounter(A, vocab)
    Qb = np.full((nq, L), -1, dtype=np.int32)
    sel = np.empty(nq, dtype=np.float64)
    for qi in range(nq):
        for _attempt in range(10000):
            src = int(rng.integers(0, N))
            c = int(rng.integers(cmin, cmax + 1))
            fields = rng.choice(L, size=c, replace=False)
            b = np.full(L, -1, dtype=np.int32)
            b[fields] = A[src, fields]
            s = counter.count(b) / N
            if sel_range is None or (sel_range[0] <= s <= sel_range[1]):
                break
        Qb[qi] = b
        sel[qi] = s
    return Qb, sel


def make_dense_workload(
    *, name, N, d, ncomp, center, sigma, vocab, zipf_s, nq, cmin, cmax,
    B, h, iters, m, k, seed, sel_range=None, integer=False, normalize=False,
    metric=0, recipe="",
) -> Workload:
    """Gaussian-mixture vectors with dense categorical attributes.

    ``center`` is ("normal", scale) -> centers ~ N(0, scale^2 I), or
    ("uniform", hi) -> centers ~ U[0, hi)^d.  ``integer`` clips to [0, 255]
    and rounds (SIFT-like byte vectors stored as fp32).  ``normalize`` scales
    every vector to unit L2 norm.  Seeds: data ``seed``, queries
    ``seed + 1000``, k-means seed points ``seed + 2000``.
    """
    rng = np.random.default_rng(seed)
    kind, scale = center
    if kind == "normal":
        centers = scale * rng.standard_normal((ncomp, d))
    elif kind == "uniform":
        centers = rng.uniform(0.0, scale, size=(ncomp, d))
    else:
        raise ValueError(kind)
    X = _mixture(rng, N, centers, sigma)
    A = _dense_attrs(rng, N, vocab, zipf_s)
    rq = np.random.default_rng(seed + 1000)
    Q = _mixture(rq, nq, centers, sigma)
    if integer:
        X = np.rint(np.clip(X, 0.0, 255.0))
        Q = np.rint(np.clip(Q, 0.0, 255.0))
    if normalize:
        X /= np.linalg.norm(X, axis=1, keepdims=True)
        Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    Qb, sel = _dense_constraints(rq, A, vocab, nq, cmin, cmax, sel_range)
    ri = np.random.default_rng(seed + 2000)
    init_idx = ri.permutation(N)[:B].astype(np.int64)
    return Workload(
        name=name, X=np.ascontiguousarray(X, dtype=np.float32),
        Q=np.ascontiguousarray(Q, dtype=np.float32), metric=metric, B=B, h=h,
        iters=iters, m=m, k=k, init_idx=init_idx, A=A,
        vocab=np.asarray(vocab, dtype=np.int32), Qb=Qb, selectivity=sel,
        recipe=recipe)


def with_constraints(w: Workload, cmin: int, cmax: int, seed: int, sel_range=None,
                     name: str = "") -> Workload:
    """The same vectors, attributes and query vectors with new query
    constraints: each copies cmin..cmax fields from a random data point
    (cmin = cmax fixes the absence fraction (L - c) / L, Sec. 6.1),
    rejection-sampled into sel_range when given."""
    rq = np.random.default_rng(seed)
    Qb, sel = _dense_constraints(rq, w.A, w.vocab, w.nq, cmin, cmax, sel_range)
    return dataclasses.replace(w, Qb=Qb, selectivity=sel, name=name or w.name,
                               recipe=w.recipe + f"; constraints re-drawn: {cmin}-{cmax} copied "
                                                 f"fields (seed {seed})")


def _sparse_labels(rng, N, V, zipf_s, nmax, exponent):
    """1..nmax labels per point, count law P(n) ~ n^-exponent, labels drawn
    without replacement from a bounded Zipf law over V labels."""
    pn = np.arange(1, nmax + 1, dtype=np.float64) ** (-exponent)
    pn /= pn.sum()
    cnt = rng.choice(np.arange(1, nmax + 1), size=N, p=pn)
    draws = rng.choice(V, size=(N, 4 * nmax), p=zipf_probs(V, zipf_s))
    rows = []
    for i in range(N):
        _, first = np.unique(draws[i], return_index=True)
        uniq = draws[i][np.sort(first)]
        while len(uniq) < cnt[i]:
            extra = rng.choice(V, size=4 * nmax, p=zipf_probs(V, zipf_s))
            allv = np.concatenate([uniq, extra])
            _, first = np.unique(allv, return_index=True)
            uniq = allv[np.sort(first)]
        rows.append(np.sort(uniq[: cnt[i]]))
    off = np.zeros(N + 1, dtype=np.int64)
    off[1:] = np.cumsum(cnt)
    lab = np.concatenate(rows).astype(np.int32)
    return off, lab


def make_sparse_workload(
    *, name, N, d, ncomp, center, sigma, V, zipf_s, nmax, exponent, nq,
    cmin, cmax, B, h, iters, m, k, seed, sel_range=None, recipe="",
) -> Workload:
    """Gaussian-mixture vectors with sparse multi-hot label sets (Table 1,
    "sparse attributes"); each query requires 1..cmax labels copied from a
    random data point."""
    rng = np.random.default_rng(seed)
    kind, scale = center
    centers = (scale * rng.standard_normal((ncomp, d)) if kind == "normal"
               else rng.uniform(0.0, scale, size=(ncomp, d)))
    X = _mixture(rng, N, centers, sigma)
    sp_off, sp_lab = _sparse_labels(rng, N, V, zipf_s, nmax, exponent)
    # inverted lists for selectivity
    owner = np.repeat(np.arange(N, dtype=np.int64), np.diff(sp_off))
    order = np.argsort(sp_lab, kind="stable")
    lab_sorted = sp_lab[order]
    inv_start = np.searchsorted(lab_sorted, np.arange(V + 1))
    inv_pts = owner[order]
    rq = np.random.default_rng(seed + 1000)
    Q = _mixture(rq, nq, centers, sigma)
    q_rows, sel = [], np.empty(nq)
    for qi in range(nq):
        for _attempt in range(10000):
            src = int(rq.integers(0, N))
            labs = sp_lab[sp_off[src]:sp_off[src + 1]]
            c = min(int(rq.integers(cmin, cmax + 1)), len(labs))
            req = np.sort(rq.choice(labs, size=c, replace=False))
            pts = inv_pts[inv_start[req[0]]:inv_start[req[0] + 1]]
            for lbl in req[1:]:
                pts = np.intersect1d(pts, inv_pts[inv_start[lbl]:inv_start[lbl + 1]],
                                     assume_unique=True)
            s = len(pts) / N
            if sel_range is None or (sel_range[0] <= s <= sel_range[1]):
                break
        q_rows.append(req.astype(np.int32))
        sel[qi] = s
    q_off = np.zeros(nq + 1, dtype=np.int64)
    q_off[1:] = np.cumsum([len(r) for r in q_rows])
    ri = np.random.default_rng(seed + 2000)
    init_idx = ri.permutation(N)[:B].astype(np.int64)
    return Workload(
        name=name, X=np.ascontiguousarray(X, dtype=np.float32),
        Q=np.ascontiguousarray(Q, dtype=np.float32), metric=0, B=B, h=h,
        iters=iters, m=m, k=k, init_idx=init_idx, sp_off=sp_off, sp_lab=sp_lab,
        sp_vocab=V, q_off=q_off, q_lab=np.concatenate(q_rows), selectivity=sel,
        recipe=recipe)


def config_small(seed: int = 1001, **over) -> Workload:
    """10,000 x 32 fp32, 16-component mixture (centers N(0, 4I), unit-variance
    clusters), 3 fields with vocab 8/16/32 Zipf s=1.0, k-means B=16 (20
    iterations), probe 4, 200 queries with 1-3 copied constraints, k=10, L2."""
    kw = dict(name="small_10k_d32", N=10_000, d=32, ncomp=16, center=("normal", 2.0),
              sigma=1.0, vocab=[8, 16, 32], zipf_s=1.0, nq=200, cmin=1, cmax=3,
              B=16, h=15, iters=20, m=4, k=10, seed=seed,
              recipe="mixture 16 comps, centers N(0,4I), sigma 1; Zipf(1.0) fields 8/16/32; "
                     "queries from the mixture, 1-3 constraints copied from a random point")
    kw.update(over)
    return make_dense_workload(**kw)


def config_sift1m_like(seed: int = 1002, **over) -> Workload:
    """1,000,000 x 128 byte-valued vectors stored as fp32 (1000-component
    mixture, centers U[0,128)^d, sigma 16, clipped to [0,255], rounded), 3
    fields vocab 20/50/100 Zipf s=1.0, B=1024, h=15, 10,000 queries with 1-3
    constraints rejection-sampled into selectivity [0.1%, 30%], k=10, L2."""
    kw = dict(name="sift1m_like_1M_d128", N=1_000_000, d=128, ncomp=1000,
              center=("uniform", 128.0), sigma=16.0, vocab=[20, 50, 100], zipf_s=1.0,
              nq=10_000, cmin=1, cmax=3, B=1024, h=15, iters=20, m=32, k=10, seed=seed,
              sel_range=(0.001, 0.30), integer=True,
              recipe="mixture 1000 comps, centers U[0,128)^128, sigma 16, clip [0,255], round; "
                     "Zipf(1.0) fields 20/50/100; 1-3 copied constraints, selectivity in [0.1%,30%]")
    kw.update(over)
    return make_dense_workload(**kw)


def config_sift1m_fields(L: int, seed: int = 1002, **over) -> Workload:
    """The 1M x 128 byte-valued vectors of config_sift1m_like with L
    attribute fields (vocab 20/50/100 repeating, Zipf s=1.0); queries copy
    1-3 fields from a random point, selectivity in [0.1%, 30%], so longer
    attribute vectors leave more fields free (the paper's appendix varies the
    attribute length L)."""
    vocab = [(20, 50, 100)[f % 3] for f in range(L)]
    kw = dict(name=f"sift1m_like_1M_d128_L{L}", N=1_000_000, d=128, ncomp=1000,
              center=("uniform", 128.0), sigma=16.0, vocab=vocab, zipf_s=1.0,
              nq=10_000, cmin=1, cmax=min(3, L), B=1024, h=15, iters=20, m=32, k=10, seed=seed,
              sel_range=(0.001, 0.30), integer=True,
              recipe=f"as sift1m_like with {L} fields vocab 20/50/100 repeating, 1-3 copied "
                     "constraints, selectivity in [0.1%,30%]")
    kw.update(over)
    return make_dense_workload(**kw)


def config_sift1m_wide(L: int = 100, nq: int = 1000, p_field: float = 0.03,
                       seed: int = 1002, base: Optional[Workload] = None) -> Workload:
    """The 1M x 128 vectors and first nq queries of config_sift1m_like with L
    attribute fields (vocab 20/50/100 repeating, Zipf s=1.0) held as label
    sets: field f with value v is label f * 100 + v (every point carries L
    labels).  Each query keeps each field of a random data point with
    probability p_field (at least one), as in the paper's appendix (0.03 for
    L = 100), rejection-sampled into selectivity [0.1%, 30%]; a field
    constraint is then the requirement of that label.  base: the
    config_sift1m_like workload of the same seed, whose vectors are reused
    (they are the same draws); attributes and constraints come from seeds
    seed + 3000 and seed + 4000 either way."""
    N, d, ncomp = 1_000_000, 128, 1000
    if base is not None:
        assert base.N == N and base.d == d and base.nq >= nq
        X, Q = base.X, base.Q[:nq]
    else:
        rng = np.random.default_rng(seed)
        centers = rng.uniform(0.0, 128.0, size=(ncomp, d))
        X = np.rint(np.clip(_mixture(rng, N, centers, 16.0), 0.0, 255.0))
        rq = np.random.default_rng(seed + 1000)  # (the 10,000 queries of the base workload)
        Q = np.rint(np.clip(_mixture(rq, 10_000, centers, 16.0), 0.0, 255.0))[:nq]
    vocab = [(20, 50, 100)[f % 3] for f in range(L)]
    A = _dense_attrs(np.random.default_rng(seed + 3000), N, vocab, 1.0)
    lab = (np.arange(L, dtype=np.int64)[None, :] * 100 + A).astype(np.int32)
    sp_off = np.arange(N + 1, dtype=np.int64) * L
    AT = np.ascontiguousarray(A.T.astype(np.uint8))  # field-major, for the selectivity counts
    rq = np.random.default_rng(seed + 4000)
    # counts per (field, value) pair, and the points of each, for selectivity
    rows, sel = [], np.empty(nq)
    for qi in range(nq):
        for _attempt in range(10000):
            src = int(rq.integers(0, N))
            keep = np.nonzero(rq.random(L) < p_field)[0]
            if len(keep) == 0:
                keep = np.array([int(rq.integers(0, L))])
            ok = np.ones(N, dtype=bool)
            for f in keep:
                ok &= AT[f] == AT[f, src]
            s = float(ok.sum()) / N
            if 0.001 <= s <= 0.30:
                break
        rows.append(np.sort(lab[src, keep]).astype(np.int32))
        sel[qi] = s
    q_off = np.zeros(nq + 1, dtype=np.int64)
    q_off[1:] = np.cumsum([len(r) for r in rows])
    ri = np.random.default_rng(seed + 2000)
    init_idx = ri.permutation(N)[:1024].astype(np.int64)
    return Workload(
        name=f"sift1m_like_1M_d128_L{L}_labels", X=np.ascontiguousarray(X, dtype=np.float32),
        Q=np.ascontiguousarray(Q, dtype=np.float32), metric=0, B=1024, h=15, iters=20, m=32, k=10,
        init_idx=init_idx, sp_off=sp_off, sp_lab=np.ascontiguousarray(lab.ravel()),
        sp_vocab=100 * L, q_off=q_off, q_lab=np.concatenate(rows).astype(np.int32),
        selectivity=sel,
        recipe=f"sift1m_like vectors; {L} fields vocab 20/50/100 Zipf(1.0) as labels f*100+v; "
               f"queries keep each field of a random point with p={p_field}, selectivity "
               "[0.1%,30%]")


def config_learned4m(seed: int = 1004, **over) -> Workload:
    """4,000,000 x 96 unit-norm vectors (4000 components, centers N(0, I),
    sigma 0.3 before normalisation), inner product, 5 fields vocab
    10/30/100/300/1000 Zipf s=1.1, B=1024, 10,000 queries with 1-5 constraints
    copied from a random point, rejection-sampled into selectivity [0.1%, 30%]
    as in the 1M x 128 workload (without it, half of the queries match fewer
    than 100 points and their neighbours lie in arbitrary partitions)."""
    kw = dict(name="learned_4M_d96_ip", N=4_000_000, d=96, ncomp=4000,
              center=("normal", 1.0), sigma=0.3, vocab=[10, 30, 100, 300, 1000],
              zipf_s=1.1, nq=10_000, cmin=1, cmax=5, B=1024, h=15, iters=20, m=32,
              k=10, seed=seed, normalize=True, metric=1, sel_range=(0.001, 0.30),
              recipe="mixture 4000 comps, centers N(0,I), sigma 0.3, L2-normalised; "
                     "Zipf(1.1) fields 10/30/100/300/1000; 1-5 copied constraints, "
                     "selectivity in [0.1%,30%]")
    kw.update(over)
    return make_dense_workload(**kw)


def config_sparse2m(seed: int = 1005, **over) -> Workload:
    """2,000,000 x 128 fp32 (mixture as the 1M config, not rounded), multi-hot
    labels from a 10,000-label vocabulary, 1-20 labels per point (P(n) ~
    n^-1.5), queries requiring 1-8 labels copied from a random point with
    selectivity in [0.01%, 50%]."""
    kw = dict(name="sparse_2M_d128", N=2_000_000, d=128, ncomp=1000,
              center=("uniform", 128.0), sigma=16.0, V=10_000, zipf_s=1.0, nmax=20,
              exponent=1.5, nq=4096, cmin=1, cmax=8, B=1024, h=15, iters=20, m=32,
              k=10, seed=seed, sel_range=(0.0001, 0.5),
              recipe="mixture 1000 comps, centers U[0,128)^128, sigma 16; labels: count "
                     "P(n)~n^-1.5 on 1..20, Zipf(1.0) over 10,000 without replacement")
    kw.update(over)
    return make_sparse_workload(**kw)


CONFIGS = {
    "small": config_small,
    "sift1m": config_sift1m_like,
    "sift1m_fields": config_sift1m_fields,
    "learned4m": config_learned4m,
    "sparse2m": config_sparse2m,
}
