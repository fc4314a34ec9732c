"""CPU oracle for CAPS (arXiv 2308.15014) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``caps_oracle.c`` (plain C,
compiled by ``oracle/build.py``) with numpy marshalling and adds the recall
metric of the paper's appendix ("Metric").  It shares nothing with the CUDA
library and never calls it.

Function map (paper passage -> function):
  Def. 1 query filter ............... filter_dense, filter_sparse
  distances (fp32 fixed order, fp64) dist32, dist64
  Alg. 1 first level (k-means) ...... kmeans, assign, centroid_update
  Alg. 1 second level (AFT) ......... aft
  contiguous sub-partition layout ... layout
  dynamic insertion (Table 1) ....... block_of, insert
  Alg. 2 top-m probe ................ probe
  Alg. 2 sub-partition selection .... select
  Alg. 2 full query ................. search
  Sec. 5.3 OR constraints ........... OrCons, select_or, search_or
  Def. 2 / appendix ground truth .... bruteforce
  appendix RecallK@K ................ recall
  Sec. 5.2 learned partitioner ...... mlp_forward64, mlp_loss_grad, adam,
                                      mlp_assign32, mlp_logits32, mlp_labels,
                                      mlp_train, probe_logits, balanced_assign
"""
from __future__ import annotations

import ctypes as ct
import dataclasses
from typing import Optional

import numpy as np

from .build import build_oracle

L2, IP = 0, 1

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build_oracle())
        P = ct.c_void_p
        i64, i32 = ct.c_int64, ct.c_int
        _lib.orc_filter_dense.argtypes = [P, P, i32]
        _lib.orc_filter_sparse.argtypes = [P, i64, P, i64]
        _lib.orc_dist32.argtypes = [P, P, i32, i32]
        _lib.orc_dist32.restype = ct.c_float
        _lib.orc_dist64.argtypes = [P, P, i32, i32]
        _lib.orc_dist64.restype = ct.c_double
        _lib.orc_assign.argtypes = [P, i64, i32, P, i32, i32, P]
        _lib.orc_centroid_update.argtypes = [P, i64, i32, P, i32, i32, P]
        _lib.orc_kmeans.argtypes = [P, i64, i32, i32, i32, P, i32, P, P]
        _lib.orc_aft.argtypes = [P, i64, i32, i32, i32, P, P, P, P, ct.c_int32, P, P]
        _lib.orc_layout.argtypes = [P, P, i64, i32, i32, P, P]
        _lib.orc_probe.argtypes = [P, i64, i32, P, i32, i32, i32, P]
        _lib.orc_select.argtypes = [P, i32, i32, P, ct.c_int32, P, i64, i32, P, P, P, P]
        _lib.orc_search.argtypes = [P, i64, i32, i32, P, P, P, P, ct.c_int32, P, i32, i32,
                                    P, i32, P, P, P, i64, P, P, P, i32, i32, P, P, P, P, P]
        _lib.orc_bruteforce.argtypes = [P, i64, i32, i32, P, P, P, P, ct.c_int32, P, i64,
                                        P, P, P, i32, i32, i32, P, P, P, P]
        _lib.orc_block_of.argtypes = [P, i32, i32, P, P, P, P, ct.c_int32, P, i64, P]
        _lib.orc_select_or.argtypes = [P, i32, i32, P, P, i64, i32, P, P, P]
        _lib.orc_search_or.argtypes = [P, i64, i32, i32, P, P, P, i32, i32, P, i32, P, P, P, i64,
                                       P, P, i32, i32, P, P, P]
        _lib.orc_set_threads.argtypes = [i32]
        _lib.orc_set_threads.restype = i32
        _lib.orc_mlp_forward64.argtypes = [P, i64, i32, i32, i32, P, P, P, P, P, P]
        _lib.orc_mlp_loss_grad.argtypes = [P, i64, i32, i32, i32, P, P, P, P, P, P, P, P, P]
        _lib.orc_mlp_loss_grad.restype = ct.c_double
        _lib.orc_mlp_loss_grad_bf16.argtypes = [P, i64, i32, i32, i32, P, P, P, P, P, P, P, P, P]
        _lib.orc_mlp_loss_grad_bf16.restype = ct.c_double
        _lib.orc_bf16.argtypes = [ct.c_double]
        _lib.orc_bf16.restype = ct.c_double
        _lib.orc_adam.argtypes = [P, P, P, P, i64, ct.c_double, ct.c_double, ct.c_double,
                                  ct.c_double, i32]
        _lib.orc_mlp_assign32.argtypes = [P, i64, i32, i32, i32, P, P, P, P, P]
        _lib.orc_mlp_logits32.argtypes = [P, i64, i32, i32, i32, P, P, P, P, P]
        _lib.orc_balanced_assign.argtypes = [P, i64, i32, i32, P, P]
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 keeps it); returns the count in use."""
    return lib().orc_set_threads(int(n))


@dataclasses.dataclass
class Attrs:
    """Data attributes: dense ``A [N,L]`` + ``vocab [L]``, or sparse CSR."""
    A: Optional[np.ndarray] = None
    vocab: Optional[np.ndarray] = None
    sp_off: Optional[np.ndarray] = None
    sp_lab: Optional[np.ndarray] = None
    sp_vocab: int = 0

    def __post_init__(self):
        self.A = _c(self.A, np.int32)
        self.vocab = _c(self.vocab, np.int32)
        self.sp_off = _c(self.sp_off, np.int64)
        self.sp_lab = _c(self.sp_lab, np.int32)

    @property
    def L(self) -> int:
        return 0 if self.A is None else int(self.A.shape[1])

    def args(self):
        return (self.L, _p(self.A), _p(self.vocab), _p(self.sp_off), _p(self.sp_lab),
                int(self.sp_vocab))

    @staticmethod
    def of(w) -> "Attrs":
        if w.A is not None:
            return Attrs(A=w.A, vocab=w.vocab)
        return Attrs(sp_off=w.sp_off, sp_lab=w.sp_lab, sp_vocab=w.sp_vocab)


@dataclasses.dataclass
class Cons:
    """Query constraints: dense ``Qb [nq,L]`` (-1 = unconstrained) or sparse CSR."""
    Qb: Optional[np.ndarray] = None
    q_off: Optional[np.ndarray] = None
    q_lab: Optional[np.ndarray] = None

    def __post_init__(self):
        self.Qb = _c(self.Qb, np.int32)
        self.q_off = _c(self.q_off, np.int64)
        self.q_lab = _c(self.q_lab, np.int32)

    def args(self):
        return (_p(self.Qb), _p(self.q_off), _p(self.q_lab))

    @staticmethod
    def of(w) -> "Cons":
        if w.Qb is not None:
            return Cons(Qb=w.Qb)
        return Cons(q_off=w.q_off, q_lab=w.q_lab)

    def subset(self, idx) -> "Cons":
        idx = np.asarray(idx)
        if self.Qb is not None:
            return Cons(Qb=self.Qb[idx])
        rows = [self.q_lab[self.q_off[i]:self.q_off[i + 1]] for i in idx]
        off = np.zeros(len(rows) + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(r) for r in rows])
        lab = np.concatenate(rows) if rows else np.zeros(0, np.int32)
        return Cons(q_off=off, q_lab=lab)


# ---- Def. 1 ---------------------------------------------------------------

def filter_dense(a, b) -> bool:
    a = _c(a, np.int32)
    b = _c(b, np.int32)
    return bool(lib().orc_filter_dense(_p(a), _p(b), len(a)))


def filter_sparse(a, b) -> bool:
    a = _c(a, np.int32)
    b = _c(b, np.int32)
    return bool(lib().orc_filter_sparse(_p(a), len(a), _p(b), len(b)))


# ---- distances ------------------------------------------------------------

def dist32(x, q, metric=L2) -> float:
    x = _c(x, np.float32)
    q = _c(q, np.float32)
    return float(lib().orc_dist32(_p(x), _p(q), len(x), metric))


def dist64(x, q, metric=L2) -> float:
    x = _c(x, np.float32)
    q = _c(q, np.float32)
    return float(lib().orc_dist64(_p(x), _p(q), len(x), metric))


# ---- Alg. 1 ---------------------------------------------------------------

def assign(X, C, metric=L2) -> np.ndarray:
    X = _c(X, np.float32)
    C = _c(C, np.float32)
    out = np.empty(X.shape[0], dtype=np.int32)
    lib().orc_assign(_p(X), X.shape[0], X.shape[1], _p(C), C.shape[0], metric, _p(out))
    return out


def centroid_update(X, bin, C, metric=L2) -> np.ndarray:
    X = _c(X, np.float32)
    bin = _c(bin, np.int32)
    C = np.array(C, dtype=np.float32, copy=True, order="C")
    lib().orc_centroid_update(_p(X), X.shape[0], X.shape[1], _p(bin), C.shape[0],
                              metric, _p(C))
    return C


def kmeans(X, B, iters, init_idx, metric=L2):
    X = _c(X, np.float32)
    init_idx = _c(init_idx, np.int64)
    C = np.empty((B, X.shape[1]), dtype=np.float32)
    bin = np.empty(X.shape[0], dtype=np.int32)
    lib().orc_kmeans(_p(X), X.shape[0], X.shape[1], B, iters, _p(init_idx), metric,
                     _p(C), _p(bin))
    return C, bin


def aft(bin, B, h, attrs: Attrs):
    bin = _c(bin, np.int32)
    N = len(bin)
    tags = np.empty((B, h), dtype=np.int32)
    key = np.zeros(N, dtype=np.uint8)
    lib().orc_aft(_p(bin), N, B, h, *attrs.args(), _p(tags), _p(key))
    return tags, key


def block_of(tags, h, attrs: Attrs, bins):
    """Block (1..h+1) of each point of `attrs` in its partition bins[i] under
    the fixed tags: the first block whose tag it carries, else h+1 (the
    insertion rule; for the built points it is the tree's own key)."""
    tags = _c(tags, np.int32)
    bins = _c(bins, np.int32)
    key = np.empty(len(bins), np.uint8)
    lib().orc_block_of(_p(tags), h, *attrs.args(), _p(bins), len(bins), _p(key))
    return key


def insert(index: Index, X_all, attrs_all: Attrs, n_new, metric=L2, bins_new=None) -> Index:
    """The index after inserting the last n_new points of X_all / attrs_all:
    their partitions f(x) (nearest centroid, or the given bins_new from a
    learned f), their blocks under the unchanged tags, and the layout by
    (partition, block, id) of all points.  Centroids and tags stay."""
    X_all = _c(X_all, np.float32)
    N = X_all.shape[0]
    n0 = N - n_new
    if bins_new is None:
        bins_new = assign(X_all[n0:], index.C, metric)
    bin_all = np.concatenate([np.asarray(index.bin, np.int32), np.asarray(bins_new, np.int32)])
    sub = Attrs(A=attrs_all.A[n0:], vocab=attrs_all.vocab) if attrs_all.A is not None else None
    assert sub is not None, "insertion serves dense attributes"
    key_new = block_of(index.tags, index.h, sub, bins_new)
    key_all = np.concatenate([np.asarray(index.key, np.uint8), key_new])
    perm, offsets = layout(bin_all, key_all, index.B, index.h)
    return Index(C=index.C, bin=bin_all, tags=index.tags, key=key_all, perm=perm,
                 offsets=offsets, B=index.B, h=index.h, metric=index.metric)


def layout(bin, key, B, h):
    bin = _c(bin, np.int32)
    key = _c(key, np.uint8)
    N = len(bin)
    perm = np.empty(N, dtype=np.int32)
    offsets = np.empty(B * (h + 1) + 1, dtype=np.int32)
    lib().orc_layout(_p(bin), _p(key), N, B, h, _p(perm), _p(offsets))
    return perm, offsets


# ---- Alg. 2 ---------------------------------------------------------------

def probe(Q, C, m, metric=L2) -> np.ndarray:
    Q = _c(Q, np.float32)
    C = _c(C, np.float32)
    out = np.empty((Q.shape[0], m), dtype=np.int32)
    lib().orc_probe(_p(Q), Q.shape[0], Q.shape[1], _p(C), C.shape[0], metric, m, _p(out))
    return out


def select(tags, h, attrs: Attrs, probe_bins, cons: Cons) -> np.ndarray:
    tags = _c(tags, np.int32)
    probe_bins = _c(probe_bins, np.int32)
    nq, m = probe_bins.shape
    out = np.empty((nq, m), dtype=np.uint64)
    lib().orc_select(_p(tags), h, attrs.L, _p(attrs.vocab), int(attrs.sp_vocab),
                     _p(probe_bins), nq, m, *cons.args(), _p(out))
    return out


@dataclasses.dataclass
class Index:
    """Oracle-built CAPS index (Alg. 1)."""
    C: np.ndarray
    bin: np.ndarray
    tags: np.ndarray
    key: np.ndarray
    perm: np.ndarray
    offsets: np.ndarray
    B: int
    h: int
    metric: int


def build(X, attrs: Attrs, B, h, iters, init_idx, metric=L2, C=None, bins=None) -> Index:
    """Alg. 1: k-means first level (or given centroids, or given partitions
    `bins` from a learned f), AFT, layout."""
    if bins is not None:
        C = np.zeros((B, np.asarray(X).shape[1]), np.float32) if C is None else _c(C, np.float32)
        bin = _c(bins, np.int32)
    elif C is None:
        C, bin = kmeans(X, B, iters, init_idx, metric)
    else:
        C = _c(C, np.float32)
        bin = assign(X, C, metric)
    tags, key = aft(bin, B, h, attrs)
    perm, offsets = layout(bin, key, B, h)
    return Index(C=C, bin=bin, tags=tags, key=key, perm=perm, offsets=offsets, B=B, h=h,
                 metric=metric)


def search(X, attrs: Attrs, index: Index, Q, cons: Cons, k, m, probe_in=None):
    """Alg. 2 for every query: returns ids [nq,k] (original ids, -1 pad),
    fp32 distances [nq,k], rows attribute-tested and rows matched per query.
    probe_in [nq,m] (optional): the partitions to probe (e.g. from a learned
    f(q)); by default the m nearest centroids."""
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.float32)
    n_scan = np.empty(nq, dtype=np.int64)
    n_match = np.empty(nq, dtype=np.int64)
    C = _c(index.C, np.float32)
    tags = _c(index.tags, np.int32)
    perm = _c(index.perm, np.int32)
    offsets = _c(index.offsets, np.int32)
    lib().orc_search(_p(X), X.shape[0], X.shape[1], *attrs.args(), _p(C), index.B,
                     index.metric, _p(tags), index.h, _p(perm), _p(offsets), _p(Q), nq,
                     *cons.args(), k, m, _p(ids), _p(dist), _p(n_scan), _p(n_match),
                     _p(_c(probe_in, np.int32)))
    return ids, dist, n_scan, n_match


# ---- Sec. 5.3: disjunctive constraints ---------------------------------------

@dataclasses.dataclass
class OrCons:
    """Per-(query, field) allowed values: field f of query q allows
    ``vals[voff[q*L+f]:voff[q*L+f+1]]``; an empty list leaves it free."""
    voff: np.ndarray
    vals: np.ndarray

    def __post_init__(self):
        self.voff = _c(self.voff, np.int64)
        self.vals = _c(self.vals, np.int32)

    @staticmethod
    def of_lists(lists):
        """lists[q][f] = list of allowed values (empty = free)."""
        L = len(lists[0]) if len(lists) else 0
        voff = [0]
        vals = []
        for row in lists:
            assert len(row) == L
            for f in range(L):
                vals.extend(int(v) for v in row[f])
                voff.append(len(vals))
        return OrCons(np.asarray(voff, np.int64), np.asarray(vals, np.int32))


def select_or(tags, h, attrs: Attrs, probe_bins, oc: OrCons) -> np.ndarray:
    """Blocks scanned per (query, probed partition) under OR constraints: the
    union of Alg. 2's selections over the cross product of the lists."""
    tags = _c(tags, np.int32)
    probe_bins = _c(probe_bins, np.int32)
    nq, m = probe_bins.shape
    out = np.empty((nq, m), dtype=np.uint64)
    lib().orc_select_or(_p(tags), h, attrs.L, _p(attrs.vocab), _p(probe_bins), nq, m,
                        _p(oc.voff), _p(oc.vals), _p(out))
    return out


def search_or(X, attrs: Attrs, index: Index, Q, oc: OrCons, k, m, probe_in=None):
    """Alg. 2 with OR constraints (dense attributes): ids [nq,k], fp32
    distances [nq,k]."""
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    dist = np.empty((nq, k), dtype=np.float32)
    lib().orc_search_or(_p(X), X.shape[0], X.shape[1], attrs.L, _p(attrs.A), _p(attrs.vocab),
                        _p(_c(index.C, np.float32)), index.B, index.metric,
                        _p(_c(index.tags, np.int32)), index.h, _p(_c(index.perm, np.int32)),
                        _p(_c(index.offsets, np.int32)), _p(Q), nq, _p(oc.voff), _p(oc.vals), k,
                        m, _p(ids), _p(dist), _p(_c(probe_in, np.int32)))
    return ids, dist


def bruteforce(X, attrs: Attrs, Q, cons: Cons, k, metric=L2, order64=True):
    """Exact filtered kNN (Def. 2, appendix "Groundtruth")."""
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    d32 = np.empty((nq, k), dtype=np.float32)
    d64 = np.empty((nq, k), dtype=np.float64)
    cnt = np.empty(nq, dtype=np.int64)
    lib().orc_bruteforce(_p(X), X.shape[0], X.shape[1], *attrs.args(), _p(Q), nq,
                         *cons.args(), k, metric, int(bool(order64)), _p(ids), _p(d32),
                         _p(d64), _p(cnt))
    return ids, d32, d64, cnt


# ---- appendix "Metric": RecallK@K -------------------------------------------

def recall(ids, gt_ids, gt_d64, gt_count, k, X=None, Q=None, metric=L2):
    """RecallK@K = |index top-K  intersect  true top-K| / K, with two readings:

    strict: id-set intersection, divided by min(K, |D_C|);
    tie-aware (needs X, Q): a returned id is a hit when its exact distance is
    no worse than the true K-th distance (ids tied at the boundary count).
    Returns (strict_mean, tie_mean, per-query strict, per-query tie).
    """
    ids = np.asarray(ids)
    nq = ids.shape[0]
    strict = np.ones(nq)
    tie = np.ones(nq)
    for q in range(nq):
        denom = int(min(k, gt_count[q]))
        if denom == 0:
            continue
        truth = set(int(v) for v in gt_ids[q, :denom])
        got = [int(v) for v in ids[q, :k] if v >= 0]
        strict[q] = len(truth.intersection(got)) / denom
        if X is not None:
            kth = gt_d64[q, denom - 1]
            hits = 0
            for v in got:
                dv = dist64(X[v], Q[q], metric)
                if (dv <= kth) if metric == L2 else (dv >= kth):
                    hits += 1
            tie[q] = min(hits, denom) / denom
    return float(strict.mean()), float(tie.mean()), strict, tie


# ---- Sec. 5.2: learned partitioner (BLISS-style MLP) -------------------------

@dataclasses.dataclass
class MLP:
    """f(x) = W2 relu(W1 x + b1) + b2; W1 [H,d], b1 [H], W2 [B,H], b2 [B]."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray

    @property
    def dims(self):
        return self.W1.shape[1], self.W1.shape[0], self.W2.shape[0]

    def astype(self, dt):
        return MLP(*(np.ascontiguousarray(a, dtype=dt) for a in (self.W1, self.b1, self.W2, self.b2)))


def mlp_forward64(X, net: MLP):
    X = _c(X, np.float32)
    d, H, B = net.dims
    n64 = net.astype(np.float64)
    Z = np.empty((X.shape[0], B))
    Hd = np.empty((X.shape[0], H))
    lib().orc_mlp_forward64(_p(X), X.shape[0], d, H, B, _p(n64.W1), _p(n64.b1), _p(n64.W2),
                            _p(n64.b2), _p(Z), _p(Hd))
    return Z, Hd


def round_bf16(v):
    """Nearest bf16 value (ties to even) of each element, as fp64."""
    f = np.vectorize(lib().orc_bf16, otypes=[np.float64])
    return f(np.asarray(v, np.float64))


def mlp_loss_grad(X, Y, net: MLP, bf16=False):
    """Mean softmax cross-entropy and its fp64 gradients (gW1, gb1, gW2, gb2).
    bf16: the step with bf16 weights and activations -- every operand of a
    matrix product rounded to bf16, products summed exactly."""
    X = _c(X, np.float32)
    Y = _c(Y, np.float32)
    d, H, B = net.dims
    n64 = net.astype(np.float64)
    g = MLP(np.empty((H, d)), np.empty(H), np.empty((B, H)), np.empty(B))
    fn = lib().orc_mlp_loss_grad_bf16 if bf16 else lib().orc_mlp_loss_grad
    loss = fn(_p(X), X.shape[0], d, H, B, _p(n64.W1), _p(n64.b1), _p(n64.W2), _p(n64.b2), _p(Y),
              _p(g.W1), _p(g.b1), _p(g.W2), _p(g.b2))
    return loss, g


def adam(w, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in place on fp64 arrays (t counts from 1)."""
    for a in (w, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(_p(w), _p(g), _p(m), _p(v), w.size, lr, beta1, beta2, eps, int(t))


def mlp_logits32(X, net: MLP):
    X = _c(X, np.float32)
    d, H, B = net.dims
    n32 = net.astype(np.float32)
    Z = np.empty((X.shape[0], B), np.float32)
    lib().orc_mlp_logits32(_p(X), X.shape[0], d, H, B, _p(n32.W1), _p(n32.b1), _p(n32.W2),
                           _p(n32.b2), _p(Z))
    return Z


def mlp_assign32(X, net: MLP):
    X = _c(X, np.float32)
    d, H, B = net.dims
    n32 = net.astype(np.float32)
    out = np.empty(X.shape[0], np.int32)
    lib().orc_mlp_assign32(_p(X), X.shape[0], d, H, B, _p(n32.W1), _p(n32.b1), _p(n32.W2),
                           _p(n32.b2), _p(out))
    return out


def probe_logits(Q, net: MLP, m):
    """Top-m partitions by fp32 logit, largest first, ties to the lower id."""
    Z = mlp_logits32(Q, net)
    out = np.empty((Z.shape[0], m), np.int32)
    idx = np.arange(Z.shape[1])
    for q in range(Z.shape[0]):
        out[q] = np.lexsort((idx, -Z[q].astype(np.float64)))[:m]
    return out


def balanced_assign(top, B, load0=None):
    """Greedy balanced assignment (BLISS-style rounds): top [n, R] each
    point's R best partitions, best first; in id order every point goes to
    its least-loaded candidate (ties to the earlier one).  load0: loads
    before the first point (default zeros)."""
    top = _c(top, np.int32)
    n, R = top.shape
    bins = np.empty(n, np.int32)
    lib().orc_balanced_assign(_p(top), n, R, B, _p(_c(load0, np.int64)), _p(bins))
    return bins


def mlp_labels(X, attrs: Attrs, bins, samples, sample_cons, B, k=10, metric=L2):
    """Label of sample s: normalised histogram of the partitions (bins) of its
    k exact filtered nearest neighbours, the filter being the sample's own
    attributes on a chosen subset of fields (sample_cons row, -1 = free) and
    the sample itself excluded; a sample with no neighbour gets its own bin."""
    samples = np.asarray(samples, np.int64)
    Qs = np.ascontiguousarray(np.asarray(X, np.float32)[samples])
    ids, _, _, cnt = bruteforce(X, attrs, Qs, Cons(Qb=sample_cons), k + 1, metric=metric,
                                order64=False)
    Y = np.zeros((len(samples), B), np.float32)
    for r, s in enumerate(samples):
        nb = [int(i) for i in ids[r] if i >= 0 and i != s][:k]
        if not nb:
            Y[r, bins[s]] = 1.0
            continue
        for i in nb:
            Y[r, bins[i]] += 1.0
        Y[r] /= len(nb)
    return Y


def mlp_train(X, Y, net: MLP, epochs, batch, lr, order=None, bf16=False):
    """Adam on the mean cross-entropy, fp64, minibatches in the given order
    (default: sample order); returns the trained net and the loss per step.
    bf16: each step's gradients from the bf16 step (mlp_loss_grad), the
    fp64 weights being the masters."""
    X = _c(X, np.float32)
    Y = _c(Y, np.float32)
    # a copy: the caller's net is not updated in place
    w = MLP(*(np.array(a, dtype=np.float64, copy=True) for a in (net.W1, net.b1, net.W2, net.b2)))
    params = [w.W1, w.b1, w.W2, w.b2]
    ms = [np.zeros_like(a) for a in params]
    vs = [np.zeros_like(a) for a in params]
    n = X.shape[0]
    losses, t = [], 0
    for e in range(epochs):
        idx = np.arange(n) if order is None else np.asarray(order[e])
        for b0 in range(0, n, batch):
            sel = idx[b0:b0 + batch]
            loss, g = mlp_loss_grad(X[sel], Y[sel], w, bf16=bf16)
            t += 1
            for a, ga, ma, va in zip(params, [g.W1, g.b1, g.W2, g.b2], ms, vs):
                adam(a, np.ascontiguousarray(ga), ma, va, lr, t)
            losses.append(loss)
    return w, losses
