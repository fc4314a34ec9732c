"""Python binding of the CAPS GB300 library (include/caps.h).

Argument marshalling only: every step of index construction (Alg. 1) and of
the batched query (Alg. 2) runs in the CUDA kernels of libcaps_gb300.so.
There is no CPU fallback: importing works anywhere, but the first call fails
loudly if the compiled library is missing or no GPU is present.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; CPU/numpy arrays
are host memory and go through the library's own host<->device staging.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcaps_gb300.so")

CAPS_OK, CAPS_EINVAL, CAPS_ENOMEM, CAPS_ECUDA, CAPS_ETIMEOUT = 0, 1, 2, 3, 4
L2, IP = 0, 1
FP32, BF16, FP8, FP32_SPLIT = 0, 1, 2, 3
KMEANS, MLP = 0, 1
(ARR_CENTROIDS, ARR_BIN, ARR_TAGS, ARR_KEY, ARR_PERM, ARR_OFFSETS, ARR_MLP, ARR_LABELS,
 ARR_LABEL_BINS) = range(9)

# Every symbol declared in include/caps.h.
EXPORTS = ("caps_build", "caps_search_batch", "caps_free", "caps_last_error", "caps_get_info",
           "caps_export", "caps_assign", "caps_probe", "caps_probe_set", "caps_select",
           "caps_set_timing", "caps_get_stage_times", "caps_search_batch_noalloc",
           "caps_device_status", "caps_mlp_loss_grad", "caps_mlp_train", "caps_mlp_assign", "caps_plan_create",
           "caps_plan_search", "caps_plan_get_info", "caps_plan_free", "caps_alloc_count",
           "caps_inject_alloc_failure", "caps_test_scan_stall", "caps_search_batch_or",
           "caps_insert", "caps_mlp_balance", "caps_mlp_loss_grad_bf16", "caps_mlp_train_bf16")


class CapsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"CAPS error {code}: {msg}")
        self.code = code


class caps_attrs(ct.Structure):
    _fields_ = [("L", ct.c_int32), ("dense", ct.c_void_p), ("vocab", ct.c_void_p),
                ("sp_offsets", ct.c_void_p), ("sp_labels", ct.c_void_p), ("sp_vocab", ct.c_int32)]


class caps_or_constraints(ct.Structure):
    _fields_ = [("L", ct.c_int32), ("offsets", ct.c_void_p), ("values", ct.c_void_p)]


class caps_build_params(ct.Structure):
    _fields_ = [("B", ct.c_int32), ("h", ct.c_int32), ("kmeans_iters", ct.c_int32),
                ("seed", ct.c_uint64), ("metric", ct.c_int), ("part", ct.c_int),
                ("prec", ct.c_int), ("rerank_factor", ct.c_int32), ("mlp_hidden", ct.c_int32),
                ("mlp_epochs", ct.c_int32), ("init_idx", ct.c_void_p), ("centroids", ct.c_void_p),
                ("mlp_samples", ct.c_int32), ("mlp_batch", ct.c_int32), ("mlp_lr", ct.c_float),
                ("mlp_label_k", ct.c_int32), ("mlp_sample_idx", ct.c_void_p),
                ("mlp_sample_cons", ct.c_void_p), ("mlp_init", ct.c_void_p),
                ("mlp_rounds", ct.c_int32), ("mlp_balance_r", ct.c_int32),
                ("mlp_arbiter_queries", ct.c_int32), ("mlp_arbiter_m", ct.c_int32),
                ("mlp_bf16", ct.c_int32)]


class caps_stage_times(ct.Structure):
    _fields_ = [("prep_ms", ct.c_float), ("scores_ms", ct.c_float), ("topm_ms", ct.c_float),
                ("select_ms", ct.c_float), ("group_ms", ct.c_float), ("scan_ms", ct.c_float),
                ("merge_ms", ct.c_float), ("launches", ct.c_int32)]


class caps_index_info(ct.Structure):
    _fields_ = [("N", ct.c_int64), ("d", ct.c_int32), ("B", ct.c_int32), ("h", ct.c_int32),
                ("L", ct.c_int32), ("metric", ct.c_int32), ("n_codes", ct.c_int64),
                ("attr_words", ct.c_int32), ("device_bytes", ct.c_int64), ("part", ct.c_int32),
                ("mlp_hidden", ct.c_int32), ("n_labels", ct.c_int64),
                ("n_label_bins", ct.c_int64), ("mlp_balance_r", ct.c_int32),
                ("arbiter_recall_kmeans", ct.c_float), ("arbiter_recall_mlp", ct.c_float)]


class caps_plan_info(ct.Structure):
    _fields_ = [("nq", ct.c_int64), ("k", ct.c_int32), ("m", ct.c_int32),
                ("tile_n", ct.c_int32), ("item_cap", ct.c_int32), ("n_candidates", ct.c_int32),
                ("cand_tile_n", ct.c_int32 * 8), ("cand_item_cap", ct.c_int32 * 8),
                ("cand_ms", ct.c_float * 8), ("graph_nodes", ct.c_int32), ("pen", ct.c_int32),
                ("cand_pen", ct.c_int32 * 8)]


_lib = None


def lib(path: Optional[str] = None):
    """Load libcaps_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"CAPS CUDA library not built: {p} is missing "
                          "(run paper_2308_15014_gb300/build.py); there is no CPU fallback")
    L = ct.CDLL(p)
    P, i64, i32 = ct.c_void_p, ct.c_int64, ct.c_int32
    L.caps_build.argtypes = [ct.POINTER(caps_build_params), P, i64, i32, ct.POINTER(caps_attrs),
                             P, ct.POINTER(P)]
    L.caps_search_batch.argtypes = [P, P, i64, ct.POINTER(caps_attrs), i32, i32, P, P, P]
    L.caps_free.argtypes = [P]
    L.caps_free.restype = None
    L.caps_last_error.restype = ct.c_char_p
    L.caps_get_info.argtypes = [P, ct.POINTER(caps_index_info)]
    L.caps_export.argtypes = [P, i32, P, ct.c_size_t, P]
    L.caps_assign.argtypes = [P, i64, i32, P, i32, i32, P, P]
    L.caps_probe.argtypes = [P, P, i64, i32, P, P]
    L.caps_probe_set.argtypes = [P, P, i64, i32, P, P]
    L.caps_select.argtypes = [P, P, i64, i32, ct.POINTER(caps_attrs), P, P]
    L.caps_search_batch_noalloc.argtypes = [P, P, i64, ct.POINTER(caps_attrs), i32, i32, P, P,
                                            P]
    L.caps_device_status.argtypes = [P, P]
    L.caps_mlp_loss_grad.argtypes = [i32, i32, i32, P, P, P, P, P, i64, P, P, P, P, P, P, P]
    L.caps_mlp_train.argtypes = [i32, i32, i32, P, P, i64, P, i32, i32, ct.c_float, P, P]
    L.caps_mlp_loss_grad_bf16.argtypes = L.caps_mlp_loss_grad.argtypes
    L.caps_mlp_train_bf16.argtypes = L.caps_mlp_train.argtypes
    L.caps_mlp_assign.argtypes = [i32, i32, i32, P, P, i64, P, P]
    L.caps_mlp_balance.argtypes = [i32, i32, i32, P, P, i64, i32, P, P, P]
    L.caps_plan_create.argtypes = [P, P, i64, ct.POINTER(caps_attrs), i32, i32, i32, P,
                                   ct.POINTER(P)]
    L.caps_plan_search.argtypes = [P, P, i64, ct.POINTER(caps_attrs), P, P, P]
    L.caps_plan_get_info.argtypes = [P, ct.POINTER(caps_plan_info)]
    L.caps_plan_free.argtypes = [P]
    L.caps_plan_free.restype = None
    L.caps_set_timing.argtypes = [i32]
    L.caps_get_stage_times.argtypes = [ct.POINTER(caps_stage_times)]
    L.caps_alloc_count.argtypes = []
    L.caps_alloc_count.restype = i64
    L.caps_inject_alloc_failure.argtypes = [i64]
    L.caps_inject_alloc_failure.restype = None
    L.caps_search_batch_or.argtypes = [P, P, i64, ct.POINTER(caps_or_constraints), i32, i32, P,
                                       P, P]
    L.caps_insert.argtypes = [P, P, i64, ct.POINTER(caps_attrs), P]
    L.caps_test_scan_stall.argtypes = [i64, ct.c_uint64]
    L.caps_test_scan_stall.restype = None
    _lib = L
    return L


def _check(rc: int):
    if rc != CAPS_OK:
        raise CapsError(rc, lib().caps_last_error().decode())


def _torch():
    try:
        import torch
        return torch
    except ImportError:  # pragma: no cover
        return None


def _ptr(a):
    """Raw address of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    t = _torch()
    if t is not None and isinstance(a, t.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream=None):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    t = _torch()
    if t is not None and t.cuda.is_available():
        return t.cuda.current_stream().cuda_stream
    return 0


def _np_or_keep(a, dtype):
    t = _torch()
    if t is not None and isinstance(a, t.Tensor):
        want = {np.float32: t.float32, np.int32: t.int32, np.int64: t.int64}[dtype]
        if a.dtype != want:
            raise TypeError(f"expected {want}, got {a.dtype}")
        return a.contiguous()
    return np.ascontiguousarray(a, dtype=dtype)


def _dense_attrs(A, vocab=None):
    A = _np_or_keep(A, np.int32)
    at = caps_attrs()
    at.L = int(A.shape[1])
    at.dense = _ptr(A)
    keep = [A]
    if vocab is not None:
        v = np.ascontiguousarray(vocab, dtype=np.int32)
        at.vocab = _ptr(v)
        keep.append(v)
    return at, keep


def _sparse_attrs(off, lab, vocab=0):
    """Label-set attributes or constraints: CSR offsets [n+1] (int64) and
    labels (int32); for data the labels of each point ascend strictly."""
    off = _np_or_keep(off, np.int64)
    lab = _np_or_keep(lab, np.int32)
    at = caps_attrs()
    at.L = 0
    at.sp_offsets = _ptr(off)
    at.sp_labels = _ptr(lab) if lab.shape[0] > 0 else None
    at.sp_vocab = int(vocab)
    return at, [off, lab]


def _cons(Qb):
    """Dense constraint rows [nq, L], or a (q_off, q_lab) pair of label sets."""
    if isinstance(Qb, tuple):
        return _sparse_attrs(Qb[0], Qb[1])
    return _dense_attrs(Qb)


def assign(X, C, metric=L2, out=None, stream=None):
    """f(x) = best centroid for every row of X (caps_assign)."""
    X = _np_or_keep(X, np.float32)
    C = _np_or_keep(C, np.float32)
    N, d = X.shape
    if out is None:
        out = np.empty(N, dtype=np.int32)
    _check(lib().caps_assign(_ptr(X), N, d, _ptr(C), C.shape[0], metric, _ptr(out),
                             _stream(stream)))
    return out


def set_timing(enable: bool):
    """Record per-stage CUDA events in later searches on this thread."""
    _check(lib().caps_set_timing(1 if enable else 0))


def stage_times() -> dict:
    """Stage times (ms) of the last timed search on this thread."""
    t = caps_stage_times()
    _check(lib().caps_get_stage_times(ct.byref(t)))
    return {f: getattr(t, f) for f, _ in caps_stage_times._fields_}


def mlp_flat(W1, b1, W2, b2):
    """Concatenate the MLP weights in the library's order W1|b1|W2|b2."""
    return np.ascontiguousarray(np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2),
                                                np.ravel(b2)]).astype(np.float32))


def mlp_loss_grad(W1, b1, W2, b2, X, Y, stream=None, bf16=False):
    """caps_mlp_loss_grad (bf16: caps_mlp_loss_grad_bf16): loss and fp32
    gradients (gW1, gb1, gW2, gb2)."""
    W1, b1, W2, b2 = (np.ascontiguousarray(a, np.float32) for a in (W1, b1, W2, b2))
    X = np.ascontiguousarray(X, np.float32)
    Y = np.ascontiguousarray(Y, np.float32)
    H, d = W1.shape
    B = W2.shape[0]
    g = [np.empty_like(a) for a in (W1, b1, W2, b2)]
    loss = ct.c_float()
    fn = lib().caps_mlp_loss_grad_bf16 if bf16 else lib().caps_mlp_loss_grad
    _check(fn(d, H, B, _ptr(W1), _ptr(b1), _ptr(W2), _ptr(b2), _ptr(X), X.shape[0], _ptr(Y),
              _ptr(g[0]), _ptr(g[1]), _ptr(g[2]), _ptr(g[3]), ct.byref(loss), _stream(stream)))
    return float(loss.value), g


def mlp_train(W, d, H, B, X, Y, epochs, batch, lr, stream=None, bf16=False):
    """caps_mlp_train (bf16: caps_mlp_train_bf16) on a flat W1|b1|W2|b2 copy;
    returns (W, losses)."""
    W = np.array(W, np.float32, copy=True)
    X = np.ascontiguousarray(X, np.float32)
    Y = np.ascontiguousarray(Y, np.float32)
    steps = epochs * ((X.shape[0] + batch - 1) // batch)
    losses = np.zeros(max(1, steps), np.float32)
    fn = lib().caps_mlp_train_bf16 if bf16 else lib().caps_mlp_train
    _check(fn(d, H, B, _ptr(W), _ptr(X), X.shape[0], _ptr(Y), epochs, batch, lr, _ptr(losses),
              _stream(stream)))
    return W, losses[:steps]


def mlp_assign(W, d, H, B, X, stream=None):
    """caps_mlp_assign: argmax partition of every row of X."""
    W = np.ascontiguousarray(W, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    out = np.empty(X.shape[0], np.int32)
    _check(lib().caps_mlp_assign(d, H, B, _ptr(W), _ptr(X), X.shape[0], _ptr(out), _stream(stream)))
    return out


def mlp_balance(W, d, H, B, X, R, load0=None, stream=None):
    """caps_mlp_balance: the balanced assignment over each row's R largest
    logits, loads starting at load0 (zeros when None)."""
    W = np.ascontiguousarray(W, np.float32)
    X = np.ascontiguousarray(X, np.float32)
    if load0 is not None:
        load0 = np.ascontiguousarray(load0, np.int64)
    out = np.empty(X.shape[0], np.int32)
    _check(lib().caps_mlp_balance(d, H, B, _ptr(W), _ptr(X), X.shape[0], R,
                                  _ptr(load0) if load0 is not None else None, _ptr(out),
                                  _stream(stream)))
    return out


class Index:
    """A CAPS index living in GPU memory (caps_build / caps_free)."""

    def __init__(self, handle, keep=None):
        self._h = handle
        info = caps_index_info()
        _check(lib().caps_get_info(self._h, ct.byref(info)))
        self.info = info

    @classmethod
    def build(cls, X, A, vocab, B, h=15, iters=20, metric=L2, init_idx=None, centroids=None,
              seed=0, prec=FP32, rerank_factor=0, part=KMEANS, mlp_hidden=0, mlp_epochs=0,
              mlp_samples=0, mlp_batch=0, mlp_lr=0.0, mlp_label_k=0, mlp_sample_idx=None,
              mlp_sample_cons=None, mlp_init=None, mlp_rounds=0, mlp_balance_r=0,
              mlp_arbiter_queries=0, mlp_arbiter_m=0, mlp_bf16=0, labels=None,
              stream=None) -> "Index":
        """labels = (sp_off, sp_lab, sp_vocab): label-set attributes instead of
        the dense A / vocab."""
        X = _np_or_keep(X, np.float32)
        N, d = X.shape
        if labels is not None:
            at, keep = _sparse_attrs(*labels)
        else:
            at, keep = _dense_attrs(A, vocab)
        p = caps_build_params()
        p.B, p.h, p.kmeans_iters, p.seed, p.metric = B, h, iters, seed, metric
        p.part, p.prec, p.rerank_factor = part, prec, rerank_factor
        p.mlp_hidden, p.mlp_epochs, p.mlp_samples, p.mlp_batch = (mlp_hidden, mlp_epochs,
                                                                  mlp_samples, mlp_batch)
        p.mlp_lr, p.mlp_label_k = mlp_lr, mlp_label_k
        p.mlp_rounds, p.mlp_balance_r = mlp_rounds, mlp_balance_r
        p.mlp_arbiter_queries, p.mlp_arbiter_m = mlp_arbiter_queries, mlp_arbiter_m
        p.mlp_bf16 = mlp_bf16
        if mlp_sample_idx is not None:
            mlp_sample_idx = _np_or_keep(mlp_sample_idx, np.int64)
            p.mlp_sample_idx = _ptr(mlp_sample_idx)
        if mlp_sample_cons is not None:
            mlp_sample_cons = _np_or_keep(mlp_sample_cons, np.int32)
            p.mlp_sample_cons = _ptr(mlp_sample_cons)
        if mlp_init is not None:
            mlp_init = _np_or_keep(mlp_init, np.float32)
            p.mlp_init = _ptr(mlp_init)
        if init_idx is not None:
            init_idx = _np_or_keep(init_idx, np.int64)
            p.init_idx = _ptr(init_idx)
        if centroids is not None:
            centroids = _np_or_keep(centroids, np.float32)
            p.centroids = _ptr(centroids)
        h_out = ct.c_void_p()
        _check(lib().caps_build(ct.byref(p), _ptr(X), N, d, ct.byref(at), _stream(stream),
                                ct.byref(h_out)))
        return cls(h_out)

    def close(self):
        if self._h:
            lib().caps_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def export(self, which: int) -> np.ndarray:
        i = self.info
        shapes = {ARR_CENTROIDS: ((i.B, i.d), np.float32), ARR_BIN: ((i.N,), np.int32),
                  ARR_TAGS: ((i.B, i.h), np.int32), ARR_KEY: ((i.N,), np.uint8),
                  ARR_PERM: ((i.N,), np.int32),
                  ARR_OFFSETS: ((i.B * (i.h + 1) + 1,), np.int32)}
        Hm = i.mlp_hidden
        shapes[ARR_MLP] = ((Hm * i.d + Hm + i.B * Hm + i.B,), np.float32)
        shapes[ARR_LABELS] = ((i.n_labels, i.B), np.float32)
        shapes[ARR_LABEL_BINS] = ((i.n_label_bins,), np.int32)
        shape, dt = shapes[which]
        out = np.empty(shape, dtype=dt)
        _check(lib().caps_export(self._h, which, _ptr(out) if out.size else 1, out.nbytes,
                                 _stream(None)))
        return out

    def status(self, stream=None):
        """Raise CapsError(CAPS_ETIMEOUT) if a bounded device wait expired."""
        _check(lib().caps_device_status(self._h, _stream(stream)))

    def probe(self, Q, m, out=None, stream=None):
        Q = _np_or_keep(Q, np.float32)
        nq = Q.shape[0]
        if out is None:
            out = np.empty((nq, m), dtype=np.int32)
        _check(lib().caps_probe(self._h, _ptr(Q), nq, m, _ptr(out), _stream(stream)))
        return out

    def probe_set(self, Q, m, out=None, stream=None):
        """The probe set the batched search uses (row order unspecified)."""
        Q = _np_or_keep(Q, np.float32)
        nq = Q.shape[0]
        if out is None:
            out = np.empty((nq, m), dtype=np.int32)
        _check(lib().caps_probe_set(self._h, _ptr(Q), nq, m, _ptr(out), _stream(stream)))
        return out

    def select(self, probe, Qb, out=None, stream=None):
        probe = _np_or_keep(probe, np.int32)
        nq, m = probe.shape
        at, keep = _cons(Qb)
        if out is None:
            out = np.empty((nq, m), dtype=np.uint64)
        _check(lib().caps_select(self._h, _ptr(probe), nq, m, ct.byref(at), _ptr(out),
                                 _stream(stream)))
        return out

    def search(self, Q, Qb, k, m, out_ids=None, out_dist=None, stream=None):
        """Alg. 2 for a batch; returns (ids [nq,k] int64, dist [nq,k] fp32).
        Qb: dense constraint rows, or (q_off, q_lab) label sets.  Outputs land
        where the inputs live unless given explicitly."""
        Q = _np_or_keep(Q, np.float32)
        nq = Q.shape[0]
        at, keep = _cons(Qb)
        t = _torch()
        if out_ids is None:
            if t is not None and isinstance(Q, t.Tensor) and Q.is_cuda:
                out_ids = t.empty((nq, k), dtype=t.int64, device=Q.device)
                out_dist = t.empty((nq, k), dtype=t.float32, device=Q.device)
            else:
                out_ids = np.empty((nq, k), dtype=np.int64)
                out_dist = np.empty((nq, k), dtype=np.float32)
        _check(lib().caps_search_batch(self._h, _ptr(Q), nq, ct.byref(at), k, m, _ptr(out_ids),
                                       _ptr(out_dist), _stream(stream)))
        return out_ids, out_dist

    def insert(self, X, A, stream=None):
        """caps_insert: add the rows X [n, d] with dense attributes A [n, L];
        they get the ids N .. N+n-1.  Plans made before refuse to run."""
        X = _np_or_keep(X, np.float32)
        at, keep = _dense_attrs(A)
        _check(lib().caps_insert(self._h, _ptr(X), X.shape[0], ct.byref(at), _stream(stream)))
        inf = caps_index_info()
        _check(lib().caps_get_info(self._h, ct.byref(inf)))
        self.info = inf

    def search_or(self, Q, lists, k, m, out_ids=None, out_dist=None, stream=None):
        """caps_search_batch_or: Alg. 2 with per-field value lists (Sec. 5.3).
        lists: (offsets int64 [nq*L+1], values int32), or a list over queries
        of lists over fields of allowed values (empty = unconstrained).
        Returns (ids [nq,k] int64, dist [nq,k] fp32), where the inputs live
        unless the outputs are given."""
        Q = _np_or_keep(Q, np.float32)
        nq = Q.shape[0]
        if isinstance(lists, (list, tuple)) and not (len(lists) == 2 and hasattr(lists[0], "dtype")):
            off, vals = [0], []
            for row in lists:
                for f in row:
                    vals.extend(int(v) for v in f)
                    off.append(len(vals))
            lists = (np.asarray(off, np.int64), np.asarray(vals, np.int32))
        off, vals = lists
        off = _np_or_keep(off, np.int64)
        vals = _np_or_keep(vals, np.int32)
        oc = caps_or_constraints(self.info.L, _ptr(off) if len(off) else None,
                                 _ptr(vals) if len(vals) else None)
        t = _torch()
        if out_ids is None:
            if t is not None and isinstance(Q, t.Tensor) and Q.is_cuda:
                out_ids = t.empty((nq, k), dtype=t.int64, device=Q.device)
                out_dist = t.empty((nq, k), dtype=t.float32, device=Q.device)
            else:
                out_ids = np.empty((nq, k), dtype=np.int64)
                out_dist = np.empty((nq, k), dtype=np.float32)
        _check(lib().caps_search_batch_or(self._h, _ptr(Q), nq, ct.byref(oc), k, m,
                                          _ptr(out_ids), _ptr(out_dist), _stream(stream)))
        return out_ids, out_dist

    def search_noalloc(self, Q, Qb, k, m, out_ids, out_dist, stream=None):
        """caps_search_batch_noalloc: same query, no device allocation.
        Q (float32 [nq, d]), Qb (int32 [nq, L]), out_ids (int64 [nq, k]) and
        out_dist (float32 [nq, k]) must be contiguous CUDA tensors on one
        device; nothing is converted (a conversion would allocate)."""
        check_noalloc_args(Q, Qb, k, out_ids, out_dist, self.info.d, self.info.L)
        at, keep = _dense_attrs(Qb)
        _check(lib().caps_search_batch_noalloc(self._h, _ptr(Q), Q.shape[0], ct.byref(at), k, m,
                                               _ptr(out_ids), _ptr(out_dist), _stream(stream)))
        return out_ids, out_dist

    def plan(self, Q, Qb, k, m, autotune=True, stream=None) -> "Plan":
        """caps_plan_create: a tuned, graph-captured plan for batches shaped
        like Q (its rows are the autotuner's sample)."""
        Q = _np_or_keep(Q, np.float32)
        at, keep = _cons(Qb)
        h = ct.c_void_p()
        _check(lib().caps_plan_create(self._h, _ptr(Q), Q.shape[0], ct.byref(at), k, m,
                                      1 if autotune else 0, _stream(stream), ct.byref(h)))
        return Plan(h, self, k)


def check_noalloc_args(Q, Qb, k, out_ids, out_dist, d, L):
    """Argument checks of Index.search_noalloc, made before any pointer
    reaches the library: the C call cannot tell a float64 query or a short
    output from a correct one, and would read or write past its end."""
    t = _torch()
    if t is None:
        raise ValueError("search_noalloc takes CUDA tensors (torch is not available)")
    want = (("Q", Q, t.float32, d), ("Qb", Qb, t.int32, L), ("out_ids", out_ids, t.int64, k),
            ("out_dist", out_dist, t.float32, k))
    nq = Q.shape[0] if isinstance(Q, t.Tensor) and Q.dim() == 2 else None
    for name, a, dt, cols in want:
        if not isinstance(a, t.Tensor):
            raise ValueError(f"{name} must be a torch tensor")
        if a.dtype != dt:
            raise ValueError(f"{name} must be {dt}, got {a.dtype}")
        if a.dim() != 2 or a.shape[1] != cols or (nq is not None and a.shape[0] != nq):
            raise ValueError(f"{name} must have shape ({nq}, {cols}), got {tuple(a.shape)}")
        if not a.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    devs = {a.device for _, a, _, _ in want}
    if any(dv.type != "cuda" for dv in devs):
        raise ValueError("Q, Qb, out_ids and out_dist must be CUDA tensors")
    if len(devs) != 1:
        raise ValueError("Q, Qb, out_ids and out_dist must be on one device")


def alloc_count() -> int:
    """caps_alloc_count: device allocations the library has made so far."""
    return int(lib().caps_alloc_count())


def inject_alloc_failure(n: int):
    """caps_inject_alloc_failure: fail the n-th device allocation from now
    (1 = the next) as an out-of-memory device would; n <= 0 disarms."""
    lib().caps_inject_alloc_failure(int(n))


def scan_stall_hook(item: int, wait_ns: int = 0):
    """caps_test_scan_stall: later tensor-core scans withhold every copy and
    MMA of work item `item` and give up each bounded wait after wait_ns
    (item < 0: normal operation)."""
    lib().caps_test_scan_stall(int(item), int(wait_ns))


class Plan:
    """A tuned, graph-captured batch query (caps_plan_*); keeps its index alive."""

    def __init__(self, handle, index, k):
        self._h = handle
        self._index = index
        self.k = k
        inf = caps_plan_info()
        _check(lib().caps_plan_get_info(self._h, ct.byref(inf)))
        self.nq = inf.nq
        n = inf.n_candidates
        self.info = {"nq": inf.nq, "k": inf.k, "m": inf.m, "tile_n": inf.tile_n,
                     "item_cap": inf.item_cap, "pen": inf.pen, "graph_nodes": inf.graph_nodes,
                     "candidates": [{"tile_n": inf.cand_tile_n[i],
                                     "item_cap": inf.cand_item_cap[i], "pen": inf.cand_pen[i],
                                     "ms": round(float(inf.cand_ms[i]), 4)} for i in range(n)]}

    def search(self, Q, Qb, out_ids=None, out_dist=None, stream=None):
        """Replay the plan on a batch of <= nq queries; returns (ids, dist)."""
        Q = _np_or_keep(Q, np.float32)
        nq = Q.shape[0]
        at, keep = _dense_attrs(Qb)
        t = _torch()
        if out_ids is None:
            if t is not None and isinstance(Q, t.Tensor) and Q.is_cuda:
                out_ids = t.empty((nq, self.k), dtype=t.int64, device=Q.device)
                out_dist = t.empty((nq, self.k), dtype=t.float32, device=Q.device)
            else:
                out_ids = np.empty((nq, self.k), dtype=np.int64)
                out_dist = np.empty((nq, self.k), dtype=np.float32)
        _check(lib().caps_plan_search(self._h, _ptr(Q), nq, ct.byref(at), _ptr(out_ids),
                                      _ptr(out_dist), _stream(stream)))
        return out_ids, out_dist

    def close(self):
        if self._h:
            lib().caps_plan_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
