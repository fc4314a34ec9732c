#!/usr/bin/env python
"""Benchmark of the CAPS filtered-search hot path on one GB300.

Workload: 1,000,000 x 128 byte-valued vectors (fp32), 3 attribute fields
(vocab 20/50/100, Zipf 1.0), B = 1024 k-means partitions (20 Lloyd
iterations), AFT height 15, 10,000 queries with 1-3 AND constraints
(selectivity 0.1%-30%), k = 10, squared L2.  A step is one batched query of
all 10,000 queries (Alg. 2: filter packing, centroid scores, top-m, block
selection, fused scan + top-k) with queries resident in HBM; the index build
(Alg. 1) runs once before and is reported as build time.  m is the smallest
probe count in {8,12,16,24,32,40,48,64} whose tie-aware recall@10 (against the
exact filtered kNN of a seeded sample of queries, from the CPU oracle's brute
force ordered by fp64 distance, untimed) is >= 0.9.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle
(the plain C restatement of the method) on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("filtered QPS at recall@10>=0.9 (learned partitioner + BF16 tensor-core path; "
          "plain FP32 k-means paths alongside: fp32 on the tensor cores as split bf16 terms, "
          "and the SIMT fp32 scan)")
UNIT = "queries/s"
M_SWEEP = (8, 12, 16, 24, 32, 40, 48, 64)
SPARSE_M_SWEEP = (8, 16, 32, 64, 128, 256)
RECALL_SAMPLE = 500
FALLBACK_HBM_GBS = 6800.0
# fp32 peak from unit counts and clock: 152 SMs x 128 fp32 lanes x 2 flop
# (fma) x 2.07 GHz maximum SM clock
SMS, FP32_LANES, MAX_SM_GHZ = 152, 128, 2.07
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * MAX_SM_GHZ / 1e3
SCAN_KERNEL = "k_scan_bin"
SCAN_SRC = "scan_bin.cu"
TC_KERNEL = "k_scan_tc"
TC_SRC = "scan_tc_kernel.cuh"


def _json_default(o):
    if isinstance(o, np.integer):
        return int(o)
    if isinstance(o, np.floating):
        return float(o)
    raise TypeError(type(o).__name__)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["caps", "reference"], default="caps")
    ap.add_argument("--config", choices=["sift1m", "small"], default="sift1m")
    ap.add_argument("--m", type=int, default=0, help="fixed probe count (0 = sweep)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--paths", default="mlp_bf16,fp32_split,fp32,bf16,fp8",
                    help="comma list of search paths (fp32, fp32_split, bf16, fp8, mlp_fp32, "
                         "mlp_fp32_split, mlp_bf16, mlp_fp8); the first is the headline")
    ap.add_argument("--no-ablations", action="store_true",
                    help="skip the ablations (k-means + bf16, QPS at recall@10 >= 0.9 for AFT "
                         "heights h, constrained-field counts and 10 attribute fields)")
    ap.add_argument("--no-sparse", action="store_true",
                    help="skip the label-set workload (2M x 128, 10,000 labels, 4,096 queries)")
    ap.add_argument("--no-learned4m", action="store_true",
                    help="skip the learned-partitioner workload (4M x 96 inner product, 5 fields, "
                         "MLP 96 -> 512 -> 1024): k-means vs learned at equal recall, build times")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_workload(name):
    from workloads import config_sift1m_like, config_small
    return config_sift1m_like() if name == "sift1m" else config_small()


def bf16_peak_tflops():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["bf16_tflops"]), "measured (cuBLAS bf16 burst)"
    return 1900.0, "fallback"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) != 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def scan_traffic_bytes(w, perm, offsets, probe, sel, words_pad, bf16=False, split=False):
    """Algorithmic bytes of the scan for one batch.

    fp32 scan -- union: attribute words of every row some query selects, plus
    the fp32 vector of every row that passes some query's filter (each byte
    once: the HBM floor of the whole batch); per_query: the same sums taken
    query by query (the paper's query-time term sum |p| (L + d*match)).
    bf16 tensor-core scan -- every selected row is scored, so the union is
    each selected row's bf16 vector, attribute words, id and norm once; the
    split fp32 form reads two bf16 terms per coordinate."""
    N, d, h = w.N, w.d, w.h
    nb = h + 1
    Ar = w.A[perm]
    q_list, s_list = [], []
    for j in range(nb):
        qq, ii = np.nonzero((sel >> np.uint64(j)) & np.uint64(1))
        q_list.append(qq)
        s_list.append(probe[qq, ii].astype(np.int64) * nb + j)
    qs = np.concatenate(q_list)
    ss = np.concatenate(s_list)
    order = np.argsort(ss, kind="stable")
    qs, ss = qs[order], ss[order]
    bounds = np.flatnonzero(np.diff(ss)) + 1
    touched = np.zeros(N, bool)
    passed = np.zeros(N, bool)
    pq_scan = pq_pass = 0
    for grp_q, s in zip(np.split(qs, bounds), ss[np.concatenate([[0], bounds])] if len(ss) else []):
        r0, r1 = int(offsets[s]), int(offsets[s + 1])
        if r1 <= r0:
            continue
        touched[r0:r1] = True
        b = w.Qb[grp_q]
        ok = np.all((b[:, None, :] < 0) | (Ar[None, r0:r1, :] == b[:, None, :]), axis=2)
        passed[r0:r1] |= ok.any(0)
        pq_scan += (r1 - r0) * len(grp_q)
        pq_pass += int(ok.sum())
    attr_b = 4 * words_pad
    if bf16 or split:
        row_b = (4 if split else 2) * d + attr_b + 8
        return int(touched.sum()) * row_b, pq_scan * row_b, pq_scan, pq_pass
    union = int(touched.sum()) * attr_b + int(passed.sum()) * d * 4
    per_query = pq_scan * attr_b + pq_pass * d * 4
    return union, per_query, pq_scan, pq_pass


def dense_item_stats(w, offsets, probe, sel, group=128):
    """Work of the partition-major tensor-core scan as it forms its items:
    probes sorted by partition (query order kept), cut into groups of
    `group`; each item streams the union of its probes' selected blocks.
    Returns (items, sum of union rows, sum of union rows x probes)."""
    nb = w.h + 1
    B = w.B
    pr = probe.reshape(-1)
    sl = sel.reshape(-1)
    if group == 128 and nb <= 16:  # the tensor-core scan orders by (partition, mask)
        order = np.lexsort((np.arange(len(pr)), sl, pr))
    else:
        order = np.argsort(pr, kind="stable")
    pr, sl = pr[order], sl[order]
    starts = np.searchsorted(pr, np.arange(B + 1))
    sizes = np.diff(offsets.astype(np.int64).reshape(-1)[: B * nb + 1]).reshape(B, nb)
    items = rows = pairs = 0
    for b in range(B):
        s0, s1 = starts[b], starts[b + 1]
        for g0 in range(s0, s1, group):
            g1 = min(s1, g0 + group)
            u = np.bitwise_or.reduce(sl[g0:g1])
            bits = (u >> np.arange(nb, dtype=np.uint64)) & np.uint64(1)
            ur = int(sizes[b][bits.astype(bool)].sum())
            items += 1
            rows += ur
            pairs += ur * (g1 - g0)
    return int(items), int(rows), int(pairs)


def traffic_from_profile(kernel=SCAN_KERNEL, src_name=SCAN_SRC, m=None, variant=None):
    """dram bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current source of that kernel, of the same form
    (variant) and, where the entry names one, at the same probe count m
    (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    src = os.path.join(ROOT, "paper_2308_15014_gb300", "csrc", src_name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        entries = json.load(f)
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    for e in entries:
        if e.get("kernel") == kernel and e.get("src_sha") == sha and \
                e.get("variant") == variant and (m is None or e.get("m") in (None, m)):
            return e.get("dram_bytes_per_launch")
    return None


def e4m3(v):
    """Round to the nearest e4m3 value (ties to even, saturating at 448): three
    mantissa bits, exponent bias 7, subnormal spacing 2^-9."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    e = np.minimum(np.floor(np.log2(np.maximum(a, 2.0 ** -6))), 8.0)
    quantum = 2.0 ** (e - 3)
    return np.sign(v) * np.minimum(np.round(a / quantum) * quantum, 448.0)


def form1_error(w, rng_seed=11, nq=64, nrow=2048):
    """Relative error of the BF16 and the e4m3 tile score against the FP64
    distance.

    The tensor-core tile multiplies rounded vectors and accumulates in fp32;
    the score is |x|^2 + |q|^2 - 2 q.x with fp32 norms.  BF16: x and q rounded
    to bf16.  e4m3: each row (and query) scaled by s = max |x| / 448 (fp32),
    x / s (fp32) rounded to e4m3, the dot product multiplied back by the two
    scales.  The products are summed in fp64 here (the fp32 accumulation adds
    at most ~d * 2^-24 relative) and compared with the exact squared distance
    in fp64 on random (query, row) pairs.  The returned distances themselves
    are exact fp32 (re-ranked)."""
    rng = np.random.default_rng(rng_seed)
    qi = rng.choice(w.Q.shape[0], min(nq, w.Q.shape[0]), replace=False)
    ri = rng.choice(w.X.shape[0], min(nrow, w.X.shape[0]), replace=False)
    X32, Q32 = w.X[ri].astype(np.float32), w.Q[qi].astype(np.float32)
    X, Q = X32.astype(np.float64), Q32.astype(np.float64)

    def bf16(a):
        u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000  # round to nearest even
        return u.astype(np.uint32).view(np.float32).astype(np.float64)

    def scaled_e4m3(a32):
        amax = np.abs(a32).max(1)
        sc = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
        return e4m3((a32 / sc[:, None]).astype(np.float32)), sc.astype(np.float64)

    xn = (X * X).sum(1)
    qn = (Q * Q).sum(1)
    exact = ((Q[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    out = {}
    x8, xs = scaled_e4m3(X32)
    q8, qs = scaled_e4m3(Q32)
    for name, dot in (("bf16", bf16(Q) @ bf16(X).T), ("e4m3", (q8 @ x8.T) * qs[:, None] * xs[None, :])):
        approx = xn[None, :] + qn[:, None] - 2.0 * dot
        rel = np.abs(approx - exact) / np.maximum(exact, 1e-30)
        out[name] = {"pairs": int(rel.size), "max_rel": float(rel.max()),
                     "mean_rel": float(rel.mean())}
    return out


def oracle_truth(w, samp, k=None):
    """Exact filtered kNN of the sampled queries (Def. 2, appendix
    "Groundtruth") from the CPU oracle's brute force: every point filtered,
    the valid ones ordered by fp64 distance (ties to the lower id).  Runs
    outside every timed region.  Returns ids [n, k] (-1 padded), their fp64
    distances and |D_C| per query."""
    import oracle as O
    from oracle.build import build_oracle
    build_oracle()
    O.set_threads(0)
    cons = O.Cons.of(w).subset(samp)
    ids, _, d64, cnt = O.bruteforce(w.X, O.Attrs.of(w), np.ascontiguousarray(w.Q[samp]), cons,
                                    k or w.k, metric=w.metric, order64=True)
    return ids, d64, cnt


def library_truth(caps, torch, w, samp, labels=False):
    """The same sample answered by the library with every partition probed
    (m = B: the exact filtered top-k by construction), its 2k best reordered
    by fp64 distance.  Used only to cross-check oracle_truth."""
    k, k2, Bt = w.k, min(2 * w.k, 128), 64
    init = (np.arange(Bt, dtype=np.int64) * (w.N // Bt)).astype(np.int64)
    X = torch.from_numpy(w.X).cuda()
    if labels:
        ix = caps.Index.build(X, None, None, Bt, h=w.h, iters=0, init_idx=init, metric=w.metric,
                              labels=(w.sp_off, w.sp_lab, w.sp_vocab))
        rows = [w.q_lab[w.q_off[q]:w.q_off[q + 1]] for q in samp]
        q_off = np.zeros(len(samp) + 1, dtype=np.int64)
        q_off[1:] = np.cumsum([len(r) for r in rows])
        q_lab = np.concatenate(rows).astype(np.int32) if len(rows) else np.zeros(0, np.int32)
        ids, _ = ix.search(np.ascontiguousarray(w.Q[samp]), (q_off, q_lab), k2, Bt)
    else:
        ix = caps.Index.build(X, torch.from_numpy(w.A).cuda(), w.vocab, Bt, h=w.h, iters=0,
                              init_idx=init, metric=w.metric)
        ids, _ = ix.search(np.ascontiguousarray(w.Q[samp]), np.ascontiguousarray(w.Qb[samp]),
                           k2, Bt)
    ix.close()
    n = len(samp)
    g64 = np.full((n, k), np.inf if w.metric == 0 else -np.inf)
    for i, q in enumerate(samp):
        got = ids[i][ids[i] >= 0]
        d = exact_dist(w.X[got], w.Q[q], w.metric)
        order = np.lexsort((got, d if w.metric == 0 else -d))[:k]
        g64[i, :len(order)] = d[order]
    return g64


def exact_truth(caps, torch, w, samp, labels=False):
    """Ground truth for the recall of the sampled queries: the oracle's brute
    force, cross-checked against the library's m = B search (the k best fp64
    distances of the two must agree to 1e-6 relative, position by position;
    the bench stops if they do not).  Returns (ids, fp64 distances, |D_C|,
    the cross-check's summary)."""
    gt, g64, cnt = oracle_truth(w, samp)
    lib64 = library_truth(caps, torch, w, samp, labels=labels)
    fin = np.isfinite(g64) | np.isfinite(lib64)
    both = np.isfinite(g64) & np.isfinite(lib64)
    tol = 1e-6 * np.maximum(1.0, np.abs(np.where(both, g64, 0.0)))
    bad = (fin & ~both) | (both & (np.abs(g64 - lib64) > tol))
    n_bad = int(bad.any(1).sum())
    if n_bad:
        raise RuntimeError(f"ground truth: the library's exact (m = B) search disagrees with the "
                           f"oracle's brute force on {n_bad} of {len(samp)} sampled queries")
    check = {"truth": "oracle brute force (fp64 order)", "queries": int(len(samp)),
             "library_m_eq_B_agrees": True}
    return gt, g64, cnt, check


def exact_dist(rows, q, metric):
    """fp64 squared L2 distance (or inner product) of each row to q."""
    r = rows.astype(np.float64)
    qq = q.astype(np.float64)
    return ((r - qq) ** 2).sum(1) if metric == 0 else r @ qq


def recall_at_k(ids, gt, g64, cnt, k, X, Q, metric=0):
    """RecallK@K over the sampled queries, two readings: strict (returned ids
    in the true top-k, divided by min(k, |D_C|)); tie-aware (a returned id
    whose exact distance is no worse than the true k-th counts).  Returns the
    two means."""
    strict, tie = [], []
    for q in range(ids.shape[0]):
        den = int(min(k, cnt[q]))
        if den == 0:
            strict.append(1.0)
            tie.append(1.0)
            continue
        got = ids[q, :k][ids[q, :k] >= 0]
        strict.append(len(set(gt[q, :den].tolist()).intersection(got.tolist())) / den)
        d = exact_dist(X[got], Q[q], metric) if len(got) else np.zeros(0)
        kth = g64[q, den - 1]
        hits = int((d <= kth).sum() if metric == 0 else (d >= kth).sum())
        tie.append(min(hits, den) / den)
    return float(np.mean(strict)), float(np.mean(tie))


def query_stats(w, rows_scanned, rows_passed):
    """Selectivity |D_C| / N of the batch's filters (percentiles and a
    per-decade histogram) and the mean candidates per query of the measured
    probe count: rows in the selected blocks, and rows passing the filter."""
    sel = np.asarray(w.selectivity, dtype=np.float64) if w.selectivity is not None else None
    out = {"rows_selected_per_query": round(float(rows_scanned) / w.nq, 1),
           "rows_passing_per_query": round(float(rows_passed) / w.nq, 1)}
    if sel is not None and sel.size:
        edges = [0.0, 1e-4, 1e-3, 1e-2, 1e-1, 1.0 + 1e-12]
        hist = np.histogram(sel, bins=edges)[0]
        out["selectivity"] = {
            "p0": float(sel.min()), "p50": float(np.median(sel)), "p100": float(sel.max()),
            "mean": float(sel.mean()),
            "hist": {"<0.01%": int(hist[0]), "0.01-0.1%": int(hist[1]), "0.1-1%": int(hist[2]),
                     "1-10%": int(hist[3]), ">=10%": int(hist[4])}}
    return out


ABLATION_M_SWEEP = M_SWEEP + (96, 128, 192, 256)


def qps_at_recall(caps, torch, ix, w, samp, gt, g64, cnt, flush, m_sweep=ABLATION_M_SWEEP, target=0.9,
                  reps=5, nq=None, k=None):
    """Smallest probe count in m_sweep whose tie-aware recall@k on the sample
    reaches the target, and the batch QPS there (device buffers, CUDA events,
    L2 flushed before each timed search).  Returns a small dict."""
    k = k or w.k
    nq = nq or w.nq
    Qd = torch.from_numpy(np.ascontiguousarray(w.Q[:nq])).cuda()
    Qbd = torch.from_numpy(np.ascontiguousarray(w.Qb[:nq])).cuda() if w.Qb is not None else \
        (torch.from_numpy(w.q_off).cuda(), torch.from_numpy(w.q_lab).cuda())
    ids = torch.empty((nq, k), dtype=torch.int64, device="cuda")
    dist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    row = {"m": None}
    for m in m_sweep:
        ix.search(Qd, Qbd, k, m, out_ids=ids, out_dist=dist)
        _, tie = recall_at_k(ids.cpu().numpy()[samp], gt, g64, cnt, k, w.X, w.Q[samp], w.metric)
        if tie >= target:
            ms = time_search(torch, lambda: ix.search(Qd, Qbd, k, m, out_ids=ids, out_dist=dist),
                             flush, reps)
            row = {"m": m, "recall_tie": round(tie, 4), "qps": round(nq / (ms / 1e3), 1)}
            break
        row = {"m": None, "recall_tie_at_max_m": round(tie, 4)}
    return row


def time_search(torch, fn, flush, reps=5, warm=2):
    """Median device time (ms) of fn(), L2 flushed before each timed call."""
    for _ in range(warm):
        fn()
    evs = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in evs]))


def ablations(args, w, caps, torch, flush):
    """Sec. 6.1 ablations and the appendix's longer attribute vectors, on
    k-means + bf16 indexes (the same seed points) of the 1M x 128 data:
    QPS at recall@10 >= 0.9 for (1) AFT heights h (blocks h+1), (2) queries
    constraining exactly 3, 2 or 1 of the 3 fields (absence fraction 0,
    1/3, 2/3), (3) 10 attribute fields instead of 3 (queries constrain 1-3
    of them) and 100 fields as label sets (1,000 queries, each field kept
    with probability 0.03).  Ground truth of a 300-query sample from the
    oracle's brute force for every query set."""
    from workloads import config_sift1m_fields, with_constraints
    rng = np.random.default_rng(9)
    samp = np.sort(rng.choice(w.nq, 300, replace=False))

    def build(wl, h=None):
        return caps.Index.build(torch.from_numpy(wl.X).cuda(), torch.from_numpy(wl.A).cuda(),
                                wl.vocab, wl.B, h=wl.h if h is None else h, iters=wl.iters,
                                init_idx=wl.init_idx, prec=caps.BF16)

    out = {"index": "k-means + bf16", "h": [], "constrained_fields": [], "attribute_fields": []}
    gt = oracle_truth(w, samp)
    for h in (0, 1, 3, 7, 15, 31):
        ix = build(w, h)
        out["h"].append({"h": h, **qps_at_recall(caps, torch, ix, w, samp, *gt, flush)})
        ix.close()
    ix = build(w)
    for c in (3, 2, 1):
        wc = with_constraints(w, c, c, 4000 + c, sel_range=(0.001, 0.30))
        out["constrained_fields"].append(
            {"constrained": c, "absence_fraction": round((3 - c) / 3, 3),
             **qps_at_recall(caps, torch, ix, wc, samp, *oracle_truth(wc, samp), flush)})
    ix.close()
    for L in (10,):
        wl = config_sift1m_fields(L)
        ix = build(wl)
        out["attribute_fields"].append(
            {"L": L, "attr_words": int(ix.info.attr_words),
             **qps_at_recall(caps, torch, ix, wl, samp, *oracle_truth(wl, samp), flush)})
        ix.close()
    # L = 100 (the appendix's longest attribute vectors): too many packed bits
    # for the dense words, so the fields go in as label sets (field f with
    # value v = label f * 100 + v); 1,000 queries keeping each field with
    # probability 0.03
    from workloads import config_sift1m_wide
    t0 = time.perf_counter()
    wl = config_sift1m_wide(100, nq=1000, base=w)
    gen_s = time.perf_counter() - t0
    samp100 = np.sort(rng.choice(wl.nq, 300, replace=False))
    ix = caps.Index.build(torch.from_numpy(wl.X).cuda(), None, None, wl.B, h=wl.h, iters=wl.iters,
                          init_idx=wl.init_idx, prec=caps.BF16,
                          labels=(wl.sp_off, wl.sp_lab, wl.sp_vocab))
    out["attribute_fields"].append(
        {"L": 100, "form": "label sets", "queries_per_step": wl.nq, "generate_s": round(gen_s, 1),
         **qps_at_recall(caps, torch, ix, wl, samp100, *oracle_truth(wl, samp100), flush)})
    ix.close()
    out["attribute_fields"].insert(0, {"L": 3, **{k_: v_ for k_, v_ in out["h"][4].items()
                                                   if k_ != "h"}})
    return out


def sparse_line(args, caps, torch, flush):
    """Label-set workload (2M x 128 fp32 mixture, 10,000-label vocabulary,
    1-20 labels per point, queries requiring 1-8 labels).  Per index form
    (fp32, bf16): build time, recall@10 and QPS over a probe sweep, the
    smallest m reaching recall@10 >= 0.9, and the QPS there for batches of
    1, 16, 256 and 4,096 queries; for the fp32 index also k = 100 (recall@100
    >= 0.9).  Recall against the oracle's brute force on a 200-query sample;
    device buffers, CUDA events, L2 flushed before each timed search."""
    from workloads import config_sparse2m
    t0 = time.perf_counter()
    w = config_sparse2m()
    gen_s = time.perf_counter() - t0
    rng = np.random.default_rng(6)
    samp = np.sort(rng.choice(w.nq, 200, replace=False))
    gt10 = exact_truth(caps, torch, w, samp, labels=True)[:3]
    gt100 = oracle_truth(w, samp, k=100)
    Qd = torch.from_numpy(w.Q).cuda()
    qoff = torch.from_numpy(w.q_off).cuda()
    qlab = torch.from_numpy(w.q_lab).cuda()
    out = {"workload": w.name, "N": w.N, "d": w.d, "labels": int(w.sp_vocab),
           "queries_per_step": w.nq, "generate_s": round(gen_s, 1), "paths": {}}

    def sub(nq):  # the first nq queries' label lists
        end = int(w.q_off[nq])
        return (torch.from_numpy(np.ascontiguousarray(w.q_off[:nq + 1])).cuda(),
                torch.from_numpy(np.ascontiguousarray(w.q_lab[:end])).cuda())

    for name, prec in (("fp32", caps.FP32), ("bf16", caps.BF16)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = caps.Index.build(torch.from_numpy(w.X).cuda(), None, None, w.B, h=w.h,
                              iters=w.iters, init_idx=w.init_idx, prec=prec,
                              labels=(w.sp_off, w.sp_lab, w.sp_vocab))
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t0
        res = {"build_s": round(build_s, 2)}
        for k, gt, label in ((10, gt10, "k10"), (100, gt100, "k100")):
            if k == 100 and name != "fp32":
                continue  # k > 32 runs the fp32 scan on a bf16 index too
            ids = torch.empty((w.nq, k), dtype=torch.int64, device="cuda")
            dist = torch.empty((w.nq, k), dtype=torch.float32, device="cuda")
            sweep, chosen = [], None
            for m in SPARSE_M_SWEEP:
                ix.search(Qd, (qoff, qlab), k, m, out_ids=ids, out_dist=dist)
                _, tie = recall_at_k(ids.cpu().numpy()[samp], *gt, k, w.X, w.Q[samp], w.metric)
                ms = time_search(torch, lambda: ix.search(Qd, (qoff, qlab), k, m, out_ids=ids,
                                                          out_dist=dist), flush)
                sweep.append({"m": m, "recall_tie": round(tie, 4),
                              "qps": round(w.nq / (ms / 1e3), 1)})
                if chosen is None and tie >= 0.9:
                    chosen = m
                    break
            row = {"m_at_0.9": chosen, "sweep": sweep}
            if chosen is not None and k == 10:
                bq = {}
                for nb in (1, 16, 256, 4096):
                    qc, lc = Qd[:nb], sub(nb)
                    bi = torch.empty((nb, k), dtype=torch.int64, device="cuda")
                    bd = torch.empty((nb, k), dtype=torch.float32, device="cuda")
                    ms = time_search(torch, lambda: ix.search(qc, lc, k, chosen, out_ids=bi,
                                                              out_dist=bd), flush, reps=7)
                    bq[str(nb)] = {"qps": round(nb / (ms / 1e3), 1), "ms": round(ms, 4)}
                row["batches"] = bq
            res[label] = row
        out["paths"][name] = res
        ix.close()
    return out


LEARNED4M_M_SWEEP = (1, 2, 4, 8, 12, 16, 24, 32, 48, 64, 96, 128)


def learned4m_line(args, caps, torch, flush):
    """The learned-partitioner workload (4M x 96 unit vectors, inner product,
    5 fields, B = 1024): k-means against the MLP 96 -> 512 -> 1024 trained on
    filtered-neighbour labels with bf16 weights and fp32 masters (one round
    with argmax; a shorter training, also with the fp32 training step; two
    BLISS rounds with the balanced assignment over 8 logits), all bf16
    indexes; per
    index its build time, the largest partition, the recall@10 / QPS sweep
    over m and the QPS at recall@10 >= 0.9 (the comparison at equal recall),
    plus the build's own arbiter (k-means fallback).  Recall against the
    oracle's brute force on a 200-query sample."""
    from workloads import config_learned4m
    t0 = time.perf_counter()
    w = config_learned4m()
    gen_s = time.perf_counter() - t0
    rng = np.random.default_rng(8)
    samp = np.sort(rng.choice(w.nq, 200, replace=False))
    t0 = time.perf_counter()
    gt = oracle_truth(w, samp)
    truth_s = time.perf_counter() - t0
    X = torch.from_numpy(w.X).cuda()
    A = torch.from_numpy(w.A).cuda()
    Qd = torch.from_numpy(w.Q).cuda()
    Qbd = torch.from_numpy(w.Qb).cuda()
    ids = torch.empty((w.nq, w.k), dtype=torch.int64, device="cuda")
    dist = torch.empty((w.nq, w.k), dtype=torch.float32, device="cuda")
    mlp = dict(part=caps.MLP, mlp_hidden=512, mlp_epochs=40, mlp_samples=524288,
               mlp_batch=4096, mlp_lr=1e-3, mlp_label_k=10, seed=17, mlp_arbiter_queries=1000,
               mlp_arbiter_m=8, mlp_bf16=1)
    variants = (("kmeans", {}), ("learned", mlp),
                ("learned_short", dict(mlp, mlp_epochs=20, mlp_samples=131072, mlp_lr=2e-3)),
                ("learned_fp32_training", dict(mlp, mlp_epochs=20, mlp_samples=131072, mlp_lr=2e-3,
                                               mlp_bf16=0)),
                ("learned_balanced", dict(mlp, mlp_rounds=2, mlp_balance_r=8)))
    out = {"workload": w.name, "N": w.N, "d": w.d, "B": w.B, "metric": "ip",
           "queries_per_step": w.nq, "generate_s": round(gen_s, 1),
           "truth_s": round(truth_s, 1), "mlp": "96 -> 512 -> 1024, 524,288 training points, "
           "40 epochs, Adam lr 1e-3, 10-NN filtered labels, bf16 weights / fp32 masters "
           "(learned_short: 131,072 points, 20 epochs, lr 2e-3)", "paths": {}}
    for name, extra in variants:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = caps.Index.build(X, A, w.vocab, w.B, h=w.h, iters=w.iters, metric=w.metric,
                              init_idx=w.init_idx, prec=caps.BF16, **extra)
        torch.cuda.synchronize()
        res = {"build_s": round(time.perf_counter() - t0, 2),
               "largest_partition": int(np.bincount(ix.export(caps.ARR_BIN),
                                                    minlength=w.B).max()),
               "mean_partition": w.N // w.B}
        if extra:
            i = ix.info
            res["arbiter"] = {"queries": 1000, "m": 8,
                            "recall_kmeans": round(float(i.arbiter_recall_kmeans), 4),
                            "recall_learned": round(float(i.arbiter_recall_mlp), 4),
                            "kept": "learned" if i.part == caps.MLP else "kmeans"}
        sweep, chosen = [], None
        for m in LEARNED4M_M_SWEEP:
            ix.search(Qd, Qbd, w.k, m, out_ids=ids, out_dist=dist)
            _, tie = recall_at_k(ids.cpu().numpy()[samp], *gt, w.k, w.X, w.Q[samp], w.metric)
            ms = time_search(torch, lambda: ix.search(Qd, Qbd, w.k, m, out_ids=ids,
                                                      out_dist=dist), flush)
            sweep.append({"m": m, "recall_tie": round(tie, 4), "qps": round(w.nq / (ms / 1e3), 1)})
            if tie >= 0.9:
                chosen = sweep[-1]
                break
        res["sweep"] = sweep
        res["at_0.9"] = chosen
        out["paths"][name] = res
        ix.close()
    return out


def oracle_index_of(caps, ix, w):
    """The oracle's own index over the partitions of a built library index:
    the oracle runs Alg. 1's second level itself (attribute-frequency trees
    and layout) from the library's f(x_i) (ARR_BIN), and for a learned
    partitioner also takes the trained network, whose m largest fp32 logits
    it computes itself per query (Alg. 2 probe).  So the CPU times the same
    index, probe rule and m as the GPU; only the first-level training
    (k-means, network) is not redone on the host cores.
    Returns (oracle index, network or None)."""
    import oracle as O
    bins = ix.export(caps.ARR_BIN)
    net = None
    if ix.info.part == caps.MLP:
        H, d, B = ix.info.mlp_hidden, w.d, w.B
        Wf = ix.export(caps.ARR_MLP)
        net = O.MLP(Wf[:H * d].reshape(H, d), Wf[H * d:H * d + H],
                    Wf[H * d + H:H * d + H + B * H].reshape(B, H), Wf[H * d + H + B * H:])
        oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, w.metric, bins=bins)
    else:
        oi = O.build(w.X, O.Attrs.of(w), w.B, w.h, 0, w.init_idx, w.metric,
                     C=ix.export(caps.ARR_CENTROIDS))
    return oi, net


def oracle_query(w, at, oi, net, sub, m):
    """One batch of Alg. 2 on the host cores: the probe (the network's m
    largest logits, or the m nearest centroids inside the oracle's search),
    block selection, filtered scan and top-k."""
    import oracle as O
    Q = np.ascontiguousarray(w.Q[sub])
    probe_in = O.probe_logits(Q, net, m) if net is not None else None
    return O.search(w.X, at, oi, Q, O.Cons(Qb=w.Qb[sub]), w.k, m, probe_in=probe_in)


def oracle_baseline(caps, ix, w, m, budget_s=15.0):
    """CPU oracle (plain C, all host cores) on a bounded sample of queries,
    over the same partitions as the measured library index."""
    import oracle as O
    from oracle.build import build_oracle
    build_oracle()
    cores = O.set_threads(0)
    at = O.Attrs.of(w)
    t0 = time.perf_counter()
    oi, net = oracle_index_of(caps, ix, w)
    build_s = time.perf_counter() - t0
    rng = np.random.default_rng(7)
    order = rng.permutation(w.nq)
    n, done, spent = 256, 0, 0.0
    while done < w.nq and spent < budget_s:
        sub = order[done:done + n]
        t0 = time.perf_counter()
        oracle_query(w, at, oi, net, sub, m)
        spent += time.perf_counter() - t0
        done += len(sub)
        n *= 2
    # one core as well (the paper times its CPU program single-threaded)
    one = order[:500]
    O.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle_query(w, at, oi, net, one, m)
        one_s = time.perf_counter() - t0
    finally:
        O.set_threads(cores)
    part = "learned partitioner's logits" if net is not None else "k-means centroids"
    return {"value": done / spent, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} of {w.nq} queries at m={m}, k={w.k}; the oracle's index laid out "
                      f"by the oracle from the measured GPU index's partitions (probe: the "
                      f"{part}; {build_s:.1f} s, untimed)",
            "single_core": {"value": len(one) / one_s, "unit": UNIT, "cores": 1,
                            "sample": f"{len(one)} of the same queries"}}


# the probe count at which the headline (learned + bf16) reaches recall@10
# >= 0.9 on this workload: the reference arm's m unless one is given
REFERENCE_M = 16


def max_over_ranks(x, world, device):
    """The largest value of x over the ranks (the slowest rank's time), or x
    itself on one rank; every rank gets the same result."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, nq, seconds):
    """Whole-job queries/s: each of the world ranks answered nq queries, the
    slowest of them in `seconds`."""
    return world * nq / seconds


def headline_config(w, m, path, world):
    """The `config` object of both arms' JSON lines (the same workload, index,
    probe count and batch)."""
    return {"workload": w.name, "N": w.N, "d": w.d, "L": int(w.A.shape[1]), "B": w.B, "h": w.h,
            "kmeans_iters": w.iters, "m": m, "k": w.k, "path": path,
            "partitioner": "mlp 128-512-1024" if path.startswith("mlp") else "k-means",
            "queries_per_step": w.nq, "l2": "flushed between timed steps (256 MB write)",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def build_index(caps, torch, w, path):
    """Alg. 1 on the GPU for one of the search paths (precision, partitioner)."""
    prec, part = {"fp32": (caps.FP32, caps.KMEANS), "bf16": (caps.BF16, caps.KMEANS),
                  "fp8": (caps.FP8, caps.KMEANS), "mlp_fp32": (caps.FP32, caps.MLP),
                  "mlp_bf16": (caps.BF16, caps.MLP), "mlp_fp8": (caps.FP8, caps.MLP)}[path]
    X = torch.from_numpy(w.X).cuda()
    A = torch.from_numpy(w.A).cuda()
    extra = MLP_ARGS if part == caps.MLP else {}
    return caps.Index.build(X, A, w.vocab, w.B, h=w.h, iters=w.iters, metric=w.metric,
                            init_idx=w.init_idx, prec=prec, part=part, **extra)


def run_reference(args):
    """The reference arm: the CPU oracle (plain C restatement of Alg. 2 with
    OpenMP over queries) times whole 10,000-query batches on the host cores,
    over the index of the headline path -- its partitions built on the GPU
    (k-means / network training are untimed set-up), its attribute-frequency
    trees, layout, probes, selections and scans all the oracle's own."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import torch
    import oracle as O
    from oracle.build import build_oracle
    from paper_2308_15014_gb300 import build as capsbuild
    build_oracle()
    capsbuild.build()
    import paper_2308_15014_gb300 as caps
    torch.cuda.set_device(0)
    w = load_workload(args.config)
    path = [p for p in args.paths.split(",") if p][0]
    # the probe count of the headline line on this workload (the smallest m
    # at which the learned bf16 path reaches recall@10 >= 0.9), unless given
    m = args.m or REFERENCE_M
    ix = build_index(caps, torch, w, path)
    torch.cuda.synchronize()
    oi, net = oracle_index_of(caps, ix, w)
    ix.close()
    at = O.Attrs.of(w)
    cores = O.set_threads(0)
    allq = np.arange(w.nq)
    for _ in range(args.warmup):
        oracle_query(w, at, oi, net, allq, m)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_query(w, at, oi, net, allq, m)
        times.append(time.perf_counter() - t0)
    v = w.nq * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": headline_config(w, m, path, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"all {w.nq} queries per step at m={m}; the oracle's "
                                       "index laid out by the oracle from the GPU-built "
                                       "partitions of the same path (untimed set-up)"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line, default=_json_default), flush=True)
    return 0


# the e4m3 form re-scores 16 k candidates per query exactly (its tile scores
# carry about 1 % error, so the right neighbours rank lower than with bf16)
FP8_RERANK_FACTOR = 16

# learned partitioner: 128 -> 512 -> 1024 (ReLU), 524,288 training points,
# 10-NN filtered labels, Adam lr 1e-3, batches of 4096, 40 epochs, bf16
# weights and activations with fp32 masters (recall@10 on the bench's sample
# at m = 12 / 16 / 24: 0.894 / 0.911 / 0.930; with 131,072 points, 20 epochs,
# lr 2e-3 and fp32 training it was 0.887 at m = 24 and 0.906 at m = 40)
MLP_ARGS = dict(mlp_hidden=512, mlp_epochs=40, mlp_samples=524288, mlp_batch=4096, mlp_lr=1e-3,
                mlp_label_k=10, seed=17, mlp_bf16=1)


def measure_path(args, w, caps, prec, samp, gt, g64, cnt, flush, world, local, part=0):
    """Build the index in the given precision and partitioner, pick m, time
    the batch."""
    import torch
    import torch.distributed as dist
    X = torch.from_numpy(w.X).cuda()
    A = torch.from_numpy(w.A).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    extra = dict(MLP_ARGS) if part == caps.MLP else {}
    if prec == caps.FP8:
        extra["rerank_factor"] = FP8_RERANK_FACTOR
    ix = caps.Index.build(X, A, w.vocab, w.B, h=w.h, iters=w.iters, metric=w.metric,
                          init_idx=w.init_idx, prec=prec, part=part, **extra)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del X, A
    Qd = torch.from_numpy(w.Q).cuda()
    Qbd = torch.from_numpy(w.Qb).cuda()
    out_ids = torch.empty((w.nq, w.k), dtype=torch.int64, device="cuda")
    out_dist = torch.empty((w.nq, w.k), dtype=torch.float32, device="cuda")

    def search(m):
        ix.search(Qd, Qbd, w.k, m, out_ids=out_ids, out_dist=out_dist)

    sweep, chosen = [], args.m
    for m in ((args.m,) if args.m else M_SWEEP):
        search(m)
        ids = out_ids.cpu().numpy()[samp]
        strict, tie = recall_at_k(ids, gt, g64, cnt, w.k, w.X, w.Q[samp], w.metric)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        search(m)
        ev0.record()
        for _ in range(3):
            search(m)
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / 3
        sweep.append({"m": m, "recall_tie": round(tie, 4), "recall_strict": round(strict, 4),
                      "qps": round(w.nq / (ms / 1e3), 1)})
        if not chosen and tie >= 0.9:
            chosen = m
    m = chosen or M_SWEEP[-1]
    rec = next(x for x in sweep if x["m"] == m)

    # ---- the batch as a tuned, graph-captured plan --------------------------
    # the autotuner times the scan's launch shapes on this batch and the
    # whole query is captured into one CUDA graph; the direct call (same
    # kernels, launched one by one) is timed alongside
    plan = ix.plan(Qd, Qbd, w.k, m, autotune=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    search(m)
    ev0.record()
    for _ in range(3):
        search(m)
    ev1.record()
    torch.cuda.synchronize()
    direct_ms = ev0.elapsed_time(ev1) / 3

    def run(m):
        plan.search(Qd, Qbd, out_ids=out_ids, out_dist=out_dist)

    run(m)
    torch.cuda.synchronize()
    p_ids = out_ids.cpu().numpy()[samp]
    p_dist = out_dist.cpu().numpy()[samp]
    search(m)
    assert np.array_equal(p_ids, out_ids.cpu().numpy()[samp]), "plan and direct call disagree"

    # ---- timed region: K batches, L2 flushed between them -------------------
    for _ in range(args.warmup):
        run(m)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    with Clocks(local) as clk:
        for e0, e1 in evs:
            flush.zero_()
            e0.record()
            run(m)
            e1.record()
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(float(np.mean([e0.elapsed_time(e1) for e0, e1 in evs])), world, "cuda")
    value = job_throughput(world, w.nq, ms / 1e3)

    # ---- per-stage device times (events on the launching stream) -----------
    caps.set_timing(True)
    stage, reps = {}, 5
    for _ in range(reps):
        flush.zero_()
        search(m)
        st = caps.stage_times()
        for kk, vv in st.items():
            stage[kk] = stage.get(kk, 0.0) + vv / reps
    caps.set_timing(False)
    launches = int(round(stage.pop("launches")))
    return dict(ix=ix, plan=plan, m=m, rec=rec, sweep=sweep, value=value, ms=ms, stage=stage,
                launches=launches, build_s=build_s, clocks=clk.summary(),
                direct_ms=direct_ms, tuning=plan.info, ids_s=p_ids, dist_s=p_dist)


def run_caps(args):
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2308_15014_gb300 import build as capsbuild
    capsbuild.build()
    import paper_2308_15014_gb300 as caps

    w = load_workload(args.config)
    # recall on a seeded sample of queries against their exact filtered kNN
    rng = np.random.default_rng(5)
    samp = np.sort(rng.choice(w.nq, min(RECALL_SAMPLE, w.nq), replace=False))
    gt, g64, cnt, truth_check = exact_truth(caps, torch, w, samp)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    kinds = {"fp32": (caps.FP32, caps.KMEANS), "bf16": (caps.BF16, caps.KMEANS),
             "fp8": (caps.FP8, caps.KMEANS), "fp32_split": (caps.FP32_SPLIT, caps.KMEANS),
             "mlp_fp32": (caps.FP32, caps.MLP), "mlp_bf16": (caps.BF16, caps.MLP),
             "mlp_fp8": (caps.FP8, caps.MLP), "mlp_fp32_split": (caps.FP32_SPLIT, caps.MLP)}
    paths = [p for p in args.paths.split(",") if p]
    res = {}
    for pth in paths:
        prec, part = kinds[pth]
        res[pth] = measure_path(args, w, caps, prec, samp, gt, g64, cnt, flush, world, local,
                                part=part)
    head = res[paths[0]]
    ix, m, stage = head["ix"], head["m"], head["stage"]

    # ---- algorithmic work of the scan (the dominant kernel) ----------------
    perm = ix.export(caps.ARR_PERM)
    offsets = ix.export(caps.ARR_OFFSETS)
    probe = ix.probe(w.Q, m)
    sel = ix.select(probe, w.Qb)
    split_head = paths[0].endswith("split")
    union, per_query, rows_scanned, rows_passed = scan_traffic_bytes(
        w, perm, offsets, probe, sel, ix.info.attr_words, bf16=paths[0].endswith("bf16"),
        split=split_head)
    hbm, hbm_src = peaks()
    scan_s = stage["scan_ms"] / 1e3
    tc_head = paths[0].endswith("bf16") or split_head
    d_items, d_rows, d_pairs = dense_item_stats(w, offsets, probe, sel, 128 if tc_head else 32)
    achieved_gbs = union / scan_s / 1e9
    if tc_head:
        # the scan's roofline: the HBM floor of the batch -- every selected
        # row's bf16 vector, attribute words, id and norm once (the bytes the
        # method must move) -- over the scan's CUDA-event time, against the
        # measured copy bandwidth; traffic = ncu DRAM bytes of one launch of
        # the same kernel source at this m
        roof = {"kernel": TC_KERNEL, "bound": "hbm", "achieved": round(achieved_gbs, 1),
                "peak": hbm, "peak_source": hbm_src, "unit": "GB/s",
                "frac": round(achieved_gbs / hbm, 4),
                "traffic": traffic_from_profile(TC_KERNEL, TC_SRC, m,
                                                "split" if split_head else "bf16"),
                "algorithmic_bytes": union, "algorithmic_bytes_per_query_sum": per_query,
                "rows_attr_tested": rows_scanned, "rows_distance": rows_passed,
                "work_items": d_items, "item_union_rows": d_rows, "item_dense_pairs": d_pairs}
        # the method's own distance work (2d flop per filter-passing pair)
        # against the bf16 tensor peak; the tensor cores evaluate every
        # (probe, row) pair of each work item (item_dense_pairs)
        flops = rows_passed * w.d * 2
        tflops = flops / scan_s / 1e12
        bf16_peak, bf16_src = bf16_peak_tflops()
        roof_other = {"kernel": TC_KERNEL, "bound": "tensor", "achieved": round(tflops, 3),
                      "peak": bf16_peak, "peak_source": bf16_src, "unit": "TFLOP/s",
                      "frac": round(tflops / bf16_peak, 5), "algorithmic_flops": flops,
                      "dense_flops_evaluated": d_pairs * w.d * 2}
        other_key = "roofline_tensor"
    else:
        flops = rows_passed * w.d * (3 if w.metric == 0 else 2)
        tflops = flops / scan_s / 1e12
        roof = {"kernel": SCAN_KERNEL, "bound": "alu", "achieved": round(tflops, 2),
                "peak": round(FP32_PEAK_TFLOPS, 1),
                "peak_source": "derived: 152 SMs x 128 fp32 lanes x 2 flop x 2.07 GHz",
                "unit": "TFLOP/s", "frac": round(tflops / FP32_PEAK_TFLOPS, 4),
                "traffic": traffic_from_profile(SCAN_KERNEL, SCAN_SRC, m), "algorithmic_flops": flops,
                "rows_attr_tested": rows_scanned, "rows_distance": rows_passed}
        roof_other = {"kernel": roof["kernel"], "bound": "hbm", "achieved": round(achieved_gbs, 1),
                      "peak": hbm, "peak_source": hbm_src, "unit": "GB/s",
                      "frac": round(achieved_gbs / hbm, 4), "algorithmic_bytes_union": union,
                      "algorithmic_bytes_per_query_sum": per_query}
        other_key = "roofline_hbm"

    # ---- end to end: pinned host buffers through the plan's C-ABI call -----
    plan = head["plan"]
    Qh = torch.from_numpy(np.ascontiguousarray(w.Q)).pin_memory()
    Qbh = torch.from_numpy(np.ascontiguousarray(w.Qb)).pin_memory()
    ids_h = torch.empty((w.nq, w.k), dtype=torch.int64).pin_memory()
    dist_h = torch.empty((w.nq, w.k), dtype=torch.float32).pin_memory()
    for _ in range(args.warmup):
        plan.search(Qh, Qbh, out_ids=ids_h, out_dist=dist_h)
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.search(Qh, Qbh, out_ids=ids_h, out_dist=dist_h)  # returns after the D2H copies
        e2e_t.append(time.perf_counter() - t0)
    e2e_v = job_throughput(world, w.nq, max_over_ranks(float(np.mean(e2e_t)), world, "cuda"))

    # ---- form 1: bf16 / e4m3 tile scores and returned distances against fp64 -
    from workloads import make_dense_workload
    wf = make_dense_workload(name="float_mixture", N=20_000, d=w.d, ncomp=100,
                             center=("uniform", 128.0), sigma=16.0, vocab=[20, 50, 100],
                             zipf_s=1.0, nq=200, cmin=1, cmax=3, B=64, h=15, iters=1, m=4,
                             k=10, seed=77, integer=False)
    hid, hdist = head["ids_s"], head["dist_s"]
    okm = hid >= 0
    qs = np.repeat(samp[:, None], hid.shape[1], 1)[okm]
    d64 = ((w.X[hid[okm]].astype(np.float64) - w.Q[qs].astype(np.float64)) ** 2).sum(1)
    rel = np.abs(hdist[okm].astype(np.float64) - d64) / np.maximum(d64, 1e-30)
    form1 = {"tile_score_vs_fp64": {w.name: form1_error(w), "float_mixture_d128": form1_error(wf)},
             "returned_dist_vs_fp64": {"pairs": int(rel.size), "max_rel": float(rel.max()),
                                       "mean_rel": float(rel.mean())}}
    sparse = sparse_line(args, caps, torch, flush) if not args.no_sparse and world == 1 else None
    abl = ablations(args, w, caps, torch, flush) if not args.no_ablations and world == 1 else None
    l4m = learned4m_line(args, caps, torch, flush) if not args.no_learned4m and world == 1 \
        else None

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_baseline(caps, ix, w, m)
    others = {}
    for pth in paths[1:]:
        r = res[pth]
        others[pth] = {"value": round(r["value"], 1), "m": r["m"], "ms_per_step": round(r["ms"], 4),
                       "recall_at_10": {"tie_aware": r["rec"]["recall_tie"],
                                        "strict": r["rec"]["recall_strict"]},
                       "stage_ms": {k_: round(v_, 4) for k_, v_ in r["stage"].items()},
                       "sweep": r["sweep"], "build_s": round(r["build_s"], 3),
                       "direct_call_ms": round(r["direct_ms"], 4), "tuning": r["tuning"]}
    line = {
        "metric": METRIC, "value": round(head["value"], 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(head["ms"], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp8": "e4m3"}.get(paths[0].split("_")[-1], "f32"),
        "data": "synthetic",
        "config": headline_config(w, m, paths[0], world),
        "recall_at_10": {"tie_aware": head["rec"]["recall_tie"],
                         "strict": head["rec"]["recall_strict"], "sample_queries": int(len(samp)),
                         "truth": truth_check},
        "sweep": head["sweep"],
        "build_s": round(head["build_s"], 3),
        "stage_ms": {k_: round(v_, 4) for k_, v_ in stage.items()},
        "timing": "one CUDA-graph replay of a tuned plan per step (caps_plan_search, device "
                  "buffers); stage_ms from the same kernels launched directly with stage events",
        "direct_call_ms": round(head["direct_ms"], 4),
        "tuning": head["tuning"],
        "roofline": roof,
        other_key: roof_other,
        "other_paths": others,
        "e2e": {"value": round(e2e_v, 1), "unit": UNIT,
                "h2d_bytes_per_step": int(Qh.nbytes + Qbh.nbytes),
                "d2h_bytes_per_step": int(ids_h.nbytes + dist_h.nbytes)},
        "gpu_launches": head["launches"] * args.steps,
        "clocks": head["clocks"],
        "cpu_baseline": cpu,
        "form1_error": form1,
        "queries": query_stats(w, rows_scanned, rows_passed),
    }
    if sparse is not None:
        line["label_sets"] = sparse
    if abl is not None:
        line["ablations"] = abl
    if l4m is not None:
        line["learned_4m"] = l4m
    print(json.dumps(line, default=_json_default), flush=True)
    for r in res.values():
        r["plan"].close()
        r["ix"].close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_caps(args)


if __name__ == "__main__":
    sys.exit(main())
