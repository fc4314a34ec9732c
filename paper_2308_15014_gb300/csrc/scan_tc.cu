// Host side of the BF16 tensor-core form of the CAPS scan: bf16 copies of
// the queries and rows, grouping of the probes into work items, the
// persistent scan launch (explicit-filter instantiations here, the penalty
// form in scan_tc_pen.cu), and the per-query merge with an exact fp32
// re-rank of the best rerank_factor * k candidates (coordinates in order,
// one fma each) before the final top-k.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <type_traits>

#include "scan_tc_kernel.cuh"

#include <cuda_fp8.h>

namespace caps {
namespace {

// ---- e4m3 rows (form 1, per-row scale) --------------------------------------
// Scale of a row: max |x_j| / 448 (the largest finite e4m3 value), 1 for a
// zero row; coordinate j is stored as e4m3(x_j / scale), round to nearest
// even, saturating.
__device__ __forceinline__ float f8_scale(float amax) { return amax > 0.f ? amax / 448.f : 1.f; }
__device__ __forceinline__ uint8_t f8_code(float v) {
  return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
}
// one warp per query: e4m3 copy (cols bytes, zero padded), the scale, and
// the fp32 squared norm over the coordinates in order (one fma each)
__global__ void k_query_fp8(const float* __restrict__ Q, int64_t nq, int d,
                            uint8_t* __restrict__ Qh, float* __restrict__ qs,
                            float* __restrict__ qn) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= nq) return;
  const float* x = Q + q * d;
  float amax = 0.f;
  for (int j = lane; j < d; j += 32) amax = fmaxf(amax, fabsf(x[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const float sc = f8_scale(amax);
  for (int j = lane; j < d; j += 32) Qh[q * d + j] = f8_code(x[j] / sc);
  if (lane == 0) {
    float acc = 0.f;
    for (int j = 0; j < d; j++) acc = fmaf(x[j], x[j], acc);
    qn[q] = acc;
    qs[q] = sc;
  }
}
// one thread per row: e4m3 row (cols bytes, zero padded), its scale and its
// fp32 squared norm (coordinates in order, one fma each)
__global__ void k_rows_fp8(const float* __restrict__ Xp, int64_t N, int d, int cols,
                           uint8_t* __restrict__ Xb, float* __restrict__ xn,
                           float* __restrict__ xs) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const float* x = Xp + r * d;
  float amax = 0.f, acc = 0.f;
  for (int j = 0; j < d; j++) {
    amax = fmaxf(amax, fabsf(x[j]));
    acc = fmaf(x[j], x[j], acc);
  }
  const float sc = f8_scale(amax);
  uint8_t* row = Xb + r * cols;
  for (int j = 0; j < d; j++) row[j] = f8_code(x[j] / sc);
  for (int j = d; j < cols; j++) row[j] = 0;
  xn[r] = acc;
  xs[r] = sc;
}

// ---- bf16 query copy and fp32 squared norms -------------------------------
// split: rows of 2*hcols bf16, hi = bf16(q) in [0, d), lo = bf16(q - hi) in
// [hcols, hcols + d), zeros elsewhere
__global__ void k_query_bf16(const float* __restrict__ Q, int64_t nq, int d, int split,
                             __nv_bfloat16* __restrict__ Qh, float* __restrict__ qn) {
  // one warp per query: coalesced bf16 conversion, then lane 0 forms the
  // squared norm over the coordinates in order (one fma each)
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (q >= nq) return;
  const float* x = Q + q * d;
  if (split) {
    const int hcols = (d + 63) / 64 * 64;
    __nv_bfloat16* o = Qh + q * 2 * hcols;
    for (int j = lane; j < hcols; j += 32) {
      const float v = j < d ? x[j] : 0.f;
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      o[j] = hi;
      o[hcols + j] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
  } else {
    for (int j = lane; j < d; j += 32) Qh[q * d + j] = __float2bfloat16_rn(x[j]);
  }
  if (lane == 0) {
    float acc = 0.f;
    for (int j = 0; j < d; j++) acc = fmaf(x[j], x[j], acc);
    qn[q] = acc;
  }
}

// ---- per-query merge of the m candidate lists (keys out) -------------------
template <int KPL>
struct TopKm {
  uint64_t v[KPL];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int s = 0; s < KPL; s++) v[s] = kEmptyKey;
  }
  __device__ __forceinline__ uint64_t kth(int k) const {
    const int P = k - 1, l = P / KPL, s = P % KPL;
    uint64_t mine = v[0];
#pragma unroll
    for (int u = 1; u < KPL; u++)
      if (u == s) mine = v[u];
    return __shfl_sync(0xffffffffu, mine, l);
  }
  __device__ __forceinline__ void insert(uint64_t x, int lane) {
    int p = 0;
#pragma unroll
    for (int s = 0; s < KPL; s++) p += __popc(__ballot_sync(0xffffffffu, v[s] < x));
    const uint64_t prev_last = __shfl_up_sync(0xffffffffu, v[KPL - 1], 1);
    uint64_t nv[KPL];
#pragma unroll
    for (int s = 0; s < KPL; s++) {
      const int P = lane * KPL + s;
      const uint64_t before = (s == 0) ? prev_last : v[s - 1];
      nv[s] = P < p ? v[s] : (P == p ? x : before);
    }
#pragma unroll
    for (int s = 0; s < KPL; s++) v[s] = nv[s];
  }
  __device__ __forceinline__ void offer(uint64_t key, uint64_t& kthv, int k, int lane) {
    unsigned cand = __ballot_sync(0xffffffffu, key < kthv);
    while (cand) {
      const int src = __ffs(cand) - 1;
      cand &= cand - 1;
      const uint64_t x = __shfl_sync(0xffffffffu, key, src);
      if (x < kthv) {
        insert(x, lane);
        kthv = kth(k);
      }
    }
  }
};

// Merge each query's m lists of kp keys, re-score the kp best exactly in
// fp32 (coordinates in order, one fma each) and keep the k best.  When the
// scan stopped on an expired bounded wait (*err set) its lists are not all
// written: every query then gets padding only (the call reports the
// timeout), and no key is read.  The scan's
// per-query bound T (the largest of the query's bound slots, once all are
// set) has at least kp keys of the lists at or below it, so only those keys
// compete: they are compacted and sorted in the warp (up to 128), else the
// lists are merged by insertion.
template <int METRIC, int KPL_K>
__global__ void __launch_bounds__(128)
k_merge_rerank(const uint64_t* __restrict__ part, const uint8_t* __restrict__ dead, int64_t nq,
               int m, int lp, int kp, int k, const uint64_t* __restrict__ qslot, int nslot,
               const float* __restrict__ Q, int d, const float* __restrict__ Xp,
               const int32_t* __restrict__ iperm, int64_t n_rows, int64_t* __restrict__ out_ids,
               float* __restrict__ out_dist, const int32_t* __restrict__ err) {
  // [4][d] queries, [4][kMaxRerank] candidate keys
  extern __shared__ float qsm[];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 4 + wp;
  if (q >= nq) return;
  if (err != nullptr && *reinterpret_cast<const volatile int32_t*>(err) != 0) {
    for (int i = lane; i < k; i += 32) {
      out_ids[q * k + i] = -1;
      out_dist[q * k + i] = METRIC == CAPS_L2 ? INFINITY : -INFINITY;
    }
    return;
  }
  float* qs = qsm + (size_t)wp * d;
  uint64_t* cbuf = reinterpret_cast<uint64_t*>(qsm + 4 * (size_t)d) + (size_t)wp * kMaxRerank;
  for (int j = lane; j < d; j += 32) qs[j] = Q[q * d + j];
  const uint64_t* src = part + q * (int64_t)m * lp;
  const int tot = m * lp;
  const bool live = !dead[q];
  uint64_t T = kEmptyKey;
  if (nslot > 0) {
    T = 0ull;
    for (int i = 0; i < nslot; i++) {
      const uint64_t v = qslot[q * 8 + i];
      T = v > T ? v : T;
    }
  }
  int cnt = 0;
  if (live && T != kEmptyKey) {
    const unsigned lt = (1u << lane) - 1u;
    for (int b0 = 0; b0 < tot; b0 += 32) {
      const uint64_t key = (b0 + lane < tot) ? src[b0 + lane] : kEmptyKey;
      const bool keep = key <= T;
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      const int pos = cnt + __popc(bal & lt);
      if (keep && pos < kMaxRerank) cbuf[pos] = key;
      cnt += __popc(bal);
    }
  }
  __syncwarp();
  // the kp best keys, ascending, at the front of cbuf: the compacted keys
  // sorted in the warp when at most kMaxRerank of them compete, else every
  // list key offered to a warp top-kp
  auto sort_front = [&](auto vtag) {
    constexpr int V = decltype(vtag)::value;
    uint64_t v[V];
#pragma unroll
    for (int s = 0; s < V; s++) v[s] = (V * lane + s < cnt) ? cbuf[V * lane + s] : kEmptyKey;
    warp_sort<V>(v, lane);
    __syncwarp();
#pragma unroll
    for (int s = 0; s < V; s++) cbuf[V * lane + s] = v[s];
  };
  if (live && T != kEmptyKey && cnt <= 64) {
    sort_front(std::integral_constant<int, 2>{});
  } else if (live && T != kEmptyKey && cnt <= 128) {
    sort_front(std::integral_constant<int, 4>{});
  } else if (live && T != kEmptyKey && cnt <= kMaxRerank) {
    sort_front(std::integral_constant<int, kMaxRerank / 32>{});
  } else {
    TopKm<kMaxRerank / 32> cand;
    cand.init();
    uint64_t kthv = kEmptyKey;
    if (live) {
      for (int b0 = 0; b0 < tot; b0 += 32) {
        const uint64_t key = (b0 + lane < tot) ? src[b0 + lane] : kEmptyKey;
        cand.offer(key, kthv, kp, lane);
      }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < kMaxRerank / 32; s++) cbuf[(kMaxRerank / 32) * lane + s] = cand.v[s];
  }
  __syncwarp();
  // exact fp32 scores of the kp candidates, 64 at a time, two per lane (c
  // and c + 32): their rows in 16-byte loads, four per candidate in flight,
  // and their two fma chains interleaved, each over the coordinates in order
  TopKm<KPL_K> top;
  top.init();
  uint64_t kth2 = kEmptyKey;
  for (int c0 = 0; c0 < kp; c0 += 64) {
    uint64_t ck[2];
    const float4* xr[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int c = c0 + lane + 32 * h;
      ck[h] = c < kp ? cbuf[c] : kEmptyKey;
      // (an id outside the rows can only come from a list the scan did not
      // finish; it is dropped, never dereferenced)
      if (ck[h] != kEmptyKey && (int64_t)(uint32_t)(ck[h] & 0xffffffffu) >= n_rows) ck[h] = kEmptyKey;
      xr[h] = reinterpret_cast<const float4*>(Xp);
      if (ck[h] != kEmptyKey)
        xr[h] = reinterpret_cast<const float4*>(Xp + (int64_t)iperm[(uint32_t)(ck[h] & 0xffffffffu)] * d);
    }
    const bool has0 = ck[0] != kEmptyKey, has1 = ck[1] != kEmptyKey;
    float acc0 = 0.f, acc1 = 0.f;
    for (int j0 = 0; j0 < d / 4; j0 += 4) {
      float4 x0[4], x1[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (has0 && j0 + u < d / 4) x0[u] = xr[0][j0 + u];
        if (has1 && j0 + u < d / 4) x1[u] = xr[1][j0 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; u++) {
        if (j0 + u < d / 4) {
          const float4 q4 = *reinterpret_cast<const float4*>(qs + 4 * (j0 + u));
          const float qv[4] = {q4.x, q4.y, q4.z, q4.w};
          const float a0[4] = {x0[u].x, x0[u].y, x0[u].z, x0[u].w};
          const float a1[4] = {x1[u].x, x1[u].y, x1[u].z, x1[u].w};
#pragma unroll
          for (int e = 0; e < 4; e++) {
            if (METRIC == CAPS_L2) {
              const float t0 = a0[e] - qv[e], t1 = a1[e] - qv[e];
              acc0 = fmaf(t0, t0, acc0);
              acc1 = fmaf(t1, t1, acc1);
            } else {
              acc0 = fmaf(a0[e], qv[e], acc0);
              acc1 = fmaf(a1[e], qv[e], acc1);
            }
          }
        }
      }
    }
    const uint64_t k0 = has0 ? make_key(METRIC == CAPS_L2 ? acc0 : -acc0, (uint32_t)(ck[0] & 0xffffffffu))
                             : kEmptyKey;
    const uint64_t k1 = has1 ? make_key(METRIC == CAPS_L2 ? acc1 : -acc1, (uint32_t)(ck[1] & 0xffffffffu))
                             : kEmptyKey;
    top.offer(k0, kth2, k, lane);
    top.offer(k1, kth2, k, lane);
  }
#pragma unroll
  for (int s = 0; s < KPL_K; s++) {
    const int P = lane * KPL_K + s;
    if (P < k) {
      const uint64_t key = top.v[s];
      int64_t id = -1;
      float dist = METRIC == CAPS_L2 ? INFINITY : -INFINITY;
      if (key != kEmptyKey) {
        id = (int64_t)(uint32_t)(key & 0xffffffffu);
        const float sc = unord_bits((uint32_t)(key >> 32));
        dist = METRIC == CAPS_L2 ? sc : -sc;
      }
      out_ids[q * k + P] = id;
      out_dist[q * k + P] = dist;
    }
  }
}

// ---- grouping of the probes by partition -----------------------------------
__global__ void k_bin_count(const int32_t* __restrict__ probe, int64_t ne, int32_t* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ne) atomicAdd(&cnt[probe[i]], 1);
}
__global__ void k_bin_scatter(const int32_t* __restrict__ probe, int64_t ne,
                              int32_t* __restrict__ cursor, int32_t* __restrict__ ent) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ne) ent[atomicAdd(&cursor[probe[i]], 1)] = (int32_t)i;
}
// The same grouping without contended global atomics (B <= kBinShared): G
// blocks each count their slice of the entries in shared memory; a scan over
// the blocks gives every (partition, block) its first output position, and
// each block scatters its slice through shared-memory cursors.
constexpr int GRP_T = 512, kBinShared = 12288, kBinBlocks = 128;
__global__ void __launch_bounds__(GRP_T)
k_bin_hist(const int32_t* __restrict__ probe, int64_t ne, int64_t chunk, int B, int G,
           int32_t* __restrict__ bin_cnt, int32_t* __restrict__ blk) {
  extern __shared__ int h[];
  for (int i = threadIdx.x; i < B; i += GRP_T) h[i] = 0;
  __syncthreads();
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(ne, beg + chunk);
  for (int64_t e = beg + threadIdx.x; e < end; e += GRP_T) atomicAdd(&h[probe[e]], 1);
  __syncthreads();
  for (int i = threadIdx.x; i < B; i += GRP_T) {
    const int c = h[i];
    blk[(int64_t)i * G + blockIdx.x] = c;
    if (c) atomicAdd(&bin_cnt[i], c);
  }
}
// One warp per partition: blk[b][g] becomes bin_off[b] + the counts of the
// blocks before g.
__global__ void k_bin_blockscan(const int32_t* __restrict__ bin_off, int B, int G,
                                int32_t* __restrict__ blk) {
  const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (b >= B) return;
  int carry = bin_off[b];
  for (int g0 = 0; g0 < G; g0 += 32) {
    const int g = g0 + lane;
    const int c = g < G ? blk[(int64_t)b * G + g] : 0;
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (g < G) blk[(int64_t)b * G + g] = carry + inc - c;
    carry += __shfl_sync(0xffffffffu, inc, 31);
  }
}
__global__ void __launch_bounds__(GRP_T)
k_bin_scatter_blk(const int32_t* __restrict__ probe, int64_t ne, int64_t chunk, int B, int G,
                  const int32_t* __restrict__ blk, int32_t* __restrict__ ent) {
  extern __shared__ int cur[];
  for (int i = threadIdx.x; i < B; i += GRP_T) cur[i] = blk[(int64_t)i * G + blockIdx.x];
  __syncthreads();
  const int64_t beg = (int64_t)blockIdx.x * chunk, end = min(ne, beg + chunk);
  for (int64_t e = beg + threadIdx.x; e < end; e += GRP_T) ent[atomicAdd(&cur[probe[e]], 1)] = (int32_t)e;
}

// Within each partition, order the probe entries by a 12-bit code of their
// selected-block mask (lowest block, highest block, number of blocks): probes
// that scan the same blocks end up in the same work item.  One CTA per
// partition: count the codes in shared memory, scan, scatter.  Only the speed
// of the scan depends on this order (equal codes land in any order), never its
// results.
constexpr int TC_MCODES = 4096;
__device__ __forceinline__ int mask_code(uint64_t m) {
  if (m == 0) return 0;
  const int lo = min(15, __ffsll((long long)m) - 1), hi = min(15, 63 - __clzll((long long)m));
  const int n = min(15, __popcll(m));
  return lo | (hi << 4) | (n << 8);
}
__global__ void __launch_bounds__(512)
k_bin_group_mask(const int32_t* __restrict__ bin_off, const uint64_t* __restrict__ sel,
                 const int32_t* __restrict__ ent_in, int32_t* __restrict__ ent_out) {
  __shared__ int cnt[TC_MCODES];
  __shared__ int wsum[16];
  const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int beg = bin_off[b], end = bin_off[b + 1];
  if (end - beg <= 1) {
    if (end > beg && tid == 0) ent_out[beg] = ent_in[beg];
    return;
  }
  for (int i = tid; i < TC_MCODES; i += 512) cnt[i] = 0;
  __syncthreads();
  for (int i = beg + tid; i < end; i += 512) atomicAdd(&cnt[mask_code(sel[ent_in[i]])], 1);
  __syncthreads();
  // exclusive scan of the 4096 counts: 8 per thread, then across threads
  int loc[TC_MCODES / 512], run = 0;
#pragma unroll
  for (int j = 0; j < TC_MCODES / 512; j++) {
    loc[j] = run;
    run += cnt[tid * (TC_MCODES / 512) + j];
  }
  int inc = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  int wbase = 0;
  for (int w = 0; w < warp; w++) wbase += wsum[w];
  const int tbase = beg + wbase + inc - run;
#pragma unroll
  for (int j = 0; j < TC_MCODES / 512; j++) cnt[tid * (TC_MCODES / 512) + j] = tbase + loc[j];
  __syncthreads();
  for (int i = beg + tid; i < end; i += 512) {
    const int e = ent_in[i];
    ent_out[atomicAdd(&cnt[mask_code(sel[e])], 1)] = e;
  }
}

__global__ void k_tc_items_count(const int32_t* __restrict__ bin_off, int B, int cap,
                                 int32_t* __restrict__ cnt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) cnt[b] = (bin_off[b + 1] - bin_off[b] + cap - 1) / cap;
  if (b == B) cnt[B] = 0;
}
__global__ void k_tc_items_fill(const int32_t* __restrict__ bin_off,
                                const int32_t* __restrict__ item_off, int B, int cap,
                                TcItem* __restrict__ items, int32_t* __restrict__ n_items,
                                int32_t* __restrict__ next_item) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == B) {
    *n_items = item_off[B];
    *next_item = 0;
  }
  if (b >= B) return;
  const int c = bin_off[b + 1] - bin_off[b];
  for (int t = 0; t * cap < c; t++) {
    TcItem x;
    x.b = b;
    x.e0 = bin_off[b] + t * cap;
    x.ne = min(cap, c - t * cap);
    x.pad = 0;
    items[item_off[b] + t] = x;
  }
}

// ---- build-side helpers ----------------------------------------------------
// bf16 copy of each row in `cols` columns (vector, zero padding, and in the
// penalty form the 64-column code chunk: a one-hot code of the row's packed
// attribute bits, two columns per bit, then for L2 the row's -|x|^2/2 as
// three bf16 parts that sum to it exactly), its fp32 squared norm
// (coordinates in order, one fma each) and the largest squared norm
// split: the row as two bf16 terms, hi = bf16(x) in columns [0, d) and
// lo = bf16(x - hi) in [hcols, hcols + d), hcols = ceil(d/64)*64
__global__ void k_rows_bf16(const float* __restrict__ Xp, int64_t N, int d, int cols, int kcd,
                            const uint32_t* __restrict__ Ap, int WP, int pen, int pen_bits,
                            uint4 pen_mask, int pen_norm, int split, __nv_bfloat16* __restrict__ Xb,
                            float* __restrict__ xn, unsigned int* __restrict__ xn_max_bits) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  __nv_bfloat16* row = Xb + r * cols;
  for (int j = 0; j < cols; j++) row[j] = __float2bfloat16_rn(0.f);
  const int hcols = (d + 63) / 64 * 64;
  float acc = 0.f;
  for (int j = 0; j < d; j++) {
    const float x = Xp[r * d + j];
    acc = fmaf(x, x, acc);
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    row[j] = hi;
    if (split) row[hcols + j] = __float2bfloat16_rn(x - __bfloat162float(hi));
  }
  xn[r] = acc;
  if (!(acc != acc)) atomicMax(xn_max_bits, __float_as_uint(acc));  // acc >= 0: bits order as floats
  if (!pen) return;
  __nv_bfloat16* code = row + (size_t)kcd * 64;
  const __nv_bfloat16 one = __float2bfloat16_rn(1.f);
  const uint32_t um[4] = {pen_mask.x, pen_mask.y, pen_mask.z, pen_mask.w};
  int gb = 0;
  for (int w = 0; w < WP; w++) {
    uint32_t m = um[w];
    const uint32_t a = Ap[r * WP + w];
    while (m) {
      const int i = __ffs(m) - 1;
      m &= m - 1;
      code[2 * gb + ((a >> i) & 1u)] = one;
      gb++;
    }
  }
  if (pen_norm) {
    // v = -|x|^2/2 = h1 + h2 + h3 exactly: h1 = bf16(v) leaves v - h1 with
    // at most 16 significant bits (exact in fp32), h2 = bf16(v - h1) leaves at
    // most 8, which bf16 holds exactly
    const float v = -0.5f * acc;
    const __nv_bfloat16 h1 = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h1);
    const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(h2);
    code[2 * pen_bits + 0] = h1;
    code[2 * pen_bits + 1] = h2;
    code[2 * pen_bits + 2] = __float2bfloat16_rn(r2);
  }
}
__global__ void k_inverse_perm(const int32_t* __restrict__ perm, int64_t N,
                               int32_t* __restrict__ iperm) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < N) iperm[perm[r]] = (int32_t)r;
}

int sm_count() {
  static int n[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  if (n[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 1;
    }
    n[dev] = v;
  }
  return n[dev];
}

}  // namespace

int tc_kp(int k, int depth) {
  // at least k keys per partition, and at least a quarter of the re-rank
  // depth so that a deep re-rank is not starved by the per-partition cap
  const int need = std::max(k, (depth + 3) / 4);
  return need <= 10 ? 10 : (need <= 16 ? 16 : 32);
}
int tc_rerank_depth(int k, int factor) {
  const int f = factor > 0 ? factor : 4;
  return std::min(kMaxRerank, std::max(k, f * k));
}

bool tc_tile_fits(int d, int words_pad, int N, int f8) {
  const int kc = f8 ? (d + 127) / 128 : (d + 63) / 64;
  return tc_fits(kc, words_pad, N, false, f8 != 0);
}

bool tc_scan_supported(int d, int k, int kp, int words_pad, int f8) {
  if (d % 8 != 0 || d < 64 || d > 128 || k > 32 || (kp != 10 && kp != 16 && kp != 32))
    return false;
  if (f8 && d % 16 != 0) return false;
  return tc_tile_fits(d, words_pad, 128, f8) || tc_tile_fits(d, words_pad, 256, f8);
}

bool tc_pen_supported(int d, int kp, int words_pad) {
  if (d % 8 != 0 || d < 64 || d > 128 || (kp != 10 && kp != 16)) return false;
  return tc_fits((d + 63) / 64 + 1, words_pad, 128, true);
}

// the split form: penalty form with 64-row tiles over [hi | lo | code] rows
bool tc_split_supported(int d, int kp, int words_pad) {
  if (d % 8 != 0 || d < 64 || d > 128 || (kp != 10 && kp != 16)) return false;
  return tc_fits(2 * ((d + 63) / 64) + 1, words_pad, 64, true);
}

int tc_pen_columns(int pen_bits, int metric) { return 2 * pen_bits + (metric == CAPS_L2 ? 3 : 0); }

namespace {
std::atomic<long long> g_tc_withhold{-1};
std::atomic<unsigned long long> g_tc_wait_ns{kTcWaitNs};
}  // namespace

void tc_set_stall(long long item, unsigned long long wait_ns) {
  if (item < 0) {
    g_tc_withhold.store(-1);
    g_tc_wait_ns.store(kTcWaitNs);
  } else {
    g_tc_withhold.store(item);
    g_tc_wait_ns.store(wait_ns > 0 ? wait_ns : kTcWaitNs);
  }
}

int tc_prepare_index(const TcIndexPrep& p, cudaStream_t s) {
  const int64_t N = p.N;
  if (p.f8) {
    // e4m3 rows of ceil(d / 128) * 128 bytes, per-row scales and fp32 norms
    const int cols8 = (p.d + 127) / 128 * 128;
    k_rows_fp8<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(p.Xp, N, p.d, cols8,
                                                            static_cast<uint8_t*>(p.Xb), p.xn, p.xs);
    CAPS_LAUNCH("k_rows_fp8");
    *p.xn_max = 0.f;
    k_inverse_perm<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(p.perm, N, p.iperm);
    CAPS_LAUNCH("k_inverse_perm");
    // 2-D tensor map: boxes of 128 coordinates (128 bytes) x 128 rows,
    // 128-byte swizzle
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult qres;
    CAPS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                               cudaEnableDefault, &qres));
    if (!fn || qres != cudaDriverEntryPointSuccess)
      return fail(CAPS_ECUDA, "cuTensorMapEncodeTiled is not available");
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    cuuint64_t gdim[2] = {(cuuint64_t)cols8, (cuuint64_t)N};
    cuuint64_t gstride[1] = {(cuuint64_t)cols8};
    cuuint32_t box[2] = {128, (cuuint32_t)TC_BOX};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(static_cast<CUtensorMap*>(p.tmap), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, p.Xb,
                        gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(CAPS_ECUDA, "cuTensorMapEncodeTiled failed (e4m3 rows)");
    CAPS_CUDA(cudaStreamSynchronize(s));
    return CAPS_OK;
  }
  const int kcd = (p.d + 63) / 64 * (p.split ? 2 : 1);  // chunks before the code chunk
  const int cols = p.pen ? (kcd + 1) * 64 : p.d;
  if (p.split && !p.pen) return fail(CAPS_EINVAL, "the split form needs the penalty form");
  unsigned int* xmax = nullptr;
  {
    void* q = nullptr;
    if (dev_alloc(&q, sizeof(unsigned int), s, true) != cudaSuccess) {
      cudaGetLastError();
      return fail(CAPS_ENOMEM, "device allocation failed for the norm maximum");
    }
    xmax = static_cast<unsigned int*>(q);
  }
  CAPS_CUDA(cudaMemsetAsync(xmax, 0, sizeof(unsigned int), s));
  const uint4 pm = make_uint4(p.pen_mask[0], p.pen_mask[1], p.pen_mask[2], p.pen_mask[3]);
  k_rows_bf16<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
      p.Xp, N, p.d, cols, kcd, p.Ap, p.words_pad, p.pen, p.pen_bits, pm,
      p.pen && p.metric == CAPS_L2 ? 1 : 0, p.split, static_cast<__nv_bfloat16*>(p.Xb), p.xn,
      xmax);
  cudaError_t le = cudaGetLastError();
  unsigned int xmax_h = 0;
  if (le == cudaSuccess) le = cudaMemcpyAsync(&xmax_h, xmax, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (le == cudaSuccess) le = cudaStreamSynchronize(s);
  cudaFreeAsync(xmax, s);
  if (le != cudaSuccess) return cuda_fail(le, "k_rows_bf16");
  ++g_kernel_launches;
  uint32_t bits = xmax_h;
  float xm;
  std::memcpy(&xm, &bits, sizeof(float));
  *p.xn_max = xm;
  k_inverse_perm<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(p.perm, N, p.iperm);
  CAPS_LAUNCH("k_inverse_perm");
  // 2-D tensor map over the bf16 rows: inner dimension cols, outer N rows;
  // boxes of 64 coordinates (128 bytes) x 128 rows, 128-byte swizzle
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qres;
  CAPS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &qres));
  if (!fn || qres != cudaDriverEntryPointSuccess)
    return fail(CAPS_ECUDA, "cuTensorMapEncodeTiled is not available");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)N};
  cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
  // (the split form scans 64-row tiles: a 64-row box)
  cuuint32_t box[2] = {64, (cuuint32_t)(p.split ? tc_box_rows(64) : TC_BOX)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(static_cast<CUtensorMap*>(p.tmap), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p.Xb,
                      gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CAPS_ECUDA, "cuTensorMapEncodeTiled failed");
  return CAPS_OK;
}

int tc_query_prep(const float* Q, int64_t nq, int d, void* Qh, float* qn, int f8, float* qs,
                  cudaStream_t s, int split) {
  if (nq == 0) return CAPS_OK;
  if (f8) {
    k_query_fp8<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(Q, nq, d, static_cast<uint8_t*>(Qh), qs, qn);
    CAPS_LAUNCH("k_query_fp8");
    return CAPS_OK;
  }
  k_query_bf16<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(Q, nq, d, split,
                                                        static_cast<__nv_bfloat16*>(Qh), qn);
  CAPS_LAUNCH("k_query_bf16");
  return CAPS_OK;
}

int tc_group(const int32_t* probe, const uint64_t* sel, int h, int64_t ne, int B, int item_cap,
             BinWork* w, Scratch& scr, cudaStream_t s) {
  if (ne > INT_MAX) return fail(CAPS_EINVAL, "too many probes in one chunk");
  (void)h;
  const int cap = item_cap > 0 ? std::min(item_cap, TC_M) : TC_M;
  int32_t *bin_off = nullptr, *cursor = nullptr, *cnt = nullptr;
  if (int rc = scr.get(&w->ent, (size_t)ne)) return rc;
  if (int rc = scr.get(&bin_off, (size_t)B + 1)) return rc;
  if (int rc = scr.get(&cursor, (size_t)B + 1)) return rc;
  // partition histogram, offsets, scatter; then mask order inside each partition
  CAPS_CUDA(cudaMemsetAsync(bin_off, 0, sizeof(int32_t) * ((size_t)B + 1), s));
  const bool shared_bins = B <= kBinShared;
  const int G = (int)std::min<int64_t>(kBinBlocks, std::max<int64_t>(1, (ne + 2047) / 2048));
  const int64_t chunk = (ne + G - 1) / G;
  const size_t hsm = sizeof(int32_t) * (size_t)B;
  int32_t* blk = nullptr;
  const unsigned g = (unsigned)((ne + 255) / 256);
  if (ne > 0 && shared_bins) {
    if (int rc = scr.get(&blk, (size_t)B * G)) return rc;
    k_bin_hist<<<(unsigned)G, GRP_T, hsm, s>>>(probe, ne, chunk, B, G, bin_off, blk);
    CAPS_LAUNCH("k_bin_hist");
  } else if (ne > 0) {
    k_bin_count<<<g, 256, 0, s>>>(probe, ne, bin_off);
    CAPS_LAUNCH("k_bin_count");
  }
  if (int rc = scan_exclusive_i32(bin_off, (int64_t)B + 1, scr, s)) return rc;
  if (ne > 0) {
    int32_t* tmp = nullptr;
    if (int rc = scr.get(&tmp, (size_t)ne)) return rc;
    if (shared_bins) {
      k_bin_blockscan<<<(unsigned)(((int64_t)B * 32 + 255) / 256), 256, 0, s>>>(bin_off, B, G, blk);
      CAPS_LAUNCH("k_bin_blockscan");
      k_bin_scatter_blk<<<(unsigned)G, GRP_T, hsm, s>>>(probe, ne, chunk, B, G, blk, tmp);
      CAPS_LAUNCH("k_bin_scatter_blk");
    } else {
      CAPS_CUDA(cudaMemcpyAsync(cursor, bin_off, sizeof(int32_t) * ((size_t)B + 1),
                                cudaMemcpyDeviceToDevice, s));
      k_bin_scatter<<<g, 256, 0, s>>>(probe, ne, cursor, tmp);
      CAPS_LAUNCH("k_bin_scatter");
    }
    k_bin_group_mask<<<(unsigned)B, 512, 0, s>>>(bin_off, sel, tmp, w->ent);
    CAPS_LAUNCH("k_bin_group_mask");
  }
  if (int rc = scr.get(&cnt, (size_t)B + 1)) return rc;
  if (int rc = scr.get(&w->n_items, 2)) return rc;
  w->next_item = w->n_items + 1;
  k_tc_items_count<<<(B + 1 + 255) / 256, 256, 0, s>>>(bin_off, B, cap, cnt);
  CAPS_LAUNCH("k_tc_items_count");
  if (int rc = scan_exclusive_i32(cnt, (int64_t)B + 1, scr, s)) return rc;
  w->max_items = ne / cap + B + 1;
  TcItem* items = nullptr;
  if (int rc = scr.get(&items, (size_t)w->max_items)) return rc;
  w->items = items;
  k_tc_items_fill<<<(B + 1 + 255) / 256, 256, 0, s>>>(bin_off, cnt, B, cap, items, w->n_items,
                                                       w->next_item);
  CAPS_LAUNCH("k_tc_items_fill");
  return CAPS_OK;
}

int tc_scan(const TcScanArgs& t, const BinWork& w, cudaStream_t s) {
  TcArgs a;
  a.ent = w.ent;
  a.items = static_cast<const TcItem*>(w.items);
  a.n_items = w.n_items;
  a.next_item = w.next_item;
  a.sel = t.sel;
  a.qmask = t.qmask;
  a.qval = t.qval;
  a.Qh = t.Qh;
  a.qs = t.qs;
  a.xs = t.xs;
  a.qn = t.qn;
  a.Ap = t.Ap;
  a.perm = t.perm;
  a.xn = t.xn;
  a.offsets = t.offsets;
  a.m = t.m;
  a.h = t.h;
  a.split = t.split;
  // (split: the A operand's rows are the queries' [hi | lo] bf16 columns)
  a.d = t.split ? tc_vec_cols(t.d, 1) : t.d;
  a.kcd = t.f8 ? (t.d + 127) / 128 : (t.d + 63) / 64 * (t.split ? 2 : 1);
  a.kc = a.kcd + (t.pen ? 1 : 0);
  a.kp = t.kp;
  a.pen_bits = t.pen_bits;
  for (int i = 0; i < 4; i++) a.pen_mask[i] = t.pen_mask[i];
  a.xn_max = t.xn_max;
  a.qslot = t.qslot;
  a.sp = t.sp;
  {
    const int depth = std::min(t.rerank, t.m * t.kp);  // keys the merge keeps per query
    a.nslot = std::min(TC_SLOTS, std::max(1, (depth + t.kp - 1) / t.kp));
  }
  a.part = t.part;
  a.err = t.err;
  a.pen_ks = t.pen ? (tc_pen_columns(t.pen_bits, t.metric) + 15) / 16 : 0;
  a.pen_norm = t.pen && t.metric == CAPS_L2 ? 1 : 0;
  a.wait_ns = g_tc_wait_ns.load();
  {
    const long long w = g_tc_withhold.load();
    a.withhold = w >= 0 && w < INT_MAX ? (int)w : -1;
  }
  const CUtensorMap& map = *static_cast<const CUtensorMap*>(t.tmap);
  // persistent: one CTA per SM (the shared memory admits no second), never
  // more CTAs than work items
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>(w.max_items, sm_count()));
  if (t.split) {  // (the kernel multiplies the split chunk pairs with 64-row tiles only)
    if (!t.pen || !tc_split_supported(t.d, t.kp, t.words_pad))
      return fail(CAPS_EINVAL, "the split form does not fit this index or k");
    return tc_launch_pen(map, a, t.metric, t.words_pad, t.kp, g,
                         tc_smem_bytes(a.kc, t.words_pad, 64, true), s, 64);
  }
  if (t.pen) {
    if (!tc_pen_supported(t.d, t.kp, t.words_pad))
      return fail(CAPS_EINVAL, "the penalty form does not fit this index or k");
    return tc_launch_pen(map, a, t.metric, t.words_pad, t.kp, g,
                         tc_smem_bytes(a.kc, t.words_pad, 128, true), s);
  }
  // 256-row tiles unless 128 were asked for; whichever of the two fits
  const bool f8 = t.f8 != 0;
  const bool fit128 = tc_fits(a.kc, t.words_pad, 128, false, f8);
  const bool fit256 = tc_fits(a.kc, t.words_pad, 256, false, f8);
  if (!fit128 && !fit256)
    return fail(CAPS_EINVAL, "the per-pair filter form does not fit this index");
  const int N = (t.tile_n != 128 && fit256) || !fit128 ? 256 : 128;
  const size_t smem = tc_smem_bytes(a.kc, t.words_pad, N, false, f8);
  if (f8) return tc_launch_f8(map, a, t.metric, t.words_pad, t.kp, N, g, smem, s);
#define CAPS_TC(WPV, KPV)                                                                      \
  if (N == 128)                                                                                \
    return t.metric == CAPS_L2 ? launch_tc<CAPS_L2, WPV, KPV, 128, false>(map, a, g, smem, s)  \
                               : launch_tc<CAPS_IP, WPV, KPV, 128, false>(map, a, g, smem, s); \
  return t.metric == CAPS_L2 ? launch_tc<CAPS_L2, WPV, KPV, 256, false>(map, a, g, smem, s)    \
                             : launch_tc<CAPS_IP, WPV, KPV, 256, false>(map, a, g, smem, s)
  if (t.kp == 10) {
    switch (t.words_pad) {
      case 1: CAPS_TC(1, 10);
      case 2: CAPS_TC(2, 10);
      case 4: CAPS_TC(4, 10);
    }
  } else if (t.kp == 16) {
    switch (t.words_pad) {
      case 1: CAPS_TC(1, 16);
      case 2: CAPS_TC(2, 16);
      case 4: CAPS_TC(4, 16);
    }
  } else if (t.kp == 32) {
    switch (t.words_pad) {
      case 1: CAPS_TC(1, 32);
      case 2: CAPS_TC(2, 32);
      case 4: CAPS_TC(4, 32);
    }
  }
#undef CAPS_TC
  return fail(CAPS_EINVAL, "unsupported attribute word count or list length");
}

int tc_merge_rerank(const TcScanArgs& t, const uint8_t* dead, int64_t nq, int k, const float* Q,
                    const float* Xp, const int32_t* iperm, int64_t* out_ids, float* out_dist,
                    cudaStream_t s) {
  if (nq == 0) return CAPS_OK;
  const int depth = std::min(t.rerank, t.m * t.kp);  // candidates re-scored per query
  const int nslot = t.qslot ? std::min(TC_SLOTS, std::max(1, (depth + t.kp - 1) / t.kp)) : 0;
  const unsigned grid = (unsigned)((nq + 3) / 4);
  if (t.d % 4 != 0 || t.d > 128) return fail(CAPS_EINVAL, "re-rank needs d % 4 == 0, d <= 128");
  if (depth > kMaxRerank) return fail(CAPS_EINVAL, "re-rank depth above 256");
  const size_t smem = sizeof(float) * 4 * (size_t)t.d + sizeof(uint64_t) * 4 * kMaxRerank;
#define CAPS_MR(MET)                                                                            \
  do {                                                                                          \
    CAPS_CUDA(cudaFuncSetAttribute(k_merge_rerank<MET, 1>,                                      \
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));    \
    k_merge_rerank<MET, 1><<<grid, 128, smem, s>>>(t.part, dead, nq, t.m, t.kp, depth, k,       \
                                                   t.qslot, nslot, Q, t.d, Xp, iperm, t.n_rows, \
                                                   out_ids, out_dist, t.err);                   \
  } while (0)
  if (t.metric == CAPS_L2) CAPS_MR(CAPS_L2);
  else CAPS_MR(CAPS_IP);
#undef CAPS_MR
  CAPS_LAUNCH("k_merge_rerank");
  return CAPS_OK;
}

}  // namespace caps
