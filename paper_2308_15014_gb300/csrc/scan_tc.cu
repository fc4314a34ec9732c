// Host side of the BF16 tensor-core form of the CAPS scan: bf16 copies of
// the queries and rows, grouping of the probes into work items, the
// persistent scan launch (explicit-filter instantiations here, the penalty
// form in scan_tc_pen.cu), and the per-query merge with an exact fp32
// re-rank of the best rerank_factor * k candidates (coordinates in order,
// one fma each) before the final top-k.
#include <algorithm>
#include <climits>
#include <cstring>

#include "scan_tc_kernel.cuh"

namespace caps {
namespace {

// ---- bf16 query copy and fp32 squared norms -------------------------------
__global__ void k_query_bf16(const float* __restrict__ Q, int64_t nq, int d,
                             __nv_bfloat16* __restrict__ Qh, float* __restrict__ qn) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  float acc = 0.f;
  for (int j = 0; j < d; j++) {
    const float x = Q[q * d + j];
    acc = fmaf(x, x, acc);
    Qh[q * d + j] = __float2bfloat16_rn(x);
  }
  qn[q] = acc;
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
// fp32 (coordinates in order, one fma each) and keep the k best.
template <int METRIC, int KPL_M, int KPL_K>
__global__ void __launch_bounds__(128)
k_merge_rerank(const uint64_t* __restrict__ part, const uint8_t* __restrict__ dead, int64_t nq,
               int m, int lp, int kp, int k, const float* __restrict__ Q, int d,
               const float* __restrict__ Xp, const int32_t* __restrict__ iperm,
               int64_t* __restrict__ out_ids, float* __restrict__ out_dist) {
  extern __shared__ float qsm[];  // [4][d]
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 4 + wp;
  if (q >= nq) return;
  float* qs = qsm + (size_t)wp * d;
  for (int j = lane; j < d; j += 32) qs[j] = Q[q * d + j];
  __syncwarp();
  TopKm<KPL_M> cand;
  cand.init();
  uint64_t kthv = kEmptyKey;
  if (!dead[q]) {
    const uint64_t* src = part + q * (int64_t)m * lp;
    const int tot = m * lp;
    for (int b0 = 0; b0 < tot; b0 += 32) {
      const uint64_t key = (b0 + lane < tot) ? src[b0 + lane] : kEmptyKey;
      cand.offer(key, kthv, kp, lane);
    }
  }
  // exact fp32 scores of the kp candidates
  TopKm<KPL_K> top;
  top.init();
  uint64_t kth2 = kEmptyKey;
#pragma unroll
  for (int s = 0; s < KPL_M; s++) {
    const int P = lane * KPL_M + s;
    uint64_t key = kEmptyKey;
    const uint64_t ck = cand.v[s];
    if (P < kp && ck != kEmptyKey) {
      const uint32_t id = (uint32_t)(ck & 0xffffffffu);
      const float* xr = Xp + (int64_t)iperm[id] * d;
      float acc = 0.f;
      for (int j = 0; j < d; j++) {
        if (METRIC == CAPS_L2) {
          const float t = xr[j] - qs[j];
          acc = fmaf(t, t, acc);
        } else {
          acc = fmaf(xr[j], qs[j], acc);
        }
      }
      key = make_key(METRIC == CAPS_L2 ? acc : -acc, id);
    }
    top.offer(key, kth2, k, lane);
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

__global__ void k_mask_key(const uint64_t* __restrict__ sel, int64_t ne, int32_t* __restrict__ key) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ne) key[i] = (int32_t)sel[i];
}
__global__ void k_gather_i32(const int32_t* __restrict__ src, const int32_t* __restrict__ idx,
                             int64_t n, int32_t* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[idx[i]];
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
// penalty form the 64-column one-hot code of the row's packed attribute bits
// and of its block), its fp32 squared norm (coordinates in order, one fma
// each) and the largest squared norm
__global__ void k_rows_bf16(const float* __restrict__ Xp, int64_t N, int d, int cols, int kcd,
                            const uint32_t* __restrict__ Ap, int WP, int pen, int pen_bits,
                            uint4 pen_mask, const int32_t* __restrict__ offsets, int n_blocks,
                            int nb, __nv_bfloat16* __restrict__ Xb, float* __restrict__ xn,
                            unsigned int* __restrict__ xn_max_bits) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  __nv_bfloat16* row = Xb + r * cols;
  float acc = 0.f;
  for (int j = 0; j < d; j++) {
    const float x = Xp[r * d + j];
    acc = fmaf(x, x, acc);
    row[j] = __float2bfloat16_rn(x);
  }
  for (int j = d; j < cols; j++) row[j] = __float2bfloat16_rn(0.f);
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
  // block of row r: the last offset <= r (offsets[n_blocks] = N)
  int lo = 0, hi = n_blocks;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (offsets[mid] <= r) lo = mid;
    else hi = mid;
  }
  code[2 * pen_bits + lo % nb] = one;
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

int tc_kp(int k) { return k <= 12 ? 12 : (k <= 16 ? 16 : 32); }
int tc_rerank_depth(int k, int factor) {
  const int f = factor > 0 ? factor : 4;
  return std::min(64, std::max(k, f * k));
}

bool tc_scan_supported(int d, int k, int kp, int words_pad) {
  if (d % 8 != 0 || d < 64 || d > 128 || k > 32 || (kp != 12 && kp != 16 && kp != 32))
    return false;
  return tc_fits((d + 63) / 64, words_pad, 128, false);
}

bool tc_pen_supported(int d, int kp, int words_pad) {
  if (d % 8 != 0 || d < 64 || d > 128 || (kp != 12 && kp != 16)) return false;
  return tc_fits((d + 63) / 64 + 1, words_pad, 128, true);
}

int tc_prepare_index(const TcIndexPrep& p, cudaStream_t s) {
  const int64_t N = p.N;
  const int kcd = (p.d + 63) / 64;
  const int cols = p.pen ? (kcd + 1) * 64 : p.d;
  unsigned int* xmax = nullptr;
  CAPS_CUDA(cudaMallocAsync(&xmax, sizeof(unsigned int), s));
  CAPS_CUDA(cudaMemsetAsync(xmax, 0, sizeof(unsigned int), s));
  const uint4 pm = make_uint4(p.pen_mask[0], p.pen_mask[1], p.pen_mask[2], p.pen_mask[3]);
  k_rows_bf16<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(
      p.Xp, N, p.d, cols, kcd, p.Ap, p.words_pad, p.pen, p.pen_bits, pm, p.offsets,
      p.B * p.nb, p.nb, static_cast<__nv_bfloat16*>(p.Xb), p.xn, xmax);
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
  cuuint32_t box[2] = {64, (cuuint32_t)TC_BOX};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(static_cast<CUtensorMap*>(p.tmap), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, p.Xb,
                      gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CAPS_ECUDA, "cuTensorMapEncodeTiled failed");
  return CAPS_OK;
}

int tc_query_prep(const float* Q, int64_t nq, int d, void* Qh, float* qn, cudaStream_t s) {
  if (nq == 0) return CAPS_OK;
  k_query_bf16<<<(unsigned)((nq + 127) / 128), 128, 0, s>>>(Q, nq, d,
                                                            static_cast<__nv_bfloat16*>(Qh), qn);
  CAPS_LAUNCH("k_query_bf16");
  return CAPS_OK;
}

int tc_group(const int32_t* probe, const uint64_t* sel, int h, int64_t ne, int B, int item_cap,
             BinWork* w, Scratch& scr, cudaStream_t s) {
  if (ne > INT_MAX) return fail(CAPS_EINVAL, "too many probes in one chunk");
  const int cap = item_cap > 0 ? std::min(item_cap, TC_M) : TC_M;
  int32_t *bin_off = nullptr, *cnt = nullptr;
  if (int rc = scr.get(&w->ent, (size_t)ne)) return rc;
  if (int rc = scr.get(&bin_off, (size_t)B + 1)) return rc;
  if (h + 1 <= 16) {
    // probes of a partition ordered by their selected-block mask, so that
    // probes scanning the same blocks share a work item: sort by mask, then
    // (stably) by partition
    int32_t *mkey = nullptr, *p1 = nullptr, *moff = nullptr, *pkey = nullptr, *p2 = nullptr;
    if (int rc = scr.get(&mkey, (size_t)ne)) return rc;
    if (int rc = scr.get(&p1, (size_t)ne)) return rc;
    if (int rc = scr.get(&moff, ((size_t)1 << (h + 1)) + 1)) return rc;
    if (int rc = scr.get(&pkey, (size_t)ne)) return rc;
    if (int rc = scr.get(&p2, (size_t)ne)) return rc;
    const unsigned g = (unsigned)((ne + 255) / 256);
    k_mask_key<<<g, 256, 0, s>>>(sel, ne, mkey);
    CAPS_LAUNCH("k_mask_key");
    if (int rc = stable_sort_by_key(mkey, ne, (int64_t)1 << (h + 1), p1, moff, scr, s)) return rc;
    k_gather_i32<<<g, 256, 0, s>>>(probe, p1, ne, pkey);
    CAPS_LAUNCH("k_gather_i32");
    if (int rc = stable_sort_by_key(pkey, ne, B, p2, bin_off, scr, s)) return rc;
    k_gather_i32<<<g, 256, 0, s>>>(p1, p2, ne, w->ent);
    CAPS_LAUNCH("k_gather_i32");
  } else {
    if (int rc = stable_sort_by_key(probe, ne, B, w->ent, bin_off, scr, s)) return rc;
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
  a.Qh = static_cast<const __nv_bfloat16*>(t.Qh);
  a.qn = t.qn;
  a.Ap = t.Ap;
  a.perm = t.perm;
  a.xn = t.xn;
  a.offsets = t.offsets;
  a.m = t.m;
  a.h = t.h;
  a.d = t.d;
  a.kcd = (t.d + 63) / 64;
  a.kc = a.kcd + (t.pen ? 1 : 0);
  a.kp = t.kp;
  a.pen_bits = t.pen_bits;
  for (int i = 0; i < 4; i++) a.pen_mask[i] = t.pen_mask[i];
  a.xn_max = t.xn_max;
  a.qslot = t.qslot;
  {
    const int depth = std::min(t.rerank, t.m * t.kp);  // keys the merge keeps per query
    a.nslot = std::min(TC_SLOTS, std::max(1, (depth + t.kp - 1) / t.kp));
  }
  a.part = t.part;
  a.err = t.err;
  const CUtensorMap& map = *static_cast<const CUtensorMap*>(t.tmap);
  // persistent: one CTA per SM (the shared memory admits no second), never
  // more CTAs than work items
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>(w.max_items, sm_count()));
  if (t.pen) {
    if (!tc_pen_supported(t.d, t.kp, t.words_pad))
      return fail(CAPS_EINVAL, "the penalty form does not fit this index or k");
    return tc_launch_pen(map, a, t.metric, t.words_pad, t.kp, g,
                         tc_smem_bytes(a.kc, t.words_pad, 128, true), s);
  }
  if (!tc_fits(a.kc, t.words_pad, 128, false))
    return fail(CAPS_EINVAL, "the per-pair filter form does not fit this index");
  // 256-row tiles where they fit, else 128
  const int N = t.tile_n != 128 && tc_fits(a.kc, t.words_pad, 256, false) ? 256 : 128;
  const size_t smem = tc_smem_bytes(a.kc, t.words_pad, N, false);
#define CAPS_TC(WPV, KPV)                                                                      \
  if (N == 128)                                                                                \
    return t.metric == CAPS_L2 ? launch_tc<CAPS_L2, WPV, KPV, 128, false>(map, a, g, smem, s)  \
                               : launch_tc<CAPS_IP, WPV, KPV, 128, false>(map, a, g, smem, s); \
  return t.metric == CAPS_L2 ? launch_tc<CAPS_L2, WPV, KPV, 256, false>(map, a, g, smem, s)    \
                             : launch_tc<CAPS_IP, WPV, KPV, 256, false>(map, a, g, smem, s)
  if (t.kp == 12) {
    switch (t.words_pad) {
      case 1: CAPS_TC(1, 12);
      case 2: CAPS_TC(2, 12);
      case 4: CAPS_TC(4, 12);
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
  const unsigned grid = (unsigned)((nq + 3) / 4);
  const size_t smem = sizeof(float) * 4 * (size_t)t.d;
#define CAPS_MR(MET, KM, KK)                                                                   \
  k_merge_rerank<MET, KM, KK><<<grid, 128, smem, s>>>(t.part, dead, nq, t.m, t.kp, depth, k, Q, \
                                                       t.d, Xp, iperm, out_ids, out_dist)
  const int km = depth <= 32 ? 1 : 2;
  if (t.metric == CAPS_L2) {
    if (km == 1) CAPS_MR(CAPS_L2, 1, 1);
    else CAPS_MR(CAPS_L2, 2, 1);
  } else {
    if (km == 1) CAPS_MR(CAPS_IP, 1, 1);
    else CAPS_MR(CAPS_IP, 2, 1);
  }
#undef CAPS_MR
  CAPS_LAUNCH("k_merge_rerank");
  return CAPS_OK;
}

}  // namespace caps
