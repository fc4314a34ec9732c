// Partition-major scan of CAPS Alg. 2 ("attribute match" + "top-k vector
// match") for a whole query batch.
//
// The m probes of every query are grouped by partition; one CTA takes one
// partition and up to G probes of it.  The partition's rows in the blocks any
// of those probes selected stream through shared memory once (1-D TMA bulk
// copies, double-buffered, completion on an mbarrier), and every probe is
// tested against every row there: block selected? attribute filter passes?
// distance.  Each tile runs in three balanced phases: (1) every warp tests
// its 4 probes against the tile's rows and the passing (probe, row) pairs are
// compacted into one list, probe by probe; (2) the list is split evenly over
// all warps, each 8-lane group scores one pair at a time (lane s reads the
// row's and the query's coordinates 32c + 4s .. + 3, sums its d/8 products in
// order, and a 3-step shuffle reduction finishes the row); (3) each warp
// offers the keys of its own 4 probes to their running top-k lists.  Work per
// warp no longer depends on how unevenly the probes pass (a single-constraint
// query passes a whole AFT block).  The per-probe top-k goes to part[e][0..k),
// e = query * m + probe slot; k_merge_topk then keeps the k best of each
// query's m lists (each point lives in exactly one partition, so the top-k of
// the union is the top-k of the per-partition top-k lists).
//
// Summation order: each lane adds its d/8 coordinates in order, then the 8
// lane sums are added pairwise -- an fp32 sum whose rounding may differ from
// the fully sequential order by a few units in the last place.
#include <algorithm>
#include <climits>

#include "caps_internal.cuh"

namespace caps {
namespace {

constexpr int NW = 8;          // warps per CTA
constexpr int G = 32;          // probes per work item
constexpr int PPW = G / NW;    // probes per warp

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
// Wait for the mbarrier phase with the given parity, at most limit_ns of
// wall-clock time; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const uint32_t a = smem_u32(bar);
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    for (int i = 0; i < 256; i++) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(a), "r"(parity)
          : "memory");
      if (done) return true;
    }
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s: a 32-KB copy takes microseconds

template <int KPL>
struct TopK {
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
  // offer one key per lane (kEmptyKey = none); keeps the k best
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

struct Item {
  int32_t b, e0, ne, pad;
};

// dynamic shared memory: two row tiles; per tile buffer its attribute words
// and original ids (bulk-copied from a 16-B aligned start, so up to 3 extra
// rows on each side) and block ids; then (16-B aligned) the query tile, the
// pair list and the pair keys
__host__ __device__ __forceinline__ int bin_aux_rows(int R) { return R + 8; }
__host__ __device__ __forceinline__ size_t bin_smem_fixed(int R, int d, int WP) {
  const size_t b = (size_t)2 * R * d * sizeof(float) + (size_t)2 * bin_aux_rows(R) * WP * 4 +
                   (size_t)2 * bin_aux_rows(R) * 4 + 2 * (size_t)R;
  return (b + 15) & ~(size_t)15;
}
__host__ __device__ __forceinline__ size_t bin_smem_total(int R, int d, int WP) {
  const size_t q = bin_smem_fixed(R, d, WP) + (size_t)G * d * sizeof(float) + (size_t)G * R * 2;
  return ((q + 7) & ~(size_t)7) + (size_t)G * R * 8;
}

struct BinScanArgs {
  const float* Xp;
  const uint32_t* Ap;
  const int32_t* perm;
  const int32_t* offsets;
  const float* Q;
  const uint32_t* qmask;
  const uint32_t* qval;
  const uint64_t* sel;
  const int32_t* ent;      // entries (q*m + slot) sorted by partition
  const Item* items;
  const int32_t* n_items;
  int m, h, d, k, R;
  uint64_t* part;          // [nq*m*k] keys
  int32_t* err;
  SparseRef sp;            // label sets: exact check after the signature test
};

// DV = d / 32 float4 pieces per lane (d a multiple of 32).
template <int METRIC, int WP, int DV, int KPL>
__global__ void __launch_bounds__(NW * 32)
k_scan_bin(BinScanArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int item_id = blockIdx.x;
  if (item_id >= *a.n_items) return;  // uniform per CTA
  const Item it = a.items[item_id];
  const int d = a.d, R = a.R, nb = a.h + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // shared layout
  float* rows0 = reinterpret_cast<float*>(smem_raw);
  float* rows1 = rows0 + (size_t)R * d;
  const int RA = bin_aux_rows(R);
  uint32_t* attr0 = reinterpret_cast<uint32_t*>(rows1 + (size_t)R * d);
  uint32_t* attr1 = attr0 + RA * WP;
  int32_t* prm0 = reinterpret_cast<int32_t*>(attr1 + RA * WP);
  int32_t* prm1 = prm0 + RA;
  uint8_t* blk0 = reinterpret_cast<uint8_t*>(prm1 + RA);
  uint8_t* blk1 = blk0 + R;
  // query tile [G][d], pair list [G*R] (probe*64 + row), pair keys [G*R]
  float* qtile = reinterpret_cast<float*>(smem_raw + bin_smem_fixed(R, d, WP));
  uint16_t* pairs = reinterpret_cast<uint16_t*>(qtile + (size_t)G * d);
  uint64_t* pkeys = reinterpret_cast<uint64_t*>(
      smem_raw + ((bin_smem_fixed(R, d, WP) + (size_t)G * d * sizeof(float) + (size_t)G * R * 2 + 7) &
                  ~(size_t)7));
  __shared__ uint64_t bar[2];
  __shared__ uint64_t p_sel[G];
  __shared__ uint32_t p_qm[G * WP], p_qv[G * WP];
  __shared__ int32_t p_q[G], p_e[G];
  __shared__ unsigned long long u_sel;
  __shared__ int run_lo[64], run_hi[64], run_j0[64];
  __shared__ int n_runs;
  __shared__ int32_t boff[65];           // block row offsets of this partition
  __shared__ int warp_cnt[NW], warp_base[NW + 1];
  __shared__ int p_start[G], p_cnt[G];

  if (tid == 0) {
    u_sel = 0ull;
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (tid < it.ne) {
    const int e = a.ent[it.e0 + tid];
    const int q = e / a.m;
    p_e[tid] = e;
    p_q[tid] = q;
    const uint64_t s = a.sel[e];
    p_sel[tid] = s;
    atomicOr(&u_sel, (unsigned long long)s);
#pragma unroll
    for (int w = 0; w < WP; w++) {
      p_qm[tid * WP + w] = a.qmask[(int64_t)q * WP + w];
      p_qv[tid * WP + w] = a.qval[(int64_t)q * WP + w];
    }
  }
  __syncthreads();
  const int32_t* off = a.offsets + (int64_t)it.b * nb;
  for (int j = tid; j <= nb; j += NW * 32) boff[j] = off[j];
  for (int x = tid; x < G * d / 4; x += NW * 32) {
    const int p = x / (d / 4), c4 = x % (d / 4);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p < it.ne) v = *reinterpret_cast<const float4*>(a.Q + (int64_t)p_q[p] * d + 4 * c4);
    reinterpret_cast<float4*>(qtile)[x] = v;
  }
  if (tid == 0) {
    // row runs = maximal stretches of blocks selected by some probe
    const uint64_t U = u_sel;
    int nr = 0, j = 0;
    while (j < nb) {
      if (!((U >> j) & 1ull)) { j++; continue; }
      int j2 = j;
      while (j2 + 1 < nb && ((U >> (j2 + 1)) & 1ull)) j2++;
      if (off[j2 + 1] > off[j]) {
        run_lo[nr] = off[j];
        run_hi[nr] = off[j2 + 1];
        run_j0[nr] = j;
        nr++;
      }
      j = j2 + 1;
    }
    n_runs = nr;
  }
  __syncthreads();

  const int grp = lane >> 3, sub = lane & 7;
  TopK<KPL> top[PPW];
  uint64_t kthv[PPW];
#pragma unroll
  for (int u = 0; u < PPW; u++) {
    top[u].init();
    kthv[u] = kEmptyKey;
  }

  // tile schedule: (run, start) pairs walked in order; tile t uses buffer t&1
  const int first_lo = n_runs > 0 ? run_lo[0] : 0;
  auto next_tile = [&](int& lo, int& n, int& j0, int& rr, int& rlo) -> bool {
    while (rr < n_runs && rlo >= run_hi[rr]) {
      rr++;
      if (rr < n_runs) rlo = run_lo[rr];
    }
    if (rr >= n_runs) return false;
    lo = rlo;
    n = min(R, run_hi[rr] - rlo);
    j0 = run_j0[rr];
    rlo += n;
    return true;
  };
  // issue tile into buffer `bi` (thread 0 only): rows, attribute words and
  // original ids of rows [lo, lo+n); the two small arrays are copied from the
  // 16-B boundary at or below lo (the arrays are padded so the rounded-up
  // end stays inside them)
  auto aux_lo = [&](int lo) { return lo & ~3; };
  auto issue = [&](int bi, int lo, int n) {
    const int alo = aux_lo(lo);
    const int arows = ((lo + n + 3) & ~3) - alo;
    const uint32_t rb = (uint32_t)(n * d * sizeof(float));
    const uint32_t ab = (uint32_t)(arows * WP * 4);
    const uint32_t pb = (uint32_t)(arows * 4);
    fence_proxy_async();
    mbar_expect_tx(&bar[bi], rb + ab + pb);
    bulk_g2s(bi ? rows1 : rows0, a.Xp + (int64_t)lo * d, rb, &bar[bi]);
    bulk_g2s(bi ? attr1 : attr0, a.Ap + (int64_t)alo * WP, ab, &bar[bi]);
    bulk_g2s(bi ? prm1 : prm0, a.perm + alo, pb, &bar[bi]);
  };

  int t_lo[2], t_n[2], t_j0[2];
  bool have[2] = {false, false};
  int rr_issue = 0, rlo_issue = first_lo;
  // prefetch two tiles
  for (int bi = 0; bi < 2; bi++) {
    have[bi] = next_tile(t_lo[bi], t_n[bi], t_j0[bi], rr_issue, rlo_issue);
    if (have[bi] && tid == 0) issue(bi, t_lo[bi], t_n[bi]);
  }
  uint32_t phase[2] = {0u, 0u};
  int bi = 0;
  while (have[bi]) {
    const int lo = t_lo[bi], n = t_n[bi];
    const uint32_t* attr = (bi ? attr1 : attr0) + (lo - aux_lo(lo)) * WP;
    const int32_t* prm = (bi ? prm1 : prm0) + (lo - aux_lo(lo));
    uint8_t* blk = bi ? blk1 : blk0;
    const float* rows = bi ? rows1 : rows0;
    // block index of the tile's rows (from the partition's block offsets)
    for (int r = tid; r < n; r += NW * 32) {
      const int gr = lo + r;
      int j = t_j0[bi];
      while (j + 1 < nb && boff[j + 1] <= gr) j++;
      blk[r] = (uint8_t)j;
    }
    const bool timed_out = !mbar_wait(&bar[bi], phase[bi], kWaitLimitNs);
    phase[bi] ^= 1u;
    if (__syncthreads_or(timed_out)) {
      // a copy never completed: flag it, let the other buffer's copy land
      // (bounded), and leave without touching shared memory again
      if (tid == 0) {
        atomicExch(a.err, 1);
        if (have[bi ^ 1]) mbar_wait(&bar[bi ^ 1], phase[bi ^ 1], kWaitLimitNs);
      }
      return;
    }
    {
      // phase 1: pass masks of this warp's probes (4w .. 4w+3) over the rows
      uint64_t pm[PPW];
      uint64_t ps[PPW];
      uint32_t pqm[PPW][WP], pqv[PPW][WP];
#pragma unroll
      for (int u = 0; u < PPW; u++) {
        const int p = PPW * warp + u;
        pm[u] = 0ull;
        ps[u] = p < it.ne ? p_sel[p] : 0ull;  // no block selected: never passes
#pragma unroll
        for (int w = 0; w < WP; w++) {
          pqm[u][w] = p_qm[p * WP + w];
          pqv[u][w] = p_qv[p * WP + w];
        }
      }
#pragma unroll
      for (int g0 = 0; g0 < 64; g0 += 32) {
        const int r = g0 + lane;
        const bool in = r < n;
        const int bj = in ? blk[r] : 0;
        uint32_t aw[WP];
#pragma unroll
        for (int w = 0; w < WP; w++) aw[w] = in ? attr[r * WP + w] : 0u;
#pragma unroll
        for (int u = 0; u < PPW; u++) {
          bool pass = in && ((ps[u] >> bj) & 1ull);
#pragma unroll
          for (int w = 0; w < WP; w++) pass = pass && ((aw[w] & pqm[u][w]) == pqv[u][w]);
          // label sets: the signature test is necessary, this is exact
          if (pass && a.sp.roff) pass = sp_subset(a.sp, lo + r, p_q[PPW * warp + u]);
          pm[u] |= (uint64_t)__ballot_sync(0xffffffffu, pass) << g0;
        }
      }
      int mycnt = 0;
#pragma unroll
      for (int u = 0; u < PPW; u++) mycnt += __popcll(pm[u]);
      if (lane == 0) warp_cnt[warp] = mycnt;
      __syncthreads();
      if (warp == 0) {
        const int c = lane < NW ? warp_cnt[lane] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (lane < NW) warp_base[lane] = incl - c;
        if (lane == NW - 1) warp_base[NW] = incl;
      }
      __syncthreads();
      {
        int base = warp_base[warp];
#pragma unroll
        for (int u = 0; u < PPW; u++) {
          const int p = PPW * warp + u;
          if (lane == 0) {
            p_start[p] = base;
            p_cnt[p] = __popcll(pm[u]);
          }
#pragma unroll
          for (int g0 = 0; g0 < 64; g0 += 32) {
            const int r = g0 + lane;
            if ((pm[u] >> r) & 1ull) {
              const uint64_t below = r == 0 ? 0ull : (pm[u] & ((~0ull) >> (64 - r)));
              pairs[base + __popcll(below)] = (uint16_t)(p * 64 + r);
            }
          }
          base += __popcll(pm[u]);
        }
      }
      __syncthreads();
      // phase 2: pairs split evenly over the warps, one pair per 8-lane group
      const int P = warp_base[NW];
      const int lo_w = (int)((int64_t)P * warp / NW), hi_w = (int)((int64_t)P * (warp + 1) / NW);
      for (int i0 = lo_w; i0 < hi_w; i0 += 4) {
        const int i = i0 + grp;
        const bool has = i < hi_w;
        const int pr = has ? pairs[i] : 0;
        const int pp = pr >> 6, r = pr & 63;
        const float* xr = rows + (size_t)r * d + 4 * sub;
        const float* qr = qtile + (size_t)pp * d + 4 * sub;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < DV; c++) {
          const float4 x = *reinterpret_cast<const float4*>(xr + 32 * c);
          const float4 y = *reinterpret_cast<const float4*>(qr + 32 * c);
          if (METRIC == CAPS_L2) {
            float t0 = x.x - y.x; acc = fmaf(t0, t0, acc);
            t0 = x.y - y.y; acc = fmaf(t0, t0, acc);
            t0 = x.z - y.z; acc = fmaf(t0, t0, acc);
            t0 = x.w - y.w; acc = fmaf(t0, t0, acc);
          } else {
            acc = fmaf(x.x, y.x, acc);
            acc = fmaf(x.y, y.y, acc);
            acc = fmaf(x.z, y.z, acc);
            acc = fmaf(x.w, y.w, acc);
          }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        if (has && sub == 0)
          pkeys[i] = make_key(METRIC == CAPS_L2 ? acc : -acc, (uint32_t)prm[r]);
      }
      __syncthreads();
      // phase 3: each warp offers its own probes' keys to their top-k lists
#pragma unroll
      for (int u = 0; u < PPW; u++) {
        const int p = PPW * warp + u;
        if (p >= it.ne) break;
        const int st = p_start[p], cn = p_cnt[p];
        for (int b0 = 0; b0 < cn; b0 += 32) {
          const uint64_t key = (b0 + lane < cn) ? pkeys[st + b0 + lane] : kEmptyKey;
          top[u].offer(key, kthv[u], a.k, lane);
        }
      }
    }
    __syncthreads();  // every warp is done with buffer bi
    // refill buffer bi with the tile after the one in the other buffer
    have[bi] = next_tile(t_lo[bi], t_n[bi], t_j0[bi], rr_issue, rlo_issue);
    if (have[bi] && tid == 0) issue(bi, t_lo[bi], t_n[bi]);
    bi ^= 1;
  }

  // per-probe top-k lists -> part[e*k ..]
#pragma unroll
  for (int u = 0; u < PPW; u++) {
    const int p = PPW * warp + u;
    if (p >= it.ne) break;
    uint64_t* dst = a.part + (int64_t)p_e[p] * a.k;
#pragma unroll
    for (int s = 0; s < KPL; s++) {
      const int P = lane * KPL + s;
      if (P < a.k) dst[P] = top[u].v[s];
    }
  }
}

// ---- work items: probes grouped by partition, at most G per item ----------
__global__ void k_items_count(const int32_t* __restrict__ bin_off, int B,
                              int32_t* __restrict__ cnt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) cnt[b] = (bin_off[b + 1] - bin_off[b] + G - 1) / G;
  if (b == B) cnt[B] = 0;
}
__global__ void k_items_fill(const int32_t* __restrict__ bin_off, const int32_t* __restrict__ item_off,
                             int B, Item* __restrict__ items, int32_t* __restrict__ n_items) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b == B) *n_items = item_off[B];
  if (b >= B) return;
  const int c = bin_off[b + 1] - bin_off[b];
  for (int t = 0; t * G < c; t++) {
    Item x;
    x.b = b;
    x.e0 = bin_off[b] + t * G;
    x.ne = min(G, c - t * G);
    x.pad = 0;
    items[item_off[b] + t] = x;
  }
}

// ---- per-query merge of the m partial lists ------------------------------
template <int METRIC, int KPL>
__global__ void __launch_bounds__(128)
k_merge_topk(const uint64_t* __restrict__ part, const uint8_t* __restrict__ dead, int64_t nq,
             int m, int k, int64_t* __restrict__ out_ids, float* __restrict__ out_dist) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
  if (q >= nq) return;
  TopK<KPL> top;
  top.init();
  uint64_t kthv = kEmptyKey;
  if (!dead[q]) {
    const uint64_t* src = part + q * m * k;
    const int tot = m * k;
    for (int base = 0; base < tot; base += 32) {
      const uint64_t key = (base + lane < tot) ? src[base + lane] : kEmptyKey;
      top.offer(key, kthv, k, lane);
    }
  }
#pragma unroll
  for (int s = 0; s < KPL; s++) {
    const int P = lane * KPL + s;
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

template <int METRIC, int WP, int DV, int KPL>
int launch_bin_k(const BinScanArgs& a, int64_t grid, size_t smem, cudaStream_t s) {
  auto kern = k_scan_bin<METRIC, WP, DV, KPL>;
  if (smem > 48 * 1024)
    CAPS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)grid, NW * 32, smem, s>>>(a);
  CAPS_LAUNCH("k_scan_bin");
  return CAPS_OK;
}

template <int METRIC, int WP, int DV>
int launch_bin_kpl(const BinScanArgs& a, int64_t grid, size_t smem, cudaStream_t s) {
  if (a.k <= 32) return launch_bin_k<METRIC, WP, DV, 1>(a, grid, smem, s);
  if (a.k <= 64) return launch_bin_k<METRIC, WP, DV, 2>(a, grid, smem, s);
  return launch_bin_k<METRIC, WP, DV, 4>(a, grid, smem, s);
}

template <int METRIC, int WP>
int launch_bin_d(const BinScanArgs& a, int64_t grid, size_t smem, cudaStream_t s) {
  switch (a.d) {
    case 32: return launch_bin_kpl<METRIC, WP, 1>(a, grid, smem, s);
    case 64: return launch_bin_kpl<METRIC, WP, 2>(a, grid, smem, s);
    case 96: return launch_bin_kpl<METRIC, WP, 3>(a, grid, smem, s);
    case 128: return launch_bin_kpl<METRIC, WP, 4>(a, grid, smem, s);
    case 256: return launch_bin_kpl<METRIC, WP, 8>(a, grid, smem, s);
  }
  return fail(CAPS_EINVAL, "partition-major scan: unsupported d");
}

template <int METRIC>
int launch_bin_w(const BinScanArgs& a, int wp, int64_t grid, size_t smem, cudaStream_t s) {
  switch (wp) {
    case 1: return launch_bin_d<METRIC, 1>(a, grid, smem, s);
    case 2: return launch_bin_d<METRIC, 2>(a, grid, smem, s);
    case 4: return launch_bin_d<METRIC, 4>(a, grid, smem, s);
  }
  return fail(CAPS_EINVAL, "unsupported attribute word count");
}

}  // namespace

bool bin_scan_supported(int d) { return d == 32 || d == 64 || d == 96 || d == 128 || d == 256; }

int64_t bin_work_items_bound(int64_t ne, int B) { return ne / G + B + 1; }

// Group the batch's probes by partition and cut work items of <= G probes.
int bin_group(const int32_t* probe, int64_t ne, int B, BinWork* w, Scratch& scr, cudaStream_t s) {
  if (ne > INT_MAX) return fail(CAPS_EINVAL, "too many probes in one chunk");
  int32_t *bin_off = nullptr, *cnt = nullptr;
  if (int rc = scr.get(&w->ent, (size_t)ne)) return rc;
  if (int rc = scr.get(&bin_off, (size_t)B + 1)) return rc;
  if (int rc = stable_sort_by_key(probe, ne, B, w->ent, bin_off, scr, s)) return rc;
  if (int rc = scr.get(&cnt, (size_t)B + 1)) return rc;
  if (int rc = scr.get(&w->n_items, 1)) return rc;
  k_items_count<<<(B + 1 + 255) / 256, 256, 0, s>>>(bin_off, B, cnt);
  CAPS_LAUNCH("k_items_count");
  if (int rc = scan_exclusive_i32(cnt, (int64_t)B + 1, scr, s)) return rc;
  w->max_items = bin_work_items_bound(ne, B);
  Item* items = nullptr;
  if (int rc = scr.get(&items, (size_t)w->max_items)) return rc;
  w->items = items;
  k_items_fill<<<(B + 1 + 255) / 256, 256, 0, s>>>(bin_off, cnt, B, items, w->n_items);
  CAPS_LAUNCH("k_items_fill");
  return CAPS_OK;
}

int bin_scan(const ScanArgs& a, const BinWork& w, uint64_t* part, int32_t* err, cudaStream_t s) {
  if (a.nq == 0) return CAPS_OK;
  if (!bin_scan_supported(a.d)) return fail(CAPS_EINVAL, "partition-major scan: unsupported d");
  BinScanArgs b;
  b.Xp = a.Xp;
  b.Ap = a.Ap;
  b.perm = a.perm;
  b.offsets = a.offsets;
  b.Q = a.Q;
  b.qmask = a.qp.qmask;
  b.qval = a.qp.qval;
  b.sel = a.sel;
  b.ent = w.ent;
  b.items = static_cast<const Item*>(w.items);
  b.n_items = w.n_items;
  b.m = a.m;
  b.h = a.h;
  b.d = a.d;
  b.k = a.k;
  b.R = a.d <= 128 ? 64 : 32;
  b.part = part;
  b.err = err;
  b.sp = a.sp;
  const size_t smem = bin_smem_total(b.R, a.d, a.words_pad);
  return a.metric == CAPS_L2 ? launch_bin_w<CAPS_L2>(b, a.words_pad, w.max_items, smem, s)
                             : launch_bin_w<CAPS_IP>(b, a.words_pad, w.max_items, smem, s);
}

int bin_merge(const ScanArgs& a, const uint64_t* part, cudaStream_t s) {
  if (a.nq == 0) return CAPS_OK;
  const unsigned mg = (unsigned)((a.nq + 3) / 4);
#define CAPS_MERGE(MET, KP) \
  k_merge_topk<MET, KP><<<mg, 128, 0, s>>>(part, a.qp.dead, a.nq, a.m, a.k, a.out_ids, a.out_dist)
  if (a.metric == CAPS_L2) {
    if (a.k <= 32) CAPS_MERGE(CAPS_L2, 1);
    else if (a.k <= 64) CAPS_MERGE(CAPS_L2, 2);
    else CAPS_MERGE(CAPS_L2, 4);
  } else {
    if (a.k <= 32) CAPS_MERGE(CAPS_IP, 1);
    else if (a.k <= 64) CAPS_MERGE(CAPS_IP, 2);
    else CAPS_MERGE(CAPS_IP, 4);
  }
#undef CAPS_MERGE
  CAPS_LAUNCH("k_merge_topk");
  return CAPS_OK;
}

}  // namespace caps
