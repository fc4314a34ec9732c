// The persistent BF16 tensor-core scan kernel (Alg. 2 "attribute match" +
// "top-k vector match" on bf16 tiles with fp32 accumulation), shared by the
// two translation units that instantiate it: scan_tc.cu (block selection and
// attribute filter tested per (probe, row) in the epilogue) and
// scan_tc_pen.cu (both folded into the MMA as a penalty chunk).
//
// One CTA per SM takes work items (a partition and up to 128 of its probes)
// from a global counter.  The probes' query vectors (bf16) form the MMA A
// operand (M = 128, K-major, 128-byte swizzle) in shared memory; the
// partition's rows in the blocks any probe selected arrive as N-row bf16
// tiles by 2-D TMA (K-major, 128-byte swizzle), together with their attribute
// words, original ids and fp32 squared norms (1-D bulk copies).
// tcgen05.mma (kind::f16, bf16 x bf16 -> fp32, M = 128, K = 16 per
// instruction) writes the 128 x N dot products into tensor memory, one
// accumulator per pipeline stage.  In the epilogue four threads own probe p
// (TMEM lane p), one per quarter of the tile's rows: for every row the
// thread keeps the pair only if the probe selected the row's block and the
// row passes the probe's filter, forms the approximate score (L2:
// |x|^2 - 2 q.x in fp32, the query's own |q|^2 left out because keys are only
// ever compared with keys of the same query; IP: -q.x) and, if it beats the thread's
// current threshold, appends the key to a small queue in shared memory; when
// any lane's queue fills, the warp merges every queue into the lanes' sorted
// KP-key register lists with a fixed compare-exchange network (no divergent
// insertion).  Each partition so contributes its KP best keys per probe
// (KP >= k).
//
// Penalty form (PEN): every bf16 row carries one extra 64-column chunk: a
// one-hot code of its attribute bits (two columns per packed bit: "bit is
// 0", "bit is 1") and, for L2, -|x|^2/2 split exactly into three bf16 parts
// (h1 = bf16(v), h2 = bf16(v - h1), h3 = v - h1 - h2).  The A operand's
// matching chunk holds -P in the columns of the bit values a probe's filter
// rules out, 1 in the three norm columns, 0 elsewhere, so the accumulator of
// a pair is acc = q.x - |x|^2/2 - (P for every ruled-out bit the row has).
// A pair that passes has only exact zero products in the code columns, so
// its acc is the same fp32 value as without them; the approximate score is
// -2 acc = |x|^2 - 2 q.x (L2) or -acc = -q.x (IP), an exact scaling.  With
// P = 2^e >= 4 (max_x |x|^2 + |q|^2) a passing pair has acc >= -P/4 and a
// failing one acc <= -7P/8, so acc >= -P/2 is the whole filter.  The block
// selection needs no columns: Alg. 2's selection never leaves out a row that
// passes the filter, so a row of an unselected block never passes it.  The
// epilogue so reads one fp32 value per pair and compares it with one floor
// per probe (the list's bound turned into accumulator units, or the cut);
// only the rare pairs above the floor become keys.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "caps_internal.cuh"
#include <type_traits>

namespace caps {

struct TcItem {
  int32_t b, e0, ne, pad;
};

struct TcArgs {
  const int32_t* ent;
  const TcItem* items;
  const int32_t* n_items;
  int32_t* next_item;  // work counter, zeroed by the grouping step
  const uint64_t* sel;
  const uint32_t* qmask;
  const uint32_t* qval;
  const void* Qh;           // [nq*d] bf16 or e4m3 (F8) query rows
  const float* qs;          // F8: [nq] per-query scale
  const float* xs;          // F8: [N+4] per-row scale, layout order
  const float* qn;          // [nq]
  const uint32_t* Ap;
  const int32_t* perm;
  const float* xn;
  const int32_t* offsets;
  int m, h, d;
  int kcd;               // 64-column chunks of the vector part
  int kc;                // chunks in the MMA: kcd, + 1 in the penalty form
  int kp;
  int pen_bits;          // penalty form: packed attribute bits encoded (two columns each)
  uint32_t pen_mask[4];  // which bits of each packed word are encoded
  float xn_max;          // largest squared row norm
  uint64_t* qslot;       // [nq*8] per-query bound slots, all ones at the start
  int nslot;             // slots in use: ceil(rerank depth / kp)
  SparseRef sp;          // label sets: exact check before a key is queued
  uint64_t* part;        // [nq*m*kp]
  int32_t* err;
  int pen_ks;            // penalty form: 16-column MMA steps of the code chunk (used columns)
  int pen_norm;          // penalty form, L2: the chunk carries -|x|^2/2 after the bit columns
  uint64_t wait_ns;      // limit of every bounded wait (ns)
  int withhold;          // test hook: the producer issues no copy or MMA for this item (-1: none)
  int split;             // fp32 rows as two bf16 terms: chunks [hi | lo | code] on both sides,
                         // products hi.hi + hi.lo + lo.hi (64-row tiles)
};

namespace {

constexpr int TC_M = 128;     // probes per work item (MMA M, TMEM lanes)
constexpr int TC_C = 512;     // epilogue threads: four per probe (one per quarter tile)
constexpr int TC_T = TC_C + 64;  // + a producer warp (copies and MMAs) and a prep warp
constexpr int TC_PARTS = TC_C / TC_M;
// The entry (0..ne-1 of the item's probes) held by accumulator lane t: with
// c = ceil(ne / 4), lane quarter q holds entries q c .. q c + c - 1, so that an
// item's probes spread evenly over the four 32-lane quarters and their
// epilogue warps while neighbouring entries (similar block selections) stay
// in one warp.  A lane without an entry gets a value >= ne.
__device__ __forceinline__ int slot_entry(int t, int ne) {
  const int c = (ne + 3) >> 2, l = t & 31;
  return l < c ? (t >> 5) * c + l : TC_M;
}
constexpr int TC_Q = 12;      // per-thread candidate queue (merged when > 4 wait)
constexpr int TC_BOX = 128;   // rows per 2-D copy (the tensor map's box)
constexpr int TC_COLS = 512;  // tensor-memory columns: TC_COLS / N accumulator stages
constexpr int TC_PRODUCER = TC_C / 32;  // warp index of the producer
constexpr int TC_PREP = TC_PRODUCER + 1;  // warp index of the prep warp (next item's data)
constexpr int TC_SLOTS = 8;   // per-query bound slots (stride)
constexpr uint64_t kTcWaitNs = 1000000000ull;  // default limit of a bounded wait
// a waiting thread may sleep up to this long per try (it wakes when the
// phase completes), so spinning warps leave the issue slots to working ones
constexpr uint32_t kTcSuspendNs = 500;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}
// Bounded wait for the completion of the barrier phase with the given parity.
// Gives up after `limit` ns, or early once *fail is set (fail may be null).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const volatile int* fail,
                                          uint64_t limit) {
  const uint32_t a = su32(bar);
  const uint64_t t0 = gtimer();
  while (true) {
    for (int i = 0; i < 64; i++) {
      uint32_t done;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
          " selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(a), "r"(parity), "r"(kTcSuspendNs)
          : "memory");
      if (done) return true;
    }
    if (fail != nullptr && *fail) return false;
    if (gtimer() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void consumers_sync() {  // named barrier 1: the 16 epilogue warps
  asm volatile("bar.sync 1, %0;" ::"n"(TC_C) : "memory");
}
// named barrier 1 with an AND over the 16 epilogue warps' predicates
__device__ __forceinline__ bool consumers_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(TC_C)
      : "memory");
  return r != 0;
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}
// Instruction descriptor: bf16 x bf16 -> f32, A and B K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t id,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(id), "r"(acc));
}
// Instruction descriptor: e4m3 x e4m3 -> f32 (format code 0 for A and B), A
// and B K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f8(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f8(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t id,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
      "l"(ad), "l"(bd), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
// Eight accumulator columns of this warp's 32 lanes; the load is only issued
// here, tmem_wait() completes it (no use of v before that).
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}
// 16 accumulator columns of this warp's 32 lanes (issue only, as above).
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&v)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
                 "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]),
                 "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
}
// max of three floats in one instruction (a NaN operand is ignored)
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// Completes the outstanding loads; v is tied in so that no use of it moves above.
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7])
               :
               : "memory");
}

__host__ __device__ constexpr int tc_stages(int N, bool pen) { return pen ? 2 : TC_COLS / N; }
// accumulator stages in tensor memory (64-row tiles: four, to leave shared
// memory for the wider rows of the split form)
__host__ __device__ constexpr int tc_acc_stages(int N) { return N == 64 ? 4 : TC_COLS / N; }
// rows per 2-D copy: the tensor map's box (64-row tiles use a 64-row box)
__host__ __device__ constexpr int tc_box_rows(int N) { return N < TC_BOX ? N : TC_BOX; }
__host__ __device__ constexpr size_t tc_a_bytes(int kc) { return (size_t)kc * TC_M * 128; }
__host__ __device__ constexpr size_t tc_b_bytes(int kc, int N) { return (size_t)kc * N * 128; }
// per stage: attribute words, ids, norms and (e4m3 rows) scales of N + 8
// rows (4-row aligned superset of the tile), block id of each row
__host__ __device__ constexpr size_t tc_aux_bytes(int WP, int N, bool f8 = false) {
  return (((size_t)(N + 8) * WP * 4 + (size_t)(N + 8) * (f8 ? 12 : 8) + (size_t)(N + 8)) + 15) &
         ~(size_t)15;
}
// shared memory one CTA may hold (227 KB), and an upper bound of the
// kernel's static part (barriers, per-probe arrays, the tile schedule)
constexpr size_t kTcSmemLimit = 227 * 1024;
__host__ __device__ constexpr size_t tc_static_bound(int WP, bool pen) {
  return 7168 + 1024 * (size_t)WP + (pen ? (size_t)4096 : 0);
}
__host__ __device__ constexpr size_t tc_smem_bytes(int kc, int WP, int N, bool pen, bool f8 = false);
__host__ __device__ constexpr bool tc_fits(int kc, int WP, int N, bool pen, bool f8 = false) {
  return tc_smem_bytes(kc, WP, N, pen, f8) + tc_static_bound(WP, pen) <= kTcSmemLimit;
}
__host__ __device__ constexpr size_t tc_smem_bytes(int kc, int WP, int N, bool pen, bool f8) {
  // 1024-byte alignment slack + A + B stages + candidate queues + aux stages
  // (one per accumulator stage; the final merge of the quarter lists reuses
  // the queues)
  return 1024 + tc_a_bytes(kc) + (size_t)tc_stages(N, pen) * tc_b_bytes(kc, N) +
         (size_t)TC_Q * TC_C * 8 + (size_t)tc_acc_stages(N) * tc_aux_bytes(WP, N, f8);
}

template <int KP>
__device__ __forceinline__ void net_insert(uint64_t (&L)[KP], uint64_t x) {
  // sorted ascending; x goes to the first position whose key is not below
  // it, the keys from there on move down by one and the largest falls off
  // the end (an empty key changes nothing).  Every position is decided from
  // its own and its predecessor's key alone, so the KP compares and selects
  // are independent of one another (no chain through the list).
  bool lt[KP];
#pragma unroll
  for (int i = 0; i < KP; i++) lt[i] = L[i] < x;
#pragma unroll
  for (int i = KP - 1; i > 0; i--) L[i] = lt[i] ? L[i] : (lt[i - 1] ? x : L[i - 1]);
  L[0] = lt[0] ? L[0] : x;
}

// L (ascending) becomes the KP smallest keys of L and the ascending list at
// other[i * TC_M]: the pairwise minima of L and the reversed other list are
// those keys as a bitonic sequence (rising, then falling); zero keys in front
// (below every key) pad it to a power of two, and a bitonic merger sorts it.
template <int KP>
__device__ __forceinline__ void net_merge(uint64_t (&L)[KP], const uint64_t* other) {
  constexpr int P = KP <= 16 ? 16 : 32;
  static_assert(KP <= P && P <= 32, "list too long");
  uint64_t c[P];
#pragma unroll
  for (int i = 0; i < P - KP; i++) c[i] = 0ull;
#pragma unroll
  for (int i = 0; i < KP; i++) {
    const uint64_t o = other[(size_t)(KP - 1 - i) * TC_M];
    c[P - KP + i] = L[i] < o ? L[i] : o;
  }
#pragma unroll
  for (int st = P / 2; st > 0; st >>= 1)
#pragma unroll
    for (int i = 0; i < P; i++)
      if ((i & st) == 0) {
        const uint64_t x = c[i], y = c[i + st];
        c[i] = x < y ? x : y;
        c[i + st] = x < y ? y : x;
      }
#pragma unroll
  for (int i = 0; i < KP; i++) L[i] = c[P - KP + i];
}

// One persistent CTA per SM walks the work items (partition, <= 128 probes)
// in the order a global counter hands them out, so partitions of very
// different sizes balance across the SMs within one launch.  Warp 16 is the
// producer.  Its copies run ahead of its MMAs: before tile t's MMAs it starts
// the copies of tile t + SB - 1 — the rows into the B stage of tile t - 1
// (free once that tile's MMAs completed) and the rows' ids, norms, attribute
// words and block ids into the aux stage of that tile's accumulator (free
// once the epilogue has read it) — then waits for tile t's rows and issues
// its MMAs into accumulator stage t mod ST.  After the item's last tile it
// already takes and prepares the next item (its rows' ranges and the probes'
// data) while the epilogue finishes the current one.  Warps 0-15 are the
// epilogue; they meet the producer only through mbarriers (full: rows
// landed; bfree: B stage's MMAs done; aux: ids and norms landed; mma:
// accumulator written; empty: all 16 warps done with the accumulator and aux
// stage; taken: the probes' data read; meta: the next item's data ready;
// afull: the next item's A operand built), and at item boundaries, where
// they merge the probes' quarter lists and build the next item's A operand.
//
// Bound across a query's partitions: the rerank keeps the best R keys of the
// query's m lists.  Each finished list offers its KP-th key to one of the
// query's ns = ceil(R / KP) slots (slot = the probe's rank mod ns, atomic
// min).  Once every slot holds a key, the largest of them, T, has at least
// ns * KP >= R keys of distinct lists at or below it, so a later partition
// of that query drops every key above T: such a key cannot be among the R
// best.
template <int METRIC, int WP, int KP, int N, bool PEN, bool F8>
__global__ void __launch_bounds__(TC_T, 1)
k_scan_tc(const __grid_constant__ CUtensorMap tmX, TcArgs a) {
  // SB shared-memory stages hold B tiles (free once the tile's MMAs are
  // done); ST accumulator stages in tensor memory, each with the tile's ids,
  // norms, attribute words and block ids (free once the epilogue read them)
  constexpr int SB = tc_stages(N, PEN), ST = tc_acc_stages(N);
  constexpr int BOXR = tc_box_rows(N);
  constexpr int RA = N + 8;
  constexpr int CPT = N / TC_PARTS;  // accumulator columns per epilogue thread and tile
  extern __shared__ unsigned char smem_raw[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kc = a.kc, nb = a.h + 1;
  const int n_items = *a.n_items;

  // 1024-byte alignment by pointer arithmetic on the shared array itself, so
  // that every pointer derived from it stays a shared-memory pointer (shared
  // loads and stores, not generic ones)
  unsigned char* base = smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  unsigned char* sA = base;
  unsigned char* sB0 = sA + tc_a_bytes(kc);
  const size_t bstride = tc_b_bytes(kc, N);
  uint64_t* queue = reinterpret_cast<uint64_t*>(sB0 + SB * bstride);
  unsigned char* aux0 = reinterpret_cast<unsigned char*>(queue + (size_t)TC_Q * TC_C);
  constexpr size_t astride = tc_aux_bytes(WP, N, F8);
  auto s_attr = [&](int b) { return reinterpret_cast<uint32_t*>(aux0 + b * astride); };
  auto s_perm = [&](int b) {
    return reinterpret_cast<int32_t*>(aux0 + b * astride + (size_t)RA * WP * 4);
  };
  auto s_xn = [&](int b) {
    return reinterpret_cast<float*>(aux0 + b * astride + (size_t)RA * WP * 4 + RA * 4);
  };
  auto s_xs = [&](int b) {
    return reinterpret_cast<float*>(aux0 + b * astride + (size_t)RA * WP * 4 + RA * 8);
  };
  auto s_blk = [&](int b) { return aux0 + b * astride + (size_t)RA * WP * 4 + RA * (F8 ? 12 : 8); };
  static_assert(!(PEN && F8), "the penalty form is bf16 only");

  __shared__ uint64_t full_bar[SB], bfree_bar[SB], aux_bar[ST], mma_bar[ST], empty_bar[ST];
  __shared__ uint64_t taken_bar, meta_bar[2], afull_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;
  // the current and the next item (index: item parity)
  __shared__ int s_ne[2], s_ntiles[2], s_bin[2], s_item[2];
  __shared__ uint64_t p_thr[2][TC_M];
  // penalty form: the score bits of each quarter list's ceil(KP/4)-th and
  // ceil(KP/4) - 1-th keys (all ones until it has that many); the per-pair
  // form has no shared memory to spare for them
  __shared__ uint32_t s_qa[PEN ? TC_PARTS : 1][TC_M], s_qb[PEN ? TC_PARTS : 1][TC_M];
  __shared__ int32_t p_e[2][TC_M];
  // probe data of the item about to start (read once into registers)
  __shared__ uint64_t p_sel[TC_M];
  __shared__ uint32_t p_qm[TC_M * WP], p_qv[TC_M * WP];
  __shared__ float p_qn[TC_M];
  __shared__ float p_cut[TC_M];  // penalty form: scores at or above are masked pairs
  // producer only: tile schedule of its item
  __shared__ int s_tlo[ST], s_tn[ST];
  // the tile schedule (runs of selected blocks) of the current and the next item
  __shared__ int run_lo[2][64], run_hi[2][64], run_j0[2][64];
  __shared__ int n_runs[2];
  __shared__ int32_t boff[2][65];
  __shared__ uint8_t s_pbit[32];  // penalty form: word * 32 + bit of the g-th encoded bit

  if (tid == 0) {
    for (int i = 0; i < SB; i++) {
      mbar_init(&full_bar[i], 1);
      mbar_init(&bfree_bar[i], 1);
    }
    for (int i = 0; i < ST; i++) {
      mbar_init(&aux_bar[i], 1);
      mbar_init(&mma_bar[i], 1);
      mbar_init(&empty_bar[i], TC_C / 32);
    }
    mbar_init(&taken_bar, TC_C / 32);
    mbar_init(&meta_bar[0], 1);
    mbar_init(&meta_bar[1], 1);
    mbar_init(&afull_bar, TC_C / 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i < (PEN ? TC_PARTS : 1) * TC_M; i++) (&s_qa[0][0])[i] = (&s_qb[0][0])[i] = ~0u;
    s_fail = 0;
    int gb = 0;
    for (int w = 0; w < WP; w++)
      for (uint32_t um = a.pen_mask[w]; um && gb < 32; um &= um - 1) s_pbit[gb++] = (uint8_t)(32 * w + __ffs(um) - 1);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base)),
                 "n"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = F8 ? idesc_f8(TC_M, N) : idesc_bf16(TC_M, N);

  // ---- producer: take the next item and prepare everything but A ----------
  // (fills s_ne/s_ntiles/s_bin/p_e/p_thr[par], the probe data, the runs)
  auto prep_meta = [&](int par) -> bool {
    int id = 0;
    if (lane == 0) id = atomicAdd(a.next_item, 1);
    id = __shfl_sync(0xffffffffu, id, 0);
    if (id >= n_items) {
      if (lane == 0) {
        s_ne[par] = -1;
        s_item[par] = -1;
      }
      return false;
    }
    const TcItem pit = a.items[id];
    const int32_t* off = a.offsets + (int64_t)pit.b * nb;
    int32_t* bo = boff[par];
    for (int j = lane; j <= nb; j += 32) bo[j] = off[j];
    uint64_t U = 0ull;
#pragma unroll
    for (int i = 0; i < TC_M / 32; i++) {
      const int t = lane + 32 * i;
      uint64_t sel = 0ull, T = kEmptyKey;
      float qn = 0.f;
      int e = 0;
      uint32_t qm[WP], qv[WP];
#pragma unroll
      for (int w = 0; w < WP; w++) qm[w] = qv[w] = 0u;
      const int jt = slot_entry(t, pit.ne);
      if (jt < pit.ne) {
        e = a.ent[pit.e0 + jt];
        const int q = e / a.m;
        sel = a.sel[e];
        qn = a.qn[q];
#pragma unroll
        for (int w = 0; w < WP; w++) {
          qm[w] = a.qmask[(int64_t)q * WP + w];
          qv[w] = a.qval[(int64_t)q * WP + w];
        }
        const uint64_t* sl = a.qslot + (int64_t)q * TC_SLOTS;
        T = 0ull;
        for (int i = 0; i < a.nslot; i++) {
          const uint64_t v = sl[i];
          T = v > T ? v : T;
        }
      }
      U |= sel;
      p_e[par][t] = e;
      p_thr[par][t] = T;
      p_sel[t] = sel;
      p_qn[t] = qn;
#pragma unroll
      for (int w = 0; w < WP; w++) {
        p_qm[t * WP + w] = qm[w];
        p_qv[t * WP + w] = qv[w];
      }
      // penalty form: P = 2^ex >= 4 (max |x|^2 + |q|^2); a pair passes the
      // filter iff its accumulator is >= -P/2 (the cut; +inf: no probe)
      float cut = INFINITY;
      if (PEN && jt < pit.ne) {
        const float bound = 4.f * (a.xn_max + qn);
        int ex = (int)((__float_as_uint(bound) >> 23) & 0xffu) - 126;  // 2^ex >= bound
        ex = max(0, min(126, ex));
        cut = __uint_as_float(0x80000000u | ((uint32_t)(ex + 126) << 23));
      }
      p_cut[t] = cut;
    }
    const uint32_t ulo = __reduce_or_sync(0xffffffffu, (uint32_t)U);
    const uint32_t uhi = __reduce_or_sync(0xffffffffu, (uint32_t)(U >> 32));
    U = ((uint64_t)uhi << 32) | ulo;
    __syncwarp();
    if (lane == 0) {
      int nr = 0, nt = 0, j = 0;
      while (j < nb) {
        if (!((U >> j) & 1ull)) {
          j++;
          continue;
        }
        int j2 = j;
        while (j2 + 1 < nb && ((U >> (j2 + 1)) & 1ull)) j2++;
        if (bo[j2 + 1] > bo[j]) {
          run_lo[par][nr] = bo[j];
          run_hi[par][nr] = bo[j2 + 1];
          run_j0[par][nr] = j;
          nt += (bo[j2 + 1] - bo[j] + N - 1) / N;
          nr++;
        }
        j = j2 + 1;
      }
      n_runs[par] = nr;
      s_ntiles[par] = nt;
      s_ne[par] = pit.ne;
      s_bin[par] = pit.b;
      s_item[par] = id;
    }
    __syncwarp();
    return true;
  };
  // ---- epilogue threads: the A operand of the prepared item ---------------
  // row t = probe t's query, bf16, zero-padded to kcd*64 coordinates, 16-byte
  // unit u of chunk c stored at unit u ^ (t%8); four threads per row, one per
  // quarter of the units.  In the penalty form one more chunk: -P in the
  // column of every attribute bit value the probe's filter rules out, 1 in
  // the three columns of the rows' -|x|^2/2 parts (L2), 0 elsewhere.
  auto build_a = [&](int par) {
    const int t = tid & (TC_M - 1), qq = tid / TC_M;
    const int ne_n = s_ne[par];
    const int q = slot_entry(t, ne_n) < ne_n ? p_e[par][t] / a.m : -1;
    // 16-byte units: 8 bf16 or 16 e4m3 coordinates
    const int rowb = a.d * (F8 ? 1 : 2);
    const int units = a.kcd * 8, dunits = rowb / 16;
    const unsigned char* qrow = static_cast<const unsigned char*>(a.Qh) + (int64_t)(q < 0 ? 0 : q) * rowb;
    const int u0 = qq * units / TC_PARTS, u1 = (qq + 1) * units / TC_PARTS;
#pragma unroll 4
    for (int u = u0; u < u1; u++) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (q >= 0 && u < dunits) v = *reinterpret_cast<const uint4*>(qrow + 16 * u);
      const int c = u >> 3, uu = u & 7;
      *reinterpret_cast<uint4*>(sA + (size_t)c * TC_M * 128 + t * 128 + ((uu ^ (t & 7)) << 4)) = v;
    }
    if (PEN) {
      // each of the row's four threads computes 16 of the chunk's columns
      uint16_t negP = 0;
      if (q >= 0) {
        const float bound = 4.f * (a.xn_max + p_qn[t]);
        int ex = (int)((__float_as_uint(bound) >> 23) & 0xffu) - 126;  // 2^ex >= bound
        ex = max(0, min(126, ex));
        negP = (uint16_t)(0x8000u | ((uint32_t)(ex + 127) << 7));
      }
      const int nbit = 2 * a.pen_bits;
      const int nnorm = a.pen_norm ? 3 : 0;
      uint32_t w32[8];
#pragma unroll
      for (int h = 0; h < 16; h++) {
        const int c = 16 * qq + h;
        uint32_t v = 0u;
        if (q >= 0) {
          if (c < nbit) {  // the column of the bit value the filter rules out
            const int pb = s_pbit[c >> 1], w = pb >> 5, i = pb & 31;
            const uint32_t qm = p_qm[t * WP + w], qv = p_qv[t * WP + w];
            if (((qm >> i) & 1u) && (uint32_t)(c & 1) != ((qv >> i) & 1u)) v = (uint32_t)negP;
          } else if (c < nbit + nnorm) {  // times the row's -|x|^2/2 parts
            v = 0x3F80u;                  // bf16 1.0
          }
        }
        if (h & 1) w32[h >> 1] |= v << 16;
        else w32[h >> 1] = v;
      }
      unsigned char* rowp = sA + (size_t)a.kcd * TC_M * 128 + t * 128;
      *reinterpret_cast<uint4*>(rowp + (((2 * qq) ^ (t & 7)) << 4)) =
          make_uint4(w32[0], w32[1], w32[2], w32[3]);
      *reinterpret_cast<uint4*>(rowp + (((2 * qq + 1) ^ (t & 7)) << 4)) =
          make_uint4(w32[4], w32[5], w32[6], w32[7]);
    }
    fence_async_smem();  // generic stores of A before the MMAs read it
  };

  if (warp == TC_PREP) prep_meta(0);
  __syncthreads();
  if (warp < TC_PRODUCER && s_ne[0] >= 0) {
    build_a(0);
    __syncwarp();
    if (lane == 0) mbar_arrive(&afull_bar);  // the producer may issue the item's MMAs
  }
  // ---- prep warp: item i + 1's data while item i runs ---------------------
  // Once the epilogue has taken item i's probe data (which also means the
  // producer is done with item i - 1's tile schedule), the next item's
  // metadata, probe data and tile schedule go into the other buffer, and
  // meta_bar[i % 2] completes.  Two barriers: the producer waits for item
  // i's data only at item i's start, by which time item i + 1's data may
  // already be complete too.
  if (warp == TC_PREP) {
    for (int i = 0; s_ne[i & 1] >= 0; i++) {
      bool ok = s_fail == 0 && mbar_wait(&taken_bar, (uint32_t)(i & 1), &s_fail, a.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) s_fail = 1;
        break;
      }
      prep_meta((i & 1) ^ 1);
      __syncwarp();
      if (lane == 0) mbar_arrive(&meta_bar[i & 1]);  // item i + 1's data is ready
    }
  }

  int g0 = 0;           // tiles this CTA finished before the current item
  int par = 0, n_done = 0;
  int tma_hi = -1, mma_hi = -1;  // producer: last tile whose copies / MMAs were issued
  while (warp <= TC_PRODUCER) {
    if (warp == TC_PRODUCER && n_done > 0) {  // this item's data, from the prep warp
      const int j = n_done - 1;
      const bool ok = s_fail == 0 &&
                      mbar_wait(&meta_bar[j & 1], (uint32_t)((j >> 1) & 1), &s_fail, a.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) s_fail = 1;
        break;
      }
    }
    const int ne = s_ne[par];
    if (ne < 0 || s_fail) break;
    const int n_tiles = s_ntiles[par];

    if (warp == TC_PRODUCER) {
      // ---- producer ------------------------------------------------------
      // copies run ahead of the MMAs: before tile t's MMAs the copy of tile
      // t + SB - 1 is issued, into the B stage of tile t - 1 (free once that
      // tile's MMAs are done) and the aux stage of tile t + SB - 1 - ST (free
      // once the epilogue has read it)
      const int* rl = run_lo[par];
      const int* rh = run_hi[par];
      const int* rj = run_j0[par];
      const int32_t* bo = boff[par];
      int rr = 0, rlo = n_runs[par] > 0 ? rl[0] : 0;
      bool ok = true;
      int tl = 0;  // next tile of this item to copy
      auto load = [&](int t) -> bool {  // warp-uniform
        const int g = g0 + t, sb = g % SB, st = g % ST;
        while (rlo >= rh[rr]) {
          rr++;
          rlo = rl[rr];
        }
        const int lo = rlo, n = min(N, rh[rr] - rlo), j0 = rj[rr];
        rlo += n;
        bool k = true;
        if (g >= SB) k = mbar_wait(&bfree_bar[sb], (uint32_t)((g / SB - 1) & 1), &s_fail, a.wait_ns);
        if (k && g >= ST)
          k = mbar_wait(&empty_bar[st], (uint32_t)((g / ST - 1) & 1), &s_fail, a.wait_ns);
        if (!__all_sync(0xffffffffu, k)) return false;
        if (!PEN) {
          uint8_t* blk = s_blk(st);
          for (int r = lane; r < n; r += 32) {
            int j = j0;
            while (j + 1 < nb && bo[j + 1] <= lo + r) j++;
            blk[r] = (uint8_t)j;
          }
        }
        if (lane == 0) {
          s_tlo[st] = lo;
          s_tn[st] = n;
        }
        __syncwarp();
        if (lane == 0) {
          const int alo = lo & ~3;
          const int arows = ((lo + n + 3) & ~3) - alo;
          const uint32_t ab = PEN ? 0u : (uint32_t)(arows * WP * 4), pb = (uint32_t)(arows * 4);
          unsigned char* sB = sB0 + sb * bstride;
          expect_tx(&full_bar[sb], (uint32_t)(kc * N * 128));
          for (int c = 0; c < kc; c++)
#pragma unroll
            for (int hb = 0; hb < N / BOXR; hb++)
              tma_2d(sB + (size_t)c * N * 128 + (size_t)hb * BOXR * 128, &tmX, 64 * c,
                     lo + hb * BOXR, &full_bar[sb]);
          // ids (and, per-pair form, attribute words and norms; e4m3 scales):
          // the penalty form needs only the ids
          expect_tx(&aux_bar[st], ab + (PEN ? 1 : (F8 ? 3 : 2)) * pb);
          if (!PEN) bulk_copy(s_attr(st), a.Ap + (int64_t)alo * WP, ab, &aux_bar[st]);
          bulk_copy(s_perm(st), a.perm + alo, pb, &aux_bar[st]);
          if (!PEN) bulk_copy(s_xn(st), a.xn + alo, pb, &aux_bar[st]);
          if (F8) bulk_copy(s_xs(st), a.xs + alo, pb, &aux_bar[st]);
          tma_hi = g;
        }
        return true;
      };
      // test hook: a withheld item gets no copy and no MMA, so the epilogue's
      // bounded wait for its first tile expires with nothing left in flight
      const int n_issue = s_item[par] == a.withhold ? 0 : n_tiles;
      // MMA steps per tile: four per vector chunk, and the used part of the
      // penalty chunk; the split form multiplies three chunk pairs for each
      // chunk of the vector: hi.hi, hi.lo, lo.hi
      const int hcd = a.kcd >> 1;  // split form: chunks of the hi part
      const bool split = N == 64 && a.split;  // (64-row tiles only)
      const int ksteps = split ? 12 * hcd + (PEN ? a.pen_ks : 0)
                               : (PEN ? (kc - 1) * 4 + a.pen_ks : kc * 4);
      while (ok && tl < n_issue && tl < SB - 1) ok = load(tl++);
      for (int t = 0; ok && t < n_issue; t++) {
        if (tl < n_issue) ok = load(tl++);
        if (!ok) break;
        const int g = g0 + t, sb = g % SB, st = g % ST;
        if (lane == 0) {
          ok = mbar_wait(&full_bar[sb], (uint32_t)((g / SB) & 1), &s_fail, a.wait_ns);
          // the item's first MMA waits for its A operand
          if (ok && t == 0) ok = mbar_wait(&afull_bar, (uint32_t)(n_done & 1), &s_fail, a.wait_ns);
          if (ok) {
            tc_fence_after();
            // descriptors of the stage bases once; a step's operand is the
            // base plus its byte offset / 16 (the address field of the
            // descriptor; shared addresses stay below 256 KB, so no carry)
            const uint64_t adb = sdesc(su32(sA)), bdb = sdesc(su32(sB0 + sb * bstride));
            const uint32_t dt = tbase + (uint32_t)(st * N);
            if (split) {
              // two accumulators, so that consecutive MMAs do not wait on
              // one another: D0 (columns st N) takes hi.hi and hi.lo, D1
              // (columns 256 + st N) takes lo.hi and the code chunk; the
              // epilogue adds them.  The MMAs alternate between the two.
              const uint32_t dt1 = dt + 256u;
              const int n1 = hcd + (PEN ? 1 : 0);
              for (int i = 0; i < 2 * hcd; i++) {
                const int c0a = i < hcd ? i : i - hcd, c0b = i;  // D0's chunk pair
                const bool has1 = i < n1;
                const int c1a = i < hcd ? hcd + i : a.kcd, c1b = i < hcd ? i : a.kcd;
                const int nk1 = i < hcd ? 4 : a.pen_ks;
                const uint64_t ad0 = adb + (uint64_t)(c0a * TC_M * 8), bd0 = bdb + (uint64_t)(c0b * N * 8);
                const uint64_t ad1 = adb + (uint64_t)(c1a * TC_M * 8), bd1 = bdb + (uint64_t)(c1b * N * 8);
#pragma unroll
                for (int kin = 0; kin < 4; kin++) {
                  mma_bf16(dt, ad0 + (uint64_t)(2 * kin), bd0 + (uint64_t)(2 * kin), idesc,
                           (i > 0 || kin > 0) ? 1u : 0u);
                  if (has1 && kin < nk1)
                    mma_bf16(dt1, ad1 + (uint64_t)(2 * kin), bd1 + (uint64_t)(2 * kin), idesc,
                             (i > 0 || kin > 0) ? 1u : 0u);
                }
              }
            }
            const int nch = split ? 0 : (ksteps + 3) >> 2;  // 64-column chunks (the code chunk may be partial)
            for (int c = 0; c < nch; c++) {
              int ca = c, cb = c;  // the chunks of A and B this chunk step multiplies
              if (split) {
                if (c >= 3 * hcd) ca = cb = a.kcd;                  // code chunk
                else if (c >= 2 * hcd) ca = c - hcd, cb = c - 2 * hcd;  // lo . hi
                else if (c >= hcd) ca = c - hcd;                   // hi . lo
              }
              const uint64_t ad = adb + (uint64_t)(ca * TC_M * 8), bd = bdb + (uint64_t)(cb * N * 8);
              const int nk = min(4, ksteps - 4 * c);
#pragma unroll
              for (int kin = 0; kin < 4; kin++) {
                if (kin < nk) {
                  const uint32_t acc = (c > 0 || kin > 0) ? 1u : 0u;
                  if (F8) mma_f8(dt, ad + (uint64_t)(2 * kin), bd + (uint64_t)(2 * kin), idesc, acc);
                  else mma_bf16(dt, ad + (uint64_t)(2 * kin), bd + (uint64_t)(2 * kin), idesc, acc);
                }
              }
            }
            mma_commit(&mma_bar[st]);
            mma_commit(&bfree_bar[sb]);
            mma_hi = g;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
      }
      if (!ok && lane == 0) s_fail = 1;
    } else {
      // ---- epilogue ------------------------------------------------------
      // (items follow one another without a CTA barrier: the next item's A
      // operand is built as soon as this item's MMAs are done, while the
      // producer already streams the next item's tiles)
      const int probe = tid & (TC_M - 1), part = tid / TC_M;
      const bool active = slot_entry(probe, ne) < ne;
      const uint64_t my_sel = p_sel[probe];
      uint32_t my_qm[WP], my_qv[WP];
#pragma unroll
      for (int w = 0; w < WP; w++) {
        my_qm[w] = p_qm[probe * WP + w];
        my_qv[w] = p_qv[probe * WP + w];
      }
      const float my_cut = PEN ? p_cut[probe] : 0.f;
      const int my_q = active ? p_e[par][probe] / a.m : 0;
      const float my_qs = F8 && active ? a.qs[my_q] : 1.f;  // e4m3: the query's scale
      __syncwarp();
      if (lane == 0) mbar_arrive(&taken_bar);  // the producer may refill the probe data
      uint64_t* pthr = p_thr[par];
      uint64_t L[KP];
#pragma unroll
      for (int i = 0; i < KP; i++) L[i] = kEmptyKey;
      uint64_t thr = kEmptyKey;
      int qcnt = 0;
      // Merge every queue into its lanes' lists (warp-uniform call: as many
      // rounds as the fullest queue; the next round's key is loaded while the
      // current one is inserted).
      auto flush = [&]() {
        const int mx = __reduce_max_sync(0xffffffffu, (unsigned)qcnt);
        uint64_t nx = qcnt > 0 ? queue[tid] : kEmptyKey;
#pragma unroll 1
        for (int i = 0; i < mx; i++) {
          const uint64_t x = nx;
          nx = i + 1 < qcnt ? queue[(size_t)(i + 1) * TC_C + tid] : kEmptyKey;
          net_insert<KP>(L, x);
        }
        qcnt = 0;
        thr = L[KP - 1];
        // the four threads of a probe share the smallest of their KP-th keys:
        // a key above it has KP better keys in one quarter list already
        if (thr != kEmptyKey) atomicMin(reinterpret_cast<unsigned long long*>(&pthr[probe]), thr);
        // and a bound from all four lists (of distinct rows): with QB =
        // ceil(KP/4), the NHI quarters whose QB-th keys are smallest count QB
        // keys each and the others QB - 1, KP keys in all at or below the
        // largest of those keys' scores.  A slot read before its quarter's
        // latest flush is larger, so the bound holds
        if constexpr (PEN) {
          constexpr int QB = (KP + TC_PARTS - 1) / TC_PARTS;
          constexpr int NHI = KP - TC_PARTS * (QB - 1);
          static_assert(QB >= 2 && NHI >= 1 && NHI <= TC_PARTS, "quarter split");
          s_qa[part][probe] = (uint32_t)(L[QB - 1] >> 32);
          s_qb[part][probe] = (uint32_t)(L[QB - 2] >> 32);
          uint32_t qa[TC_PARTS], qb[TC_PARTS];
#pragma unroll
          for (int pp = 0; pp < TC_PARTS; pp++) {
            qa[pp] = s_qa[pp][probe];
            qb[pp] = s_qb[pp][probe];
          }
          // order the quarters by their QB-th key (compare-exchange network)
          auto cx = [&](int i, int j) {
            if (qa[j] < qa[i]) {
              const uint32_t ta = qa[i], tb = qb[i];
              qa[i] = qa[j];
              qb[i] = qb[j];
              qa[j] = ta;
              qb[j] = tb;
            }
          };
          cx(0, 1);
          cx(2, 3);
          cx(0, 2);
          cx(1, 3);
          cx(1, 2);
          uint32_t bs = qa[NHI - 1];
#pragma unroll
          for (int pp = NHI; pp < TC_PARTS; pp++) bs = qb[pp] > bs ? qb[pp] : bs;
          const uint64_t mq = ((uint64_t)bs << 32) | 0xffffffffull;
          if (mq != kEmptyKey) {
            atomicMin(reinterpret_cast<unsigned long long*>(&pthr[probe]), mq);
            if (mq < thr) thr = mq;
          }
        }
      };
      const bool warp_live = __any_sync(0xffffffffu, active);
      const int cbeg = part * CPT;
      // The next item's A operand, built as soon as every MMA of this item
      // has completed (right after the wait for the last tile's accumulator;
      // at once for an item without tiles), so that its MMAs run while this
      // item's last tile and list merge are still in the epilogue.
      auto next_a = [&]() {
        const bool ok = s_fail == 0 && mbar_wait(&meta_bar[n_done & 1], (uint32_t)((n_done >> 1) & 1),
                                                 &s_fail, a.wait_ns);
        if (!__all_sync(0xffffffffu, ok)) {
          s_fail = 1;
          return;
        }
        if (s_ne[par ^ 1] >= 0) {
          build_a(par ^ 1);
          __syncwarp();
          if (lane == 0) mbar_arrive(&afull_bar);  // the producer may issue the item's MMAs
        }
      };
      // penalty form: the smallest accumulator value that can still enter
      // this thread's list (the list's bound in accumulator units, never
      // below the filter cut; +inf for a lane without a probe)
      auto floor_of = [&](uint64_t tk) -> float {
        if (tk == kEmptyKey) return my_cut;
        const float ts = unord_bits((uint32_t)(tk >> 32));
        return fmaxf(METRIC == CAPS_L2 ? -0.5f * ts : -ts, my_cut);
      };
      if (n_tiles == 0) next_a();
      for (int t = 0; t < n_tiles; t++) {
        const int g = g0 + t, b = g % ST, u = g / ST;
        const bool ok = mbar_wait(&aux_bar[b], (uint32_t)(u & 1), &s_fail, a.wait_ns) &&
                        mbar_wait(&mma_bar[b], (uint32_t)(u & 1), &s_fail, a.wait_ns);
        if (!__all_sync(0xffffffffu, ok)) {  // warp-uniform: the loads below are collective
          s_fail = 1;
          break;
        }
        tc_fence_after();
        if (t == n_tiles - 1) next_a();  // every MMA of the item has completed
        const int lo = s_tlo[b], n = s_tn[b];
        const int alo = lo & ~3;
        const uint32_t* attr = s_attr(b) + (lo - alo) * WP;
        const int32_t* prm = s_perm(b) + (lo - alo);
        const float* xnr = s_xn(b) + (lo - alo);
        const float* xsr = s_xs(b) + (lo - alo);
        const uint8_t* blk = s_blk(b);
        const uint32_t tacc = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(b * N + cbeg);
        const int ncol = warp_live ? min(CPT, n - cbeg) : 0;  // warp-uniform
        if constexpr (PEN) {
          // the thread's CPT accumulators in loads of 16; the largest of
          // each 8 against the floor; only lanes with a value at or above it
          // turn pairs into keys
          static_assert(CPT % 16 == 0, "the penalty form reads 16 columns at a time");
          float fl;
#pragma unroll 1
          for (int h16 = 0; h16 < CPT / 16 && 16 * h16 < ncol; h16++) {  // warp-uniform bounds
            // the probe's shared bound, fresh for every 16 columns
            {
              const uint64_t st = pthr[probe];
              if (st < thr) thr = st;
            }
            fl = floor_of(thr);
            uint32_t v[16];
            tmem_ld16_issue(tacc + (uint32_t)(16 * h16), v);
            if constexpr (N == 64) {
              // the split form's second accumulator (columns + 256)
              uint32_t v2[16];
              tmem_ld16_issue(tacc + 256u + (uint32_t)(16 * h16), v2);
              tmem_wait16(v);
              tmem_wait16(v2);
#pragma unroll
              for (int j = 0; j < 16; j++)
                v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(v2[j]));
            } else {
              tmem_wait16(v);
            }
            const int c0 = cbeg + 16 * h16, lim = ncol - 16 * h16;
            if (lim < 16) {  // rows past the end of the tile's run
#pragma unroll
              for (int j = 0; j < 16; j++)
                if (j >= lim) v[j] = 0xff800000u;  // -inf
            }
            const float mx = fmax3(fmax3(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2])),
                                   fmax3(__uint_as_float(v[3]), __uint_as_float(v[4]), __uint_as_float(v[5])),
                                   fmax3(__uint_as_float(v[6]), __uint_as_float(v[7]), __uint_as_float(v[8])));
            const float my = fmax3(fmax3(__uint_as_float(v[9]), __uint_as_float(v[10]), __uint_as_float(v[11])),
                                   fmax3(__uint_as_float(v[12]), __uint_as_float(v[13]), __uint_as_float(v[14])),
                                   __uint_as_float(v[15]));
            if (__any_sync(0xffffffffu, fmaxf(mx, my) >= fl)) {
#pragma unroll
              for (int hh = 0; hh < 2; hh++) {
                // the lane's hot columns of this half as a bit mask; a half no
                // lane needs is skipped by the whole warp.  Keys of a hot half
                // are built for all 8 columns at once (the columns' ids are
                // broadcast loads) and stored only where the lane's bit is
                // set, at positions from a prefix count: no column waits for
                // another.
                uint32_t hm = 0u;
#pragma unroll
                for (int j = 0; j < 8; j++)
                  hm |= (__uint_as_float(v[8 * hh + j]) >= fl ? 1u : 0u) << j;
                if (__any_sync(0xffffffffu, hm != 0u)) {
#pragma unroll
                  for (int j = 0; j < 8; j++) {
                    const float acc = __uint_as_float(v[8 * hh + j]);
                    const uint64_t key = make_key(METRIC == CAPS_L2 ? -2.f * acc : -acc,
                                                  (uint32_t)prm[c0 + 8 * hh + j]);
                    if ((hm >> j) & 1u)
                      queue[(size_t)(qcnt + __popc(hm & ((1u << j) - 1u))) * TC_C + tid] = key;
                  }
                  qcnt += __popc(hm);
                  // at most 8 more keys per lane before the next check
                  if (__any_sync(0xffffffffu, qcnt > TC_Q - 8)) {
                    flush();
                    fl = floor_of(thr);
                  }
                }
              }
            }
          }
        }
        const int ngr = (!PEN && ncol > 0) ? (ncol + 7) >> 3 : 0;
#pragma unroll 1
        for (int gi = 0; gi < ngr; gi++) {
          uint32_t cur[8];
          tmem_ld8_issue(tacc + (uint32_t)(8 * gi), cur);
          tmem_wait(cur);
          const int c0 = cbeg + 8 * gi;
          {
            const uint64_t st = pthr[probe];
            if (st < thr) thr = st;
          }
          const int lim = n - c0;  // rows of this group inside the tile
          {
            // the 8 rows' block ids and attribute words in few wide loads
            // (the same addresses for every lane: broadcast)
            const uint2 bw = *reinterpret_cast<const uint2*>(blk + c0);
            const uint32_t bb[2] = {bw.x, bw.y};
            uint32_t aw[8 * WP];
            if (WP == 1 && ((lo - alo + c0) & 3) == 0) {
              const uint4 a0 = *reinterpret_cast<const uint4*>(attr + c0);
              const uint4 a1 = *reinterpret_cast<const uint4*>(attr + c0 + 4);
              aw[0] = a0.x; aw[1] = a0.y; aw[2] = a0.z; aw[3] = a0.w;
              aw[4] = a1.x; aw[5] = a1.y; aw[6] = a1.z; aw[7] = a1.w;
            } else {
#pragma unroll
              for (int x = 0; x < 8 * WP; x++) aw[x] = attr[c0 * WP + x];
            }
#pragma unroll
            for (int j = 0; j < 8; j++) {
              const int bj = (bb[j >> 2] >> (8 * (j & 3))) & 0xff;
              bool pass = j < lim && ((my_sel >> bj) & 1ull);
#pragma unroll
              for (int w = 0; w < WP; w++) pass = pass && ((aw[j * WP + w] & my_qm[w]) == my_qv[w]);
              if (pass) {
                const int r = c0 + j;
                float dot = __uint_as_float(cur[j]);
                if (F8) dot *= my_qs * xsr[r];  // the rows' and the query's scales
                const float sc = METRIC == CAPS_L2 ? fmaf(-2.f, dot, xnr[r]) : -dot;
                const uint64_t key = make_key(sc, (uint32_t)prm[r]);
                // label sets: the signature test above is necessary; the
                // exact test runs only for keys that would enter the list
                if (key < thr && (!a.sp.roff || sp_subset(a.sp, lo + r, my_q))) {
                  queue[(size_t)qcnt * TC_C + tid] = key;
                  qcnt++;
                }
              }
            }
          }
          // at most 8 more keys per lane before the next check: merge once
          // any queue holds more than TC_Q - 8
          if (__any_sync(0xffffffffu, qcnt > TC_Q - 8)) flush();
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[b]);
      }
      flush();
      consumers_sync();  // every queue drained: the queue area holds the quarter lists
      // merge the four quarter lists of each probe: in two levels (parts 1
      // and 3 hand theirs to parts 0 and 2, then part 2 to part 0) when two
      // lists per probe fit in the queue area, else one list at a time
      uint64_t* parts = queue;
      bool fine = s_fail == 0;
      static_assert(TC_PARTS == 4 && KP * TC_M <= TC_Q * TC_C, "quarter lists");
      if constexpr (2 * KP * TC_M <= TC_Q * TC_C) {
        if (fine && (part & 1)) {
#pragma unroll
          for (int i = 0; i < KP; i++) parts[((size_t)(part >> 1) * KP + i) * TC_M + probe] = L[i];
        }
        consumers_sync();
        if (fine && !(part & 1) && active)
          net_merge<KP>(L, parts + (size_t)(part >> 1) * KP * TC_M + probe);
        if (fine && part == 2) {  // into the slot only this thread read
#pragma unroll
          for (int i = 0; i < KP; i++) parts[((size_t)KP + i) * TC_M + probe] = L[i];
        }
        consumers_sync();
        if (fine && part == 0 && active) net_merge<KP>(L, parts + (size_t)KP * TC_M + probe);
        // (the barrier before the next item's first queue write follows below)
      } else {
        for (int src = 1; src < TC_PARTS; src++) {
          if (fine && part == src) {
#pragma unroll
            for (int i = 0; i < KP; i++) parts[(size_t)i * TC_M + probe] = L[i];
          }
          consumers_sync();
          if (fine && part == 0 && active) net_merge<KP>(L, parts + probe);
          consumers_sync();
        }
      }
      if (fine && part == 0 && active) {
        const int e = p_e[par][probe];
        uint64_t* dst = a.part + (int64_t)e * KP;
#pragma unroll
        for (int i = 0; i < KP; i++) dst[i] = L[i];
        // offer the list's KP-th key to the query's bound (slot = the probe's
        // rank mod the slot count: distinct lists per slot)
        if (L[KP - 1] != kEmptyKey)
          atomicMin(reinterpret_cast<unsigned long long*>(
                        a.qslot + (int64_t)(e / a.m) * TC_SLOTS + (e % a.m) % a.nslot),
                    (unsigned long long)L[KP - 1]);
      }
      if (PEN) s_qa[part][probe] = s_qb[part][probe] = ~0u;  // read again only after the barrier below
      // (the next item's A operand was built at its last tile) every thread
      // is done with this item's lists and quarter bounds before any starts
      // the next item's queue writes and flushes
      consumers_sync();
    }
    g0 += n_tiles;
    n_done++;
    par ^= 1;
  }

  // every thread is out of the item loop before the failure flag is read:
  // a producer that ran out of items may leave the loop before a wait of
  // the epilogue expires
  __syncthreads();
  if (s_fail) {
    // a copy or an MMA did not complete in time: flag it, let what is in
    // flight land (bounded waits), release tensor memory and leave
    if (warp == TC_PRODUCER && lane == 0) {
      atomicExch(a.err, 1);
      for (int g = max(0, tma_hi - SB + 1); g <= tma_hi; g++)
        mbar_wait(&full_bar[g % SB], (uint32_t)((g / SB) & 1), nullptr, a.wait_ns);
      for (int g = max(0, tma_hi - ST + 1); g <= tma_hi; g++)
        mbar_wait(&aux_bar[g % ST], (uint32_t)((g / ST) & 1), nullptr, a.wait_ns);
      for (int g = max(0, mma_hi - ST + 1); g <= mma_hi; g++)
        mbar_wait(&mma_bar[g % ST], (uint32_t)((g / ST) & 1), nullptr, a.wait_ns);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(TC_COLS));
}

template <int METRIC, int WP, int KP, int N, bool PEN, bool F8 = false>
int launch_tc(const CUtensorMap& map, const TcArgs& a, int64_t grid, size_t smem, cudaStream_t s) {
  auto kern = k_scan_tc<METRIC, WP, KP, N, PEN, F8>;
  cudaFuncAttributes fa;
  CAPS_CUDA(cudaFuncGetAttributes(&fa, kern));
  if (smem + fa.sharedSizeBytes > kTcSmemLimit)
    return fail(CAPS_EINVAL, "tensor-core tile shape does not fit in shared memory");
  CAPS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)grid, TC_T, smem, s>>>(map, a);
  CAPS_LAUNCH("k_scan_tc");
  return CAPS_OK;
}

}  // namespace

// Launch of the e4m3 form (scan_tc_f8.cu): per-pair filter, N = 256 or 128
// rows per tile; kp 10, 16 or 32.
int tc_launch_f8(const CUtensorMap& map, const TcArgs& a, int metric, int words_pad, int kp, int N,
                 int64_t grid, size_t smem, cudaStream_t s);
// Launch of the penalty form (scan_tc_pen.cu): N = 128 rows per tile (64
// for the split form), two B-tile stages and four accumulator stages; kp 10
// or 16.
int tc_launch_pen(const CUtensorMap& map, const TcArgs& a, int metric, int words_pad, int kp,
                  int64_t grid, size_t smem, cudaStream_t s, int N = 128);

}  // namespace caps
