// Internal declarations of the CAPS GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "caps.h"

namespace caps {

constexpr int kMaxFields = 16;  // dense attribute fields per point
constexpr int kMaxK = 128;      // neighbours per query
constexpr int kMaxH = 63;       // AFT height (h+1 blocks fit a 64-bit mask)

// Dense attribute model (Def. 1): field f takes values 0..vocab[f]-1.
// code(f, v) = code_off[f] + v enumerates all (field, value) pairs; the AFT
// tags are such codes.  For the scan, each row's values are packed into
// `words` 32-bit words: field f occupies `bits[f]` bits at `shift[f]` of word
// `word[f]` (fields never straddle a word).
struct DenseMeta {
  int L = 0;
  int vocab[kMaxFields] = {};
  int code_off[kMaxFields] = {};
  int word[kMaxFields] = {};
  int shift[kMaxFields] = {};
  int bits[kMaxFields] = {};
  int words = 0;       // packed words actually used (1..4)
  int words_pad = 0;   // row stride in words: 1, 2 or 4 (vector loads)
  int64_t n_codes = 0;
  // sparse label sets: L = 0, n_codes = the label vocabulary, and the two
  // packed words of a row hold its 64-bit label signature (bit
  // sig_bit(label) set for every label), so "(a & mask) == val" with
  // mask = val = the query's signature is a necessary condition for b <= a
  int sparse = 0;
};

// Signature bit of a sparse label (Fibonacci hashing of the label id).
__host__ __device__ __forceinline__ int sig_bit(int32_t label) {
  return (int)(((uint32_t)label * 2654435769u) >> 26);
}

// Sparse label filter (Def. 1, label sets): is every label the query requires
// present in the row's sorted label list?  roff/rlab: rows in layout order;
// qoff/qlab: the queries of the current chunk.  roff == nullptr: dense.
struct SparseRef {
  const int32_t* roff = nullptr;  // [N+1]
  const int32_t* rlab = nullptr;
  const int32_t* qoff = nullptr;  // [nq+1] (positions into qlab)
  const int32_t* qlab = nullptr;
};
__device__ __forceinline__ bool sp_subset(const SparseRef& s, int64_t row, int64_t q) {
  const int rb = s.roff[row], re = s.roff[row + 1];
  const int qe = s.qoff[q + 1];
  for (int i = s.qoff[q]; i < qe; i++) {
    const int32_t c = s.qlab[i];
    int lo = rb, hi = re;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s.rlab[mid] < c) lo = mid + 1;
      else hi = mid;
    }
    if (lo == re || s.rlab[lo] != c) return false;
  }
  return true;
}

// ---- orderable keys: (score, id) -> uint64, smaller key = better --------
// score is the fp32 distance for L2 and minus the inner product for IP; the
// low 32 bits hold the original point id so equal scores order by id.
__device__ __forceinline__ uint32_t ord_bits(float s) {
  uint32_t u = __float_as_uint(s + 0.0f);  // folds -0 into +0
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_bits(uint32_t u) {
  uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  return __uint_as_float(b);
}
__device__ __forceinline__ uint64_t make_key(float score, uint32_t id) {
  return ((uint64_t)ord_bits(score) << 32) | (uint64_t)id;
}

// Ascending bitonic sort of 32 * V keys held V per lane (key P = V * lane + s).
template <int V>
__device__ __forceinline__ void warp_sort(uint64_t (&v)[V], int lane) {
#pragma unroll
  for (int size = 2; size <= 32 * V; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride < V) {
#pragma unroll
        for (int s = 0; s < V; s++) {
          const int o = s ^ stride;
          if (o > s) {
            const bool up = ((V * lane + s) & size) == 0;
            const uint64_t a = v[s], b = v[o];
            if ((a > b) == up) {
              v[s] = b;
              v[o] = a;
            }
          }
        }
      } else {
#pragma unroll
        for (int s = 0; s < V; s++) {
          const int P = V * lane + s;
          const uint64_t o = __shfl_xor_sync(0xffffffffu, v[s], stride / V);
          const bool up = (P & size) == 0, lower = (P & stride) == 0;
          v[s] = (lower == up) ? (o < v[s] ? o : v[s]) : (o > v[s] ? o : v[s]);
        }
      }
    }
}

constexpr uint64_t kEmptyKey = ~0ull;

// Running k smallest keys of a warp: positions lane*KPL + s, ascending, the
// k-th at position k-1 (k <= 32*KPL).  offer() takes one key per lane and
// inserts every key that beats the current k-th, one at a time.
template <int KPL>
struct WarpTopK {
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

// ---- error handling --------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define CAPS_CUDA(call)                                          \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return ::caps::cuda_fail(_e, #call);  \
  } while (0)
// Kernels launched by this thread (every launch site checks through
// CAPS_LAUNCH, which also counts it).
extern thread_local long long g_kernel_launches;
#define CAPS_LAUNCH(what)                                        \
  do {                                                           \
    cudaError_t _e = cudaGetLastError();                         \
    if (_e != cudaSuccess) return ::caps::cuda_fail(_e, what);   \
    ++::caps::g_kernel_launches;                                 \
  } while (0)

// ---- device allocation gate ------------------------------------------------
// Every device allocation of the library goes through dev_alloc: it counts
// the calls (caps_alloc_count) and fails the n-th one on request
// (caps_inject_alloc_failure) as if the device were out of memory, without
// calling the allocator, so the CAPS_ENOMEM paths can be tested on the host.
// stream == nullptr: cudaMalloc; otherwise cudaMallocAsync on that stream.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t stream, bool async);

// ---- stream-ordered scratch ------------------------------------------------
// Temporary device buffers for one call, allocated from the stream-ordered
// pool and released on the same stream.
struct Scratch {
  cudaStream_t s;
  void* ptrs[256];
  int n = 0;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (int i = 0; i < n; i++) cudaFreeAsync(ptrs[i], s);
  }
  template <class T>
  int get(T** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    if (n == 256) return fail(CAPS_ENOMEM, "scratch slots exhausted");
    void* p = nullptr;
    cudaError_t e = dev_alloc(&p, count * sizeof(T), s, true);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(CAPS_ENOMEM, "device allocation failed for scratch");
    }
    ptrs[n++] = p;
    *out = (T*)p;
    return CAPS_OK;
  }
};

// ---- build-side launchers (build_kernels.cu) ------------------------------
int launch_gather_rows(const float* X, const int64_t* idx, int64_t n, int d,
                       float* out, cudaStream_t s);
// disjunctive constraints: per query, the best k of its sub-queries' results
// (sub-query rows soff[q] .. soff[q+1], k results each)
int launch_or_merge(const int64_t* sids, const float* sdist, const int64_t* soff, int64_t nq,
                    int k, int metric, int64_t* out_ids, float* out_dist, cudaStream_t s);
constexpr int kMaxOrCombos = 256;  // single-valued sub-queries per OR query
int launch_assign(const float* X, int64_t N, int d, const float* C, int B,
                  int metric, int32_t* bin, cudaStream_t s);
int launch_scores(const float* Q, int64_t nq, int d, const float* C, int B,
                  int metric, float* scores, cudaStream_t s);
// Stable counting sort of keys in [0, K): perm[r] = index of the r-th element
// in (key, index) order; seg_off[s] = first position of key s, seg_off[K] = n.
int stable_sort_by_key(const int32_t* keys, int64_t n, int64_t K, int32_t* perm,
                       int32_t* seg_off, Scratch& scr, cudaStream_t s);
int launch_centroid_update(const float* X, int d, const int32_t* perm_bin,
                           const int32_t* bin_off, int B, int metric, float* C,
                           Scratch& scr, cudaStream_t s);
int launch_check_dense(const int32_t* A, int64_t N, const DenseMeta& meta,
                       int32_t* bad, cudaStream_t s);
// sparse label sets (CSR, int64 offsets): every label in [0, V), strictly
// ascending per point; *bad = 1 otherwise.  Also writes int32 offsets.
int launch_check_sparse(const int64_t* off, const int32_t* lab, int64_t N, int32_t V,
                        int32_t* off32, int32_t* bad, cudaStream_t s);
int launch_aft_sparse(const int32_t* perm_bin, const int32_t* bin_off, int B, int h,
                      const int32_t* off, const int32_t* lab, int32_t V, int32_t* tags,
                      uint8_t* key, cudaStream_t s);
// signature words and label lists of the rows in layout order
int launch_layout_sparse(const int32_t* off, const int32_t* lab, const int32_t* perm, int64_t N,
                         uint32_t* Ap, int32_t* off_p, int32_t* lab_p, Scratch& scr,
                         cudaStream_t s);
int launch_aft(const int32_t* perm_bin, const int32_t* bin_off, int B, int h,
               const int32_t* A, const DenseMeta& meta, const uint8_t* code_field,
               int32_t* tags, uint8_t* key, cudaStream_t s);
int launch_segment_keys(const int32_t* bin, const uint8_t* key, int64_t N, int h,
                        int32_t* seg, cudaStream_t s);
int launch_layout(const float* X, const int32_t* A, const int32_t* perm, int64_t N,
                  int d, const DenseMeta& meta, float* Xp, uint32_t* Ap,
                  cudaStream_t s);
int launch_pos_table(const int32_t* tags, int B, int h, int64_t n_codes,
                     uint8_t* pos, cudaStream_t s);
int launch_code_field(const DenseMeta& meta, uint8_t* code_field, cudaStream_t s);
// dynamic insertion: the layout's rows and packed attributes back in id
// order (dense attributes), and the block of each new point
int launch_unlayout(const float* Xp, const uint32_t* Ap, const int32_t* perm, int64_t N, int d,
                    const DenseMeta& meta, float* X, int32_t* A, cudaStream_t s);
int launch_block_of(const int32_t* A, const int32_t* bin, int64_t n, const int32_t* tags, int h,
                    const DenseMeta& meta, const uint8_t* code_field, uint8_t* key, cudaStream_t s);

// ---- search-side launchers (search_kernels.cu) ----------------------------
struct QueryPrep {
  uint32_t* qmask;   // [nq * words_pad]
  uint32_t* qval;    // [nq * words_pad]
  int32_t* qcode;    // [nq * L] code of each constrained field, -1 = free
  uint8_t* dead;     // [nq] 1 = a constraint value lies outside the vocabulary
};
int launch_query_prep(const int32_t* Qb, int64_t nq, const DenseMeta& meta,
                      QueryPrep qp, cudaStream_t s);
// sparse constraints: qoff [nq+1] / qlab (int32, device); signature words,
// dead = a label outside [0, vocab)
int launch_query_prep_sparse(const int32_t* qoff, const int32_t* qlab, int64_t nq,
                             const DenseMeta& meta, QueryPrep qp, cudaStream_t s);
// sparse rule of Alg. 2: j* = the first block whose tag the query requires;
// blocks 1..min(j*, h) that have a tag (every tag is compatible with a label
// set) and h+1 iff j* = h+1
int launch_select_sparse(const int32_t* probe, int64_t nq, int m, int h, const int32_t* tags,
                         const uint8_t* pos, int64_t n_codes, const int32_t* qoff,
                         const int32_t* qlab, uint64_t* sel, cudaStream_t s);
int launch_topm(const float* scores, int64_t nq, int B, int m, int metric,
                int32_t* probe, cudaStream_t s);
int launch_select(const int32_t* probe, int64_t nq, int m, int h, const int32_t* tags,
                  const uint8_t* pos, int64_t n_codes, const uint8_t* code_field,
                  const int32_t* Qb, const DenseMeta& meta, const int32_t* qcode,
                  uint64_t* sel, cudaStream_t s);

struct ScanArgs {
  const float* Xp;
  const uint32_t* Ap;
  const int32_t* perm;
  const int32_t* offsets;
  const float* Q;
  QueryPrep qp;
  const int32_t* probe;
  const uint64_t* sel;
  int64_t nq;
  int m, h, d, k, metric, words_pad;
  int64_t* out_ids;
  float* out_dist;
  SparseRef sp;  // sparse label sets: exact check after the signature test
};
int launch_scan_topk(const ScanArgs& a, cudaStream_t s);

// ---- partition-major scan (scan_bin.cu) ------------------------------------
int scan_exclusive_i32(int32_t* data, int64_t n, Scratch& scr, cudaStream_t s);
struct BinWork {
  int32_t* ent = nullptr;      // [nq*m] probe entries sorted by partition
  void* items = nullptr;       // work items
  int32_t* n_items = nullptr;  // device count of work items
  int32_t* next_item = nullptr;  // work counter of a persistent scan (zeroed with the items)
  int64_t max_items = 0;       // grid bound
};
bool bin_scan_supported(int d);
int64_t bin_work_items_bound(int64_t ne, int B);
int bin_group(const int32_t* probe, int64_t ne, int B, BinWork* w, Scratch& scr, cudaStream_t s);
int bin_scan(const ScanArgs& a, const BinWork& w, uint64_t* part, int32_t* err, cudaStream_t s);
int bin_merge(const ScanArgs& a, const uint64_t* part, cudaStream_t s);

// ---- learned partitioner (mlp.cu) ------------------------------------------
// W1 [H,d] | b1 [H] | W2 [B,H] | b2 [B], one contiguous device block.
struct MlpNet {
  int d = 0, H = 0, B = 0;
  float* W1 = nullptr;
  float* b1 = nullptr;
  float* W2 = nullptr;
  float* b2 = nullptr;
  int64_t size() const { return (int64_t)H * d + H + (int64_t)B * H + B; }
  void bind(float* base) {
    W1 = base;
    b1 = W1 + (int64_t)H * d;
    W2 = b1 + H;
    b2 = W2 + (int64_t)B * H;
  }
};
int mlp_logits(const MlpNet& net, const float* X, int64_t n, float* Hd, float* Z, cudaStream_t s);
// Balanced assignment of n points (BLISS-style rounds): each point's R
// largest logits (ties to the lower partition), then in id order the
// least-loaded of them (ties to the earlier); loads start at load0 ([B]
// int64 device, or null for zeros).
int mlp_balanced_assign(const MlpNet& net, const float* X, int64_t n, int R, const int64_t* load0,
                        int32_t* bin, Scratch& scr, cudaStream_t s);
int mlp_hidden(const MlpNet& net, const float* X, int64_t n, float* Hd, cudaStream_t s);

// ---- exact top-m probe screened on the tensor cores (probe_tc.cu) ----------
// mode 0: logits of hidden rows A [n,K] against W [B,K] + bias (larger
// better); 1: L2 centroid distances of queries A [n,K] to W = centroids; 2:
// IP.  Writes the m-partition set of each query to probe [n,m] (order:
// certain partitions first, by index); Dt [n,B] is scratch.
bool probe_screen_supported(int K, int B, int m);
// Weight side of the screened probe (centroids or the MLP's output layer,
// B rows of K): bf16 [hi | lo | hi] rows of 3 * Kp (Kp = K rounded up to 64)
// and the rows' squared norms and norms; fixed once the index is built.
struct ProbeWeights {
  void* Wh = nullptr;
  float* wn2 = nullptr;
  float* wn = nullptr;
};
size_t probe_weights_elems(int K, int B);
int probe_weights_prepare(const float* W, int B, int K, const ProbeWeights& pw, cudaStream_t s);
// pw: the weight side prepared at build time, or null (prepared here)
int probe_screened(int mode, const float* A, int64_t n, int K, const float* W, const float* bias,
                   int B, int m, float* Dt, int32_t* probe, int32_t* err, Scratch& scr,
                   cudaStream_t s, const ProbeWeights* pw = nullptr);
int mlp_assign(const MlpNet& net, const float* X, int64_t n, int32_t* bin, Scratch& scr,
               cudaStream_t s);
int mlp_loss_grad(const MlpNet& net, const float* X, int64_t n, const float* Y, MlpNet* grad,
                  float* loss_dev, Scratch& scr, cudaStream_t s);
// The training step with bf16 weights and activations on the tensor cores
// (fp32 masters in net): Xb optional bf16 rows [n, ceil(d/64)*64] of X.
int mlp_loss_grad_bf16(const MlpNet& net, const float* X, const void* Xb, int64_t n,
                       const float* Y, MlpNet* grad, float* loss_dev, int32_t* err, Scratch& scr,
                       cudaStream_t s);
int mlp_train(MlpNet& net, const float* X, int64_t n, const float* Y, int epochs, int batch,
              float lr, float* losses_host, cudaStream_t s, bool bf16 = false);
// D[M, N] (fp32, row stride N) = A[M, Kt] . B[N, Kt]^T, bf16 operands in rows
// of Kt elements (Kt a multiple of 64, 16-byte aligned bases); tcgen05 tiles
// of 128 x 256; a bounded wait that expires sets *err.
int bf16_gemm_nt(const void* A, int64_t M, const void* Bm, int N, int Kt, float* D, int32_t* err,
                 cudaStream_t s);
int mlp_gather_rows(const float* X, const int64_t* idx, int64_t n, int d, float* out,
                    cudaStream_t s);

// ---- bf16 tensor-core scan + exact re-rank (scan_tc.cu) ---------------------
struct TcScanArgs {
  const uint64_t* sel;
  const uint32_t* qmask;
  const uint32_t* qval;
  const void* Qh;       // [nq*d] bf16 (or e4m3 with f8) queries
  int f8;               // 1: e4m3 rows and queries with per-row / per-query scales
  const float* qs;      // f8: [nq] per-query scales
  const float* xs;      // f8: [N+4] per-row scales
  const float* qn;      // [nq] fp32 squared norms
  const uint32_t* Ap;
  const int32_t* perm;
  const float* xn;      // [N+4] fp32 squared norms of the rows
  const int32_t* offsets;
  const void* tmap;     // CUtensorMap over the bf16 rows
  int m, h, d, kp, words_pad, metric;  // kp: keys kept per probe (16 or 32)
  int rerank;           // candidates re-scored exactly per query
  int tile_n;           // rows per tensor-core tile: 128 or 256 (0: 256)
  int pen;              // 1: filter folded into the MMA (the index has the code chunk)
  int pen_bits;         // packed attribute bits in the code chunk
  uint32_t pen_mask[4]; // which bits of each packed word are encoded
  float xn_max;         // largest squared row norm
  uint64_t* qslot;      // [nq*8] bound slots per query, set to all ones before the scan
  SparseRef sp;         // sparse label sets: exact check before a key is queued
  uint64_t* part;       // [nq*m*kp]
  int32_t* err;
  int64_t n_rows = 0;   // rows of the index (ids are below it)
  int split = 0;        // 1: rows and queries as two bf16 terms [hi | lo | code] (fp32 form)
};
constexpr int kMaxRerank = 256;  // candidates re-scored exactly per query (form 1)
// keys each partition keeps per probe: 10, 16 or 32, at least k and at least
// a quarter of the re-rank depth
int tc_kp(int k, int depth);
int tc_rerank_depth(int k, int factor);
bool tc_scan_supported(int d, int k, int kp, int words_pad, int f8 = 0);
// whether the per-pair filter form with N-row tiles fits in shared memory
bool tc_tile_fits(int d, int words_pad, int N, int f8);
bool tc_pen_supported(int d, int kp, int words_pad);
// columns of the penalty form's code chunk: two per encoded attribute bit,
// and for L2 three for the row's -|x|^2/2 (the chunk holds 64)
int tc_pen_columns(int pen_bits, int metric);
// test hook of the bounded waits: later scans withhold every copy and MMA of
// work item `item` and wait at most wait_ns at each bounded wait (item < 0:
// normal operation, default limit)
void tc_set_stall(long long item, unsigned long long wait_ns);
// What the bf16 form of an index is made from, and where it goes.
struct TcIndexPrep {
  const float* Xp;         // [N*d] rows in layout order
  int64_t N;
  int d;
  const int32_t* perm;     // layout row -> original id
  const uint32_t* Ap;      // [N*words_pad] packed attributes
  int words_pad;
  const int32_t* offsets;  // [B*nb+1] block offsets
  int B, nb;
  int pen, pen_bits;       // code chunk for the penalty form
  uint32_t pen_mask[4];
  int metric;              // CAPS_L2: the code chunk also carries -|x|^2/2
  int f8;                  // 1: e4m3 rows of ceil(d/128)*128 bytes + per-row scales
  int split = 0;           // 1: bf16 rows [hi | lo | code] of (2*ceil(d/64)+1)*64 columns
  float* xs;               // out (f8): [N] per-row scales
  void* Xb;                // out: [N*cols] bf16 rows, cols = d, or (ceil(d/64)+1)*64 with pen
  float* xn;               // out: [N] squared norms
  int32_t* iperm;          // out: original id -> layout row
  float* xn_max;           // out (host): largest squared norm
  void* tmap;              // out: CUtensorMap over Xb
};
int tc_prepare_index(const TcIndexPrep& p, cudaStream_t s);
int tc_query_prep(const float* Q, int64_t nq, int d, void* Qh, float* qn, int f8, float* qs,
                  cudaStream_t s, int split = 0);
// bf16 columns of a query or row's vector part (split: [hi | lo], each part
// padded to a multiple of 64)
inline int tc_vec_cols(int d, int split) { return split ? 2 * ((d + 63) / 64) * 64 : d; }
bool tc_split_supported(int d, int kp, int words_pad);
// item_cap: most probes per work item (1..128; 0: 128)
int tc_group(const int32_t* probe, const uint64_t* sel, int h, int64_t ne, int B, int item_cap,
             BinWork* w, Scratch& scr, cudaStream_t s);
int tc_scan(const TcScanArgs& t, const BinWork& w, cudaStream_t s);
int tc_merge_rerank(const TcScanArgs& t, const uint8_t* dead, int64_t nq, int k, const float* Q,
                    const float* Xp, const int32_t* iperm, int64_t* out_ids, float* out_dist,
                    cudaStream_t s);

}  // namespace caps

// The index object behind the opaque caps_index handle: owns every device
// array of one CAPS index (Alg. 1 output) and frees them on destruction.
struct caps_index {
  int64_t N = 0;
  int d = 0, B = 0, h = 0, metric = 0;
  caps::DenseMeta meta;
  float* C = nullptr;
  int32_t* bin = nullptr;
  uint8_t* key = nullptr;
  int32_t* tags = nullptr;
  int32_t* perm = nullptr;
  int32_t* offsets = nullptr;
  uint8_t* pos = nullptr;
  uint8_t* code_field = nullptr;
  float* Xp = nullptr;
  uint32_t* Ap = nullptr;
  int32_t* err = nullptr;  // device word: 1 after a bounded device wait expired
  // bf16 form (prec = CAPS_BF16): bf16 copy of the rows, their fp32 squared
  // norms, row of each original id, and a TMA tensor map over the bf16 rows
  int prec = CAPS_FP32;
  int rerank_factor = 4;
  // learned partitioner (part = CAPS_PART_MLP): weights and training labels
  int part = CAPS_PART_KMEANS;
  caps::MlpNet mlp;
  float* labels = nullptr;
  int64_t n_labels = 0;
  int32_t* label_bins = nullptr;  // [n_label_bins] the partitions the last labels were made from
  int64_t n_label_bins = 0;       // N at build time
  int balance_r = 0;              // > 0: BLISS's balanced assignment over R logits
  float arbiter_recall[2] = {-1.f, -1.f};  // build arbiter: k-means, learned
  void* Xb = nullptr;
  float* xn = nullptr;
  float* xs = nullptr;  // e4m3 form: per-row scales [N+4]
  caps::ProbeWeights pw;  // weight side of the screened probe (when it applies)
  int32_t* iperm = nullptr;
  alignas(128) unsigned char tmap[128] = {};
  // penalty form of the bf16 scan: each bf16 row carries a 64-column one-hot
  // code of its packed attribute bits and its block
  int pen = 0;
  int pen_bits = 0;
  uint32_t pen_mask[4] = {};
  float xn_max = 0.f;
  // sparse label sets of the rows, in layout order (CSR)
  int32_t* sp_off = nullptr;  // [N+1]
  int32_t* sp_lab = nullptr;  // [nnz]
  int64_t sp_nnz = 0;
  // launch shapes the autotuner chose, per (k, m): rows per tile, probes per
  // item, penalty form; later caps_search_batch calls with that (k, m) use them
  struct Shape {
    int tile_n, item_cap, pen;
  };
  mutable std::mutex tune_mu;
  mutable std::map<std::pair<int, int>, Shape> tuned;
  int64_t bytes = 0;
  std::vector<std::pair<void*, size_t>> allocs;
  // bumped by every insertion (the arrays move): plans made before it refuse to run
  int64_t generation = 0;

  template <class T>
  int alloc(T** p, size_t count) {
    if (count == 0) count = 1;
    void* q = nullptr;
    cudaError_t e = caps::dev_alloc(&q, count * sizeof(T), nullptr, false);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return caps::fail(CAPS_ENOMEM, "device allocation failed for an index array");
    }
    allocs.emplace_back(q, count * sizeof(T));
    bytes += (int64_t)(count * sizeof(T));
    *p = (T*)q;
    return CAPS_OK;
  }
  // free one array of this index (no-op for null)
  void release(void* q) {
    if (!q) return;
    for (size_t i = 0; i < allocs.size(); i++)
      if (allocs[i].first == q) {
        cudaFree(q);
        bytes -= (int64_t)allocs[i].second;
        allocs.erase(allocs.begin() + (ptrdiff_t)i);
        return;
      }
  }
  ~caps_index() {
    for (auto& a : allocs) cudaFree(a.first);
  }
};

