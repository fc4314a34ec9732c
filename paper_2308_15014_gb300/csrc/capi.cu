// C ABI of the CAPS GB300 library: argument checks, host/device staging and
// the order of the kernels for index construction (Alg. 1) and batched query
// (Alg. 2).  All arithmetic of the method runs in the kernels.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_set>
#include <vector>

#include "caps_internal.cuh"

namespace caps {

static thread_local std::string g_err;
thread_local long long g_kernel_launches = 0;

void set_error(const std::string& msg) { g_err = msg; }
int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return CAPS_ECUDA;
}

static std::atomic<long long> g_alloc_calls{0};
static std::atomic<long long> g_alloc_fail_at{0};  // 0: no failure armed

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t stream, bool async) {
  *p = nullptr;
  const long long n = ++g_alloc_calls;
  long long at = g_alloc_fail_at.load();
  if (at != 0 && n >= at && g_alloc_fail_at.compare_exchange_strong(at, 0))
    return cudaErrorMemoryAllocation;
  return async ? cudaMallocAsync(p, bytes, stream) : cudaMalloc(p, bytes);
}

namespace {

// int64 offsets -> int32, flagging negative, oversized or decreasing ones
__global__ void k_offsets_i32(const int64_t* __restrict__ in, int64_t n, int32_t* __restrict__ out,
                              int32_t* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t v = in[i];
  if (v < 0 || v > INT32_MAX || (i > 0 && v < in[i - 1])) atomicExch(bad, 1);
  out[i] = (int32_t)v;
}

// Is p a pointer the current device can dereference (device or managed)?
int is_device_ptr(const void* p, bool* dev) {
  *dev = false;
  if (!p) return CAPS_OK;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CAPS_OK;  // unknown to CUDA: plain host memory
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
    int cur = 0;
    CAPS_CUDA(cudaGetDevice(&cur));
    if (at.type == cudaMemoryTypeDevice && at.device != cur)
      return fail(CAPS_EINVAL, "device pointer belongs to another GPU");
    *dev = true;
  }
  return CAPS_OK;
}

// Device view of an input array: the pointer itself, or a stream-ordered copy.
template <class T>
int stage_in(const T* src, size_t count, Scratch& scr, cudaStream_t s, const T** out) {
  *out = nullptr;
  if (count == 0) return CAPS_OK;
  if (!src) return fail(CAPS_EINVAL, "null input array");
  bool dev = false;
  if (int rc = is_device_ptr(src, &dev)) return rc;
  if (dev) {
    *out = src;
    return CAPS_OK;
  }
  T* d = nullptr;
  if (int rc = scr.get(&d, count)) return rc;
  CAPS_CUDA(cudaMemcpyAsync(d, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
  *out = d;
  return CAPS_OK;
}

// Host copy of a small input array (for validation and metadata).
template <class T>
int to_host(const T* src, size_t count, std::vector<T>* out, cudaStream_t s) {
  out->assign(count, T());
  if (count == 0) return CAPS_OK;
  if (!src) return fail(CAPS_EINVAL, "null input array");
  bool dev = false;
  if (int rc = is_device_ptr(src, &dev)) return rc;
  if (!dev) {
    std::memcpy(out->data(), src, count * sizeof(T));
    return CAPS_OK;
  }
  CAPS_CUDA(cudaMemcpyAsync(out->data(), src, count * sizeof(T), cudaMemcpyDeviceToHost, s));
  CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

// Output array: the caller's device pointer, or scratch copied back later.
template <class T>
struct Out {
  T* user = nullptr;
  T* dev = nullptr;
  size_t count = 0;
  bool host = false;
  int init(T* u, size_t n, Scratch& scr) {
    user = u;
    count = n;
    if (n == 0) return CAPS_OK;
    if (!u) return fail(CAPS_EINVAL, "null output array");
    bool d = false;
    if (int rc = is_device_ptr(u, &d)) return rc;
    host = !d;
    if (d) {
      dev = u;
      return CAPS_OK;
    }
    return scr.get(&dev, n);
  }
  int finish(cudaStream_t s) {
    if (host && count)
      CAPS_CUDA(cudaMemcpyAsync(user, dev, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    return CAPS_OK;
  }
};

void keep_pool_warm() {
  static bool done = false;
  if (done) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done = true;
}

// SplitMix64 (Steele, Lea, Flood 2014) driving Floyd's sampling of B
// distinct seed ids out of N.
uint64_t splitmix64(uint64_t* st) {
  uint64_t z = (*st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
std::vector<int64_t> floyd_sample(int64_t N, int64_t B, uint64_t seed) {
  std::vector<int64_t> out;
  std::unordered_set<int64_t> seen;
  uint64_t st = seed;
  for (int64_t j = N - B; j < N; j++) {
    const int64_t t = (int64_t)(splitmix64(&st) % (uint64_t)(j + 1));
    const int64_t v = seen.count(t) ? j : t;
    seen.insert(v);
    out.push_back(v);
  }
  return out;
}

int make_meta(const caps_attrs* at, cudaStream_t s, DenseMeta* meta) {
  if (!at) return fail(CAPS_EINVAL, "attributes are required");
  if (at->dense == nullptr) {
    // sparse label sets: codes = labels, two packed words = the signature
    if (!at->sp_offsets) return fail(CAPS_EINVAL, "attributes need dense values or sparse labels");
    if (at->sp_vocab < 1 || at->sp_vocab > (1 << 24))
      return fail(CAPS_EINVAL, "sp_vocab must be in [1, 2^24]");
    DenseMeta m;
    m.L = 0;
    m.words = 2;
    m.words_pad = 2;
    m.n_codes = at->sp_vocab;
    m.sparse = 1;
    *meta = m;
    return CAPS_OK;
  }
  if (at->L <= 0) return fail(CAPS_EINVAL, "dense attributes need L >= 1");
  if (at->L > kMaxFields) return fail(CAPS_EINVAL, "more than 16 attribute fields");
  std::vector<int32_t> vocab;
  if (int rc = to_host(at->vocab, (size_t)at->L, &vocab, s)) return rc;
  DenseMeta m;
  m.L = at->L;
  int64_t off = 0;
  int word = 0, used = 0;
  for (int f = 0; f < m.L; f++) {
    if (vocab[f] < 1) return fail(CAPS_EINVAL, "vocab entries must be >= 1");
    m.vocab[f] = vocab[f];
    m.code_off[f] = (int)off;
    off += vocab[f];
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)vocab[f]) bits++;
    if (used + bits > 32) {
      word++;
      used = 0;
    }
    m.word[f] = word;
    m.shift[f] = used;
    m.bits[f] = bits;
    used += bits;
  }
  if (off > (int64_t)1 << 24) return fail(CAPS_EINVAL, "too many attribute codes (sum of vocab)");
  m.words = word + 1;
  if (m.words > 4) return fail(CAPS_EINVAL, "packed attributes exceed 128 bits");
  m.words_pad = m.words == 1 ? 1 : (m.words == 2 ? 2 : 4);
  m.n_codes = off;
  *meta = m;
  return CAPS_OK;
}

}  // namespace
}  // namespace caps

using namespace caps;

extern "C" const char* caps_last_error(void) { return g_err.c_str(); }

extern "C" int64_t caps_alloc_count(void) { return (int64_t)g_alloc_calls.load(); }

extern "C" void caps_inject_alloc_failure(int64_t n) {
  g_alloc_fail_at.store(n > 0 ? g_alloc_calls.load() + n : 0);
}

extern "C" void caps_test_scan_stall(int64_t item, uint64_t wait_ns) {
  tc_set_stall((long long)item, (unsigned long long)wait_ns);
}

namespace caps {
namespace {
// Label of training point s: normalised histogram of the partitions of its
// first label_k search results other than itself (its own partition when it
// has none).
__global__ void k_mlp_labels(const int64_t* __restrict__ ids, int kq, const int64_t* __restrict__ samples,
                             int64_t S, int label_k, const int32_t* __restrict__ bin, int B,
                             float* __restrict__ Y) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= S) return;
  const int64_t self = samples[r];
  int cnt = 0;
  for (int j = 0; j < kq && cnt < label_k; j++) {
    const int64_t i = ids[r * kq + j];
    if (i < 0 || i == self) continue;
    cnt++;
  }
  float* y = Y + r * B;
  if (cnt == 0) {
    y[bin[self]] = 1.f;
    return;
  }
  const float w = 1.f / (float)cnt;
  int seen = 0;
  for (int j = 0; j < kq && seen < cnt; j++) {
    const int64_t i = ids[r * kq + j];
    if (i < 0 || i == self) continue;
    y[bin[i]] += w;
    seen++;
  }
}
__global__ void k_mlp_cons(const int32_t* __restrict__ A, int L, const int64_t* __restrict__ samples,
                           const uint8_t* __restrict__ keep, int64_t S, int32_t* __restrict__ cons) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= S * L) return;
  const int64_t r = t / L, f = t % L;
  cons[t] = keep[t] ? A[samples[r] * L + f] : -1;
}
// Points per partition from the (partition, block) offsets.
__global__ void k_part_loads(const int32_t* __restrict__ offsets, int B, int h,
                             int64_t* __restrict__ load) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) load[b] = (int64_t)offsets[(int64_t)(b + 1) * (h + 1)] - offsets[(int64_t)b * (h + 1)];
}
double u01(uint64_t* st) { return (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0); }
}  // namespace
}  // namespace caps

// Filters of S data points on their own attributes: each field kept with
// probability 1/2 (SplitMix64(seed), row by row), at least one per point.
static int draw_cons(const int32_t* dA, int L, const int64_t* dS, int64_t S, uint64_t seed,
                     Scratch& scr, cudaStream_t s, int32_t** out) {
  std::vector<uint8_t> keep((size_t)S * L, 0);
  uint64_t st = seed;
  for (int64_t r = 0; r < S; r++) {
    int any = 0;
    for (int f = 0; f < L; f++) {
      keep[r * L + f] = u01(&st) < 0.5 ? 1 : 0;
      any |= keep[r * L + f];
    }
    if (!any) keep[r * L + (int)(splitmix64(&st) % (uint64_t)L)] = 1;
  }
  uint8_t* dkeep = nullptr;
  if (int rc = scr.get(&dkeep, (size_t)S * L)) return rc;
  if (int rc = scr.get(out, (size_t)S * L)) return rc;
  CAPS_CUDA(cudaMemcpyAsync(dkeep, keep.data(), keep.size(), cudaMemcpyHostToDevice, s));
  k_mlp_cons<<<(unsigned)((S * L + 255) / 256), 256, 0, s>>>(dA, L, dS, dkeep, S, *out);
  CAPS_LAUNCH("k_mlp_cons");
  CAPS_CUDA(cudaStreamSynchronize(s));  // `keep` leaves scope
  return CAPS_OK;
}

// The build's arbiter between k-means and the learned partitioner: held-out
// data points as queries, filtered on their own attributes, recall@10 of the
// m-probe search against their exact filtered neighbours (themselves left
// out).
namespace {
constexpr int kArbiterK = 10;
struct Arbiter {
  int64_t J = 0;
  std::vector<int64_t> qid;    // query point ids
  const float* Q = nullptr;    // [J*d]
  const int32_t* cons = nullptr;
  std::vector<int64_t> exact;  // [J*(kArbiterK+1)]
};
}  // namespace

static int arbiter_prepare(const caps_build_params* p, const float* dX, const int32_t* dA, int64_t N,
                         int d, int L, Scratch& scr, cudaStream_t s, Arbiter* jg) {
  jg->J = std::min<int64_t>(p->mlp_arbiter_queries, N);
  jg->qid = floyd_sample(N, jg->J, p->seed + 5);
  int64_t* dq = nullptr;
  if (int rc = scr.get(&dq, (size_t)jg->J)) return rc;
  CAPS_CUDA(cudaMemcpyAsync(dq, jg->qid.data(), sizeof(int64_t) * jg->J, cudaMemcpyHostToDevice, s));
  float* Q = nullptr;
  if (int rc = scr.get(&Q, (size_t)jg->J * d)) return rc;
  if (int rc = mlp_gather_rows(dX, dq, jg->J, d, Q, s)) return rc;
  int32_t* cons = nullptr;
  if (int rc = draw_cons(dA, L, dq, jg->J, p->seed + 6, scr, s, &cons)) return rc;
  jg->Q = Q;
  jg->cons = cons;
  return CAPS_OK;
}

// ids of the arbiter queries' k+1 best at m probes (fp32 scan)
static int arbiter_search(caps_index* ix, const Arbiter& jg, int m, cudaStream_t s,
                        std::vector<int64_t>* out) {
  const int kq = kArbiterK + 1;
  Scratch scr(s);
  int64_t* ids = nullptr;
  float* dist = nullptr;
  if (int rc = scr.get(&ids, (size_t)jg.J * kq)) return rc;
  if (int rc = scr.get(&dist, (size_t)jg.J * kq)) return rc;
  caps_attrs ca;
  ca.L = ix->meta.L;
  ca.dense = jg.cons;
  ca.vocab = nullptr;
  ca.sp_offsets = nullptr;
  ca.sp_labels = nullptr;
  ca.sp_vocab = 0;
  const int keep_prec = ix->prec;
  ix->prec = CAPS_FP32;
  const int rc_s = caps_search_batch(ix, jg.Q, jg.J, &ca, kq, m, ids, dist, s);
  ix->prec = keep_prec;
  if (rc_s) return rc_s;
  out->resize((size_t)jg.J * kq);
  CAPS_CUDA(cudaMemcpyAsync(out->data(), ids, sizeof(int64_t) * out->size(), cudaMemcpyDeviceToHost, s));
  CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

// mean over the queries with a neighbour of |found ∩ exact| / |exact|, both
// the first 10 valid ids other than the query point itself
static float arbiter_recall(const Arbiter& jg, const std::vector<int64_t>& got) {
  const int kq = kArbiterK + 1;
  double sum = 0.0;
  int64_t cnt = 0;
  for (int64_t j = 0; j < jg.J; j++) {
    auto first = [&](const std::vector<int64_t>& v, std::vector<int64_t>* o) {
      o->clear();
      for (int t = 0; t < kq && (int)o->size() < kArbiterK; t++) {
        const int64_t i = v[j * kq + t];
        if (i >= 0 && i != jg.qid[j]) o->push_back(i);
      }
    };
    std::vector<int64_t> g, f;
    first(jg.exact, &g);
    first(got, &f);
    if (g.empty()) continue;
    int hit = 0;
    for (int64_t i : f)
      for (int64_t e : g) hit += i == e;
    sum += (double)hit / (double)g.size();
    cnt++;
  }
  return cnt ? (float)(sum / (double)cnt) : 1.f;
}

// Learned partitioner (Sec. 5.2): labels from exact filtered neighbours over
// the k-means index, Adam training, f(x) = argmax logits into ix->bin.
static int build_mlp(const caps_build_params* p, const float* dX, const int32_t* dA, int64_t N,
                     int d, const DenseMeta& meta, cudaStream_t s, caps_index* ix) {
  const int B = p->B, L = meta.L;
  const int H = p->mlp_hidden > 0 ? p->mlp_hidden : 512;
  const int64_t S = p->mlp_samples > 0 ? std::min<int64_t>(p->mlp_samples, N)
                                       : std::min<int64_t>(N, 32768);
  const int batch = p->mlp_batch > 0 ? p->mlp_batch : 4096;
  const float lr = p->mlp_lr > 0.f ? p->mlp_lr : 1e-3f;
  const int lk = p->mlp_label_k > 0 ? p->mlp_label_k : 10;
  Scratch scr(s);
  // training points
  std::vector<int64_t> samp;
  if (p->mlp_sample_idx) {
    if (int rc = to_host(p->mlp_sample_idx, (size_t)S, &samp, s)) return rc;
    for (int64_t v : samp)
      if (v < 0 || v >= N) return fail(CAPS_EINVAL, "mlp_sample_idx entry outside [0, N)");
  } else {
    samp = floyd_sample(N, S, p->seed + 1);
  }
  int64_t* dS = nullptr;
  if (int rc = scr.get(&dS, (size_t)S)) return rc;
  CAPS_CUDA(cudaMemcpyAsync(dS, samp.data(), sizeof(int64_t) * S, cudaMemcpyHostToDevice, s));
  // label filters
  const int32_t* dCons = nullptr;
  if (p->mlp_sample_cons) {
    if (int rc = stage_in(p->mlp_sample_cons, (size_t)S * L, scr, s, &dCons)) return rc;
  } else {
    int32_t* cons_buf = nullptr;
    if (int rc = draw_cons(dA, L, dS, S, p->seed + 3, scr, s, &cons_buf)) return rc;
    dCons = cons_buf;
  }
  // exact filtered neighbours of the training points (m = B, fp32 scan)
  float* Xs = nullptr;
  if (int rc = scr.get(&Xs, (size_t)S * d)) return rc;
  if (int rc = mlp_gather_rows(dX, dS, S, d, Xs, s)) return rc;
  const int kq = lk + 1;
  int64_t* nid = nullptr;
  float* ndist = nullptr;
  if (int rc = scr.get(&nid, (size_t)S * kq)) return rc;
  if (int rc = scr.get(&ndist, (size_t)S * kq)) return rc;
  caps_attrs ca;
  ca.L = L;
  ca.dense = dCons;
  ca.vocab = nullptr;
  ca.sp_offsets = nullptr;
  ca.sp_labels = nullptr;
  ca.sp_vocab = 0;
  const int keep_prec = ix->prec;
  ix->prec = CAPS_FP32;
  const int rc_s = caps_search_batch(ix, Xs, S, &ca, kq, B, nid, ndist, s);
  ix->prec = keep_prec;
  if (rc_s) return rc_s;
  if (int rc = ix->alloc(&ix->labels, (size_t)S * B)) return rc;
  ix->n_labels = S;
  CAPS_CUDA(cudaMemsetAsync(ix->labels, 0, sizeof(float) * S * B, s));
  k_mlp_labels<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(nid, kq, dS, S, lk, ix->bin, B,
                                                           ix->labels);
  CAPS_LAUNCH("k_mlp_labels");
  // network
  ix->mlp.d = d;
  ix->mlp.H = H;
  ix->mlp.B = B;
  float* wbase = nullptr;
  if (int rc = ix->alloc(&wbase, (size_t)ix->mlp.size())) return rc;
  ix->mlp.bind(wbase);
  if (p->mlp_init) {
    const float* dW = nullptr;
    if (int rc = stage_in(p->mlp_init, (size_t)ix->mlp.size(), scr, s, &dW)) return rc;
    CAPS_CUDA(cudaMemcpyAsync(wbase, dW, sizeof(float) * ix->mlp.size(), cudaMemcpyDeviceToDevice, s));
  } else {
    std::vector<float> w((size_t)ix->mlp.size(), 0.f);
    uint64_t st = p->seed + 2;
    const double a1 = 1.0 / std::sqrt((double)d), a2 = 1.0 / std::sqrt((double)H);
    for (int64_t i = 0; i < (int64_t)H * d; i++) w[i] = (float)((2.0 * u01(&st) - 1.0) * a1);
    float* w2 = w.data() + (int64_t)H * d + H;
    for (int64_t i = 0; i < (int64_t)B * H; i++) w2[i] = (float)((2.0 * u01(&st) - 1.0) * a2);
    CAPS_CUDA(cudaMemcpyAsync(wbase, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, s));
    CAPS_CUDA(cudaStreamSynchronize(s));
  }
  // the partitions the first labels were made from: the k-means ones
  if (int rc = ix->alloc(&ix->label_bins, (size_t)N)) return rc;
  ix->n_label_bins = N;
  CAPS_CUDA(cudaMemcpyAsync(ix->label_bins, ix->bin, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
  // rounds (BLISS's iterative scheme): train, assign every point (argmax, or
  // the balanced assignment over its R largest logits), and before the next
  // round relabel the training points from their neighbours' new partitions
  const int rounds = std::max(1, p->mlp_rounds);
  ix->balance_r = p->mlp_balance_r;
  for (int r = 0; r < rounds; r++) {
    if (p->mlp_epochs > 0)
      if (int rc = mlp_train(ix->mlp, Xs, S, ix->labels, p->mlp_epochs, batch, lr, nullptr, s,
                             p->mlp_bf16 != 0))
        return rc;
    if (ix->balance_r > 0) {
      if (int rc = mlp_balanced_assign(ix->mlp, dX, N, ix->balance_r, nullptr, ix->bin, scr, s))
        return rc;
    } else if (int rc = mlp_assign(ix->mlp, dX, N, ix->bin, scr, s)) {
      return rc;
    }
    if (r + 1 < rounds) {
      CAPS_CUDA(cudaMemcpyAsync(ix->label_bins, ix->bin, sizeof(int32_t) * N,
                                cudaMemcpyDeviceToDevice, s));
      CAPS_CUDA(cudaMemsetAsync(ix->labels, 0, sizeof(float) * S * B, s));
      k_mlp_labels<<<(unsigned)((S + 127) / 128), 128, 0, s>>>(nid, kq, dS, S, lk, ix->bin, B,
                                                               ix->labels);
      CAPS_LAUNCH("k_mlp_labels");
    }
  }
  ix->part = CAPS_PART_MLP;
  CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

// The arrays of the bf16 / e4m3 forms for the index's current rows (Xp, Ap,
// perm, offsets in layout order): bf16 rows (with the penalty chunk when
// ix->pen) or e4m3 rows and per-row scales, fp32 squared norms, the inverse
// permutation and the tensor map over the rows.  Nothing for CAPS_FP32.
static int prepare_precision(caps_index* ix, cudaStream_t s) {
  if (ix->prec == CAPS_FP32) return CAPS_OK;
  // the split form rides on the penalty form; without it the index searches
  // with the fp32 scan alone
  const bool split = ix->prec == CAPS_FP32_SPLIT;
  if (split && !ix->pen) return CAPS_OK;
  const int64_t N = ix->N;
  const int d = ix->d;
  const bool f8 = ix->prec == CAPS_FP8E4M3;
  if (f8) {
    // e4m3 rows (ceil(d/128)*128 bytes) + per-row scales + fp32 squared
    // norms + inverse permutation; the filter is tested per pair
    const int cols8 = (d + 127) / 128 * 128;
    uint8_t* xb = nullptr;
    if (int rc = ix->alloc(&xb, (size_t)N * cols8)) return rc;
    ix->Xb = xb;
    if (int rc = ix->alloc(&ix->xs, (size_t)N + 4)) return rc;
  } else {
    const int cols = ix->pen ? ((d + 63) / 64 * (split ? 2 : 1) + 1) * 64 : d;
    uint16_t* xb = nullptr;
    if (int rc = ix->alloc(&xb, (size_t)N * cols)) return rc;
    ix->Xb = xb;
  }
  if (int rc = ix->alloc(&ix->xn, (size_t)N + 4)) return rc;
  if (int rc = ix->alloc(&ix->iperm, (size_t)N)) return rc;
  TcIndexPrep tp;
  tp.Xp = ix->Xp;
  tp.N = N;
  tp.d = d;
  tp.perm = ix->perm;
  tp.Ap = ix->Ap;
  tp.words_pad = ix->meta.words_pad;
  tp.offsets = ix->offsets;
  tp.B = ix->B;
  tp.nb = ix->h + 1;
  tp.pen = ix->pen;
  tp.pen_bits = ix->pen_bits;
  for (int w = 0; w < 4; w++) tp.pen_mask[w] = ix->pen_mask[w];
  tp.f8 = f8 ? 1 : 0;
  tp.split = split ? 1 : 0;
  tp.metric = ix->metric;
  tp.xs = ix->xs;
  tp.Xb = ix->Xb;
  tp.xn = ix->xn;
  tp.iperm = ix->iperm;
  tp.xn_max = &ix->xn_max;
  tp.tmap = ix->tmap;
  return tc_prepare_index(tp, s);
}

static int build_impl(const caps_build_params* p, const float* X, int64_t N, int32_t d,
                      const caps_attrs* attrs, cudaStream_t s, caps_index* ix) {
  if (!p || !X || !attrs) return fail(CAPS_EINVAL, "null argument");
  if (N < 1 || N >= (int64_t)INT32_MAX) return fail(CAPS_EINVAL, "N must be in [1, 2^31-1)");
  if (d < 1) return fail(CAPS_EINVAL, "d must be >= 1");
  if (p->B < 1 || p->B > N) return fail(CAPS_EINVAL, "B must be in [1, N]");
  if (p->h < 0 || p->h > kMaxH) return fail(CAPS_EINVAL, "h must be in [0, 63]");
  if ((int64_t)p->B * (p->h + 1) >= (int64_t)INT32_MAX) return fail(CAPS_EINVAL, "B*(h+1) too large");
  if (p->kmeans_iters < 0) return fail(CAPS_EINVAL, "kmeans_iters must be >= 0");
  if (p->metric != CAPS_L2 && p->metric != CAPS_IP) return fail(CAPS_EINVAL, "unknown metric");
  if (p->part != CAPS_PART_KMEANS && p->part != CAPS_PART_MLP)
    return fail(CAPS_EINVAL, "unknown partitioner");
  if (p->part == CAPS_PART_MLP) {
    if (p->mlp_hidden < 0 || p->mlp_epochs < 0 || p->mlp_samples < 0 || p->mlp_batch < 0 ||
        p->mlp_label_k < 0 || p->mlp_label_k > kMaxK - 1 || !(p->mlp_lr >= 0.f))
      return fail(CAPS_EINVAL, "bad MLP parameters");
    if (p->mlp_epochs == 0 && !p->mlp_init)
      return fail(CAPS_EINVAL, "an MLP build needs mlp_epochs > 0 or mlp_init");
    if (p->mlp_rounds < 0 || p->mlp_rounds > 64) return fail(CAPS_EINVAL, "mlp_rounds must be in [0, 64]");
    if (p->mlp_balance_r < 0 || p->mlp_balance_r > 64 || p->mlp_balance_r > p->B ||
        (p->mlp_balance_r > 0 && p->B > 25600))
      return fail(CAPS_EINVAL, "mlp_balance_r must be in [0, min(64, B)] (B <= 25600 to balance)");
    if (p->mlp_arbiter_queries < 0 ||
        (p->mlp_arbiter_queries > 0 && (p->mlp_arbiter_m < 1 || p->mlp_arbiter_m > p->B)))
      return fail(CAPS_EINVAL, "mlp_arbiter_queries >= 0, and mlp_arbiter_m in [1, B] when arbitrating");
  }
  if (p->prec != CAPS_FP32 && p->prec != CAPS_BF16 && p->prec != CAPS_FP8E4M3 &&
      p->prec != CAPS_FP32_SPLIT)
    return fail(CAPS_EINVAL,
                "precision must be CAPS_FP32, CAPS_BF16, CAPS_FP8E4M3 or CAPS_FP32_SPLIT");
  if ((p->prec == CAPS_BF16 || p->prec == CAPS_FP32_SPLIT) && (d % 8 != 0 || d < 64 || d > 128))
    return fail(CAPS_EINVAL, "the bf16 form needs d a multiple of 8 in [64, 128]");
  if (p->prec == CAPS_FP8E4M3 && (d % 16 != 0 || d < 64 || d > 128))
    return fail(CAPS_EINVAL, "the e4m3 form needs d a multiple of 16 in [64, 128]");
  if (p->rerank_factor < 0 || p->rerank_factor > 16)
    return fail(CAPS_EINVAL, "rerank_factor must be in [0, 16] (0 = 4)");
  keep_pool_warm();
  DenseMeta meta;
  if (int rc = make_meta(attrs, s, &meta)) return rc;
  if (meta.sparse && p->part == CAPS_PART_MLP)
    return fail(CAPS_EINVAL, "the learned partitioner serves dense attributes only");
  const int B = p->B, h = p->h, L = meta.L;
  ix->N = N;
  ix->d = d;
  ix->B = B;
  ix->h = h;
  ix->metric = p->metric;
  ix->meta = meta;
  ix->prec = p->prec;
  ix->rerank_factor = p->rerank_factor > 0 ? p->rerank_factor : 4;

  Scratch scr(s);
  const float* dX = nullptr;
  const int32_t* dA = nullptr;
  if (int rc = stage_in(X, (size_t)N * d, scr, s, &dX)) return rc;
  int32_t* bad = nullptr;
  if (int rc = scr.get(&bad, 1)) return rc;
  CAPS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
  int32_t* sp_off32 = nullptr;  // sparse: int32 offsets of the input label lists
  const int32_t* sp_lab_in = nullptr;
  if (meta.sparse) {
    int64_t nnz = 0;
    bool dev = false;
    if (int rc = is_device_ptr(attrs->sp_offsets, &dev)) return rc;
    if (dev) {
      CAPS_CUDA(cudaMemcpyAsync(&nnz, attrs->sp_offsets + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
      CAPS_CUDA(cudaStreamSynchronize(s));
    } else {
      nnz = attrs->sp_offsets[N];
    }
    if (nnz < 0 || nnz >= (int64_t)INT32_MAX) return fail(CAPS_EINVAL, "bad sparse label offsets");
    if (nnz > 0 && !attrs->sp_labels) return fail(CAPS_EINVAL, "null sp_labels");
    const int64_t* doff = nullptr;
    if (int rc = stage_in(attrs->sp_offsets, (size_t)N + 1, scr, s, &doff)) return rc;
    if (nnz > 0) {
      if (int rc = stage_in(attrs->sp_labels, (size_t)nnz, scr, s, &sp_lab_in)) return rc;
    } else {
      int32_t* z = nullptr;
      if (int rc = scr.get(&z, 1)) return rc;
      sp_lab_in = z;
    }
    if (int rc = scr.get(&sp_off32, (size_t)N + 1)) return rc;
    if (int rc = launch_check_sparse(doff, sp_lab_in, N, (int32_t)meta.n_codes, sp_off32, bad, s))
      return rc;
    ix->sp_nnz = nnz;
  } else {
    if (int rc = stage_in(attrs->dense, (size_t)N * L, scr, s, &dA)) return rc;
    if (int rc = launch_check_dense(dA, N, meta, bad, s)) return rc;
  }
  int32_t bad_h = 0;
  CAPS_CUDA(cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CAPS_CUDA(cudaStreamSynchronize(s));
  if (bad_h)
    return fail(CAPS_EINVAL, meta.sparse ? "labels must lie in [0, sp_vocab) and ascend strictly "
                                           "within each point"
                                         : "attribute value outside [0, vocab[f])");

  const int64_t nseg = (int64_t)B * (h + 1);
  if (int rc = ix->alloc(&ix->C, (size_t)B * d)) return rc;
  if (int rc = ix->alloc(&ix->bin, (size_t)N)) return rc;
  if (int rc = ix->alloc(&ix->key, (size_t)N)) return rc;
  if (int rc = ix->alloc(&ix->tags, (size_t)B * h)) return rc;
  // perm and Ap carry 4 spare rows: the scan bulk-copies them from 16-B
  // boundaries, which may reach up to 3 rows past the last one
  if (int rc = ix->alloc(&ix->perm, (size_t)N + 4)) return rc;
  if (int rc = ix->alloc(&ix->offsets, (size_t)nseg + 1)) return rc;
  if (int rc = ix->alloc(&ix->pos, (size_t)B * meta.n_codes)) return rc;
  if (int rc = ix->alloc(&ix->code_field, (size_t)meta.n_codes)) return rc;
  if (int rc = ix->alloc(&ix->Xp, (size_t)N * d)) return rc;
  if (int rc = ix->alloc(&ix->Ap, (size_t)(N + 4) * meta.words_pad)) return rc;
  if (int rc = ix->alloc(&ix->err, 1)) return rc;
  CAPS_CUDA(cudaMemsetAsync(ix->err, 0, sizeof(int32_t), s));
  if (meta.sparse) {
    CAPS_CUDA(cudaMemsetAsync(ix->code_field, 0, (size_t)meta.n_codes, s));
    if (int rc = ix->alloc(&ix->sp_off, (size_t)N + 1)) return rc;
    if (int rc = ix->alloc(&ix->sp_lab, (size_t)std::max<int64_t>(1, ix->sp_nnz))) return rc;
  } else {
    if (int rc = launch_code_field(meta, ix->code_field, s)) return rc;
  }

  int32_t *perm_bin = nullptr, *bin_off = nullptr;
  if (int rc = scr.get(&perm_bin, (size_t)N)) return rc;
  if (int rc = scr.get(&bin_off, (size_t)B + 1)) return rc;

  // ---- first level: fixed centroids or k-means (Sec. 5.2) ----
  if (p->centroids) {
    const float* dC = nullptr;
    if (int rc = stage_in(p->centroids, (size_t)B * d, scr, s, &dC)) return rc;
    CAPS_CUDA(cudaMemcpyAsync(ix->C, dC, sizeof(float) * B * d, cudaMemcpyDeviceToDevice, s));
  } else {
    std::vector<int64_t> init;
    if (p->init_idx) {
      if (int rc = to_host(p->init_idx, (size_t)B, &init, s)) return rc;
      std::unordered_set<int64_t> seen;
      for (int64_t v : init) {
        if (v < 0 || v >= N) return fail(CAPS_EINVAL, "init_idx entry outside [0, N)");
        if (!seen.insert(v).second) return fail(CAPS_EINVAL, "init_idx entries must be distinct");
      }
    } else {
      init = floyd_sample(N, B, p->seed);
    }
    int64_t* dinit = nullptr;
    if (int rc = scr.get(&dinit, (size_t)B)) return rc;
    CAPS_CUDA(cudaMemcpyAsync(dinit, init.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice, s));
    if (int rc = launch_gather_rows(dX, dinit, B, d, ix->C, s)) return rc;
    CAPS_CUDA(cudaStreamSynchronize(s));  // `init` leaves scope
    for (int it = 0; it < p->kmeans_iters; it++) {
      Scratch it_scr(s);  // per-iteration temporaries, released in stream order
      if (int rc = launch_assign(dX, N, d, ix->C, B, p->metric, ix->bin, s)) return rc;
      if (int rc = stable_sort_by_key(ix->bin, N, B, perm_bin, bin_off, it_scr, s)) return rc;
      if (int rc = launch_centroid_update(dX, d, perm_bin, bin_off, B, p->metric, ix->C, it_scr, s))
        return rc;
    }
  }
  // ---- f(x_i) for every point (Alg. 1, first loop) ----
  if (int rc = launch_assign(dX, N, d, ix->C, B, p->metric, ix->bin, s)) return rc;
  int32_t* seg = nullptr;
  if (int rc = scr.get(&seg, (size_t)N)) return rc;
  // partitions -> attribute frequency tree -> contiguous layout
  auto finish = [&]() -> int {
    if (int rc = stable_sort_by_key(ix->bin, N, B, perm_bin, bin_off, scr, s)) return rc;
    // ---- attribute frequency tree per partition (Alg. 1, second loop) ----
    CAPS_CUDA(cudaMemsetAsync(ix->key, 0, (size_t)N, s));
    if (meta.sparse) {
      if (int rc = launch_aft_sparse(perm_bin, bin_off, B, h, sp_off32, sp_lab_in,
                                     (int32_t)meta.n_codes, ix->tags, ix->key, s))
        return rc;
    } else if (int rc = launch_aft(perm_bin, bin_off, B, h, dA, meta, ix->code_field, ix->tags,
                                   ix->key, s)) {
      return rc;
    }
    // ---- contiguous sub-partitions: stable order by (partition, block, id) ----
    if (int rc = launch_segment_keys(ix->bin, ix->key, N, h, seg, s)) return rc;
    if (int rc = stable_sort_by_key(seg, N, nseg, ix->perm, ix->offsets, scr, s)) return rc;
    if (int rc = launch_layout(dX, dA, ix->perm, N, d, meta, ix->Xp, ix->Ap, s)) return rc;
    if (meta.sparse)
      if (int rc = launch_layout_sparse(sp_off32, sp_lab_in, ix->perm, N, ix->Ap, ix->sp_off,
                                        ix->sp_lab, scr, s))
        return rc;
    CAPS_CUDA(cudaMemsetAsync(ix->pos, 0, (size_t)B * meta.n_codes, s));
    if (int rc = launch_pos_table(ix->tags, B, h, meta.n_codes, ix->pos, s)) return rc;
    return CAPS_OK;
  };
  if (int rc = finish()) return rc;
  if (p->part == CAPS_PART_MLP) {
    // k-means as the fallback, exact recall as the arbiter
    Arbiter jg;
    std::vector<int64_t> got;
    int32_t* kbins = nullptr;
    const bool arbiter = p->mlp_arbiter_queries > 0;
    if (arbiter) {
      if (int rc = arbiter_prepare(p, dX, dA, N, d, L, scr, s, &jg)) return rc;
      if (int rc = arbiter_search(ix, jg, B, s, &jg.exact)) return rc;
      if (int rc = arbiter_search(ix, jg, p->mlp_arbiter_m, s, &got)) return rc;
      ix->arbiter_recall[0] = arbiter_recall(jg, got);
      if (int rc = scr.get(&kbins, (size_t)N)) return rc;
      CAPS_CUDA(cudaMemcpyAsync(kbins, ix->bin, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
    }
    if (int rc = build_mlp(p, dX, dA, N, d, meta, s, ix)) return rc;
    if (int rc = finish()) return rc;
    if (arbiter) {
      if (int rc = arbiter_search(ix, jg, p->mlp_arbiter_m, s, &got)) return rc;
      ix->arbiter_recall[1] = arbiter_recall(jg, got);
      if (ix->arbiter_recall[0] > ix->arbiter_recall[1]) {
        CAPS_CUDA(cudaMemcpyAsync(ix->bin, kbins, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, s));
        ix->part = CAPS_PART_KMEANS;
        if (int rc = finish()) return rc;
      }
    }
  }
  if (p->prec == CAPS_BF16 || p->prec == CAPS_FP32_SPLIT) {
    // penalty form when the one-hot code of the packed attribute bits (two
    // columns per bit) and, for L2, the three parts of -|x|^2/2 fit one
    // 64-column chunk
    int T = 0;
    uint32_t um[4] = {};
    for (int f = 0; f < meta.L; f++) {
      um[meta.word[f]] |= ((1u << meta.bits[f]) - 1u) << meta.shift[f];
      T += meta.bits[f];
    }
    // (label sets need the exact subset test per key: never the penalty form)
    ix->pen = !meta.sparse && tc_pen_columns(T, p->metric) <= 64 ? 1 : 0;
    ix->pen_bits = T;
    for (int w = 0; w < 4; w++) ix->pen_mask[w] = um[w];
  } else {
    ix->pen = 0;
    ix->pen_bits = 0;
  }
  if (int rc = prepare_precision(ix, s)) return rc;
  {
    // the weight side of the screened probe, fixed from here on
    const bool mlp = ix->part == CAPS_PART_MLP;
    const int sK = mlp ? ix->mlp.H : d;
    if (probe_screen_supported(sK, B, 1)) {
      uint16_t* wh = nullptr;
      if (int rc = ix->alloc(&wh, probe_weights_elems(sK, B))) return rc;
      ix->pw.Wh = wh;
      if (int rc = ix->alloc(&ix->pw.wn2, (size_t)B)) return rc;
      if (int rc = ix->alloc(&ix->pw.wn, (size_t)B)) return rc;
      if (int rc = probe_weights_prepare(mlp ? ix->mlp.W2 : ix->C, B, sK, ix->pw, s)) return rc;
    }
  }
  CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

extern "C" int caps_build(const caps_build_params* params, const float* X, int64_t N, int32_t d,
                          const caps_attrs* attrs, void* stream, caps_index** out) {
  if (!out) return fail(CAPS_EINVAL, "null output handle");
  *out = nullptr;
  caps_index* ix = new (std::nothrow) caps_index();
  if (!ix) return fail(CAPS_ENOMEM, "host allocation failed");
  const int rc = build_impl(params, X, N, d, attrs, (cudaStream_t)stream, ix);
  if (rc != CAPS_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    cudaGetLastError();
    delete ix;
    return rc;
  }
  *out = ix;
  return CAPS_OK;
}

extern "C" void caps_free(caps_index* index) {
  if (!index) return;
  cudaDeviceSynchronize();
  delete index;
}

extern "C" int caps_get_info(const caps_index* ix, caps_index_info* out) {
  if (!ix || !out) return fail(CAPS_EINVAL, "null argument");
  out->N = ix->N;
  out->d = ix->d;
  out->B = ix->B;
  out->h = ix->h;
  out->L = ix->meta.L;
  out->metric = ix->metric;
  out->n_codes = ix->meta.n_codes;
  out->attr_words = ix->meta.words_pad;
  out->device_bytes = ix->bytes;
  out->part = ix->part;
  out->mlp_hidden = ix->part == CAPS_PART_MLP ? ix->mlp.H : 0;
  out->n_labels = ix->n_labels;
  out->n_label_bins = ix->n_label_bins;
  out->mlp_balance_r = ix->balance_r;
  out->arbiter_recall_kmeans = ix->arbiter_recall[0];
  out->arbiter_recall_mlp = ix->arbiter_recall[1];
  return CAPS_OK;
}

extern "C" int caps_export(const caps_index* ix, int32_t which, void* dst, size_t bytes,
                           void* stream) {
  if (!ix || !dst) return fail(CAPS_EINVAL, "null argument");
  const void* src = nullptr;
  size_t want = 0;
  switch (which) {
    case CAPS_ARR_CENTROIDS: src = ix->C; want = sizeof(float) * ix->B * ix->d; break;
    case CAPS_ARR_BIN: src = ix->bin; want = sizeof(int32_t) * ix->N; break;
    case CAPS_ARR_TAGS: src = ix->tags; want = sizeof(int32_t) * ix->B * ix->h; break;
    case CAPS_ARR_KEY: src = ix->key; want = (size_t)ix->N; break;
    case CAPS_ARR_PERM: src = ix->perm; want = sizeof(int32_t) * ix->N; break;
    case CAPS_ARR_OFFSETS:
      src = ix->offsets;
      want = sizeof(int32_t) * ((size_t)ix->B * (ix->h + 1) + 1);
      break;
    case CAPS_ARR_MLP:
      if (ix->part != CAPS_PART_MLP) return fail(CAPS_EINVAL, "not an MLP index");
      src = ix->mlp.W1;
      want = sizeof(float) * (size_t)ix->mlp.size();
      break;
    case CAPS_ARR_LABELS:
      if (ix->part != CAPS_PART_MLP) return fail(CAPS_EINVAL, "not an MLP index");
      src = ix->labels;
      want = sizeof(float) * (size_t)ix->n_labels * ix->B;
      break;
    case CAPS_ARR_LABEL_BINS:
      if (ix->part != CAPS_PART_MLP) return fail(CAPS_EINVAL, "not an MLP index");
      src = ix->label_bins;
      want = sizeof(int32_t) * (size_t)ix->n_label_bins;
      break;
    default: return fail(CAPS_EINVAL, "unknown array id");
  }
  if (bytes != want) return fail(CAPS_EINVAL, "byte count does not match the array size");
  if (want == 0) return CAPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CAPS_CUDA(cudaMemcpyAsync(dst, src, want, cudaMemcpyDefault, s));
  CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

extern "C" int caps_assign(const float* X, int64_t N, int32_t d, const float* C, int32_t B,
                           int32_t metric, int32_t* out_bin, void* stream) {
  if (N < 0 || d < 1 || B < 1) return fail(CAPS_EINVAL, "bad sizes");
  if (metric != CAPS_L2 && metric != CAPS_IP) return fail(CAPS_EINVAL, "unknown metric");
  if (N == 0) return CAPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  keep_pool_warm();
  Scratch scr(s);
  const float *dX = nullptr, *dC = nullptr;
  if (int rc = stage_in(X, (size_t)N * d, scr, s, &dX)) return rc;
  if (int rc = stage_in(C, (size_t)B * d, scr, s, &dC)) return rc;
  Out<int32_t> ob;
  if (int rc = ob.init(out_bin, (size_t)N, scr)) return rc;
  if (int rc = launch_assign(dX, N, d, dC, B, metric, ob.dev, s)) return rc;
  if (int rc = ob.finish(s)) return rc;
  if (ob.host) CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

namespace {
int check_cons(const caps_index* ix, const caps_attrs* cons) {
  if (!cons) return fail(CAPS_EINVAL, "constraints are required");
  if (ix->meta.sparse) {
    if (cons->sp_offsets == nullptr)
      return fail(CAPS_EINVAL, "a label-set index needs sparse constraints (sp_offsets, sp_labels)");
    return CAPS_OK;
  }
  if (cons->dense == nullptr || cons->L != ix->meta.L)
    return fail(CAPS_EINVAL, "constraints must be dense with the index's L fields");
  return CAPS_OK;
}

// Device int32 copy of sparse query constraints (offsets [nq+1], labels).
struct SparseQueries {
  int32_t* off = nullptr;
  const int32_t* lab = nullptr;
};
int stage_sparse_queries(const caps_attrs* cons, int64_t nq, Scratch& scr, cudaStream_t s,
                         SparseQueries* out) {
  bool dev = false;
  if (int rc = is_device_ptr(cons->sp_offsets, &dev)) return rc;
  int64_t nnz = 0;
  if (dev) {
    CAPS_CUDA(cudaMemcpyAsync(&nnz, cons->sp_offsets + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CAPS_CUDA(cudaStreamSynchronize(s));
  } else {
    nnz = cons->sp_offsets[nq];
  }
  if (nnz < 0 || nnz > INT32_MAX) return fail(CAPS_EINVAL, "bad sparse constraint offsets");
  if (nnz > 0 && !cons->sp_labels) return fail(CAPS_EINVAL, "null sp_labels");
  const int64_t* doff = nullptr;
  if (int rc = stage_in(cons->sp_offsets, (size_t)nq + 1, scr, s, &doff)) return rc;
  const int32_t* dlab = nullptr;
  if (nnz > 0) {
    if (int rc = stage_in(cons->sp_labels, (size_t)nnz, scr, s, &dlab)) return rc;
  } else {
    int32_t* z = nullptr;
    if (int rc = scr.get(&z, 1)) return rc;
    dlab = z;
  }
  int32_t *o32 = nullptr, *bad = nullptr;
  if (int rc = scr.get(&o32, (size_t)nq + 1)) return rc;
  if (int rc = scr.get(&bad, 1)) return rc;
  CAPS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
  k_offsets_i32<<<(unsigned)((nq + 1 + 255) / 256), 256, 0, s>>>(doff, nq + 1, o32, bad);
  CAPS_LAUNCH("k_offsets_i32");
  int32_t bad_h = 0;
  CAPS_CUDA(cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CAPS_CUDA(cudaStreamSynchronize(s));
  if (bad_h) return fail(CAPS_EINVAL, "sparse constraint offsets must be non-decreasing");
  out->off = o32;
  out->lab = dlab;
  return CAPS_OK;
}

// Device buffers for one chunk of queries.
struct Batch {
  float* scores;
  int32_t* probe;
  uint64_t* sel;
  QueryPrep qp;
};

int alloc_batch(const caps_index* ix, int64_t nq, int m, Scratch& scr, Batch* b) {
  const int WP = ix->meta.words_pad, L = ix->meta.L;
  if (int rc = scr.get(&b->scores, (size_t)nq * ix->B)) return rc;
  if (int rc = scr.get(&b->probe, (size_t)nq * m)) return rc;
  if (int rc = scr.get(&b->sel, (size_t)nq * m)) return rc;
  if (int rc = scr.get(&b->qp.qmask, (size_t)nq * WP)) return rc;
  if (int rc = scr.get(&b->qp.qval, (size_t)nq * WP)) return rc;
  if (int rc = scr.get(&b->qp.qcode, (size_t)nq * L)) return rc;
  if (int rc = scr.get(&b->qp.dead, (size_t)nq)) return rc;
  return CAPS_OK;
}

int64_t chunk_rows(const caps_index* ix, int64_t nq, int m = 1, int k = 1) {
  // per-query scratch: centroid scores + partial top-k lists + probe data
  const int64_t per_q = 4 * (int64_t)ix->B + 8 * (int64_t)m * k + 16 * (int64_t)m + 64;
  const int64_t budget = (int64_t)1 << 29;  // 512 MiB per chunk
  int64_t c = budget / per_q;
  if (c < 1) c = 1;
  return std::min(c, nq);
}
}  // namespace

// Alg. 2 "select top m partitions": scores of every partition for each
// query -- centroid distances (k-means) or MLP logits (learned) -- and the
// order in which they rank (smaller L2 distance / larger IP or logit).
static int partition_scores(const caps_index* ix, const float* Q, int64_t n, float* scores,
                            float* hid, cudaStream_t s) {
  if (ix->part == CAPS_PART_MLP) return mlp_logits(ix->mlp, Q, n, hid, scores, s);
  return launch_scores(Q, n, ix->d, ix->C, ix->B, ix->metric, scores, s);
}
static int probe_metric(const caps_index* ix) {
  return ix->part == CAPS_PART_MLP ? CAPS_IP : ix->metric;
}

extern "C" int caps_probe(const caps_index* ix, const float* Q, int64_t nq, int32_t m,
                          int32_t* out_probe, void* stream) {
  if (!ix) return fail(CAPS_EINVAL, "null index");
  if (nq < 0 || m < 1 || m > ix->B) return fail(CAPS_EINVAL, "m must be in [1, B]");
  if (nq == 0) return CAPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  const float* dQ = nullptr;
  if (int rc = stage_in(Q, (size_t)nq * ix->d, scr, s, &dQ)) return rc;
  Out<int32_t> op;
  if (int rc = op.init(out_probe, (size_t)nq * m, scr)) return rc;
  const int64_t qc = chunk_rows(ix, nq);
  float* scores = nullptr;
  if (int rc = scr.get(&scores, (size_t)qc * ix->B)) return rc;
  float* hid = nullptr;
  if (ix->part == CAPS_PART_MLP)
    if (int rc = scr.get(&hid, (size_t)qc * ix->mlp.H)) return rc;
  for (int64_t c0 = 0; c0 < nq; c0 += qc) {
    const int64_t n = std::min(qc, nq - c0);
    if (int rc = partition_scores(ix, dQ + c0 * ix->d, n, scores, hid, s)) return rc;
    if (int rc = launch_topm(scores, n, ix->B, m, probe_metric(ix), op.dev + c0 * m, s)) return rc;
  }
  if (int rc = op.finish(s)) return rc;
  if (op.host) CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

extern "C" int caps_probe_set(const caps_index* ix, const float* Q, int64_t nq, int32_t m,
                              int32_t* out_probe, void* stream) {
  if (!ix) return fail(CAPS_EINVAL, "null index");
  if (nq < 0 || m < 1 || m > ix->B) return fail(CAPS_EINVAL, "m must be in [1, B]");
  const bool mlp = ix->part == CAPS_PART_MLP;
  const int sK = mlp ? ix->mlp.H : ix->d;
  if (!probe_screen_supported(sK, ix->B, m)) return caps_probe(ix, Q, nq, m, out_probe, stream);
  if (nq == 0) return CAPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  const float* dQ = nullptr;
  if (int rc = stage_in(Q, (size_t)nq * ix->d, scr, s, &dQ)) return rc;
  Out<int32_t> op;
  if (int rc = op.init(out_probe, (size_t)nq * m, scr)) return rc;
  const int64_t qc = chunk_rows(ix, nq);
  float* scores = nullptr;
  if (int rc = scr.get(&scores, (size_t)qc * ix->B)) return rc;
  float* hid = nullptr;
  if (mlp)
    if (int rc = scr.get(&hid, (size_t)qc * ix->mlp.H)) return rc;
  for (int64_t c0 = 0; c0 < nq; c0 += qc) {
    const int64_t n = std::min(qc, nq - c0);
    const float* Qc = dQ + c0 * ix->d;
    Scratch cscr(s);
    if (mlp)
      if (int rc = ::caps::mlp_hidden(ix->mlp, Qc, n, hid, s)) return rc;
    if (int rc = probe_screened(mlp ? 0 : (ix->metric == CAPS_L2 ? 1 : 2), mlp ? hid : Qc, n, sK,
                                mlp ? ix->mlp.W2 : ix->C, mlp ? ix->mlp.b2 : nullptr, ix->B, m,
                                scores, op.dev + c0 * m, ix->err, cscr, s, &ix->pw))
      return rc;
  }
  if (int rc = op.finish(s)) return rc;
  if (op.host) CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

extern "C" int caps_select(const caps_index* ix, const int32_t* probe, int64_t nq, int32_t m,
                           const caps_attrs* cons, uint64_t* out_sel, void* stream) {
  if (!ix) return fail(CAPS_EINVAL, "null index");
  if (nq < 0 || m < 1 || m > ix->B) return fail(CAPS_EINVAL, "m must be in [1, B]");
  if (int rc = check_cons(ix, cons)) return rc;
  if (nq == 0) return CAPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  std::vector<int32_t> ph;
  if (int rc = to_host(probe, (size_t)nq * m, &ph, s)) return rc;
  for (int32_t b : ph)
    if (b < 0 || b >= ix->B) return fail(CAPS_EINVAL, "probe entry outside [0, B)");
  const int32_t *dP = nullptr, *dQb = nullptr;
  if (int rc = stage_in(probe, (size_t)nq * m, scr, s, &dP)) return rc;
  Out<uint64_t> os;
  if (int rc = os.init(out_sel, (size_t)nq * m, scr)) return rc;
  if (ix->meta.sparse) {
    SparseQueries sq;
    if (int rc = stage_sparse_queries(cons, nq, scr, s, &sq)) return rc;
    if (int rc = launch_select_sparse(dP, nq, m, ix->h, ix->tags, ix->pos, ix->meta.n_codes,
                                      sq.off, sq.lab, os.dev, s))
      return rc;
    if (int rc = os.finish(s)) return rc;
    if (os.host) CAPS_CUDA(cudaStreamSynchronize(s));
    return CAPS_OK;
  }
  if (int rc = stage_in(cons->dense, (size_t)nq * ix->meta.L, scr, s, &dQb)) return rc;
  QueryPrep qp;
  const int WP = ix->meta.words_pad, L = ix->meta.L;
  if (int rc = scr.get(&qp.qmask, (size_t)nq * WP)) return rc;
  if (int rc = scr.get(&qp.qval, (size_t)nq * WP)) return rc;
  if (int rc = scr.get(&qp.qcode, (size_t)nq * L)) return rc;
  if (int rc = scr.get(&qp.dead, (size_t)nq)) return rc;
  if (int rc = launch_query_prep(dQb, nq, ix->meta, qp, s)) return rc;
  if (int rc = launch_select(dP, nq, m, ix->h, ix->tags, ix->pos, ix->meta.n_codes,
                             ix->code_field, dQb, ix->meta, qp.qcode, os.dev, s))
    return rc;
  if (int rc = os.finish(s)) return rc;
  if (os.host) CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

namespace {
// Stage timing of caps_search_batch: one event before each stage of each
// chunk, plus one at the end.
struct StageTimer {
  bool on = false;
  static constexpr int kStages = 7;
  std::vector<cudaEvent_t> ev;  // kStages per chunk + 1
  int used = 0;
  int launches = 0;
  bool valid = false;
  int record(cudaStream_t s) {
    if (!on) return CAPS_OK;
    if (used == (int)ev.size()) {
      cudaEvent_t e;
      CAPS_CUDA(cudaEventCreate(&e));
      ev.push_back(e);
    }
    CAPS_CUDA(cudaEventRecord(ev[used++], s));
    return CAPS_OK;
  }
  ~StageTimer() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};
thread_local StageTimer g_timer;
}  // namespace

extern "C" int caps_set_timing(int32_t enable) {
  g_timer.on = enable != 0;
  g_timer.valid = false;
  return CAPS_OK;
}

extern "C" int caps_get_stage_times(caps_stage_times* out) {
  if (!out) return fail(CAPS_EINVAL, "null argument");
  const int S = StageTimer::kStages;
  if (!g_timer.valid || g_timer.used < S + 1) return fail(CAPS_EINVAL, "no timed search on this thread");
  CAPS_CUDA(cudaEventSynchronize(g_timer.ev[g_timer.used - 1]));
  float acc[StageTimer::kStages] = {};
  const int chunks = (g_timer.used - 1) / S;
  for (int c = 0; c < chunks; c++)
    for (int st = 0; st < S; st++) {
      float ms = 0.f;
      const int a = c * S + st;
      CAPS_CUDA(cudaEventElapsedTime(&ms, g_timer.ev[a], g_timer.ev[a + 1]));
      acc[st] += ms;
    }
  out->prep_ms = acc[0];
  out->scores_ms = acc[1];
  out->topm_ms = acc[2];
  out->select_ms = acc[3];
  out->group_ms = acc[4];
  out->scan_ms = acc[5];
  out->merge_ms = acc[6];
  out->launches = g_timer.launches;
  return CAPS_OK;
}

extern "C" int caps_device_status(const caps_index* ix, void* stream) {
  if (!ix) return fail(CAPS_EINVAL, "null index");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t e = 0;
  CAPS_CUDA(cudaMemcpyAsync(&e, ix->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CAPS_CUDA(cudaStreamSynchronize(s));
  if (e) {
    CAPS_CUDA(cudaMemsetAsync(ix->err, 0, sizeof(int32_t), s));
    CAPS_CUDA(cudaStreamSynchronize(s));
    return fail(CAPS_ETIMEOUT, "a bounded device wait expired in an earlier search");
  }
  return CAPS_OK;
}

namespace {
// Launch-shape choices of one batched search (the autotuner's search space).
struct SearchOpts {
  int tile_n = 256;    // rows per tensor-core tile (128 or 256)
  int item_cap = 0;    // most probes per tensor-core work item (0: 128)
  int pen = -1;        // filter folded into the MMA: 1 yes, 0 no, -1 when the index has it
  bool timed = true;   // stage events allowed (not while a graph is captured)
  bool cached = false; // use the shape the autotuner chose for this (k, m), if any
};

int search_impl(const caps_index* ix, const float* Q, int64_t nq, const caps_attrs* cons,
                int32_t k, int32_t m, int64_t* out_ids, float* out_dist, cudaStream_t s,
                const SearchOpts& o);

// which forms of the tensor-core scan serve this index and k
int kp_of(const caps_index* ix, int k) {
  return tc_kp(k, tc_rerank_depth(k, ix->rerank_factor));
}
bool tc_explicit_ok(const caps_index* ix, int k) {
  const bool f8 = ix->prec == CAPS_FP8E4M3;
  return (ix->prec == CAPS_BF16 || f8) &&
         tc_scan_supported(ix->d, k, kp_of(ix, k), ix->meta.words_pad, f8 ? 1 : 0);
}
bool uses_pen(const caps_index* ix, int k) {
  if (ix->prec == CAPS_FP32_SPLIT)
    return k <= 32 && ix->pen && tc_split_supported(ix->d, kp_of(ix, k), ix->meta.words_pad);
  return ix->prec == CAPS_BF16 && k <= 32 && ix->pen &&
         tc_pen_supported(ix->d, kp_of(ix, k), ix->meta.words_pad);
}
bool uses_tc(const caps_index* ix, int k) { return tc_explicit_ok(ix, k) || uses_pen(ix, k); }
}  // namespace

extern "C" int caps_search_batch(const caps_index* ix, const float* Q, int64_t nq,
                                 const caps_attrs* cons, int32_t k, int32_t m, int64_t* out_ids,
                                 float* out_dist, void* stream) {
  SearchOpts o;
  o.cached = true;
  return search_impl(ix, Q, nq, cons, k, m, out_ids, out_dist, (cudaStream_t)stream, o);
}

namespace {
int search_impl(const caps_index* ix, const float* Q, int64_t nq, const caps_attrs* cons,
                int32_t k, int32_t m, int64_t* out_ids, float* out_dist, cudaStream_t s,
                const SearchOpts& o) {
  if (!ix) return fail(CAPS_EINVAL, "null index");
  if (nq < 0) return fail(CAPS_EINVAL, "nq < 0");
  if (k < 1 || k > kMaxK) return fail(CAPS_EINVAL, "k must be in [1, 128]");
  if (m < 1 || m > ix->B) return fail(CAPS_EINVAL, "m must be in [1, B]");
  if (int rc = check_cons(ix, cons)) return rc;
  if (nq == 0) return CAPS_OK;
  keep_pool_warm();
  Scratch scr(s);
  const float* dQ = nullptr;
  const int32_t* dQb = nullptr;
  SparseQueries sq;
  if (int rc = stage_in(Q, (size_t)nq * ix->d, scr, s, &dQ)) return rc;
  if (ix->meta.sparse) {
    if (int rc = stage_sparse_queries(cons, nq, scr, s, &sq)) return rc;
  } else if (int rc = stage_in(cons->dense, (size_t)nq * ix->meta.L, scr, s, &dQb)) {
    return rc;
  }
  Out<int64_t> oi;
  Out<float> od;
  if (int rc = oi.init(out_ids, (size_t)nq * k, scr)) return rc;
  if (int rc = od.init(out_dist, (size_t)nq * k, scr)) return rc;
  const bool tc = uses_tc(ix, k);
  const int kp = tc ? kp_of(ix, k) : k;
  int tile_n = o.tile_n, item_cap = o.item_cap, pen = o.pen;
  if (o.cached) {
    std::lock_guard<std::mutex> lock(ix->tune_mu);
    auto f = ix->tuned.find({k, m});
    if (f != ix->tuned.end()) {
      tile_n = f->second.tile_n;
      item_cap = f->second.item_cap;
      pen = f->second.pen;
    }
  }
  const bool pen_ok = tc && uses_pen(ix, k);
  const bool use_pen = pen_ok && (pen != 0 || !tc_explicit_ok(ix, k));
  const int64_t qc = chunk_rows(ix, nq, m, kp);
  Batch bt;
  if (int rc = alloc_batch(ix, qc, m, scr, &bt)) return rc;
  const bool binmajor = !tc && bin_scan_supported(ix->d);
  float* mlp_hidden = nullptr;
  if (ix->part == CAPS_PART_MLP)
    if (int rc = scr.get(&mlp_hidden, (size_t)qc * ix->mlp.H)) return rc;
  uint64_t* part = nullptr;
  if (binmajor || tc)
    if (int rc = scr.get(&part, (size_t)qc * m * kp)) return rc;
  uint16_t* Qh = nullptr;  // bf16 queries, or e4m3 bytes in the first half
  float* qn = nullptr;
  float* qs = nullptr;
  const int f8 = ix->prec == CAPS_FP8E4M3 ? 1 : 0;
  const int split = ix->prec == CAPS_FP32_SPLIT ? 1 : 0;
  if (tc) {
    if (int rc = scr.get(&Qh, (size_t)qc * tc_vec_cols(ix->d, split))) return rc;
    if (int rc = scr.get(&qn, (size_t)qc)) return rc;
    if (f8)
      if (int rc = scr.get(&qs, (size_t)qc)) return rc;
  }
  const int L = ix->meta.L;
  StageTimer& tm = g_timer;
  const bool timer_on = tm.on;
  if (!o.timed) tm.on = false;  // no event records inside a graph capture
  struct Restore {
    StageTimer& t;
    bool on;
    ~Restore() { t.on = on; }
  } restore{tm, timer_on};
  tm.used = 0;
  tm.launches = 0;
  tm.valid = false;
  const long long launches0 = g_kernel_launches;
  for (int64_t c0 = 0; c0 < nq; c0 += qc) {
    const int64_t n = std::min(qc, nq - c0);
    const float* Qc = dQ + c0 * ix->d;
    const int32_t* Qbc = dQb ? dQb + c0 * L : nullptr;
    SparseRef sp;  // label sets: rows (layout order) and this chunk's queries
    if (ix->meta.sparse) {
      sp.roff = ix->sp_off;
      sp.rlab = ix->sp_lab;
      sp.qoff = sq.off + c0;
      sp.qlab = sq.lab;
    }
    Scratch cscr(s);  // per-chunk grouping temporaries
    if (int rc = tm.record(s)) return rc;
    if (ix->meta.sparse) {
      if (int rc = launch_query_prep_sparse(sp.qoff, sp.qlab, n, ix->meta, bt.qp, s)) return rc;
    } else if (int rc = launch_query_prep(Qbc, n, ix->meta, bt.qp, s)) {
      return rc;
    }
    if (int rc = tm.record(s)) return rc;
    const bool mlp = ix->part == CAPS_PART_MLP;
    const int sK = mlp ? ix->mlp.H : ix->d;
    if (probe_screen_supported(sK, ix->B, m)) {
      // exact probe set, screened on the tensor cores (the top-m stage is
      // part of it, so its stage time reads ~0)
      if (mlp)
        if (int rc = ::caps::mlp_hidden(ix->mlp, Qc, n, mlp_hidden, s)) return rc;
      if (int rc = probe_screened(mlp ? 0 : (ix->metric == CAPS_L2 ? 1 : 2), mlp ? mlp_hidden : Qc,
                                  n, sK, mlp ? ix->mlp.W2 : ix->C, mlp ? ix->mlp.b2 : nullptr,
                                  ix->B, m, bt.scores, bt.probe, ix->err, cscr, s, &ix->pw))
        return rc;
      if (int rc = tm.record(s)) return rc;
    } else {
      if (int rc = partition_scores(ix, Qc, n, bt.scores, mlp_hidden, s)) return rc;
      if (int rc = tm.record(s)) return rc;
      if (int rc = launch_topm(bt.scores, n, ix->B, m, probe_metric(ix), bt.probe, s)) return rc;
    }
    if (int rc = tm.record(s)) return rc;
    if (ix->meta.sparse) {
      if (int rc = launch_select_sparse(bt.probe, n, m, ix->h, ix->tags, ix->pos,
                                        ix->meta.n_codes, sp.qoff, sp.qlab, bt.sel, s))
        return rc;
    } else if (int rc = launch_select(bt.probe, n, m, ix->h, ix->tags, ix->pos, ix->meta.n_codes,
                                      ix->code_field, Qbc, ix->meta, bt.qp.qcode, bt.sel, s)) {
      return rc;
    }
    if (int rc = tm.record(s)) return rc;
    ScanArgs a;
    a.sp = sp;
    a.Xp = ix->Xp;
    a.Ap = ix->Ap;
    a.perm = ix->perm;
    a.offsets = ix->offsets;
    a.Q = Qc;
    a.qp = bt.qp;
    a.probe = bt.probe;
    a.sel = bt.sel;
    a.nq = n;
    a.m = m;
    a.h = ix->h;
    a.d = ix->d;
    a.k = k;
    a.metric = ix->metric;
    a.words_pad = ix->meta.words_pad;
    a.out_ids = oi.dev + c0 * k;
    a.out_dist = od.dev + c0 * k;
    if (tc) {
      BinWork w;
      if (int rc = tc_query_prep(Qc, n, ix->d, Qh, qn, f8, qs, s, split)) return rc;
      const int rerank = tc_rerank_depth(k, ix->rerank_factor);
      if (int rc = tc_group(bt.probe, bt.sel, ix->h, n * m, ix->B, item_cap, &w, cscr, s))
        return rc;
      if (int rc = tm.record(s)) return rc;
      TcScanArgs t;
      t.sel = bt.sel;
      t.qmask = bt.qp.qmask;
      t.qval = bt.qp.qval;
      t.Qh = Qh;
      t.f8 = f8;
      t.qs = qs;
      t.xs = ix->xs;
      t.qn = qn;
      t.Ap = ix->Ap;
      t.perm = ix->perm;
      t.xn = ix->xn;
      t.offsets = ix->offsets;
      t.tmap = ix->tmap;
      t.m = m;
      t.h = ix->h;
      t.d = ix->d;
      t.kp = kp;
      t.rerank = rerank;
      t.tile_n = tile_n;
      t.pen = use_pen ? 1 : 0;
      t.pen_bits = ix->pen_bits;
      for (int i = 0; i < 4; i++) t.pen_mask[i] = ix->pen_mask[i];
      t.xn_max = ix->xn_max;
      uint64_t* qslot = nullptr;
      if (int rc = cscr.get(&qslot, (size_t)n * 8)) return rc;
      CAPS_CUDA(cudaMemsetAsync(qslot, 0xFF, sizeof(uint64_t) * (size_t)n * 8, s));
      t.qslot = qslot;
      t.sp = sp;
      t.words_pad = ix->meta.words_pad;
      t.metric = ix->metric;
      t.part = part;
      t.err = ix->err;
      t.n_rows = ix->N;
      t.split = split;
      if (int rc = tc_scan(t, w, s)) return rc;
      if (int rc = tm.record(s)) return rc;
      if (int rc = tc_merge_rerank(t, bt.qp.dead, n, k, Qc, ix->Xp, ix->iperm, a.out_ids,
                                   a.out_dist, s))
        return rc;
    } else if (binmajor) {
      BinWork w;
      if (int rc = bin_group(bt.probe, n * m, ix->B, &w, cscr, s)) return rc;
      if (int rc = tm.record(s)) return rc;
      if (int rc = bin_scan(a, w, part, ix->err, s)) return rc;
      if (int rc = tm.record(s)) return rc;
      if (int rc = bin_merge(a, part, s)) return rc;
    } else {
      if (int rc = tm.record(s)) return rc;
      if (int rc = launch_scan_topk(a, s)) return rc;
      if (int rc = tm.record(s)) return rc;
    }
  }
  if (int rc = tm.record(s)) return rc;
  tm.launches = (int)(g_kernel_launches - launches0);
  tm.valid = tm.on;
  if (int rc = oi.finish(s)) return rc;
  if (int rc = od.finish(s)) return rc;
  if (oi.host || od.host) {
    CAPS_CUDA(cudaStreamSynchronize(s));
    return caps_device_status(ix, s);
  }
  return CAPS_OK;
}
}  // namespace

// ---- tuned, graph-captured query plans -------------------------------------

struct caps_plan {
  const caps_index* ix = nullptr;
  int64_t generation = 0;  // the index's generation when the graph was captured
  int64_t nq = 0;
  int32_t k = 0, m = 0;
  float* Q = nullptr;        // [nq*d]
  int32_t* cons = nullptr;   // [nq*L]
  int64_t* ids = nullptr;    // [nq*k]
  float* dist = nullptr;     // [nq*k]
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  caps_plan_info info{};
  ~caps_plan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFree(Q);
    cudaFree(cons);
    cudaFree(ids);
    cudaFree(dist);
    cudaGetLastError();
  }
};

namespace {
template <class T>
int plan_alloc(T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = dev_alloc(&q, std::max<size_t>(1, count) * sizeof(T), nullptr, false);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(CAPS_ENOMEM, "device allocation failed for a plan buffer");
  }
  *p = static_cast<T*>(q);
  return CAPS_OK;
}

// Median device time (ms) of `reps` searches with launch shape o, after one
// untimed run.
int time_shape(caps_plan* p, const caps_attrs& pc, const SearchOpts& o, cudaStream_t s, int reps,
               float* ms_out) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CAPS_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "cudaEventCreate");
  }
  std::vector<float> t;
  int rc = search_impl(p->ix, p->Q, p->nq, &pc, p->k, p->m, p->ids, p->dist, s, o);
  for (int r = 0; rc == CAPS_OK && r < reps; r++) {
    if (cudaEventRecord(e0, s) != cudaSuccess) rc = fail(CAPS_ECUDA, "cudaEventRecord");
    if (rc == CAPS_OK) rc = search_impl(p->ix, p->Q, p->nq, &pc, p->k, p->m, p->ids, p->dist, s, o);
    if (rc == CAPS_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = fail(CAPS_ECUDA, "cudaEventRecord");
    float ms = 0.f;
    if (rc == CAPS_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(CAPS_ECUDA, "cudaEventSynchronize");
    if (rc == CAPS_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      rc = fail(CAPS_ECUDA, "cudaEventElapsedTime");
    t.push_back(ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  if (rc) return rc;
  std::sort(t.begin(), t.end());
  *ms_out = t[t.size() / 2];
  return CAPS_OK;
}
}  // namespace

extern "C" int caps_plan_create(const caps_index* ix, const float* Q, int64_t nq,
                                const caps_attrs* cons, int32_t k, int32_t m, int32_t autotune,
                                void* stream, caps_plan** out) {
  if (!out) return fail(CAPS_EINVAL, "null output handle");
  *out = nullptr;
  if (!ix || !Q) return fail(CAPS_EINVAL, "null argument");
  if (nq < 1) return fail(CAPS_EINVAL, "a plan needs nq >= 1");
  if (k < 1 || k > kMaxK) return fail(CAPS_EINVAL, "k must be in [1, 128]");
  if (m < 1 || m > ix->B) return fail(CAPS_EINVAL, "m must be in [1, B]");
  if (ix->meta.sparse) return fail(CAPS_EINVAL, "plans serve dense constraints only");
  if (int rc = check_cons(ix, cons)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  std::unique_ptr<caps_plan> p(new caps_plan());
  p->ix = ix;
  p->generation = ix->generation;
  p->nq = nq;
  p->k = k;
  p->m = m;
  const int L = ix->meta.L;
  if (int rc = plan_alloc(&p->Q, (size_t)nq * ix->d)) return rc;
  if (int rc = plan_alloc(&p->cons, (size_t)nq * L)) return rc;
  if (int rc = plan_alloc(&p->ids, (size_t)nq * k)) return rc;
  if (int rc = plan_alloc(&p->dist, (size_t)nq * k)) return rc;
  CAPS_CUDA(cudaMemcpyAsync(p->Q, Q, sizeof(float) * nq * ix->d, cudaMemcpyDefault, s));
  CAPS_CUDA(cudaMemcpyAsync(p->cons, cons->dense, sizeof(int32_t) * nq * L, cudaMemcpyDefault, s));
  caps_attrs pc = *cons;
  pc.dense = p->cons;
  caps_plan_info& inf = p->info;
  inf.nq = nq;
  inf.k = k;
  inf.m = m;
  SearchOpts best;
  best.timed = false;
  if (uses_tc(ix, k)) {
    const bool pen_ok = uses_pen(ix, k);
    best.pen = pen_ok ? 1 : 0;
    best.tile_n = pen_ok ? 128 : 256;
    inf.tile_n = best.tile_n;
    inf.item_cap = 128;
    inf.pen = best.pen;
    if (autotune) {
      // the scan's launch shapes: filter in the epilogue (rows per tile:
      // accumulator stages) or folded into the MMA (128 rows), x most probes
      // per work item
      const int all[6][3] = {{256, 128, 0}, {128, 128, 0}, {256, 64, 0},
                             {128, 64, 0},  {128, 128, 1}, {128, 64, 1}};
      int shapes[6][3];
      int n_shapes = 0;
      for (const auto& sh : all)
        if (sh[2] ? pen_ok
                  : tc_explicit_ok(ix, k) &&
                        tc_tile_fits(ix->d, ix->meta.words_pad, sh[0],
                                     ix->prec == CAPS_FP8E4M3 ? 1 : 0)) {
          for (int j = 0; j < 3; j++) shapes[n_shapes][j] = sh[j];
          n_shapes++;
        }
      float best_ms = 0.f;
      // every shape computes the same per-probe lists, so the results must
      // agree to the bit: the tuner checks that against the first shape
      std::vector<int64_t> ref_i((size_t)nq * k), got_i((size_t)nq * k);
      std::vector<float> ref_d((size_t)nq * k), got_d((size_t)nq * k);
      for (int c = 0; c < n_shapes; c++) {
        SearchOpts o;
        o.timed = false;
        o.tile_n = shapes[c][0];
        o.item_cap = shapes[c][1];
        o.pen = shapes[c][2];
        float ms = 0.f;
        if (int rc = time_shape(p.get(), pc, o, s, 3, &ms)) return rc;
        std::vector<int64_t>& vi = c == 0 ? ref_i : got_i;
        std::vector<float>& vd = c == 0 ? ref_d : got_d;
        CAPS_CUDA(cudaMemcpyAsync(vi.data(), p->ids, sizeof(int64_t) * vi.size(),
                                  cudaMemcpyDeviceToHost, s));
        CAPS_CUDA(cudaMemcpyAsync(vd.data(), p->dist, sizeof(float) * vd.size(),
                                  cudaMemcpyDeviceToHost, s));
        CAPS_CUDA(cudaStreamSynchronize(s));
        if (c > 0 && (std::memcmp(vi.data(), ref_i.data(), sizeof(int64_t) * vi.size()) != 0 ||
                      std::memcmp(vd.data(), ref_d.data(), sizeof(float) * vd.size()) != 0))
          return fail(CAPS_ECUDA, "tensor-core launch shapes disagree on the tuning batch");
        inf.cand_tile_n[c] = o.tile_n;
        inf.cand_item_cap[c] = o.item_cap;
        inf.cand_pen[c] = o.pen;
        inf.cand_ms[c] = ms;
        inf.n_candidates = c + 1;
        if (c == 0 || ms < best_ms) {
          best_ms = ms;
          best = o;
        }
      }
      inf.tile_n = best.tile_n;
      inf.item_cap = best.item_cap;
      inf.pen = best.pen;
      std::lock_guard<std::mutex> lock(ix->tune_mu);
      ix->tuned[{k, m}] = {best.tile_n, best.item_cap, best.pen};
    }
  }
  CAPS_CUDA(cudaStreamSynchronize(s));  // the input copies, and any tuning runs
  if (int rc = caps_device_status(ix, s)) return rc;
  // capture on a private stream (the legacy default stream cannot be captured)
  cudaStream_t cs = nullptr;
  CAPS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (ce != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(ce, "cudaStreamBeginCapture");
  }
  int rc = search_impl(ix, p->Q, nq, &pc, k, m, p->ids, p->dist, cs, best);
  cudaGraph_t g = nullptr;
  ce = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (rc != CAPS_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc;
  }
  if (ce != cudaSuccess || !g) return cuda_fail(ce, "cudaStreamEndCapture");
  p->graph = g;
  CAPS_CUDA(cudaGraphInstantiate(&p->exec, g, 0));
  size_t nodes = 0;
  CAPS_CUDA(cudaGraphGetNodes(g, nullptr, &nodes));
  inf.graph_nodes = (int32_t)nodes;
  *out = p.release();
  return CAPS_OK;
}

extern "C" int caps_plan_search(caps_plan* p, const float* Q, int64_t nq, const caps_attrs* cons,
                                int64_t* out_ids, float* out_dist, void* stream) {
  if (!p) return fail(CAPS_EINVAL, "null plan");
  if (p->generation != p->ix->generation)
    return fail(CAPS_EINVAL, "points were inserted after the plan was made: make a new plan");
  if (nq < 0 || nq > p->nq) return fail(CAPS_EINVAL, "nq must be in [0, plan nq]");
  if (int rc = check_cons(p->ix, cons)) return rc;
  if (nq == 0) return CAPS_OK;
  if (!Q || !out_ids || !out_dist) return fail(CAPS_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int L = p->ix->meta.L;
  CAPS_CUDA(cudaMemcpyAsync(p->Q, Q, sizeof(float) * nq * p->ix->d, cudaMemcpyDefault, s));
  CAPS_CUDA(cudaMemcpyAsync(p->cons, cons->dense, sizeof(int32_t) * nq * L, cudaMemcpyDefault, s));
  CAPS_CUDA(cudaGraphLaunch(p->exec, s));
  ++g_kernel_launches;
  CAPS_CUDA(cudaMemcpyAsync(out_ids, p->ids, sizeof(int64_t) * nq * p->k, cudaMemcpyDefault, s));
  CAPS_CUDA(cudaMemcpyAsync(out_dist, p->dist, sizeof(float) * nq * p->k, cudaMemcpyDefault, s));
  bool di = false, dd = false;
  if (int rc = is_device_ptr(out_ids, &di)) return rc;
  if (int rc = is_device_ptr(out_dist, &dd)) return rc;
  if (!di || !dd) {
    CAPS_CUDA(cudaStreamSynchronize(s));
    return caps_device_status(p->ix, s);
  }
  return CAPS_OK;
}

extern "C" int caps_plan_get_info(const caps_plan* p, caps_plan_info* out) {
  if (!p || !out) return fail(CAPS_EINVAL, "null argument");
  *out = p->info;
  return CAPS_OK;
}

extern "C" void caps_plan_free(caps_plan* p) { delete p; }

// ---- learned partitioner step entry points ---------------------------------

static int mlp_dims_ok(int32_t d, int32_t H, int32_t B) {
  if (d < 1 || H < 1 || B < 1) return fail(CAPS_EINVAL, "MLP dimensions must be >= 1");
  return CAPS_OK;
}

static int mlp_loss_grad_entry(int32_t d, int32_t H, int32_t B, const float* W1, const float* b1,
                               const float* W2, const float* b2, const float* X, int64_t n,
                               const float* Y, float* gW1, float* gb1, float* gW2, float* gb2,
                               float* loss, void* stream, bool bf16) {
  if (int rc = mlp_dims_ok(d, H, B)) return rc;
  if (n < 1) return fail(CAPS_EINVAL, "n must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  keep_pool_warm();
  Scratch scr(s);
  MlpNet net;
  net.d = d;
  net.H = H;
  net.B = B;
  float* w = nullptr;
  if (int rc = scr.get(&w, (size_t)net.size())) return rc;
  net.bind(w);
  const float *t1, *t2, *t3, *t4, *dX, *dY;
  if (int rc = stage_in(W1, (size_t)H * d, scr, s, &t1)) return rc;
  if (int rc = stage_in(b1, (size_t)H, scr, s, &t2)) return rc;
  if (int rc = stage_in(W2, (size_t)B * H, scr, s, &t3)) return rc;
  if (int rc = stage_in(b2, (size_t)B, scr, s, &t4)) return rc;
  if (int rc = stage_in(X, (size_t)n * d, scr, s, &dX)) return rc;
  if (int rc = stage_in(Y, (size_t)n * B, scr, s, &dY)) return rc;
  CAPS_CUDA(cudaMemcpyAsync(net.W1, t1, sizeof(float) * H * d, cudaMemcpyDeviceToDevice, s));
  CAPS_CUDA(cudaMemcpyAsync(net.b1, t2, sizeof(float) * H, cudaMemcpyDeviceToDevice, s));
  CAPS_CUDA(cudaMemcpyAsync(net.W2, t3, sizeof(float) * B * H, cudaMemcpyDeviceToDevice, s));
  CAPS_CUDA(cudaMemcpyAsync(net.b2, t4, sizeof(float) * B, cudaMemcpyDeviceToDevice, s));
  Out<float> o1, o2, o3, o4;
  if (int rc = o1.init(gW1, (size_t)H * d, scr)) return rc;
  if (int rc = o2.init(gb1, (size_t)H, scr)) return rc;
  if (int rc = o3.init(gW2, (size_t)B * H, scr)) return rc;
  if (int rc = o4.init(gb2, (size_t)B, scr)) return rc;
  MlpNet g = net;
  g.W1 = o1.dev;
  g.b1 = o2.dev;
  g.W2 = o3.dev;
  g.b2 = o4.dev;
  float* dl = nullptr;
  if (int rc = scr.get(&dl, 1)) return rc;
  int32_t* err = nullptr;
  if (bf16) {
    if (int rc = scr.get(&err, 1)) return rc;
    CAPS_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
    if (int rc = mlp_loss_grad_bf16(net, dX, nullptr, n, dY, &g, dl, err, scr, s)) return rc;
    int32_t he = 0;
    CAPS_CUDA(cudaMemcpyAsync(&he, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CAPS_CUDA(cudaStreamSynchronize(s));
    if (he) return fail(CAPS_ETIMEOUT, "a bounded device wait expired in the bf16 step");
  } else if (int rc = mlp_loss_grad(net, dX, n, dY, &g, dl, scr, s)) {
    return rc;
  }
  if (int rc = o1.finish(s)) return rc;
  if (int rc = o2.finish(s)) return rc;
  if (int rc = o3.finish(s)) return rc;
  if (int rc = o4.finish(s)) return rc;
  float lh = 0.f;
  CAPS_CUDA(cudaMemcpyAsync(&lh, dl, sizeof(float), cudaMemcpyDeviceToHost, s));
  CAPS_CUDA(cudaStreamSynchronize(s));
  if (loss) *loss = lh;
  return CAPS_OK;
}

extern "C" int caps_mlp_loss_grad(int32_t d, int32_t H, int32_t B, const float* W1,
                                  const float* b1, const float* W2, const float* b2,
                                  const float* X, int64_t n, const float* Y, float* gW1,
                                  float* gb1, float* gW2, float* gb2, float* loss, void* stream) {
  return mlp_loss_grad_entry(d, H, B, W1, b1, W2, b2, X, n, Y, gW1, gb1, gW2, gb2, loss, stream,
                             false);
}

extern "C" int caps_mlp_loss_grad_bf16(int32_t d, int32_t H, int32_t B, const float* W1,
                                       const float* b1, const float* W2, const float* b2,
                                       const float* X, int64_t n, const float* Y, float* gW1,
                                       float* gb1, float* gW2, float* gb2, float* loss,
                                       void* stream) {
  return mlp_loss_grad_entry(d, H, B, W1, b1, W2, b2, X, n, Y, gW1, gb1, gW2, gb2, loss, stream,
                             true);
}

static int mlp_train_entry(int32_t d, int32_t H, int32_t B, float* W, const float* X, int64_t n,
                           const float* Y, int32_t epochs, int32_t batch, float lr, float* losses,
                           void* stream, bool bf16) {
  if (int rc = mlp_dims_ok(d, H, B)) return rc;
  if (n < 1 || epochs < 0 || batch < 1 || !(lr > 0.f)) return fail(CAPS_EINVAL, "bad training arguments");
  cudaStream_t s = (cudaStream_t)stream;
  keep_pool_warm();
  Scratch scr(s);
  MlpNet net;
  net.d = d;
  net.H = H;
  net.B = B;
  Out<float> ow;
  if (int rc = ow.init(W, (size_t)net.size(), scr)) return rc;
  if (ow.host)
    CAPS_CUDA(cudaMemcpyAsync(ow.dev, W, sizeof(float) * net.size(), cudaMemcpyHostToDevice, s));
  net.bind(ow.dev);
  const float *dX, *dY;
  if (int rc = stage_in(X, (size_t)n * d, scr, s, &dX)) return rc;
  if (int rc = stage_in(Y, (size_t)n * B, scr, s, &dY)) return rc;
  if (int rc = mlp_train(net, dX, n, dY, epochs, batch, lr, losses, s, bf16)) return rc;
  if (int rc = ow.finish(s)) return rc;
  CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

extern "C" int caps_mlp_train(int32_t d, int32_t H, int32_t B, float* W, const float* X,
                              int64_t n, const float* Y, int32_t epochs, int32_t batch, float lr,
                              float* losses, void* stream) {
  return mlp_train_entry(d, H, B, W, X, n, Y, epochs, batch, lr, losses, stream, false);
}

extern "C" int caps_mlp_train_bf16(int32_t d, int32_t H, int32_t B, float* W, const float* X,
                                   int64_t n, const float* Y, int32_t epochs, int32_t batch,
                                   float lr, float* losses, void* stream) {
  return mlp_train_entry(d, H, B, W, X, n, Y, epochs, batch, lr, losses, stream, true);
}

extern "C" int caps_mlp_assign(int32_t d, int32_t H, int32_t B, const float* W, const float* X,
                               int64_t n, int32_t* out_bin, void* stream) {
  if (int rc = mlp_dims_ok(d, H, B)) return rc;
  if (n < 0) return fail(CAPS_EINVAL, "n < 0");
  if (n == 0) return CAPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  keep_pool_warm();
  Scratch scr(s);
  MlpNet net;
  net.d = d;
  net.H = H;
  net.B = B;
  const float *dW, *dX;
  if (int rc = stage_in(W, (size_t)net.size(), scr, s, &dW)) return rc;
  if (int rc = stage_in(X, (size_t)n * d, scr, s, &dX)) return rc;
  net.bind(const_cast<float*>(dW));
  Out<int32_t> ob;
  if (int rc = ob.init(out_bin, (size_t)n, scr)) return rc;
  if (int rc = mlp_assign(net, dX, n, ob.dev, scr, s)) return rc;
  if (int rc = ob.finish(s)) return rc;
  if (ob.host) CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

extern "C" int caps_mlp_balance(int32_t d, int32_t H, int32_t B, const float* W, const float* X,
                                int64_t n, int32_t R, const int64_t* load0, int32_t* out_bin,
                                void* stream) {
  if (int rc = mlp_dims_ok(d, H, B)) return rc;
  if (n < 0) return fail(CAPS_EINVAL, "n < 0");
  if (R < 1 || R > 64 || R > B) return fail(CAPS_EINVAL, "R must be in [1, min(64, B)]");
  if (B > 25600) return fail(CAPS_EINVAL, "balanced assignment needs B <= 25600");
  if (n == 0) return CAPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  keep_pool_warm();
  Scratch scr(s);
  MlpNet net;
  net.d = d;
  net.H = H;
  net.B = B;
  const float *dW, *dX;
  const int64_t* dL = nullptr;
  if (int rc = stage_in(W, (size_t)net.size(), scr, s, &dW)) return rc;
  if (int rc = stage_in(X, (size_t)n * d, scr, s, &dX)) return rc;
  if (load0)
    if (int rc = stage_in(load0, (size_t)B, scr, s, &dL)) return rc;
  net.bind(const_cast<float*>(dW));
  Out<int32_t> ob;
  if (int rc = ob.init(out_bin, (size_t)n, scr)) return rc;
  if (int rc = mlp_balanced_assign(net, dX, n, R, dL, ob.dev, scr, s)) return rc;
  if (int rc = ob.finish(s)) return rc;
  if (ob.host) CAPS_CUDA(cudaStreamSynchronize(s));
  return CAPS_OK;
}

// ---- disjunctive (OR) constraints (Sec. 5.3) -------------------------------
extern "C" int caps_search_batch_or(const caps_index* ix, const float* Q, int64_t nq,
                                    const caps_or_constraints* oc, int32_t k, int32_t m,
                                    int64_t* out_ids, float* out_dist, void* stream) {
  if (!ix || !oc) return fail(CAPS_EINVAL, "null argument");
  if (nq < 0) return fail(CAPS_EINVAL, "nq < 0");
  if (k < 1 || k > kMaxK) return fail(CAPS_EINVAL, "k must be in [1, 128]");
  if (m < 1 || m > ix->B) return fail(CAPS_EINVAL, "m must be in [1, B]");
  if (ix->meta.sparse) return fail(CAPS_EINVAL, "OR constraints need dense attributes");
  const int L = ix->meta.L;
  if (oc->L != L) return fail(CAPS_EINVAL, "constraints must have the index's L fields");
  if (nq == 0) return CAPS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  // the value lists on the host, expanded into single-valued sub-queries
  std::vector<int64_t> voff;
  if (int rc = to_host(oc->offsets, (size_t)(nq * L + 1), &voff, s)) return rc;
  if (voff[0] != 0) return fail(CAPS_EINVAL, "offsets[0] must be 0");
  for (size_t i = 1; i < voff.size(); i++)
    if (voff[i] < voff[i - 1]) return fail(CAPS_EINVAL, "offsets must not decrease");
  std::vector<int32_t> vals;
  if (int rc = to_host(oc->values, (size_t)voff.back(), &vals, s)) return rc;
  for (int32_t v : vals)
    if (v < 0) return fail(CAPS_EINVAL, "OR values must be >= 0");
  std::vector<int32_t> sub_cons;
  std::vector<int64_t> sub_q, soff((size_t)nq + 1, 0);
  std::vector<int64_t> pos((size_t)L);
  std::vector<int32_t> b((size_t)L);
  for (int64_t q = 0; q < nq; q++) {
    int64_t combos = 1;
    for (int f = 0; f < L; f++) {
      const int64_t n = voff[q * L + f + 1] - voff[q * L + f];
      combos *= n > 0 ? n : 1;
      if (combos > kMaxOrCombos)
        return fail(CAPS_EINVAL, "an OR query expands into more than 256 single-valued queries");
    }
    for (int f = 0; f < L; f++) {
      pos[f] = voff[q * L + f];
      b[f] = pos[f] < voff[q * L + f + 1] ? vals[pos[f]] : -1;
    }
    for (;;) {  // mixed-radix walk over the constrained fields' lists
      sub_cons.insert(sub_cons.end(), b.begin(), b.end());
      sub_q.push_back(q);
      int f = 0;
      for (; f < L; f++) {
        const int64_t e = voff[q * L + f + 1];
        if (voff[q * L + f] == e) continue;
        if (++pos[f] < e) {
          b[f] = vals[pos[f]];
          break;
        }
        pos[f] = voff[q * L + f];
        b[f] = vals[pos[f]];
      }
      if (f == L) break;
    }
    soff[q + 1] = (int64_t)sub_q.size();
  }
  const int64_t n_sub = (int64_t)sub_q.size();
  Scratch scr(s);
  const float* dQ = nullptr;
  if (int rc = stage_in(Q, (size_t)nq * ix->d, scr, s, &dQ)) return rc;
  int64_t *d_subq = nullptr, *d_soff = nullptr, *d_ids = nullptr;
  int32_t* d_cons = nullptr;
  float *d_Qs = nullptr, *d_dist = nullptr;
  if (int rc = scr.get(&d_subq, (size_t)n_sub)) return rc;
  if (int rc = scr.get(&d_soff, (size_t)nq + 1)) return rc;
  if (int rc = scr.get(&d_cons, (size_t)n_sub * L)) return rc;
  if (int rc = scr.get(&d_Qs, (size_t)n_sub * ix->d)) return rc;
  if (int rc = scr.get(&d_ids, (size_t)n_sub * k)) return rc;
  if (int rc = scr.get(&d_dist, (size_t)n_sub * k)) return rc;
  CAPS_CUDA(cudaMemcpyAsync(d_subq, sub_q.data(), sizeof(int64_t) * (size_t)n_sub,
                            cudaMemcpyHostToDevice, s));
  CAPS_CUDA(cudaMemcpyAsync(d_soff, soff.data(), sizeof(int64_t) * soff.size(),
                            cudaMemcpyHostToDevice, s));
  CAPS_CUDA(cudaMemcpyAsync(d_cons, sub_cons.data(), sizeof(int32_t) * sub_cons.size(),
                            cudaMemcpyHostToDevice, s));
  if (int rc = launch_gather_rows(dQ, d_subq, n_sub, ix->d, d_Qs, s)) return rc;
  caps_attrs at{};
  at.L = L;
  at.dense = d_cons;
  SearchOpts o;
  o.cached = true;
  if (int rc = search_impl(ix, d_Qs, n_sub, &at, k, m, d_ids, d_dist, s, o)) return rc;
  Out<int64_t> oi;
  Out<float> od;
  if (int rc = oi.init(out_ids, (size_t)nq * k, scr)) return rc;
  if (int rc = od.init(out_dist, (size_t)nq * k, scr)) return rc;
  if (int rc = launch_or_merge(d_ids, d_dist, d_soff, nq, k, ix->metric, oi.dev, od.dev, s)) return rc;
  if (int rc = oi.finish(s)) return rc;
  if (int rc = od.finish(s)) return rc;
  CAPS_CUDA(cudaStreamSynchronize(s));  // the host copies above outlive the call
  return caps_device_status(ix, s);
}

// ---- dynamic insertion (Table 1; the mechanism is this library's reading) ---
extern "C" int caps_insert(caps_index* ix, const float* X, int64_t n, const caps_attrs* attrs,
                           void* stream) {
  if (!ix || !attrs) return fail(CAPS_EINVAL, "null argument");
  if (n < 0) return fail(CAPS_EINVAL, "n < 0");
  if (ix->meta.sparse) return fail(CAPS_EINVAL, "insertion serves dense attributes only");
  const DenseMeta& meta = ix->meta;
  const int L = meta.L, d = ix->d, B = ix->B, h = ix->h;
  if (attrs->L != L || (n > 0 && (!attrs->dense || !X)))
    return fail(CAPS_EINVAL, "attributes must be dense with the index's L fields");
  if (n == 0) return CAPS_OK;
  const int64_t N0 = ix->N, N1 = N0 + n;
  if (N1 >= (int64_t)INT32_MAX) return fail(CAPS_EINVAL, "the index would exceed 2^31-1 points");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  const float* dX = nullptr;
  const int32_t* dA = nullptr;
  if (int rc = stage_in(X, (size_t)n * d, scr, s, &dX)) return rc;
  if (int rc = stage_in(attrs->dense, (size_t)n * L, scr, s, &dA)) return rc;
  int32_t* bad = nullptr;
  if (int rc = scr.get(&bad, 1)) return rc;
  CAPS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
  if (int rc = launch_check_dense(dA, n, meta, bad, s)) return rc;
  int32_t bad_h = 0;
  CAPS_CUDA(cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CAPS_CUDA(cudaStreamSynchronize(s));
  if (bad_h) return fail(CAPS_EINVAL, "attribute value outside [0, vocab[f])");
  // every point in id order: the built ones back from the layout, then the new
  float* Xall = nullptr;
  int32_t* Aall = nullptr;
  if (int rc = scr.get(&Xall, (size_t)N1 * d)) return rc;
  if (int rc = scr.get(&Aall, (size_t)N1 * L)) return rc;
  if (int rc = launch_unlayout(ix->Xp, ix->Ap, ix->perm, N0, d, meta, Xall, Aall, s)) return rc;
  CAPS_CUDA(cudaMemcpyAsync(Xall + N0 * d, dX, sizeof(float) * (size_t)n * d,
                            cudaMemcpyDeviceToDevice, s));
  CAPS_CUDA(cudaMemcpyAsync(Aall + N0 * L, dA, sizeof(int32_t) * (size_t)n * L,
                            cudaMemcpyDeviceToDevice, s));
  // New arrays for every point; the index keeps its old ones until all of
  // them (and the bf16 / e4m3 rows) are ready, so a failure leaves it as it
  // was.
  struct Arrays {
    int32_t* bin = nullptr;
    uint8_t* key = nullptr;
    int32_t* perm = nullptr;
    int32_t* offsets = nullptr;
    float* Xp = nullptr;
    uint32_t* Ap = nullptr;
    void* Xb = nullptr;
    float *xn = nullptr, *xs = nullptr;
    int32_t* iperm = nullptr;
  };
  auto release_all = [&](const Arrays& x) {
    ix->release(x.bin);
    ix->release(x.key);
    ix->release(x.perm);
    ix->release(x.offsets);
    ix->release(x.Xp);
    ix->release(x.Ap);
    ix->release(x.Xb);
    ix->release(x.xn);
    ix->release(x.xs);
    ix->release(x.iperm);
  };
  Arrays nw;
  auto build_new = [&]() -> int {
    const int64_t nseg = (int64_t)B * (h + 1);
    if (int rc = ix->alloc(&nw.bin, (size_t)N1)) return rc;
    if (int rc = ix->alloc(&nw.key, (size_t)N1)) return rc;
    if (int rc = ix->alloc(&nw.perm, (size_t)N1 + 4)) return rc;
    if (int rc = ix->alloc(&nw.offsets, (size_t)nseg + 1)) return rc;
    if (int rc = ix->alloc(&nw.Xp, (size_t)N1 * d)) return rc;
    if (int rc = ix->alloc(&nw.Ap, (size_t)(N1 + 4) * meta.words_pad)) return rc;
    CAPS_CUDA(cudaMemcpyAsync(nw.bin, ix->bin, sizeof(int32_t) * (size_t)N0, cudaMemcpyDeviceToDevice, s));
    CAPS_CUDA(cudaMemcpyAsync(nw.key, ix->key, (size_t)N0, cudaMemcpyDeviceToDevice, s));
    // f(x) of the new points (the index's partition function), then their
    // blocks under the unchanged tags
    if (ix->part == CAPS_PART_MLP && ix->balance_r > 0) {
      // the balanced rule, loads starting from the current partition sizes
      int64_t* load = nullptr;
      if (int rc = scr.get(&load, (size_t)B)) return rc;
      k_part_loads<<<(B + 127) / 128, 128, 0, s>>>(ix->offsets, B, h, load);
      CAPS_LAUNCH("k_part_loads");
      if (int rc = mlp_balanced_assign(ix->mlp, dX, n, ix->balance_r, load, nw.bin + N0, scr, s))
        return rc;
    } else if (ix->part == CAPS_PART_MLP) {
      if (int rc = mlp_assign(ix->mlp, dX, n, nw.bin + N0, scr, s)) return rc;
    } else if (int rc = launch_assign(dX, n, d, ix->C, B, ix->metric, nw.bin + N0, s)) {
      return rc;
    }
    if (int rc = launch_block_of(dA, nw.bin + N0, n, ix->tags, h, meta, ix->code_field,
                                 nw.key + N0, s))
      return rc;
    // the stable order by (partition, block, id) of all N1 points
    int32_t* seg = nullptr;
    if (int rc = scr.get(&seg, (size_t)N1)) return rc;
    if (int rc = launch_segment_keys(nw.bin, nw.key, N1, h, seg, s)) return rc;
    if (int rc = stable_sort_by_key(seg, N1, nseg, nw.perm, nw.offsets, scr, s)) return rc;
    if (int rc = launch_layout(Xall, Aall, nw.perm, N1, d, meta, nw.Xp, nw.Ap, s)) return rc;
    CAPS_CUDA(cudaMemsetAsync(nw.perm + N1, 0, sizeof(int32_t) * 4, s));
    CAPS_CUDA(cudaMemsetAsync(nw.Ap + N1 * meta.words_pad, 0, sizeof(uint32_t) * 4 * meta.words_pad, s));
    return CAPS_OK;
  };
  if (int rc = build_new()) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    release_all(nw);
    return rc;
  }
  // switch to the new arrays and derive the bf16 / e4m3 form from them
  Arrays old;
  old.bin = ix->bin;
  old.key = ix->key;
  old.perm = ix->perm;
  old.offsets = ix->offsets;
  old.Xp = ix->Xp;
  old.Ap = ix->Ap;
  old.Xb = ix->Xb;
  old.xn = ix->xn;
  old.xs = ix->xs;
  old.iperm = ix->iperm;
  const float old_xn_max = ix->xn_max;
  alignas(128) unsigned char old_tmap[sizeof(ix->tmap)];
  std::memcpy(old_tmap, ix->tmap, sizeof(ix->tmap));
  auto set = [&](const Arrays& x, int64_t N) {
    ix->bin = x.bin;
    ix->key = x.key;
    ix->perm = x.perm;
    ix->offsets = x.offsets;
    ix->Xp = x.Xp;
    ix->Ap = x.Ap;
    ix->Xb = x.Xb;
    ix->xn = x.xn;
    ix->xs = x.xs;
    ix->iperm = x.iperm;
    ix->N = N;
  };
  set(nw, N1);
  int rc = prepare_precision(ix, s);
  if (rc == CAPS_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "caps_insert");
  }
  nw.Xb = ix->Xb;
  nw.xn = ix->xn;
  nw.xs = ix->xs;
  nw.iperm = ix->iperm;
  if (rc != CAPS_OK) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    set(old, N0);
    ix->xn_max = old_xn_max;
    std::memcpy(ix->tmap, old_tmap, sizeof(ix->tmap));
    release_all(nw);
    return rc;
  }
  release_all(old);
  ix->generation++;
  return CAPS_OK;
}
