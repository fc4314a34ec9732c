// caps_search_batch_noalloc: the batched query of caps_search_batch for
// callers that cannot allocate device memory.
//
// Who needs it: a caller whose device memory is fully reserved up front by
// another framework (nothing is left for a per-call pool), a latency-bound
// serving loop that must never wait on the allocator or on cudaFree's
// implicit device synchronisation, or an integration whose rules forbid any
// allocator call after start-up.  Such a caller passes device inputs and
// device outputs; the per-query intermediates (centroid scores, probes,
// selections, packed filters) live in one fixed array compiled into this
// library instead of coming from cudaMalloc or a memory pool.
//
// The array is a file-scope __device__ object: every GPU that loads the
// library holds it until the process exits.  Host code never dereferences
// its name (on the host the name is only a stand-in, not a device address);
// the device address is looked up once per device with
// cudaGetSymbolAddress and handed to the kernels.
#include <mutex>

#include "caps_internal.cuh"

namespace caps {
namespace {

// 16 MiB: enough for ~3,800 queries per pass at B = 1024; larger batches run
// in several passes over the same array.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up on the
// first call made with that device current).
int scratch_address(void** out) {
  *out = nullptr;
  int dev = 0;
  CAPS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(CAPS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return fail(CAPS_ECUDA, std::string("cudaGetSymbolAddress(scratch) failed: ") +
                                  cudaGetErrorString(e));
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CAPS_OK;
}

int require_device(const void* p, const char* what) {
  if (!p) return fail(CAPS_EINVAL, std::string("null ") + what);
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(CAPS_EINVAL, std::string(what) + " must be device memory (no staging without allocation)");
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(CAPS_EINVAL, std::string(what) + " must be device memory (no staging without allocation)");
  int cur = 0;
  CAPS_CUDA(cudaGetDevice(&cur));
  if (at.type == cudaMemoryTypeDevice && at.device != cur)
    return fail(CAPS_EINVAL, std::string(what) + " belongs to another GPU");
  return CAPS_OK;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// Scratch bytes one query needs (each array rounded up per pass below).
size_t bytes_per_query(const caps_index* ix, int m) {
  const int WP = ix->meta.words_pad, L = ix->meta.L;
  return sizeof(float) * ix->B + sizeof(int32_t) * m + sizeof(uint64_t) * m +
         2 * sizeof(uint32_t) * WP + sizeof(int32_t) * L + 1;
}

}  // namespace
}  // namespace caps

using namespace caps;

extern "C" int caps_search_batch_noalloc(const caps_index* ix, const float* Q, int64_t nq,
                                         const caps_attrs* cons, int32_t k, int32_t m,
                                         int64_t* out_ids, float* out_dist, void* stream) {
  if (!ix) return fail(CAPS_EINVAL, "null index");
  if (nq < 0) return fail(CAPS_EINVAL, "nq < 0");
  if (k < 1 || k > kMaxK) return fail(CAPS_EINVAL, "k must be in [1, 128]");
  if (m < 1 || m > ix->B) return fail(CAPS_EINVAL, "m must be in [1, B]");
  if (ix->meta.sparse) return fail(CAPS_EINVAL, "the no-allocation query serves dense attributes only");
  if (!cons || cons->dense == nullptr || cons->L != ix->meta.L)
    return fail(CAPS_EINVAL, "constraints must be dense with the index's L fields");
  if (ix->part != CAPS_PART_KMEANS)
    return fail(CAPS_EINVAL, "the no-allocation query serves k-means indexes only");
  if (nq == 0) return CAPS_OK;
  if (int rc = require_device(Q, "Q")) return rc;
  if (int rc = require_device(cons->dense, "constraints")) return rc;
  if (int rc = require_device(out_ids, "out_ids")) return rc;
  if (int rc = require_device(out_dist, "out_dist")) return rc;
  // one pass must hold at least one query: 7 arrays, each padded to 256 B
  const size_t per_q = bytes_per_query(ix, m);
  if (per_q + 7 * 256 > kNoAllocScratchBytes)
    return fail(CAPS_EINVAL,
                "B and m need more than the 16 MiB no-allocation scratch for one query");
  void* base = nullptr;
  if (int rc = scratch_address(&base)) return rc;
  const int64_t qc = std::min<int64_t>(nq, (int64_t)((kNoAllocScratchBytes - 7 * 256) / per_q));
  const int WP = ix->meta.words_pad, L = ix->meta.L;
  unsigned char* p = static_cast<unsigned char*>(base);
  auto carve = [&](size_t bytes) {
    unsigned char* r = p;
    p += round256(bytes);
    return r;
  };
  float* scores = reinterpret_cast<float*>(carve(sizeof(float) * qc * ix->B));
  int32_t* probe = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * qc * m));
  uint64_t* sel = reinterpret_cast<uint64_t*>(carve(sizeof(uint64_t) * qc * m));
  QueryPrep qp;
  qp.qmask = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * qc * WP));
  qp.qval = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * qc * WP));
  qp.qcode = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * qc * L));
  qp.dead = carve((size_t)qc);
  if ((size_t)(p - static_cast<unsigned char*>(base)) > kNoAllocScratchBytes)
    return fail(CAPS_EINVAL, "no-allocation scratch layout overflow");

  cudaStream_t s = (cudaStream_t)stream;
  const int32_t* Qb = cons->dense;
  for (int64_t c0 = 0; c0 < nq; c0 += qc) {
    const int64_t n = std::min(qc, nq - c0);
    const float* Qc = Q + c0 * ix->d;
    const int32_t* Qbc = Qb + c0 * L;
    if (int rc = launch_query_prep(Qbc, n, ix->meta, qp, s)) return rc;
    if (int rc = launch_scores(Qc, n, ix->d, ix->C, ix->B, ix->metric, scores, s)) return rc;
    if (int rc = launch_topm(scores, n, ix->B, m, ix->metric, probe, s)) return rc;
    if (int rc = launch_select(probe, n, m, ix->h, ix->tags, ix->pos, ix->meta.n_codes,
                               ix->code_field, Qbc, ix->meta, qp.qcode, sel, s))
      return rc;
    ScanArgs a;
    a.Xp = ix->Xp;
    a.Ap = ix->Ap;
    a.perm = ix->perm;
    a.offsets = ix->offsets;
    a.Q = Qc;
    a.qp = qp;
    a.probe = probe;
    a.sel = sel;
    a.nq = n;
    a.m = m;
    a.h = ix->h;
    a.d = ix->d;
    a.k = k;
    a.metric = ix->metric;
    a.words_pad = ix->meta.words_pad;
    a.out_ids = out_ids + c0 * k;
    a.out_dist = out_dist + c0 * k;
    if (int rc = launch_scan_topk(a, s)) return rc;
  }
  return CAPS_OK;
}
