// Index construction kernels: CAPS Alg. 1 on the GPU.
//
//   k-means first level (Sec. 5.2)  : k_dist_tile<ARGMIN> + stable sort by
//                                     partition + fp64 centroid sums
//   f(x_i) assignment (Alg. 1 loop) : k_dist_tile<ARGMIN>
//   attribute frequency tree        : k_aft (one CTA per partition)
//   contiguous sub-partitions       : stable sort by (partition, block) +
//                                     k_layout_rows / k_layout_attrs
#include <algorithm>
#include <cfloat>
#include <climits>

#include "caps_internal.cuh"

namespace caps {

// ---------------------------------------------------------------------------
// Distance tiles.  Every (row, centroid) score is accumulated over the
// coordinates in order j = 0..d-1 with one fused multiply-add per coordinate
// (L2: t = x_j - c_j, acc = fma(t, t, acc); IP: acc = fma(x_j, c_j, acc)).
// A 64x64 output tile per CTA, 4x4 per thread, k staged through shared
// memory 16 coordinates at a time; zero padding past d leaves acc unchanged.
// ---------------------------------------------------------------------------
namespace {
constexpr int TM = 64, TN = 64, TK = 16, TPAD = 4;

template <int METRIC>
__device__ __forceinline__ bool better(float s1, int i1, float s2, int i2) {
  if (s1 != s2) return METRIC == CAPS_L2 ? (s1 < s2) : (s1 > s2);
  return i1 < i2;
}

template <bool VEC>
__device__ __forceinline__ void load_tile(const float* __restrict__ src, int64_t rows,
                                          int d, int64_t r0, int k0,
                                          float (*dst)[TM + TPAD], int tid) {
  // 64 rows x 16 coordinates; thread -> (row tid/4, coords (tid%4)*4..+3)
  const int r = tid >> 2, c = (tid & 3) * 4;
  const int64_t gr = r0 + r;
  const int gc = k0 + c;
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  if (gr < rows) {
    const float* p = src + gr * (int64_t)d + gc;
    if (VEC) {
      if (gc < d) {
        float4 t = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
      }
    } else {
#pragma unroll
      for (int e = 0; e < 4; e++)
        if (gc + e < d) v[e] = __ldg(p + e);
    }
  }
#pragma unroll
  for (int e = 0; e < 4; e++) dst[c + e][r] = v[e];
}

// MODE 0: argmin/argmax over all centroids -> out_bin.  MODE 1: all scores.
template <int METRIC, int MODE, bool VEC>
__global__ void __launch_bounds__(256)
k_dist_tile(const float* __restrict__ X, int64_t N, int d, const float* __restrict__ C,
            int B, int32_t* __restrict__ out_bin, float* __restrict__ out_s) {
  __shared__ __align__(16) float Xs[TK][TM + TPAD];
  __shared__ __align__(16) float Cs[TK][TM + TPAD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * TM;
  const float worst = METRIC == CAPS_L2 ? INFINITY : -INFINITY;
  float best[4];
  int bidx[4];
#pragma unroll
  for (int i = 0; i < 4; i++) { best[i] = worst; bidx[i] = INT_MAX; }
  const int n_lo = MODE == 0 ? 0 : blockIdx.y * TN;
  const int n_hi = MODE == 0 ? B : min(B, n_lo + TN);
  for (int n0 = n_lo; n0 < n_hi; n0 += TN) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
      for (int j = 0; j < 4; j++) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < d; k0 += TK) {
      load_tile<VEC>(X, N, d, m0, k0, Xs, tid);
      load_tile<VEC>(C, B, d, n0, k0, Cs, tid);
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < TK; kk++) {
        const float4 xa = *reinterpret_cast<const float4*>(&Xs[kk][ty * 4]);
        const float4 cb = *reinterpret_cast<const float4*>(&Cs[kk][tx * 4]);
        const float xv[4] = {xa.x, xa.y, xa.z, xa.w};
        const float cv[4] = {cb.x, cb.y, cb.z, cb.w};
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
          for (int j = 0; j < 4; j++) {
            if (METRIC == CAPS_L2) {
              const float t = xv[i] - cv[j];
              acc[i][j] = fmaf(t, t, acc[i][j]);
            } else {
              acc[i][j] = fmaf(xv[i], cv[j], acc[i][j]);
            }
          }
      }
      __syncthreads();
    }
    if (MODE == 0) {
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int c = n0 + tx * 4 + j;
          if (c < B && better<METRIC>(acc[i][j], c, best[i], bidx[i])) {
            best[i] = acc[i][j];
            bidx[i] = c;
          }
        }
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const int64_t r = m0 + ty * 4 + i;
        if (r >= N) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
          const int c = n0 + tx * 4 + j;
          if (c < B) out_s[r * B + c] = acc[i][j];
        }
      }
    }
  }
  if (MODE == 0) {
    // the 16 threads sharing a row group are lanes tx = 0..15 of one half-warp
#pragma unroll
    for (int i = 0; i < 4; i++) {
      float s = best[i];
      int c = bidx[i];
#pragma unroll
      for (int off = 8; off > 0; off >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, off);
        const int c2 = __shfl_xor_sync(0xffffffffu, c, off);
        if (better<METRIC>(s2, c2, s, c)) { s = s2; c = c2; }
      }
      const int64_t r = m0 + ty * 4 + i;
      if (tx == 0 && r < N) out_bin[r] = (c == INT_MAX) ? 0 : c;
    }
  }
}

template <int MODE>
int launch_dist(const float* X, int64_t N, int d, const float* C, int B, int metric,
                int32_t* bin, float* scores, cudaStream_t s) {
  if (N == 0) return CAPS_OK;
  const bool vec = (d % 4) == 0 && ((uintptr_t)X % 16) == 0 && ((uintptr_t)C % 16) == 0;
  const int64_t gx = (N + TM - 1) / TM;
  if (gx > INT_MAX) return fail(CAPS_EINVAL, "too many rows for the distance grid");
  dim3 grid((unsigned)gx, MODE == 0 ? 1u : (unsigned)((B + TN - 1) / TN));
  if (grid.y > 65535) return fail(CAPS_EINVAL, "too many centroids for the score grid");
#define CAPS_DIST(MET, V) k_dist_tile<MET, MODE, V><<<grid, 256, 0, s>>>(X, N, d, C, B, bin, scores)
  if (metric == CAPS_L2) {
    if (vec) CAPS_DIST(CAPS_L2, true); else CAPS_DIST(CAPS_L2, false);
  } else {
    if (vec) CAPS_DIST(CAPS_IP, true); else CAPS_DIST(CAPS_IP, false);
  }
#undef CAPS_DIST
  CAPS_LAUNCH("k_dist_tile");
  return CAPS_OK;
}
}  // namespace

int launch_assign(const float* X, int64_t N, int d, const float* C, int B, int metric,
                  int32_t* bin, cudaStream_t s) {
  return launch_dist<0>(X, N, d, C, B, metric, bin, nullptr, s);
}

int launch_scores(const float* Q, int64_t nq, int d, const float* C, int B, int metric,
                  float* scores, cudaStream_t s) {
  return launch_dist<1>(Q, nq, d, C, B, metric, nullptr, scores, s);
}

// ---------------------------------------------------------------------------
// Row gather (k-means seed points).
// ---------------------------------------------------------------------------
namespace {
__global__ void k_gather_rows(const float* __restrict__ X, const int64_t* __restrict__ idx,
                              int64_t n, int d, float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * d) return;
  const int64_t r = t / d, j = t % d;
  out[t] = X[idx[r] * d + j];
}
}  // namespace

int launch_gather_rows(const float* X, const int64_t* idx, int64_t n, int d, float* out,
                       cudaStream_t s) {
  const int64_t tot = n * d;
  if (tot == 0) return CAPS_OK;
  k_gather_rows<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, idx, n, d, out);
  CAPS_LAUNCH("k_gather_rows");
  return CAPS_OK;
}

// ---------------------------------------------------------------------------
// Exclusive prefix sum of int32 (totals < 2^31), three phases, recursive.
// ---------------------------------------------------------------------------
namespace {
constexpr int SCAN_T = 256, SCAN_ITEMS = 16, SCAN_BLOCK = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ int block_incl_scan(int v, int* wsum) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) wsum[w] = v;
  __syncthreads();
  if (w == 0) {
    int x = lane < SCAN_T / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    if (lane < SCAN_T / 32) wsum[lane] = x;
  }
  __syncthreads();
  if (w > 0) v += wsum[w - 1];
  __syncthreads();
  return v;
}

// In-place exclusive scan of each SCAN_BLOCK chunk; block totals to sums.
__global__ void __launch_bounds__(SCAN_T)
k_scan_blocks(int32_t* __restrict__ data, int64_t n, int32_t* __restrict__ sums) {
  __shared__ int wsum[SCAN_T / 32];
  __shared__ int tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  int carry = 0;
  for (int it = 0; it < SCAN_ITEMS && base + (int64_t)it * SCAN_T < n; it++) {  // block-uniform
    const int64_t e = base + (int64_t)it * SCAN_T + threadIdx.x;
    const int v = e < n ? data[e] : 0;
    const int inc = block_incl_scan(v, wsum);
    if (e < n) data[e] = carry + inc - v;
    if (threadIdx.x == SCAN_T - 1) tot = inc;
    __syncthreads();
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[blockIdx.x] = carry;
}

__global__ void k_scan_add(int32_t* __restrict__ data, int64_t n,
                           const int32_t* __restrict__ sums) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) data[e] += sums[e / SCAN_BLOCK];
}

int scan_exclusive(int32_t* data, int64_t n, Scratch& scr, cudaStream_t s) {
  if (n == 0) return CAPS_OK;
  const int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  int32_t* sums = nullptr;
  if (int rc = scr.get(&sums, (size_t)nb)) return rc;
  k_scan_blocks<<<(unsigned)nb, SCAN_T, 0, s>>>(data, n, sums);
  CAPS_LAUNCH("k_scan_blocks");
  if (nb > 1) {
    if (int rc = scan_exclusive(sums, nb, scr, s)) return rc;
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(data, n, sums);
    CAPS_LAUNCH("k_scan_add");
  }
  return CAPS_OK;
}
}  // namespace

int scan_exclusive_i32(int32_t* data, int64_t n, Scratch& scr, cudaStream_t s) {
  return scan_exclusive(data, n, scr, s);
}

// ---------------------------------------------------------------------------
// Stable counting sort by key.  The n elements are cut into tiles; counts
// are kept per (key, tile) in key-major order, so one exclusive scan of the
// count matrix gives, for every (key, tile), the first output position of
// that tile's elements with that key.  The scatter walks each tile in index
// order (warps in turn), which keeps equal keys in index order.
// ---------------------------------------------------------------------------
namespace {
constexpr int SORT_T = 256;

__global__ void __launch_bounds__(SORT_T)
k_sort_hist(const int32_t* __restrict__ keys, int64_t n, int tile, int64_t ntile,
            int32_t* __restrict__ counts) {
  const int64_t t = blockIdx.x;
  const int64_t beg = t * tile, end = min(n, beg + tile);
  for (int64_t e = beg + threadIdx.x; e < end; e += SORT_T)
    atomicAdd(&counts[(int64_t)keys[e] * ntile + t], 1);
}

__global__ void k_sort_segoff(const int32_t* __restrict__ scanned, int64_t K, int64_t ntile,
                              int64_t n, int32_t* __restrict__ seg_off) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < K) seg_off[s] = scanned[s * ntile];
  if (s == K) seg_off[K] = (int32_t)n;
}

__global__ void __launch_bounds__(SORT_T)
k_sort_scatter(const int32_t* __restrict__ keys, int64_t n, int tile, int64_t ntile,
               int32_t* __restrict__ cursor, int32_t* __restrict__ perm) {
  const int64_t t = blockIdx.x;
  const int64_t beg = t * tile, end = min(n, beg + tile);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t c0 = beg; c0 < end; c0 += SORT_T) {
    const int64_t e = c0 + threadIdx.x;
    const bool valid = e < end;
    const int key = valid ? keys[e] : 0;
    for (int w = 0; w < SORT_T / 32; w++) {
      if (warp == w) {
        const unsigned act = __ballot_sync(0xffffffffu, valid);
        if (valid) {
          const unsigned peers = __match_any_sync(act, key);
          const int leader = __ffs(peers) - 1;
          const int rank = __popc(peers & lt);
          int base = 0;
          int32_t* cur = &cursor[(int64_t)key * ntile + t];
          if (lane == leader) {
            base = *cur;
            *cur = base + __popc(peers);
          }
          base = __shfl_sync(peers, base, leader);
          perm[base + rank] = (int32_t)e;
        }
      }
      __syncthreads();
    }
  }
}
}  // namespace

int stable_sort_by_key(const int32_t* keys, int64_t n, int64_t K, int32_t* perm,
                       int32_t* seg_off, Scratch& scr, cudaStream_t s) {
  if (K < 1) return fail(CAPS_EINVAL, "sort: K < 1");
  if (n > INT_MAX) return fail(CAPS_EINVAL, "sort: n >= 2^31");
  // bound the count matrix to ~16M entries by growing the tile
  const int64_t max_tiles = std::max<int64_t>(1, (int64_t)(1 << 24) / K);
  int64_t tile = 2048;
  while ((n + tile - 1) / tile > max_tiles) tile *= 2;
  const int64_t ntile = std::max<int64_t>(1, (n + tile - 1) / tile);
  int32_t* counts = nullptr;
  if (int rc = scr.get(&counts, (size_t)(K * ntile))) return rc;
  CAPS_CUDA(cudaMemsetAsync(counts, 0, sizeof(int32_t) * K * ntile, s));
  if (n > 0) {
    k_sort_hist<<<(unsigned)ntile, SORT_T, 0, s>>>(keys, n, (int)tile, ntile, counts);
    CAPS_LAUNCH("k_sort_hist");
  }
  if (int rc = scan_exclusive(counts, K * ntile, scr, s)) return rc;
  k_sort_segoff<<<(unsigned)((K + 1 + 255) / 256), 256, 0, s>>>(counts, K, ntile, n, seg_off);
  CAPS_LAUNCH("k_sort_segoff");
  if (n > 0) {
    k_sort_scatter<<<(unsigned)ntile, SORT_T, 0, s>>>(keys, n, (int)tile, ntile, counts, perm);
    CAPS_LAUNCH("k_sort_scatter");
  }
  return CAPS_OK;
}

// ---------------------------------------------------------------------------
// k-means centroid update: fp64 sum of each partition's members in id order,
// mean = sum / count, rounded to fp32 (IP: normalised to unit length first);
// an empty partition keeps its centroid.
// ---------------------------------------------------------------------------
namespace {
__global__ void k_centroid_sums(const float* __restrict__ X, int d,
                                const int32_t* __restrict__ perm_bin,
                                const int32_t* __restrict__ bin_off,
                                double* __restrict__ sums) {
  const int c = blockIdx.x;
  const int beg = bin_off[c], end = bin_off[c + 1];
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double acc = 0.0;
    int u = beg;
    for (; u + 4 <= end; u += 4) {
      const float v0 = __ldg(X + (int64_t)perm_bin[u] * d + j);
      const float v1 = __ldg(X + (int64_t)perm_bin[u + 1] * d + j);
      const float v2 = __ldg(X + (int64_t)perm_bin[u + 2] * d + j);
      const float v3 = __ldg(X + (int64_t)perm_bin[u + 3] * d + j);
      acc = __dadd_rn(acc, (double)v0);
      acc = __dadd_rn(acc, (double)v1);
      acc = __dadd_rn(acc, (double)v2);
      acc = __dadd_rn(acc, (double)v3);
    }
    for (; u < end; u++) acc = __dadd_rn(acc, (double)__ldg(X + (int64_t)perm_bin[u] * d + j));
    sums[(int64_t)c * d + j] = acc;
  }
}

__global__ void k_centroid_finalize(double* __restrict__ sums, const int32_t* __restrict__ bin_off,
                                    int B, int d, int metric, float* __restrict__ C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= B) return;
  const int cnt = bin_off[c + 1] - bin_off[c];
  if (cnt == 0) return;
  double* s = sums + (int64_t)c * d;
  for (int j = 0; j < d; j++) s[j] = __ddiv_rn(s[j], (double)cnt);
  if (metric == CAPS_IP) {
    double nrm = 0.0;
    for (int j = 0; j < d; j++) nrm = __dadd_rn(nrm, __dmul_rn(s[j], s[j]));
    nrm = __dsqrt_rn(nrm);
    if (nrm > 0.0)
      for (int j = 0; j < d; j++) s[j] = __ddiv_rn(s[j], nrm);
  }
  for (int j = 0; j < d; j++) C[(int64_t)c * d + j] = __double2float_rn(s[j]);
}
}  // namespace

int launch_centroid_update(const float* X, int d, const int32_t* perm_bin,
                           const int32_t* bin_off, int B, int metric, float* C,
                           Scratch& scr, cudaStream_t s) {
  double* sums = nullptr;
  if (int rc = scr.get(&sums, (size_t)B * d)) return rc;
  const int threads = std::min(256, ((d + 31) / 32) * 32);
  k_centroid_sums<<<B, threads, 0, s>>>(X, d, perm_bin, bin_off, sums);
  CAPS_LAUNCH("k_centroid_sums");
  k_centroid_finalize<<<(B + 127) / 128, 128, 0, s>>>(sums, bin_off, B, d, metric, C);
  CAPS_LAUNCH("k_centroid_finalize");
  return CAPS_OK;
}

// ---------------------------------------------------------------------------
// Attribute checks and code tables.
// ---------------------------------------------------------------------------
namespace {
__global__ void k_check_dense(const int32_t* __restrict__ A, int64_t N, DenseMeta meta,
                              int32_t* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * meta.L) return;
  const int f = (int)(t % meta.L);
  const int v = A[t];
  if (v < 0 || v >= meta.vocab[f]) atomicExch(bad, 1);
}

__global__ void k_code_field(DenseMeta meta, uint8_t* __restrict__ code_field) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= meta.n_codes) return;
  int f = 0;
  while (f + 1 < meta.L && meta.code_off[f + 1] <= c) f++;
  code_field[c] = (uint8_t)f;
}
}  // namespace

int launch_check_dense(const int32_t* A, int64_t N, const DenseMeta& meta, int32_t* bad,
                       cudaStream_t s) {
  const int64_t tot = N * meta.L;
  if (tot == 0) return CAPS_OK;
  k_check_dense<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A, N, meta, bad);
  CAPS_LAUNCH("k_check_dense");
  return CAPS_OK;
}

int launch_code_field(const DenseMeta& meta, uint8_t* code_field, cudaStream_t s) {
  if (meta.n_codes == 0) return CAPS_OK;
  k_code_field<<<(unsigned)((meta.n_codes + 255) / 256), 256, 0, s>>>(meta, code_field);
  CAPS_LAUNCH("k_code_field");
  return CAPS_OK;
}

// ---------------------------------------------------------------------------
// Attribute frequency tree (Alg. 1, second loop), one CTA per partition.
// Round j: histogram of the codes carried by the points not yet peeled,
// t_j = most frequent code (ties -> lowest code), points carrying t_j get
// block j.  No point left (or no code left) -> t_j..t_h = -1.  Points never
// peeled get block h+1.  key[] must be zero on entry; 0 marks "not peeled".
// ---------------------------------------------------------------------------
namespace {
constexpr int AFT_T = 256;

__global__ void __launch_bounds__(AFT_T)
k_aft(const int32_t* __restrict__ perm_bin, const int32_t* __restrict__ bin_off, int h,
      const int32_t* __restrict__ A, DenseMeta meta, const uint8_t* __restrict__ code_field,
      int32_t* __restrict__ tags, uint8_t* __restrict__ key) {
  extern __shared__ int hist[];  // [n_codes]
  __shared__ unsigned long long red[AFT_T / 32];
  __shared__ int t_sh;
  const int b = blockIdx.x;
  const int beg = bin_off[b], end = bin_off[b + 1];
  const int V = (int)meta.n_codes, L = meta.L;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  bool done = false;
  for (int j = 1; j <= h; j++) {
    if (done) {
      if (threadIdx.x == 0) tags[(int64_t)b * h + j - 1] = -1;
      continue;
    }
    for (int c = threadIdx.x; c < V; c += AFT_T) hist[c] = 0;
    __syncthreads();
    for (int u = beg + threadIdx.x; u < end; u += AFT_T) {
      const int i = perm_bin[u];
      if (key[i] != 0) continue;
      for (int f = 0; f < L; f++) atomicAdd(&hist[meta.code_off[f] + A[(int64_t)i * L + f]], 1);
    }
    __syncthreads();
    // argmax: larger count first, then lower code
    unsigned long long best = 0ull;
    for (int c = threadIdx.x; c < V; c += AFT_T) {
      const unsigned long long cand =
          ((unsigned long long)(unsigned)hist[c] << 32) | (unsigned long long)(0xffffffffu - (unsigned)c);
      if (cand > best) best = cand;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, o);
      if (x > best) best = x;
    }
    if (lane == 0) red[w] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = red[0];
      for (int q = 1; q < AFT_T / 32; q++) m = red[q] > m ? red[q] : m;
      const unsigned cnt = (unsigned)(m >> 32);
      t_sh = cnt > 0 ? (int)(0xffffffffu - (unsigned)(m & 0xffffffffull)) : -1;
      tags[(int64_t)b * h + j - 1] = t_sh;
    }
    __syncthreads();
    const int t = t_sh;
    if (t < 0) {
      done = true;
      continue;
    }
    const int tf = code_field[t];
    const int tv = t - meta.code_off[tf];
    for (int u = beg + threadIdx.x; u < end; u += AFT_T) {
      const int i = perm_bin[u];
      if (key[i] == 0 && A[(int64_t)i * L + tf] == tv) key[i] = (uint8_t)j;
    }
    __syncthreads();
  }
  for (int u = beg + threadIdx.x; u < end; u += AFT_T) {
    const int i = perm_bin[u];
    if (key[i] == 0) key[i] = (uint8_t)(h + 1);
  }
}
}  // namespace

int launch_aft(const int32_t* perm_bin, const int32_t* bin_off, int B, int h,
               const int32_t* A, const DenseMeta& meta, const uint8_t* code_field,
               int32_t* tags, uint8_t* key, cudaStream_t s) {
  const size_t smem = sizeof(int) * (size_t)std::max<int64_t>(1, meta.n_codes);
  if (smem > 200 * 1024) return fail(CAPS_EINVAL, "too many attribute codes for the AFT kernel");
  if (smem > 48 * 1024)
    CAPS_CUDA(cudaFuncSetAttribute(k_aft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_aft<<<B, AFT_T, smem, s>>>(perm_bin, bin_off, h, A, meta, code_field, tags, key);
  CAPS_LAUNCH("k_aft");
  return CAPS_OK;
}

// ---------------------------------------------------------------------------
// Layout: segment key, permuted rows, packed attributes, position table.
// ---------------------------------------------------------------------------
namespace {
__global__ void k_segment_keys(const int32_t* __restrict__ bin, const uint8_t* __restrict__ key,
                               int64_t N, int h, int32_t* __restrict__ seg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) seg[i] = bin[i] * (h + 1) + (int)key[i] - 1;
}

__global__ void k_layout_rows4(const float4* __restrict__ X, const int32_t* __restrict__ perm,
                               int64_t N, int d4, float4* __restrict__ Xp) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * d4) return;
  const int64_t r = t / d4, c = t % d4;
  Xp[t] = __ldg(X + (int64_t)perm[r] * d4 + c);
}

__global__ void k_layout_rows1(const float* __restrict__ X, const int32_t* __restrict__ perm,
                               int64_t N, int d, float* __restrict__ Xp) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * d) return;
  const int64_t r = t / d, c = t % d;
  Xp[t] = __ldg(X + (int64_t)perm[r] * d + c);
}

__global__ void k_layout_attrs(const int32_t* __restrict__ A, const int32_t* __restrict__ perm,
                               int64_t N, DenseMeta meta, uint32_t* __restrict__ Ap) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int64_t i = perm[r];
  uint32_t w[4] = {0u, 0u, 0u, 0u};
  for (int f = 0; f < meta.L; f++)
    w[meta.word[f]] |= (uint32_t)A[i * meta.L + f] << meta.shift[f];
  for (int q = 0; q < meta.words_pad; q++) Ap[r * meta.words_pad + q] = w[q];
}

__global__ void k_pos_table(const int32_t* __restrict__ tags, int B, int h, int64_t n_codes,
                            uint8_t* __restrict__ pos) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)B * h) return;
  const int b = (int)(t / h), j = (int)(t % h) + 1;
  const int c = tags[t];
  if (c >= 0 && c < n_codes) pos[(int64_t)b * n_codes + c] = (uint8_t)j;
}
}  // namespace

int launch_segment_keys(const int32_t* bin, const uint8_t* key, int64_t N, int h,
                        int32_t* seg, cudaStream_t s) {
  if (N == 0) return CAPS_OK;
  k_segment_keys<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(bin, key, N, h, seg);
  CAPS_LAUNCH("k_segment_keys");
  return CAPS_OK;
}

int launch_layout(const float* X, const int32_t* A, const int32_t* perm, int64_t N, int d,
                  const DenseMeta& meta, float* Xp, uint32_t* Ap, cudaStream_t s) {
  if (N == 0) return CAPS_OK;
  if (d % 4 == 0 && (uintptr_t)X % 16 == 0 && (uintptr_t)Xp % 16 == 0) {
    const int64_t tot = N * (d / 4);
    k_layout_rows4<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const float4*>(X), perm, N, d / 4, reinterpret_cast<float4*>(Xp));
  } else {
    const int64_t tot = N * d;
    k_layout_rows1<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, perm, N, d, Xp);
  }
  CAPS_LAUNCH("k_layout_rows");
  if (meta.sparse) return CAPS_OK;  // label sets: launch_layout_sparse
  k_layout_attrs<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(A, perm, N, meta, Ap);
  CAPS_LAUNCH("k_layout_attrs");
  return CAPS_OK;
}

namespace {
// ---- dynamic insertion: the built points back in id order, the new ones'
// blocks ----------------------------------------------------------------------
// X[perm[r]] = Xp[r]: the rows of the layout back at their original ids
__global__ void k_unlayout_rows(const float* __restrict__ Xp, const int32_t* __restrict__ perm,
                                int64_t N, int d, float* __restrict__ X) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N * d) return;
  const int64_t r = t / d, c = t % d;
  X[(int64_t)perm[r] * d + c] = Xp[t];
}
// A[perm[r]][f] = field f's bits of the packed row Ap[r]
__global__ void k_unpack_attrs(const uint32_t* __restrict__ Ap, const int32_t* __restrict__ perm,
                               int64_t N, DenseMeta meta, int32_t* __restrict__ A) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int64_t i = perm[r];
  for (int f = 0; f < meta.L; f++) {
    const uint32_t w = Ap[r * meta.words_pad + meta.word[f]];
    const uint32_t mask = meta.bits[f] >= 32 ? 0xffffffffu : ((1u << meta.bits[f]) - 1u);
    A[i * meta.L + f] = (int32_t)((w >> meta.shift[f]) & mask);
  }
}
// key[i] = the first block j of partition bin[i] whose tag point i carries,
// else h + 1 (the block the attribute-frequency peel would give it under the
// partition's tags; a tag of -1 ends the partition's tree)
__global__ void k_block_of(const int32_t* __restrict__ A, const int32_t* __restrict__ bin, int64_t n,
                           const int32_t* __restrict__ tags, int h, DenseMeta meta,
                           const uint8_t* __restrict__ code_field, uint8_t* __restrict__ key) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t* t = tags + (int64_t)bin[i] * h;
  int j = 1;
  for (; j <= h; j++) {
    const int c = t[j - 1];
    if (c < 0) {
      j = h + 1;
      break;
    }
    const int f = code_field[c];
    if (A[i * meta.L + f] == c - meta.code_off[f]) break;
  }
  key[i] = (uint8_t)j;
}
}  // namespace

int launch_unlayout(const float* Xp, const uint32_t* Ap, const int32_t* perm, int64_t N, int d,
                    const DenseMeta& meta, float* X, int32_t* A, cudaStream_t s) {
  if (N == 0) return CAPS_OK;
  k_unlayout_rows<<<(unsigned)((N * d + 255) / 256), 256, 0, s>>>(Xp, perm, N, d, X);
  CAPS_LAUNCH("k_unlayout_rows");
  k_unpack_attrs<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(Ap, perm, N, meta, A);
  CAPS_LAUNCH("k_unpack_attrs");
  return CAPS_OK;
}

int launch_block_of(const int32_t* A, const int32_t* bin, int64_t n, const int32_t* tags, int h,
                    const DenseMeta& meta, const uint8_t* code_field, uint8_t* key, cudaStream_t s) {
  if (n == 0) return CAPS_OK;
  k_block_of<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A, bin, n, tags, h, meta, code_field, key);
  CAPS_LAUNCH("k_block_of");
  return CAPS_OK;
}

int launch_pos_table(const int32_t* tags, int B, int h, int64_t n_codes, uint8_t* pos,
                     cudaStream_t s) {
  const int64_t tot = (int64_t)B * h;
  if (tot == 0) return CAPS_OK;
  k_pos_table<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(tags, B, h, n_codes, pos);
  CAPS_LAUNCH("k_pos_table");
  return CAPS_OK;
}

// ---------------------------------------------------------------------------
// Sparse label sets (Def. 1 with label-set attributes): validation, the
// attribute frequency tree over label codes, and the layout-order copies.
// ---------------------------------------------------------------------------
namespace {
__global__ void k_check_sparse(const int64_t* __restrict__ off, const int32_t* __restrict__ lab,
                               int64_t N, int32_t V, int32_t* __restrict__ off32,
                               int32_t* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > N) return;
  const int64_t o = off[i];
  if (o < 0 || o > INT_MAX) atomicExch(bad, 1);
  off32[i] = (int32_t)o;
  if (i == N) return;
  const int64_t e = off[i + 1];
  if (e < o) {
    atomicExch(bad, 1);
    return;
  }
  int32_t prev = -1;
  for (int64_t r = o; r < e; r++) {
    const int32_t c = lab[r];
    if (c < 0 || c >= V || c <= prev) {
      atomicExch(bad, 1);
      return;
    }
    prev = c;
  }
}

// One CTA per partition; as k_aft, but a point carries its labels as codes.
__global__ void __launch_bounds__(AFT_T)
k_aft_sparse(const int32_t* __restrict__ perm_bin, const int32_t* __restrict__ bin_off, int h,
             const int32_t* __restrict__ off, const int32_t* __restrict__ lab, int32_t V,
             int32_t* __restrict__ tags, uint8_t* __restrict__ key) {
  extern __shared__ int hist[];  // [V]
  __shared__ unsigned long long red[AFT_T / 32];
  __shared__ int t_sh;
  const int b = blockIdx.x;
  const int beg = bin_off[b], end = bin_off[b + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  bool done = false;
  for (int j = 1; j <= h; j++) {
    if (done) {
      if (threadIdx.x == 0) tags[(int64_t)b * h + j - 1] = -1;
      continue;
    }
    for (int c = threadIdx.x; c < V; c += AFT_T) hist[c] = 0;
    __syncthreads();
    for (int u = beg + threadIdx.x; u < end; u += AFT_T) {
      const int i = perm_bin[u];
      if (key[i] != 0) continue;
      for (int r = off[i]; r < off[i + 1]; r++) atomicAdd(&hist[lab[r]], 1);
    }
    __syncthreads();
    unsigned long long best = 0ull;
    for (int c = threadIdx.x; c < V; c += AFT_T) {
      const unsigned long long cand =
          ((unsigned long long)(unsigned)hist[c] << 32) | (unsigned long long)(0xffffffffu - (unsigned)c);
      if (cand > best) best = cand;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, best, o);
      if (x > best) best = x;
    }
    if (lane == 0) red[w] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = red[0];
      for (int q = 1; q < AFT_T / 32; q++) m = red[q] > m ? red[q] : m;
      const unsigned cnt = (unsigned)(m >> 32);
      t_sh = cnt > 0 ? (int)(0xffffffffu - (unsigned)(m & 0xffffffffull)) : -1;
      tags[(int64_t)b * h + j - 1] = t_sh;
    }
    __syncthreads();
    const int t = t_sh;
    if (t < 0) {
      done = true;
      continue;
    }
    for (int u = beg + threadIdx.x; u < end; u += AFT_T) {
      const int i = perm_bin[u];
      if (key[i] != 0) continue;
      for (int r = off[i]; r < off[i + 1]; r++)
        if (lab[r] == t) {
          key[i] = (uint8_t)j;
          break;
        }
    }
    __syncthreads();
  }
  for (int u = beg + threadIdx.x; u < end; u += AFT_T) {
    const int i = perm_bin[u];
    if (key[i] == 0) key[i] = (uint8_t)(h + 1);
  }
}

__global__ void k_layout_sparse_sig(const int32_t* __restrict__ off, const int32_t* __restrict__ lab,
                                    const int32_t* __restrict__ perm, int64_t N,
                                    uint32_t* __restrict__ Ap, int32_t* __restrict__ cnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > N) return;
  if (r == N) {
    cnt[N] = 0;
    return;
  }
  const int i = perm[r];
  uint64_t sig = 0ull;
  for (int u = off[i]; u < off[i + 1]; u++) sig |= 1ull << sig_bit(lab[u]);
  Ap[2 * r] = (uint32_t)sig;
  Ap[2 * r + 1] = (uint32_t)(sig >> 32);
  cnt[r] = off[i + 1] - off[i];
}

__global__ void k_layout_sparse_lab(const int32_t* __restrict__ off, const int32_t* __restrict__ lab,
                                    const int32_t* __restrict__ perm, int64_t N,
                                    const int32_t* __restrict__ off_p, int32_t* __restrict__ lab_p) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int i = perm[r];
  const int o = off_p[r];
  for (int u = off[i]; u < off[i + 1]; u++) lab_p[o + (u - off[i])] = lab[u];
}
}  // namespace

int launch_check_sparse(const int64_t* off, const int32_t* lab, int64_t N, int32_t V,
                        int32_t* off32, int32_t* bad, cudaStream_t s) {
  k_check_sparse<<<(unsigned)((N + 1 + 255) / 256), 256, 0, s>>>(off, lab, N, V, off32, bad);
  CAPS_LAUNCH("k_check_sparse");
  return CAPS_OK;
}

int launch_aft_sparse(const int32_t* perm_bin, const int32_t* bin_off, int B, int h,
                      const int32_t* off, const int32_t* lab, int32_t V, int32_t* tags,
                      uint8_t* key, cudaStream_t s) {
  const size_t smem = sizeof(int) * (size_t)std::max<int32_t>(1, V);
  if (smem > 200 * 1024) return fail(CAPS_EINVAL, "label vocabulary too large for the AFT kernel");
  if (smem > 48 * 1024)
    CAPS_CUDA(cudaFuncSetAttribute(k_aft_sparse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  k_aft_sparse<<<B, AFT_T, smem, s>>>(perm_bin, bin_off, h, off, lab, V, tags, key);
  CAPS_LAUNCH("k_aft_sparse");
  return CAPS_OK;
}

int launch_layout_sparse(const int32_t* off, const int32_t* lab, const int32_t* perm, int64_t N,
                         uint32_t* Ap, int32_t* off_p, int32_t* lab_p, Scratch& scr,
                         cudaStream_t s) {
  k_layout_sparse_sig<<<(unsigned)((N + 1 + 255) / 256), 256, 0, s>>>(off, lab, perm, N, Ap, off_p);
  CAPS_LAUNCH("k_layout_sparse_sig");
  if (int rc = scan_exclusive_i32(off_p, N + 1, scr, s)) return rc;
  if (N > 0) {
    k_layout_sparse_lab<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(off, lab, perm, N, off_p, lab_p);
    CAPS_LAUNCH("k_layout_sparse_lab");
  }
  return CAPS_OK;
}

}  // namespace caps
