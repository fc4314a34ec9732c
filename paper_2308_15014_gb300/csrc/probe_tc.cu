// Alg. 2 "select top m partitions" on the tensor cores, exact.
//
// The probe ranks every partition of a query by an fp32 score with a fixed
// summation order: the centroid distance (L2: t = c - q, acc = fma(t, t, acc)
// over the coordinates in order; IP: acc = fma(c, q, acc)) or the learned
// partitioner's logit (acc = fma(h, w, acc) over the hidden units in order,
// then + bias).  Here the scores are first approximated for all partitions
// by one bf16 tensor-core GEMM of split operands: every fp32 value v becomes
// hi = bf16(v) and lo = bf16(v - hi), and the query side [hi | hi | lo]
// times the weight side [hi | lo | hi] gives hi*hi + hi*lo + lo*hi, the dot
// product up to the lo*lo term and rounding (relative error about 2^-14 of
// sum |a_k w_k|).  With eps = 2^-11 |a| |w| (Cauchy-Schwarz, about four
// times the derived bound) every partition gets an interval [lb, ub] that
// holds its exact score.  A partition whose lb exceeds the m-th largest ub
// is certainly among the m best; one whose ub is below the m-th largest lb
// certainly is not; only the few in between are re-scored with the exact
// fixed-order fp32 chain and ranked (ties to the lower partition).  So the
// probe set is exactly the one the fp32 scores give.  The order within the
// set is not the score order (the certain partitions come first, by index):
// the rest of the query does not depend on it.
#include "scan_tc_kernel.cuh"

namespace caps {
namespace {

constexpr int PG_M = 128, PG_N = 256, PG_S = 2, PG_T = 128;
constexpr float kScreenEps = 4.8828125e-4f;  // 2^-11

__host__ __device__ constexpr size_t pg_smem_bytes() {
  return 1024 + (size_t)PG_S * (16384 + 32768);
}

// fp32 rows [rows, K] -> bf16 rows [rows, 3*Kp] (zero padded to Kp):
// query side [hi | hi | lo], weight side [hi | lo | hi].
__global__ void k_split3(const float* __restrict__ X, int64_t rows, int K, int Kp, int wside,
                         __nv_bfloat16* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * Kp) return;
  const int64_t r = t / Kp;
  const int k = (int)(t % Kp);
  const float x = k < K ? X[r * K + k] : 0.f;
  const __nv_bfloat16 hi = __float2bfloat16_rn(x);
  const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
  __nv_bfloat16* o = out + r * 3 * (int64_t)Kp;
  o[k] = hi;
  o[Kp + k] = wside ? lo : hi;
  o[2 * Kp + k] = wside ? hi : lo;
}

// Query side in one pass, a warp per row: bf16 [hi | hi | lo] (two
// coordinates per lane and store) and the row's squared norm (fp32; its
// rounding is inside eps).
__global__ void k_split3_rows(const float* __restrict__ X, int64_t rows, int K, int Kp,
                              __nv_bfloat16* __restrict__ out, float* __restrict__ n2) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  const float* x = X + r * K;
  __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(out + r * 3 * (int64_t)Kp);
  const int hp = Kp / 2;
  float acc = 0.f;
  for (int k2 = lane; k2 < hp; k2 += 32) {
    const int k = 2 * k2;
    const float v0 = k < K ? x[k] : 0.f, v1 = k + 1 < K ? x[k + 1] : 0.f;
    acc = fmaf(v0, v0, acc);
    acc = fmaf(v1, v1, acc);
    const __nv_bfloat162 hi = __floats2bfloat162_rn(v0, v1);
    const __nv_bfloat162 lo =
        __floats2bfloat162_rn(v0 - __low2float(hi), v1 - __high2float(hi));
    o[k2] = hi;
    o[hp + k2] = hi;
    o[2 * hp + k2] = lo;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) n2[r] = acc;
}

// Squared norm of each row and, when nr is given, the norm (fp32; the
// rounding is inside eps).
__global__ void k_rownorm2(const float* __restrict__ X, int64_t rows, int K, float* __restrict__ n2,
                           float* __restrict__ nr) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  float s = 0.f;
  for (int k = lane; k < K; k += 32) {
    const float x = X[r * K + k];
    s = fmaf(x, x, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    n2[r] = s;
    if (nr) nr[r] = sqrtf(s);
  }
}

// D[M, N] = A[M, Kt] . B[N, Kt]^T (bf16 in, fp32 out): one 128 x 256 tile per
// CTA, K in chunks of 64 through two shared-memory stages (2-D TMA, 128-byte
// swizzle), tcgen05.mma into a 256-column tensor-memory accumulator, thread 0
// issuing copies and MMAs; every wait bounded.
__global__ void __launch_bounds__(PG_T, 1)
k_pgemm(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, int M,
        int N, int Kt, float* __restrict__ D, int32_t* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      smem_raw + ((1024u - (su32(smem_raw) & 1023u)) & 1023u);
  __shared__ uint64_t full[PG_S], freeb[PG_S], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * PG_M, n0 = blockIdx.x * PG_N;
  const int nk = Kt / 64;
  auto sA = [&](int s) { return base + (size_t)s * 49152; };
  auto sB = [&](int s) { return base + (size_t)s * 49152 + 16384; };
  if (tid == 0) {
    for (int i = 0; i < PG_S; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&freeb[i], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base)),
                 "n"(PG_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  if (tid == 0) {
    const uint32_t idesc = idesc_bf16(PG_M, PG_N);
    int issued = 0, waited = 0;
    auto issue = [&](int c) {
      const int s = c % PG_S;
      expect_tx(&full[s], 49152u);
      tma_2d(sA(s), &tA, 64 * c, m0, &full[s]);
      tma_2d(sB(s), &tB, 64 * c, n0, &full[s]);
      tma_2d(sB(s) + 16384, &tB, 64 * c, n0 + 128, &full[s]);
      issued = c + 1;
    };
    bool ok = true;
    for (int c = 0; c < PG_S && c < nk; c++) issue(c);
    for (int c = 0; c < nk && ok; c++) {
      const int s = c % PG_S;
      const uint32_t u = (uint32_t)(c / PG_S);
      ok = mbar_wait(&full[s], u & 1, &s_fail, kTcWaitNs);
      if (!ok) break;
      waited = c + 1;
      tc_fence_after();
      const uint32_t a0 = su32(sA(s)), b0 = su32(sB(s));
#pragma unroll
      for (int ks = 0; ks < 4; ks++)
        mma_bf16(tbase, sdesc(a0 + (uint32_t)(ks * 32)), sdesc(b0 + (uint32_t)(ks * 32)), idesc,
                 (c > 0 || ks > 0) ? 1u : 0u);
      mma_commit(&freeb[s]);
      if (c + PG_S < nk) {
        ok = mbar_wait(&freeb[s], u & 1, &s_fail, kTcWaitNs);  // the stage is free again
        if (ok) issue(c + PG_S);
      }
    }
    if (!ok) {
      s_fail = 1;
      atomicExch(err, 1);
      for (int c = waited; c < issued; c++)  // let the copies in flight land
        mbar_wait(&full[c % PG_S], (uint32_t)((c / PG_S) & 1), nullptr, kTcWaitNs);
    }
    mma_commit(&done);  // arrives once every MMA issued so far has completed
  }
  const bool ok = mbar_wait(&done, 0u, nullptr, kTcWaitNs) && s_fail == 0;
  tc_fence_after();
  if (__all_sync(0xffffffffu, ok)) {
    const int row = m0 + 32 * warp + lane;
    const uint32_t tl = tbase + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < PG_N && n0 + c0 < N; c0 += 8) {
      uint32_t v[8];
      tmem_ld8_issue(tl + (uint32_t)c0, v);
      tmem_wait(v);
      if (row < M) {
        float* dst = D + (int64_t)row * N + n0 + c0;
        if (n0 + c0 + 8 <= N && ((((uintptr_t)dst) & 15) == 0)) {
          reinterpret_cast<float4*>(dst)[0] = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]),
                                                          __uint_as_float(v[2]), __uint_as_float(v[3]));
          reinterpret_cast<float4*>(dst)[1] = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]),
                                                          __uint_as_float(v[6]), __uint_as_float(v[7]));
        } else {
          for (int j = 0; j < 8 && n0 + c0 + j < N; j++) dst[j] = __uint_as_float(v[j]);
        }
      }
    }
  } else if (lane == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(PG_N));
}

// MODE 0: learned partitioner (score = logit, larger is better, bias added);
// MODE 1: L2 centroids (score = distance, smaller is better);
// MODE 2: IP centroids (score = inner product, larger is better).
template <int MODE>
struct Screen {
  // approximate score as "larger is better", and its error bound
  __device__ __forceinline__ static void approx(float dt, float an2, float an, float wn2, float wn,
                                                const float* bias, int b, float& s, float& e) {
    if (MODE == 0) {
      s = dt + bias[b];
      e = kScreenEps * an * wn + 1.0e-6f * fabsf(s);
    } else if (MODE == 1) {
      s = -(wn2 + an2 - 2.f * dt);
      e = kScreenEps * (an + wn) * (an + wn);
    } else {
      s = dt;
      e = kScreenEps * an * wn;
    }
    e = e * 1.001f + 1e-30f;
  }
  // exact key of partition b (ascending = better), the fixed-order chain
  __device__ __forceinline__ static float term(float acc, float av, float wv) {
    if (MODE == 1) {
      const float t = wv - av;
      return fmaf(t, t, acc);
    }
    return fmaf(av, wv, acc);
  }
  __device__ __forceinline__ static uint64_t exact_key(const float* a, const float* w, int K,
                                                       const float* bias, int b) {
    float acc = 0.f;
    int k = 0;
    if (((((uintptr_t)w) | ((uintptr_t)a)) & 15) == 0 && K >= 16) {
      // the weight row in 16-byte loads, the next 16 values in flight while
      // the current ones are summed; terms still in order
      float4 x[4], y[4];
#pragma unroll
      for (int u = 0; u < 4; u++) x[u] = reinterpret_cast<const float4*>(w)[u];
      for (; k + 16 <= K; k += 16) {
        const bool more = k + 32 <= K;
        if (more) {
#pragma unroll
          for (int u = 0; u < 4; u++) y[u] = reinterpret_cast<const float4*>(w + k + 16)[u];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const float4 av = *reinterpret_cast<const float4*>(a + k + 4 * u);
          acc = term(acc, av.x, x[u].x);
          acc = term(acc, av.y, x[u].y);
          acc = term(acc, av.z, x[u].z);
          acc = term(acc, av.w, x[u].w);
        }
        if (more) {
#pragma unroll
          for (int u = 0; u < 4; u++) x[u] = y[u];
        }
      }
    }
    for (; k < K; k++) acc = term(acc, a[k], w[k]);
    if (MODE == 0) acc = acc + bias[b];
    return make_key(MODE == 1 ? acc : -acc, (uint32_t)b);
  }
};

// Descending bitonic sort of 32*V floats held V per lane (position V*lane+s).
// No NaN may take part.
template <int V>
__device__ __forceinline__ void warp_sort_desc(float (&v)[V], int lane) {
#pragma unroll
  for (int size = 2; size <= 32 * V; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride < V) {
#pragma unroll
        for (int s = 0; s < V; s++) {
          const int o = s ^ stride;
          if (o > s) {
            const bool down = ((V * lane + s) & size) == 0;
            const float hi = fmaxf(v[s], v[o]), lo = fminf(v[s], v[o]);
            v[s] = down ? hi : lo;
            v[o] = down ? lo : hi;
          }
        }
      } else {
#pragma unroll
        for (int s = 0; s < V; s++) {
          const int P = V * lane + s;
          const float o = __shfl_xor_sync(0xffffffffu, v[s], stride / V);
          const bool down = (P & size) == 0, lower = (P & stride) == 0;
          v[s] = (lower == down) ? fmaxf(o, v[s]) : fminf(o, v[s]);
        }
      }
    }
}

// The value at position P of a four-per-lane sorted warp array.
__device__ __forceinline__ float at_pos4(const float (&v)[4], int P) {
  const int s = P & 3;
  const float x = s == 0 ? v[0] : (s == 1 ? v[1] : (s == 2 ? v[2] : v[3]));
  return __shfl_sync(0xffffffffu, x, P >> 2);
}

constexpr int kScreenList = 256;  // partitions with ub >= T kept per query
constexpr int kScreenVList = 128;  // upper bounds >= the estimate of V

// Warp per query: intervals, the certain partitions, exact re-score of the
// uncertain ones, and the m-partition probe set.  m <= 64.
//
// Two passes over the B intervals: the first gives, from each lane's four
// largest bounds, T (at or below the m-th largest lower bound) and Vlo (at or
// below the m-th largest upper bound V); the second lists every partition
// with ub >= T (a superset of the certain and uncertain ones, since Vlo >= T
// and lb > V >= Vlo) and the upper bounds >= Vlo (all that decide V).  The
// rest works on the list.  Lists that overflow fall back to full passes.
template <int MODE>
__global__ void __launch_bounds__(128)
k_screen_topm(const float* __restrict__ Dt, int64_t nq, int B, int m, const float* __restrict__ A,
              int K, const float* __restrict__ W, const float* __restrict__ bias,
              const float* __restrict__ an2v, const float* __restrict__ wn2v,
              const float* __restrict__ wnv, int32_t* __restrict__ probe) {
  extern __shared__ float asm_[];  // [4][K] query features
  __shared__ int l_id[4][kScreenList];
  __shared__ float l_lb[4][kScreenList], l_ub[4][kScreenList];
  __shared__ float l_v[4][kScreenVList];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 4 + wp;
  if (q >= nq) return;
  float* a = asm_ + (size_t)wp * K;
  for (int k = lane; k < K; k += 32) a[k] = A[q * K + k];
  __syncwarp();
  const float an2 = an2v[q], an = sqrtf(an2);
  const float* dq = Dt + q * B;
  int* lid = l_id[wp];
  float *llb = l_lb[wp], *lub = l_ub[wp], *lv4 = l_v[wp];
  const unsigned lt = (1u << lane) - 1u;
  const int P = m - 1;
  // (1) each lane's four largest lower and upper bounds (NaN bounds take no
  // part), sorted across the warp
  float lv[4], uv[4];
#pragma unroll
  for (int i = 0; i < 4; i++) lv[i] = uv[i] = -INFINITY;
  for (int b = lane; b < B; b += 32) {
    float s, e;
    Screen<MODE>::approx(dq[b], an2, an, wn2v[b], wnv[b], bias, b, s, e);
    float x = s - e, y = s + e;
    if (!(x == x)) x = -INFINITY;
    if (!(y == y)) y = -INFINITY;
#pragma unroll
    for (int i = 0; i < 4; i++) {
      const float hx = fmaxf(lv[i], x);
      x = fminf(lv[i], x);
      lv[i] = hx;
      const float hy = fmaxf(uv[i], y);
      y = fminf(uv[i], y);
      uv[i] = hy;
    }
  }
  // the m-th best of the 128 lane values is no better than the m-th best of all
  warp_sort_desc<4>(lv, lane);
  const float T = at_pos4(lv, P);
  warp_sort_desc<4>(uv, lane);
  const float Vlo = at_pos4(uv, P);
  // (2) the list (ub >= T) and the upper bounds that decide V (ub >= Vlo)
  int cnt = 0, cv = 0;
  for (int b0 = 0; b0 < B; b0 += 32) {
    const int b = b0 + lane;
    float x = 0.f, y = -INFINITY;
    if (b < B) {
      float s, e;
      Screen<MODE>::approx(dq[b], an2, an, wn2v[b], wnv[b], bias, b, s, e);
      x = s - e;
      y = s + e;
    }
    const bool keep = b < B && y >= T, kv = b < B && y >= Vlo;  // false for NaN
    const unsigned bk = __ballot_sync(0xffffffffu, keep), bv = __ballot_sync(0xffffffffu, kv);
    const int pos = cnt + __popc(bk & lt), pv = cv + __popc(bv & lt);
    if (keep && pos < kScreenList) {
      lid[pos] = b;
      llb[pos] = x;
      lub[pos] = y;
    }
    if (kv && pv < kScreenVList) lv4[pv] = y;
    cnt += __popc(bk);
    cv += __popc(bv);
  }
  __syncwarp();
  // V: the exact m-th largest upper bound; without it no partition is certain
  float V = INFINITY;
  if (cv <= kScreenVList) {
    float v4[4];
#pragma unroll
    for (int s2 = 0; s2 < 4; s2++) v4[s2] = (4 * lane + s2 < cv) ? lv4[4 * lane + s2] : -INFINITY;
    warp_sort_desc<4>(v4, lane);
    V = at_pos4(v4, P);
  }
  // (3) certain partitions (lb > V: at most m - 1 upper bounds exceed V) go
  // straight to the probe list; uncertain ones (ub >= T) are collected in
  // place of the list, in partition order
  int ci = 0, nu = 0;
  int32_t* out = probe + q * m;
  if (cnt <= kScreenList) {
    for (int r0 = 0; r0 < cnt; r0 += 32) {
      const int r = r0 + lane;
      int b = 0;
      bool cert = false, unc = false;
      if (r < cnt) {
        b = lid[r];
        cert = llb[r] > V;
        unc = !cert;  // every listed partition has ub >= T
      }
      __syncwarp();
      const unsigned bc = __ballot_sync(0xffffffffu, cert);
      if (cert) out[ci + __popc(bc & lt)] = b;
      ci += __popc(bc);
      const unsigned bu = __ballot_sync(0xffffffffu, unc);
      if (unc) lid[nu + __popc(bu & lt)] = b;  // at or before this lane's own slot
      nu += __popc(bu);
    }
  } else {
    for (int b0 = 0; b0 < B; b0 += 32) {
      const int b = b0 + lane;
      bool cert = false, unc = false;
      if (b < B) {
        float s, e;
        Screen<MODE>::approx(dq[b], an2, an, wn2v[b], wnv[b], bias, b, s, e);
        cert = (s - e) > V;
        unc = !cert && (s + e) >= T;
      }
      const unsigned bc = __ballot_sync(0xffffffffu, cert);
      if (cert) out[ci + __popc(bc & lt)] = b;
      ci += __popc(bc);
      const unsigned bu = __ballot_sync(0xffffffffu, unc);
      const int pos = nu + __popc(bu & lt);
      if (unc && pos < kScreenList) lid[pos] = b;
      nu += __popc(bu);
    }
  }
  __syncwarp();
  const int need = m - ci;
  // (4) exact scores of the uncertain partitions; the best `need` complete
  // the set (ties to the lower partition)
  WarpTopK<2> top;
  top.init();
  uint64_t kth = kEmptyKey;
  if (nu <= kScreenList) {
    for (int r0 = 0; r0 < nu; r0 += 32) {
      uint64_t key = kEmptyKey;
      if (r0 + lane < nu) {
        const int b = lid[r0 + lane];
        key = Screen<MODE>::exact_key(a, W + (int64_t)b * K, K, bias, b);
      }
      top.offer(key, kth, need, lane);
    }
  } else {
    // many uncertain partitions (wide intervals): re-score all of them
    for (int b0 = 0; b0 < B; b0 += 32) {
      const int b = b0 + lane;
      uint64_t key = kEmptyKey;
      if (b < B) {
        float s, e;
        Screen<MODE>::approx(dq[b], an2, an, wn2v[b], wnv[b], bias, b, s, e);
        if (!((s - e) > V) && (s + e) >= T) key = Screen<MODE>::exact_key(a, W + (int64_t)b * K, K, bias, b);
      }
      top.offer(key, kth, need, lane);
    }
  }
  // a non-finite score can leave the list short: re-score every partition
  // that is not certain (every key, NaN ones included, is then a valid one)
  bool short_list = false;
#pragma unroll
  for (int s2 = 0; s2 < 2; s2++) short_list |= (2 * lane + s2 < need) && top.v[s2] == kEmptyKey;
  if (__any_sync(0xffffffffu, short_list)) {
    top.init();
    kth = kEmptyKey;
    for (int b0 = 0; b0 < B; b0 += 32) {
      const int b = b0 + lane;
      uint64_t key = kEmptyKey;
      if (b < B) {
        float s, e;
        Screen<MODE>::approx(dq[b], an2, an, wn2v[b], wnv[b], bias, b, s, e);
        if (!((s - e) > V)) key = Screen<MODE>::exact_key(a, W + (int64_t)b * K, K, bias, b);
        if (key == kEmptyKey && !((s - e) > V)) key = kEmptyKey - 1 - (uint64_t)(B - b);
      }
      top.offer(key, kth, need, lane);
    }
  }
#pragma unroll
  for (int s2 = 0; s2 < 2; s2++) {
    const int Pp = 2 * lane + s2;
    if (Pp < need) out[ci + Pp] = (int32_t)(top.v[s2] & 0xffffffffu);
  }
  // (5) the set in the order of the approximate scores, best first (ties to
  // the lower partition): only the order inside the row changes, so that the
  // scan can take every query's nearest partitions first
  __syncwarp();
  uint64_t ord[2];
#pragma unroll
  for (int s2 = 0; s2 < 2; s2++) {
    const int Pp = 2 * lane + s2;
    ord[s2] = kEmptyKey;
    if (Pp < m) {
      const int b = out[Pp];
      float sc, e;
      Screen<MODE>::approx(dq[b], an2, an, wn2v[b], wnv[b], bias, b, sc, e);
      if (!(sc == sc)) sc = -INFINITY;
      ord[s2] = make_key(-sc, (uint32_t)b);
    }
  }
  warp_sort<2>(ord, lane);
  __syncwarp();
#pragma unroll
  for (int s2 = 0; s2 < 2; s2++) {
    const int Pp = 2 * lane + s2;
    if (Pp < m) out[Pp] = (int32_t)(ord[s2] & 0xffffffffu);
  }
}

int encode_bf16_map(void* map, const void* ptr, int64_t rows, int64_t cols) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qres;
  CAPS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &qres));
  if (!fn || qres != cudaDriverEntryPointSuccess)
    return fail(CAPS_ECUDA, "cuTensorMapEncodeTiled is not available");
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, 128};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                      const_cast<void*>(ptr), gdim, gstride, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CAPS_ECUDA, "cuTensorMapEncodeTiled failed");
  return CAPS_OK;
}

}  // namespace

int bf16_gemm_nt(const void* A, int64_t M, const void* Bm, int N, int Kt, float* D, int32_t* err,
                 cudaStream_t s) {
  if (M == 0 || N == 0) return CAPS_OK;
  if (M < 0 || N < 0 || Kt < 64 || Kt % 64 != 0 || ((uintptr_t)A & 15) || ((uintptr_t)Bm & 15))
    return fail(CAPS_EINVAL, "bf16 gemm: bad sizes or alignment");
  alignas(64) CUtensorMap mA, mB;
  if (int rc = encode_bf16_map(&mA, A, M, Kt)) return rc;
  if (int rc = encode_bf16_map(&mB, Bm, N, Kt)) return rc;
  const size_t smem = pg_smem_bytes();
  CAPS_CUDA(cudaFuncSetAttribute(k_pgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid((unsigned)((N + PG_N - 1) / PG_N), (unsigned)((M + PG_M - 1) / PG_M));
  if (grid.y > 65535) return fail(CAPS_EINVAL, "bf16 gemm: too many rows in one call");
  k_pgemm<<<grid, PG_T, smem, s>>>(mA, mB, (int)M, N, Kt, D, err);
  CAPS_LAUNCH("k_pgemm");
  return CAPS_OK;
}

bool probe_screen_supported(int K, int B, int m) { return m >= 1 && m <= 64 && m <= B && K >= 1 && K <= 2048; }

size_t probe_weights_elems(int K, int B) { return (size_t)B * 3 * (size_t)((K + 63) / 64 * 64); }

int probe_weights_prepare(const float* W, int B, int K, const ProbeWeights& pw, cudaStream_t s) {
  const int Kp = (K + 63) / 64 * 64;
  k_split3<<<(unsigned)(((int64_t)B * Kp + 255) / 256), 256, 0, s>>>(
      W, B, K, Kp, 1, static_cast<__nv_bfloat16*>(pw.Wh));
  CAPS_LAUNCH("k_split3");
  k_rownorm2<<<(unsigned)((B + 7) / 8), 256, 0, s>>>(W, B, K, pw.wn2, pw.wn);
  CAPS_LAUNCH("k_rownorm2");
  return CAPS_OK;
}

int probe_screened(int mode, const float* A, int64_t n, int K, const float* W, const float* bias,
                   int B, int m, float* Dt, int32_t* probe, int32_t* err, Scratch& scr,
                   cudaStream_t s, const ProbeWeights* pre) {
  if (n == 0) return CAPS_OK;
  if (!probe_screen_supported(K, B, m)) return fail(CAPS_EINVAL, "screened probe: bad sizes");
  const int Kp = (K + 63) / 64 * 64, Kt = 3 * Kp;
  __nv_bfloat16* Ah = nullptr;
  float* an2 = nullptr;
  if (int rc = scr.get(&Ah, (size_t)n * Kt)) return rc;
  if (int rc = scr.get(&an2, (size_t)n)) return rc;
  ProbeWeights pw;
  if (pre && pre->Wh) {
    pw = *pre;
  } else {
    __nv_bfloat16* wh = nullptr;
    if (int rc = scr.get(&wh, (size_t)B * Kt)) return rc;
    pw.Wh = wh;
    if (int rc = scr.get(&pw.wn2, (size_t)B)) return rc;
    if (int rc = scr.get(&pw.wn, (size_t)B)) return rc;
    if (int rc = probe_weights_prepare(W, B, K, pw, s)) return rc;
  }
  __nv_bfloat16* Wh = static_cast<__nv_bfloat16*>(pw.Wh);
  const float *wn2 = pw.wn2, *wn = pw.wn;
  k_split3_rows<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(A, n, K, Kp, Ah, an2);
  CAPS_LAUNCH("k_split3_rows");
  alignas(64) CUtensorMap mA, mB;
  if (int rc = encode_bf16_map(&mA, Ah, n, Kt)) return rc;
  if (int rc = encode_bf16_map(&mB, Wh, B, Kt)) return rc;
  const size_t smem = pg_smem_bytes();
  CAPS_CUDA(cudaFuncSetAttribute(k_pgemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid((unsigned)((B + PG_N - 1) / PG_N), (unsigned)((n + PG_M - 1) / PG_M));
  if (grid.y > 65535) return fail(CAPS_EINVAL, "screened probe: too many queries in one chunk");
  k_pgemm<<<grid, PG_T, smem, s>>>(mA, mB, (int)std::min<int64_t>(n, INT32_MAX), B, Kt, Dt, err);
  CAPS_LAUNCH("k_pgemm");
  const size_t ssm = sizeof(float) * 4 * (size_t)K;
  const unsigned g = (unsigned)((n + 3) / 4);
#define CAPS_SCR(MD)                                                                          \
  do {                                                                                        \
    if (ssm > 48 * 1024)                                                                      \
      CAPS_CUDA(cudaFuncSetAttribute(k_screen_topm<MD>,                                       \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm)); \
    k_screen_topm<MD><<<g, 128, ssm, s>>>(Dt, n, B, m, A, K, W, bias, an2, wn2, wn, probe);  \
  } while (0)
  if (mode == 0) CAPS_SCR(0);
  else if (mode == 1) CAPS_SCR(1);
  else CAPS_SCR(2);
#undef CAPS_SCR
  CAPS_LAUNCH("k_screen_topm");
  return CAPS_OK;
}

}  // namespace caps
