// Learned first-level partitioner (Sec. 5.2, BLISS-style): a two-layer MLP
// f(x) = W2 relu(W1 x + b1) + b2 trained on the GPU with the library's own
// forward, backward and Adam kernels; the partition of x is argmax f(x).
//
// Every GEMM output element accumulates its products in index order with one
// fused multiply-add each and adds the bias afterwards, so the fp32 forward
// (and hence the argmax decision) is reproducible term for term.  Gradients
// are the mean softmax cross-entropy against a label distribution Y over the
// B partitions: dz = (softmax(z) * sum(y) - y) / n.
#include <algorithm>
#include <climits>
#include <cmath>

#include <cuda_bf16.h>

#include "caps_internal.cuh"

namespace caps {
namespace {

constexpr int GM = 64, GN = 64, GK = 16, GP = 4;

// op(A)[m][k]: TA = false -> A[m*lda + k]; TA = true -> A[k*lda + m]
// op(B)[k][n]: TB = false -> B[n*ldb + k] (B stored [N,K]); TB = true -> B[k*ldb + n]
// EPI: 0 = plain, 1 = + bias[n] then relu, 2 = + bias[n], 3 = * (mask[m*ldm + n] > 0)
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256)
k_gemm(const float* __restrict__ A, int lda, const float* __restrict__ Bm, int ldb,
       float* __restrict__ C, int ldc, int M, int N, int K, const float* __restrict__ bias,
       const float* __restrict__ mask, int ldm) {
  __shared__ __align__(16) float As[GK][GM + GP];
  __shared__ __align__(16) float Bs[GK][GN + GP];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GK) {
    // 64 x 16 of op(A) and 16 x 64 of op(B): 1024 elements each, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int x = tid + 256 * e;
      int mm, kk;
      if (TA) { kk = x >> 6; mm = x & 63; } else { mm = x >> 4; kk = x & 15; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = v;
      int nn, kb;
      if (TB) { kb = x >> 6; nn = x & 63; } else { nn = x >> 4; kb = x & 15; }
      const int gn = n0 + nn, gkb = k0 + kb;
      float w = 0.f;
      if (gn < N && gkb < K) w = TB ? Bm[(int64_t)gkb * ldb + gn] : Bm[(int64_t)gn * ldb + gkb];
      Bs[kb][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk++) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      if (EPI == 1) {
        v = v + bias[n];
        v = v > 0.f ? v : 0.f;
      } else if (EPI == 2) {
        v = v + bias[n];
      } else if (EPI == 3) {
        v = mask[(int64_t)m * ldm + n] > 0.f ? v : 0.f;
      }
      C[(int64_t)m * ldc + n] = v;
    }
  }
}

// Softmax cross-entropy per row (warp per row): dz and the row's share of
// the mean loss (summed over the rows afterwards in a fixed fp32 order).
__global__ void k_softmax_xent(const float* __restrict__ Z, const float* __restrict__ Y, int n,
                               int B, float inv_n, float* __restrict__ dZ,
                               float* __restrict__ row_loss) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const float* z = Z + (int64_t)i * B;
  const float* y = Y + (int64_t)i * B;
  float mx = -INFINITY;
  for (int c = lane; c < B; c += 32) mx = fmaxf(mx, z[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float se = 0.f, ys = 0.f;
  for (int c = lane; c < B; c += 32) {
    se += expf(z[c] - mx);
    ys += y[c];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xffffffffu, se, o);
    ys += __shfl_xor_sync(0xffffffffu, ys, o);
  }
  const float lse = mx + logf(se);
  float l = 0.f;
  for (int c = lane; c < B; c += 32) {
    const float p = expf(z[c] - lse);
    dZ[(int64_t)i * B + c] = (p * ys - y[c]) * inv_n;
    l -= y[c] * (z[c] - lse);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if (lane == 0) row_loss[i] = l * inv_n;
}

// Column sums (bias gradients) in a fixed order: chunks of CS_ROWS rows, in
// each chunk 8 row lanes (rows r = lane, lane + 8, ...) summed in order and
// then the 8 lanes in order; k_colsum_fin adds the chunks in order.
constexpr int CS_ROWS = 256;
__global__ void __launch_bounds__(256)
k_colsum_part(const float* __restrict__ D, int n, int ncol, float* __restrict__ part) {
  __shared__ float red[8][33];
  const int cx = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + cx;
  const int r0 = blockIdx.y * CS_ROWS, r1 = min(n, r0 + CS_ROWS);
  float s = 0.f;
  if (c < ncol)
    for (int i = r0 + g; i < r1; i += 8) s += D[(int64_t)i * ncol + c];
  red[g][cx] = s;
  __syncthreads();
  if (g == 0 && c < ncol) {
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; q++) t += red[q][cx];
    part[(int64_t)blockIdx.y * ncol + c] = t;
  }
}
__global__ void k_colsum_fin(const float* __restrict__ part, int nchunk, int ncol,
                             float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  float s = 0.f;
  for (int q = 0; q < nchunk; q++) s += part[(int64_t)q * ncol + c];
  out[c] = s;
}

// C[M,N] = A[M,K] . B[N,K]^T (+ bias, relu) for the forward pass: 128 x 128
// tiles, 8 x 8 outputs per thread, k in steps of 8 through double-buffered
// shared memory.  Every output is the same fma chain over k in order as in
// k_gemm, so the two kernels agree bit for bit.  Needs K % 8 == 0 and
// 16-byte aligned rows (lda, ldb multiples of 4).
constexpr int TM = 128, TN = 128, TK = 8, TPAD = 4;
template <int EPI>
__global__ void __launch_bounds__(256)
k_gemm_big(const float* __restrict__ A, int lda, const float* __restrict__ Bm, int ldb,
           float* __restrict__ C, int ldc, int M, int N, int K, const float* __restrict__ bias) {
  __shared__ __align__(16) float As[2][TK][TM + TPAD];
  __shared__ __align__(16) float Bs[2][TK][TN + TPAD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  // loader: thread t brings row t/2, k-offset 4*(t%2) of both tiles
  const int lr = tid >> 1, lk = (tid & 1) * 4;
  const bool am = m0 + lr < M, bn = n0 + lr < N;
  const float* ap = A + (int64_t)(am ? m0 + lr : 0) * lda + lk;
  const float* bp = Bm + (int64_t)(bn ? n0 + lr : 0) * ldb + lk;
  float4 ra = am ? *reinterpret_cast<const float4*>(ap) : make_float4(0.f, 0.f, 0.f, 0.f);
  float4 rb = bn ? *reinterpret_cast<const float4*>(bp) : make_float4(0.f, 0.f, 0.f, 0.f);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[i][j] = 0.f;
  int buf = 0;
  As[0][lk + 0][lr] = ra.x; As[0][lk + 1][lr] = ra.y; As[0][lk + 2][lr] = ra.z; As[0][lk + 3][lr] = ra.w;
  Bs[0][lk + 0][lr] = rb.x; Bs[0][lk + 1][lr] = rb.y; Bs[0][lk + 2][lr] = rb.z; Bs[0][lk + 3][lr] = rb.w;
  __syncthreads();
  for (int k0 = 0; k0 < K; k0 += TK) {
    const bool more = k0 + TK < K;
    if (more) {
      ra = am ? *reinterpret_cast<const float4*>(ap + k0 + TK) : make_float4(0.f, 0.f, 0.f, 0.f);
      rb = bn ? *reinterpret_cast<const float4*>(bp + k0 + TK) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int kk = 0; kk < TK; kk++) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4 + 64]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4 + 64]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (more) {
      const int nb = buf ^ 1;
      As[nb][lk + 0][lr] = ra.x; As[nb][lk + 1][lr] = ra.y; As[nb][lk + 2][lr] = ra.z; As[nb][lk + 3][lr] = ra.w;
      Bs[nb][lk + 0][lr] = rb.x; Bs[nb][lk + 1][lr] = rb.y; Bs[nb][lk + 2][lr] = rb.z; Bs[nb][lk + 3][lr] = rb.w;
      __syncthreads();
      buf = nb;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const int m = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; j++) {
      const int n = n0 + tx * 4 + (j & 3) + (j >> 2) * 64;
      if (n >= N) continue;
      float v = acc[i][j];
      if (EPI == 1) {
        v = v + bias[n];
        v = v > 0.f ? v : 0.f;
      } else if (EPI == 2) {
        v = v + bias[n];
      }
      C[(int64_t)m * ldc + n] = v;
    }
  }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// argmax per row, ties to the lower index (warp per row).
__global__ void k_argmax_rows(const float* __restrict__ Z, int64_t n, int B,
                              int32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;
  const float* z = Z + i * B;
  float best = -INFINITY;
  int bi = INT_MAX;
  for (int c = lane; c < B; c += 32) {
    const float v = z[c];
    if (v > best || (v == best && c < bi)) {
      best = v;
      bi = c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int c2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (v2 > best || (v2 == best && c2 < bi)) {
      best = v2;
      bi = c2;
    }
  }
  if (lane == 0) out[i] = bi == INT_MAX ? 0 : bi;
}

__global__ void k_gather_rows_f(const float* __restrict__ X, const int64_t* __restrict__ idx,
                                int64_t n, int d, float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * d) return;
  out[t] = X[idx[t / d] * d + t % d];
}

template <bool TA, bool TB, int EPI>
int gemm(const float* A, int lda, const float* Bm, int ldb, float* C, int ldc, int M, int N, int K,
         const float* bias, const float* mask, int ldm, cudaStream_t s) {
  if (M == 0 || N == 0) return CAPS_OK;
  if (!TA && !TB && EPI != 3 && K > 0 && K % TK == 0 && lda % 4 == 0 && ldb % 4 == 0 &&
      (uintptr_t)A % 16 == 0 && (uintptr_t)Bm % 16 == 0 && M >= TM) {
    dim3 g2((unsigned)((N + TN - 1) / TN), (unsigned)((M + TM - 1) / TM));
    if (g2.y > 65535) return fail(CAPS_EINVAL, "gemm: too many rows in one call");
    k_gemm_big<EPI == 3 ? 0 : EPI><<<g2, 256, 0, s>>>(A, lda, Bm, ldb, C, ldc, M, N, K, bias);
    CAPS_LAUNCH("k_gemm_big");
    return CAPS_OK;
  }
  dim3 grid((unsigned)((N + GN - 1) / GN), (unsigned)((M + GM - 1) / GM));
  if (grid.y > 65535) return fail(CAPS_EINVAL, "gemm: too many rows in one call");
  k_gemm<TA, TB, EPI><<<grid, 256, 0, s>>>(A, lda, Bm, ldb, C, ldc, M, N, K, bias, mask, ldm);
  CAPS_LAUNCH("k_gemm");
  return CAPS_OK;
}

int colsum(const float* D, int n, int ncol, float* out, Scratch& scr, cudaStream_t s) {
  const int nchunk = std::max(1, (n + CS_ROWS - 1) / CS_ROWS);
  float* part = nullptr;
  if (int rc = scr.get(&part, (size_t)nchunk * ncol)) return rc;
  k_colsum_part<<<dim3((unsigned)((ncol + 31) / 32), (unsigned)nchunk), 256, 0, s>>>(D, n, ncol, part);
  CAPS_LAUNCH("k_colsum_part");
  k_colsum_fin<<<(unsigned)((ncol + 127) / 128), 128, 0, s>>>(part, nchunk, ncol, out);
  CAPS_LAUNCH("k_colsum_fin");
  return CAPS_OK;
}

// ---- the bf16 training step ----
// bf16 copy of fp32 [rows, cols]: out [rows, ldo], columns past cols zero
__global__ void k_to_bf16(const float* __restrict__ src, int64_t rows, int cols, int ldo,
                          __nv_bfloat16* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * ldo) return;
  const int64_t r = t / ldo;
  const int c = (int)(t % ldo);
  out[t] = __float2bfloat16_rn(c < cols ? src[r * cols + c] : 0.f);
}
// bf16 transpose of fp32 [rows, cols]: out [cols, ldo], out[c][r] = src[r][c],
// columns r >= rows zero; 32 x 32 tiles through shared memory
__global__ void __launch_bounds__(256)
k_to_bf16_t(const float* __restrict__ src, int64_t rows, int cols, int64_t ldo,
            __nv_bfloat16* __restrict__ out) {
  __shared__ float t[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    const int64_t r = r0 + ty + k;
    const int c = c0 + tx;
    t[ty + k][tx] = (r < rows && c < cols) ? src[r * cols + c] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    const int c = c0 + ty + k;
    const int64_t r = r0 + tx;
    if (c < cols && r < ldo) out[(int64_t)c * ldo + r] = __float2bfloat16_rn(t[tx][ty + k]);
  }
}
// P [n, H] <- relu(P + b) (EPI 1) or P + b (EPI 2), in place
template <int EPI>
__global__ void k_bias_rows(float* __restrict__ P, int64_t n, int H, const float* __restrict__ b) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * H) return;
  float v = P[t] + b[t % H];
  if (EPI == 1) v = v > 0.f ? v : 0.f;
  P[t] = v;
}
// D <- D where the hidden unit was on (Hd > 0), else 0
__global__ void k_relu_mask(float* __restrict__ D, const float* __restrict__ Hd, int64_t n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) D[t] = Hd[t] > 0.f ? D[t] : 0.f;
}

int to_bf16(const float* src, int64_t rows, int cols, int ldo, __nv_bfloat16* out, cudaStream_t s) {
  const int64_t tot = rows * ldo;
  if (tot == 0) return CAPS_OK;
  k_to_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(src, rows, cols, ldo, out);
  CAPS_LAUNCH("k_to_bf16");
  return CAPS_OK;
}
int to_bf16_t(const float* src, int64_t rows, int cols, int64_t ldo, __nv_bfloat16* out,
              cudaStream_t s) {
  if (cols == 0 || ldo == 0) return CAPS_OK;
  const dim3 g((unsigned)((ldo + 31) / 32), (unsigned)((cols + 31) / 32));
  if (g.y > 65535) return fail(CAPS_EINVAL, "transpose: too many columns");
  k_to_bf16_t<<<g, 256, 0, s>>>(src, rows, cols, ldo, out);
  CAPS_LAUNCH("k_to_bf16_t");
  return CAPS_OK;
}
inline int pad64(int64_t v) { return (int)((v + 63) / 64 * 64); }

}  // namespace

// logits Z [n, B] of rows X [n, d]; Hd [n, H] scratch.  Rows in chunks.
int mlp_logits(const MlpNet& net, const float* X, int64_t n, float* Hd, float* Z, cudaStream_t s) {
  const int64_t chunk = 65535LL * GM;
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int rows = (int)std::min(chunk, n - r0);
    if (int rc = gemm<false, false, 1>(X + r0 * net.d, net.d, net.W1, net.d, Hd + r0 * net.H,
                                       net.H, rows, net.H, net.d, net.b1, nullptr, 0, s))
      return rc;
    if (int rc = gemm<false, false, 2>(Hd + r0 * net.H, net.H, net.W2, net.H, Z + r0 * net.B,
                                       net.B, rows, net.B, net.H, net.b2, nullptr, 0, s))
      return rc;
  }
  return CAPS_OK;
}

// hidden layer Hd [n, H] = relu(W1 X + b1) of rows X [n, d] (rows in chunks)
int mlp_hidden(const MlpNet& net, const float* X, int64_t n, float* Hd, cudaStream_t s) {
  const int64_t chunk = 65535LL * GM;
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int rows = (int)std::min(chunk, n - r0);
    if (int rc = gemm<false, false, 1>(X + r0 * net.d, net.d, net.W1, net.d, Hd + r0 * net.H,
                                       net.H, rows, net.H, net.d, net.b1, nullptr, 0, s))
      return rc;
  }
  return CAPS_OK;
}

int mlp_assign(const MlpNet& net, const float* X, int64_t n, int32_t* bin, Scratch& scr,
               cudaStream_t s) {
  if (n == 0) return CAPS_OK;
  // rows per pass so that hidden + logits stay under ~256 MB
  const int64_t per = std::max<int64_t>(1, ((int64_t)1 << 26) / (net.H + net.B));
  const int64_t pass = std::min(n, per);
  float *Hd = nullptr, *Z = nullptr;
  if (int rc = scr.get(&Hd, (size_t)pass * net.H)) return rc;
  if (int rc = scr.get(&Z, (size_t)pass * net.B)) return rc;
  for (int64_t r0 = 0; r0 < n; r0 += pass) {
    const int64_t rows = std::min(pass, n - r0);
    if (int rc = mlp_logits(net, X + r0 * net.d, rows, Hd, Z, s)) return rc;
    k_argmax_rows<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(Z, rows, net.B, bin + r0);
    CAPS_LAUNCH("k_argmax_rows");
  }
  return CAPS_OK;
}

int mlp_loss_grad(const MlpNet& net, const float* X, int64_t n, const float* Y, MlpNet* grad,
                  float* loss_dev, Scratch& scr, cudaStream_t s) {
  if (n < 1 || n > INT_MAX) return fail(CAPS_EINVAL, "mlp: batch size out of range");
  const int d = net.d, H = net.H, B = net.B, nn = (int)n;
  float *Hd = nullptr, *Z = nullptr, *dZ = nullptr, *dH = nullptr, *rl = nullptr;
  if (int rc = scr.get(&rl, (size_t)n)) return rc;
  if (int rc = scr.get(&Hd, (size_t)n * H)) return rc;
  if (int rc = scr.get(&Z, (size_t)n * B)) return rc;
  if (int rc = scr.get(&dZ, (size_t)n * B)) return rc;
  if (int rc = scr.get(&dH, (size_t)n * H)) return rc;
  if (int rc = mlp_logits(net, X, n, Hd, Z, s)) return rc;
  k_softmax_xent<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(Z, Y, nn, B, 1.f / (float)n, dZ, rl);
  CAPS_LAUNCH("k_softmax_xent");
  // the mean loss: the rows' shares summed in a fixed order (one column)
  if (int rc = colsum(rl, nn, 1, loss_dev, scr, s)) return rc;
  // gW2 [B,H] = dZ^T [B,n] . Hd [n,H];  gb2 = column sums of dZ
  if (int rc = gemm<true, true, 0>(dZ, B, Hd, H, grad->W2, H, B, H, nn, nullptr, nullptr, 0, s))
    return rc;
  if (int rc = colsum(dZ, nn, B, grad->b2, scr, s)) return rc;
  // dH [n,H] = dZ [n,B] . W2 [B,H], zero where the hidden unit was off
  if (int rc = gemm<false, true, 3>(dZ, B, net.W2, H, dH, H, nn, H, B, nullptr, Hd, H, s)) return rc;
  // gW1 [H,d] = dH^T [H,n] . X [n,d];  gb1 = column sums of dH
  if (int rc = gemm<true, true, 0>(dH, H, X, d, grad->W1, d, H, d, nn, nullptr, nullptr, 0, s))
    return rc;
  if (int rc = colsum(dH, nn, H, grad->b1, scr, s)) return rc;
  return CAPS_OK;
}

// Every product on the tensor cores with bf16 operands and fp32
// accumulation: H = relu(X W1^T + b1), Z = bf16(H) W2^T + b2, dZ from the
// softmax, gW2 = bf16(dZ)^T bf16(H), dH = (bf16(dZ) W2) where H > 0,
// gW1 = bf16(dH)^T bf16(X); the bias gradients are fp32 column sums of dZ
// and dH.  Operands are padded with zeros to multiples of 64 along the
// contracted index.
int mlp_loss_grad_bf16(const MlpNet& net, const float* X, const void* Xb_in, int64_t n,
                       const float* Y, MlpNet* grad, float* loss_dev, int32_t* err, Scratch& scr,
                       cudaStream_t s) {
  if (n < 1 || n > INT_MAX) return fail(CAPS_EINVAL, "mlp: batch size out of range");
  using bf = __nv_bfloat16;
  const int d = net.d, H = net.H, B = net.B, nn = (int)n;
  const int dp = pad64(d), Hp = pad64(H), Bp = pad64(B), np_ = pad64(n);
  bf *W1b, *W2b, *W2bT, *Hb, *HbT, *dZb, *dZbT, *dHbT, *XbT;
  float *Hd, *Z, *dZ, *dH, *rl;
  if (int rc = scr.get(&W1b, (size_t)H * dp)) return rc;
  if (int rc = scr.get(&W2b, (size_t)B * Hp)) return rc;
  if (int rc = scr.get(&W2bT, (size_t)H * Bp)) return rc;
  if (int rc = scr.get(&Hb, (size_t)n * Hp)) return rc;
  if (int rc = scr.get(&HbT, (size_t)H * np_)) return rc;
  if (int rc = scr.get(&dZb, (size_t)n * Bp)) return rc;
  if (int rc = scr.get(&dZbT, (size_t)B * np_)) return rc;
  if (int rc = scr.get(&dHbT, (size_t)H * np_)) return rc;
  if (int rc = scr.get(&XbT, (size_t)d * np_)) return rc;
  if (int rc = scr.get(&Hd, (size_t)n * H)) return rc;
  if (int rc = scr.get(&Z, (size_t)n * B)) return rc;
  if (int rc = scr.get(&dZ, (size_t)n * B)) return rc;
  if (int rc = scr.get(&dH, (size_t)n * H)) return rc;
  if (int rc = scr.get(&rl, (size_t)n)) return rc;
  const bf* Xb = static_cast<const bf*>(Xb_in);
  if (!Xb) {
    bf* xb = nullptr;
    if (int rc = scr.get(&xb, (size_t)n * dp)) return rc;
    if (int rc = to_bf16(X, n, d, dp, xb, s)) return rc;
    Xb = xb;
  }
  // bf16 copies of the master weights, and of the rows transposed
  if (int rc = to_bf16(net.W1, H, d, dp, W1b, s)) return rc;
  if (int rc = to_bf16(net.W2, B, H, Hp, W2b, s)) return rc;
  if (int rc = to_bf16_t(net.W2, B, H, Bp, W2bT, s)) return rc;
  if (int rc = to_bf16_t(X, n, d, np_, XbT, s)) return rc;
  // forward
  if (int rc = bf16_gemm_nt(Xb, n, W1b, H, dp, Hd, err, s)) return rc;
  k_bias_rows<1><<<(unsigned)((n * H + 255) / 256), 256, 0, s>>>(Hd, n, H, net.b1);
  CAPS_LAUNCH("k_bias_rows");
  if (int rc = to_bf16(Hd, n, H, Hp, Hb, s)) return rc;
  if (int rc = to_bf16_t(Hd, n, H, np_, HbT, s)) return rc;
  if (int rc = bf16_gemm_nt(Hb, n, W2b, B, Hp, Z, err, s)) return rc;
  k_bias_rows<2><<<(unsigned)((n * B + 255) / 256), 256, 0, s>>>(Z, n, B, net.b2);
  CAPS_LAUNCH("k_bias_rows");
  k_softmax_xent<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(Z, Y, nn, B, 1.f / (float)n, dZ, rl);
  CAPS_LAUNCH("k_softmax_xent");
  if (int rc = colsum(rl, nn, 1, loss_dev, scr, s)) return rc;
  // backward
  if (int rc = to_bf16(dZ, n, B, Bp, dZb, s)) return rc;
  if (int rc = to_bf16_t(dZ, n, B, np_, dZbT, s)) return rc;
  if (int rc = bf16_gemm_nt(dZbT, B, HbT, H, np_, grad->W2, err, s)) return rc;
  if (int rc = colsum(dZ, nn, B, grad->b2, scr, s)) return rc;
  if (int rc = bf16_gemm_nt(dZb, n, W2bT, H, Bp, dH, err, s)) return rc;
  k_relu_mask<<<(unsigned)((n * H + 255) / 256), 256, 0, s>>>(dH, Hd, n * H);
  CAPS_LAUNCH("k_relu_mask");
  if (int rc = to_bf16_t(dH, n, H, np_, dHbT, s)) return rc;
  if (int rc = bf16_gemm_nt(dHbT, H, XbT, d, np_, grad->W1, err, s)) return rc;
  if (int rc = colsum(dH, nn, H, grad->b1, scr, s)) return rc;
  return CAPS_OK;
}

int mlp_adam(float* w, const float* g, float* m, float* v, int64_t n, float lr, int t,
             cudaStream_t s) {
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, t)), c2 = (float)(1.0 - std::pow(b2, t));
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, g, m, v, n, lr, (float)b1, (float)b2,
                                                     1e-8f, c1, c2);
  CAPS_LAUNCH("k_adam");
  return CAPS_OK;
}

int mlp_gather_rows(const float* X, const int64_t* idx, int64_t n, int d, float* out,
                    cudaStream_t s) {
  if (n == 0) return CAPS_OK;
  k_gather_rows_f<<<(unsigned)((n * d + 255) / 256), 256, 0, s>>>(X, idx, n, d, out);
  CAPS_LAUNCH("k_gather_rows_f");
  return CAPS_OK;
}

// Minibatches of `batch` samples in sample order, the same every epoch.
int mlp_train(MlpNet& net, const float* X, int64_t n, const float* Y, int epochs, int batch,
              float lr, float* losses_host, cudaStream_t s, bool bf16) {
  const int64_t P1 = (int64_t)net.H * net.d, P2 = (int64_t)net.B * net.H;
  const int64_t total = P1 + net.H + P2 + net.B;
  Scratch scr(s);
  float *g = nullptr, *mo = nullptr, *ve = nullptr;
  float* loss = nullptr;
  if (int rc = scr.get(&g, (size_t)total)) return rc;
  if (int rc = scr.get(&mo, (size_t)total)) return rc;
  if (int rc = scr.get(&ve, (size_t)total)) return rc;
  if (int rc = scr.get(&loss, 1)) return rc;
  // bf16 form: the rows' bf16 copy once, a flag for the tensor-core waits
  __nv_bfloat16* Xb = nullptr;
  int32_t* err = nullptr;
  const int dp = pad64(net.d);
  if (bf16) {
    if (int rc = scr.get(&Xb, (size_t)n * dp)) return rc;
    if (int rc = to_bf16(X, n, net.d, dp, Xb, s)) return rc;
    if (int rc = scr.get(&err, 1)) return rc;
    CAPS_CUDA(cudaMemsetAsync(err, 0, sizeof(int32_t), s));
  }
  CAPS_CUDA(cudaMemsetAsync(mo, 0, sizeof(float) * total, s));
  CAPS_CUDA(cudaMemsetAsync(ve, 0, sizeof(float) * total, s));
  MlpNet gr = net;
  gr.W1 = g;
  gr.b1 = g + P1;
  gr.W2 = g + P1 + net.H;
  gr.b2 = g + P1 + net.H + P2;
  float* w = net.W1;  // W1|b1|W2|b2 are one contiguous block
  int t = 0;
  for (int e = 0; e < epochs; e++) {
    for (int64_t b0 = 0; b0 < n; b0 += batch) {
      const int64_t nb = std::min<int64_t>(batch, n - b0);
      Scratch step(s);
      if (bf16) {
        if (int rc = mlp_loss_grad_bf16(net, X + b0 * net.d, Xb + b0 * dp, nb, Y + b0 * net.B,
                                        &gr, loss, err, step, s))
          return rc;
      } else if (int rc = mlp_loss_grad(net, X + b0 * net.d, nb, Y + b0 * net.B, &gr, loss, step,
                                        s)) {
        return rc;
      }
      t++;
      if (int rc = mlp_adam(w, g, mo, ve, total, lr, t, s)) return rc;
      if (losses_host) {
        CAPS_CUDA(cudaMemcpyAsync(&losses_host[t - 1], loss, sizeof(float),
                                  cudaMemcpyDeviceToHost, s));
        CAPS_CUDA(cudaStreamSynchronize(s));
      }
    }
  }
  if (bf16) {
    int32_t he = 0;
    CAPS_CUDA(cudaMemcpyAsync(&he, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CAPS_CUDA(cudaStreamSynchronize(s));
    if (he) return fail(CAPS_ETIMEOUT, "a bounded device wait expired in the bf16 training");
  }
  return CAPS_OK;
}


namespace {
// Greedy balanced assignment (one thread, in id order): point i goes to the
// least-loaded of its R candidates top[i*R..] (best first, ties to the
// earlier), loads in shared memory starting at load0 (or zero).
__global__ void __launch_bounds__(32)
k_balanced_assign(const int32_t* __restrict__ top, int64_t n, int R, int B,
                  const int64_t* __restrict__ load0, int32_t* __restrict__ bins) {
  extern __shared__ long long load[];
  for (int b = threadIdx.x; b < B; b += 32) load[b] = load0 ? load0[b] : 0;
  __syncwarp();
  if (threadIdx.x != 0) return;
  for (int64_t i = 0; i < n; i++) {
    const int32_t* t = top + i * R;
    int32_t best = t[0];
    long long lb = load[best];
    for (int r = 1; r < R; r++) {
      const int32_t c = t[r];
      const long long lc = load[c];
      if (lc < lb) {
        best = c;
        lb = lc;
      }
    }
    bins[i] = best;
    load[best] = lb + 1;
  }
}
}  // namespace

int mlp_balanced_assign(const MlpNet& net, const float* X, int64_t n, int R, const int64_t* load0,
                        int32_t* bin, Scratch& scr, cudaStream_t s) {
  if (n == 0) return CAPS_OK;
  if (R < 1 || R > 64 || R > net.B) return fail(CAPS_EINVAL, "balance R must be in [1, min(64, B)]");
  if ((size_t)net.B * sizeof(long long) > 200 * 1024)
    return fail(CAPS_EINVAL, "balanced assignment needs B <= 25600");
  // each point's R largest logits (ties to the lower partition), in passes
  const int64_t per = std::max<int64_t>(1, ((int64_t)1 << 26) / (net.H + net.B));
  const int64_t pass = std::min(n, per);
  float *Hd = nullptr, *Z = nullptr;
  int32_t* top = nullptr;
  if (int rc = scr.get(&Hd, (size_t)pass * net.H)) return rc;
  if (int rc = scr.get(&Z, (size_t)pass * net.B)) return rc;
  if (int rc = scr.get(&top, (size_t)n * R)) return rc;
  for (int64_t r0 = 0; r0 < n; r0 += pass) {
    const int64_t rows = std::min(pass, n - r0);
    if (int rc = mlp_logits(net, X + r0 * net.d, rows, Hd, Z, s)) return rc;
    if (int rc = launch_topm(Z, rows, net.B, R, CAPS_IP, top + r0 * R, s)) return rc;
  }
  const size_t smem = sizeof(long long) * (size_t)net.B;
  if (smem > 48 * 1024)
    CAPS_CUDA(cudaFuncSetAttribute(k_balanced_assign, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
  k_balanced_assign<<<1, 32, smem, s>>>(top, n, R, net.B, load0, bin);
  CAPS_LAUNCH("k_balanced_assign");
  return CAPS_OK;
}

}  // namespace caps
