// Batched Householder QR with a non-negative diagonal of R (thin Q only).
//
// The variational fit of App. B (arXiv:1908.09359) moves the orthogonality
// centre of the truncated MPS with a QR of every optimal site tensor; the
// random starting guess is made right-orthonormal the same way.  Choosing the
// sign of each column so that diag(R) >= 0 makes Q unique for full-rank input,
// so the truncated MPS does not depend on the QR routine used.
//
// One CTA per matrix.  General form: the matrix and the growing Q live in shared
// memory in column-major order; for rows <= 256, cols <= 32 a register-resident form
// (below) is used instead.  Reflector j: v = x + sign(x0)|x| e1, beta = 2/(v.v);
// a zero column gets no reflector and a zero diagonal.
#include "common.cuh"
#include "pepsvmc.h"

namespace pv {
namespace {

constexpr int kQrThreads = 256;
constexpr int kQrMaxCols = 64;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kQrThreads) qr_pos_kernel(const float* __restrict__ Y, long long bsY,
                                                            long long yrs, long long ycs, float* __restrict__ Q,
                                                            long long bsQ, long long qrs, long long qcs, int R,
                                                            int C) {
  extern __shared__ float sm[];
  float* A = sm;           // A[j*R + i]
  float* Qs = sm + R * C;  // Qs[j*R + i]
  __shared__ float beta[kQrMaxCols];
  __shared__ int flip[kQrMaxCols];
  __shared__ float red[kQrThreads / 32];

  const int b = blockIdx.x;
  const float* Yb = Y + (long long)b * bsY;
  for (int idx = threadIdx.x; idx < R * C; idx += blockDim.x) {
    const int i = idx % R, j = idx / R;
    A[idx] = Yb[(long long)i * yrs + (long long)j * ycs];
    Qs[idx] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < C; ++j) {
    float* a = A + j * R;
    float s = 0.f;
    for (int i = j + threadIdx.x; i < R; i += blockDim.x) s = fmaf(a[i], a[i], s);
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      float tot = 0.f;
      for (int w = 0; w < nw; ++w) tot += red[w];
      const float alpha = sqrtf(tot);
      const float x0 = a[j];
      if (alpha == 0.f) {
        beta[j] = 0.f;
        flip[j] = 0;
      } else {
        const float sg = (x0 >= 0.f) ? 1.f : -1.f;
        a[j] = x0 + sg * alpha;
        beta[j] = 1.f / (alpha * (alpha + fabsf(x0)));
        flip[j] = (sg > 0.f) ? 1 : 0;  // R_jj = -sign(x0)|x| < 0 -> negate column j of Q
      }
    }
    __syncthreads();
    const float bj = beta[j];
    if (bj != 0.f) {
      for (int jj = j + 1 + warp; jj < C; jj += nw) {
        float* c = A + jj * R;
        float w = 0.f;
        for (int i = j + lane; i < R; i += 32) w = fmaf(a[i], c[i], w);
        w = warp_sum(w) * bj;
        for (int i = j + lane; i < R; i += 32) c[i] = fmaf(-w, a[i], c[i]);
      }
    }
    __syncthreads();
  }
  for (int j = C - 1; j >= 0; --j) {
    const float bj = beta[j];
    if (bj == 0.f) continue;
    const float* a = A + j * R;
    for (int jj = j + warp; jj < C; jj += nw) {
      float* q = Qs + jj * R;
      float w = 0.f;
      for (int i = j + lane; i < R; i += 32) w = fmaf(a[i], q[i], w);
      w = warp_sum(w) * bj;
      for (int i = j + lane; i < R; i += 32) q[i] = fmaf(-w, a[i], q[i]);
    }
    __syncthreads();
  }
  float* Qb = Q + (long long)b * bsQ;
  for (int idx = threadIdx.x; idx < R * C; idx += blockDim.x) {
    const int i = idx % R, j = idx / R;
    const float v = Qs[idx];
    Qb[(long long)i * qrs + (long long)j * qcs] = flip[j] ? -v : v;
  }
}

// Register-resident form for rows <= 256, cols <= 32 (every bulk shape of D <= 8,
// Dc <= 32), in blocks of 64, 128 or 256 threads (the smallest that covers the rows):
// thread t holds row t of the matrix and of Q in registers, so a reflector
// costs two block reductions instead of a pass over shared memory per column.  The
// 32-wide reductions (w = v^T A over the remaining columns) run as a transposing warp
// butterfly (31 shuffles leave column l's warp sum in lane l), then across the eight
// warps through shared memory.  Same reflectors, signs and zero-column rule as above.
constexpr int kQrRegCols = 32;

__device__ __forceinline__ float warp_transpose_sum32(float (&p)[kQrRegCols]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float send = up ? p[i] : p[i + w];
      const float keep = up ? p[i + w] : p[i];
      p[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return p[0];
}

// Sum over the block (NT threads) of p[k] for every k: returns, in lane l of every warp,
// the block sum of column l (the eight warp sums added in warp order, so every warp
// holds the same value); red: NT/32 x 32 floats, written before and read after the one
// barrier.  Consecutive calls must alternate between two red buffers (a warp may still
// be reading one when another warp writes the next).
template <int NT>
__device__ __forceinline__ float block_sum32(float (&p)[kQrRegCols], float* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float v = warp_transpose_sum32(p);
  red[warp * 32 + lane] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) s += red[w * 32 + lane];
  return s;
}

// Y and Q may be the same array (in-place QR): every row is read before any is written.
// NT threads (64, 128 or 256) hold up to NT rows.  One barrier per block reduction: the
// partial sums are written before it and every thread forms the total after it (in the
// same order, so all agree bit for bit).  The partials go to two alternating buffers --
// by the parity of j in the factorisation, where every column passes the norm's barrier,
// and per reduction done in the Q accumulation, where a zero column has none -- so a
// buffer is rewritten only after a barrier that follows every read of it.
template <int NT>
__global__ void __launch_bounds__(NT) qr_pos_reg_kernel(const float* Y, long long bsY, long long yrs,
                                                                long long ycs, float* Q, long long bsQ,
                                                                long long qrs, long long qcs, int R, int C) {
  __shared__ float red[2][NT];
  __shared__ float redn[2][NT / 32];
  __shared__ float beta[kQrRegCols];
  __shared__ int flip[kQrRegCols];
  __shared__ float x0s[2];  // x0 by parity of j: a zero column skips the dot products' barrier
  const int t = threadIdx.x;
  const int lane = t & 31, warp = t >> 5;
  const float* Yb = Y + (long long)blockIdx.x * bsY;
  float a[kQrRegCols], q[kQrRegCols], p[kQrRegCols];
#pragma unroll
  for (int k = 0; k < kQrRegCols; ++k) {
    a[k] = (t < R && k < C) ? Yb[(long long)t * yrs + (long long)k * ycs] : 0.f;
    q[k] = (t == k) ? 1.f : 0.f;
  }
  // factorisation: reflector j from column j, rows >= j; v overwrites a[j] of rows >= j
#pragma unroll
  for (int j = 0; j < kQrRegCols; ++j) {
    if (j >= C) break;
    float s = (t >= j) ? a[j] * a[j] : 0.f;
    s = warp_sum(s);
    if (lane == 0) redn[j & 1][warp] = s;
    if (t == j) x0s[j & 1] = a[j];
    __syncthreads();
    float n2 = 0.f;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) n2 += redn[j & 1][w];
    const float alpha = sqrtf(n2), x0 = x0s[j & 1];
    const float sg = (x0 >= 0.f) ? 1.f : -1.f;
    const float bj = alpha == 0.f ? 0.f : 1.f / (alpha * (alpha + fabsf(x0)));
    if (t == 0) {
      beta[j] = bj;
      flip[j] = (alpha != 0.f && sg > 0.f) ? 1 : 0;  // R_jj = -sign(x0)|x| < 0 -> negate column j of Q
    }
    if (bj == 0.f) continue;  // uniform over the block: zero column, no reflector
    if (t == j) a[j] = x0 + sg * alpha;
    const float v = (t >= j) ? a[j] : 0.f;
#pragma unroll
    for (int k = 0; k < kQrRegCols; ++k) p[k] = (k > j) ? v * a[k] : 0.f;
    const float c = -bj * block_sum32<NT>(p, red[j & 1]);  // lane l: -beta w_l
#pragma unroll
    for (int k = 0; k < kQrRegCols; ++k)
      if (k > j) a[k] = fmaf(__shfl_sync(0xffffffffu, c, k), v, a[k]);
  }
  __syncthreads();
  // thin Q = H_0 ... H_{C-1} [I; 0], accumulated backwards; H_j touches rows >= j and,
  // at that point, only columns >= j of Q
  int par = 0;  // alternates per reduction done (a skipped reflector has no barrier)
#pragma unroll
  for (int j = kQrRegCols - 1; j >= 0; --j) {
    if (j >= C) continue;
    const float bj = beta[j];
    if (bj == 0.f) continue;
    const float v = (t >= j) ? a[j] : 0.f;
#pragma unroll
    for (int k = 0; k < kQrRegCols; ++k) p[k] = (k >= j) ? v * q[k] : 0.f;
    const float c = -bj * block_sum32<NT>(p, red[par]);
    par ^= 1;
#pragma unroll
    for (int k = 0; k < kQrRegCols; ++k)
      if (k >= j) q[k] = fmaf(__shfl_sync(0xffffffffu, c, k), v, q[k]);
  }
  if (t < R) {
    float* Qb = Q + (long long)blockIdx.x * bsQ;
#pragma unroll
    for (int k = 0; k < kQrRegCols; ++k)
      if (k < C) Qb[(long long)t * qrs + (long long)k * qcs] = flip[k] ? -q[k] : q[k];
  }
}

}  // namespace

cudaError_t qr_pos_batched(const float* Y, long long bsY, long long yrs, long long ycs, float* Q,
                           long long bsQ, long long qrs, long long qcs, int rows, int cols, int batch,
                           cudaStream_t st) {
  if (g_dry_run || batch <= 0) return cudaSuccess;
  if (cols > kQrMaxCols || rows < cols || cols <= 0) return cudaErrorInvalidValue;
  if (rows <= 256 && cols <= kQrRegCols) {
    if (rows <= 64)
      qr_pos_reg_kernel<64><<<batch, 64, 0, st>>>(Y, bsY, yrs, ycs, Q, bsQ, qrs, qcs, rows, cols);
    else if (rows <= 128)
      qr_pos_reg_kernel<128><<<batch, 128, 0, st>>>(Y, bsY, yrs, ycs, Q, bsQ, qrs, qcs, rows, cols);
    else
      qr_pos_reg_kernel<256><<<batch, 256, 0, st>>>(Y, bsY, yrs, ycs, Q, bsQ, qrs, qcs, rows, cols);
    return cudaGetLastError();
  }
  const size_t smem = (size_t)2 * rows * cols * sizeof(float);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    PV_CUDA(cudaFuncSetAttribute(qr_pos_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    configured = smem;
  }
  qr_pos_kernel<<<batch, kQrThreads, smem, st>>>(Y, bsY, yrs, ycs, Q, bsQ, qrs, qcs, rows, cols);
  return cudaGetLastError();
}

}  // namespace pv

extern "C" int pepsvmc_qr_pos(const float* Y, float* Q, int32_t batch, int32_t rows, int32_t cols, int32_t col_major,
                              void* stream) {
  if (!Y || !Q || batch < 1 || cols < 1 || cols > 64 || rows < cols) return PEPSVMC_EINVAL;
  const long long bs = (long long)rows * cols;
  const long long rs = col_major ? 1 : cols, cs = col_major ? rows : 1;
  const cudaError_t e =
      pv::qr_pos_batched(Y, bs, rs, cs, Q, bs, rs, cs, rows, cols, batch, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? PEPSVMC_OK : PEPSVMC_ECUDA;
}
