// Batched Householder QR with a non-negative diagonal of R (thin Q only).
//
// The variational fit of App. B (arXiv:1908.09359) moves the orthogonality
// centre of the truncated MPS with a QR of every optimal site tensor; the
// random starting guess is made right-orthonormal the same way.  Choosing the
// sign of each column so that diag(R) >= 0 makes Q unique for full-rank input,
// so the truncated MPS does not depend on the QR routine used.
//
// One CTA per matrix; the matrix and the growing Q live in shared memory in
// column-major order.  Reflector j: v = x + sign(x0)|x| e1, beta = 2/(v.v);
// a zero column gets no reflector and a zero diagonal.
#include "common.cuh"

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

}  // namespace

cudaError_t qr_pos_batched(const float* Y, long long bsY, long long yrs, long long ycs, float* Q,
                           long long bsQ, long long qrs, long long qcs, int rows, int cols, int batch,
                           cudaStream_t st) {
  if (g_dry_run || batch <= 0) return cudaSuccess;
  if (cols > kQrMaxCols || rows < cols || cols <= 0) return cudaErrorInvalidValue;
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
