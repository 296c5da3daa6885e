// Batched tensor-contraction kernel on the 5th-generation tensor cores (sm_103a).
//
// Same interface as the FP32 kernel (GemmDesc: strided A/B, per-chain spin-selected
// site tensor, scattered C), so every contraction of the boundary-MPS method (App. B)
// and of the three- and four-line environments (App. C) can run here.  Operands are
// read from global memory as float32, rounded to BF16 (kind::f16) or kept as TF32
// (kind::tf32), and staged into shared memory in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices; K-adjacent core matrices 128 B apart,
// row-group-adjacent ones 1024 B apart).  One thread issues tcgen05.mma into an FP32
// accumulator in tensor memory; completion is tracked with tcgen05.commit on an
// mbarrier (two shared-memory stages, so loading stage k+1 overlaps the MMAs of stage
// k).  The epilogue reads the accumulator with tcgen05.ld and scatters it like the
// FP32 kernel.  Every mbarrier wait has a clock budget; on expiry the CTA raises
// ST_TIMEOUT, drains, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_util.cuh"

namespace pv {
namespace {

using namespace tc;

constexpr int kBM = 128;       // rows per tile = MMA M
constexpr int kKBytes = 128;   // bytes of K per stage (64 BF16 or 32 TF32)
constexpr int kThreads = 256;  // 8 warps; warps w and w+4 share TMEM lane quarter w%4 in the epilogue

// Fill one operand tile (rows x kKBytes) of stage memory, K-major core-matrix layout:
// core matrix (r/8, kc) at ((r/8) * KC + kc) * 128 bytes, row r%8 at +16 (r%8).
// Every thread first issues all of its global loads (16-byte loads where the operand
// is K-contiguous, or row-contiguous with 4 rows per load), then converts and stores.
// K-contiguous units are assigned so that eight consecutive lanes fill the eight rows
// of one core matrix: a warp's 16-byte shared stores cover whole 128-byte core
// matrices (no bank conflicts).
template <int EB, int ROWS, bool X3>
__device__ __forceinline__ void load_tile(uint8_t* tile, const float* base, long long s_row, long long s_k, int row0,
                                          int nrows, int k0, int K, int lo_off) {
  constexpr int CE = 16 / EB;
  constexpr int KC = kKBytes / 16;  // core columns per stage
  if (s_k == 1) {
    constexpr int U = ROWS * KC / kThreads;
    float f[U][CE];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int u = threadIdx.x + j * kThreads;
      const int kc = (u >> 3) % KC, r = ((u >> 3) / KC) * 8 + (u & 7);
      const int row = row0 + r, k = k0 + kc * CE;
      const float* src = base + (long long)row * s_row + k;
      if (row < nrows && k + CE <= K && aligned16(src)) {
#pragma unroll
        for (int i = 0; i < CE; i += 4) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(src + i));
          f[j][i] = v.x; f[j][i + 1] = v.y; f[j][i + 2] = v.z; f[j][i + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < CE; ++i) f[j][i] = (row < nrows && k + i < K) ? src[i] : 0.f;
      }
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int u = threadIdx.x + j * kThreads;
      const int kc = (u >> 3) % KC, r = ((u >> 3) / KC) * 8 + (u & 7);
      put16<EB, X3>(tile + ((r >> 3) * KC + kc) * 128 + (r & 7) * 16, f[j], lo_off);
    }
  } else if (s_row == 1 && (s_k & 3) == 0) {
    constexpr int U = (ROWS / 4) * KC / kThreads > 0 ? (ROWS / 4) * KC / kThreads : 1;
    float f[U][4][CE];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int u = threadIdx.x + j * kThreads;
      if (u >= (ROWS / 4) * KC) break;
      const int r4 = u % (ROWS / 4), kc = u / (ROWS / 4);
      const int r = r4 * 4, row = row0 + r, k = k0 + kc * CE;
      const float* src = base + row + (long long)k * s_k;
      if (row + 4 <= nrows && k + CE <= K && aligned16(src)) {
#pragma unroll
        for (int i = 0; i < CE; ++i) {
          const float4 v = __ldg(reinterpret_cast<const float4*>(src + (long long)i * s_k));
          f[j][0][i] = v.x; f[j][1][i] = v.y; f[j][2][i] = v.z; f[j][3][i] = v.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < CE; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            f[j][q][i] = (row + q < nrows && k + i < K) ? src[q + (long long)i * s_k] : 0.f;
      }
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const int u = threadIdx.x + j * kThreads;
      if (u >= (ROWS / 4) * KC) break;
      const int r = (u % (ROWS / 4)) * 4, kc = u / (ROWS / 4);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        put16<EB, X3>(tile + (((r + q) >> 3) * KC + kc) * 128 + ((r + q) & 7) * 16, f[j][q], lo_off);
    }
  } else {
    for (int u = threadIdx.x; u < ROWS * KC; u += kThreads) {
      int r, kc;
      if (s_row == 1) { r = u % ROWS; kc = u / ROWS; } else { kc = u % KC; r = u / KC; }
      const int row = row0 + r, k = k0 + kc * CE;
      const float* src = base + (long long)row * s_row + (long long)k * s_k;
      float f[CE];
#pragma unroll
      for (int i = 0; i < CE; ++i) f[i] = (row < nrows && k + i < K) ? src[(long long)i * s_k] : 0.f;
      put16<EB, X3>(tile + ((r >> 3) * KC + kc) * 128 + (r & 7) * 16, f, lo_off);
    }
  }
}

// X3: split BF16 operands, x = hi + lo, and D += A_hi B_hi + A_hi B_lo + A_lo B_hi (the
// lo*lo term, ~2^-18 relative, is dropped): close to FP32 accuracy at BF16 cost.  One
// shared-memory stage holds [A_hi | B_hi | A_lo | B_lo]; plain modes double-buffer, and
// so does the split mode with DB (twice the shared memory, so fewer resident blocks:
// a candidate for long-K products, where loading stage k+1 then overlaps the MMAs of k).
template <int EB, int BN, bool X3, bool DB = false>
__global__ void __launch_bounds__(kThreads) gemm_tc_kernel(const GemmDesc d, unsigned* status) {
  constexpr int BK = kKBytes / EB;   // K elements per stage
  constexpr int MMA_K = 32 / EB;     // K elements per tcgen05.mma (32 bytes)
  constexpr int A_BYTES = kBM * kKBytes, B_BYTES = BN * kKBytes;
  constexpr int STAGES = (X3 && !DB) ? 1 : 2;
  constexpr int STAGE_BYTES = (X3 ? 2 : 1) * (A_BYTES + B_BYTES);
  constexpr uint32_t TCOLS = BN < 32 ? 32 : BN;
  extern __shared__ __align__(1024) uint8_t smem[];
  // stage s: A tile at s * (A_BYTES + B_BYTES), B tile right after it
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base;
  __shared__ long long s_on[BN];  // C offset of each tile column (the same for every row)

  const int b = blockIdx.y + blockIdx.z * gridDim.y;
  if (b >= d.batch) return;
  const int tiles_n = (d.N + BN - 1) / BN;
  const int m0 = (blockIdx.x / tiles_n) * kBM;
  const int n0 = (blockIdx.x % tiles_n) * BN;
  const float* A = d.A + (long long)b * d.bsA;
  long long boff = (long long)b * d.bsB;
  if (d.sel) boff += (long long)(((d.sel[(long long)b * d.sel_stride] < 0) ? 1 : 0) ^ d.sel_xor) * d.ssB;
  const float* B = d.B + boff;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = threadIdx.x; c < BN; c += kThreads) {
    const int n = n0 + c, cn23 = d.cn2 * d.cn3;
    s_on[c] = n < d.N ? (long long)(n / cn23) * d.sCn1 + (long long)((n / d.cn3) % d.cn2) * d.sCn2 +
                            (long long)(n % d.cn3) * d.sCn3
                      : 0;
  }

  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base;
  const uint32_t id = idesc<EB>(kBM, BN);

  const int nk = (d.K + BK - 1) / BK;
  const long long budget = d.wait_cycles > 0 ? d.wait_cycles : kDefaultWaitCycles;
  // draining after a timeout waits at least the default budget for the MMAs in flight
  const long long drain = budget > kDefaultWaitCycles ? budget : kDefaultWaitCycles;
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  for (int kt = 0; kt < nk && ok; ++kt) {
    const int s = kt % STAGES;
    if (kt >= STAGES) {
      const bool w = wait_parity(&bar[s], phase[s], budget);
      phase[s] ^= 1u;
      ok = !__syncthreads_or(!w);
      if (!ok) break;
    }
    uint8_t* As = smem + s * STAGE_BYTES;
    uint8_t* Bs = As + A_BYTES;
    constexpr int LO = A_BYTES + B_BYTES;  // offset of the lo copies (X3 only)
    load_tile<EB, kBM, X3>(As, A, d.sAm, d.sAk, m0, d.M, kt * BK, d.K, LO);
    load_tile<EB, BN, X3>(Bs, B, d.sBn, d.sBk, n0, d.N, kt * BK, d.K, LO);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_after_sync();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      const int kleft = d.K - kt * BK;
      const int nmma = kleft >= BK ? BK / MMA_K : (kleft + MMA_K - 1) / MMA_K;
      for (int i = 0; i < nmma; ++i) {
        // one MMA consumes two K core columns (32 bytes of K)
        const uint64_t ad = sdesc(a0 + i * 256, 128, (kKBytes / 16) * 128);
        const uint64_t bd = sdesc(b0 + i * 256, 128, (kKBytes / 16) * 128);
        mma<EB>(tmem, ad, bd, id, (kt > 0 || i > 0) ? 1u : 0u);
        if constexpr (X3) {
          mma<EB>(tmem, ad, sdesc(b0 + LO + i * 256, 128, (kKBytes / 16) * 128), id, 1u);
          mma<EB>(tmem, sdesc(a0 + LO + i * 256, 128, (kKBytes / 16) * 128), bd, id, 1u);
        }
      }
      commit(&bar[s]);
    }
  }
  if (ok && nk > 0) {
    const int s = (nk - 1) % STAGES;
    ok = !__syncthreads_or(!wait_parity(&bar[s], phase[s], budget));
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
    // drain whatever is still in flight before giving the tensor memory back
    if (nk > 0) wait_parity(&bar[(nk - 1) % STAGES], phase[(nk - 1) % STAGES], drain);
  } else if (nk > 0) {
    tc_after_sync();
    float alpha = d.alpha;
    if (d.inv_scale) alpha = (float)((double)alpha / d.inv_scale[b]);
    float* C = d.C + (long long)b * d.bsC;
    const int quarter = warp & 3, half = warp >> 2;
    const int m = m0 + quarter * 32 + lane;
    const int cm23 = d.cm2 * d.cm3, cn23 = d.cn2 * d.cn3;
    const long long om = (long long)(m / cm23) * d.sCm1 + (long long)((m / d.cm3) % d.cm2) * d.sCm2 +
                         (long long)(m % d.cm3) * d.sCm3;
    // innermost non-trivial part of n: contiguous in C with a run length that is a multiple of 4?
    const int run = d.cn3 > 1 ? d.cn3 : (d.cn2 > 1 ? d.cn2 : d.N);
    const long long srun = d.cn3 > 1 ? d.sCn3 : (d.cn2 > 1 ? d.sCn2 : d.sCn1);
    const bool vec = (srun == 1) && (run % 4 == 0) && !d.accumulate;
    // Outputs whose contiguous index is the OUTER part of n (n = n1 * cn23 + inner, stride
    // of n1 = 1): gather the e1 columns of one inner value from tensor memory and store
    // them as one contiguous run.
    const int e1 = cn23 > 1 ? d.N / cn23 : 0;
    const bool outer_run = d.N <= BN && cn23 > 1 && d.N % cn23 == 0 && d.sCn1 == 1 && e1 >= 4 && e1 <= 16 &&
                           (e1 & 3) == 0 && !d.accumulate;
    if (outer_run) {
      for (int i = half; i < cn23; i += 2) {
        float v[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1)
          if (n1 < e1) tmem_ld1_nowait(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(n1 * cn23 + i), v[n1]);
        tmem_wait_ld();
        if (m < d.M) {
          const long long oi = (long long)((i / d.cn3) % d.cn2) * d.sCn2 + (long long)(i % d.cn3) * d.sCn3;
          float* dst = C + om + oi;
          if (aligned16(dst)) {
#pragma unroll
            for (int n1 = 0; n1 < 16; n1 += 4)
              if (n1 < e1)
                *reinterpret_cast<float4*>(dst + n1) =
                    make_float4(alpha * v[n1], alpha * v[n1 + 1], alpha * v[n1 + 2], alpha * v[n1 + 3]);
          } else {
#pragma unroll
            for (int n1 = 0; n1 < 16; ++n1)
              if (n1 < e1) dst[n1] = alpha * v[n1];
          }
        }
      }
    }
    constexpr int HALF = BN >= 32 ? BN / 2 : 16;
    for (int c0 = half * HALF; !outer_run && c0 < (half + 1) * HALF && c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
      if (m < d.M) {
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const int n = n0 + c0 + j;
          const long long on = s_on[c0 + j];
          float* dst = C + om + on;
          if (vec && n + 4 <= d.N && aligned16(dst)) {
            *reinterpret_cast<float4*>(dst) =
                make_float4(alpha * v[j], alpha * v[j + 1], alpha * v[j + 2], alpha * v[j + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int nq = n + q;
              if (nq < d.N) {
                const long long oq = s_on[c0 + j + q];
                if (d.accumulate) C[om + oq] += alpha * v[j + q]; else C[om + oq] = alpha * v[j + q];
              }
            }
          }
        }
      }
    }
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

template <int EB, int BN, bool X3, bool DB = false>
cudaError_t launch(const GemmDesc& d, unsigned* status, cudaStream_t st) {
  // two plain stages, one split stage, or two split stages (DB)
  constexpr int smem = (DB ? 4 : 2) * (kBM + BN) * kKBytes;
  static bool configured = false;
  if (!configured) {
    PV_CUDA(cudaFuncSetAttribute(gemm_tc_kernel<EB, BN, X3, DB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem));
    configured = true;
  }
  const int tiles = ((d.M + kBM - 1) / kBM) * ((d.N + BN - 1) / BN);
  dim3 grid(tiles, d.batch < 65535 ? d.batch : 65535, (d.batch + 65534) / 65535);
  gemm_tc_kernel<EB, BN, X3, DB><<<grid, kThreads, smem, st>>>(d, status);
  return cudaGetLastError();
}

template <int EB, bool X3>
cudaError_t launch_bn(const GemmDesc& d, int bn, unsigned* status, cudaStream_t st) {
  if (bn <= 0) bn = d.N <= 32 ? 32 : d.N <= 64 ? 64 : d.N <= 128 ? 128 : 256;
  switch (bn) {
    case 32: return launch<EB, 32, X3>(d, status, st);
    case 64: return launch<EB, 64, X3>(d, status, st);
    case 128: return launch<EB, 128, X3>(d, status, st);
    default: return launch<EB, 256, X3>(d, status, st);
  }
}

}  // namespace

// Shared memory per CTA is 2 x (128 + BN) rows x 128 B, i.e. 40/48/64/96 KB for
// BN = 32/64/128/256, so at most 5/4/3/2 CTAs share an SM and their tensor memory
// (BN columns each) never exceeds the SM's 512 columns: allocation never waits.  The
// double-buffered split mode (BN = 32/64 only) takes 80/96 KB: at most 2 CTAs per SM.
// mode: 2 = BF16, 3 = split BF16 (hi + lo), 4 = TF32, 6 = split BF16 double-buffered.
// bn: tile width 32/64/128/256, or 0 for the smallest that covers N.
cudaError_t gemm_tc(const GemmDesc& d, int mode, int bn, unsigned* status, cudaStream_t st) {
  if (g_dry_run || d.M <= 0 || d.N <= 0 || d.batch <= 0) return cudaSuccess;
  if (bn != 0 && bn != 32 && bn != 64 && bn != 128 && bn != 256) return cudaErrorInvalidValue;
  if (mode == 6) {
    if (bn == 0) bn = d.N <= 32 ? 32 : 64;
    if (bn == 32) return launch<2, 32, true, true>(d, status, st);
    if (bn == 64) return launch<2, 64, true, true>(d, status, st);
    return cudaErrorInvalidValue;
  }
  if (mode == 2) return launch_bn<2, false>(d, bn, status, st);
  if (mode == 3) return launch_bn<2, true>(d, bn, status, st);
  return launch_bn<4, false>(d, bn, status, st);
}

}  // namespace pv
