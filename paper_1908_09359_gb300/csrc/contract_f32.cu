// FP32 batched tensor-contraction kernel (CUDA cores).
//
// Every contraction of the boundary-MPS method (App. B of arXiv:1908.09359:
// MPO x MPS fit steps, three-line and four-line environments of App. C, the
// defect network Delta of Eq. (7)) is written by the engine as a chain of
// batched matrix products over the Markov chains.  The kernel reads A and B
// through arbitrary (m,k)/(k,n) strides, selects the site tensor A_k^{s_k} per
// chain from the spin array (slot = sigma < 0), and scatters C into the layout
// the next stage wants (up to three nested indices on each of m and n), so no
// separate transpose kernels are needed.
#include "common.cuh"

namespace pv {
namespace {

template <int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(256) gemm_f32_kernel(const GemmDesc d) {
  constexpr int TX = BN / TN;
  constexpr int TY = BM / TM;
  static_assert(TX * TY == 256, "256 threads per tile");
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  __shared__ long long s_on[BN];  // C offset of each tile column (the same for every row)

  const int b = blockIdx.y + blockIdx.z * gridDim.y;
  if (b >= d.batch) return;
  const int tiles_n = (d.N + BN - 1) / BN;
  const int m0 = (blockIdx.x / tiles_n) * BM;
  const int n0 = (blockIdx.x % tiles_n) * BN;

  const float* __restrict__ A = d.A + (long long)b * d.bsA;
  long long boff = (long long)b * d.bsB;
  if (d.sel) boff += (long long)(((d.sel[(long long)b * d.sel_stride] < 0) ? 1 : 0) ^ d.sel_xor) * d.ssB;
  const float* __restrict__ B = d.B + boff;

  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  for (int c = t; c < BN; c += 256) {
    const int n = n0 + c, cn23 = d.cn2 * d.cn3;
    s_on[c] = n < d.N ? (long long)(n / cn23) * d.sCn1 + (long long)((n / d.cn3) % d.cn2) * d.sCn2 +
                            (long long)(n % d.cn3) * d.sCn3
                      : 0;
  }
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  const bool a_m_fast = (d.sAm == 1);
  const bool b_n_fast = (d.sBn == 1);
  for (int k0 = 0; k0 < d.K; k0 += BK) {
    for (int i = t; i < BM * BK; i += 256) {
      int mm, kk;
      if (a_m_fast) { mm = i % BM; kk = i / BM; } else { kk = i % BK; mm = i / BK; }
      const int m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < d.M && k < d.K) ? A[(long long)m * d.sAm + (long long)k * d.sAk] : 0.f;
    }
    for (int i = t; i < BN * BK; i += 256) {
      int nn, kk;
      if (b_n_fast) { nn = i % BN; kk = i / BN; } else { kk = i % BK; nn = i / BK; }
      const int n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < d.N && k < d.K) ? B[(long long)k * d.sBk + (long long)n * d.sBn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], bb[TN];
      if constexpr (TM % 4 == 0) {
#pragma unroll
        for (int i = 0; i < TM; i += 4) {
          const float4 v = *reinterpret_cast<const float4*>(&As[kk][ty * TM + i]);
          a[i] = v.x; a[i + 1] = v.y; a[i + 2] = v.z; a[i + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
      }
      if constexpr (TN % 4 == 0) {
#pragma unroll
        for (int j = 0; j < TN; j += 4) {
          const float4 v = *reinterpret_cast<const float4*>(&Bs[kk][tx * TN + j]);
          bb[j] = v.x; bb[j + 1] = v.y; bb[j + 2] = v.z; bb[j + 3] = v.w;
        }
      } else if constexpr (TN % 2 == 0) {
#pragma unroll
        for (int j = 0; j < TN; j += 2) {
          const float2 v = *reinterpret_cast<const float2*>(&Bs[kk][tx * TN + j]);
          bb[j] = v.x; bb[j + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tx * TN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }

  float alpha = d.alpha;
  if (d.inv_scale) alpha = (float)((double)alpha / d.inv_scale[b]);
  float* __restrict__ C = d.C + (long long)b * d.bsC;
  const int cm23 = d.cm2 * d.cm3;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty * TM + i;
    if (m >= d.M) continue;
    const long long om = (long long)(m / cm23) * d.sCm1 + (long long)((m / d.cm3) % d.cm2) * d.sCm2 +
                         (long long)(m % d.cm3) * d.sCm3;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx * TN + j;
      if (n >= d.N) continue;
      const long long on = s_on[tx * TN + j];
      const float v = alpha * acc[i][j];
      if (d.accumulate) C[om + on] += v; else C[om + on] = v;
    }
  }
}

struct Cfg {
  int BM, BN;
  const char* name;
};
const Cfg kCfgs[] = {{64, 64, "f32_64x64"},  {128, 64, "f32_128x64"}, {64, 32, "f32_64x32"},
                     {32, 32, "f32_32x32"},  {128, 32, "f32_128x32"}, {128, 128, "f32_128x128"}};

template <int BM, int BN, int TM, int TN>
cudaError_t launch(const GemmDesc& d, cudaStream_t st) {
  const int tiles = ((d.M + BM - 1) / BM) * ((d.N + BN - 1) / BN);
  dim3 grid(tiles, d.batch < 65535 ? d.batch : 65535, (d.batch + 65534) / 65535);
  gemm_f32_kernel<BM, BN, 16, TM, TN><<<grid, 256, 0, st>>>(d);
  return cudaGetLastError();
}

}  // namespace

int gemm_f32_num_configs() { return (int)(sizeof(kCfgs) / sizeof(kCfgs[0])); }
const char* gemm_f32_config_name(int cfg) { return kCfgs[cfg].name; }

int gemm_f32_pick(const GemmDesc& d) {
  if (d.N <= 32) return d.M >= 128 ? 4 : (d.M >= 64 ? 2 : 3);
  if (d.N <= 64) return d.M >= 128 ? 1 : 0;
  return d.M >= 128 ? 5 : 0;
}

cudaError_t gemm_f32(const GemmDesc& d, int cfg, cudaStream_t st) {
  if (g_dry_run || d.M <= 0 || d.N <= 0 || d.batch <= 0) return cudaSuccess;
  switch (cfg) {
    case 0: return launch<64, 64, 4, 4>(d, st);
    case 1: return launch<128, 64, 8, 4>(d, st);
    case 2: return launch<64, 32, 4, 2>(d, st);
    case 3: return launch<32, 32, 2, 2>(d, st);
    case 4: return launch<128, 32, 8, 2>(d, st);
    case 5: return launch<128, 128, 8, 8>(d, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pv
