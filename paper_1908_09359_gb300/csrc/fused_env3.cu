// Fused three-line column step on the tcgen05 tensor cores (App. C, Fig. "contraction"
// (c); the same network closes the three-line environments of the sampler's ratios,
// Eq. (9), and of the measurement, Eqs. (3)-(7)).
//
// One CTA owns one chain (and a group of a' tiles); per tile of 8 values of the outgoing
// top bond a' it runs the three products back to back:
//   S1  X[(b,l)][(a',u)]  = sum_a     E(a,l,b) T(a,u,a')          M 256, N 64, K 32
//   S2  Y[(b,a')][(r,d)]  = sum_(l,u) X A_s(l,u,r,d)              M 256, N 64, K 64
//   S3  O[(r,a')][b']     = sum_(b,d) Y B(b,d,b')                 M  64, N 32, K 256
// Accumulators live in tensor memory (columns 0-127 S1, 128-255 S2, 256-287 S3).  Between
// stages the epilogue warps read an accumulator row per thread (tcgen05.ld), split each
// FP32 value into BF16 hi + lo and store it as the next stage's A operand in shared
// memory, re-indexed: S2's operand uses the 128-byte swizzled layout so that the eight
// lanes writing one row group hit eight different bank groups; S3's operand needs no
// swizzle for that.  E, A_s and B are loaded once per CTA; only T is reloaded per tile.
// Bonds below the maxima are zero-padded, so padded rows and columns of every
// intermediate are exact zeros and only valid outputs are written.  Shared memory is
// 216 KB (one CTA per SM), tensor memory 512 columns.
#include "fused.cuh"
#include "tc_util.cuh"

namespace pv {
namespace {

using namespace tc;

constexpr int kThreads = 256;
constexpr int kAT = 8;  // a' values per tile

// byte offsets of the operand tiles (hi part; the lo part follows at + size)
constexpr uint32_t SZ_X = 256 * 128, OFF_X = 0;             // S2 A: 256 rows x 64 K, swizzled
constexpr uint32_t SZ_E = 256 * 64, OFF_E = OFF_X + 2 * SZ_X;  // S1 A: 256 rows x 32 K
constexpr uint32_t SZ_T = 64 * 64, OFF_T = OFF_E + 2 * SZ_E;   // S1 B: 64 rows x 32 K
constexpr uint32_t SZ_A = 64 * 128, OFF_A = OFF_T + 2 * SZ_T;  // S2 B: 64 rows x 64 K
constexpr uint32_t SZ_Y = 64 * 512, OFF_Y = OFF_A + 2 * SZ_A;  // S3 A: 64 rows x 256 K
constexpr uint32_t SZ_B = 32 * 512, OFF_B = OFF_Y + 2 * SZ_Y;  // S3 B: 32 rows x 256 K
constexpr uint32_t SMEM_USED = OFF_B + 2 * SZ_B;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;  // slack to align the swizzled tile to 1 KB
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t COL_S1 = 0, COL_S2 = 128, COL_S3 = 256;
static_assert(SMEM_BYTES <= 232448, "fused three-line step exceeds the shared memory of one CTA");

// Bounded wait on barrier `bar` by every thread; false (for the whole block) on expiry.
__device__ __forceinline__ bool block_wait(uint64_t* bar, uint32_t parity, long long budget) {
  const bool w = wait_parity(bar, parity, budget);
  return !__syncthreads_or(!w);
}

template <bool X3>
__device__ __forceinline__ void issue3(uint32_t d, uint64_t a_hi, uint64_t a_lo, uint64_t b_hi, uint64_t b_lo,
                                       uint32_t id, uint32_t acc) {
  mma<2>(d, a_hi, b_hi, id, acc);
  if constexpr (X3) {
    mma<2>(d, a_hi, b_lo, id, 1u);
    mma<2>(d, a_lo, b_hi, id, 1u);
  }
}

template <bool X3>
__global__ void __launch_bounds__(kThreads, 1) env3_fused_kernel(const Env3Fused a, unsigned* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar[3];
  __shared__ uint32_t tmem_base;
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(sm);

  const int n_at = (a.cT2 + kAT - 1) / kAT;
  const int tpc = a.tiles_per_cta;
  const int groups = (n_at + tpc - 1) / tpc;
  const int c = blockIdx.x / groups, grp = blockIdx.x % groups;
  if (c >= a.batch) return;
  const int t0 = grp * tpc, t1 = min(n_at, t0 + tpc);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long budget = a.wait_cycles > 0 ? a.wait_cycles : kDefaultWaitCycles;
  const long long drain = budget > kDefaultWaitCycles ? budget : kDefaultWaitCycles;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);

  // ---- per-chain operands: E^T (S1 A), A_s^T (S2 B), B^T (S3 B)
  {
    const float* E = a.E + (long long)c * a.bsE;
    for (int u = tid; u < 256 * 4; u += kThreads) {
      const int row = u & 255, kc = u >> 8;  // row = b*8 + l, K = a
      const int b = row >> 3, l = row & 7;
      const bool rv = b < a.cB && l < a.Dl;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = kc * 8 + i;
        v[i] = (rv && k < a.cT) ? E[k * a.sEa + l * a.sEl + b * a.sEb] : 0.f;
      }
      put16<2, X3>(sm + OFF_E + kmajor_off(row, kc * 8, 4), v, SZ_E);
    }
    const int slot = a.sel ? (((a.sel[(long long)c * a.sel_stride] < 0) ? 1 : 0) ^ a.sel_xor) : 0;
    const float* A = a.A + (long long)slot * a.ssA;
    for (int u = tid; u < 64 * 8; u += kThreads) {
      const int row = u & 63, l = u >> 6;  // row = r*8 + d, K = l*8 + u
      const int r = row >> 3, d = row & 7;
      const bool rv = r < a.Dr && d < a.Dd && l < a.Dl;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = (rv && i < a.Du) ? A[l * a.sAl + i * a.sAu + r * a.sAr + d * a.sAd] : 0.f;
      put16<2, X3>(sm + OFF_A + kmajor_off(row, l * 8, 8), v, SZ_A);
    }
    const float* B = a.B + (long long)c * a.bsB;
    for (int u = tid; u < 32 * 32; u += kThreads) {
      const int b2 = u & 31, b = u >> 5;  // row = b', K = b*8 + d
      const bool rv = b2 < a.cB2 && b < a.cB;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = (rv && i < a.Dd) ? B[b * a.sBb + i * a.sBd + b2 * a.sBb2] : 0.f;
      put16<2, X3>(sm + OFF_B + kmajor_off(b2, b * 8, 32), v, SZ_B);
    }
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base;
  const float* T = a.T + (long long)c * a.bsT;
  float* O = a.out + (long long)c * a.bsO;
  const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter, second index (M half or column half)
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  bool ok = true;
  int waited = -1;  // barrier of the MMAs in flight when a wait expired
  uint32_t phase = 0;

  for (int t = t0; t < t1 && ok; ++t, phase ^= 1u) {
    // ---- T tile (S1 B): rows (a'_loc*8 + u), K = a
    {
      const int row = tid & 63, kc = tid >> 6;
      const int al = row >> 3, uu = row & 7, a2 = t * kAT + al;
      const bool rv = a2 < a.cT2 && uu < a.Du;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = kc * 8 + i;
        v[i] = (rv && k < a.cT) ? T[k * a.sTa + uu * a.sTu + a2 * a.sTa2] : 0.f;
      }
      put16<2, X3>(sm + OFF_T + kmajor_off(row, kc * 8, 4), v, SZ_T);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    // ---- S1: two M halves of 128 rows, K = 32
    if (tid == 0) {
      tc_after_sync();
      const uint32_t id = idesc<2>(128, 64);
      for (int hh = 0; hh < 2; ++hh)
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t ao = sbase + OFF_E + hh * 8192 + ks * 256, bo = sbase + OFF_T + ks * 256;
          issue3<X3>(tmem + COL_S1 + hh * 64, sdesc(ao, 128, 512), sdesc(ao + SZ_E, 128, 512), sdesc(bo, 128, 512),
                     sdesc(bo + SZ_T, 128, 512), id, ks > 0 ? 1u : 0u);
        }
      commit(&bar[0]);
    }
    if (!(ok = block_wait(&bar[0], phase, budget))) { waited = 0; break; }
    tc_after_sync();
    // ---- S1 epilogue: row (b,l) of half h -> S2 operand rows (b,a'), chunk l, swizzled
    {
      const int m1 = h * 128 + q * 32 + lane, b = m1 >> 3, l = m1 & 7;
      float v[64];
      tmem_ld32(tmem + lane_base + COL_S1 + h * 64, v);
      tmem_ld32(tmem + lane_base + COL_S1 + h * 64 + 32, v + 32);
#pragma unroll
      for (int al = 0; al < 8; ++al) put16<2, X3>(sm + OFF_X + sw128_chunk_off(b * 8 + al, l), v + al * 8, SZ_X);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    // ---- S2: two M halves, K = 64 in four steps of 16
    if (tid == 0) {
      tc_after_sync();
      const uint32_t id = idesc<2>(128, 64);
      for (int hh = 0; hh < 2; ++hh)
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t ao = sbase + OFF_X + hh * 16384 + ks * 32, bo = sbase + OFF_A + ks * 256;
          issue3<X3>(tmem + COL_S2 + hh * 64, sdesc_sw128(ao), sdesc_sw128(ao + SZ_X), sdesc(bo, 128, 1024),
                     sdesc(bo + SZ_A, 128, 1024), id, ks > 0 ? 1u : 0u);
        }
      commit(&bar[1]);
    }
    if (!(ok = block_wait(&bar[1], phase, budget))) { waited = 1; break; }
    tc_after_sync();
    // ---- S2 epilogue: row (b,a') of half h -> S3 operand row (r,a'), chunk b
    {
      const int m2 = h * 128 + q * 32 + lane, b = m2 >> 3, al = m2 & 7;
      float v[64];
      tmem_ld32(tmem + lane_base + COL_S2 + h * 64, v);
      tmem_ld32(tmem + lane_base + COL_S2 + h * 64 + 32, v + 32);
#pragma unroll
      for (int r = 0; r < 8; ++r) put16<2, X3>(sm + OFF_Y + kmajor_off(r * 8 + al, b * 8, 32), v + r * 8, SZ_Y);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    // ---- S3: M = 64, N = 32, K = 256 in sixteen steps
    if (tid == 0) {
      tc_after_sync();
      const uint32_t id = idesc<2>(64, 32);
      for (int ks = 0; ks < 16; ++ks) {
        const uint32_t ao = sbase + OFF_Y + ks * 256, bo = sbase + OFF_B + ks * 256;
        issue3<X3>(tmem + COL_S3, sdesc(ao, 128, 4096), sdesc(ao + SZ_Y, 128, 4096), sdesc(bo, 128, 4096),
                   sdesc(bo + SZ_B, 128, 4096), id, ks > 0 ? 1u : 0u);
      }
      commit(&bar[2]);
    }
    if (!(ok = block_wait(&bar[2], phase, budget))) { waited = 2; break; }
    tc_after_sync();
    // ---- S3 epilogue: an M = 64 accumulator keeps rows 16q..16q+15 in lanes 0-15 of
    // quarter q; warps h = 0 / 1 take columns 0-15 / 16-31
    {
      float v[16];
      tmem_ld16(tmem + lane_base + COL_S3 + h * 16, v);
      const int m3 = q * 16 + lane, r = m3 >> 3, a2 = t * kAT + (m3 & 7);
      if (lane < 16 && a2 < a.cT2 && r < a.Dr) {
        float* dst = O + a2 * a.sOa2 + r * a.sOr;
        const int b0 = h * 16;
        if (a.sOb2 == 1 && b0 + 16 <= a.cB2 && ((reinterpret_cast<uintptr_t>(dst + b0) & 15u) == 0)) {
#pragma unroll
          for (int j = 0; j < 16; j += 4)
            *reinterpret_cast<float4*>(dst + b0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (b0 + j < a.cB2) dst[(b0 + j) * a.sOb2] = v[j];
        }
      }
    }
    tc_before_sync();
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
    // the MMAs of the expired wait may still be running: let them finish before the
    // tensor memory is released
    wait_parity(&bar[waited], phase, drain);
    tc_before_sync();
    __syncthreads();
  }
  tc_after_sync();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

template <bool X3>
cudaError_t launch(const Env3Fused& a0, unsigned* status, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    PV_CUDA(cudaFuncSetAttribute(env3_fused_kernel<X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMEM_BYTES));
    configured = true;
  }
  Env3Fused a = a0;
  const int n_at = (a.cT2 + kAT - 1) / kAT;
  if (a.tiles_per_cta <= 0) a.tiles_per_cta = a.batch >= 2 * 152 ? n_at : 1;
  if (a.tiles_per_cta > n_at) a.tiles_per_cta = n_at;
  const long long groups = (n_at + a.tiles_per_cta - 1) / a.tiles_per_cta;
  const long long blocks = groups * a.batch;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  env3_fused_kernel<X3><<<(unsigned)blocks, kThreads, SMEM_BYTES, st>>>(a, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t env3_fused(const Env3Fused& a, bool split, unsigned* status, cudaStream_t st) {
  if (g_dry_run || a.batch <= 0) return cudaSuccess;
  if (!env3_fused_fits(a.cT, a.cB, a.cT2, a.cB2, a.Dl, a.Dr, a.Du, a.Dd)) return cudaErrorInvalidValue;
  return split ? launch<true>(a, status, st) : launch<false>(a, status, st);
}

}  // namespace pv
