// Fused three-line column step on the tcgen05 tensor cores (App. C, Fig. "contraction"
// (c); the same network closes the three-line environments of the sampler's ratios,
// Eq. (9), and of the measurement, Eqs. (3)-(7)).
//
// One CTA owns one chain and one tile of 8 values of the outgoing top bond a'.  It walks
// the incoming bottom bond b in tiles of 16 and runs three products per tile:
//   S1  X[(b,l)][(a',u)]   = sum_a     E(a,l,b) T(a,u,a')          M 128, N 64, K 32
//   S2  Y[(b,a')][(r,d)]   = sum_(l,u) X A_s(l,u,r,d)              M 128, N 64, K 64
//   S3  O[(r,a')][b']     += sum_(b,d) Y B(b,d,b')                 M  64, N 32, K 128
// S3 accumulates over the b tiles in tensor memory.  S1 and S2 accumulators are drained
// by the epilogue warps (one accumulator row per thread, tcgen05.ld), split into BF16
// hi + lo and stored, re-indexed, as the next product's A operand: S2's in the 128-byte
// swizzled layout, S3's without swizzle; in both the eight lanes that write one row group
// hit eight different bank groups.  X and Y share one buffer (each is dead once its
// product completed).  The E and B slices of the next b tile are fetched into registers
// while the current tile computes.  Bonds below the maxima are zero-padded on chip, so
// padded rows and columns of every intermediate are exact zeros and only valid outputs
// are written.  Shared memory 104 KB and 256 tensor-memory columns per CTA: two CTAs
// share an SM, so one CTA's epilogues overlap the other's products.
#include "fused.cuh"
#include "tc_util.cuh"

namespace pv {
namespace {

using namespace tc;

constexpr int kThreads = 256;
constexpr int kAT = 8;   // a' per tile
constexpr int kBT = 16;  // b per tile

// byte offsets of the operand tiles (hi part; the lo part follows at + size)
constexpr uint32_t SZ_W = 128 * 128, OFF_W = 0;               // X (S2 A, swizzled) or Y (S3 A)
constexpr uint32_t SZ_E = 128 * 64, OFF_E = OFF_W + 2 * SZ_W;   // S1 A: 128 rows x 32 K
constexpr uint32_t SZ_T = 64 * 64, OFF_T = OFF_E + 2 * SZ_E;    // S1 B: 64 rows x 32 K
constexpr uint32_t SZ_A = 64 * 128, OFF_A = OFF_T + 2 * SZ_T;   // S2 B: 64 rows x 64 K
constexpr uint32_t SZ_B = 32 * 256, OFF_B = OFF_A + 2 * SZ_A;   // S3 B: 32 rows x 128 K, two buffers
constexpr uint32_t SMEM_USED = OFF_B + 4 * SZ_B;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;  // slack to align the swizzled tile to 1 KB
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t COL_S1 = 0, COL_S2 = 64, COL_S3 = 128;
static_assert(2 * (SMEM_BYTES + 1024) <= 233472, "two fused three-line CTAs must fit one SM");

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

// One b tile's operands in registers: the E slice (rows b*8 + l, K = a; two units of 8
// per thread) and the B slice (rows b', K = b*8 + d; two units of 8 per thread).
struct Slice {
  float e[2][8];
  float b[2][8];
};

__device__ __forceinline__ void fetch_slice(const Env3Fused& a, const float* E, const float* B, int j, int tid,
                                            Slice& s) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    const int row = u & 127, kc = u >> 7;
    const int b = j * kBT + (row >> 3), l = row & 7;
    const bool rv = b < a.cB && l < a.Dl;
    const float* src = E + b * a.sEb + l * a.sEl;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      s.e[i][e] = (rv && k < a.cT) ? src[k * a.sEa] : 0.f;
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    const int b2 = u & 31, b = j * kBT + (u >> 5);
    const bool rv = b2 < a.cB2 && b < a.cB;
    const float* src = B + b * a.sBb + b2 * a.sBb2;
#pragma unroll
    for (int e = 0; e < 8; ++e) s.b[i][e] = (rv && e < a.Dd) ? src[e * a.sBd] : 0.f;
  }
}

template <bool X3>
__device__ __forceinline__ void store_e(uint8_t* sm, int tid, const Slice& s) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    put16<2, X3>(sm + OFF_E + kmajor_off(u & 127, (u >> 7) * 8, 4), s.e[i], SZ_E);
  }
}
template <bool X3>
__device__ __forceinline__ void store_b(uint8_t* sm, int buf, int tid, const Slice& s) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    put16<2, X3>(sm + OFF_B + buf * 2 * SZ_B + kmajor_off(u & 31, (u >> 5) * 8, 16), s.b[i], SZ_B);
  }
}

template <bool X3>
__global__ void __launch_bounds__(kThreads, 2) env3_fused_kernel(const Env3Fused a, unsigned* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar[3];
  __shared__ uint32_t tmem_base;
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(sm);

  const int n_at = (a.cT2 + kAT - 1) / kAT, n_bt = (a.cB + kBT - 1) / kBT;
  const int c = blockIdx.x / n_at, t = blockIdx.x % n_at;
  if (c >= a.batch) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long budget = a.wait_cycles > 0 ? a.wait_cycles : kDefaultWaitCycles;
  const long long drain = budget > kDefaultWaitCycles ? budget : kDefaultWaitCycles;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);

  const float* E = a.E + (long long)c * a.bsE;
  const float* B = a.B + (long long)c * a.bsB;
  Slice nxt;
  fetch_slice(a, E, B, 0, tid, nxt);
  {
    // T tile (S1 B): rows a'_loc*8 + u, K = a
    const float* T = a.T + (long long)c * a.bsT;
    const int row = tid & 63, kc = tid >> 6;
    const int a2 = t * kAT + (row >> 3), uu = row & 7;
    const bool rv = a2 < a.cT2 && uu < a.Du;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      v[e] = (rv && k < a.cT) ? T[k * a.sTa + uu * a.sTu + a2 * a.sTa2] : 0.f;
    }
    put16<2, X3>(sm + OFF_T + kmajor_off(row, kc * 8, 4), v, SZ_T);
    // A_s (S2 B): rows r*8 + d, K = l*8 + u
    const int slot = a.sel ? (((a.sel[(long long)c * a.sel_stride] < 0) ? 1 : 0) ^ a.sel_xor) : 0;
    const float* A = a.A + (long long)slot * a.ssA;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int u = tid + i * kThreads;
      const int rw = u & 63, l = u >> 6, r = rw >> 3, d = rw & 7;
      const bool ok = r < a.Dr && d < a.Dd && l < a.Dl;
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (ok && e < a.Du) ? A[l * a.sAl + e * a.sAu + r * a.sAr + d * a.sAd] : 0.f;
      put16<2, X3>(sm + OFF_A + kmajor_off(rw, l * 8, 8), v, SZ_A);
    }
  }
  store_e<X3>(sm, tid, nxt);
  store_b<X3>(sm, 0, tid, nxt);
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base;
  const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter; column half
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  bool ok = true;
  int failed = -1;
  uint32_t fphase = 0;

  for (int j = 0; j < n_bt && ok; ++j) {
    const int buf = j & 1;
    const uint32_t ph = (uint32_t)(j & 1);
    if (j + 1 < n_bt) fetch_slice(a, E, B, j + 1, tid, nxt);
    // ---- S1: M 128 (b,l), N 64 (a',u), K 32
    if (tid == 0) {
      tc_after_sync();
      const uint32_t id = idesc<2>(128, 64);
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t ao = sbase + OFF_E + ks * 256, bo = sbase + OFF_T + ks * 256;
        issue3<X3>(tmem + COL_S1, sdesc(ao, 128, 512), sdesc(ao + SZ_E, 128, 512), sdesc(bo, 128, 512),
                   sdesc(bo + SZ_T, 128, 512), id, ks > 0 ? 1u : 0u);
      }
      commit(&bar[0]);
    }
    if (!(ok = block_wait(&bar[0], ph, budget))) { failed = 0; fphase = ph; break; }
    tc_after_sync();
    {  // S1 epilogue: row (b,l) -> S2 rows (b,a'), chunk l (swizzled)
      const int m1 = q * 32 + lane, bl = m1 >> 3, l = m1 & 7;
      float v[32];
      tmem_ld32(tmem + lane_base + COL_S1 + h * 32, v);
#pragma unroll
      for (int i = 0; i < 4; ++i) put16<2, X3>(sm + OFF_W + sw128_chunk_off(bl * 8 + h * 4 + i, l), v + i * 8, SZ_W);
    }
    // the E buffer was read only by S1, complete now
    if (j + 1 < n_bt) store_e<X3>(sm, tid, nxt);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    // ---- S2: M 128 (b,a'), N 64 (r,d), K 64
    if (tid == 0) {
      tc_after_sync();
      const uint32_t id = idesc<2>(128, 64);
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t ao = sbase + OFF_W + ks * 32, bo = sbase + OFF_A + ks * 256;
        issue3<X3>(tmem + COL_S2, sdesc_sw128(ao), sdesc_sw128(ao + SZ_W), sdesc(bo, 128, 1024),
                   sdesc(bo + SZ_A, 128, 1024), id, ks > 0 ? 1u : 0u);
      }
      commit(&bar[1]);
    }
    if (!(ok = block_wait(&bar[1], ph, budget))) { failed = 1; fphase = ph; break; }
    tc_after_sync();
    {  // S2 epilogue: row (b,a') -> S3 rows (r,a'), chunk b
      const int m2 = q * 32 + lane, bl = m2 >> 3, al = m2 & 7;
      float v[32];
      tmem_ld32(tmem + lane_base + COL_S2 + h * 32, v);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        put16<2, X3>(sm + OFF_W + kmajor_off((h * 4 + i) * 8 + al, bl * 8, 16), v + i * 8, SZ_W);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    // ---- S3: M 64 (r,a'), N 32 (b'), K 128 (b,d), accumulated over the b tiles.  Its
    // completion is covered by the next tile's S1 commit (the products of one CTA run
    // in issue order), which is waited for before Y's buffer is overwritten, and after
    // the last tile by bar[2].
    if (tid == 0) {
      tc_after_sync();
      const uint32_t id = idesc<2>(64, 32);
      const uint32_t bb = sbase + OFF_B + buf * 2 * SZ_B;
      for (int ks = 0; ks < 8; ++ks) {
        const uint32_t ao = sbase + OFF_W + ks * 256, bo = bb + ks * 256;
        issue3<X3>(tmem + COL_S3, sdesc(ao, 128, 2048), sdesc(ao + SZ_W, 128, 2048), sdesc(bo, 128, 2048),
                   sdesc(bo + SZ_B, 128, 2048), id, (j > 0 || ks > 0) ? 1u : 0u);
      }
      if (j + 1 == n_bt) commit(&bar[2]);
    }
    // the other B buffer was last read by S3 of tile j-1, complete since bar[0] of tile j
    if (j + 1 < n_bt) {
      store_b<X3>(sm, buf ^ 1, tid, nxt);
      fence_async_smem();
    }
    tc_before_sync();
    __syncthreads();
  }
  if (ok && !(ok = block_wait(&bar[2], 0u, budget))) {
    failed = 2;
    fphase = 0;
  }
  if (ok) {
    tc_after_sync();
    // an M = 64 accumulator keeps rows 16q..16q+15 in lanes 0-15 of quarter q; warps
    // h = 0 / 1 take columns 0-15 / 16-31
    float v[16];
    tmem_ld16(tmem + lane_base + COL_S3 + h * 16, v);
    const int m3 = q * 16 + lane, r = m3 >> 3, a2 = t * kAT + (m3 & 7);
    if (lane < 16 && a2 < a.cT2 && r < a.Dr) {
      float* dst = a.out + (long long)c * a.bsO + a2 * a.sOa2 + r * a.sOr;
      const int b0 = h * 16;
      if (a.sOb2 == 1 && b0 + 16 <= a.cB2 && ((reinterpret_cast<uintptr_t>(dst + b0) & 15u) == 0)) {
#pragma unroll
        for (int e = 0; e < 16; e += 4)
          *reinterpret_cast<float4*>(dst + b0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (b0 + e < a.cB2) dst[(b0 + e) * a.sOb2] = v[e];
      }
    }
  } else {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
    // the products of the expired wait may still run: let them finish before the tensor
    // memory is released
    wait_parity(&bar[failed], fphase, drain);
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

template <bool X3>
cudaError_t launch(const Env3Fused& a, unsigned* status, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    PV_CUDA(cudaFuncSetAttribute(env3_fused_kernel<X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMEM_BYTES));
    configured = true;
  }
  const long long blocks = (long long)a.batch * ((a.cT2 + kAT - 1) / kAT);
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
