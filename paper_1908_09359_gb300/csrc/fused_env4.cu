// Fused four-line column step on the tcgen05 tensor cores (App. C: the four-line
// environments of a row pair give the vertical and diagonal amplitude ratios of E_loc,
// Eqs. (3)-(7), and the band ratios of the learned moves).
//
// One CTA owns one chain and one tile of 8 values of the outgoing top bond a'.  It walks
// the incoming bottom bond b in tiles of 2 and runs four products per tile:
//   S1  X[(b,l2,l1)][(a',u1)]   = sum_a       E(a,l1,l2,b) T(a,u1,a')     M 128, N 64, K 32
//   S2  Y[(l2,b,a')][(r1,d1)]   = sum_(l1,u1) X a1(l1,u1,r1,d1)           M 128, N 64, K 64
//   S3  Z[(b,r1,a')][(r2,d2)]   = sum_(l2,d1) Y a2(l2,d1,r2,d2)           M 128, N 64, K 64
//   S4  O[(r1,r2,a')][b']      += sum_(b,d2)  Z B(b,d2,b')                M 512, N 32, K 16
// S4 accumulates over the b tiles in tensor memory (four 128-row quarters); the other
// accumulators are drained after each product by the epilogue warps, split into BF16
// hi + lo and stored, re-indexed, as the next product's A operand (S2's in the 128-byte
// swizzled layout, S3's and S4's without swizzle; in every case the eight lanes that write
// one row group hit eight different bank groups).  X, Y and Z share one buffer and S1, S2
// and S3 one accumulator region (each is dead once the next product was issued).
// Split BF16 needs three BF16 products per step; an MMA instruction costs about the same
// for any N up to 128, so S1-S3 issue A_hi x [B_hi | B_lo] as one MMA of twice the width
// plus A_lo x B_hi, and the epilogue adds the two column halves (the lo copy of each B
// tile directly follows its hi copy with the same row-group stride).  The E and B slices
// of the next b tile are fetched into registers while the current tile computes.  Bonds
// below the maxima are zero-padded on chip.  Shared memory 93 KB and 256 tensor-memory
// columns per CTA: two CTAs share an SM, so one CTA's epilogues overlap the other's
// products.
#include "fused.cuh"
#include "tc_util.cuh"

namespace pv {
namespace {

using namespace tc;

constexpr int kThreads = 256;
constexpr int kAT = 8;  // a' per tile
constexpr int kBT = 2;  // b per tile

constexpr uint32_t SZ_W = 128 * 128, OFF_W = 0;                   // X (S2 A, swizzled), Y (S3 A) or Z (S4 A)
constexpr uint32_t SZ_E = 128 * 64, OFF_E = OFF_W + 2 * SZ_W;       // S1 A
constexpr uint32_t SZ_T = 64 * 64, OFF_T = OFF_E + 2 * SZ_E;        // S1 B
constexpr uint32_t SZ_A1 = 64 * 128, OFF_A1 = OFF_T + 2 * SZ_T;     // S2 B
constexpr uint32_t SZ_A2 = 64 * 128, OFF_A2 = OFF_A1 + 2 * SZ_A1;   // S3 B
constexpr uint32_t SZ_B = 32 * 32, OFF_B = OFF_A2 + 2 * SZ_A2;      // S4 B, two buffers
constexpr uint32_t SMEM_USED = OFF_B + 4 * SZ_B;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t COL_S123 = 0, COL_S4 = 128;
static_assert(2 * (SMEM_BYTES + 1024) <= 233472, "two fused four-line CTAs must fit one SM");

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

// One K step of a split (or plain) BF16 product into accumulator d (N columns; with X3
// columns N..2N-1 receive A_hi x B_lo).
template <bool X3>
__device__ __forceinline__ void mma_merged(uint32_t d, uint64_t a_hi, uint64_t a_lo, uint64_t b, uint32_t id_n,
                                           uint32_t id_2n, uint32_t acc) {
  if constexpr (X3) {
    mma<2>(d, a_hi, b, id_2n, acc);
    mma<2>(d, a_lo, b, id_n, 1u);
  } else {
    mma<2>(d, a_hi, b, id_n, acc);
  }
}

// 32 accumulator columns of this thread's row, the split halves added (X3).
template <bool X3>
__device__ __forceinline__ void load_acc(uint32_t taddr, float* v) {
  tmem_ld32(taddr, v);
  if constexpr (X3) {
    float w[32];
    tmem_ld32(taddr + 64, w);
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] += w[i];
  }
}

// Registers of one b tile's operands: E slice (two units of 8 per thread) and B slice
// (threads 0-63, one unit of 8).
struct Slice {
  float e[2][8];
  float b[8];
};

__device__ __forceinline__ void fetch_slice(const Env4Fused& a, const float* E, const float* B, int j, int tid,
                                            Slice& s) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    const int row = u & 127, kc = u >> 7;  // row = b_loc*64 + l2*8 + l1, K = a
    const int b = j * kBT + (row >> 6), l2 = (row >> 3) & 7, l1 = row & 7;
    const bool rv = b < a.cB && l1 < a.D1l && l2 < a.D2l;
    const float* src = E + b * a.sEb + l1 * a.sEl1 + l2 * a.sEl2;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      s.e[i][e] = (rv && k < a.cT) ? src[k * a.sEa] : 0.f;
    }
  }
  if (tid < 64) {
    const int b2 = tid & 31, b = j * kBT + (tid >> 5);  // row = b', K = b_loc*8 + d2
    const bool rv = b2 < a.cB2 && b < a.cB;
#pragma unroll
    for (int e = 0; e < 8; ++e) s.b[e] = (rv && e < a.Dd2) ? B[b * a.sBb + e * a.sBd + b2 * a.sBb2] : 0.f;
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
  if (tid < 64) put16<2, X3>(sm + OFF_B + buf * 2 * SZ_B + kmajor_off(tid & 31, (tid >> 5) * 8, 2), s.b, SZ_B);
}

template <bool X3>
__global__ void __launch_bounds__(kThreads, 2) env4_fused_kernel(const Env4Fused a, unsigned* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar[4];
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
    for (int i = 0; i < 4; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);

  const float* E = a.E + (long long)c * a.bsE;
  const float* B = a.B + (long long)c * a.bsB;
  Slice nxt;
  fetch_slice(a, E, B, 0, tid, nxt);
  {
    // T tile (S1 B): rows a'_loc*8 + u1, K = a
    const float* T = a.T + (long long)c * a.bsT;
    const int row = tid & 63, kc = tid >> 6;
    const int a2 = t * kAT + (row >> 3), u1 = row & 7;
    const bool rv = a2 < a.cT2 && u1 < a.Du1;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      v[e] = (rv && k < a.cT) ? T[k * a.sTa + u1 * a.sTu + a2 * a.sTa2] : 0.f;
    }
    put16<2, X3>(sm + OFF_T + kmajor_off(row, kc * 8, 4), v, SZ_T);
    // a1 (S2 B): rows r1*8 + d1, K = l1*8 + u1; a2 (S3 B): rows r2*8 + d2, K = l2*8 + d1
    const int s1 = a.sel1 ? (((a.sel1[(long long)c * a.sel_stride] < 0) ? 1 : 0) ^ a.xor1) : 0;
    const int s2 = a.sel2 ? (((a.sel2[(long long)c * a.sel_stride] < 0) ? 1 : 0) ^ a.xor2) : 0;
    const float* A1 = a.A1 + (long long)s1 * a.ss1;
    const float* A2 = a.A2 + (long long)s2 * a.ss2;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int u = tid + i * kThreads;
      const int rw = u & 63, l = u >> 6, r = rw >> 3, d = rw & 7;
      const bool v1 = r < a.D1r && d < a.Dd1 && l < a.D1l;
      const bool v2 = r < a.D2r && d < a.Dd2 && l < a.D2l;
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (v1 && e < a.Du1) ? A1[l * a.s1l + e * a.s1u + r * a.s1r + d * a.s1d] : 0.f;
      put16<2, X3>(sm + OFF_A1 + kmajor_off(rw, l * 8, 8), v, SZ_A1);
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (v2 && e < a.Dd1) ? A2[l * a.s2l + e * a.s2u + r * a.s2r + d * a.s2d] : 0.f;
      put16<2, X3>(sm + OFF_A2 + kmajor_off(rw, l * 8, 8), v, SZ_A2);
    }
  }
  store_e<X3>(sm, tid, nxt);
  store_b<X3>(sm, 0, tid, nxt);
  fence_async_smem();
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base;
  const int q = warp & 3, h = warp >> 2;
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  const uint32_t id_n = idesc<2>(128, 64), id_2n = idesc<2>(128, 128);
  bool ok = true;
  int failed = -1;
  uint32_t fphase = 0;

  for (int j = 0; j < n_bt && ok; ++j) {
    const int buf = j & 1;
    const uint32_t ph = (uint32_t)(j & 1);
    if (j + 1 < n_bt) fetch_slice(a, E, B, j + 1, tid, nxt);
    // ---- S1
    if (tid == 0) {
      tc_after_sync();
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t ao = sbase + OFF_E + ks * 256, bo = sbase + OFF_T + ks * 256;
        mma_merged<X3>(tmem + COL_S123, sdesc(ao, 128, 512), sdesc(ao + SZ_E, 128, 512), sdesc(bo, 128, 512), id_n,
                       id_2n, ks > 0 ? 1u : 0u);
      }
      commit(&bar[0]);
    }
    if (!(ok = block_wait(&bar[0], ph, budget))) { failed = 0; fphase = ph; break; }
    tc_after_sync();
    {  // S1 epilogue: row (b,l2,l1) -> S2 rows (l2,b,a'), chunk l1
      const int m1 = q * 32 + lane, bl = m1 >> 6, l2 = (m1 >> 3) & 7, l1 = m1 & 7;
      float v[32];
      load_acc<X3>(tmem + lane_base + COL_S123 + h * 32, v);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        put16<2, X3>(sm + OFF_W + sw128_chunk_off(l2 * 16 + bl * 8 + h * 4 + i, l1), v + i * 8, SZ_W);
    }
    // the E buffer was read only by S1, complete now
    if (j + 1 < n_bt) store_e<X3>(sm, tid, nxt);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    // ---- S2
    if (tid == 0) {
      tc_after_sync();
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t ao = sbase + OFF_W + ks * 32, bo = sbase + OFF_A1 + ks * 256;
        mma_merged<X3>(tmem + COL_S123, sdesc_sw128(ao), sdesc_sw128(ao + SZ_W), sdesc(bo, 128, 1024), id_n, id_2n,
                       ks > 0 ? 1u : 0u);
      }
      commit(&bar[1]);
    }
    if (!(ok = block_wait(&bar[1], ph, budget))) { failed = 1; fphase = ph; break; }
    tc_after_sync();
    {  // S2 epilogue: row (l2,b,a') -> S3 rows (b,r1,a'), chunk l2
      const int m2 = q * 32 + lane, l2 = m2 >> 4, bl = (m2 >> 3) & 1, al = m2 & 7;
      float v[32];
      load_acc<X3>(tmem + lane_base + COL_S123 + h * 32, v);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        put16<2, X3>(sm + OFF_W + kmajor_off(bl * 64 + (h * 4 + i) * 8 + al, l2 * 8, 8), v + i * 8, SZ_W);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    // ---- S3
    if (tid == 0) {
      tc_after_sync();
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t ao = sbase + OFF_W + ks * 256, bo = sbase + OFF_A2 + ks * 256;
        mma_merged<X3>(tmem + COL_S123, sdesc(ao, 128, 1024), sdesc(ao + SZ_W, 128, 1024), sdesc(bo, 128, 1024), id_n,
                       id_2n, ks > 0 ? 1u : 0u);
      }
      commit(&bar[2]);
    }
    if (!(ok = block_wait(&bar[2], ph, budget))) { failed = 2; fphase = ph; break; }
    tc_after_sync();
    {  // S3 epilogue: row (b,r1,a') -> S4 rows (r1,r2,a'), chunk b
      const int m3 = q * 32 + lane, bl = m3 >> 6, r1 = (m3 >> 3) & 7, al = m3 & 7;
      float v[32];
      load_acc<X3>(tmem + lane_base + COL_S123 + h * 32, v);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        put16<2, X3>(sm + OFF_W + kmajor_off(r1 * 64 + (h * 4 + i) * 8 + al, bl * 8, 2), v + i * 8, SZ_W);
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    // ---- S4, accumulated over the b tiles; its completion is covered by the next commit
    if (tid == 0) {
      tc_after_sync();
      const uint32_t id = idesc<2>(128, 32);
      const uint32_t bo = sbase + OFF_B + buf * 2 * SZ_B;
      for (int qq = 0; qq < 4; ++qq) {
        const uint32_t ao = sbase + OFF_W + qq * 4096;
        issue3<X3>(tmem + COL_S4 + qq * 32, sdesc(ao, 128, 256), sdesc(ao + SZ_W, 128, 256), sdesc(bo, 128, 256),
                   sdesc(bo + SZ_B, 128, 256), id, j > 0 ? 1u : 0u);
      }
      if (j + 1 == n_bt) commit(&bar[3]);
    }
    // the other B buffer was last read by S4 of tile j-1, complete since bar[0] of j; Z
    // stays in the shared buffer until S4 completes, which the next S1 commit covers (one
    // CTA's products run in issue order) before the next S1 epilogue overwrites it
    if (j + 1 < n_bt) {
      store_b<X3>(sm, buf ^ 1, tid, nxt);
      fence_async_smem();
    }
    tc_before_sync();
    __syncthreads();
  }
  if (ok) {
    if (!(ok = block_wait(&bar[3], 0u, budget))) {
      failed = 3;
      fphase = 0;
    }
  }
  if (ok) {
    tc_after_sync();
    float* O = a.out + (long long)c * a.bsO;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int qq = h + 2 * k;
      const int m4 = qq * 128 + q * 32 + lane, r1 = m4 >> 6, r2 = (m4 >> 3) & 7, a2 = t * kAT + (m4 & 7);
      float v[32];
      tmem_ld32(tmem + lane_base + COL_S4 + qq * 32, v);
      if (a2 < a.cT2 && r1 < a.D1r && r2 < a.D2r) {
        float* dst = O + a2 * a.sOa2 + r1 * a.sOr1 + r2 * a.sOr2;
        if (a.sOb2 == 1 && a.cB2 == 32 && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
#pragma unroll
          for (int e = 0; e < 32; e += 4)
            *reinterpret_cast<float4*>(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        } else {
#pragma unroll
          for (int e = 0; e < 32; ++e)
            if (e < a.cB2) dst[e * a.sOb2] = v[e];
        }
      }
    }
  } else {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
    wait_parity(&bar[failed], fphase, drain);
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

template <bool X3>
cudaError_t launch(const Env4Fused& a, unsigned* status, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    PV_CUDA(cudaFuncSetAttribute(env4_fused_kernel<X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMEM_BYTES));
    // the whole shared memory for this kernel, so that two CTAs fit an SM
    PV_CUDA(cudaFuncSetAttribute(env4_fused_kernel<X3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    configured = true;
  }
  const long long blocks = (long long)a.batch * ((a.cT2 + kAT - 1) / kAT);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  env4_fused_kernel<X3><<<(unsigned)blocks, kThreads, SMEM_BYTES, st>>>(a, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t env4_fused(const Env4Fused& a, bool split, unsigned* status, cudaStream_t st) {
  if (g_dry_run || a.batch <= 0) return cudaSuccess;
  if (!env4_fused_fits(a)) return cudaErrorInvalidValue;
  return split ? launch<true>(a, status, st) : launch<false>(a, status, st);
}

}  // namespace pv
