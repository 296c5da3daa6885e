// Fused three-line column step on the tcgen05 tensor cores (App. C, Fig. "contraction"
// (c); the same network closes the three-line environments of the sampler's ratios,
// Eq. (9), and of the measurement, Eqs. (3)-(7)).
//
// Work unit: one chain and one tile of 8 values of the outgoing top bond a'.  A unit walks
// the incoming bottom bond b in tiles of 16 and runs three products per tile:
//   S1  X[(b,l)][(a',u)]   = sum_a     E(a,l,b) T(a,u,a')          M 128, N 64, K 32
//   S2  Y[(b,a')][(r,d)]   = sum_(l,u) X A_s(l,u,r,d)              M 128, N 64, K 64
//   S3  O[(r,a')][b']     += sum_(b,d) Y B(b,d,b')                 M  64, N 32, K 128
// S3 accumulates over the b tiles in tensor memory.  S1 and S2 accumulators are drained
// by the epilogue warps (one accumulator row per thread, tcgen05.ld) and stored,
// re-indexed and split into BF16 hi + lo, as the next product's A operand: S2's in the
// 128-byte swizzled layout, S3's without swizzle; in both the eight lanes that write one
// row group hit eight different bank groups.
//
// Split BF16 (x = hi + lo, the lo*lo term dropped) needs three BF16 products per step;
// an MMA instruction costs about the same for any N up to 128, so they are merged:
//   S1, S2: A_hi x [B_hi | B_lo] as one MMA of twice the width, plus A_lo x B_hi; the
//           epilogue adds the two column halves;
//   S3:     [Y_hi ; Y_lo] x [B_hi | B_lo] as one MMA of M 128, N 64 (the lo*lo quadrant
//           is computed and ignored); the final epilogue adds three quadrants.
// The lo copy of every operand tile directly follows its hi copy with the same row-group
// stride, so one descriptor addresses both.
//
// CTAs are persistent (two per SM: 104 KB of shared memory, 256 tensor-memory columns
// each, so one CTA's epilogues overlap the other's products) and walk the units in a
// grid-stride loop; the E and B slices of the next b tile -- of the next unit after a
// unit's last tile -- are fetched into registers while the current tile computes.  Bonds
// below the maxima are zero-padded on chip, so padded rows and columns of every
// intermediate are exact zeros and only valid outputs are written.
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
// S3 B: 32 rows (b') x 128 K ((b,d)) in the 128-byte swizzled layout, two K atoms of 64;
// with X3 the lo rows follow the hi rows inside each atom (one operand of 64 rows), so an
// atom holds 64 rows x 128 bytes.  Two buffers.
constexpr uint32_t SZ_B = 32 * 256, OFF_B = OFF_A + 2 * SZ_A;
constexpr uint32_t B_ATOM = 64 * 128, B_LO = 32 * 128;
constexpr uint32_t SMEM_USED = OFF_B + 4 * SZ_B;
constexpr uint32_t SMEM_BYTES = SMEM_USED + 1024;  // slack to align the swizzled tile to 1 KB
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t COL_S12 = 0, COL_S3 = 128;  // S1 and S2 share columns 0-127 (each is drained before the next)
static_assert(2 * (SMEM_BYTES + 1024) <= 233472, "two fused three-line CTAs must fit one SM");

__device__ __forceinline__ bool block_wait(uint64_t* bar, uint32_t parity, long long budget) {
  const bool w = wait_parity(bar, parity, budget);
  return !__syncthreads_or(!w);
}

// One K step of a split (or plain) BF16 product into accumulator d (N columns; with X3
// columns N..2N-1 receive A_hi x B_lo).
template <bool X3>
__device__ __forceinline__ void mma_merged(uint32_t d, uint64_t a_hi, uint64_t a_lo, uint64_t b, uint32_t id_n,
                                           uint32_t id_2n, uint32_t acc) {
  if constexpr (X3) {
    mma<2>(d, a_hi, b, id_2n, acc);  // [hi x hi | hi x lo]
    mma<2>(d, a_lo, b, id_n, 1u);    // lo x hi into the first half
  } else {
    mma<2>(d, a_hi, b, id_n, acc);
  }
}

struct Unit {
  int c, t;
};
__device__ __forceinline__ Unit unit_of(int u, int n_at) { return Unit{u / n_at, u % n_at}; }

// One b tile's operands in registers: the E slice (rows b*8 + l, K = a: the two rows of
// a pair of consecutive b at one l, one K chunk of 8) and the B slice (rows b', K = b*8 + d;
// two units of 8 per thread).
struct Slice {
  float e[2][8];
  float b[2][8];
};

// (b', b within the tile) of B-slice unit u: lanes along b' when b' is contiguous, else
// along b.
__device__ __forceinline__ void b_slot(const Env3Fused& a, int u, int& b2, int& bl) {
  if (a.sBb2 == 1 || a.sBb != 1) {
    b2 = u & 31;
    bl = u >> 5;
  } else {
    bl = u & 15;
    b2 = u >> 4;
  }
}

// E slice lanes: l fastest, then the b pair, then the K chunk.  The eight lanes of one
// shared-memory store phase then write rows of eight different l, i.e. eight different
// 16-byte bank groups of the K-major tile, and the global reads of one K value cover
// eight runs of eight consecutive b (full 32-byte sectors when b is contiguous).
__device__ __forceinline__ void fetch_slice(const Env3Fused& a, int c, int j, int tid, Slice& s) {
  const float* E = a.E + (long long)c * a.bsE;
  const float* B = a.B + (long long)c * a.bsB;
  {
    const int l = tid & 7, bp = (tid >> 3) & 7, kc = tid >> 6;
    const int b0 = j * kBT + 2 * bp;
    const bool lv = l < a.Dl;
    const float* src = E + (long long)b0 * a.sEb + l * a.sEl;
    // pairs of b as one 8-byte load when b is contiguous and every pair start is aligned
    const bool vec = a.sEb == 1 && ((a.sEl | a.sEa | a.bsE) & 1) == 0 && (reinterpret_cast<uintptr_t>(a.E) & 7) == 0 &&
                     b0 + 1 < a.cB;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      const bool kv = lv && k < a.cT;
      if (vec) {
        float2 v = kv ? *reinterpret_cast<const float2*>(src + k * a.sEa) : make_float2(0.f, 0.f);
        s.e[0][e] = v.x;
        s.e[1][e] = v.y;
      } else {
        s.e[0][e] = (kv && b0 < a.cB) ? src[k * a.sEa] : 0.f;
        s.e[1][e] = (kv && b0 + 1 < a.cB) ? src[k * a.sEa + a.sEb] : 0.f;
      }
    }
  }
  // B slice lanes along whichever of b' and b is contiguous in memory (the right step
  // reads a mirrored view whose b is contiguous); the swizzled operand layout keeps the
  // shared-memory stores conflict-free either way
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    int b2, bl;
    b_slot(a, tid + i * kThreads, b2, bl);
    const int b = j * kBT + bl;
    const bool rv = b2 < a.cB2 && b < a.cB;
    const float* src = B + b * a.sBb + b2 * a.sBb2;
#pragma unroll
    for (int e = 0; e < 8; ++e) s.b[i][e] = (rv && e < a.Dd) ? src[e * a.sBd] : 0.f;
  }
}

template <bool X3>
__device__ __forceinline__ void store_e(uint8_t* sm, int tid, const Slice& s) {
  const int l = tid & 7, bp = (tid >> 3) & 7, kc = tid >> 6;
#pragma unroll
  for (int i = 0; i < 2; ++i) put16<2, X3>(sm + OFF_E + kmajor_off((2 * bp + i) * 8 + l, kc * 8, 4), s.e[i], SZ_E);
}
// chunk (row b', K chunk b) of the swizzled S3 B operand
__device__ __forceinline__ uint32_t b_off(int b2, int b) { return (uint32_t)(b >> 3) * B_ATOM + sw128_chunk_off(b2, b & 7); }

template <bool X3>
__device__ __forceinline__ void store_b(const Env3Fused& a, uint8_t* sm, int buf, int tid, const Slice& s) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    int b2, bl;
    b_slot(a, tid + i * kThreads, b2, bl);
    put16<2, X3>(sm + OFF_B + buf * 2 * SZ_B + b_off(b2, bl), s.b[i], B_LO);
  }
}

// T tile of unit (c, t) (S1 B: rows a'_loc*8 + u, K = a) and the chain's A_s (S2 B: rows
// r*8 + d, K = l*8 + u): fetched into registers (during the previous unit's last
// epilogue), then stored as operands.
struct UnitRegs {
  float t[8];
  float a[2][8];
};
__device__ __forceinline__ void fetch_unit(const Env3Fused& a, int c, int t, int tid, UnitRegs& r) {
  const float* T = a.T + (long long)c * a.bsT;
  const int row = tid & 63, kc = tid >> 6;
  const int a2 = t * kAT + (row >> 3), uu = row & 7;
  const bool rv = a2 < a.cT2 && uu < a.Du;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = kc * 8 + e;
    r.t[e] = (rv && k < a.cT) ? T[k * a.sTa + uu * a.sTu + a2 * a.sTa2] : 0.f;
  }
  const int slot = a.sel ? (((a.sel[(long long)c * a.sel_stride] < 0) ? 1 : 0) ^ a.sel_xor) : 0;
  const float* A = a.A + (long long)slot * a.ssA;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    const int rw = u & 63, l = u >> 6, rr = rw >> 3, d = rw & 7;
    const bool ok = rr < a.Dr && d < a.Dd && l < a.Dl;
#pragma unroll
    for (int e = 0; e < 8; ++e) r.a[i][e] = (ok && e < a.Du) ? A[l * a.sAl + e * a.sAu + rr * a.sAr + d * a.sAd] : 0.f;
  }
}
template <bool X3>
__device__ __forceinline__ void store_unit(uint8_t* sm, int tid, const UnitRegs& r) {
  const int row = tid & 63, kc = tid >> 6;
  put16<2, X3>(sm + OFF_T + kmajor_off(row, kc * 8, 4), r.t, SZ_T);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    put16<2, X3>(sm + OFF_A + kmajor_off(u & 63, (u >> 6) * 8, 8), r.a[i], SZ_A);
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

template <bool X3>
__global__ void __launch_bounds__(kThreads, 2) env3_fused_kernel(const Env3Fused a, unsigned* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar[3];
  __shared__ uint32_t tmem_base;
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(sm);

  const int n_at = (a.cT2 + kAT - 1) / kAT, n_bt = (a.cB + kBT - 1) / kBT;
  const int n_units = a.batch * n_at;
  if ((int)blockIdx.x >= n_units) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long budget = a.wait_cycles > 0 ? a.wait_cycles : kDefaultWaitCycles;
  const long long drain = budget > kDefaultWaitCycles ? budget : kDefaultWaitCycles;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);

  Slice nxt;
  fetch_slice(a, unit_of(blockIdx.x, n_at).c, 0, tid, nxt);
  store_e<X3>(sm, tid, nxt);
  store_b<X3>(a, sm, 0, tid, nxt);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base;
  const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter; column half
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  const uint32_t id_n = idesc<2>(128, 64), id_2n = idesc<2>(128, 128);
  const uint32_t id3 = X3 ? idesc<2>(128, 64) : idesc<2>(64, 32);
  bool ok = true;
  int failed = -1;
  uint32_t fphase = 0, blk = 0, uph = 0;

  UnitRegs ur;
  {
    const Unit first = unit_of(blockIdx.x, n_at);
    fetch_unit(a, first.c, first.t, tid, ur);
  }
  for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, uph ^= 1u) {
    const Unit cur = unit_of(u, n_at);
    // T and A of this unit (the previous unit's S1 and S2 have completed)
    store_unit<X3>(sm, tid, ur);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    for (int j = 0; j < n_bt; ++j, ++blk) {
      const int buf = blk & 1;
      const uint32_t ph = blk & 1;
      // the next b tile: of this unit, or the first of the next unit of this CTA
      const bool more = j + 1 < n_bt || u + (int)gridDim.x < n_units;
      if (more) fetch_slice(a, j + 1 < n_bt ? cur.c : unit_of(u + gridDim.x, n_at).c, j + 1 < n_bt ? j + 1 : 0, tid, nxt);
      // ---- S1: M 128 (b,l), N 64 (a',u), K 32
      if (tid == 0) {
        tc_after_sync();
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t ao = sbase + OFF_E + ks * 256, bo = sbase + OFF_T + ks * 256;
          mma_merged<X3>(tmem + COL_S12, sdesc(ao, 128, 512), sdesc(ao + SZ_E, 128, 512), sdesc(bo, 128, 512), id_n,
                         id_2n, ks > 0 ? 1u : 0u);
        }
        commit(&bar[0]);
      }
      if (!(ok = block_wait(&bar[0], ph, budget))) { failed = 0; fphase = ph; break; }
      tc_after_sync();
      {  // S1 epilogue: row (b,l) -> S2 rows (b,a'), chunk l (swizzled)
        const int m1 = q * 32 + lane, bl = m1 >> 3, l = m1 & 7;
        float v[32];
        load_acc<X3>(tmem + lane_base + COL_S12 + h * 32, v);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          put16<2, X3>(sm + OFF_W + sw128_chunk_off(bl * 8 + h * 4 + i, l), v + i * 8, SZ_W);
      }
      // the E buffer was read only by S1, complete now
      if (more) store_e<X3>(sm, tid, nxt);
      fence_async_smem();
      tc_before_sync();
      __syncthreads();
      // ---- S2: M 128 (b,a'), N 64 (r,d), K 64
      if (tid == 0) {
        tc_after_sync();
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t ao = sbase + OFF_W + ks * 32, bo = sbase + OFF_A + ks * 256;
          mma_merged<X3>(tmem + COL_S12, sdesc_sw128(ao), sdesc_sw128(ao + SZ_W), sdesc(bo, 128, 1024), id_n, id_2n,
                         ks > 0 ? 1u : 0u);
        }
        commit(&bar[1]);
      }
      if (!(ok = block_wait(&bar[1], ph, budget))) { failed = 1; fphase = ph; break; }
      tc_after_sync();
      {  // S2 epilogue: row (b,a') -> S3 rows (r,a'), chunk b
        const int m2 = q * 32 + lane, bl = m2 >> 3, al = m2 & 7;
        float v[32];
        load_acc<X3>(tmem + lane_base + COL_S12 + h * 32, v);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          put16<2, X3>(sm + OFF_W + kmajor_off((h * 4 + i) * 8 + al, bl * 8, 16), v + i * 8, SZ_W);
      }
      fence_async_smem();
      tc_before_sync();
      __syncthreads();
      // ---- S3, accumulated over the b tiles: with X3 [Y_hi ; Y_lo] x [B_hi | B_lo] (M 128,
      // N 64), else Y x B (M 64, N 32).  Its completion is covered by the next S1 commit
      // (one CTA's products run in issue order), waited for before Y's buffer is
      // overwritten, and after the unit's last tile by bar[2].
      if (tid == 0) {
        tc_after_sync();
        const uint32_t bb = sbase + OFF_B + buf * 2 * SZ_B;
        for (int ks = 0; ks < 8; ++ks)
          mma<2>(tmem + COL_S3, sdesc(sbase + OFF_W + ks * 256, 128, 2048),
                 sdesc_sw128(bb + (ks >> 2) * B_ATOM + (ks & 3) * 32), id3, (j > 0 || ks > 0) ? 1u : 0u);
        if (j + 1 == n_bt) commit(&bar[2]);
      }
      // the other B buffer was last read by S3 of the previous tile, complete since bar[0]
      if (more) {
        store_b<X3>(a, sm, buf ^ 1, tid, nxt);
        fence_async_smem();
      }
      tc_before_sync();
      __syncthreads();
    }
    if (!ok) break;
    // T and A of the next unit, in flight during this unit's final epilogue
    if (u + (int)gridDim.x < n_units) {
      const Unit nu = unit_of(u + gridDim.x, n_at);
      fetch_unit(a, nu.c, nu.t, tid, ur);
    }
    if (!(ok = block_wait(&bar[2], uph, budget))) {
      failed = 2;
      fphase = uph;
      break;
    }
    tc_after_sync();
    // ---- output O[(r,a')][b'] of this unit
    float* O = a.out + (long long)cur.c * a.bsO;
    if constexpr (X3) {
      // lanes 0-63 hold [Y_hi B_hi | Y_hi B_lo], lanes 64-127 [Y_lo B_hi | -]: warps of
      // quarters 2 and 3 hand their first columns over through shared memory (the Y buffer
      // is dead now)
      float* xch = reinterpret_cast<float*>(sm + OFF_W);
      float v[16];
      tmem_ld16(tmem + lane_base + COL_S3 + h * 16, v);
      if (q >= 2) {
#pragma unroll
        for (int e = 0; e < 16; ++e) xch[((q - 2) * 32 + lane) * 33 + h * 16 + e] = v[e];
      }
      float w[16];
      tmem_ld16(tmem + lane_base + COL_S3 + 32 + h * 16, w);
      __syncthreads();
      if (q < 2) {
        const int m3 = q * 32 + lane, r = m3 >> 3, a2 = cur.t * kAT + (m3 & 7);
        if (a2 < a.cT2 && r < a.Dr) {
          float* dst = O + a2 * a.sOa2 + r * a.sOr;
          const int b0 = h * 16;
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] += w[e] + xch[m3 * 33 + b0 + e];
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
      }
    } else {
      // an M = 64 accumulator keeps rows 16q..16q+15 in lanes 0-15 of quarter q
      float v[16];
      tmem_ld16(tmem + lane_base + COL_S3 + h * 16, v);
      const int m3 = q * 16 + lane, r = m3 >> 3, a2 = cur.t * kAT + (m3 & 7);
      if (lane < 16 && a2 < a.cT2 && r < a.Dr) {
        float* dst = O + a2 * a.sOa2 + r * a.sOr;
        const int b0 = h * 16;
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if (b0 + e < a.cB2) dst[(b0 + e) * a.sOb2] = v[e];
      }
    }
    tc_before_sync();
    __syncthreads();
  }
  if (!ok) {
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
  static int ctas = 0;
  if (!ctas) {
    PV_CUDA(cudaFuncSetAttribute(env3_fused_kernel<X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMEM_BYTES));
    // the whole shared memory for this kernel, so that two CTAs fit an SM
    PV_CUDA(cudaFuncSetAttribute(env3_fused_kernel<X3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int dev = 0, sms = 0;
    PV_CUDA(cudaGetDevice(&dev));
    PV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ctas = 2 * sms;  // two resident CTAs per SM (104 KB shared memory, 128 registers x 256 threads each)
  }
  const long long units = (long long)a.batch * ((a.cT2 + kAT - 1) / kAT);
  if (units > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)(units < ctas ? units : ctas);
  env3_fused_kernel<X3><<<grid, kThreads, SMEM_BYTES, st>>>(a, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------ optimal site of the fit
// Fused optimal-site contraction of the variational fit (App. B): per work unit (one
// chain, one tile of 16 values of the new MPS's left bond v) the a' tiles of 8 are walked:
//   S1  X[(v,l)][(a',u)]    = sum_a     L(a,l,v) T(a,u,a')          M 128, N 64, K 32
//   S2  Y[(v,a')][(r,d)]    = sum_(l,u) X A_s(l,u,r,d)              M 128, N 64, K 64
//   S3  O[(v,d)][v']       += sum_(a',r) Y R(a',r,v')               M 128, N 32, K 64
// S3 accumulates over the a' tiles.  S1's epilogue is the three-line step's; S2's
// re-indexes each row (v,a') into rows (v,d) and K chunk a' of S3's operand, in the
// 128-byte swizzled layout (the eight lanes of one row group write eight different bank
// groups).  Split BF16 products are merged as in the three-line step.  The T tile and R
// slice of the next a' tile (of the next unit after the last) are fetched into registers
// while the current one computes.  88 KB of shared memory and 256 tensor-memory columns:
// two CTAs per SM.
constexpr int kPV = 16;  // v per unit
constexpr uint32_t P_SZ_W = 128 * 128, P_OFF_W = 0;                   // X or Y (swizzled)
constexpr uint32_t P_SZ_L = 128 * 64, P_OFF_L = P_OFF_W + 2 * P_SZ_W;  // S1 A: 128 rows x 32 K
constexpr uint32_t P_SZ_T = 64 * 64, P_OFF_T = P_OFF_L + 2 * P_SZ_L;   // S1 B: 64 rows x 32 K
constexpr uint32_t P_SZ_A = 64 * 128, P_OFF_A = P_OFF_T + 2 * P_SZ_T;  // S2 B: 64 rows x 64 K
constexpr uint32_t P_SZ_R = 32 * 128, P_OFF_R = P_OFF_A + 2 * P_SZ_A;  // S3 B: 32 rows x 64 K, two buffers
constexpr uint32_t P_SMEM_USED = P_OFF_R + 4 * P_SZ_R;
constexpr uint32_t P_SMEM_BYTES = P_SMEM_USED + 1024;
static_assert(2 * (P_SMEM_BYTES + 1024) <= 233472, "two fused optimal-site CTAs must fit one SM");

struct PSlice {
  float t[8];  // T tile: row tid & 63, chunk tid >> 6
  float r[8];  // R slice: row v' = tid & 31, chunk a' = tid >> 5
};

__device__ __forceinline__ void p_fetch(const Proj3Fused& a, int c, int t, int tid, PSlice& s) {
  const float* T = a.T + (long long)c * a.bsT;
  {
    const int row = tid & 63, kc = tid >> 6;
    const int a2 = t * kAT + (row >> 3), uu = row & 7;
    const bool rv = a2 < a.cT2 && uu < a.Du;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      s.t[e] = (rv && k < a.cT) ? T[k * a.sTa + uu * a.sTu + a2 * a.sTa2] : 0.f;
    }
  }
  const float* R = a.R + (long long)c * a.bsR;
  {
    const int v2 = tid & 31, a2 = t * kAT + (tid >> 5);
    const bool rv = v2 < a.cV2 && a2 < a.cT2;
#pragma unroll
    for (int e = 0; e < 8; ++e) s.r[e] = (rv && e < a.Dr) ? R[a2 * a.sRa + e * a.sRr + v2 * a.sRv] : 0.f;
  }
}
template <bool X3>
__device__ __forceinline__ void p_store_t(uint8_t* sm, int tid, const PSlice& s) {
  put16<2, X3>(sm + P_OFF_T + kmajor_off(tid & 63, (tid >> 6) * 8, 4), s.t, P_SZ_T);
}
template <bool X3>
__device__ __forceinline__ void p_store_r(uint8_t* sm, int buf, int tid, const PSlice& s) {
  put16<2, X3>(sm + P_OFF_R + buf * 2 * P_SZ_R + kmajor_off(tid & 31, (tid >> 5) * 8, 8), s.r, P_SZ_R);
}
// L slice of unit (c, vt) (S1 A: rows v*8 + l, K = a) and the chain's A_s (S2 B).
template <bool X3>
__device__ __forceinline__ void p_load_unit(const Proj3Fused& a, uint8_t* sm, int c, int vt, int tid) {
  // lanes: l fastest, then a pair of v, then the K chunk (the three-line step's E-slice
  // mapping: conflict-free shared-memory stores, full sectors when v is contiguous)
  const float* L = a.L + (long long)c * a.bsL;
  {
    const int l = tid & 7, vp = (tid >> 3) & 7, kc = tid >> 6;
    const int v0 = vt * kPV + 2 * vp;
    const bool lv = l < a.Dl;
    const float* src = L + (long long)v0 * a.sLv + l * a.sLl;
    const bool vec = a.sLv == 1 && ((a.sLl | a.sLa | a.bsL) & 1) == 0 && (reinterpret_cast<uintptr_t>(a.L) & 7) == 0 &&
                     v0 + 1 < a.cV;
    float x[2][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kc * 8 + e;
      const bool kv = lv && k < a.cT;
      if (vec) {
        const float2 w = kv ? *reinterpret_cast<const float2*>(src + k * a.sLa) : make_float2(0.f, 0.f);
        x[0][e] = w.x;
        x[1][e] = w.y;
      } else {
        x[0][e] = (kv && v0 < a.cV) ? src[k * a.sLa] : 0.f;
        x[1][e] = (kv && v0 + 1 < a.cV) ? src[k * a.sLa + a.sLv] : 0.f;
      }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) put16<2, X3>(sm + P_OFF_L + kmajor_off((2 * vp + i) * 8 + l, kc * 8, 4), x[i], P_SZ_L);
  }
  const int slot = a.sel ? ((a.sel[(long long)c * a.sel_stride] < 0) ? 1 : 0) : 0;
  const float* A = a.A + (long long)slot * a.ssA;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int u = tid + i * kThreads;
    const int rw = u & 63, l = u >> 6, r = rw >> 3, d = rw & 7;
    const bool ok = r < a.Dr && d < a.Dd && l < a.Dl;
    float x[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] = (ok && e < a.Du) ? A[l * a.sAl + e * a.sAu + r * a.sAr + d * a.sAd] : 0.f;
    put16<2, X3>(sm + P_OFF_A + kmajor_off(rw, l * 8, 8), x, P_SZ_A);
  }
}

template <bool X3>
__global__ void __launch_bounds__(kThreads, 2) proj3_fused_kernel(const Proj3Fused a, unsigned* status) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar[3];
  __shared__ uint32_t tmem_base;
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(sm);

  const int n_vt = (a.cV + kPV - 1) / kPV, n_at = (a.cT2 + kAT - 1) / kAT;
  const int n_units = a.batch * n_vt;
  if ((int)blockIdx.x >= n_units) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long budget = a.wait_cycles > 0 ? a.wait_cycles : kDefaultWaitCycles;
  const long long drain = budget > kDefaultWaitCycles ? budget : kDefaultWaitCycles;

  if (tid == 0) {
    for (int i = 0; i < 3; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(&tmem_base, TMEM_COLS);

  PSlice nxt;
  p_fetch(a, blockIdx.x / n_vt, 0, tid, nxt);
  p_store_t<X3>(sm, tid, nxt);
  p_store_r<X3>(sm, 0, tid, nxt);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tmem_base;
  const int q = warp & 3, h = warp >> 2;
  const uint32_t lane_base = (uint32_t)(q * 32) << 16;
  const uint32_t id_n = idesc<2>(128, 64), id_2n = idesc<2>(128, 128);
  const uint32_t id3_n = idesc<2>(128, 32), id3_2n = idesc<2>(128, 64);
  bool ok = true;
  int failed = -1;
  uint32_t fphase = 0, blk = 0, uph = 0;

  for (int u = blockIdx.x; u < n_units && ok; u += gridDim.x, uph ^= 1u) {
    const int c = u / n_vt, vt = u % n_vt;
    p_load_unit<X3>(a, sm, c, vt, tid);
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    for (int t = 0; t < n_at; ++t, ++blk) {
      const int buf = blk & 1;
      const uint32_t ph = blk & 1;
      const bool more = t + 1 < n_at || u + (int)gridDim.x < n_units;
      if (more) p_fetch(a, t + 1 < n_at ? c : (u + (int)gridDim.x) / n_vt, t + 1 < n_at ? t + 1 : 0, tid, nxt);
      // ---- S1: M 128 (v,l), N 64 (a',u), K 32
      if (tid == 0) {
        tc_after_sync();
        for (int ks = 0; ks < 2; ++ks) {
          const uint32_t ao = sbase + P_OFF_L + ks * 256, bo = sbase + P_OFF_T + ks * 256;
          mma_merged<X3>(tmem + COL_S12, sdesc(ao, 128, 512), sdesc(ao + P_SZ_L, 128, 512), sdesc(bo, 128, 512),
                         id_n, id_2n, ks > 0 ? 1u : 0u);
        }
        commit(&bar[0]);
      }
      if (!(ok = block_wait(&bar[0], ph, budget))) { failed = 0; fphase = ph; break; }
      tc_after_sync();
      {  // S1 epilogue: row (v,l) -> S2 rows (v,a'), chunk l (swizzled)
        const int m1 = q * 32 + lane, vl = m1 >> 3, l = m1 & 7;
        float v[32];
        load_acc<X3>(tmem + lane_base + COL_S12 + h * 32, v);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          put16<2, X3>(sm + P_OFF_W + sw128_chunk_off(vl * 8 + h * 4 + i, l), v + i * 8, P_SZ_W);
      }
      // the T tile was read only by S1, complete now
      if (more) p_store_t<X3>(sm, tid, nxt);
      fence_async_smem();
      tc_before_sync();
      __syncthreads();
      // ---- S2: M 128 (v,a'), N 64 (r,d), K 64
      if (tid == 0) {
        tc_after_sync();
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t ao = sbase + P_OFF_W + ks * 32, bo = sbase + P_OFF_A + ks * 256;
          mma_merged<X3>(tmem + COL_S12, sdesc_sw128(ao), sdesc_sw128(ao + P_SZ_W), sdesc(bo, 128, 1024), id_n, id_2n,
                         ks > 0 ? 1u : 0u);
        }
        commit(&bar[1]);
      }
      if (!(ok = block_wait(&bar[1], ph, budget))) { failed = 1; fphase = ph; break; }
      tc_after_sync();
      {  // S2 epilogue: row (v,a') -> S3 rows (v,d) for d in [4h, 4h+4), chunk a' (swizzled)
        const int m2 = q * 32 + lane, vl = m2 >> 3, al = m2 & 7;
        float x[8][4];  // [r][d - 4h]
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          float v[32];  // columns (r, d) with r in [4p, 4p+4)
          load_acc<X3>(tmem + lane_base + COL_S12 + p * 32, v);
#pragma unroll
          for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int dd = 0; dd < 4; ++dd) x[p * 4 + rr][dd] = v[rr * 8 + h * 4 + dd];
        }
#pragma unroll
        for (int dd = 0; dd < 4; ++dd) {
          float col[8];
#pragma unroll
          for (int r = 0; r < 8; ++r) col[r] = x[r][dd];
          put16<2, X3>(sm + P_OFF_W + sw128_chunk_off(vl * 8 + h * 4 + dd, al), col, P_SZ_W);
        }
      }
      fence_async_smem();
      tc_before_sync();
      __syncthreads();
      // ---- S3: M 128 (v,d), N 32 (v'), K 64 (a',r), accumulated over the a' tiles
      if (tid == 0) {
        tc_after_sync();
        const uint32_t rb = sbase + P_OFF_R + buf * 2 * P_SZ_R;
        for (int ks = 0; ks < 4; ++ks) {
          const uint32_t ao = sbase + P_OFF_W + ks * 32;
          mma_merged<X3>(tmem + COL_S3, sdesc_sw128(ao), sdesc_sw128(ao + P_SZ_W), sdesc(rb + ks * 256, 128, 1024),
                         id3_n, id3_2n, (t > 0 || ks > 0) ? 1u : 0u);
        }
        if (t + 1 == n_at) commit(&bar[2]);
      }
      // the other R buffer was last read by S3 of the previous tile, complete since bar[0]
      if (more) {
        p_store_r<X3>(sm, buf ^ 1, tid, nxt);
        fence_async_smem();
      }
      tc_before_sync();
      __syncthreads();
    }
    if (!ok) break;
    if (!(ok = block_wait(&bar[2], uph, budget))) {
      failed = 2;
      fphase = uph;
      break;
    }
    tc_after_sync();
    {  // ---- output Y(v,d,v') of this unit; warps h = 0 / 1 take v' 0-15 / 16-31
      float v[16];
      tmem_ld16(tmem + lane_base + COL_S3 + h * 16, v);
      if constexpr (X3) {
        float w[16];
        tmem_ld16(tmem + lane_base + COL_S3 + 32 + h * 16, w);
#pragma unroll
        for (int e = 0; e < 16; ++e) v[e] += w[e];
      }
      const int m = q * 32 + lane, vv = vt * kPV + (m >> 3), d = m & 7;
      if (vv < a.cV && d < a.Dd) {
        float* dst = a.out + (long long)c * a.bsO + vv * a.sOv + d * a.sOd;
        const int b0 = h * 16;
        if (a.sOv2 == 1 && b0 + 16 <= a.cV2 && ((reinterpret_cast<uintptr_t>(dst + b0) & 15u) == 0)) {
#pragma unroll
          for (int e = 0; e < 16; e += 4)
            *reinterpret_cast<float4*>(dst + b0 + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (b0 + e < a.cV2) dst[(b0 + e) * a.sOv2] = v[e];
        }
      }
    }
    tc_before_sync();
    __syncthreads();
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, ST_TIMEOUT);
    wait_parity(&bar[failed], fphase, drain);
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

template <bool X3>
cudaError_t launch_proj3(const Proj3Fused& a, unsigned* status, cudaStream_t st) {
  static int ctas = 0;
  if (!ctas) {
    PV_CUDA(cudaFuncSetAttribute(proj3_fused_kernel<X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)P_SMEM_BYTES));
    PV_CUDA(cudaFuncSetAttribute(proj3_fused_kernel<X3>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    int dev = 0, sms = 0;
    PV_CUDA(cudaGetDevice(&dev));
    PV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ctas = 2 * sms;
  }
  const long long units = (long long)a.batch * ((a.cV + kPV - 1) / kPV);
  if (units > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int grid = (int)(units < ctas ? units : ctas);
  proj3_fused_kernel<X3><<<grid, kThreads, P_SMEM_BYTES, st>>>(a, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t env3_fused(const Env3Fused& a, bool split, unsigned* status, cudaStream_t st) {
  if (g_dry_run || a.batch <= 0) return cudaSuccess;
  if (!env3_fused_fits(a.cT, a.cB, a.cT2, a.cB2, a.Dl, a.Dr, a.Du, a.Dd)) return cudaErrorInvalidValue;
  return split ? launch<true>(a, status, st) : launch<false>(a, status, st);
}

cudaError_t proj3_fused(const Proj3Fused& a, bool split, unsigned* status, cudaStream_t st) {
  if (g_dry_run || a.batch <= 0) return cudaSuccess;
  if (!proj3_fused_fits(a)) return cudaErrorInvalidValue;
  return split ? launch_proj3<true>(a, status, st) : launch_proj3<false>(a, status, st);
}

}  // namespace pv
