// Shared declarations of the pepsvmc CUDA library (kernels + host engine).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace pv {

// Batched contraction written as C[b] (scattered) = alpha * A[b] x B[b].
//   A(m,k) = A + b*bsA + m*sAm + k*sAk
//   B(k,n) = B + slot(b)*ssB + b*bsB + k*sBk + n*sBn,
//            slot(b) = (sel[b*sel_stride] < 0) ^ sel_xor when sel != nullptr, else 0
//   C index of (m,n): m = ((m1*cm2)+m2)*cm3+m3 -> m1*sCm1 + m2*sCm2 + m3*sCm3,
//                     n likewise with (cn2, cn3, sCn*).
//   alpha * (inv_scale ? 1/inv_scale[b] : 1).  accumulate: C += instead of C =.
struct GemmDesc {
  int M = 0, N = 0, K = 0, batch = 0;
  const float* A = nullptr;
  long long sAm = 0, sAk = 0, bsA = 0;
  const float* B = nullptr;
  long long sBk = 0, sBn = 0, bsB = 0, ssB = 0;
  const int8_t* sel = nullptr;
  long long sel_stride = 0;
  int sel_xor = 0;
  float* C = nullptr;
  long long bsC = 0;
  int cm2 = 1, cm3 = 1;
  long long sCm1 = 0, sCm2 = 0, sCm3 = 0;
  int cn2 = 1, cn3 = 1;
  long long sCn1 = 0, sCn2 = 0, sCn3 = 0;
  float alpha = 1.f;
  const double* inv_scale = nullptr;
  int accumulate = 0;
  long long wait_cycles = 0;  // clock budget of each device-side wait (0 = kDefaultWaitCycles)
};

// Default clock budget of a device-side wait (~2 s at 2 GHz).
constexpr long long kDefaultWaitCycles = 4000000000LL;

// Tile configurations of the FP32 contraction kernel (index into a fixed table).
int gemm_f32_num_configs();
const char* gemm_f32_config_name(int cfg);
cudaError_t gemm_f32(const GemmDesc& d, int cfg, cudaStream_t st);
int gemm_f32_pick(const GemmDesc& d);

// Same contraction on the tcgen05 tensor cores with FP32 accumulation in tensor memory.
// mode 2: operands rounded to BF16 (kind::f16); 3: split BF16, x = hi + lo, three MMAs
// per step; 4: operands rounded to TF32 (kind::tf32); 6: mode 3 with two shared-memory
// stages (bn 32 or 64).  Device waits are bounded; on
// expiry ST_TIMEOUT is set in *status.  bn: N tile (32, 64, 128, 256; 0 = smallest >= N).
cudaError_t gemm_tc(const GemmDesc& d, int mode, int bn, unsigned* status, cudaStream_t st);

// Batched Householder QR with diag(R) >= 0; writes the thin Q.
//   Y(i,j) = Y + b*bsY + i*yrs + j*ycs,   i < rows, j < cols, rows >= cols
//   Q(i,j) = Q + b*bsQ + i*qrs + j*qcs
cudaError_t qr_pos_batched(const float* Y, long long bsY, long long yrs, long long ycs,
                           float* Q, long long bsQ, long long qrs, long long qcs,
                           int rows, int cols, int batch, cudaStream_t st);

// Dry-run mode: every kernel wrapper returns at once without touching the device.
// The engine then runs its whole host-side orchestration (with bounds validation
// of every launch) on a machine without a GPU.
extern bool g_dry_run;

// Status word bits set by device code (checked by the host after a sync).
enum : unsigned {
  ST_ZEROPSI = 1u,
  ST_NONFINITE = 2u,
  ST_TIMEOUT = 4u,
};

}  // namespace pv

#define PV_CUDA(x)                                                        \
  do {                                                                    \
    cudaError_t e_ = (x);                                                 \
    if (e_ != cudaSuccess) return e_;                                     \
  } while (0)
