// The three-line environment step for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc at the point where they need
// an environment step: a service that reserved all of its device memory at start-up
// and must not allocate afterwards (cudaMalloc can synchronise the device and
// fragments a pre-planned pool), or host code that runs under a latency budget or
// holds a lock that an allocation could stall.  pepsvmc_env3_left needs a context,
// whose creation allocates; this entry point needs none.  Its two intermediates live
// in one fixed array of device memory that the library itself defines below.
//
// Host code cannot use the array's name as a device address (in host code it names
// a host-side stand-in), so every call looks the device address up with
// cudaGetSymbolAddress for the current device and context and passes it to the
// kernels.  The lookup allocates nothing and is cheap once the library's device code is
// loaded; doing it per call (rather than caching it per device ordinal) keeps the
// address right after a device reset or when another context is current on the device.

#include "common.cuh"
#include "pepsvmc.h"
#include "stages.cuh"

using namespace pv;

namespace {

static __device__ __align__(256) float noalloc_scratch[PEPSVMC_NOALLOC_SCRATCH_FLOATS];

// Device address of noalloc_scratch in the current context.
int scratch_on_current_device(float** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess || !p) return PEPSVMC_ECUDA;
  *out = static_cast<float*>(p);
  return PEPSVMC_OK;
}

}  // namespace

extern "C" int pepsvmc_env3_left_noalloc(const float* E, const float* T, const float* A, const int8_t* spins,
                                         const float* B, float* out, int32_t n_chains, int32_t cT, int32_t cB,
                                         int32_t cT2, int32_t cB2, int32_t Dl, int32_t Dr, int32_t Du, int32_t Dd,
                                         void* stream) {
  const Env3Dims d{cT, cB, cT2, cB2, Dl, Dr, Du, Dd};
  if (!E || !T || !A || !B || !out || n_chains < 1 || !env3_dims_ok(d)) return PEPSVMC_EINVAL;
  const long long per_chain = env3_scratch(d);
  if (per_chain > PEPSVMC_NOALLOC_SCRATCH_FLOATS / 2 / n_chains) return PEPSVMC_EINVAL;  // does not fit
  float* scratch = nullptr;
  const int rc = scratch_on_current_device(&scratch);
  if (rc != PEPSVMC_OK) return rc;
  float* t1 = scratch;
  float* t2 = scratch + (long long)n_chains * per_chain;
  GemmDesc g[3];
  env3_left_descs(g, d, E, (long long)cT * Dl * cB, T, (long long)cT * Du * cT2, A, (long long)Dl * Dr * Du * Dd,
                  spins, 1, 0, B, (long long)cB * Dd * cB2, out, (long long)cT2 * Dr * cB2, t1, t2, per_chain);
  for (int i = 0; i < 3; ++i) {
    g[i].batch = n_chains;
    if (gemm_f32(g[i], gemm_f32_pick(g[i]), (cudaStream_t)stream) != cudaSuccess) return PEPSVMC_ECUDA;
  }
  return PEPSVMC_OK;
}
