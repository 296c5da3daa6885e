// Per-chain kernels of the VMC-PEPS hot path (declarations; see kernels.cu).
#pragma once
#include "common.cuh"

namespace pv {

constexpr unsigned kTagMetropolis = 0x4D455452u;  // "METR"
constexpr unsigned kTagUpdate = 0x55504454u;      // "UPDT"

struct MetropolisArgs {
  const float* cur; long long bs_cur;    // L(m) with the current spin of column m
  const float* Rcur; long long bs_Rcur;  // R(m+1) with the current spin of column m+1
  const float* flip; long long bs_flip;  // L(m) with column m flipped
  const float* Rflip; long long bs_Rflip;// R(m+1) with column m+1 flipped
  int n;                                 // entries of one environment
  int8_t* spins; long long spin_stride;
  int site_a, site_b;                    // original lattice indices k*Lx+m of the pair
  unsigned long long key;                // Philox key (seed)
  unsigned chain_base;                   // global index of chain 0 (Philox counter word 0)
  const unsigned long long* sweep;       // device-resident sweep counter (read at run time)
  int bond;
  float* out; long long bs_out;          // selected, normalised L(m)
  double* trace_ratio; int8_t* trace_dec; long long trace_stride;  // nullable
  unsigned long long* counters;          // [0] proposals, [1] accepted
  unsigned* status;
};

cudaError_t k_fill(float* p, long long n, float v, cudaStream_t st);
cudaError_t k_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st);
cudaError_t k_fill_d(double* p, long long n, double v, cudaStream_t st);
cudaError_t k_gather_f32(float* dst, const double* src, const int* map, long long n, cudaStream_t st);
cudaError_t k_normalize_pow2(float* x, long long bs, int n, float* x2, long long bs2, int n2,
                             float* x3, long long bs3, int n3, int* exps, int batch, unsigned* status,
                             cudaStream_t st);
cudaError_t k_mps_normalize(float* x, long long bs, int n, const int* exps, const double* log_in,
                            double* log_out, int batch, unsigned* status, cudaStream_t st);
cudaError_t k_metropolis(const MetropolisArgs& a, int batch, cudaStream_t st);
cudaError_t k_dot(const float* a, long long bsa, const float* b, long long bsb, int n, double* out,
                  int batch, unsigned* status, cudaStream_t st);
// rho_out (nullable): the ratio of chain c is also written to rho_out[c * rho_stride + rho_idx].
cudaError_t k_ratio_accum(const float* a, long long bsa, const float* b, long long bsb, int n,
                          const double* den, const int8_t* spins, long long spin_stride, int si, int sj,
                          double halfJ, double* eloc, int batch, unsigned* status, cudaStream_t st,
                          float* rho_out = nullptr, long long rho_stride = 0, long long rho_idx = 0);
cudaError_t k_eloc_diag(const int8_t* spins, int Ly, int Lx, double J1, double J2, double* eloc,
                        int batch, cudaStream_t st);
cudaError_t k_logpsi(const float* x, long long bs, const int* exps, const double* logT,
                     const double* logB, double* logpsi, int8_t* sign, int batch, unsigned* status,
                     cudaStream_t st);
cudaError_t k_grad_accum(const float* G, long long bsG, long long Ph, const int* elem_site,
                         const long long* site_half_off, const long long* site_full_off,
                         const int* site_size, const int* site_spin, const int8_t* spins,
                         long long spin_stride, const double* eloc, int batch, double* sumG,
                         double* sumGE, cudaStream_t st);
cudaError_t k_energy_accum(const double* eloc, int batch, double* sums, cudaStream_t st);
cudaError_t k_grad_final(const double* sumG, const double* sumGE, const double* sums, long long P,
                         double* grad, cudaStream_t st);
cudaError_t k_sgd(double* master, const double* grad, long long P, double delta,
                  unsigned long long key, unsigned long long step, cudaStream_t st);

}  // namespace pv
