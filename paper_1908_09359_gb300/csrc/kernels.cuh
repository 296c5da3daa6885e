// Per-chain kernels of the VMC-PEPS hot path (declarations; see kernels.cu).
#pragma once
#include "common.cuh"

namespace pv {

constexpr unsigned kTagMetropolis = 0x4D455452u;  // "METR"
constexpr unsigned kTagUpdate = 0x55504454u;      // "UPDT"
constexpr unsigned kTagRandom = 0x52414E44u;      // "RAND"

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
  // Spin-inversion symmetrised sampling (|Phi|^2, Phi(S) = Psi(S) + Psi(S-bar)); chains
  // p and p + pairs hold S and S-bar.  With rho_out set, k_metropolis only writes each
  // chain's ratio rho = Psi(S')/Psi(S) (0 for a parallel pair) and k_phi_decide then
  // takes one decision per pair, min[1, ((rho_p + w rho_{p+P}) / (1 + w))^2] against
  // the pair's uniform (Philox counter word 0 = chain_base + p), applies it to both
  // chains, selects L(m) and carries w = Psi(S-bar)/Psi(S) (one copy per chain) by
  // w <- w rho_{p+P} / rho_p on acceptance.  Proposals are counted once per pair.
  double* rho_out;                       // nullable, [chain]
  double* phi_w;                         // [chain]
  int pairs;
};

// Random-NNASP scheme (Sec. II A, Eq. (prob_r)), one thread per chain.  propose: the
// K_a antiparallel NN pairs of each chain's configuration in bond order (vertical bonds
// by columns, then horizontal bonds by rows), the one with index floor(r K_a) swapped
// into prop (r from word 0 of Philox (chain, sweep, attempt, RAND)), K_b of the trial.
// accept: min[1, |Psi_b|^2 K_a / (|Psi_a|^2 K_b)] against word 1; an accepted trial
// replaces the spins and its ln|Psi| and sign the current ones.
struct RandomArgs {
  int8_t* spins; int8_t* prop; int C, Ly, Lx;
  unsigned long long key; const unsigned long long* sweep; int attempt; unsigned chain_base;
  int *Ka, *Kb, *bond;
  double* lp_cur; int8_t* sg_cur;          // current ln|Psi|, sign (updated on accept)
  const double* lp_new; const int8_t* sg_new;  // of the trial configurations
  int* tr_bond; double* tr_ratio; int8_t* tr_dec; long long tr_stride;  // nullable, [chain][attempt]
  unsigned long long* counters; unsigned* status;
};
cudaError_t k_random_propose(const RandomArgs& a, cudaStream_t st);
cudaError_t k_random_accept(const RandomArgs& a, cudaStream_t st);

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
cudaError_t k_phi_decide(const MetropolisArgs& a, int batch, cudaStream_t st);
// w of every chain from the amplitudes of both chains of its pair: sign_p sign_{p+P}
// exp(lnPsi_{p+P} - lnPsi_p).  With eloc set, also E^Phi = (E_p + w E_{p+P}) / (1 + w)
// into eloc_phi of both chains and the weights 1/(1+w) (chain p), w/(1+w) (chain p+P)
// of their G in G^Phi = (G(S) + w G(S-bar)) / (1 + w).
cudaError_t k_phi_combine(const double* logpsi, const int8_t* sign, const double* eloc, int batch, int pairs,
                          double* w, double* eloc_phi, double* wt, unsigned* status, cudaStream_t st);
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
                         double* sumGE, cudaStream_t st, const double* wt = nullptr);
cudaError_t k_energy_accum(const double* eloc, int batch, double* sums, cudaStream_t st);
cudaError_t k_grad_final(const double* sumG, const double* sumGE, const double* sums, long long P,
                         double* grad, cudaStream_t st);
cudaError_t k_sgd(double* master, const double* grad, long long P, double delta,
                  unsigned long long key, unsigned long long step, cudaStream_t st);

}  // namespace pv
