// Learned proposal (declarations; see proposal.cu).
#pragma once
#include "common.cuh"

namespace pv {

constexpr int kNetC = 32;  // hidden channels
// Parameter block, contiguous in this order: w1 (32,1,3,3), b1 (32), w2 (32,32,3,3),
// b2 (32), w3 (2,32,3,3), b3 (2).
constexpr int kNetParams = kNetC * 9 + kNetC + kNetC * kNetC * 9 + kNetC + 2 * kNetC * 9 + 2;

struct NetParams {
  float *w1, *b1, *w2, *b2, *w3, *b3;
  static NetParams at(float* base) {
    NetParams p;
    p.w1 = base;
    p.b1 = p.w1 + kNetC * 9;
    p.w2 = p.b1 + kNetC;
    p.b2 = p.w2 + kNetC * kNetC * 9;
    p.w3 = p.b2 + kNetC;
    p.b3 = p.w3 + 2 * kNetC * 9;
    return p;
  }
};

// Logits (B, 2, Ly, Lx) of spins (B, Ly, Lx); h1, h2 hold (B, 32, Ly, Lx) activations.
cudaError_t net_forward(const NetParams& w, const int8_t* spins, int B, int Ly, int Lx, float* h1, float* h2,
                        float* out, cudaStream_t st);
// One Adam step (step number t >= 1) on the loss of a batch; acc[0] receives the summed
// squared error, acc[1] the number of antiparallel bonds.  d1, d2: (B, 32, Ly, Lx).
cudaError_t net_train_step(const NetParams& w, const NetParams& g, float* m, float* v, int nparam, int t, float lr,
                           const int8_t* spins, const float* rho, int B, int Ly, int Lx, float* h1, float* h2,
                           float* out, float* d2, float* d1, double* acc, cudaStream_t st);
// Draw one move per chain in band k; prop receives S', move the swapped site pairs
// (-1: none), lq = ln q(S'|S).
cudaError_t propose_moves(const float* logits, const int8_t* spins, int8_t* prop, int C, int Ly, int Lx, int k,
                          unsigned long long key, const unsigned long long* sweep, int* move, double* lq,
                          unsigned chain_base, cudaStream_t st);
// lq_rev = ln q(S|S') from the logits of S'.
cudaError_t reverse_logq(const float* logits, const int8_t* prop, int C, int Ly, int Lx, int k, const int* move,
                         double* lq_rev, cudaStream_t st);
// Metropolis-Hastings decision from the band closures den (S) and num (S') with their
// power-of-two exponents; accepted chains copy S' into spins.
cudaError_t accept_moves(int8_t* spins, const int8_t* prop, int C, int N, const int* move, const float* den,
                         const float* num, long long bs, const int* e_den, const int* e_num, const double* lq_fwd,
                         const double* lq_rev, unsigned long long key, const unsigned long long* sweep, int k,
                         int Lb, double* tr_rho, double* tr_dlq, int8_t* tr_dec, unsigned long long* counters,
                         unsigned* status, unsigned chain_base, cudaStream_t st);

}  // namespace pv
