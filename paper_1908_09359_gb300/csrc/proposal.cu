// Learned proposal: a small convolutional network on the spin grid and exact
// Metropolis-Hastings moves of one or two antiparallel pairs inside a row band.
//
// The network (three zero-padded 3x3 convolutions, 1 -> 32 -> 32 -> 2 channels, ReLU
// after the first two) gives, at site (k, m), the logit of the horizontal bond
// (k,m)-(k,m+1) (channel 0) and of the vertical bond (k,m)-(k+1,m) (channel 1).  It is
// trained to predict log min(1, rho^2) of each antiparallel bond, rho the amplitude
// ratio the measurement computes, so it learns which swaps are likely accepted.  A
// move in band k draws a pair from the softmax of the band's candidate logits and, with
// probability 1/2, a second site-disjoint pair; acceptance is
// min[1, |Psi(S')/Psi(S)|^2 q(S|S')/q(S'|S)] (the Metropolis-Hastings form of Eq. (8)
// of arXiv:1908.09359 with a learned q), with Psi' / Psi from the band's four-line
// closure, so sampling stays exact whatever the network predicts.
#include "proposal.cuh"

namespace pv {
namespace {

constexpr unsigned kTagLearn = 0x4C45524Eu;  // "LERN"
constexpr int kMaxCand = 3 * 64;

__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ double uni(unsigned long long key, unsigned chain, unsigned sweep, unsigned ctr) {
  const uint4 w = philox(make_uint4(chain, sweep, ctr, kTagLearn),
                         make_uint2((unsigned)(key & 0xffffffffull), (unsigned)(key >> 32)));
  return (double)(w.x >> 8) * (1.0 / 16777216.0);
}

// ------------------------------------------------------------------ convolutions
__global__ void conv_fwd_kernel(const float* in, const int8_t* spins, int Cin, const float* w, const float* bias,
                                float* out, int Cout, int B, int Ly, int Lx, int relu) {
  const long long n = (long long)B * Cout * Ly * Lx;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
    const int x = idx % Lx, y = (idx / Lx) % Ly, co = (idx / ((long long)Lx * Ly)) % Cout;
    const long long b = idx / ((long long)Lx * Ly * Cout);
    float acc = bias[co];
    for (int ci = 0; ci < Cin; ++ci)
      for (int dy = 0; dy < 3; ++dy) {
        const int yy = y + dy - 1;
        if (yy < 0 || yy >= Ly) continue;
        for (int dx = 0; dx < 3; ++dx) {
          const int xx = x + dx - 1;
          if (xx < 0 || xx >= Lx) continue;
          const float v = spins ? (float)spins[(b * Ly + yy) * Lx + xx] : in[((b * Cin + ci) * Ly + yy) * Lx + xx];
          acc = fmaf(w[((co * Cin + ci) * 3 + dy) * 3 + dx], v, acc);
        }
      }
    out[idx] = relu ? fmaxf(acc, 0.f) : acc;
  }
}

// d(loss)/d(input pre-activation) of a convolution whose input is h = relu(z).
__global__ void conv_bwd_in_kernel(const float* dout, int Cout, const float* w, const float* h_in, float* din, int Cin,
                                   int B, int Ly, int Lx) {
  const long long n = (long long)B * Cin * Ly * Lx;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
    if (!(h_in[idx] > 0.f)) {
      din[idx] = 0.f;
      continue;
    }
    const int x = idx % Lx, y = (idx / Lx) % Ly, ci = (idx / ((long long)Lx * Ly)) % Cin;
    const long long b = idx / ((long long)Lx * Ly * Cin);
    float acc = 0.f;
    for (int co = 0; co < Cout; ++co)
      for (int dy = 0; dy < 3; ++dy) {
        const int yo = y - dy + 1;
        if (yo < 0 || yo >= Ly) continue;
        for (int dx = 0; dx < 3; ++dx) {
          const int xo = x - dx + 1;
          if (xo < 0 || xo >= Lx) continue;
          acc = fmaf(w[((co * Cin + ci) * 3 + dy) * 3 + dx], dout[((b * Cout + co) * Ly + yo) * Lx + xo], acc);
        }
      }
    din[idx] = acc;
  }
}

// Weight and bias gradients: one block per (co, ci) pair; block (co, Cin) does the bias.
__global__ void conv_bwd_w_kernel(const float* dout, int Cout, const float* in, const int8_t* spins, int Cin,
                                  float* dw, float* db, int B, int Ly, int Lx) {
  const int co = blockIdx.x / (Cin + 1), ci = blockIdx.x % (Cin + 1);
  __shared__ float red[9][8];
  float acc[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const long long n = (long long)B * Ly * Lx;
  for (long long p = threadIdx.x; p < n; p += blockDim.x) {
    const int x = p % Lx, y = (p / Lx) % Ly;
    const long long b = p / ((long long)Lx * Ly);
    const float g = dout[((b * Cout + co) * Ly + y) * Lx + x];
    if (ci == Cin) {
      acc[0] += g;
      continue;
    }
    for (int dy = 0; dy < 3; ++dy) {
      const int yy = y + dy - 1;
      if (yy < 0 || yy >= Ly) continue;
      for (int dx = 0; dx < 3; ++dx) {
        const int xx = x + dx - 1;
        if (xx < 0 || xx >= Lx) continue;
        const float v = spins ? (float)spins[(b * Ly + yy) * Lx + xx] : in[((b * Cin + ci) * Ly + yy) * Lx + xx];
        acc[dy * 3 + dx] = fmaf(g, v, acc[dy * 3 + dx]);
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = 0; t < 9; ++t) {
    float v = acc[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[t][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[threadIdx.x][i];
    if (ci == Cin) {
      if (threadIdx.x == 0) db[co] = s;
    } else {
      dw[(co * Cin + ci) * 9 + threadIdx.x] = s;
    }
  }
}

// Mean-squared error against log min(1, rho^2) (clipped at -20) of antiparallel bonds.
__global__ void loss_kernel(const float* out, const int8_t* spins, const float* rho, int B, int Ly, int Lx,
                            float* dout, double* acc /* [0] sum d^2, [1] count */, int pass) {
  const long long n = (long long)B * 2 * Ly * Lx;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n; idx += (long long)gridDim.x * blockDim.x) {
    const int x = idx % Lx, y = (idx / Lx) % Ly, ch = (idx / ((long long)Lx * Ly)) % 2;
    const long long b = idx / ((long long)Lx * Ly * 2);
    const int8_t* s = spins + b * Ly * Lx;
    bool anti = false;
    if (ch == 0 && x + 1 < Lx) anti = s[y * Lx + x] != s[y * Lx + x + 1];
    if (ch == 1 && y + 1 < Ly) anti = s[y * Lx + x] != s[(y + 1) * Lx + x];
    if (pass == 0) {
      if (anti) atomicAdd(&acc[1], 1.0);
      continue;
    }
    float d = 0.f;
    if (anti) {
      const float r = rho[idx];
      const float t = fmaxf(-20.f, fminf(0.f, logf(fminf(1.f, r * r))));
      d = out[idx] - (isfinite(t) ? t : -20.f);
      atomicAdd(&acc[0], (double)d * d);
    }
    dout[idx] = 2.f * d / (float)fmax(acc[1], 1.0);
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float c1, float c2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  m[i] = b1 * m[i] + (1.f - b1) * g[i];
  v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
  p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

// ------------------------------------------------------------------ moves
struct Cand {
  int a, b;      // sites (k*Lx + m)
  float logit;
};

__device__ int band_candidates(const int8_t* s, const float* lg, int Ly, int Lx, int k, Cand* c) {
  int n = 0;
  const int N = Ly * Lx;
  for (int r = k; r <= k + 1; ++r)
    for (int m = 0; m + 1 < Lx; ++m)
      if (s[r * Lx + m] != s[r * Lx + m + 1]) c[n++] = {r * Lx + m, r * Lx + m + 1, lg[r * Lx + m]};
  for (int m = 0; m < Lx; ++m)
    if (s[k * Lx + m] != s[(k + 1) * Lx + m]) c[n++] = {k * Lx + m, (k + 1) * Lx + m, lg[N + k * Lx + m]};
  return n;
}

__device__ __forceinline__ bool disjoint(const Cand& x, const Cand& y) {
  return x.a != y.a && x.a != y.b && x.b != y.a && x.b != y.b;
}

// softmax probability of candidate i among those with use[j] (double)
__device__ double soft_p(const Cand* c, int n, const bool* use, int i) {
  double mx = -1e300;
  for (int j = 0; j < n; ++j)
    if (use[j]) mx = fmax(mx, (double)c[j].logit);
  double z = 0.0;
  for (int j = 0; j < n; ++j)
    if (use[j]) z += exp((double)c[j].logit - mx);
  return exp((double)c[i].logit - mx) / z;
}

__device__ int soft_draw(const Cand* c, int n, const bool* use, double u) {
  double mx = -1e300;
  for (int j = 0; j < n; ++j)
    if (use[j]) mx = fmax(mx, (double)c[j].logit);
  double z = 0.0;
  for (int j = 0; j < n; ++j)
    if (use[j]) z += exp((double)c[j].logit - mx);
  double cum = 0.0;
  int last = -1;
  for (int j = 0; j < n; ++j) {
    if (!use[j]) continue;
    cum += exp((double)c[j].logit - mx) / z;
    last = j;
    if (cum > u) return j;
  }
  return last;
}

// ln q of a move {i} or {i, j} (candidate indices) under the candidate list c.
__device__ double move_logq(const Cand* c, int n, int i, int j) {
  bool use[kMaxCand];
  for (int t = 0; t < n; ++t) use[t] = true;
  const double p1i = soft_p(c, n, use, i);
  if (j < 0) return log(0.5 * p1i);
  const double p1j = soft_p(c, n, use, j);
  for (int t = 0; t < n; ++t) use[t] = disjoint(c[t], c[i]);
  const double p2j = soft_p(c, n, use, j);
  for (int t = 0; t < n; ++t) use[t] = disjoint(c[t], c[j]);
  const double p2i = soft_p(c, n, use, i);
  return log(0.5 * (p1i * p2j + p1j * p2i));
}

__device__ int find(const Cand* c, int n, int a, int b) {
  for (int t = 0; t < n; ++t)
    if (c[t].a == a && c[t].b == b) return t;
  return -1;
}

__global__ void propose_kernel(const float* logits, const int8_t* spins, int8_t* prop, int C, int Ly, int Lx, int k,
                               unsigned long long key, const unsigned long long* sweep, int* move, double* lq,
                               unsigned chain_base) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int N = Ly * Lx;
  const int8_t* s = spins + (long long)c * N;
  int8_t* p = prop + (long long)c * N;
  for (int i = 0; i < N; ++i) p[i] = s[i];
  int* mv = move + 4 * c;
  mv[0] = mv[1] = mv[2] = mv[3] = -1;
  lq[c] = 0.0;
  Cand cand[kMaxCand];
  const int n = band_candidates(s, logits + (long long)c * 2 * N, Ly, Lx, k, cand);
  if (n == 0) return;
  const unsigned sw = (unsigned)*sweep;
  const unsigned cg = (unsigned)c + chain_base;
  const double u0 = uni(key, cg, sw, 4 * k), u1 = uni(key, cg, sw, 4 * k + 1), u2 = uni(key, cg, sw, 4 * k + 2);
  bool use[kMaxCand];
  for (int t = 0; t < n; ++t) use[t] = true;
  const int i = soft_draw(cand, n, use, u1);
  int j = -1;
  if (u0 >= 0.5) {
    bool any = false;
    for (int t = 0; t < n; ++t) any |= (use[t] = disjoint(cand[t], cand[i]));
    if (!any) return;  // a two-pair draw with no disjoint pair left proposes nothing
    j = soft_draw(cand, n, use, u2);
  }
  mv[0] = cand[i].a;
  mv[1] = cand[i].b;
  if (j >= 0) {
    mv[2] = cand[j].a;
    mv[3] = cand[j].b;
  }
  for (int q = 0; q < 4; q += 2)
    if (mv[q] >= 0) {
      const int8_t t = p[mv[q]];
      p[mv[q]] = p[mv[q + 1]];
      p[mv[q + 1]] = t;
    }
  lq[c] = move_logq(cand, n, i, j);
}

__global__ void reverse_kernel(const float* logits, const int8_t* prop, int C, int Ly, int Lx, int k, const int* move,
                               double* lq_rev) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int N = Ly * Lx;
  const int* mv = move + 4 * c;
  lq_rev[c] = 0.0;
  if (mv[0] < 0) return;
  Cand cand[kMaxCand];
  const int n = band_candidates(prop + (long long)c * N, logits + (long long)c * 2 * N, Ly, Lx, k, cand);
  const int i = find(cand, n, mv[0], mv[1]);
  const int j = mv[2] >= 0 ? find(cand, n, mv[2], mv[3]) : -1;
  lq_rev[c] = move_logq(cand, n, i, j);
}

__global__ void accept_kernel(int8_t* spins, const int8_t* prop, int C, int N, const int* move, const float* den,
                              const float* num, long long bs, const int* e_den, const int* e_num,
                              const double* lq_fwd, const double* lq_rev, unsigned long long key,
                              const unsigned long long* sweep, int k, int Lb, double* tr_rho, double* tr_dlq,
                              int8_t* tr_dec, unsigned long long* counters, unsigned* status, unsigned chain_base) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int dec = -1;
  double rho = 0.0, dlq = 0.0;
  if (move[4 * c] >= 0) {
    const double d = den[(long long)c * bs], u = num[(long long)c * bs];
    if (d == 0.0) {
      atomicOr(status, ST_ZEROPSI);
    } else {
      rho = u / d * exp2((double)(e_num[c] - e_den[c]));
      dlq = lq_rev[c] - lq_fwd[c];
      const double a = fmin(1.0, rho * rho * exp(dlq));
      if (!isfinite(a)) atomicOr(status, ST_NONFINITE);
      dec = (uni(key, (unsigned)c + chain_base, (unsigned)*sweep, 4 * k + 3) < a) ? 1 : 0;
      atomicAdd(&counters[0], 1ull);
      if (dec) {
        atomicAdd(&counters[1], 1ull);
        for (int i = 0; i < N; ++i) spins[(long long)c * N + i] = prop[(long long)c * N + i];
      }
    }
  }
  if (tr_dec) {
    tr_rho[(long long)c * Lb + k] = rho;
    tr_dlq[(long long)c * Lb + k] = dlq;
    tr_dec[(long long)c * Lb + k] = (int8_t)dec;
  }
}

inline int blocks(long long n, int t = 256) {
  long long g = (n + t - 1) / t;
  return (int)(g > 65535 * 16 ? 65535 * 16 : (g < 1 ? 1 : g));
}

}  // namespace

cudaError_t net_forward(const NetParams& w, const int8_t* spins, int B, int Ly, int Lx, float* h1, float* h2,
                        float* out, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  const long long n1 = (long long)B * kNetC * Ly * Lx;
  conv_fwd_kernel<<<blocks(n1), 256, 0, st>>>(nullptr, spins, 1, w.w1, w.b1, h1, kNetC, B, Ly, Lx, 1);
  conv_fwd_kernel<<<blocks(n1), 256, 0, st>>>(h1, nullptr, kNetC, w.w2, w.b2, h2, kNetC, B, Ly, Lx, 1);
  conv_fwd_kernel<<<blocks((long long)B * 2 * Ly * Lx), 256, 0, st>>>(h2, nullptr, kNetC, w.w3, w.b3, out, 2, B, Ly,
                                                                      Lx, 0);
  return cudaGetLastError();
}

cudaError_t net_train_step(const NetParams& w, const NetParams& g, float* m, float* v, int nparam, int t, float lr,
                           const int8_t* spins, const float* rho, int B, int Ly, int Lx, float* h1, float* h2,
                           float* out, float* d2, float* d1, double* acc, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  PV_CUDA(net_forward(w, spins, B, Ly, Lx, h1, h2, out, st));
  const long long no = (long long)B * 2 * Ly * Lx, nh = (long long)B * kNetC * Ly * Lx;
  PV_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  loss_kernel<<<blocks(no), 256, 0, st>>>(out, spins, rho, B, Ly, Lx, nullptr, acc, 0);
  loss_kernel<<<blocks(no), 256, 0, st>>>(out, spins, rho, B, Ly, Lx, out, acc, 1);  // dout in place
  // layer 3
  conv_bwd_w_kernel<<<2 * (kNetC + 1), 256, 0, st>>>(out, 2, h2, nullptr, kNetC, g.w3, g.b3, B, Ly, Lx);
  conv_bwd_in_kernel<<<blocks(nh), 256, 0, st>>>(out, 2, w.w3, h2, d2, kNetC, B, Ly, Lx);
  // layer 2
  conv_bwd_w_kernel<<<kNetC * (kNetC + 1), 256, 0, st>>>(d2, kNetC, h1, nullptr, kNetC, g.w2, g.b2, B, Ly, Lx);
  conv_bwd_in_kernel<<<blocks(nh), 256, 0, st>>>(d2, kNetC, w.w2, h1, d1, kNetC, B, Ly, Lx);
  // layer 1 (input = spins)
  conv_bwd_w_kernel<<<kNetC * 2, 256, 0, st>>>(d1, kNetC, nullptr, spins, 1, g.w1, g.b1, B, Ly, Lx);
  const float b1 = 0.9f, b2 = 0.999f;
  adam_kernel<<<(nparam + 255) / 256, 256, 0, st>>>(w.w1, g.w1, m, v, nparam, lr, b1, b2,
                                                     1.f - powf(b1, (float)t), 1.f - powf(b2, (float)t), 1e-8f);
  return cudaGetLastError();
}

cudaError_t propose_moves(const float* logits, const int8_t* spins, int8_t* prop, int C, int Ly, int Lx, int k,
                          unsigned long long key, const unsigned long long* sweep, int* move, double* lq,
                          unsigned chain_base, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  propose_kernel<<<(C + 127) / 128, 128, 0, st>>>(logits, spins, prop, C, Ly, Lx, k, key, sweep, move, lq,
                                                  chain_base);
  return cudaGetLastError();
}

cudaError_t reverse_logq(const float* logits, const int8_t* prop, int C, int Ly, int Lx, int k, const int* move,
                         double* lq_rev, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  reverse_kernel<<<(C + 127) / 128, 128, 0, st>>>(logits, prop, C, Ly, Lx, k, move, lq_rev);
  return cudaGetLastError();
}

cudaError_t accept_moves(int8_t* spins, const int8_t* prop, int C, int N, const int* move, const float* den,
                         const float* num, long long bs, const int* e_den, const int* e_num, const double* lq_fwd,
                         const double* lq_rev, unsigned long long key, const unsigned long long* sweep, int k,
                         int Lb, double* tr_rho, double* tr_dlq, int8_t* tr_dec, unsigned long long* counters,
                         unsigned* status, unsigned chain_base, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  accept_kernel<<<(C + 127) / 128, 128, 0, st>>>(spins, prop, C, N, move, den, num, bs, e_den, e_num, lq_fwd, lq_rev,
                                                 key, sweep, k, Lb, tr_rho, tr_dlq, tr_dec, counters, status,
                                                 chain_base);
  return cudaGetLastError();
}

}  // namespace pv
