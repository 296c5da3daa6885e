// Per-chain kernels of the VMC-PEPS hot path (arXiv:1908.09359).
//
// Scaling: environments are rescaled by exact powers of two (the exponent of
// their largest entry), so a rescaled environment differs from the unscaled
// one by no rounding at all; exponents are summed per chain where a log
// amplitude is needed.  Boundary MPSs are normalised by their 2-norm and the
// log of the norm is carried in float64 (App. B keeps |U_k> bounded this way).
#include "kernels.cuh"

namespace pv {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
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

__device__ __forceinline__ double uniform24(unsigned w) { return (double)(w >> 8) * (1.0 / 16777216.0); }

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T tot = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += red[i];
  return tot;
}

__device__ __forceinline__ float block_max(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float m = 0.f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
  return m;
}

// Per-chain vector primitives of the block reductions: 16-byte loads when both arrays
// start on a 16-byte boundary and n is a multiple of 4, else scalar loads.
__device__ __forceinline__ bool vec4_ok(const void* x, const void* y, int n) {
  return (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) == 0) && (n & 3) == 0;
}
// One step of Dot2 (Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci.
// Comput. 26, 2005): the product is split exactly into p + e (TwoProduct with a fused
// multiply-add), p is added to the running sum hi with Knuth's TwoSum, and both rounding
// errors go to lo.  hi + lo then carries about twice float32's precision -- as accurate
// as float64 accumulation of the exact products, which matters where the sum cancels
// (amplitude closures, ratios), without float64 arithmetic, which runs at a small
// fraction of the float32 rate on this GPU.  The _rn intrinsics are never contracted
// into fused multiply-adds, so each transformation stays error-free.
__device__ __forceinline__ void dot2_step(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bv = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}
// this thread's part of sum_i x[i] y[i] (Dot2 in float32 pairs, returned in float64)
__device__ __forceinline__ double part_dot(const float* x, const float* y, int n) {
  float hi = 0.f, lo = 0.f;
  if (vec4_ok(x, y, n)) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* y4 = reinterpret_cast<const float4*>(y);
    for (int i = threadIdx.x; i < (n >> 2); i += blockDim.x) {
      const float4 a = x4[i], b = y4[i];
      dot2_step(hi, lo, a.x, b.x);
      dot2_step(hi, lo, a.y, b.y);
      dot2_step(hi, lo, a.z, b.z);
      dot2_step(hi, lo, a.w, b.w);
    }
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dot2_step(hi, lo, x[i], y[i]);
  }
  return (double)hi + (double)lo;
}
// this thread's part of max |x[i]|; *bad set when an entry is not finite
__device__ __forceinline__ float part_maxabs(const float* x, int n, bool* bad) {
  float mx = 0.f;
  bool nf = false;
  if (vec4_ok(x, x, n)) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (int i = threadIdx.x; i < (n >> 2); i += blockDim.x) {
      const float4 a = x4[i];
      nf |= !isfinite(a.x) || !isfinite(a.y) || !isfinite(a.z) || !isfinite(a.w);
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
    }
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float v = x[i];
      nf |= !isfinite(v);
      mx = fmaxf(mx, fabsf(v));
    }
  }
  if (bad) *bad = nf;
  return mx;
}
// dst[i] = src[i] * f (dst may equal src)
__device__ __forceinline__ void scale_copy(float* dst, const float* src, int n, float f) {
  if (vec4_ok(dst, src, n)) {
    float4* d4 = reinterpret_cast<float4*>(dst);
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (int i = threadIdx.x; i < (n >> 2); i += blockDim.x) {
      const float4 a = s4[i];
      d4[i] = make_float4(a.x * f, a.y * f, a.z * f, a.w * f);
    }
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i] * f;
  }
}

__global__ void fill_kernel(float* p, long long n, float v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void set_u64_kernel(unsigned long long* p, unsigned long long v) { *p = v; }
__global__ void fill_d_kernel(double* p, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void gather_kernel(float* dst, const double* src, const int* map, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[map[i]];
}

// Scale x (and x2, x3 by the same factor) by 2^-e, e the exponent of max|x|.  Up to
// kNormRegF4 * 4 * kThreads elements (every three-line environment of Dc <= 32, D <= 8)
// are read once into registers and written back scaled; larger arrays take a second
// pass.
constexpr int kNormRegF4 = 8;
__global__ void normalize_pow2_kernel(float* x, long long bs, int n, float* x2, long long bs2, int n2, float* x3,
                                      long long bs3, int n3, int* exps, unsigned* status) {
  __shared__ float red[kThreads / 32];
  const int b = blockIdx.x;
  float* xb = x + b * bs;
  bool bad = false;
  const bool in_regs = vec4_ok(xb, xb, n) && n <= kNormRegF4 * 4 * kThreads;
  float4 r[kNormRegF4];
  float mx = 0.f;
  if (in_regs) {
    const float4* x4 = reinterpret_cast<const float4*>(xb);
#pragma unroll
    for (int i = 0; i < kNormRegF4; ++i) {
      const int j = threadIdx.x + i * kThreads;
      r[i] = j < (n >> 2) ? x4[j] : make_float4(0.f, 0.f, 0.f, 0.f);
      bad |= !isfinite(r[i].x) || !isfinite(r[i].y) || !isfinite(r[i].z) || !isfinite(r[i].w);
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(r[i].x), fabsf(r[i].y)), fmaxf(fabsf(r[i].z), fabsf(r[i].w))));
    }
  } else {
    mx = part_maxabs(xb, n, &bad);
  }
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
    return;
  }
  mx = block_max(mx, red);
  if (mx == 0.f) {
    if (threadIdx.x == 0) atomicOr(status, ST_ZEROPSI);
    return;
  }
  int e;
  frexpf(mx, &e);
  const float s = ldexpf(1.f, -e);
  if (in_regs) {
    float4* x4 = reinterpret_cast<float4*>(xb);
#pragma unroll
    for (int i = 0; i < kNormRegF4; ++i) {
      const int j = threadIdx.x + i * kThreads;
      if (j < (n >> 2)) x4[j] = make_float4(r[i].x * s, r[i].y * s, r[i].z * s, r[i].w * s);
    }
  } else {
    scale_copy(xb, xb, n, s);
  }
  if (x2) scale_copy(x2 + b * bs2, x2 + b * bs2, n2, s);
  if (x3) scale_copy(x3 + b * bs3, x3 + b * bs3, n3, s);
  if (exps && threadIdx.x == 0) exps[b] += e;
}

__global__ void mps_normalize_kernel(float* x, long long bs, int n, const int* exps, const double* log_in,
                                     double* log_out, unsigned* status) {
  __shared__ double red[kThreads / 32];
  const int b = blockIdx.x;
  float* xb = x + b * bs;
  double s = part_dot(xb, xb, n);
  s = block_sum(s, red);
  if (!(s > 0.0) || !isfinite(s)) {
    if (threadIdx.x == 0) atomicOr(status, isfinite(s) ? ST_ZEROPSI : ST_NONFINITE);
    return;
  }
  const double nrm = sqrt(s);
  const float inv = (float)(1.0 / nrm);
  scale_copy(xb, xb, n, inv);
  if (threadIdx.x == 0) {
    const double li = log_in ? log_in[b] : 0.0;
    log_out[b] = li + log(nrm) + (exps ? exps[b] * 0.6931471805599453 : 0.0);
  }
}

// L(m) of the chosen configuration (src), scaled by a power of two to max |.| in [1/2, 1).
__device__ void select_left(const MetropolisArgs& a, int b, const float* src, float* redf) {
  float mx = part_maxabs(src, a.n, nullptr);
  mx = block_max(mx, redf);
  float s = 1.f;
  if (mx > 0.f && isfinite(mx)) {
    int e;
    frexpf(mx, &e);
    s = ldexpf(1.f, -e);
  }
  scale_copy(a.out + b * a.bs_out, src, a.n, s);
}

// Sequential Metropolis step on one pair (Eq. (9)) for every chain.
__global__ void metropolis_kernel(const MetropolisArgs a) {
  __shared__ double red[kThreads / 32];
  __shared__ float redf[kThreads / 32];
  __shared__ int acc_s;
  const int b = blockIdx.x;
  const float* cur = a.cur + b * a.bs_cur;
  const float* Rc = a.Rcur + b * a.bs_Rcur;
  const float* fl = a.flip + b * a.bs_flip;
  const float* Rf = a.Rflip + b * a.bs_Rflip;
  int8_t* sp = a.spins + b * a.spin_stride;
  const bool anti = sp[a.site_a] != sp[a.site_b];
  double den = part_dot(cur, Rc, a.n), num = 0.0;
  den = block_sum(den, red);
  if (anti) {
    num = part_dot(fl, Rf, a.n);
    num = block_sum(num, red);
  }
  if (a.rho_out) {  // symmetrised sampling: the ratio only, decided per pair
    if (threadIdx.x == 0) {
      double rho = 0.0;
      if (den == 0.0) atomicOr(a.status, ST_ZEROPSI);
      else if (anti) rho = num / den;
      if (!isfinite(rho)) {
        atomicOr(a.status, ST_NONFINITE);
        rho = 0.0;
      }
      a.rho_out[b] = rho;
    }
    return;
  }
  if (threadIdx.x == 0) {
    int accept = 0;
    if (den == 0.0) atomicOr(a.status, ST_ZEROPSI);
    if (anti) {
      double rho = 0.0;
      if (den != 0.0) {
        rho = num / den;
        if (!isfinite(rho)) {
          atomicOr(a.status, ST_NONFINITE);
        } else {
          const uint4 w = philox4x32_10(
              make_uint4((unsigned)b + a.chain_base, (unsigned)*a.sweep, (unsigned)a.bond, kTagMetropolis),
              make_uint2((unsigned)(a.key & 0xffffffffull), (unsigned)(a.key >> 32)));
          const double u = uniform24(w.x);
          const double p = fmin(1.0, rho * rho);
          accept = (u < p) ? 1 : 0;
        }
      }
      if (accept) {
        sp[a.site_a] = (int8_t)-sp[a.site_a];
        sp[a.site_b] = (int8_t)-sp[a.site_b];
      }
      atomicAdd(&a.counters[0], 1ull);
      if (accept) atomicAdd(&a.counters[1], 1ull);
      if (a.trace_ratio) a.trace_ratio[b * a.trace_stride + a.bond] = rho;
      if (a.trace_dec) a.trace_dec[b * a.trace_stride + a.bond] = (int8_t)accept;
    } else {
      if (a.trace_ratio) a.trace_ratio[b * a.trace_stride + a.bond] = 0.0;
      if (a.trace_dec) a.trace_dec[b * a.trace_stride + a.bond] = (int8_t)-1;
    }
    acc_s = accept;
  }
  __syncthreads();
  select_left(a, b, acc_s ? fl : cur, redf);
}

// Symmetrised decision of pair p = b mod pairs, taken identically by the blocks of both
// chains of the pair (each applies it to its own spins, L(m) and copy of w).
__global__ void phi_decide_kernel(const MetropolisArgs a) {
  __shared__ float redf[kThreads / 32];
  __shared__ int acc_s;
  const int b = blockIdx.x;
  const int p = b % a.pairs;
  int8_t* sp = a.spins + b * a.spin_stride;
  if (threadIdx.x == 0) {
    int accept = 0;
    const double r1 = a.rho_out[p], r2 = a.rho_out[p + a.pairs];
    const double w = a.phi_w[b];
    if (sp[a.site_a] != sp[a.site_b]) {
      const double num = r1 + w * r2, den = 1.0 + w;
      if (den == 0.0) atomicOr(a.status, ST_ZEROPSI);
      const double q = den != 0.0 ? (num / den) * (num / den) : 0.0;
      if (!isfinite(q)) {
        atomicOr(a.status, ST_NONFINITE);
      } else if (den != 0.0) {
        const uint4 u4 = philox4x32_10(
            make_uint4((unsigned)p + a.chain_base, (unsigned)*a.sweep, (unsigned)a.bond, kTagMetropolis),
            make_uint2((unsigned)(a.key & 0xffffffffull), (unsigned)(a.key >> 32)));
        accept = (uniform24(u4.x) < fmin(1.0, q)) ? 1 : 0;
      }
      if (accept) {
        if (r1 == 0.0) {  // Psi(S') = 0: w of the new configuration is undefined
          atomicOr(a.status, ST_NONFINITE);
        } else {
          a.phi_w[b] = w * r2 / r1;
        }
        sp[a.site_a] = (int8_t)-sp[a.site_a];
        sp[a.site_b] = (int8_t)-sp[a.site_b];
      }
      if (b < a.pairs) {
        atomicAdd(&a.counters[0], 1ull);
        if (accept) atomicAdd(&a.counters[1], 1ull);
      }
      if (a.trace_ratio) a.trace_ratio[b * a.trace_stride + a.bond] = b < a.pairs ? r1 : r2;
      if (a.trace_dec) a.trace_dec[b * a.trace_stride + a.bond] = (int8_t)accept;
    } else {
      if (a.trace_ratio) a.trace_ratio[b * a.trace_stride + a.bond] = 0.0;
      if (a.trace_dec) a.trace_dec[b * a.trace_stride + a.bond] = (int8_t)-1;
    }
    acc_s = accept;
  }
  __syncthreads();
  select_left(a, b, acc_s ? a.flip + b * a.bs_flip : a.cur + b * a.bs_cur, redf);
}

__global__ void phi_combine_kernel(const double* logpsi, const int8_t* sign, const double* eloc, int batch,
                                   int pairs, double* w, double* eloc_phi, double* wt, unsigned* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const int p = b % pairs, q = p + pairs;
  if (sign[p] == 0 || sign[q] == 0) {
    atomicOr(status, ST_ZEROPSI);
    return;
  }
  const double wv = (double)(sign[p] * sign[q]) * exp(logpsi[q] - logpsi[p]);
  if (!isfinite(wv)) atomicOr(status, ST_NONFINITE);
  if (1.0 + wv == 0.0) atomicOr(status, ST_ZEROPSI);
  w[b] = wv;
  if (eloc) {
    eloc_phi[b] = (eloc[p] + wv * eloc[q]) / (1.0 + wv);
    wt[b] = (b < pairs ? 1.0 : wv) / (1.0 + wv);
  }
}

__global__ void dot_kernel(const float* a, long long bsa, const float* bb, long long bsb, int n, double* out,
                           unsigned* status) {
  __shared__ double red[kThreads / 32];
  const int b = blockIdx.x;
  double s = part_dot(a + b * bsa, bb + b * bsb, n);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    out[b] = s;
    if (s == 0.0) atomicOr(status, ST_ZEROPSI);
    if (!isfinite(s)) atomicOr(status, ST_NONFINITE);
  }
}

__global__ void ratio_accum_kernel(const float* a, long long bsa, const float* bb, long long bsb, int n,
                                   const double* den, const int8_t* spins, long long spin_stride, int si, int sj,
                                   double halfJ, double* eloc, unsigned* status, float* rho_out, long long rho_stride,
                                   long long rho_idx) {
  __shared__ double red[kThreads / 32];
  const int b = blockIdx.x;
  const int8_t* sp = spins + b * spin_stride;
  if (sp[si] == sp[sj]) return;  // no off-diagonal element for a parallel pair
  double s = part_dot(a + b * bsa, bb + b * bsb, n);
  s = block_sum(s, red);
  if (threadIdx.x == 0) {
    const double r = s / den[b];
    if (!isfinite(r)) atomicOr(status, ST_NONFINITE);
    eloc[b] += halfJ * r;
    if (rho_out) rho_out[b * rho_stride + rho_idx] = (float)r;
  }
}

__global__ void eloc_diag_kernel(const int8_t* spins, int Ly, int Lx, double J1, double J2, double* eloc,
                                 int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const int8_t* s = spins + (long long)b * Ly * Lx;
  double e = 0.0;
  for (int k = 0; k < Ly; ++k)
    for (int m = 0; m < Lx; ++m) {
      const int v = s[k * Lx + m];
      if (m + 1 < Lx) e += J1 * 0.25 * v * s[k * Lx + m + 1];
      if (k + 1 < Ly) e += J1 * 0.25 * v * s[(k + 1) * Lx + m];
      if (J2 != 0.0 && k + 1 < Ly && m + 1 < Lx) {
        e += J2 * 0.25 * v * s[(k + 1) * Lx + m + 1];
        e += J2 * 0.25 * s[k * Lx + m + 1] * s[(k + 1) * Lx + m];
      }
    }
  eloc[b] = e;
}

__global__ void logpsi_kernel(const float* x, long long bs, const int* exps, const double* logT, const double* logB,
                              double* logpsi, int8_t* sign, int batch, unsigned* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const float v = x[b * bs];
  if (v == 0.f) atomicOr(status, ST_ZEROPSI);
  logpsi[b] = logT[b] + logB[b] + exps[b] * 0.6931471805599453 + log(fabs((double)v));
  sign[b] = v < 0.f ? (int8_t)-1 : (int8_t)1;
}

__global__ void grad_accum_kernel(const float* G, long long bsG, long long Ph, const int* elem_site,
                                  const long long* site_half_off, const long long* site_full_off,
                                  const int* site_size, const int* site_spin, const int8_t* spins,
                                  long long spin_stride, const double* eloc, int batch, double* sumG,
                                  double* sumGE, const double* wt) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= Ph) return;
  const int j = elem_site[e];
  const long long local = e - site_half_off[j];
  const int si = site_spin[j];
  double g0 = 0, g1 = 0, ge0 = 0, ge1 = 0;
  for (int c = 0; c < batch; ++c) {
    const double v = wt ? wt[c] * G[c * bsG + e] : (double)G[c * bsG + e];
    const double E = eloc[c];
    if (spins[c * spin_stride + si] > 0) {
      g0 += v;
      ge0 += v * E;
    } else {
      g1 += v;
      ge1 += v * E;
    }
  }
  const long long f0 = site_full_off[j] + local, f1 = f0 + site_size[j];
  sumG[f0] += g0;
  sumG[f1] += g1;
  sumGE[f0] += ge0;
  sumGE[f1] += ge1;
}

__global__ void energy_accum_kernel(const double* eloc, int batch, double* sums) {
  __shared__ double red[kThreads / 32];
  double s = 0, s2 = 0;
  for (int i = threadIdx.x; i < batch; i += blockDim.x) {
    s += eloc[i];
    s2 += eloc[i] * eloc[i];
  }
  s = block_sum(s, red);
  s2 = block_sum(s2, red);
  if (threadIdx.x == 0) {
    sums[0] += s;
    sums[1] += s2;
    sums[2] += batch;
  }
}

__global__ void grad_final_kernel(const double* sumG, const double* sumGE, const double* sums, long long P,
                                  double* grad) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= P) return;
  const double n = sums[2];
  const double E = sums[0] / n;
  grad[i] = sumGE[i] / n - (sumG[i] / n) * E;
}

__global__ void sgd_kernel(double* master, const double* grad, long long P, double delta, unsigned long long key,
                           unsigned long long step) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= P) return;
  const uint4 w = philox4x32_10(make_uint4((unsigned)(i & 0xffffffffll), (unsigned)(i >> 32), (unsigned)step, kTagUpdate),
                                make_uint2((unsigned)(key & 0xffffffffull), (unsigned)(key >> 32)));
  const double r = uniform24(w.x);
  const double g = grad[i];
  const double sg = g > 0.0 ? 1.0 : (g < 0.0 ? -1.0 : 0.0);
  master[i] -= r * delta * sg;
}

// i-th bond of the sequential order: vertical (k,m)-(k+1,m) first (columns left to
// right, top to bottom), then horizontal (k,m)-(k,m+1) (rows top to bottom).
__device__ __forceinline__ void bond_sites(int i, int Ly, int Lx, int& p, int& q) {
  const int nv = Lx * (Ly - 1);
  if (i < nv) {
    const int m = i / (Ly - 1), k = i % (Ly - 1);
    p = k * Lx + m;
    q = (k + 1) * Lx + m;
  } else {
    const int j = i - nv, k = j / (Lx - 1), m = j % (Lx - 1);
    p = k * Lx + m;
    q = k * Lx + m + 1;
  }
}

__global__ void random_propose_kernel(const RandomArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.C) return;
  const int N = a.Ly * a.Lx, nb = 2 * N - a.Ly - a.Lx;
  const int8_t* s = a.spins + (long long)c * N;
  int8_t* t = a.prop + (long long)c * N;
  for (int i = 0; i < N; ++i) t[i] = s[i];
  int K = 0;
  for (int i = 0; i < nb; ++i) {
    int p, q;
    bond_sites(i, a.Ly, a.Lx, p, q);
    K += s[p] != s[q];
  }
  a.Ka[c] = K;
  a.Kb[c] = 0;
  a.bond[c] = -1;
  if (K == 0) return;
  const uint4 w = philox4x32_10(make_uint4((unsigned)c + a.chain_base, (unsigned)*a.sweep, (unsigned)a.attempt,
                                           kTagRandom),
                                make_uint2((unsigned)(a.key & 0xffffffffull), (unsigned)(a.key >> 32)));
  const int pick = (int)(((unsigned long long)(w.x >> 8) * (unsigned long long)K) >> 24);
  int seen = 0;
  for (int i = 0; i < nb; ++i) {
    int p, q;
    bond_sites(i, a.Ly, a.Lx, p, q);
    if (s[p] == s[q]) continue;
    if (seen++ == pick) {
      t[p] = s[q];
      t[q] = s[p];
      a.bond[c] = i;
      break;
    }
  }
  int Kb = 0;
  for (int i = 0; i < nb; ++i) {
    int p, q;
    bond_sites(i, a.Ly, a.Lx, p, q);
    Kb += t[p] != t[q];
  }
  a.Kb[c] = Kb;
}

__global__ void random_accept_kernel(const RandomArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.C) return;
  const int N = a.Ly * a.Lx;
  int dec = -1;
  double rho = 0.0;
  if (a.Ka[c] > 0) {
    const uint4 w = philox4x32_10(make_uint4((unsigned)c + a.chain_base, (unsigned)*a.sweep, (unsigned)a.attempt,
                                             kTagRandom),
                                  make_uint2((unsigned)(a.key & 0xffffffffull), (unsigned)(a.key >> 32)));
    const double r = uniform24(w.y);
    rho = (double)(a.sg_new[c] * a.sg_cur[c]) * exp(a.lp_new[c] - a.lp_cur[c]);
    if (!isfinite(rho)) atomicOr(a.status, ST_NONFINITE);
    const double p = fmin(1.0, rho * rho * (double)a.Ka[c] / (double)a.Kb[c]);
    dec = r < p ? 1 : 0;
    atomicAdd(&a.counters[0], 1ull);
    if (dec) {
      atomicAdd(&a.counters[1], 1ull);
      for (int i = 0; i < N; ++i) a.spins[(long long)c * N + i] = a.prop[(long long)c * N + i];
      a.lp_cur[c] = a.lp_new[c];
      a.sg_cur[c] = a.sg_new[c];
    }
  }
  if (a.tr_bond) {
    const long long o = (long long)c * a.tr_stride + a.attempt;
    a.tr_bond[o] = a.bond[c];
    a.tr_ratio[o] = rho;
    a.tr_dec[o] = (int8_t)dec;
  }
}

inline int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g > 1048576 ? 1048576 : (g < 1 ? 1 : g));
}

}  // namespace

bool g_dry_run = false;

cudaError_t k_fill(float* p, long long n, float v, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  fill_kernel<<<grid_for(n), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}
cudaError_t k_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  set_u64_kernel<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}
cudaError_t k_fill_d(double* p, long long n, double v, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  fill_d_kernel<<<grid_for(n), 256, 0, st>>>(p, n, v);
  return cudaGetLastError();
}
cudaError_t k_gather_f32(float* dst, const double* src, const int* map, long long n, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  gather_kernel<<<grid_for(n), 256, 0, st>>>(dst, src, map, n);
  return cudaGetLastError();
}
cudaError_t k_normalize_pow2(float* x, long long bs, int n, float* x2, long long bs2, int n2, float* x3,
                             long long bs3, int n3, int* exps, int batch, unsigned* status, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  normalize_pow2_kernel<<<batch, kThreads, 0, st>>>(x, bs, n, x2, bs2, n2, x3, bs3, n3, exps, status);
  return cudaGetLastError();
}
cudaError_t k_mps_normalize(float* x, long long bs, int n, const int* exps, const double* log_in, double* log_out,
                            int batch, unsigned* status, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  mps_normalize_kernel<<<batch, kThreads, 0, st>>>(x, bs, n, exps, log_in, log_out, status);
  return cudaGetLastError();
}
cudaError_t k_metropolis(const MetropolisArgs& a, int batch, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  metropolis_kernel<<<batch, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t k_phi_decide(const MetropolisArgs& a, int batch, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  phi_decide_kernel<<<batch, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t k_phi_combine(const double* logpsi, const int8_t* sign, const double* eloc, int batch, int pairs,
                          double* w, double* eloc_phi, double* wt, unsigned* status, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  phi_combine_kernel<<<(batch + 127) / 128, 128, 0, st>>>(logpsi, sign, eloc, batch, pairs, w, eloc_phi, wt, status);
  return cudaGetLastError();
}
cudaError_t k_dot(const float* a, long long bsa, const float* b, long long bsb, int n, double* out, int batch,
                  unsigned* status, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  dot_kernel<<<batch, kThreads, 0, st>>>(a, bsa, b, bsb, n, out, status);
  return cudaGetLastError();
}
cudaError_t k_ratio_accum(const float* a, long long bsa, const float* b, long long bsb, int n, const double* den,
                          const int8_t* spins, long long spin_stride, int si, int sj, double halfJ, double* eloc,
                          int batch, unsigned* status, cudaStream_t st, float* rho_out, long long rho_stride,
                          long long rho_idx) {
  if (g_dry_run) return cudaSuccess;
  ratio_accum_kernel<<<batch, kThreads, 0, st>>>(a, bsa, b, bsb, n, den, spins, spin_stride, si, sj, halfJ, eloc,
                                                 status, rho_out, rho_stride, rho_idx);
  return cudaGetLastError();
}
cudaError_t k_eloc_diag(const int8_t* spins, int Ly, int Lx, double J1, double J2, double* eloc, int batch,
                        cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  eloc_diag_kernel<<<(batch + 127) / 128, 128, 0, st>>>(spins, Ly, Lx, J1, J2, eloc, batch);
  return cudaGetLastError();
}
cudaError_t k_logpsi(const float* x, long long bs, const int* exps, const double* logT, const double* logB,
                     double* logpsi, int8_t* sign, int batch, unsigned* status, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  logpsi_kernel<<<(batch + 127) / 128, 128, 0, st>>>(x, bs, exps, logT, logB, logpsi, sign, batch, status);
  return cudaGetLastError();
}
cudaError_t k_grad_accum(const float* G, long long bsG, long long Ph, const int* elem_site,
                         const long long* site_half_off, const long long* site_full_off, const int* site_size,
                         const int* site_spin, const int8_t* spins, long long spin_stride, const double* eloc,
                         int batch, double* sumG, double* sumGE, cudaStream_t st, const double* wt) {
  if (g_dry_run) return cudaSuccess;
  grad_accum_kernel<<<(int)((Ph + 255) / 256), 256, 0, st>>>(G, bsG, Ph, elem_site, site_half_off, site_full_off,
                                                             site_size, site_spin, spins, spin_stride, eloc, batch,
                                                             sumG, sumGE, wt);
  return cudaGetLastError();
}
cudaError_t k_energy_accum(const double* eloc, int batch, double* sums, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  energy_accum_kernel<<<1, kThreads, 0, st>>>(eloc, batch, sums);
  return cudaGetLastError();
}
cudaError_t k_grad_final(const double* sumG, const double* sumGE, const double* sums, long long P, double* grad,
                         cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  grad_final_kernel<<<(int)((P + 255) / 256), 256, 0, st>>>(sumG, sumGE, sums, P, grad);
  return cudaGetLastError();
}
cudaError_t k_random_propose(const RandomArgs& a, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  random_propose_kernel<<<(a.C + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t k_random_accept(const RandomArgs& a, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  random_accept_kernel<<<(a.C + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t k_sgd(double* master, const double* grad, long long P, double delta, unsigned long long key,
                  unsigned long long step, cudaStream_t st) {
  if (g_dry_run) return cudaSuccess;
  sgd_kernel<<<(int)((P + 255) / 256), 256, 0, st>>>(master, grad, P, delta, key, step);
  return cudaGetLastError();
}

}  // namespace pv
