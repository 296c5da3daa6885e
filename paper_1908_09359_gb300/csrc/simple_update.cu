// Simple-update imaginary-time evolution (App. A of arXiv:1908.09359), float64.
//
// The PEPS is held as site tensors B (packed like the Monte Carlo tensors: per site
// [2][Dl][Dr][Du][Dd], open legs of dimension 1) and one vector lambda of length D on
// every nearest-neighbour link.  One launch applies the evolution operators of one
// group of updates that share no site, one CTA per update:
//
//   NN bond (sites 1, 2): both tensors, with the lambdas of their three outer legs
//   absorbed, are reduced by a Householder QR (rows: outer legs, columns: bond leg and
//   spin, diag(R) >= 0); Theta[(x,s1'),(y,s2')] = sum R1[x,b,s1] lambda[b] R2[y,b,s2]
//   G[s1',s2',s1,s2]; a truncated SVD of Theta gives the new bond lambda (unit norm) and
//   the new R factors; B1 = Q1 U, B2 = Q2 V with the outer lambdas divided out.
//
//   NNN pair (sites 1, 3) through the corner site 2 (steps (b)-(h) of App. A's figure):
//   QR of B1 and B3 with their outer lambdas; T_a = R1 . (B2 with its outer lambdas and
//   both link lambdas) . R3 with the gate on the spins of 1 and 3; a truncated SVD of
//   T_a gives lambda(1,2), the new R1 and T_b; a truncated SVD of lambda(1,2) T_b gives
//   T_c, lambda(2,3) and the new L3; B1 = Q1 R1', B3 = Q3 L3', B2 = T_c, each with the
//   inverse lambdas of its outer legs (and lambda(1,2)^-1 on B2's leg to 1) divided out.
//
// Truncated SVDs: the Gram matrix of the short side (<= 32 x 32) is diagonalised by
// cyclic Jacobi rotations (round-robin ordering, 16 rotations at a time), singular values
// are the square roots of its eigenvalues in descending order, the other side's vectors
// follow by one product.  The count kept is min(D, #{sigma > 1e-7 sigma_max}); missing
// entries are zero.  Each singular vector pair is signed so that the left vector's
// largest-magnitude entry is positive.  Inverse lambdas: 1/lambda above 1e-14 of the
// largest entry, else 0.
//
// The host loop (pepsvmc_simple_update) runs the Trotter order of one step -- horizontal
// NN bonds by parity of m, vertical by parity of k (tau), then with J2 != 0 the two
// diagonals of every plaquette through each of their two corners in four parity groups
// of plaquettes (tau/2 each) -- and stops when the mean relative change of the lambdas
// over a step falls below tol.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "pepsvmc.h"

namespace pv {
namespace {

constexpr int kSuThreads = 256;
constexpr int kSuMaxD = 8;
constexpr int kMaxRows = kSuMaxD * kSuMaxD * kSuMaxD;  // outer legs of a site
constexpr int kMaxCols = 2 * kSuMaxD;                  // (bond leg, spin)
constexpr int kMaxSide = 32;                           // short side of every SVD
constexpr int kJacobiSweeps = 40;

struct SuLattice {
  int Ly, Lx, D;
  double* B;                 // packed site tensors
  const long long* site_off; // [Ly*Lx]
  double* lam_h;             // [Ly][Lx-1][D]
  double* lam_v;             // [Ly-1][Lx][D]
};

// leg indices: 0 l, 1 r, 2 u, 3 d
__device__ __forceinline__ int leg_dim(const SuLattice& L, int k, int m, int g) {
  const int D = L.D;
  switch (g) {
    case 0: return m == 0 ? 1 : D;
    case 1: return m == L.Lx - 1 ? 1 : D;
    case 2: return k == 0 ? 1 : D;
    default: return k == L.Ly - 1 ? 1 : D;
  }
}
// lambda vector on leg g of site (k, m), nullptr on an open leg
__device__ __forceinline__ double* leg_lam(const SuLattice& L, int k, int m, int g) {
  const int D = L.D;
  switch (g) {
    case 0: return m > 0 ? L.lam_h + ((long long)k * (L.Lx - 1) + (m - 1)) * D : nullptr;
    case 1: return m < L.Lx - 1 ? L.lam_h + ((long long)k * (L.Lx - 1) + m) * D : nullptr;
    case 2: return k > 0 ? L.lam_v + ((long long)(k - 1) * L.Lx + m) * D : nullptr;
    default: return k < L.Ly - 1 ? L.lam_v + ((long long)k * L.Lx + m) * D : nullptr;
  }
}
// element stride of leg g in the packed site layout [s][l][r][u][d]
__device__ __forceinline__ long long leg_stride(const SuLattice& L, int k, int m, int g) {
  long long st = 1;
  for (int h = 3; h > g; --h) st *= leg_dim(L, k, m, h);
  return st;
}
// The three outer legs of a site (all but `bond`, in l, r, u, d order) with their
// dimensions and element strides, and the bond leg's stride.  Scalars only, so that no
// per-thread array is indexed by a run-time value.
struct Outer {
  int g0, g1, g2, d0, d1, d2;
  long long s0, s1, s2, sb, ss;
};
__device__ __forceinline__ Outer outer_of(const SuLattice& L, int k, int m, int bond) {
  Outer o;
  o.g0 = bond == 0 ? 1 : 0;
  o.g1 = bond <= 1 ? 2 : 1;
  o.g2 = bond <= 2 ? 3 : 2;
  o.d0 = leg_dim(L, k, m, o.g0);
  o.d1 = leg_dim(L, k, m, o.g1);
  o.d2 = leg_dim(L, k, m, o.g2);
  o.s0 = leg_stride(L, k, m, o.g0);
  o.s1 = leg_stride(L, k, m, o.g1);
  o.s2 = leg_stride(L, k, m, o.g2);
  o.sb = leg_stride(L, k, m, bond);
  o.ss = leg_stride(L, k, m, 0) * leg_dim(L, k, m, 0);
  return o;
}
__device__ __forceinline__ int dir_of(int k1, int m1, int k2, int m2) {
  if (k2 == k1) return m2 > m1 ? 1 : 0;
  return k2 > k1 ? 3 : 2;
}
__device__ __forceinline__ double inv_lam(const double* lam, int D, int i, double mx) {
  const double v = lam[i];
  return fabs(v) > 1e-14 * mx ? 1.0 / v : 0.0;
}
__device__ double lam_max(const double* lam, int D) {
  double mx = 0.0;
  for (int i = 0; i < D; ++i) mx = fmax(mx, fabs(lam[i]));
  return mx;
}

// Block reduction of n <= 32 partial sums (one per thread slot) into out[0..n).
__device__ void block_sums(double* part, int n, double* red, double* out) {
  // part: this thread's n partial sums (registers passed by pointer to a local array)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < n; ++c) {
    double v = part[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp * kMaxSide + c] = v;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    double s = 0.0;
    for (int w = 0; w < kSuThreads / 32; ++w) s += red[w * kMaxSide + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Householder QR with diag(R) >= 0 of A (m x n, row-major, shared memory), m <= kMaxRows,
// n <= kMaxCols.  Writes R (k x n, k = min(m, n), row-major, shared) and the thin Q
// (m x k, row-major) to Qg.  A is destroyed.
__device__ void blk_qr(double* A, int m, int n, double* R, double* Qg, double* red, double* tmp) {
  const int k = min(m, n);
  double* beta = tmp;          // [kMaxCols]
  double* sgn = tmp + kMaxCols; // [kMaxCols] sign flips of rows of R / columns of Q
  double* tot = tmp + 2 * kMaxCols;  // [kMaxSide]
  for (int j = 0; j < k; ++j) {
    double p[kMaxSide];
    p[0] = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) p[0] = fma(A[i * n + j], A[i * n + j], p[0]);
    block_sums(p, 1, red, tot);
    const double alpha = sqrt(tot[0]);
    const double x0 = A[j * n + j];
    const double sg = x0 >= 0.0 ? 1.0 : -1.0;
    const double bj = alpha == 0.0 ? 0.0 : 1.0 / (alpha * (alpha + fabs(x0)));
    __syncthreads();
    if (threadIdx.x == 0) {
      beta[j] = bj;
      // R_jj = -sg * alpha; the sign flip makes it >= 0
      sgn[j] = (bj != 0.0 && sg > 0.0) ? -1.0 : 1.0;
      R[j * n + j] = alpha;  // |R_jj| after the flip
      if (bj != 0.0) A[j * n + j] = x0 + sg * alpha;  // v_0
    }
    __syncthreads();
    if (bj == 0.0) continue;
    // w_c = beta * sum_i v_i A[i][c] for c > j
    const int nc = n - j - 1;
    for (int c = 0; c < nc; ++c) p[c] = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
      const double v = A[i * n + j];
      for (int c = 0; c < nc; ++c) p[c] = fma(v, A[i * n + j + 1 + c], p[c]);
    }
    if (nc > 0) block_sums(p, nc, red, tot);
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
      const double v = A[i * n + j];
      for (int c = 0; c < nc; ++c) A[i * n + j + 1 + c] = fma(-bj * tot[c], v, A[i * n + j + 1 + c]);
    }
    __syncthreads();
  }
  // R (rows sign-flipped so that the diagonal is >= 0)
  for (int idx = threadIdx.x; idx < k * n; idx += blockDim.x) {
    const int r = idx / n, c = idx % n;
    if (c > r) R[idx] = sgn[r] * A[r * n + c];
    else if (c < r) R[idx] = 0.0;
  }
  __syncthreads();
  // thin Q = H_0 ... H_{k-1} [I; 0], accumulated backwards, columns then sign-flipped
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) Qg[idx] = (idx / k == idx % k) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double bj = beta[j];
    if (bj == 0.0) continue;
    double p[kMaxSide];
    for (int c = 0; c < k; ++c) p[c] = 0.0;
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
      const double v = A[i * n + j];
      for (int c = j; c < k; ++c) p[c] = fma(v, Qg[i * k + c], p[c]);
    }
    block_sums(p, k, red, tot);
    for (int i = j + threadIdx.x; i < m; i += blockDim.x) {
      const double v = A[i * n + j];
      for (int c = j; c < k; ++c) Qg[i * k + c] = fma(-bj * tot[c], v, Qg[i * k + c]);
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < m * k; idx += blockDim.x) Qg[idx] *= sgn[idx % k];
  __syncthreads();
}

// Eigen-decomposition of the symmetric n x n matrix G (n <= 32, shared, destroyed) by
// cyclic Jacobi rotations in round-robin order.  Writes the eigenvalues in descending
// order to ev[0..n) and the matching eigenvectors as the columns of V (n x n, shared).
__device__ void blk_eig(double* G, int n, double* ev, double* V, double* rot, int* order) {
  const int np = n + (n & 1);  // a padding player sits out when n is odd
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  __shared__ int done;
  __syncthreads();
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    if (threadIdx.x == 0) {
      double off = 0.0, all = 0.0;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
          const double g2 = G[i * n + j] * G[i * n + j];
          all += g2;
          if (i != j) off += g2;
        }
      done = (off <= 1e-30 * all) ? 1 : 0;
    }
    __syncthreads();
    if (done) break;
    for (int r = 0; r < np - 1; ++r) {
      // round r of the circle method: player 0 fixed, the others rotate
      const int pairs = np / 2;
      if (threadIdx.x < pairs) {
        const int t = threadIdx.x;
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (np - 1); };
        int p = player(t), q = player(np - 1 - t);
        if (p > q) { const int s = p; p = q; q = s; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = G[p * n + q];
          if (apq != 0.0) {
            const double th = (G[q * n + q] - G[p * n + p]) / (2.0 * apq);
            const double tt = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(tt * tt + 1.0);
            s = tt * c;
          }
        }
        rot[4 * t] = p;
        rot[4 * t + 1] = q;
        rot[4 * t + 2] = c;
        rot[4 * t + 3] = s;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = threadIdx.x; idx < pairs * n; idx += blockDim.x) {
        const int t = idx / n, col = idx % n;
        const int p = (int)rot[4 * t], q = (int)rot[4 * t + 1];
        if (q >= n) continue;
        const double c = rot[4 * t + 2], s = rot[4 * t + 3];
        const double gp = G[p * n + col], gq = G[q * n + col];
        G[p * n + col] = c * gp - s * gq;
        G[q * n + col] = s * gp + c * gq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int idx = threadIdx.x; idx < pairs * n; idx += blockDim.x) {
        const int t = idx / n, row = idx % n;
        const int p = (int)rot[4 * t], q = (int)rot[4 * t + 1];
        if (q >= n) continue;
        const double c = rot[4 * t + 2], s = rot[4 * t + 3];
        const double gp = G[row * n + p], gq = G[row * n + q];
        G[row * n + p] = c * gp - s * gq;
        G[row * n + q] = s * gp + c * gq;
        const double vp = V[row * n + p], vq = V[row * n + q];
        V[row * n + p] = c * vp - s * vq;
        V[row * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int i = 1; i < n; ++i) {  // insertion sort, descending eigenvalue
      const int o = order[i];
      int j = i - 1;
      while (j >= 0 && G[order[j] * n + order[j]] < G[o * n + o]) {
        order[j + 1] = order[j];
        --j;
      }
      order[j + 1] = o;
    }
    for (int i = 0; i < n; ++i) ev[i] = G[order[i] * n + order[i]];
  }
  __syncthreads();
}

// Truncated SVD of M (r x c, row-major, global or shared) with r <= 32 or c <= 32: the
// Gram matrix of the short side is diagonalised.  Writes the kept count n, the
// normalised singular values lam[0..D) (zero-padded), U (r x D) and Vt (D x c), both
// zero-padded beyond n.  Work arrays in shared memory.
struct SvdWork {
  double* G;     // 32 x 32
  double* V;     // 32 x 32
  double* ev;    // 32
  double* rot;   // 4 * 16
  int* order;    // 32
  double* red;   // 8 * 32
  double* tot;   // 32
};
__device__ int blk_svd(const double* M, int r, int c, int D, double* U, double* Vt, double* lam, SvdWork& w) {
  const bool left = r <= c;  // diagonalise M M^T (r x r) if r is the short side, else M^T M
  const int s = left ? r : c, l = left ? c : r;
  for (int idx = threadIdx.x; idx < s * s; idx += blockDim.x) {
    const int i = idx / s, j = idx % s;
    if (j < i) continue;
    double acc = 0.0;
    if (left)
      for (int t = 0; t < l; ++t) acc = fma(M[(long long)i * c + t], M[(long long)j * c + t], acc);
    else
      for (int t = 0; t < l; ++t) acc = fma(M[(long long)t * c + i], M[(long long)t * c + j], acc);
    w.G[i * s + j] = acc;
    w.G[j * s + i] = acc;
  }
  __syncthreads();
  blk_eig(w.G, s, w.ev, w.V, w.rot, w.order);
  __shared__ int kept;
  __shared__ double sig[kMaxSide], nrm;
  if (threadIdx.x == 0) {
    const double s0 = sqrt(fmax(w.ev[0], 0.0));
    int n = 0;
    double n2 = 0.0;
    for (int i = 0; i < s && n < D; ++i) {
      const double si = sqrt(fmax(w.ev[i], 0.0));
      if (!(s0 > 0.0) || si <= 1e-7 * s0) break;
      sig[i] = si;
      n2 += si * si;
      ++n;
    }
    kept = n;
    nrm = sqrt(n2);
  }
  __syncthreads();
  const int n = kept;
  for (int i = threadIdx.x; i < D; i += blockDim.x) lam[i] = i < n ? sig[i] / nrm : 0.0;
  // vectors of the short side: columns order[i] of V; the long side by one product
  if (left) {
    for (int idx = threadIdx.x; idx < r * D; idx += blockDim.x) {
      const int a = idx / D, i = idx % D;
      U[idx] = i < n ? w.V[a * s + w.order[i]] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < D * c; idx += blockDim.x) {
      const int i = idx / c, b = idx % c;
      double acc = 0.0;
      if (i < n) {
        for (int a = 0; a < r; ++a) acc = fma(U[a * D + i], M[(long long)a * c + b], acc);
        acc /= sig[i];
      }
      Vt[idx] = acc;
    }
  } else {
    for (int idx = threadIdx.x; idx < D * c; idx += blockDim.x) {
      const int i = idx / c, b = idx % c;
      Vt[idx] = i < n ? w.V[b * s + w.order[i]] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < r * D; idx += blockDim.x) {
      const int a = idx / D, i = idx % D;
      double acc = 0.0;
      if (i < n) {
        for (int b = 0; b < c; ++b) acc = fma(M[(long long)a * c + b], Vt[i * c + b], acc);
        acc /= sig[i];
      }
      U[idx] = acc;
    }
  }
  __syncthreads();
  // sign rule: the largest-magnitude entry of each left vector is positive
  for (int i = 0; i < n; ++i) {
    double best = 0.0, val = 0.0;
    for (int a = threadIdx.x; a < r; a += blockDim.x) {
      const double v = U[a * D + i];
      if (fabs(v) > best) { best = fabs(v); val = v; }
    }
    // block arg-max of |v| (first lane wins ties within its own rows only; ties are
    // measure-zero for generic input)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o), ov = __shfl_xor_sync(0xffffffffu, val, o);
      if (ob > best) { best = ob; val = ov; }
    }
    if ((threadIdx.x & 31) == 0) { w.red[2 * (threadIdx.x >> 5)] = best; w.red[2 * (threadIdx.x >> 5) + 1] = val; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0, v = 0.0;
      for (int q = 0; q < kSuThreads / 32; ++q)
        if (w.red[2 * q] > b) { b = w.red[2 * q]; v = w.red[2 * q + 1]; }
      w.tot[0] = v < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    const double f = w.tot[0];
    if (f < 0.0) {
      for (int a = threadIdx.x; a < r; a += blockDim.x) U[a * D + i] = -U[a * D + i];
      for (int b = threadIdx.x; b < c; b += blockDim.x) Vt[i * c + b] = -Vt[i * c + b];
    }
    __syncthreads();
  }
  return n;
}

// Site (k, m) with the lambdas of its legs other than `bond` absorbed, as the matrix
// A[(outer legs in l, r, u, d order)][(bond index, spin)] in shared memory.  Returns the
// number of rows; the outer legs are described by `o`.
__device__ int load_reduced(const SuLattice& L, int k, int m, int bond, double* A, const Outer& o) {
  const int rows = o.d0 * o.d1 * o.d2, n = 2 * leg_dim(L, k, m, bond);
  const double* B = L.B + L.site_off[k * L.Lx + m];
  const double* l0 = leg_lam(L, k, m, o.g0);
  const double* l1 = leg_lam(L, k, m, o.g1);
  const double* l2 = leg_lam(L, k, m, o.g2);
  for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
    const int row = idx / n, col = idx % n, b = col >> 1, s = col & 1;
    const int o2 = row % o.d2, o1 = (row / o.d2) % o.d1, o0 = row / (o.d1 * o.d2);
    double v = B[s * o.ss + o0 * o.s0 + o1 * o.s1 + o2 * o.s2 + b * o.sb];
    if (l0) v *= l0[o0];
    if (l1) v *= l1[o1];
    if (l2) v *= l2[o2];
    A[idx] = v;
  }
  __syncthreads();
  return rows;
}

// B(k, m) = Q Rt with Q (rows x kq), Rt[x][(spin, bond)] (kq x 2D); outer lambdas divided out.
__device__ void store_rebuilt(const SuLattice& L, int k, int m, const Outer& o, const double* Q, int rows, int kq,
                              const double* Rt) {
  const int D = L.D;
  double* B = L.B + L.site_off[k * L.Lx + m];
  const double* l0 = leg_lam(L, k, m, o.g0);
  const double* l1 = leg_lam(L, k, m, o.g1);
  const double* l2 = leg_lam(L, k, m, o.g2);
  const double m0 = l0 ? lam_max(l0, D) : 1.0, m1 = l1 ? lam_max(l1, D) : 1.0, m2 = l2 ? lam_max(l2, D) : 1.0;
  for (int idx = threadIdx.x; idx < rows * 2 * D; idx += blockDim.x) {
    const int row = idx / (2 * D), s = (idx / D) & 1, b = idx % D;
    double acc = 0.0;
    for (int x = 0; x < kq; ++x) acc = fma(Q[row * kq + x], Rt[x * 2 * D + s * D + b], acc);
    const int o2 = row % o.d2, o1 = (row / o.d2) % o.d1, o0 = row / (o.d1 * o.d2);
    if (l0) acc *= inv_lam(l0, D, o0, m0);
    if (l1) acc *= inv_lam(l1, D, o1, m1);
    if (l2) acc *= inv_lam(l2, D, o2, m2);
    B[s * o.ss + o0 * o.s0 + o1 * o.s1 + o2 * o.s2 + b * o.sb] = acc;
  }
  __syncthreads();
}

struct NNArgs {
  SuLattice L;
  const int* sites;  // per update: k1, m1, k2, m2
  double gate[16];   // G[s1'][s2'][s1][s2]
  double* scratch;   // per CTA: 2 * kMaxRows * kMaxCols
  long long scratch_stride;
};

// dynamic shared memory of one update: the QR matrix + R + Theta + SVD outputs
constexpr int kSmemDoubles = kMaxRows * kMaxCols + 2 * kMaxCols * kMaxCols + 3 * kMaxSide * kMaxSide +
                             kMaxSide * kMaxSide;

__global__ void __launch_bounds__(kSuThreads) su_nn_kernel(const NNArgs a) {
  extern __shared__ double sm[];
  __shared__ double red[kSuThreads / 32 * kMaxSide], tmp[2 * kMaxCols + kMaxSide], rot[64], ev[kMaxSide];
  __shared__ double G[kMaxSide * kMaxSide], V[kMaxSide * kMaxSide], lamn[kSuMaxD];
  __shared__ int order[kMaxSide];
  const SuLattice L = a.L;
  const int D = L.D;
  const int* st = a.sites + 4 * blockIdx.x;
  const int k1 = st[0], m1 = st[1], k2 = st[2], m2 = st[3];
  const int g1 = dir_of(k1, m1, k2, m2), g2 = dir_of(k2, m2, k1, m1);
  double* A = sm;                                  // kMaxRows x kMaxCols
  double* R1 = A + kMaxRows * kMaxCols;            // kMaxCols x kMaxCols
  double* R2 = R1 + kMaxCols * kMaxCols;
  double* Th = R2 + kMaxCols * kMaxCols;           // 32 x 32
  double* U = Th + kMaxSide * kMaxSide;            // 32 x D
  double* Vt = U + kMaxSide * kMaxSide;            // D x 32
  double* Rt = Vt + kMaxSide * kMaxSide;           // 32 x 2D (re-indexed factor)
  double* Q1 = a.scratch + blockIdx.x * a.scratch_stride;
  double* Q2 = Q1 + kMaxRows * kMaxCols;
  const Outer o1 = outer_of(L, k1, m1, g1), o2 = outer_of(L, k2, m2, g2);
  const int n = 2 * D;
  const int r1 = load_reduced(L, k1, m1, g1, A, o1);
  blk_qr(A, r1, n, R1, Q1, red, tmp);
  const int q1 = min(r1, n);
  const int r2 = load_reduced(L, k2, m2, g2, A, o2);
  blk_qr(A, r2, n, R2, Q2, red, tmp);
  const int q2 = min(r2, n);
  double* lam = g1 == 1 ? leg_lam(L, k1, m1, 1) : leg_lam(L, k1, m1, 3);
  // Theta[(x,s1'),(y,s2')] = sum_{b,s1,s2} R1[x][(b,s1)] lam[b] R2[y][(b,s2)] G[s1'][s2'][s1][s2]
  const int tr = 2 * q1, tc = 2 * q2;
  for (int idx = threadIdx.x; idx < tr * tc; idx += blockDim.x) {
    const int x = idx / tc / 2, s1p = (idx / tc) & 1, y = (idx % tc) / 2, s2p = idx & 1;
    double acc = 0.0;
    for (int b = 0; b < D; ++b)
      for (int s1 = 0; s1 < 2; ++s1)
        for (int s2 = 0; s2 < 2; ++s2)
          acc = fma(R1[x * n + 2 * b + s1] * lam[b] * R2[y * n + 2 * b + s2], a.gate[((s1p * 2 + s2p) * 2 + s1) * 2 + s2],
                    acc);
    Th[idx] = acc;
  }
  __syncthreads();
  SvdWork w{G, V, ev, rot, order, red, tmp};
  blk_svd(Th, tr, tc, D, U, Vt, lamn, w);
  for (int i = threadIdx.x; i < D; i += blockDim.x) lam[i] = lamn[i];
  __syncthreads();
  // B1 = Q1 Rt1 with Rt1[x][(s1', b')] = U[(x, s1')][b']
  for (int idx = threadIdx.x; idx < q1 * 2 * D; idx += blockDim.x) {
    const int x = idx / (2 * D), s = (idx / D) & 1, b = idx % D;
    Rt[idx] = U[(2 * x + s) * D + b];
  }
  __syncthreads();
  store_rebuilt(L, k1, m1, o1, Q1, r1, q1, Rt);
  // B2 = Q2 Rt2 with Rt2[y][(s2', b')] = Vt[b'][(y, s2')]
  for (int idx = threadIdx.x; idx < q2 * 2 * D; idx += blockDim.x) {
    const int y = idx / (2 * D), s = (idx / D) & 1, b = idx % D;
    Rt[idx] = Vt[b * tc + 2 * y + s];
  }
  __syncthreads();
  store_rebuilt(L, k2, m2, o2, Q2, r2, q2, Rt);
}

struct NNNArgs {
  SuLattice L;
  const int* sites;  // per update: k1, m1, kc, mc, k3, m3
  double gate[16];   // G[s1'][s3'][s1][s3]
  double* scratch;   // per CTA
  long long scratch_stride;
};
// per-CTA scratch of an NNN update (doubles): Q1, Q3, M2, P, Ta (also Tb), U2 (N3 x D)
constexpr long long kNQ = (long long)kMaxRows * kMaxCols;
constexpr long long kNM2 = 2LL * kSuMaxD * kSuMaxD * kSuMaxD * kSuMaxD;
constexpr long long kNP = (long long)kMaxSide * 2 * kSuMaxD * kSuMaxD * kSuMaxD;  // (x,s1) x (s2,b,o,o')
constexpr long long kNT = (long long)kMaxSide * 2 * kSuMaxD * kSuMaxD * kMaxSide; // (x,s1') x (s2,o,o',z,s3')
constexpr long long kNU2 = (long long)kSuMaxD * 2 * kSuMaxD * kSuMaxD * kSuMaxD;  // (a',s2,o,o') x b'
constexpr long long kNNNScratch = 2 * kNQ + kNM2 + kNP + 2 * kNT + kNU2;

__global__ void __launch_bounds__(kSuThreads) su_nnn_kernel(const NNNArgs a) {
  extern __shared__ double sm[];
  __shared__ double red[kSuThreads / 32 * kMaxSide], tmp[2 * kMaxCols + kMaxSide], rot[64], ev[kMaxSide];
  __shared__ double G[kMaxSide * kMaxSide], V[kMaxSide * kMaxSide], la[kSuMaxD], lb[kSuMaxD];
  __shared__ int order[kMaxSide];
  const SuLattice L = a.L;
  const int D = L.D;
  const int* st = a.sites + 6 * blockIdx.x;
  const int k1 = st[0], m1 = st[1], kc = st[2], mc = st[3], k3 = st[4], m3 = st[5];
  const int a1 = dir_of(k1, m1, kc, mc), a2 = dir_of(kc, mc, k1, m1);
  const int b2 = dir_of(kc, mc, k3, m3), b3 = dir_of(k3, m3, kc, mc);
  double* A = sm;                          // kMaxRows x kMaxCols
  double* R1 = A + kMaxRows * kMaxCols;    // kMaxCols x kMaxCols
  double* R3 = R1 + kMaxCols * kMaxCols;
  double* U1 = R3 + kMaxCols * kMaxCols;   // 32 x D
  double* V2t = U1 + kMaxSide * kSuMaxD;   // D x 32
  double* Rt = V2t + kMaxSide * kSuMaxD;   // 16 x 2D
  double* base = a.scratch + blockIdx.x * a.scratch_stride;
  double* Q1 = base;
  double* Q3 = Q1 + kNQ;
  double* M2 = Q3 + kNQ;
  double* P = M2 + kNM2;
  double* Ta = P + kNP;
  double* Tb = Ta + kNT;
  double* U2 = Tb + kNT;
  const Outer o1 = outer_of(L, k1, m1, a1), o3 = outer_of(L, k3, m3, b3);
  const int n = 2 * D;
  const int r1 = load_reduced(L, k1, m1, a1, A, o1);  // (b)
  blk_qr(A, r1, n, R1, Q1, red, tmp);
  const int q1 = min(r1, n);
  const int r3 = load_reduced(L, k3, m3, b3, A, o3);
  blk_qr(A, r3, n, R3, Q3, red, tmp);
  const int q3 = min(r3, n);
  // M2[s2][a][b][o][o'] = B2 with the outer lambdas and both link lambdas absorbed; o and o'
  // are the corner's two other legs in l, r, u, d order
  const int oc0 = (a2 != 0 && b2 != 0) ? 0 : ((a2 != 1 && b2 != 1) ? 1 : 2);
  const int oc1 = (a2 != 3 && b2 != 3) ? 3 : ((a2 != 2 && b2 != 2) ? 2 : 1);
  const int dO = leg_dim(L, kc, mc, oc0), dP = leg_dim(L, kc, mc, oc1);
  const long long sA = leg_stride(L, kc, mc, a2), sB = leg_stride(L, kc, mc, b2);
  const long long sO = leg_stride(L, kc, mc, oc0), sP = leg_stride(L, kc, mc, oc1);
  const long long sS = leg_stride(L, kc, mc, 0) * leg_dim(L, kc, mc, 0);
  double* lam_a = leg_lam(L, kc, mc, a2);
  double* lam_b = leg_lam(L, kc, mc, b2);
  const double* lo = leg_lam(L, kc, mc, oc0);
  const double* lp = leg_lam(L, kc, mc, oc1);
  {
    const double* B2 = L.B + L.site_off[kc * L.Lx + mc];
    const int tot = 2 * D * D * dO * dP;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      const int op = idx % dP, o = (idx / dP) % dO, b = (idx / (dP * dO)) % D, aa = (idx / (dP * dO * D)) % D,
                s = idx / (dP * dO * D * D);
      double v = B2[s * sS + aa * sA + b * sB + o * sO + op * sP];
      v *= lam_a[aa] * lam_b[b];
      if (lo) v *= lo[o];
      if (lp) v *= lp[op];
      M2[idx] = v;
    }
  }
  __syncthreads();
  // (c) P[(x,s1)][(s2,b,o,o')] = sum_a R1[x][(a,s1)] M2[s2][a][b][o][o']
  const int nP = 2 * D * dO * dP;  // (s2, b, o, o') per (x, s1)
  for (int idx = threadIdx.x; idx < 2 * q1 * nP; idx += blockDim.x) {
    const int row = idx / nP, col = idx % nP;
    const int x = row >> 1, s1 = row & 1;
    const int s2 = col / (D * dO * dP), rest = col % (D * dO * dP);  // rest = (b, o, o')
    double acc = 0.0;
    for (int aa = 0; aa < D; ++aa) acc = fma(R1[x * n + 2 * aa + s1], M2[((long long)(s2 * D + aa) * D * dO * dP) + rest], acc);
    P[idx] = acc;
  }
  __syncthreads();
  // T_a[(x,s1')][(s2,o,o',z,s3')] = sum_{b,s1,s3} P[(x,s1)][(s2,b,o,o')] R3[z][(b,s3)] G[s1'][s3'][s1][s3]
  const int nT = 2 * dO * dP * 2 * q3;
  const int tr = 2 * q1;
  for (int idx = threadIdx.x; idx < tr * nT; idx += blockDim.x) {
    const int row = idx / nT, col = idx % nT;
    const int x = row >> 1, s1p = row & 1;
    const int s3p = col & 1, z = (col >> 1) % q3, oo = (col / (2 * q3)) % (dO * dP), s2 = col / (2 * q3 * dO * dP);
    double acc = 0.0;
    for (int s1 = 0; s1 < 2; ++s1)
      for (int s3 = 0; s3 < 2; ++s3) {
        const double g = a.gate[((s1p * 2 + s3p) * 2 + s1) * 2 + s3];
        if (g == 0.0) continue;
        double inner = 0.0;
        for (int b = 0; b < D; ++b)
          inner = fma(P[(long long)(2 * x + s1) * nP + (s2 * D + b) * dO * dP + oo], R3[z * n + 2 * b + s3], inner);
        acc = fma(g, inner, acc);
      }
    Ta[idx] = acc;
  }
  __syncthreads();
  SvdWork w{G, V, ev, rot, order, red, tmp};
  // (d) T_a = U1 S1 V1t; lambda(1,2) = S1 normalised; T_b = lambda(1,2) V1t (D x nT)
  double* V1t = Tb;
  blk_svd(Ta, tr, nT, D, U1, V1t, la, w);
  for (int idx = threadIdx.x; idx < D * nT; idx += blockDim.x) V1t[idx] *= la[idx / nT];
  __syncthreads();
  // (e) T_b as (a', s2, o, o') x (z, s3'): rows D*2*dO*dP, columns 2*q3
  const int rB = D * 2 * dO * dP, cB = 2 * q3;
  blk_svd(Tb, rB, cB, D, U2, V2t, lb, w);
  // new link lambdas
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    lam_a[i] = la[i];
    lam_b[i] = lb[i];
  }
  __syncthreads();
  // (f) B1 = Q1 Rt1, Rt1[x][(s1', a')] = U1[(x, s1')][a']
  for (int idx = threadIdx.x; idx < q1 * 2 * D; idx += blockDim.x) {
    const int x = idx / (2 * D), s = (idx / D) & 1, b = idx % D;
    Rt[idx] = U1[(2 * x + s) * D + b];
  }
  __syncthreads();
  store_rebuilt(L, k1, m1, o1, Q1, r1, q1, Rt);
  // (h) B3 = Q3 Rt3, Rt3[z][(s3', b')] = V2t[b'][(z, s3')]
  for (int idx = threadIdx.x; idx < q3 * 2 * D; idx += blockDim.x) {
    const int z = idx / (2 * D), s = (idx / D) & 1, b = idx % D;
    Rt[idx] = V2t[b * cB + 2 * z + s];
  }
  __syncthreads();
  store_rebuilt(L, k3, m3, o3, Q3, r3, q3, Rt);
  // (g) B2[s2][...] = T_c[(a', s2, o, o')][b'] with lambda(1,2)^-1 on a' and the outer
  // lambdas divided out
  {
    double* B2 = L.B + L.site_off[kc * L.Lx + mc];
    const double mxa = lam_max(la, D), mxo = lo ? lam_max(lo, D) : 1.0, mxp = lp ? lam_max(lp, D) : 1.0;
    const int tot = D * 2 * dO * dP * D;
    for (int idx = threadIdx.x; idx < tot; idx += blockDim.x) {
      const int bp = idx % D, row = idx / D;
      const int op = row % dP, o = (row / dP) % dO, s2 = (row / (dP * dO)) & 1, ap = row / (dP * dO * 2);
      double v = U2[idx] * inv_lam(la, D, ap, mxa);
      if (lo) v *= inv_lam(lo, D, o, mxo);
      if (lp) v *= inv_lam(lp, D, op, mxp);
      B2[s2 * sS + ap * sA + bp * sB + o * sO + op * sP] = v;
    }
  }
}

// A = B with lambda^(1/2) of every link absorbed on both ends (App. A), one thread per entry.
__global__ void su_absorb_kernel(const SuLattice L, double* out, long long P) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= P) return;
  int site = 0;
  while (site + 1 < L.Ly * L.Lx && L.site_off[site + 1] <= e) ++site;
  const int k = site / L.Lx, m = site % L.Lx;
  const int dl = leg_dim(L, k, m, 0), dr = leg_dim(L, k, m, 1), du = leg_dim(L, k, m, 2), dd = leg_dim(L, k, m, 3);
  long long r = e - L.site_off[site];
  const int d = r % dd; r /= dd;
  const int u = r % du; r /= du;
  const int rr = r % dr; r /= dr;
  const int l = r % dl;
  double v = L.B[e];
  const double* lam;
  if ((lam = leg_lam(L, k, m, 0))) v *= sqrt(lam[l]);
  if ((lam = leg_lam(L, k, m, 1))) v *= sqrt(lam[rr]);
  if ((lam = leg_lam(L, k, m, 2))) v *= sqrt(lam[u]);
  if ((lam = leg_lam(L, k, m, 3))) v *= sqrt(lam[d]);
  out[e] = v;
}

// Mean over links of ||lam - old|| / ||old||, one block.
__global__ void su_change_kernel(const double* lam, const double* old, int n_links, int D, double* out) {
  __shared__ double red[kSuThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n_links; i += blockDim.x) {
    double d2 = 0.0, o2 = 0.0;
    for (int j = 0; j < D; ++j) {
      const double x = lam[(long long)i * D + j], y = old[(long long)i * D + j];
      d2 += (x - y) * (x - y);
      o2 += y * y;
    }
    s += o2 > 0.0 ? sqrt(d2 / o2) : 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kSuThreads / 32; ++w) t += red[w];
    *out = n_links > 0 ? t / n_links : 0.0;
  }
}

void heisenberg_gate(double J, double tau, double* g) {
  // exp(-tau J S.S) = e^{-tau J/4} P_t + e^{3 tau J/4} P_s in the basis (uu, ud, du, dd)
  const double et = exp(-tau * J / 4.0), es = exp(3.0 * tau * J / 4.0);
  const double h[16] = {0.25, 0, 0, 0, 0, -0.25, 0.5, 0, 0, 0.5, -0.25, 0, 0, 0, 0, 0.25};
  for (int i = 0; i < 16; ++i) {
    const double id = (i / 4 == i % 4) ? 1.0 : 0.0;
    g[i] = et * (0.75 * id + h[i]) + es * (0.25 * id - h[i]);
  }
}

}  // namespace
}  // namespace pv

using namespace pv;

extern "C" int pepsvmc_simple_update(int32_t Ly, int32_t Lx, int32_t D, double J1, double J2, double tau,
                                     int32_t max_steps, double tol, double* B, double* lam_h, double* lam_v,
                                     double* peps_out, int32_t* steps_done, double* change_out, void* stream) {
  if (Ly < 1 || Lx < 1 || Ly > 64 || Lx > 64 || Ly * Lx < 2 || D < 1 || D > kSuMaxD || max_steps < 0 || !B ||
      !(tau == tau) || !(tol == tol))
    return PEPSVMC_EINVAL;
  if ((Lx > 1 && !lam_h) || (Ly > 1 && !lam_v)) return PEPSVMC_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // packed offsets
  std::vector<long long> off(Ly * Lx + 1, 0);
  for (int k = 0; k < Ly; ++k)
    for (int m = 0; m < Lx; ++m) {
      const long long sz = 2LL * (m == 0 ? 1 : D) * (m == Lx - 1 ? 1 : D) * (k == 0 ? 1 : D) * (k == Ly - 1 ? 1 : D);
      off[k * Lx + m + 1] = off[k * Lx + m] + sz;
    }
  const long long P = off[Ly * Lx];
  const long long nh = (long long)Ly * (Lx - 1) * D, nv = (long long)(Ly - 1) * Lx * D;
  // update lists, by group
  std::vector<std::vector<int>> nn_groups, nnn_groups;
  for (int par = 0; par < 2; ++par) {
    std::vector<int> g;
    for (int k = 0; k < Ly; ++k)
      for (int m = par; m + 1 < Lx; m += 2) g.insert(g.end(), {k, m, k, m + 1});
    nn_groups.push_back(g);
  }
  for (int par = 0; par < 2; ++par) {
    std::vector<int> g;
    for (int k = par; k + 1 < Ly; k += 2)
      for (int m = 0; m < Lx; ++m) g.insert(g.end(), {k, m, k + 1, m});
    nn_groups.push_back(g);
  }
  if (J2 != 0.0)
    for (int diag = 0; diag < 2; ++diag)
      for (int path = 0; path < 2; ++path)
        for (int pk = 0; pk < 2; ++pk)
          for (int pm = 0; pm < 2; ++pm) {
            std::vector<int> g;
            for (int k = pk; k + 1 < Ly; k += 2)
              for (int m = pm; m + 1 < Lx; m += 2) {
                if (diag == 0) {
                  const int kc = path == 0 ? k : k + 1, mc = path == 0 ? m + 1 : m;
                  g.insert(g.end(), {k, m, kc, mc, k + 1, m + 1});
                } else {
                  const int kc = path == 0 ? k : k + 1, mc = path == 0 ? m : m + 1;
                  g.insert(g.end(), {k, m + 1, kc, mc, k + 1, m});
                }
              }
            nnn_groups.push_back(g);
          }
  size_t max_nn = 0, max_nnn = 0, total_idx = 0;
  for (auto& g : nn_groups) { max_nn = std::max(max_nn, g.size() / 4); total_idx += g.size(); }
  for (auto& g : nnn_groups) { max_nnn = std::max(max_nnn, g.size() / 6); total_idx += g.size(); }

  std::vector<void*> allocs;
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (bytes == 0) bytes = 8;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return p;
  };
  auto cleanup = [&]() {
    for (void* p : allocs) cudaFree(p);
  };
  double* dB = (double*)dalloc(P * sizeof(double));
  long long* doff = (long long*)dalloc(off.size() * sizeof(long long));
  double* dlam = (double*)dalloc((nh + nv) * sizeof(double));
  double* dold = (double*)dalloc((nh + nv) * sizeof(double));
  int* didx = (int*)dalloc(total_idx * sizeof(int));
  double* dchg = (double*)dalloc(sizeof(double));
  const long long nn_stride = 2 * kMaxRows * kMaxCols;
  double* dscr = (double*)dalloc(std::max((size_t)1, std::max(max_nn * (size_t)nn_stride, max_nnn * (size_t)kNNNScratch)) *
                                 sizeof(double));
  double* dout = peps_out ? (double*)dalloc(P * sizeof(double)) : nullptr;
  if (!dB || !doff || !dlam || !dold || !didx || !dchg || !dscr || (peps_out && !dout)) {
    cleanup();
    return PEPSVMC_ENOMEM;
  }
  std::vector<int> idx_all;
  std::vector<size_t> starts;
  for (auto& g : nn_groups) { starts.push_back(idx_all.size()); idx_all.insert(idx_all.end(), g.begin(), g.end()); }
  for (auto& g : nnn_groups) { starts.push_back(idx_all.size()); idx_all.insert(idx_all.end(), g.begin(), g.end()); }
  cudaError_t e = cudaSuccess;
  if (!e) e = cudaMemcpyAsync(dB, B, P * sizeof(double), cudaMemcpyHostToDevice, st);
  if (!e) e = cudaMemcpyAsync(doff, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, st);
  if (!e && nh) e = cudaMemcpyAsync(dlam, lam_h, nh * sizeof(double), cudaMemcpyHostToDevice, st);
  if (!e && nv) e = cudaMemcpyAsync(dlam + nh, lam_v, nv * sizeof(double), cudaMemcpyHostToDevice, st);
  if (!e && !idx_all.empty())
    e = cudaMemcpyAsync(didx, idx_all.data(), idx_all.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  const size_t smem = (size_t)kSmemDoubles * sizeof(double);
  if (!e) e = cudaFuncSetAttribute(su_nn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (!e) e = cudaFuncSetAttribute(su_nnn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  SuLattice L{Ly, Lx, D, dB, doff, dlam, dlam + nh};
  NNArgs na{};
  na.L = L;
  heisenberg_gate(J1, tau, na.gate);
  na.scratch = dscr;
  na.scratch_stride = nn_stride;
  NNNArgs nb{};
  nb.L = L;
  heisenberg_gate(J2, tau / 2.0, nb.gate);
  nb.scratch = dscr;
  nb.scratch_stride = kNNNScratch;
  int done = 0;
  double change = 0.0;
  for (int step = 0; step < max_steps && !e; ++step) {
    e = cudaMemcpyAsync(dold, dlam, (nh + nv) * sizeof(double), cudaMemcpyDeviceToDevice, st);
    size_t gi = 0;
    for (auto& g : nn_groups) {
      const int cnt = (int)(g.size() / 4);
      if (!e && cnt) {
        na.sites = didx + starts[gi];
        su_nn_kernel<<<cnt, kSuThreads, smem, st>>>(na);
        e = cudaGetLastError();
      }
      ++gi;
    }
    for (auto& g : nnn_groups) {
      const int cnt = (int)(g.size() / 6);
      if (!e && cnt) {
        nb.sites = didx + starts[gi];
        su_nnn_kernel<<<cnt, kSuThreads, smem, st>>>(nb);
        e = cudaGetLastError();
      }
      ++gi;
    }
    if (!e) {
      su_change_kernel<<<1, kSuThreads, 0, st>>>(dlam, dold, (int)((nh + nv) / std::max(D, 1)), D, dchg);
      e = cudaGetLastError();
    }
    if (!e) e = cudaMemcpyAsync(&change, dchg, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    ++done;
    if (!e && !(change == change)) {
      cleanup();
      return PEPSVMC_ENONFINITE;
    }
    if (!e && change < tol) break;
  }
  if (!e) e = cudaMemcpyAsync(B, dB, P * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (!e && nh) e = cudaMemcpyAsync(lam_h, dlam, nh * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (!e && nv) e = cudaMemcpyAsync(lam_v, dlam + nh, nv * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (!e && dout) {
    su_absorb_kernel<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(L, dout, P);
    e = cudaGetLastError();
    if (!e) e = cudaMemcpyAsync(peps_out, dout, P * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  if (!e) e = cudaStreamSynchronize(st);
  cleanup();
  if (e) return PEPSVMC_ECUDA;
  if (steps_done) *steps_done = done;
  if (change_out) *change_out = change;
  return PEPSVMC_OK;
}
