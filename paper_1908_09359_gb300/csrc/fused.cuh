// Fused column steps of the boundary-MPS contraction on the tcgen05 tensor cores.
#pragma once
#include "common.cuh"

namespace pv {

// Three-line column step (App. C, Fig. "contraction" (c)) for every chain c:
//   out[c](a',r,b') = sum over a,l,b,u,d of E[c](a,l,b) T[c](a,u,a') A_s(l,u,r,d) B[c](b,d,b')
// with all three products (E.T over a, .A over (l,u), .B over (b,d)) in one kernel: the
// intermediates never leave the SM (tensor memory and shared memory).  Every operand
// is addressed through its own element strides, so the same kernel runs the left step,
// the right step (a mirrored view) and any permuted storage order.  Bonds up to
// kFusedChi (boundary) and kFusedD (virtual); smaller ones are zero-padded on chip.
constexpr int kFusedChi = 32;
constexpr int kFusedD = 8;

struct Env3Fused {
  int cT = 0, cB = 0, cT2 = 0, cB2 = 0, Dl = 0, Dr = 0, Du = 0, Dd = 0;
  int batch = 0;
  const float* E = nullptr;  // E(a,l,b) = E[c*bsE + a*sEa + l*sEl + b*sEb]
  long long bsE = 0, sEa = 0, sEl = 0, sEb = 0;
  const float* T = nullptr;  // T(a,u,a') = T[c*bsT + a*sTa + u*sTu + a'*sTa2]
  long long bsT = 0, sTa = 0, sTu = 0, sTa2 = 0;
  const float* A = nullptr;  // A_s(l,u,r,d) = A[s*ssA + l*sAl + u*sAu + r*sAr + d*sAd]
  long long ssA = 0, sAl = 0, sAu = 0, sAr = 0, sAd = 0;
  const int8_t* sel = nullptr;  // slot s of chain c: (sel[c*sel_stride] < 0) ^ sel_xor; 0 when null
  long long sel_stride = 0;
  int sel_xor = 0;
  const float* B = nullptr;  // B(b,d,b') = B[c*bsB + b*sBb + d*sBd + b'*sBb2]
  long long bsB = 0, sBb = 0, sBd = 0, sBb2 = 0;
  float* out = nullptr;      // out(a',r,b') = out[c*bsO + a'*sOa2 + r*sOr + b'*sOb2]
  long long bsO = 0, sOa2 = 0, sOr = 0, sOb2 = 0;
  long long wait_cycles = 0;  // device wait budget (0 = kDefaultWaitCycles)
  int tiles_per_cta = 0;      // a' tiles of 8 per CTA (0 = automatic)
};

inline bool env3_fused_fits(int cT, int cB, int cT2, int cB2, int Dl, int Dr, int Du, int Dd) {
  return cT >= 1 && cB >= 1 && cT2 >= 1 && cB2 >= 1 && Dl >= 1 && Dr >= 1 && Du >= 1 && Dd >= 1 &&
         cT <= kFusedChi && cB <= kFusedChi && cT2 <= kFusedChi && cB2 <= kFusedChi && Dl <= kFusedD &&
         Dr <= kFusedD && Du <= kFusedD && Dd <= kFusedD;
}

// split: BF16 hi + lo operands with three MMAs per step (PEPSVMC_MIXED_BF16X3); else BF16.
// On an expired device wait ST_TIMEOUT is set in *status.
cudaError_t env3_fused(const Env3Fused& a, bool split, unsigned* status, cudaStream_t st);

}  // namespace pv

namespace pv {

// Four-line column step of rows (k, k+1) (App. C; the vertical and diagonal ratios of
// E_loc, Eqs. (3)-(7)) for every chain c:
//   out[c](a',r1,r2,b') = sum E[c](a,l1,l2,b) T[c](a,u1,a') a1(l1,u1,r1,d1) a2(l2,d1,r2,d2) B[c](b,d2,b')
// as four products in one kernel (E.T over a, .a1 over (l1,u1), .a2 over (l2,d1), .B over
// (b,d2), the last accumulated over tiles of b), intermediates on chip; a1 and a2 are
// selected per chain by the spins of their sites (sel1, sel2, each xor a flip).
struct Env4Fused {
  int cT = 0, cB = 0, cT2 = 0, cB2 = 0;
  int D1l = 0, D1r = 0, Du1 = 0, Dd1 = 0, D2l = 0, D2r = 0, Dd2 = 0;
  int batch = 0;
  const float* E = nullptr;  // E(a,l1,l2,b) = E[c*bsE + a*sEa + l1*sEl1 + l2*sEl2 + b*sEb]
  long long bsE = 0, sEa = 0, sEl1 = 0, sEl2 = 0, sEb = 0;
  const float* T = nullptr;  // T(a,u1,a') = T[c*bsT + a*sTa + u1*sTu + a'*sTa2]
  long long bsT = 0, sTa = 0, sTu = 0, sTa2 = 0;
  const float* A1 = nullptr;  // a1_s(l1,u1,r1,d1) = A1[s*ss1 + l1*s1l + u1*s1u + r1*s1r + d1*s1d]
  long long ss1 = 0, s1l = 0, s1u = 0, s1r = 0, s1d = 0;
  const int8_t* sel1 = nullptr;
  int xor1 = 0;
  const float* A2 = nullptr;  // a2_s(l2,d1,r2,d2) = A2[s*ss2 + l2*s2l + d1*s2u + r2*s2r + d2*s2d]
  long long ss2 = 0, s2l = 0, s2u = 0, s2r = 0, s2d = 0;
  const int8_t* sel2 = nullptr;
  int xor2 = 0;
  long long sel_stride = 0;
  const float* B = nullptr;  // B(b,d2,b') = B[c*bsB + b*sBb + d2*sBd + b'*sBb2]
  long long bsB = 0, sBb = 0, sBd = 0, sBb2 = 0;
  float* out = nullptr;      // out(a',r1,r2,b') = out[c*bsO + a'*sOa2 + r1*sOr1 + r2*sOr2 + b'*sOb2]
  long long bsO = 0, sOa2 = 0, sOr1 = 0, sOr2 = 0, sOb2 = 0;
  long long wait_cycles = 0;
};

inline bool env4_fused_fits(const Env4Fused& f) {
  const int x[4] = {f.cT, f.cB, f.cT2, f.cB2};
  const int d[7] = {f.D1l, f.D1r, f.Du1, f.Dd1, f.D2l, f.D2r, f.Dd2};
  for (int v : x)
    if (v < 1 || v > kFusedChi) return false;
  for (int v : d)
    if (v < 1 || v > kFusedD) return false;
  return true;
}

cudaError_t env4_fused(const Env4Fused& a, bool split, unsigned* status, cudaStream_t st);

}  // namespace pv

namespace pv {

// Optimal site of the variational fit (App. B): the boundary MPS site that best fits
// M_k |U> given its left and right environments, for every chain c:
//   Y[c](v,d,v') = sum over a,l,a',u,r of L[c](a,l,v) T[c](a,u,a') A_s(l,u,r,d) R[c](a',r,v')
// as three products in one kernel (L.T over a, .A over (l,u), .R over (a',r), the last
// accumulated over tiles of a'), intermediates on chip.
struct Proj3Fused {
  int cT = 0, cV = 0, cT2 = 0, cV2 = 0, Dl = 0, Dr = 0, Du = 0, Dd = 0;
  int batch = 0;
  const float* L = nullptr;  // L(a,l,v) = L[c*bsL + a*sLa + l*sLl + v*sLv]
  long long bsL = 0, sLa = 0, sLl = 0, sLv = 0;
  const float* T = nullptr;  // T(a,u,a') = T[c*bsT + a*sTa + u*sTu + a'*sTa2]
  long long bsT = 0, sTa = 0, sTu = 0, sTa2 = 0;
  const float* A = nullptr;  // A_s(l,u,r,d) = A[s*ssA + l*sAl + u*sAu + r*sAr + d*sAd]
  long long ssA = 0, sAl = 0, sAu = 0, sAr = 0, sAd = 0;
  const int8_t* sel = nullptr;
  long long sel_stride = 0;
  const float* R = nullptr;  // R(a',r,v') = R[c*bsR + a'*sRa + r*sRr + v'*sRv]
  long long bsR = 0, sRa = 0, sRr = 0, sRv = 0;
  float* out = nullptr;      // Y(v,d,v') = out[c*bsO + v*sOv + d*sOd + v'*sOv2]
  long long bsO = 0, sOv = 0, sOd = 0, sOv2 = 0;
  long long wait_cycles = 0;
};

inline bool proj3_fused_fits(const Proj3Fused& f) {
  const int x[4] = {f.cT, f.cV, f.cT2, f.cV2};
  const int d[4] = {f.Dl, f.Dr, f.Du, f.Dd};
  for (int v : x)
    if (v < 1 || v > kFusedChi) return false;
  for (int v : d)
    if (v < 1 || v > kFusedD) return false;
  return true;
}

cudaError_t proj3_fused(const Proj3Fused& a, bool split, unsigned* status, cudaStream_t st);

}  // namespace pv
