// Stage layouts of the three-line environment step as batched matrix products.
#pragma once
#include "common.cuh"

namespace pv {

struct Env3Dims {
  int cT, cB;    // bonds of T and B entering the column (env: cT x Dl x cB)
  int cT2, cB2;  // bonds leaving the column (result: cT2 x Dr x cB2)
  int Dl, Dr, Du, Dd;
};

// Left three-line step (App. C, Fig. "contraction" (c)) for every chain b:
//   out[b](a',r,b') = sum E[b](a,l,b) T[b](a,u,a') A_s(l,r,u,d) B[b](b,d,b')
// as three products: (1) E x T -> t1 laid out [b][a'][l][u]; (2) t1 x A_s over (l,u)
// -> t2 laid out [a'][r][b][d]; (3) t2 x B over (b,d) -> out.  A is given per slot in
// the [(l,u)][(r,d)] order; the slot of chain b is (spins[b*spin_stride] < 0) ^ flip,
// or 0 when spins is null.  t1 and t2 need env3_scratch() floats per chain.
inline void env3_left_descs(GemmDesc g[3], const Env3Dims& d, const float* E, long long bsE, const float* T,
                            long long bsT, const float* A_lurd, long long slot_size, const int8_t* spins,
                            long long spin_stride, int flip, const float* B, long long bsB, float* out,
                            long long bsO, float* t1, float* t2, long long bsTmp) {
  const int Dl = d.Dl, Dr = d.Dr, Du = d.Du, Dd = d.Dd, cT = d.cT, cB = d.cB, cT2 = d.cT2, cB2 = d.cB2;
  g[0] = GemmDesc();
  g[0].M = Dl * cB; g[0].N = Du * cT2; g[0].K = cT;
  g[0].A = E; g[0].sAm = 1; g[0].sAk = (long long)Dl * cB; g[0].bsA = bsE;
  g[0].B = T; g[0].sBk = (long long)Du * cT2; g[0].sBn = 1; g[0].bsB = bsT;
  g[0].C = t1; g[0].bsC = bsTmp;
  g[0].cm2 = cB; g[0].sCm1 = Du; g[0].sCm2 = (long long)cT2 * Dl * Du;
  g[0].cn2 = cT2; g[0].sCn1 = 1; g[0].sCn2 = (long long)Dl * Du;
  g[1] = GemmDesc();
  g[1].M = cB * cT2; g[1].N = Dr * Dd; g[1].K = Dl * Du;
  g[1].A = t1; g[1].sAm = (long long)Dl * Du; g[1].sAk = 1; g[1].bsA = bsTmp;
  g[1].B = A_lurd; g[1].sBk = (long long)Dr * Dd; g[1].sBn = 1; g[1].bsB = 0;
  g[1].ssB = slot_size; g[1].sel = spins; g[1].sel_stride = spin_stride; g[1].sel_xor = flip;
  g[1].C = t2; g[1].bsC = bsTmp;
  g[1].cm2 = cT2; g[1].sCm1 = Dd; g[1].sCm2 = (long long)Dr * cB * Dd;
  g[1].cn2 = Dd; g[1].sCn1 = (long long)cB * Dd; g[1].sCn2 = 1;
  g[2] = GemmDesc();
  g[2].M = cT2 * Dr; g[2].N = cB2; g[2].K = cB * Dd;
  g[2].A = t2; g[2].sAm = (long long)cB * Dd; g[2].sAk = 1; g[2].bsA = bsTmp;
  g[2].B = B; g[2].sBk = cB2; g[2].sBn = 1; g[2].bsB = bsB;
  g[2].C = out; g[2].bsC = bsO; g[2].sCm1 = cB2; g[2].sCn1 = 1;
}

// Floats of t1 (and, separately, of t2) one chain of env3_left_descs needs.
inline long long env3_scratch(const Env3Dims& d) {
  const long long a = (long long)d.Dl * d.cB * d.Du * d.cT2, b = (long long)d.cB * d.cT2 * d.Dr * d.Dd;
  return a > b ? a : b;
}

inline bool env3_dims_ok(const Env3Dims& d) {
  return d.cT > 0 && d.cB > 0 && d.cT2 > 0 && d.cB2 > 0 && d.Dl > 0 && d.Dr > 0 && d.Du > 0 && d.Dd > 0;
}

}  // namespace pv
