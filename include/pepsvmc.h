/*
 * pepsvmc -- C ABI of the per-sample single-layer PEPS contraction used by
 * variational Monte Carlo (Liu, Huang, Gong, Gu, arXiv:1908.09359).
 *
 * One context holds, on one CUDA device, the PEPS tensors of an open Ly x Lx
 * spin-1/2 lattice and n_chains Markov chains.  All arithmetic of the hot path
 * runs in the library's own CUDA kernels on the stream given at init.
 *
 * Conventions shared by every call
 *   - Return value: PEPSVMC_OK (0) or a negative PEPSVMC_E* code; the text of
 *     the last error is available from pepsvmc_last_error().
 *   - Host buffers are owned by the caller and only read or written during the
 *     call.  Device memory is owned by the context and freed by
 *     pepsvmc_destroy().  Calls that return host data synchronise the stream.
 *   - Tensor layout ("packed"): sites in row-major lattice order (row k = 0 at
 *     the top, column m = 0 at the left); each site is A(s, l, r, u, d) in
 *     row-major order (Sec. II A, Eq. (1)) with s = 0 for spin +1 and s = 1
 *     for spin -1; a leg on the open edge has dimension 1, every other leg D.
 *   - Spins: int8 +1/-1, layout [chain][k][m].
 *   - A context is not thread-safe; calls on one context must not overlap.
 */
#ifndef PEPSVMC_H
#define PEPSVMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PEPSVMC_OK = 0,
  PEPSVMC_EINVAL = -1,      /* bad argument or configuration                 */
  PEPSVMC_ENOMEM = -2,      /* device or host allocation failed              */
  PEPSVMC_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed   */
  PEPSVMC_ETIMEOUT = -4,    /* a device-side wait exceeded its budget        */
  PEPSVMC_ENONFINITE = -5,  /* a non-finite amplitude ratio, E_loc or log    */
  PEPSVMC_EZEROPSI = -6,    /* a configuration with Psi(S) = 0 was met       */
  PEPSVMC_ESTATE = -7       /* call out of order (e.g. no measurement yet)   */
};

/* Precision of the contractions: FP32 on CUDA cores; or, on the tcgen05 tensor
 * cores with FP32 accumulation, operands rounded to BF16 (MIXED_BF16), to TF32
 * (MIXED_TF32), or split into two BF16 parts x = hi + lo with three products per
 * step (MIXED_BF16X3, close to FP32 accuracy).  In every mode the truncation QR, the
 * ratios (float64 dot products), log amplitudes and the energy / gradient sums are
 * as in FP32 mode.                                                              */
enum { PEPSVMC_FP32 = 0, PEPSVMC_MIXED_BF16 = 1, PEPSVMC_MIXED_TF32 = 2, PEPSVMC_MIXED_BF16X3 = 3 };

typedef struct pepsvmc_ctx pepsvmc_ctx;

typedef struct {
  int32_t Ly, Lx;       /* lattice rows and columns (>= 1 each, Ly*Lx even)  */
  int32_t D;            /* virtual bond dimension (1..16)                   */
  int32_t chi;          /* boundary-MPS cutoff Dc (App. B), 1..64           */
  int32_t n_chains;     /* Markov chains advanced together (>= 1)          */
  int32_t n_fit;        /* one-site fit half-sweeps per truncation, odd    */
  double J1, J2;        /* NN and NNN couplings; J2 = 0 is Heisenberg      */
  uint64_t seed;        /* Philox key for Metropolis and sign-SGD uniforms */
  int32_t precision;    /* PEPSVMC_FP32 or one of the PEPSVMC_MIXED_* modes  */
  int32_t chi_measure;  /* Dc of the measurement (E_loc, Psi, G), 0..64;    */
                        /* 0 = chi.  chi is then the sampler's Dc (Sec. II A */
                        /* and App. D use a smaller cutoff for sampling)    */
  uint64_t wait_budget_cycles; /* clock budget of every device-side wait    */
                        /* (tensor-core completion barriers); 0 = default   */
                        /* (4e9 cycles, ~2 s).  A wait that runs out sets   */
                        /* the status that the call returns as ETIMEOUT     */
  int32_t chain_offset; /* global index of chain 0 in the Philox counters   */
                        /* (>= 0): a job whose chains are split over several */
                        /* contexts draws the same numbers as one context   */
                        /* holding all of them                              */
  int32_t symmetrize;   /* 0: sample |Psi|^2.  1: spin-inversion symmetrised */
                        /* Phi(S) = Psi(S) + Psi(S-bar), S-bar = all spins   */
                        /* reversed (end of Sec. II B): n_chains must be     */
                        /* even, chain p + n_chains/2 holds S-bar of chain p */
                        /* (pairs p = 0 .. n_chains/2 - 1), the sequential   */
                        /* sweep samples |Phi|^2 (one decision per pair, the */
                        /* uniform of Philox chain word chain_offset + p),   */
                        /* and the accumulated sums of pepsvmc_energy_and_grad */
                        /* take E^Phi and G^Phi of each pair as one sample.  */
                        /* Random-NNASP and learned sweeps return EINVAL.   */
  int32_t reserved[2];  /* must be zero                                    */
} pepsvmc_config;

/* Create a context (on failure *out may still receive a context that holds the
 * error text; pass it to pepsvmc_destroy).  Boundary-MPS truncation (App. B) is the variational fit
 * of ||M|U> - |U'>||^2 by n_fit one-site half-sweeps; its starting guess is the
 * random MPS ``sketch``.  The sampler truncates to chi, the measurement to
 * chi_measure (when nonzero; pepsvmc_amplitude uses chi).
 *   tensors: host, packed layout above, float64, copied.
 *   sketch:  host float64 array [max(Ly,Lx)][X][D][X] of iid N(0,1) entries,
 *            X = max(chi, chi_measure), copied; a fit with cutoff c uses the
 *            leading [c][D][c] corner of each site.
 *   stream:  a cudaStream_t (NULL = the legacy default stream).
 * All chains start in the Neel configuration (with symmetrize, chains
 * n_chains/2 .. n_chains-1 in its inversion); use pepsvmc_set_spins to change.
 * Errors: EINVAL (bad config), ENOMEM, ECUDA.                               */
int pepsvmc_init(const pepsvmc_config* cfg, const double* tensors, const double* sketch,
                 void* stream, pepsvmc_ctx** out);

void pepsvmc_destroy(pepsvmc_ctx* ctx);
const char* pepsvmc_last_error(const pepsvmc_ctx* ctx);

/* Number of float64 entries of the packed tensor array (both spin slots). */
int64_t pepsvmc_n_params(const pepsvmc_ctx* ctx);

int pepsvmc_set_spins(pepsvmc_ctx* ctx, const int8_t* spins);  /* host, n_chains*Ly*Lx */
int pepsvmc_get_spins(pepsvmc_ctx* ctx, int8_t* spins);
int pepsvmc_set_tensors(pepsvmc_ctx* ctx, const double* tensors);
int pepsvmc_get_tensors(pepsvmc_ctx* ctx, double* tensors);

/* Fused three-line steps (on by default in the BF16 and split-BF16 precisions): the
 * three products of a column step (App. C) run in one tensor-core kernel per chain and
 * bond tile, with the intermediates kept in tensor and shared memory; bonds up to
 * Dc = 32 and D = 8, larger ones use the separate products.  pepsvmc_set_fused(ctx, 0)
 * computes every step as three separate products (same arithmetic type, other
 * rounding order).  Forcing a contraction kernel (pepsvmc_set_contraction_kernel)
 * also disables the fused steps.  Drops a captured step graph.                  */
int pepsvmc_set_fused(pepsvmc_ctx* ctx, int32_t on);

/* Change the device wait budget of an existing context (cycles; 0 = default).  */
int pepsvmc_set_wait_budget(pepsvmc_ctx* ctx, uint64_t cycles);

/* Sweep counter used in the Metropolis Philox counter (chain, sweep, bond, tag). */
int pepsvmc_set_sweep_counter(pepsvmc_ctx* ctx, uint64_t sweep);
uint64_t pepsvmc_get_sweep_counter(const pepsvmc_ctx* ctx);

/* n_sweeps sequential Metropolis sweeps of every chain (Sec. II A, Eq. (9)):
 * each sweep visits all vertical bonds (columns left to right, bonds top to
 * bottom), then all horizontal bonds (rows top to bottom, bonds left to
 * right), proposing a swap of every antiparallel pair and accepting it when
 * r < min(1, |Psi(S_b)/Psi(S_a)|^2), r = Philox uniform.  Bond ids: vertical
 * (k,m)-(k+1,m) is m*(Ly-1)+k, horizontal (k,m)-(k,m+1) is Lx*(Ly-1)+k*(Lx-1)+m.
 *   accept_rate_out: nullable host double, accepted / proposed over the call.
 * Errors: EZEROPSI, ENONFINITE, ECUDA.                                      */
int pepsvmc_sample_sweep(pepsvmc_ctx* ctx, int32_t n_sweeps, double* accept_rate_out);

/* n_sweeps sweeps of the random-NNASP scheme (Sec. II A, Eq. (prob_r)), the paper's
 * reference for the sequential sweep: a sweep is N = Ly*Lx attempts; each picks one of
 * the K_a antiparallel nearest-neighbour pairs of a chain's configuration uniformly
 * (pairs listed in the bond order of pepsvmc_sample_sweep; index floor(r K_a) with r from
 * word 0 of Philox (chain + chain_offset, sweep, attempt, "RAND")), swaps it, and accepts
 * with r' < min[1, |Psi_b|^2 K_a / (|Psi_a|^2 K_b)] (r' from word 1).  Every Psi is a full
 * boundary-MPS contraction at chi closed at row Ly/2, so an attempt costs a whole
 * amplitude: O(N^2 D^4 Dc^2) per sweep instead of the sequential sweep's O(N D^4 Dc^2).
 *   accept_rate_out: nullable host double, accepted / proposed over the call.
 * pepsvmc_get_random_trace: per [chain][attempt] of the last sweep (tracing on): the bond
 * id swapped (-1: no antiparallel pair), Psi_b/Psi_a, decision (-1, 0, 1); all nullable.
 * Errors: EZEROPSI, ENONFINITE, ECUDA; ESTATE (trace) without a traced sweep.        */
int pepsvmc_random_sweep(pepsvmc_ctx* ctx, int32_t n_sweeps, double* accept_rate_out);
int pepsvmc_get_random_trace(pepsvmc_ctx* ctx, int32_t* bond, double* ratio, int8_t* decision);

/* Per-proposal record of the most recent sweep (after pepsvmc_enable_trace(ctx,1)):
 *   ratio:    host float64 [n_chains][2*Lx*Ly - Lx - Ly], Psi(S_b)/Psi(S_a)
 *   decision: host int8 same shape: -1 no proposal (parallel pair), 0 rejected,
 *             1 accepted.  Both nullable.                                    */
int pepsvmc_enable_trace(pepsvmc_ctx* ctx, int32_t on);
int pepsvmc_get_trace(pepsvmc_ctx* ctx, double* ratio, int8_t* decision);

/* Measure the current configurations (App. C; Eqs. (3)-(7)):
 *   eloc:   E_loc(S) = sum over NN and NNN bonds of J s_i s_j / 4 plus, for
 *           antiparallel pairs, (J/2) Psi(S')/Psi(S); horizontal ratios from
 *           the three-line environments of each row, vertical and diagonal
 *           ratios from four-line environments of each row pair.
 *   logpsi, sign: ln|Psi(S)| and its sign from the contraction of row Ly/2.
 *   All nullable, host, n_chains entries.  G(S) = Delta(S)/Psi(S) of every
 *   chain is kept on the device for pepsvmc_get_chain_grad.
 * Errors: EZEROPSI, ENONFINITE, ECUDA.                                      */
int pepsvmc_measure(pepsvmc_ctx* ctx, double* eloc, double* logpsi, int8_t* sign);

/* Symmetrised results of the last measurement (pepsvmc_measure or a step of
 * pepsvmc_energy_and_grad) of a context created with symmetrize = 1, per
 * pair p (host float64, n_chains/2 entries each, nullable):
 *   w:        Psi(S-bar)/Psi(S) = sign_{p+P} sign_p exp(lnPsi_{p+P} - lnPsi_p)
 *             from the measured amplitudes of chains p and p + P;
 *   eloc_phi: E^Phi(S) = (E_loc(S) + w E_loc(S-bar)) / (1 + w), the local
 *             energy of Phi (H commutes with the global spin inversion, so
 *             <S|H|S'> = <S-bar|H|S'-bar>).
 * The gradient sums use G^Phi(S) = (G(S) + w G(S-bar)) / (1 + w), with G(S) in
 * the slots of S and G(S-bar) in the opposite slots.
 * Errors: ESTATE (no symmetrize, or no measurement yet), ECUDA.             */
int pepsvmc_get_phi(pepsvmc_ctx* ctx, double* eloc_phi, double* w);

/* G(S) of one chain from the last measurement: host float64, packed layout of
 * ONE spin slot per site, i.e. sum over sites of Dl*Dr*Du*Dd entries, each
 * site (l, r, u, d) row-major; it belongs to slot s(k,m) of that chain.     */
int64_t pepsvmc_n_grad_entries(const pepsvmc_ctx* ctx);
int pepsvmc_get_chain_grad(pepsvmc_ctx* ctx, int32_t chain, double* out);

/* Ln|Psi| and sign of the current configurations contracted at row ``row``
 * (<B_row| M_row |T_row>, App. B), host arrays of n_chains, nullable.       */
int pepsvmc_amplitude(pepsvmc_ctx* ctx, int32_t row, double* logpsi, int8_t* sign);

/* Algorithm 1: n_sweeps times (one sweep of every chain, then a measurement),
 * accumulating E_tot, P1 = sum G E_loc and P2 = sum G over all chains and
 * sweeps in float64.  Outputs (host, nullable):
 *   E_mean, E_var:   mean and variance of E_loc over the n_sweeps*n_chains samples
 *                    (with symmetrize: of E^Phi over the n_sweeps*n_chains/2 pairs)
 *   eloc, logpsi, sign: per sample [sweep][chain] (with symmetrize, eloc holds
 *                    E^Phi of the chain's pair)
 *   grad:            dE/dA = <G E_loc> - <G><E_loc> (Eq. (5), without the
 *                    factor 2 of the exact derivative), packed layout.
 * Errors: as pepsvmc_sample_sweep and pepsvmc_measure.                       */
int pepsvmc_energy_and_grad(pepsvmc_ctx* ctx, int32_t n_sweeps, double* E_mean, double* E_var,
                            double* eloc, double* logpsi, int8_t* sign, double* grad);

/* The float64 sums behind the gradient of the last pepsvmc_energy_and_grad
 * (Algorithm 1: E_tot, E_tot^2 and the sample count, then P1 = sum G E_loc and
 * P2 = sum G per packed tensor entry), for a job whose chains are split over
 * several contexts (one per GPU): each rank reads its sums, the ranks add them
 * (an all-reduce), and every rank writes the totals back with pepsvmc_set_sums,
 * which recomputes dE/dA = P1/n - (P2/n) E_tot/n exactly as energy_and_grad does,
 * so that the following pepsvmc_update applies one identical sign-SGD step on
 * every rank.  Host buffers: scalars[3] = {sum E, sum E^2, n}, sumGE and sumG with
 * pepsvmc_n_params entries each (nullable in get).
 * pepsvmc_sums_device exposes the same three device arrays (owned by the context,
 * valid until pepsvmc_destroy) so that a collective library can reduce them in
 * place; pepsvmc_finalize_sums then recomputes the gradient from them.
 * Errors: ESTATE before any energy_and_grad; EINVAL (null pointers, n <= 0).    */
int pepsvmc_get_sums(pepsvmc_ctx* ctx, double* scalars, double* sumGE, double* sumG);
int pepsvmc_set_sums(pepsvmc_ctx* ctx, const double* scalars, const double* sumGE, const double* sumG);
int pepsvmc_sums_device(pepsvmc_ctx* ctx, double** scalars, double** sumGE, double** sumG);
int pepsvmc_finalize_sums(pepsvmc_ctx* ctx);

/* Sign-SGD (Sec. II B, Eq. (10)) with the gradient of the last
 * pepsvmc_energy_and_grad: A <- A - r * delta * sgn(dE/dA), r = Philox uniform
 * with counter (element & 0xffffffff, element >> 32, step, tag).
 * Errors: ESTATE if no gradient was computed.                               */
int pepsvmc_update(pepsvmc_ctx* ctx, double delta, uint64_t step);

/* Simple-update imaginary-time evolution (App. A), the initialiser of the
 * optimisation, in float64 on the GPU; needs no context.  The PEPS is held as site
 * tensors B (packed layout of pepsvmc_init's tensors) and one vector lambda of length
 * D on every nearest-neighbour link:
 *   lam_h [Ly][Lx-1][D] for links (k,m)-(k,m+1), lam_v [Ly-1][Lx][D] for (k,m)-(k+1,m).
 * One Trotter step applies exp(-tau J1 S_i.S_j) to the horizontal NN bonds with m
 * even, then m odd, to the vertical ones with k even, then k odd, and, when J2 != 0,
 * exp(-(tau/2) J2 S_i.S_k) to both diagonals of every plaquette through each of its
 * two corner sites (plaquettes in four groups by the parity of (k, m)).  An NN update
 * reduces both tensors (outer lambdas absorbed) by QR, applies the gate to the R
 * factors joined by the bond lambda and truncates by SVD; an NNN update follows the
 * QR / SVD / SVD steps of App. A's figure.  Each truncation keeps min(D, #{sigma >
 * 1e-7 sigma_max}) singular values (missing entries are zero) and normalises the new
 * lambda to unit norm; inverse lambdas are 1/lambda above 1e-14 of the largest entry,
 * else 0.  Steps run until the mean over links of ||lambda(t+tau) - lambda(t)|| /
 * ||lambda(t)|| is below tol or max_steps are done.
 *   B, lam_h, lam_v: host float64, in/out (lam_h may be NULL when Lx = 1, lam_v when
 *                    Ly = 1);
 *   peps_out:        host float64 (nullable), the packed tensors with lambda^(1/2) of
 *                    every link absorbed into both of its tensors, ready for
 *                    pepsvmc_init / pepsvmc_set_tensors;
 *   steps_done, change_out: host (nullable), the steps run and the last change.
 * D <= 8.  Allocates and frees its own device memory; synchronous on the stream.
 * Errors: EINVAL (sizes, null pointers), ENOMEM, ENONFINITE, ECUDA.          */
int pepsvmc_simple_update(int32_t Ly, int32_t Lx, int32_t D, double J1, double J2, double tau,
                          int32_t max_steps, double tol, double* B, double* lam_h, double* lam_v,
                          double* peps_out, int32_t* steps_done, double* change_out, void* stream);

/* Three-line environment step (App. C, Fig. "contraction" (c)) for n_chains chains,
 * on the context's stream, with the context's scratch:
 *   out[c](a',r,b') = sum over a,l,b,u,d of
 *       E[c](a,l,b) * T[c](a,u,a') * A_{s_c}(l,r,u,d) * B[c](b,d,b')
 * E: left environment (cT, Dl, cB); T: top boundary-MPS site (cT, Du, cT2);
 * B: bottom boundary-MPS site (cB, Dd, cB2); out: (cT2, Dr, cB2).  All are float32
 * device arrays, row-major per chain, chains back to back (chain stride = size).
 * A: the site tensor, float32 device array of both spin slots, each slot in the
 * order (l, u, r, d); chain c uses slot 1 when spins[c] < 0 (int8 device array of
 * n_chains), slot 0 otherwise or when spins is NULL.  Asynchronous on the stream.
 * Errors: EINVAL for null pointers, non-positive sizes, n_chains above the
 * context's chains or bonds whose intermediates exceed the context's scratch
 * (Dl*cB*Du*cT2 and cB*cT2*Dr*Dd must not exceed D^3*chi^2); ECUDA.          */
int pepsvmc_env3_left(pepsvmc_ctx* ctx, const float* E, const float* T, const float* A,
                      const int8_t* spins, const float* B, float* out, int32_t n_chains,
                      int32_t cT, int32_t cB, int32_t cT2, int32_t cB2,
                      int32_t Dl, int32_t Dr, int32_t Du, int32_t Dd);

/* Four-line environment step of a row pair (App. C: the environments that close the
 * vertical and diagonal amplitude ratios of E_loc) for n_chains chains, on the context's
 * stream with the context's scratch:
 *   out[c](a',r1,r2,b') = sum over a,l1,l2,b,u1,d1,d2 of
 *       E[c](a,l1,l2,b) * T[c](a,u1,a') * A1_{s1}(l1,r1,u1,d1) * A2_{s2}(l2,r2,d1,d2) * B[c](b,d2,b')
 * E: (cT, D1l, D2l, cB); T: top boundary-MPS site (cT, Du1, cT2); B: bottom site
 * (cB, Dd2, cB2); out: (cT2, D1r, D2r, cB2); float32 device arrays, row-major per chain,
 * chains back to back.  A1, A2: the upper and lower site tensors, both spin slots, each
 * slot in the order (l, u, r, d) (A2's up leg is A1's down leg, Dd1); chain c uses slot 1
 * of A1 when spins1[c] < 0 and of A2 when spins2[c] < 0 (int8 device arrays), slot 0
 * otherwise or when the pointer is NULL.  In the tensor-core precisions bonds up to
 * Dc = 32 and D = 8 run as one fused kernel.  bmajor = 1 stores E and out b-major instead,
 * E(a,l1,l2,b) at [b][a][l1][l2] and out(a',r1,r2,b') at [b'][a'][r1][r2] (the order the
 * context keeps its own four-line environments in when its steps are fused; the fused
 * kernel only).  Asynchronous on the stream.
 * Errors: EINVAL (null pointers, non-positive sizes, more chains than the context's,
 * intermediates larger than its scratch, bmajor not 0 or 1, or bmajor without the fused
 * kernel); ECUDA.                                                                      */
int pepsvmc_env4_left(pepsvmc_ctx* ctx, const float* E, const float* T, const float* A1, const int8_t* spins1,
                      const float* A2, const int8_t* spins2, const float* B, float* out, int32_t n_chains,
                      int32_t cT, int32_t cB, int32_t cT2, int32_t cB2, int32_t D1l, int32_t D1r, int32_t Du1,
                      int32_t Dd1, int32_t D2l, int32_t D2r, int32_t Dd2, int32_t bmajor);

/* pepsvmc_env3_left without a context and without allocating anything (the paper
 * has no counterpart; this is a library convenience).  For callers that cannot
 * call cudaMalloc where they need the step -- e.g. a service that reserved all of
 * its device memory at start-up and must not allocate later, since cudaMalloc can
 * synchronise the device and fragments a planned pool.  Same operation, layouts
 * and spin rule as pepsvmc_env3_left; runs asynchronously on ``stream`` (a
 * cudaStream_t, NULL = legacy default stream) on the current device.
 * Scratch: the two intermediates live in one fixed array of
 * PEPSVMC_NOALLOC_SCRATCH_FLOATS floats (16 MiB) of the library's own device
 * memory, present on every GPU where the library's device code is loaded until
 * the process exits.  Every call looks up that array's device address for the
 * current device and context (no allocation; after a device reset the new
 * context's address is used); the first call on a device loads the library's
 * device code there, so make that first call before any stream capture.  Every call uses the same array, and it keeps the last call's
 * contents (nothing in it needs to start at zero); calls whose execution overlaps
 * on the GPU -- on different streams or devices sharing nothing, or from several
 * host threads -- race on it and must be serialised by the caller.
 * Errors: EINVAL for null pointers, non-positive sizes, or when
 * 2 * n_chains * max(Dl*cB*Du*cT2, cB*cT2*Dr*Dd) exceeds the array; ECUDA.      */
#define PEPSVMC_NOALLOC_SCRATCH_FLOATS 4194304
int pepsvmc_env3_left_noalloc(const float* E, const float* T, const float* A,
                              const int8_t* spins, const float* B, float* out,
                              int32_t n_chains, int32_t cT, int32_t cB, int32_t cT2,
                              int32_t cB2, int32_t Dl, int32_t Dr, int32_t Du, int32_t Dd,
                              void* stream);

/* Batched thin QR with a non-negative diagonal of R, the factorisation the
 * variational fit of App. B uses to move the orthogonality centre (Householder
 * reflections in float32; no context, no allocation).  Y, Q: device float32, `batch`
 * matrices of rows x cols stored one after another (rows * cols floats each),
 * row-major (element (i,j) at i*cols + j) or, with col_major != 0, column-major (at
 * j*rows + i); Q may equal Y (in place), otherwise the two must not overlap.  Q is the
 * unique thin factor with R(j,j) > 0 for full-rank input; a column that is zero after
 * the previous reflections gets no reflector (R(j,j) = 0) and Q keeps the identity's
 * column there, transformed by the other reflectors.  Asynchronous on ``stream`` (a
 * cudaStream_t, NULL = legacy default stream), current device.
 * Errors: EINVAL for null pointers, batch < 1, cols < 1, cols > 64 or rows < cols;
 * ECUDA.                                                                          */
int pepsvmc_qr_pos(const float* Y, float* Q, int32_t batch, int32_t rows, int32_t cols,
                   int32_t col_major, void* stream);

/* ------------------------------------------------------------- learned proposal
 * Exact Metropolis-Hastings moves proposed by a small convolutional network (no
 * counterpart in the paper's Sec. II sampler; it uses the MH form of Eq. (8) with a
 * learned q).  Network: three 3x3 zero-padded convolutions on the +-1 grid, 1 -> 32 ->
 * 32 -> 2 channels, ReLU after the first two; parameters (float64 on the host, 10146
 * entries) in the order w1 (32,1,3,3), b1 (32), w2 (32,32,3,3), b2 (32), w3 (2,32,3,3),
 * b3 (2).  Output channel 0 at (k,m) is the logit of bond (k,m)-(k,m+1), channel 1 of
 * (k,m)-(k+1,m).  A learned sweep visits bands (k, k+1), k = 0..Ly-2: one or two
 * site-disjoint antiparallel pairs of the band are drawn from softmaxes of their
 * logits (two pairs with probability 1/2) and swapped; the move is accepted with
 * min[1, |Psi'/Psi|^2 q(S|S')/q(S'|S)], Psi'/Psi from the band's four-line closure,
 * Philox counter (chain, sweep, 4k+j, "LERN").
 *   set/get_proposal_params: the network (float64 host array of 10146).
 *   proposal_logits: logits of the current spins, host float64 [chain][2][Ly][Lx].
 *   proposal_collect: n sweeps of the plain sampler, each followed by a measurement;
 *     appends every chain's configuration and its measured NN amplitude ratios to a
 *     device-resident training set.
 *   proposal_train: Adam epochs (minibatches of `batch` configurations) on the mean
 *     squared error between each antiparallel bond's logit and log min(1, rho^2)
 *     (clipped at -20); loss_out (nullable) gets the last epoch's mean.
 *   set_proposal: 0 = plain sequential sweeps only; 1 = every sample step of
 *     pepsvmc_energy_and_grad adds one learned sweep after the plain sweep.
 *   learned_sweep: n learned sweeps alone; accept_rate_out (nullable).
 *   get_learned_trace: last learned sweep per [chain][band]: ratio Psi'/Psi,
 *     ln q(S|S') - ln q(S'|S), decision (-1 nothing proposed, 0, 1); needs tracing on.
 * Errors: ESTATE before set_proposal_params or with too small a training set.   */
int pepsvmc_set_proposal_params(pepsvmc_ctx* ctx, const double* params);
int pepsvmc_get_proposal_params(pepsvmc_ctx* ctx, double* params);
int pepsvmc_proposal_logits(pepsvmc_ctx* ctx, double* out);
int pepsvmc_proposal_collect(pepsvmc_ctx* ctx, int32_t n_sweeps);
int64_t pepsvmc_proposal_dataset_size(const pepsvmc_ctx* ctx);
/* Replace the training set by n host configurations (int8 [n][Ly][Lx]) and ratios
 * (float64 [n][2][Ly][Lx], same channel layout as the logits).                   */
int pepsvmc_proposal_load(pepsvmc_ctx* ctx, const int8_t* spins, const double* rho, int64_t n);
int pepsvmc_proposal_train(pepsvmc_ctx* ctx, int32_t epochs, int32_t batch, double lr, double* loss_out);
/* Train on given configurations (host int8 [n][Ly][Lx], +-1): each is measured with
 * this context's environments (batches of n_chains; its NN ratios rho give the targets
 * log min(1, rho^2)), the training set is replaced by them, then `epochs` Adam epochs
 * in minibatches of min(256, n) run; final_loss_out (nullable) gets the last epoch's
 * mean loss.  The chains' own configurations are restored afterwards (their last
 * measurement is discarded).  Errors: EINVAL (bad sizes, spins not +-1, lr <= 0),
 * ESTATE (no network), ENOMEM.                                                      */
int pepsvmc_train_proposal(pepsvmc_ctx* ctx, const int8_t* configs, int64_t n, int32_t epochs, double lr,
                           double* final_loss_out);
int pepsvmc_set_proposal(pepsvmc_ctx* ctx, int32_t mode);
int pepsvmc_learned_sweep(pepsvmc_ctx* ctx, int32_t n_sweeps, double* accept_rate_out);
int pepsvmc_get_learned_trace(pepsvmc_ctx* ctx, double* rho, double* dlq, int8_t* decision);

/* Kernel launches issued by this context since its creation (a counter kept by
 * the host side of the library). */
int64_t pepsvmc_launch_count(const pepsvmc_ctx* ctx);

/* Optional timing of every contraction and QR launch with CUDA events recorded
 * on the context's stream (adds about a microsecond of host time per launch).
 * pepsvmc_set_profiling resets the counters.  pepsvmc_get_profile fills out[6]:
 * contraction launches, their algorithmic flops (2*M*N*K per chain), their
 * summed device time in ms, QR launches, their device time in ms, and the
 * contractions' algorithmic bytes (FP32 operands read once -- an operand shared by
 * all chains once --, the result written once).                               */
int pepsvmc_set_profiling(pepsvmc_ctx* ctx, int32_t on);
int pepsvmc_get_profile(pepsvmc_ctx* ctx, double* out);
/* The same counters per launch shape, as JSON text written to buf (len bytes):
 * [{"shape": "gemm tc M.. N.. K..", "launches": n, "flops": f, "ms": t}, ...].
 * EINVAL if the text does not fit.                                          */
int pepsvmc_get_profile_shapes(pepsvmc_ctx* ctx, char* buf, int64_t len);

/* Autotuner (on by default): the first launch of every contraction shape times each
 * candidate kernel (six FP32 tile shapes; in the tensor-core modes also the TC tile
 * widths 32/64/128/256, and in split BF16 the two-stage form at 32/64 for products
 * with K > 64) with CUDA events and keeps the fastest for this context.
 * pepsvmc_set_autotune(ctx, 0) turns it off and forgets the choices (fixed
 * heuristics then); pepsvmc_get_tuning writes the choices as JSON text:
 * [{"shape": "...", "choice": "f32_cfg3" | "tc_bn64" | "tc2_bn32", "candidate_ms": [...]}, ...]. */
int pepsvmc_set_autotune(pepsvmc_ctx* ctx, int32_t on);

/* Fix the kernel of every contraction of this context (kernel-level profiling and
 * tests; the automatic choice computes the same products).  The paper has no
 * counterpart: this selects among this library's implementations of the products of
 * App. B and App. C.  kind 0: automatic (the
 * autotuner, or the size heuristic with autotuning off); 1: FP32 CUDA-core kernel
 * with tile-table entry `tile` (0..5); 2: tcgen05 kernel with N tile `tile` (32, 64,
 * 128, 256), mixed precisions only; 3: its split-BF16 form with two shared-memory
 * stages, N tile 32 or 64, PEPSVMC_MIXED_BF16X3 only.  Drops a captured step graph.
 * Errors: EINVAL (unknown kind or tile, or a kind the precision lacks).            */
int pepsvmc_set_contraction_kernel(pepsvmc_ctx* ctx, int32_t kind, int32_t tile);

/* CUDA graphs (on by default): pepsvmc_energy_and_grad runs its first sample step
 * (sweep + measurement + sums) eagerly, then captures the step's launches once into
 * a CUDA graph on an internal stream and replays it for every later step (not while
 * tracing or profiling).  pepsvmc_set_graphs(ctx, 0) runs every step eagerly.     */
int pepsvmc_set_graphs(pepsvmc_ctx* ctx, int32_t on);
int pepsvmc_get_tuning(pepsvmc_ctx* ctx, char* buf, int64_t len);

#ifdef __cplusplus
}
#endif
#endif /* PEPSVMC_H */
