/*
 * hadamag.h -- C ABI of libhadamag: magic (non-stabilizerness) of state vectors on one
 * NVIDIA GB300 GPU (sm_103a), following "Computing quantum magic of state vectors"
 * (arXiv 2601.07824).
 *
 * Conventions shared by every call
 *   - A state of N sites of dimension d has d^N amplitudes (qubits d = 2, qutrits d = 3,
 *     qudits of odd prime d); site j is base-d digit j of the index (least significant
 *     first).  A density matrix is d^N x d^N, row-major.  Amplitudes are interleaved (re, im):
 *     HADAMAG_C64 = two floats, HADAMAG_C128 = two doubles.  Device pointers must be 16-byte
 *     aligned (8-byte where a call says so).
 *   - States are NOT renormalised: every quantity is the paper's formula evaluated on the
 *     vector as given; lost_norm reports 1 - sum_P <P>^2 / 2^N (Sec. 4.1).
 *   - Ownership: every pointer belongs to the caller; the library never frees or keeps it
 *     after the call returns.  Scratch memory belongs to the context and is reused.
 *   - Ordering: work is enqueued on the caller's CUDA stream (NULL = legacy default
 *     stream).  Calls that return host values synchronise that stream before returning.
 *     A context is not thread-safe: use one per host thread.
 *   - Errors: every call returns a status code; nothing aborts, throws or traps.  Invalid
 *     arguments return HADAMAG_ERR_INVALID_ARG before any work is enqueued.
 *   - Precision: transforms run in FP32 (CUDA-core path) or on FP16 hi/lo tensor-core
 *     operands with FP32 accumulation (tensor path); every cross-tile sum and the final
 *     logarithm are FP64.  HADAMAG_C128 input is rounded to FP32 on the device first.
 */
#ifndef HADAMAG_H
#define HADAMAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HADAMAG_OK = 0,
    HADAMAG_ERR_INVALID_ARG = 1, /* bad N, n, count, null or misaligned pointer, bad list entry */
    HADAMAG_ERR_UNSUPPORTED = 2, /* valid request outside what the library implements */
    HADAMAG_ERR_OOM = 3,         /* device or pinned allocation failed */
    HADAMAG_ERR_CUDA = 4,        /* a CUDA runtime call failed (see hadamag_last_error) */
    HADAMAG_ERR_TIMEOUT = 5,     /* a bounded inter-CTA wait ran out; the launch stopped early */
    HADAMAG_ERR_NONFINITE = 6    /* the result is NaN or infinite (non-finite input) */
} hadamag_status;

typedef enum { HADAMAG_C64 = 0, HADAMAG_C128 = 1 } hadamag_dtype;

/* Transform path of the exact-SRE calls (hadamag_sre, hadamag_sre_host, hadamag_sre_terms,
 * hadamag_sre_mc).  TENSOR runs the tensor-core kernel where it exists (21 <= N <= 24, every
 * n) and the FP32 CUDA-core kernels for every other N; AUTO currently equals CUDACORE. */
typedef enum {
    HADAMAG_PATH_AUTO = 0,     /* the library picks */
    HADAMAG_PATH_CUDACORE = 1, /* FP32 butterflies on CUDA cores */
    HADAMAG_PATH_TENSOR = 2    /* +-1 Hadamard blocks on tcgen05 tensor cores, FP16 hi/lo operands */
} hadamag_path;

typedef struct hadamag_ctx_s* hadamag_ctx_t;
typedef struct CUstream_st* hadamag_stream_t; /* same type as cudaStream_t */

/* Create a context on `device` (CUDA ordinal).  Owns scratch buffers, a status word and a
 * private stream used by the host-buffer variants.  Returns INVALID_ARG for a null ctx
 * pointer or a bad ordinal, OOM/CUDA on failure. */
hadamag_status hadamag_create(hadamag_ctx_t* ctx, int device);
/* Free everything the context owns.  Null is accepted. */
hadamag_status hadamag_destroy(hadamag_ctx_t ctx);
/* Choose the transform path for later calls on this context (default AUTO); INVALID_ARG
 * for a value outside the enum. */
hadamag_status hadamag_set_path(hadamag_ctx_t ctx, hadamag_path path);
/* Fast path for non-integer n (off by default): with on = 1 the CUDA-core exact-SRE kernels
 * form |c|^{2n} as exp2f(n log2f(.)) in FP32 (summed in FP32 per thread, FP64 across threads)
 * instead of FP64 powers, where n <= 4 and n (N + 2) <= 100 (the values stay in FP32's normal
 * range for normalised states); elsewhere, and on the tensor path, FP64 powers are kept.  Error:
 * with log2f (1 ulp) and exp2f (2 ulp), and the FP32 rounding of n and of the product, a term
 * |c|^{2n} carries a relative error below (2 + 2 ln2 n |log2 |c|^2|) 2^-23, about
 * (2 + 2 ln2 n N) 2^-23 for the terms of typical size 2^-N that dominate the sum, so
 * |dM_n| <~ (2 + 2 ln2 n N) 2^-23 / (ln2 |1 - n|) beyond the FP32 transform's own error.
 * INVALID_ARG for a value other than 0 or 1. */
hadamag_status hadamag_set_fp32_powers(hadamag_ctx_t ctx, int on);
/* Bound of every inter-CTA wait, in polling iterations (~0.1 us each; default 2^25), and a
 * value added to every wait target.  A non-zero bias makes waits unsatisfiable; it exists
 * only so tests can check that a wait that runs out returns HADAMAG_ERR_TIMEOUT. */
hadamag_status hadamag_set_wait_limit(hadamag_ctx_t ctx, long long spins, unsigned bias);
/* Number of kernel launches this context has issued since creation. */
hadamag_status hadamag_launch_count(hadamag_ctx_t ctx, uint64_t* count);
const char* hadamag_status_string(hadamag_status s);
/* Text of the last error recorded on this context ("" if none). */
const char* hadamag_last_error(hadamag_ctx_t ctx);

/*
 * Launch-shape autotuning (not in the paper: the x-batch, the shared-memory split and the task
 * shapes are picked by timing candidates on the device).  On by default.  With it on, the first uncaptured exact-SRE call of a
 * context for a given N >= 16 and n times each candidate shape of the two-pass kernel on a
 * bounded range of X-strings (units per pass-1 warp {2, 4}, column tiles per pass-2 task {2, 4},
 * a lag of 1 or 2 stages between a batch's first and second pass, at N = 20 also 2, 3 or 4 ring
 * slots; where a stage holds few tasks also the lag that puts 1.5 grid rounds of tasks between
 * the two passes, with lag + 1 slots) and keeps the fastest for that context; at N = 15 it tunes
 * the shared-memory split
 * itself: the whole 2^14-value transform in one CTA (one pass) against two passes through L2.
 * The adjoint (hadamag_sre_grad, N >= 16) tunes its x-batch (8 or 2 X-strings per batch) the
 * same way, and the batched call its x-batch (8, 4 or 2) per large state size on up to two
 * states of that size.  Results agree between shapes up to the
 * order of the FP64 partial sums.  Calls over at most 64 X-strings (Algorithm 3's steps, short
 * lists) use the two-pass shape with the most, smallest tasks (or a pinned one) and do not tune.
 * hadamag_set_autotune(ctx, 0) uses the default shapes (no
 * tuning launches; one pass at N = 15).  hadamag_twopass_shape reports the shape in use for
 * (N, n): out5 = [units per pass-1 warp, column tiles per pass-2 task, ring slots, X-strings per
 * batch, lag], all 0 before the tuner ran, all -1 when N = 15 runs one pass (15 <= N <= 24;
 * host pointer to 5 ints).
 */
hadamag_status hadamag_set_autotune(hadamag_ctx_t ctx, int on);
hadamag_status hadamag_twopass_shape(hadamag_ctx_t ctx, int N, double n, int* out5);
/* Pins the shape for (N, n) instead of tuning it: upw units per pass-1 warp (2 or 4 for
 * N <= 20, 2 above), tpt column tiles per pass-2 task (a divisor of the tiles per X-string),
 * R ring slots (2..63, or 0 for the default), lag stages between the two passes of a batch
 * (1 <= lag < slots); upw = -1 at N = 15 selects the one-pass kernel.  INVALID_ARG for any other
 * value. */
hadamag_status hadamag_set_twopass_shape(hadamag_ctx_t ctx, int N, double n, int upw, int tpt, int R, int lag);
/* Pins the adjoint's x-batch for N (16 <= N <= 20): A = 8, 4 or 2 X-strings per batch of the
 * three-pass kernel instead of tuning it.  INVALID_ARG for any other N or A. */
hadamag_status hadamag_set_grad_xbatch(hadamag_ctx_t ctx, int N, int A);

/*
 * Exact stabilizer Renyi entropy, Eq. (sre) of Sec. 2, evaluated by the per-X-string
 * Walsh-Hadamard method of Sec. 3.1.2 (Algorithm 2):
 *     M_n = 1/(1-n) log2( sum_{a,b} |<psi|X_a Z_b|psi>|^{2n} / 2^N ),
 *     M_1 = -sum_P pi_P log2 pi_P - N with pi_P = <P>^2 / sum_P <P>^2 (limit n -> 1),
 *     lost_norm = 1 - sum_P <P>^2 / 2^N (Sec. 4.1).
 * psi_dev: 2^N amplitudes on the device.  1 <= N <= 24, n > 0 (n = 1, 2, 3 have dedicated
 * kernels; other n accumulate exp2(n log2 |c|^2) in FP64).  M_out and lost_norm_out are host
 * pointers (lost_norm_out may be NULL).  Synchronises `stream`.
 */
hadamag_status hadamag_sre(hadamag_ctx_t ctx, const void* psi_dev, int N, double n,
                           hadamag_dtype dtype, double* M_out, double* lost_norm_out,
                           hadamag_stream_t stream);

/*
 * hadamag_sre over the even-weight X-strings only (Sec. 3.2): for states with U(1) symmetry
 * (conserved sum_j Z_j) or the Z_2 symmetry prod_j Z_j, <psi|X_a Z_b|psi> = 0 whenever |a| is
 * odd, so the 2^(N-1) even-weight X-strings a = 2i + parity(i) carry all of Eq. (sre) and the
 * work halves.  Same outputs, limits and path selection as hadamag_sre; the symmetry is the
 * caller's claim (for other states the result is the even-sector part only).
 */
hadamag_status hadamag_sre_even_sector(hadamag_ctx_t ctx, const void* psi_dev, int N, double n,
                                       hadamag_dtype dtype, double* M_out, double* lost_norm_out,
                                       hadamag_stream_t stream);

/* Same as hadamag_sre with psi in HOST memory: the call copies it to the device on the
 * context's own stream (inside the call), computes, and returns host results. */
hadamag_status hadamag_sre_host(hadamag_ctx_t ctx, const void* psi_host, int N, double n,
                                hadamag_dtype dtype, double* M_out, double* lost_norm_out);

/*
 * Per-X-string sums of Algorithm 2 for an explicit list of X-strings:
 *     terms_dev[3i+0] = sum_b |chi_b(a_i)|^{2n},  terms_dev[3i+1] = sum_b |chi_b(a_i)|^2,
 *     terms_dev[3i+2] = sum_b |chi_b|^2 log2 |chi_b|^2 (n = 1 only, else 0),
 * with chi_b(a) = <psi| X_a Z_b |psi> (Eq. Z_FT_qubits).  1 <= N <= 28 (n = 2 only for N > 24,
 * where the scratch of one X-string exceeds L2 and a three-pass HBM schedule is used).
 * a_list_dev: `count` int64 entries
 * in [0, 2^N) on the device (an entry outside gives INVALID_ARG after the launch and its
 * terms are left unwritten).  terms_dev: count*3 doubles on the device.  Stream-ordered;
 * synchronises `stream` to read the status word.
 */
hadamag_status hadamag_sre_terms(hadamag_ctx_t ctx, const void* psi_dev, int N, double n,
                                 hadamag_dtype dtype, const int64_t* a_list_dev, int64_t count,
                                 double* terms_dev, hadamag_stream_t stream);

/*
 * X-strings of the uniform Monte-Carlo estimator: a_i = top N bits of output i of
 * SplitMix64 (Steele, Lea & Flood 2014) started at `seed`, i = 0..count-1, written to
 * a_out_dev (count int64 on the device).  1 <= N <= 30.  Stream-ordered, no sync.
 */
hadamag_status hadamag_mc_xstrings(hadamag_ctx_t ctx, uint64_t seed, int64_t count, int N,
                                   int64_t* a_out_dev, hadamag_stream_t stream);

/*
 * Uniform-X Monte-Carlo M_2 (from the per-X decomposition of Algorithm 2): with
 * S(a) = sum_b |chi_b(a)|^4, the X-string a = 0 (it holds the identity string, which the paper
 * also takes out of its sampling, Sec. 4.2 footnote) is evaluated exactly and `samples`
 * X-strings are drawn as in hadamag_mc_xstrings, those equal to 0 being dropped:
 *     S_hat = [S(0) + (2^N - 1) mean_{a_i != 0} S(a_i)] / 2^N  (unbiased for S_2 / 2^N),
 *     M2_hat = -log2(S_hat),  stderr = (1 - 2^-N) sd / sqrt(n) / (S_hat ln 2) (Eq. M2mNcerror).
 * 1 <= N <= 28 (N >= 25 uses a three-pass HBM schedule).  stderr_out may be NULL.
 * Synchronises `stream`.
 */
hadamag_status hadamag_sre_mc(hadamag_ctx_t ctx, const void* psi_dev, int N, int64_t samples,
                              uint64_t seed, hadamag_dtype dtype, double* M2_out,
                              double* stderr_out, hadamag_stream_t stream);

/*
 * Thermodynamic-integration estimate of M_2, Sec. 3.2 (Eqs. Boltz to M2_TI, Algorithm 3).
 * L Metropolis chains at beta_l = l / (L-1), l = 0..L-1, sample X-strings from
 * Pi_beta(a) ~ exp(-beta f(a)) with f(a) = -ln(S(a) + eps), S(a) = sum_b |chi_b(a)|^4; each step
 * proposes a one-bit flip and accepts it when u < min(1, exp(-beta (f' - f))) (FP64).  After
 * burn_in unrecorded steps, n_s steps are averaged into the chain means <f>_l, and
 *     I = sum_l w_l <f>_l  (composite Simpson; 3/8 rule on the last three intervals for even L),
 *     M2_out = -log2(exp(-I) - eps)  (= I / ln 2 for eps = 0).
 * Sign: the identity <f>_beta = -d ln Z_beta / d beta fixes I = ln Z_0 - ln Z_1; the printed
 * return value of Algorithm 3 has the opposite sign.  Random numbers: chain l reads SplitMix64
 * started at seed + l (as in hadamag_mc_xstrings): output 0 -> start pattern (top N bits),
 * output 1 + 2t -> bit flipped at step t (mod N), output 2 + 2t -> u = (top 53 bits) / 2^53.
 * sector = 1 restricts the chains to even-weight X-strings, the sectors that survive a U(1) or
 * prod_j Z_j symmetry (Sec. 3.2; N >= 2): the start pattern has bit 0 flipped when its weight
 * is odd, a move flips bits b1 = r mod N and b2 = (r div N) mod (N-1) (+1 if b2 >= b1) of step
 * output r, and Z_0 = 2^(N-1) gives M2_out = 1 - log2(exp(-I) - eps).  Valid only for states
 * whose odd-weight sectors vanish; sectors that also vanish (U(1) away from half filling)
 * still need eps > 0.
 * Energies come from the FP32 CUDA-core per-X kernels of hadamag_sre_terms (the path setting is
 * not used).
 * Arguments: 1 <= N <= 24; 3 <= L <= 4096; n_s >= 1, burn_in >= 0, n_s + burn_in < 2^31;
 * eps >= 0 (eps > 0 is needed when S(a) can vanish, e.g. stabilizer states).  means_out: L host
 * doubles or NULL.  traj_dev: NULL or L * (burn_in + n_s) int64 on the device, 8-byte aligned,
 * receiving traj[l * (burn_in + n_s) + t] = chain l's X-string after step t.
 * stderr_out (host double or NULL): the statistical error of Eqs. Var_I_eps / m2error,
 * delta M_2 = exp(-I) / ((exp(-I) - eps) ln 2) * sqrt(sum_l w_l^2 Var_l), with Var_l (the variance
 * of chain l's mean, autocorrelation included) from non-overlapping batch means: B = min(32, n_s)
 * batches of n_s div B consecutive recorded steps, Var_l = sum_b (m_b - mbar)^2 / (B (B - 1));
 * 0 when n_s < 2.
 * Errors: NONFINITE when an evaluated S(a) + eps is 0 or the estimate is not finite.
 * Synchronises `stream`.
 */
hadamag_status hadamag_sre_ti(hadamag_ctx_t ctx, const void* psi_dev, int N, int L, int64_t n_s,
                              int64_t burn_in, uint64_t seed, double eps, int sector,
                              hadamag_dtype dtype, double* M2_out, double* stderr_out,
                              double* means_out, int64_t* traj_dev, hadamag_stream_t stream);

/*
 * Mana of an N-qutrit pure state, Eq. (mana2) of Sec. 2 evaluated by the per-X-string
 * Z_3^N Fourier transform of Sec. 3.3.2 (Algorithm 5, Eqs. mana_FT and F3_unnorm_def):
 *     mana = log2( sum_{a,b} |chi_b(a)| / 3^N ),  chi = F_3^{(x)N} (alpha*_x alpha_{-x}).
 * mana_out is in bits (the paper's log2); sum_w_out = sum_u |W(u)| (so ln sum_w is the
 * natural-log mana).  1 <= N <= 13.  Either output may be NULL.  Synchronises `stream`.
 */
hadamag_status hadamag_mana(hadamag_ctx_t ctx, const void* psi_dev, int N, hadamag_dtype dtype,
                            double* mana_out, double* sum_w_out, hadamag_stream_t stream);

/* Raw sums behind hadamag_mana: sums_out[0] = sum_{a,b} |chi_b(a)|, sums_out[1] = sum chi_b(a),
 * sums_out[2] = sum chi_b(a)^2 (host doubles).  With W = chi / 3^N these give the Wigner sum
 * rules of Sec. 2: sum_u W(u) = 1 and, for pure states, sum_u W(u)^2 = 3^-N. */
hadamag_status hadamag_mana_sums(hadamag_ctx_t ctx, const void* psi_dev, int N, hadamag_dtype dtype,
                                 double* sums_out, hadamag_stream_t stream);

/*
 * Mana of N qudits of odd prime dimension d, Sec. 2 (the qutrit construction holds for any odd
 * prime d): with w = e^{2 pi i / d}, T_ab = w^{-2^{-1} ab} Z^a X^b, A_0 = d^-N sum_u T_u,
 * A_u = T_u A_0 T_u^dag and W(u) = <psi|A_u|psi> / d^N,  mana = log2 sum_u |W(u)|.
 * Algorithm 5 generalised: for every shift a, v_x = conj(psi_{x-a}) psi_{-x-a} (digit-wise
 * mod d), chi = F_d^{(x)N} v with (F_d)_jk = w^{2jk}, W = chi / d^N (a relabelling of u).
 * psi_dev: d^N amplitudes, qudit j = base-d digit j.  d = 3 (1 <= N <= 13, the hadamag_mana
 * kernels), 5 (N <= 6), 7 (N <= 5), 11 (N <= 4), 13 (N <= 3); other d give UNSUPPORTED.
 * sums_out (3 host doubles or NULL): [sum |chi|, sum chi, sum chi^2] over all (a, b).
 * Synchronises `stream`.
 */
hadamag_status hadamag_mana_qudit(hadamag_ctx_t ctx, const void* psi_dev, int N, int d,
                                  hadamag_dtype dtype, double* mana_out, double* sums_out,
                                  hadamag_stream_t stream);

/*
 * Mana and its Wirtinger gradient d mana / d psi* for N qudits of odd prime dimension d (not in
 * the paper; the analogue of hadamag_sre_grad for Eq. mana2).  With chi as in hadamag_mana_qudit
 * and m = sum_{a,b} |chi_b(a)|:  d chi_b(a) / d psi*_w = d conj(chi_b(a)) / d psi*_w =
 * F_{b,w+a} psi_{-w-2a}, so with G_a = F_d^{(x)N} (Re chi_a / |chi_a|),
 *     d m / d psi*_{y-a} += psi_{-y-a} G_a(y),   d mana / d psi* = (d m / d psi*) / (m ln 2),
 * on the vector as given (not renormalised); undefined where some chi_b(a) = 0 (stabilizer
 * states).  d = 3, 5, 7, 11, 13 with d^N <= 25600 (qutrits: N <= 9).  grad_dev: d^N amplitudes
 * of the same dtype as psi on the device.  Per-CTA partials are summed in FP64 in a fixed
 * order.  Synchronises `stream`.
 */
hadamag_status hadamag_mana_grad(hadamag_ctx_t ctx, const void* psi_dev, int N, int d,
                                 hadamag_dtype dtype, double* mana_out, void* grad_dev,
                                 hadamag_stream_t stream);

/*
 * Mana of an N-qutrit density matrix, Sec. 3.3.3 (Algorithm 6; Eq. mana with
 * W_u = tr(rho A_u) / 3^N over the phase-space point operators A_u):
 *     mana = log2 sum_u |W_u|  (bits; 0 for stabilizer mixtures, equal to hadamag_mana on pure states).
 * rho_dev: 3^N x 3^N complex (dtype), row-major, rho[r * 3^N + c], qutrit j = base-3 digit j of
 * r and c; Hermitian (W is real only then: the imaginary part is not used), trace not enforced.
 * Computation: for every a, v_x = rho[-x - a, x - a] (digit-wise mod 3) is transformed by
 * F_3^{(x)N} exactly as in hadamag_mana; the values are Algorithm 6's 3^N W_u up to the
 * labelling of u, and every entry of rho is read once.
 * sums_out (3 host doubles or NULL): [sum |chi|, sum chi, sum chi^2] over all (a, b), so that
 * sum chi = 3^N tr rho and sum chi^2 = 3^N tr rho^2.  1 <= N <= 10 (rho is 9^N values: 28 GB of
 * complex64 at N = 10; complex128 input is first rounded into a complex64 copy of that size).
 * Synchronises `stream`.
 */
hadamag_status hadamag_mana_mixed(hadamag_ctx_t ctx, const void* rho_dev, int N, hadamag_dtype dtype,
                                  double* mana_out, double* sums_out, hadamag_stream_t stream);

/*
 * hadamag_mana_mixed for N qudits of odd prime dimension d (Sec. 2: the construction holds for
 * any odd prime d): rho_dev is d^N x d^N complex (dtype), row-major, qudit j = base-d digit j;
 * v_x = rho[-x - a, x - a] digit-wise mod d, F_d^{(x)N} with (F_d)_jk = w^{2jk}, W = chi / d^N.
 * d = 3 is hadamag_mana_mixed (N <= 10); d = 5, 7, 11, 13 need d^N <= 25600 (N <= 6, 5, 4, 3);
 * other d give UNSUPPORTED.  sums_out as for hadamag_mana_mixed.  Synchronises `stream`.
 */
hadamag_status hadamag_mana_mixed_qudit(hadamag_ctx_t ctx, const void* rho_dev, int N, int d,
                                        hadamag_dtype dtype, double* mana_out, double* sums_out,
                                        hadamag_stream_t stream);

/*
 * Reduced density matrix of an N-qutrit pure state (the partial trace that gives the mixed
 * states of Sec. 3.3.3):  rho_A[r, c] = sum_x psi[(r, x)] conj(psi[(c, x)]), where site keep[m]
 * is base-3 digit m of r and c and x runs over the other sites.  keep: n_keep distinct sites
 * (host ints) in [0, N); 1 <= n_keep <= min(N, 10); 1 <= N <= 16.  rho_dev: 3^n_keep x 3^n_keep
 * complex64 on the device (row-major, 8-byte aligned), written with FP32 products summed in
 * FP64 over chunks of 32 traced-out indices.  Stream-ordered, no synchronisation.
 */
hadamag_status hadamag_reduced_density_matrix(hadamag_ctx_t ctx, const void* psi_dev, int N,
                                              hadamag_dtype dtype, const int* keep, int n_keep,
                                              void* rho_dev, hadamag_stream_t stream);
/* The same for sites of dimension d (2 <= d <= 13): psi_dev has d^N amplitudes (site j = base-d
 * digit j), d^N <= 3^16 and d^n_keep <= 3^10; rho_dev is d^n_keep x d^n_keep complex64. */
hadamag_status hadamag_reduced_density_matrix_qudit(hadamag_ctx_t ctx, const void* psi_dev, int N, int d,
                                                    hadamag_dtype dtype, const int* keep, int n_keep,
                                                    void* rho_dev, hadamag_stream_t stream);

/*
 * M_2 and its Wirtinger gradient dM_2/dpsi* (not in the paper; it is what magic
 * optimisation of circuits needs).  With c_a = H^{(x)N} v_a as in Algorithm 2,
 *     dS_2/dpsi*_w = sum_a psi_{w^a} [G_a(w) + conj(G_a(w^a))],  G_a = H^{(x)N}(2|c_a|^2 c_a),
 *     dM_2/dpsi* = -dS_2/dpsi* / (ln 2 S_2).
 * The adjoint recomputes c_a instead of storing 4^N values.  grad_dev: 2^N amplitudes of the
 * same dtype as psi, on the device.  1 <= N <= 20.  Synchronises `stream`.
 */
hadamag_status hadamag_sre_grad(hadamag_ctx_t ctx, const void* psi_dev, int N, hadamag_dtype dtype,
                                double* M2_out, void* grad_dev, hadamag_stream_t stream);

/*
 * One state's computation split by X-string, for several GPUs or several calls.  The a-loop of
 * Algorithm 2 is a sum of independent per-X-string terms, which Sec. 4.1 distributes over
 * threads, processes and GPUs, combining their partial sums with one reduction.
 *
 * hadamag_sre_chunk(N): the chunk size, 2^min(N, 12) X-strings (0 for N outside [1, 24]).
 * Every slice starts and ends on a multiple of it.
 *
 * hadamag_sre_slice: the sums of Eq. (sre) over the X-strings a0 <= a < a1, one triple
 * [sum |c|^{2n}, sum |c|^2, sum |c|^2 log2 |c|^2 (n = 1, else 0)] per chunk of consecutive
 * X-strings, written to chunks_dev ((a1 - a0) / chunk * 3 doubles on the device, 8-byte
 * aligned), chunk k of the slice holding the X-strings a0 + k chunk .. a0 + (k + 1) chunk - 1.
 * A chunk's triple is a fixed-order FP64 sum that depends only on the chunk, so every
 * chunk-aligned partition of [0, 2^N) yields the same triples bit for bit, on any GPU.
 * Same N, n, dtype and path rules as hadamag_sre; a0, a1 multiples of the chunk size with
 * 0 <= a0 <= a1 <= 2^N (else INVALID_ARG).  Synchronises `stream` to read the status word.
 *
 * hadamag_sre_combine (host only, no CUDA call): adds the 2^N / chunk triples of all slices in
 * chunk order (chunks_host, host memory, gathered from every slice) and returns M_n and
 * lost_norm as hadamag_sre does.  INVALID_ARG if nchunks is not 2^N / chunk.
 */
int64_t hadamag_sre_chunk(int N);
hadamag_status hadamag_sre_slice(hadamag_ctx_t ctx, const void* psi_dev, int N, double n,
                                 hadamag_dtype dtype, int64_t a0, int64_t a1, double* chunks_dev,
                                 hadamag_stream_t stream);
hadamag_status hadamag_sre_combine(int N, double n, const double* chunks_host, int64_t nchunks,
                                   double* M_out, double* lost_norm_out);

/*
 * The adjoint of hadamag_sre_grad split by X-string in the same way.
 * hadamag_sre_grad_slice: the part of dS_2/dpsi* contributed by the X-strings a0 <= a < a1
 * (unscaled; the sum over a of the adjoint formula above restricted to the slice) into dS_dev
 * (2^N complex128 on the device, overwritten), and sums_out[0] = that slice's part of S_2,
 * sums_out[1] = its part of sum |c|^2 (host doubles).  1 <= N <= 20; a0, a1 multiples of
 * hadamag_sre_chunk(N).  Synchronises `stream`.
 * hadamag_sre_grad_combine: from the dS_2/dpsi* and S_2 summed over all slices (e.g. by an
 * all-reduce), grad_dev = -dS / (ln 2 S_2) (2^N amplitudes of `dtype` on the device) and
 * M2_out = -log2(S_2 / 2^N) (host).  S_2 must be finite and > 0.  Synchronises `stream`.
 */
hadamag_status hadamag_sre_grad_slice(hadamag_ctx_t ctx, const void* psi_dev, int N, hadamag_dtype dtype,
                                      int64_t a0, int64_t a1, double* sums_out, void* dS_dev,
                                      hadamag_stream_t stream);
hadamag_status hadamag_sre_grad_combine(hadamag_ctx_t ctx, const void* dS_dev, int N, double S2,
                                        hadamag_dtype dtype, double* M2_out, void* grad_dev,
                                        hadamag_stream_t stream);

/*
 * Many states of uneven N (10 <= N_i <= 18, complex64) in ONE persistent launch (the batched
 * form for many states of uneven N; not in the paper): M_2 of state i into M2_dev[i] (device doubles) and, if
 * want_grad, dM_2/dpsi* into grad_dev[i] (complex64).  psi_dev and grad_dev are HOST arrays of
 * `count` device pointers.  States with N <= 14 are one CTA item each; larger states run the
 * three-pass adjoint; the work list is ordered largest first and taken through a dynamic
 * ticket counter.  The X-strings per pass-1 task come from the context's autotuner (timed on
 * the first uncaptured call for a given set of sizes).  Stream-ordered, no host sync and no
 * allocation once the context's buffers have grown, so after one uncaptured call with the same
 * shapes the call can be captured in a CUDA graph.  Read the device status with
 * hadamag_batched_status.
 */
hadamag_status hadamag_sre_batched(hadamag_ctx_t ctx, int count, const void* const* psi_dev,
                                   const int* N, int want_grad, void* const* grad_dev,
                                   double* M2_dev, hadamag_stream_t stream);
/* Synchronises `stream` and reports the device status word of the preceding batched call
 * (HADAMAG_OK, or HADAMAG_ERR_TIMEOUT if a bounded wait ran out). */
hadamag_status hadamag_batched_status(hadamag_ctx_t ctx, hadamag_stream_t stream);

/*
 * Allocation-free exact SRE.  The paper has no counterpart; this is a calling convenience for
 * callers that cannot allocate device memory where they need the number: code inside a host
 * application or framework that owns all device memory through its own pool or a budget fixed at
 * start-up, latency-critical loops that must not pay the device-wide synchronisation of
 * cudaMalloc / cudaFree, and plugins that must not grow the process's device footprint.  No
 * context is needed and nothing is allocated: the scratch is a fixed 8.06 MiB __device__ array
 * inside the library, held by every GPU that loads the library until the process exits.
 *   psi_dev: 2^N complex64 amplitudes on the current device, 16-byte aligned.
 *   16 <= N <= 20 (other N: HADAMAG_ERR_UNSUPPORTED, nothing enqueued: the array holds the
 *   scratch of N = 20 at most); n > 0 as hadamag_sre.
 *   out_dev: 3 doubles on the device, 8-byte aligned, written in stream order:
 *   [M_n, lost_norm, status] (status 0 = ok; otherwise the device-side check bits, and M_n is NaN).
 * The call enqueues its kernels on `stream` and returns without synchronising.  Every call
 * on a device shares the same array (it keeps the last call's contents; each call clears
 * what must start at zero), so calls that overlap on the GPU race: serialise them.  The
 * first call on a device does the set-up (it looks up the array's address with that device
 * current); make it before any stream capture.  Not valid on a device after cudaDeviceReset.
 */
hadamag_status hadamag_sre_noalloc(const void* psi_dev, int N, double n, double* out_dev,
                                   hadamag_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* HADAMAG_H */
