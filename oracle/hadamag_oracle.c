/*
 * hadamag_oracle.c -- plain, slow, FP64 CPU reference ("oracle") for the stabilizer
 * Renyi entropy (SRE) of qubit state vectors and the mana of qutrit state vectors.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file: only the tests, the entry point's smoke check and the benchmark's CPU-baseline
 * leg use it.  It shares no code, header, table or constant with the CUDA library.
 *
 * Paper: "Computing quantum magic of state vectors" (arXiv 2601.07824).
 *   - SRE, Eq. (sre) of Sec. 2:  M_q = 1/(1-q) log2[ sum_{a,b} <psi|P_{a,b}|psi>^{2q} / 2^N ].
 *   - Algorithm 2 (Sec. 3.1.2, Eqs. Z_FT_qubits / Z_ovN_simplified): for each X-string a,
 *     v_x = beta_x^* alpha_x with beta = X_a psi (so beta_x = psi_{x xor a}), then
 *     chi = H_2^{(x)N} v (unnormalised Walsh-Hadamard), S_q += sum_b |chi_b|^{2q}.
 *   - Mana, Eqs. (mana), (mana2) of Sec. 2 and Algorithm 5 (Sec. 3.3.2, Eqs.
 *     def_psiprime_mana, mana_FT, F3_unnorm_def): for each a in Z_3^N, alpha = amplitudes
 *     of X^a psi, v_x = alpha_x^* alpha_{-x}, chi = F_3^{(x)N} v with (F_3)_{jk} = w^{2jk},
 *     m += sum_b |chi_b|;  mana = log2(m / 3^N).
 *   - lost_norm = 1 - sum_P <P>^2 / 2^N (Sec. 4.1, Eq. distNAT).
 *
 * Readings where the paper is silent or garbled:
 *   R1  Algorithm 2 accumulates chi_b^{2q}; X_a Z_b is anti-Hermitian when a.b is odd, so
 *       chi_b is then imaginary.  Eq. (sre) uses Hermitian Pauli strings (real <P>), so the
 *       accumulated term is |chi_b|^{2q}.
 *   R2  M_1 is "the limit q -> 1" of Eq. (sre).  It is computed as the Shannon entropy of
 *       pi_P = |chi|^2 / sum|chi|^2 minus N (0 log 0 = 0), equal to the limit for unit norm.
 *   R3  Algorithm 5 returns log2(m) without the 1/3^N of Eq. (mana2); the oracle uses
 *       Eq. (mana2), log2(m / 3^N), which gives 0 on |0...0> as the paper's example does.
 *   R4  Base-3 digit j of an index is qutrit j; -x and x - a are digit-wise mod 3.
 *   R5  Gradient (not in the paper): f = M_2 on the unnormalised psi; Wirtinger derivative
 *       dM2/dpsi*_w = -1/(ln2 S_2) sum_a psi_{w xor a} [G_a(w) + conj(G_a(w xor a))],
 *       G_a = H^{(x)N}(2 |c_a|^2 c_a), c_a = H^{(x)N} v_a.
 *   R6  Uniform-X Monte Carlo (not an algorithm of the paper; it follows from the per-X
 *       decomposition of Algorithm 2): a_i = top N bits of SplitMix64 output i, S(a) =
 *       sum_b |chi_b(a)|^4.  As the paper does for the identity string (Sec. 4.2 footnote: it is
 *       excluded from sampling and its contribution added exactly), the X-string a = 0, which
 *       contains the identity, is evaluated exactly and the samples with a_i = 0 are dropped:
 *       S_hat = [S(0) + (2^N - 1) mean_{a_i != 0} S(a_i)] / 2^N, M2_hat = -log2(S_hat).
 *
 * All state vectors are interleaved (re, im) doubles.  Functions return 0 on success and
 * a negative number on bad arguments or allocation failure.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int orc_num_threads(int nthreads) { return set_threads(nthreads); }

static const cplx *as_cplx(const double *p) { return (const cplx *)p; }

/* In-place unnormalised Walsh-Hadamard transform H_2^{(x)n}, radix 2, bit by bit. */
static void fwht(cplx *v, int64_t len) {
    for (int64_t h = 1; h < len; h <<= 1)
        for (int64_t i = 0; i < len; i += 2 * h)
            for (int64_t j = i; j < i + h; ++j) {
                cplx x = v[j], y = v[j + h];
                v[j] = x + y;
                v[j + h] = x - y;
            }
}

/* chi_b(a) for all b into `chi` (Algorithm 2, one iteration of its loop over a). */
static void sre_chi(const cplx *psi, int N, int64_t a, cplx *chi) {
    int64_t dim = (int64_t)1 << N;
    for (int64_t x = 0; x < dim; ++x) chi[x] = conj(psi[x ^ a]) * psi[x];
    fwht(chi, dim);
}

/*
 * Per-X-string terms for a in [a0, a1):
 *   Sq[i] = sum_b |chi_b(a)|^{2q}   (q = 1: Sq[i] = S1[i]),
 *   S1[i] = sum_b |chi_b(a)|^2,
 *   T1[i] = sum_b |chi_b|^2 log2 |chi_b|^2   (0 log 0 = 0).
 * Any of the output pointers may be NULL.
 */
int orc_sre_terms(const double *psi_ri, int N, double q, int64_t a0, int64_t a1, int nthreads,
                  double *Sq, double *S1, double *T1) {
    if (N < 1 || N > 30 || a0 < 0 || a1 < a0 || a1 > ((int64_t)1 << N) || !(q > 0)) return -1;
    const cplx *psi = as_cplx(psi_ri);
    int64_t dim = (int64_t)1 << N;
    int err = 0;
    set_threads(nthreads);
#pragma omp parallel
    {
        cplx *chi = (cplx *)malloc(sizeof(cplx) * dim);
        if (!chi) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t a = a0; a < a1; ++a) {
            if (!chi) continue;
            sre_chi(psi, N, a, chi);
            double sq = 0.0, s1 = 0.0, t1 = 0.0;
            for (int64_t b = 0; b < dim; ++b) {
                double p = creal(chi[b]) * creal(chi[b]) + cimag(chi[b]) * cimag(chi[b]);
                s1 += p;
                sq += (q == 1.0) ? p : pow(p, q);
                if (p > 0.0) t1 += p * log2(p);
            }
            if (Sq) Sq[a - a0] = sq;
            if (S1) S1[a - a0] = s1;
            if (T1) T1[a - a0] = t1;
        }
        free(chi);
    }
    return err;
}

/* Sums of per-a terms in a fixed order, then Eq. (sre) (R1, R2) and lost_norm. */
int orc_sre(const double *psi_ri, int N, double q, int nthreads, double *M, double *lost_norm) {
    if (N < 1 || N > 30 || !(q > 0)) return -1;
    int64_t dim = (int64_t)1 << N;
    double *Sq = (double *)malloc(sizeof(double) * dim);
    double *S1 = (double *)malloc(sizeof(double) * dim);
    double *T1 = (double *)malloc(sizeof(double) * dim);
    if (!Sq || !S1 || !T1) {
        free(Sq); free(S1); free(T1);
        return -2;
    }
    int rc = orc_sre_terms(psi_ri, N, q, 0, dim, nthreads, Sq, S1, T1);
    if (rc == 0) {
        double sq = 0.0, s1 = 0.0, t1 = 0.0;
        for (int64_t a = 0; a < dim; ++a) { sq += Sq[a]; s1 += S1[a]; t1 += T1[a]; }
        double two_n = ldexp(1.0, N);
        if (q == 1.0)
            *M = -t1 / s1 + log2(s1) - (double)N; /* R2 */
        else
            *M = log2(sq / two_n) / (1.0 - q);
        *lost_norm = 1.0 - s1 / two_n;
    }
    free(Sq); free(S1); free(T1);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Gradient of M_2 (R5).                                                                */

int orc_sre_grad(const double *psi_ri, int N, int nthreads, double *M2, double *grad_ri) {
    if (N < 1 || N > 24) return -1;
    const cplx *psi = as_cplx(psi_ri);
    int64_t dim = (int64_t)1 << N;
    int nt = set_threads(nthreads);
    cplx *acc = (cplx *)calloc((size_t)dim * nt, sizeof(cplx)); /* one partial per thread */
    double *s2_part = (double *)calloc((size_t)nt, sizeof(double));
    if (!acc || !s2_part) {
        free(acc); free(s2_part);
        return -2;
    }
    int err = 0;
#pragma omp parallel num_threads(nt)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        cplx *c = (cplx *)malloc(sizeof(cplx) * dim);
        cplx *G = (cplx *)malloc(sizeof(cplx) * dim);
        if (!c || !G) {
#pragma omp atomic write
            err = -2;
        }
        cplx *mine = acc + (size_t)t * dim;
        double s2 = 0.0;
#pragma omp for schedule(static)
        for (int64_t a = 0; a < dim; ++a) {
            if (!c || !G) continue;
            sre_chi(psi, N, a, c);
            for (int64_t b = 0; b < dim; ++b) {
                double p = creal(c[b]) * creal(c[b]) + cimag(c[b]) * cimag(c[b]);
                s2 += p * p;
                G[b] = 2.0 * p * c[b];
            }
            fwht(G, dim); /* H is symmetric: G_a(w) = sum_b (-1)^{b.w} 2|c_b|^2 c_b */
            for (int64_t w = 0; w < dim; ++w)
                mine[w] += psi[w ^ a] * (G[w] + conj(G[w ^ a]));
        }
        s2_part[t] = s2;
        free(c); free(G);
    }
    if (err == 0) {
        double s2 = 0.0;
        for (int t = 0; t < nt; ++t) s2 += s2_part[t];
        double scale = -1.0 / (log(2.0) * s2);
        cplx *g = (cplx *)grad_ri;
        for (int64_t w = 0; w < dim; ++w) {
            cplx sum = 0.0;
            for (int t = 0; t < nt; ++t) sum += acc[(size_t)t * dim + w];
            g[w] = scale * sum;
        }
        *M2 = -log2(s2 / ldexp(1.0, N));
    }
    free(acc); free(s2_part);
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* Uniform-X Monte Carlo (R6).  SplitMix64 (Steele, Lea & Flood, OOPSLA 2014):          */
/* state_i = seed + (i + 1) * gamma; output = mix(state_i).                              */

static uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

void orc_splitmix64(uint64_t seed, int64_t count, uint64_t *out) {
    for (int64_t i = 0; i < count; ++i) out[i] = splitmix64_at(seed, (uint64_t)i);
}

void orc_mc_xstrings(uint64_t seed, int64_t count, int N, int64_t *a_out) {
    for (int64_t i = 0; i < count; ++i) a_out[i] = (int64_t)(splitmix64_at(seed, (uint64_t)i) >> (64 - N));
}

/* S(a) = sum_b |chi_b(a)|^4 for an explicit list of X-strings. */
int orc_sre_terms_list(const double *psi_ri, int N, const int64_t *a_list, int64_t count, int nthreads,
                       double *S_out) {
    if (N < 1 || N > 30) return -1;
    const cplx *psi = as_cplx(psi_ri);
    int64_t dim = (int64_t)1 << N;
    int err = 0;
    for (int64_t i = 0; i < count; ++i)
        if (a_list[i] < 0 || a_list[i] >= dim) return -1;
    set_threads(nthreads);
#pragma omp parallel
    {
        cplx *chi = (cplx *)malloc(sizeof(cplx) * dim);
        if (!chi) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t i = 0; i < count; ++i) {
            if (!chi) continue;
            sre_chi(psi, N, a_list[i], chi);
            double s = 0.0;
            for (int64_t b = 0; b < dim; ++b) {
                double p = creal(chi[b]) * creal(chi[b]) + cimag(chi[b]) * cimag(chi[b]);
                s += p * p;
            }
            S_out[i] = s;
        }
        free(chi);
    }
    return err;
}

int orc_sre_mc(const double *psi_ri, int N, int64_t samples, uint64_t seed, int nthreads,
               double *M2_hat, double *stderr_out, double *S_per_sample) {
    if (N < 1 || N > 30 || samples < 1) return -1;
    int64_t *a = (int64_t *)malloc(sizeof(int64_t) * samples);
    double *S = S_per_sample ? S_per_sample : (double *)malloc(sizeof(double) * samples);
    if (!a || !S) {
        free(a);
        if (!S_per_sample) free(S);
        return -2;
    }
    orc_mc_xstrings(seed, samples, N, a);
    int rc = orc_sre_terms_list(psi_ri, N, a, samples, nthreads, S);
    double S0 = 0.0;
    int64_t zero = 0;
    if (rc == 0) rc = orc_sre_terms_list(psi_ri, N, &zero, 1, nthreads, &S0);
    if (rc == 0) {
        double mean = 0.0, var = 0.0;
        int64_t n = 0;
        for (int64_t i = 0; i < samples; ++i)
            if (a[i] != 0) { mean += S[i]; ++n; }
        mean = n ? mean / (double)n : 0.0;
        for (int64_t i = 0; i < samples; ++i)
            if (a[i] != 0) var += (S[i] - mean) * (S[i] - mean);
        var = n > 1 ? var / (double)(n - 1) : 0.0;
        const double two_n = ldexp(1.0, N), w = (two_n - 1.0) / two_n;
        const double Shat = S0 / two_n + w * mean;
        *M2_hat = -log2(Shat);
        /* delta M ~ (1/ln 2) delta S / S with delta S = w sd / sqrt(n) (Eq. M2mNcerror) */
        *stderr_out = n ? w * sqrt(var / (double)n) / (Shat * log(2.0)) : 0.0;
    }
    free(a);
    if (!S_per_sample) free(S);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Mana (Algorithm 5 with R3, R4).                                                       */

static int64_t ipow3(int n) {
    int64_t r = 1;
    while (n-- > 0) r *= 3;
    return r;
}

/* In-place F_3^{(x)N}, (F_3)_{jk} = w^{2jk}, applied digit by digit. */
static void ft3(cplx *v, int N) {
    const double pi = 3.14159265358979323846;
    const cplx w = cexp(2.0 * pi * I / 3.0);
    const cplx w2 = w * w; /* w^2; w^4 = w */
    int64_t stride = 1;
    int64_t dim = ipow3(N);
    for (int j = 0; j < N; ++j) {
        for (int64_t base = 0; base < dim; base += 3 * stride)
            for (int64_t o = 0; o < stride; ++o) {
                int64_t i0 = base + o, i1 = i0 + stride, i2 = i1 + stride;
                cplx x0 = v[i0], x1 = v[i1], x2 = v[i2];
                v[i0] = x0 + x1 + x2;          /* k = 0 */
                v[i1] = x0 + w2 * x1 + w * x2; /* k = 1: w^{2}, w^{4} = w */
                v[i2] = x0 + w * x1 + w2 * x2; /* k = 2: w^{4} = w, w^{8} = w^2 */
            }
        stride *= 3;
    }
}

/* index of the digit-wise combination s1 * x + s2 * a (mod 3) */
static int64_t combine3(int64_t x, int64_t a, int sx, int sa, int N) {
    int64_t r = 0, p = 1;
    for (int j = 0; j < N; ++j) {
        int xd = (int)(x % 3), ad = (int)(a % 3);
        x /= 3; a /= 3;
        int d = ((sx * xd + sa * ad) % 3 + 6) % 3;
        r += d * p;
        p *= 3;
    }
    return r;
}

/*
 * Per-a terms for a in [a0, a1) (a as a base-3 index):
 *   m[i]      = sum_b |chi_b(a)|,
 *   sgn[i]    = sum_b Re chi_b(a)          (signed: sum_u W_u = 1 check),
 *   sq[i]     = sum_b |chi_b(a)|^2         (sum_u W_u^2 = 3^-N check),
 *   maxim[i]  = max_b |Im chi_b(a)|        (chi real, R4 check).
 * Any output may be NULL.
 */
int orc_mana_terms(const double *psi_ri, int N, int64_t a0, int64_t a1, int nthreads,
                   double *m, double *sgn, double *sq, double *maxim) {
    if (N < 1 || N > 16) return -1;
    int64_t dim = ipow3(N);
    if (a0 < 0 || a1 < a0 || a1 > dim) return -1;
    const cplx *psi = as_cplx(psi_ri);
    int err = 0;
    set_threads(nthreads);
#pragma omp parallel
    {
        cplx *v = (cplx *)malloc(sizeof(cplx) * dim);
        if (!v) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t a = a0; a < a1; ++a) {
            if (!v) continue;
            /* alpha = amplitudes of X^a psi: alpha_y = psi_{y - a} */
            for (int64_t x = 0; x < dim; ++x) {
                int64_t xm = combine3(x, a, 1, -1, N);   /* x - a  */
                int64_t nxm = combine3(x, a, -1, -1, N); /* -x - a */
                v[x] = conj(psi[xm]) * psi[nxm];
            }
            ft3(v, N);
            double sm = 0.0, ss = 0.0, s2 = 0.0, mi = 0.0;
            for (int64_t b = 0; b < dim; ++b) {
                sm += cabs(v[b]);
                ss += creal(v[b]);
                s2 += creal(v[b]) * creal(v[b]) + cimag(v[b]) * cimag(v[b]);
                if (fabs(cimag(v[b])) > mi) mi = fabs(cimag(v[b]));
            }
            if (m) m[a - a0] = sm;
            if (sgn) sgn[a - a0] = ss;
            if (sq) sq[a - a0] = s2;
            if (maxim) maxim[a - a0] = mi;
        }
        free(v);
    }
    return err;
}

int orc_mana(const double *psi_ri, int N, int nthreads, double *mana_log2, double *sum_abs_w) {
    if (N < 1 || N > 16) return -1;
    int64_t dim = ipow3(N);
    double *m = (double *)malloc(sizeof(double) * dim);
    if (!m) return -2;
    int rc = orc_mana_terms(psi_ri, N, 0, dim, nthreads, m, NULL, NULL, NULL);
    if (rc == 0) {
        double s = 0.0;
        for (int64_t a = 0; a < dim; ++a) s += m[a];
        double sw = s / (double)dim; /* R3: Eq. (mana2) carries 1/3^N */
        *sum_abs_w = sw;
        *mana_log2 = log2(sw);
    }
    free(m);
    return rc;
}
