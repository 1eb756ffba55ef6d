/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for full-RNS CKKS HE Mul.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no source with the CUDA path: primes, roots,
 * tables and every modular operation are written here from their definitions.
 *
 * Arithmetic convention: residues are uint64 in [0, q); every product is formed
 * as an unsigned __int128 and reduced with a plain `%`.  There is deliberately
 * no Shoup, Barrett or Montgomery trick anywhere in this file.
 *
 * Paper: "HEAAN Demystified" (arXiv 2003.04510).  Section / algorithm cites:
 *   - encryption, decryption relation, Q and rescale: Sec. 3.1
 *   - HE Mul flow (tensor product, key switching with evk): Sec. 3.2, Fig. 2
 *   - RNS congruence relation: Sec. 3.3
 *   - NTT (Algo 3) with butterfly `butt` (Algo 4); iNTT description under Algo 4
 *   - iCRT two-phase form (Algo 5) -- the shape of the fast base conversion
 *   - full-RNS "mod up / mod down": Sec. 7 (Discussion), Table 11
 * Where the paper is silent (prime choice, root choice, digit partition,
 * floor vs round, sampling), this file follows the readings listed in the
 * header comment of each function.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------------------
 * Counters: the number of butterflies executed (Table 4 op-count pin).
 * ------------------------------------------------------------------------- */
static uint64_t g_butterflies = 0;
uint64_t or_butterfly_count(void) { return g_butterflies; }
void or_reset_butterfly_count(void) { g_butterflies = 0; }

/* ---------------------------------------------------------------------------
 * Word arithmetic mod q (q < 2^63).  Plain definitions.
 * ------------------------------------------------------------------------- */
static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + b) % q); }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + q - (b % q)) % q); }
static uint64_t powmod(uint64_t b, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}
/* q is prime, so a^(q-2) is the inverse (Fermat). */
static uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a, q - 2, q); }

/* Exported so the tests can pin the word arithmetic against Python integers. */
uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t q) { return mulmod(a, b, q); }
uint64_t or_addmod(uint64_t a, uint64_t b, uint64_t q) { return addmod(a, b, q); }
uint64_t or_submod(uint64_t a, uint64_t b, uint64_t q) { return submod(a, b, q); }
uint64_t or_powmod(uint64_t b, uint64_t e, uint64_t q) { return powmod(b, e, q); }
uint64_t or_invmod(uint64_t a, uint64_t q) { return invmod(a, q); }

/* ---------------------------------------------------------------------------
 * Primality: deterministic Miller-Rabin for n < 2^64 with the first twelve
 * primes as bases.
 * ------------------------------------------------------------------------- */
static int is_prime_u64(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}
int or_is_prime(uint64_t n) { return is_prime_u64(n); }

/* ---------------------------------------------------------------------------
 * Parameters (the paper is silent; reading c-1):
 *   the `count` largest primes below 2^bits that are 1 mod 2N, in descending
 *   order, skipping any value listed in `excl`.
 * Returns 0 on success, -1 if the range runs out.
 * ------------------------------------------------------------------------- */
int or_gen_primes(int logN, int bits, int count, const uint64_t *excl, int nexcl, uint64_t *out)
{
    uint64_t twoN = 2ull << logN;
    uint64_t top = (bits >= 64) ? ~0ull : ((1ull << bits) - 1); /* largest value < 2^bits */
    uint64_t c = ((top - 1) / twoN) * twoN + 1;                  /* largest c <= top, c = 1 mod 2N */
    int found = 0;
    while (found < count && c > twoN) {
        int skip = 0;
        for (int i = 0; i < nexcl; i++)
            if (excl[i] == c) skip = 1;
        if (!skip && is_prime_u64(c)) out[found++] = c;
        c -= twoN;
    }
    return found == count ? 0 : -1;
}

/* Smallest primitive 2N-th root of unity mod q (reading c-1).  One root g is
 * found as x^((q-1)/2N) with g^N = -1; every primitive 2N-th root is an odd
 * power of g, and the smallest of those is returned. */
uint64_t or_min_psi(uint64_t q, int logN)
{
    uint64_t N = 1ull << logN, twoN = 2 * N;
    uint64_t g = 0;
    for (uint64_t x = 2; x < q; x++) {
        g = powmod(x, (q - 1) / twoN, q);
        if (powmod(g, N, q) == q - 1) break;
    }
    uint64_t g2 = mulmod(g, g, q), cur = g, best = g;
    for (uint64_t k = 1; k < N; k++) {
        cur = mulmod(cur, g2, q);
        if (cur < best) best = cur;
    }
    return best;
}

static uint64_t bitrev(uint64_t x, int bits)
{
    uint64_t r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* ---------------------------------------------------------------------------
 * NTT -- Algo 3 with the butterfly of Algo 4.  TB_W[m + j] = psi^bitrev(m + j).
 * Algo 4 prints B = A - U and A = A + U without a reduction; both are taken
 * mod p here (the printed form is an abbreviation).  Output is the
 * bit-reversed evaluation order the algorithm produces.
 * ------------------------------------------------------------------------- */
void or_ntt(uint64_t *a, int logN, uint64_t q, uint64_t psi)
{
    uint64_t N = 1ull << logN;
    uint64_t *TBW = (uint64_t *)malloc(N * sizeof(uint64_t));
    for (uint64_t i = 0; i < N; i++) TBW[i] = powmod(psi, bitrev(i, logN), q);
    uint64_t t = N;
    for (uint64_t m = 1; m < N; m *= 2) {
        t = t / 2;
        for (uint64_t j = 0; j < m; j++) {
            uint64_t W = TBW[m + j];
            for (uint64_t k = j * 2 * t; k < j * 2 * t + t; k++) {
                /* butt(IN[k], IN[k+t], p, W) */
                uint64_t U = mulmod(a[k + t], W, q);
                a[k + t] = submod(a[k], U, q);
                a[k] = addmod(a[k], U, q);
                g_butterflies++;
            }
        }
    }
    free(TBW);
}

/* iNTT as described under Algo 4: the reversed loop order (m from N/2 down to
 * 1), the inverse butterfly A' = A + B, B' = (A - B) * W with
 * TB_invW[m + j] = psi^(-bitrev(m + j)), and finally a division by N (a
 * multiplication by N^-1 mod q). */
void or_intt(uint64_t *a, int logN, uint64_t q, uint64_t psi)
{
    uint64_t N = 1ull << logN;
    uint64_t psi_inv = invmod(psi, q);
    uint64_t *TBinvW = (uint64_t *)malloc(N * sizeof(uint64_t));
    for (uint64_t i = 0; i < N; i++) TBinvW[i] = powmod(psi_inv, bitrev(i, logN), q);
    uint64_t t = 1;
    for (uint64_t m = N / 2; m >= 1; m /= 2) {
        for (uint64_t j = 0; j < m; j++) {
            uint64_t W = TBinvW[m + j];
            for (uint64_t k = j * 2 * t; k < j * 2 * t + t; k++) {
                uint64_t A = a[k], B = a[k + t];
                a[k] = addmod(A, B, q);
                a[k + t] = mulmod(submod(A, B, q), W, q);
                g_butterflies++;
            }
        }
        t = t * 2;
    }
    uint64_t Ninv = invmod(N % q, q);
    for (uint64_t i = 0; i < N; i++) a[i] = mulmod(a[i], Ninv, q);
    free(TBinvW);
}

/* ---------------------------------------------------------------------------
 * Counter-based random words: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014;
 * Vigna's reference splitmix64.c).  Word i of the generator started at state S
 * is mix64(S + (i + 1) * gamma).  A stream (seed, id) starts at the state
 * S = mix64(seed + (id + 1) * gamma), i.e. word `id` of the generator seeded
 * with `seed`.
 * ------------------------------------------------------------------------- */
#define SM_GAMMA 0x9E3779B97F4A7C15ull
static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
uint64_t or_splitmix64(uint64_t state, uint64_t i) { return mix64(state + (i + 1) * SM_GAMMA); }

typedef struct { uint64_t state; uint64_t ctr; } rng_t;
static rng_t rng_open(uint64_t seed, uint64_t stream)
{
    rng_t r;
    r.state = mix64(seed + (stream + 1) * SM_GAMMA);
    r.ctr = 0;
    return r;
}
static uint64_t rng_next(rng_t *r) { return mix64(r->state + (++r->ctr) * SM_GAMMA); }

/* uniform in [0, t): rejection on the low bitlen(t) bits */
static uint64_t rng_below(rng_t *r, uint64_t t)
{
    uint64_t mask = 0;
    while (mask < t - 1) mask = (mask << 1) | 1;
    for (;;) {
        uint64_t v = rng_next(r) & mask;
        if (v < t) return v;
    }
}

/* rounded Gaussian, Box-Muller, rejected beyond floor(6 sigma) */
static int64_t rng_gauss(rng_t *r, double sigma)
{
    int64_t bound = (int64_t)floor(6.0 * sigma);
    for (;;) {
        uint64_t w1 = rng_next(r), w2 = rng_next(r);
        double u1 = (double)((w1 >> 11) + 1) * 0x1.0p-53; /* (0, 1] */
        double u2 = (double)(w2 >> 11) * 0x1.0p-53;       /* [0, 1) */
        double rad = sqrt(-2.0 * log(u1));
        double c = cos(6.283185307179586 * u2);
        int64_t v = llround(sigma * (rad * c));
        if (v >= -bound && v <= bound) return v;
    }
}

/* ZO(0.5): 0 with probability 1/2, +1 and -1 with 1/4 each */
static int64_t rng_zo(rng_t *r)
{
    uint64_t w = rng_next(r);
    if ((w & 1) == 0) return 0;
    return ((w >> 1) & 1) ? -1 : 1;
}

/* Stream identifiers (fixed; the product library uses the same numbers). */
enum { ST_SK = 1, ST_PK_A = 2, ST_PK_E = 3, ST_ENC_U = 4, ST_ENC_E0 = 5, ST_ENC_E1 = 6,
       ST_EVK_A = 16, ST_EVK_E = 48, ST_ROT_A = 80, ST_ROT_E = 112 };

/* Exposed samplers for the distribution tests. */
void or_sample_gauss(uint64_t seed, uint64_t stream, double sigma, int64_t n, int64_t *out)
{
    rng_t r = rng_open(seed, stream);
    for (int64_t i = 0; i < n; i++) out[i] = rng_gauss(&r, sigma);
}
void or_sample_zo(uint64_t seed, uint64_t stream, int64_t n, int64_t *out)
{
    rng_t r = rng_open(seed, stream);
    for (int64_t i = 0; i < n; i++) out[i] = rng_zo(&r);
}
void or_sample_uniform(uint64_t seed, uint64_t stream, uint64_t t, int64_t n, uint64_t *out)
{
    rng_t r = rng_open(seed, stream);
    for (int64_t i = 0; i < n; i++) out[i] = rng_below(&r, t);
}

/* signed small integer -> residue mod q */
static uint64_t to_res(int64_t v, uint64_t q)
{
    int64_t m = v % (int64_t)q;
    if (m < 0) m += (int64_t)q;
    return (uint64_t)m;
}

/* ---------------------------------------------------------------------------
 * Moduli bundle.  "ext" order puts the K special primes first, then the L
 * ciphertext primes: ext[e] = p_e for e < K, q_(e-K) otherwise.  Evaluation
 * keys are stored in this order, so level l uses ext limbs 0 .. K+l-1.
 * ------------------------------------------------------------------------- */
typedef struct {
    int logN, L, K, alpha;
    const uint64_t *q, *psi_q; /* L entries */
    const uint64_t *p, *psi_p; /* K entries */
} or_mod;

static uint64_t ext_mod(const or_mod *M, int e) { return e < M->K ? M->p[e] : M->q[e - M->K]; }
static uint64_t ext_psi(const or_mod *M, int e) { return e < M->K ? M->psi_p[e] : M->psi_q[e - M->K]; }

static or_mod mk_mod(int logN, int L, int K, int alpha, const uint64_t *q, const uint64_t *psi_q,
                     const uint64_t *p, const uint64_t *psi_p)
{
    or_mod M;
    M.logN = logN; M.L = L; M.K = K; M.alpha = alpha;
    M.q = q; M.psi_q = psi_q; M.p = p; M.psi_p = psi_p;
    return M;
}

/* Digit partition at level l (reading c-1): I_j = {j*alpha, ..., min((j+1)*alpha, l) - 1}. */
static int n_digits(int l, int alpha) { return (l + alpha - 1) / alpha; }
static int digit_lo(int j, int alpha) { return j * alpha; }
static int digit_hi(int j, int alpha, int l) { int h = (j + 1) * alpha; return h < l ? h : l; }

/* ---------------------------------------------------------------------------
 * Key generation, encryption, decryption (Sec. 3.1).
 * Layouts: sk int64[N] (coefficients in {-1,0,1}); pk uint64[2][L][N] with
 * pk0 = a*s + e (the "b" part) first and pk1 = a second, NTT domain;
 * evk uint64[dnum][2][K+L][N], b part first, ext limb order, NTT domain.
 * ------------------------------------------------------------------------- */
void or_keygen_sk(int logN, int h, uint64_t seed, int64_t *s)
{
    uint64_t N = 1ull << logN;
    uint64_t *idx = (uint64_t *)malloc(N * sizeof(uint64_t));
    for (uint64_t i = 0; i < N; i++) { idx[i] = i; s[i] = 0; }
    rng_t r = rng_open(seed, ST_SK);
    for (int k = 0; k < h; k++) { /* partial Fisher-Yates: h distinct positions */
        uint64_t pick = (uint64_t)k + rng_below(&r, N - (uint64_t)k);
        uint64_t tmp = idx[k]; idx[k] = idx[pick]; idx[pick] = tmp;
        uint64_t w = rng_next(&r);
        s[idx[k]] = (w & 1) ? -1 : 1;
    }
    free(idx);
}

/* NTT of a small signed polynomial mod q */
static void small_to_ntt(const int64_t *v, uint64_t *out, int logN, uint64_t q, uint64_t psi)
{
    uint64_t N = 1ull << logN;
    for (uint64_t i = 0; i < N; i++) out[i] = to_res(v[i], q);
    or_ntt(out, logN, q, psi);
}

void or_keygen_pk(int logN, int L, const uint64_t *q, const uint64_t *psi_q, double sigma,
                  const int64_t *s, uint64_t seed, uint64_t *pk)
{
    uint64_t N = 1ull << logN;
    rng_t ra = rng_open(seed, ST_PK_A), re = rng_open(seed, ST_PK_E);
    int64_t *e = (int64_t *)malloc(N * sizeof(int64_t));
    for (uint64_t n = 0; n < N; n++) e[n] = rng_gauss(&re, sigma);
    uint64_t *S = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *E = (uint64_t *)malloc(N * sizeof(uint64_t));
    for (int i = 0; i < L; i++) {
        uint64_t *b = pk + (size_t)i * N, *a = pk + ((size_t)L + i) * N;
        for (uint64_t n = 0; n < N; n++) a[n] = rng_below(&ra, q[i]);
        small_to_ntt(s, S, logN, q[i], psi_q[i]);
        small_to_ntt(e, E, logN, q[i], psi_q[i]);
        for (uint64_t n = 0; n < N; n++) b[n] = addmod(mulmod(a[n], S[n], q[i]), E[n], q[i]);
    }
    free(e); free(S); free(E);
}

/* evk_j encrypts P * Qtilde_j * s^2 (reading c-6), with Qtilde_j = 1 mod q_i for
 * i in I_j (at level L) and 0 mod every other q_i; it is 0 mod every p_k. */
void or_keygen_evk(int logN, int L, int K, int alpha, const uint64_t *q, const uint64_t *psi_q,
                   const uint64_t *p, const uint64_t *psi_p, double sigma, const int64_t *s,
                   uint64_t seed, uint64_t *evk)
{
    or_mod M = mk_mod(logN, L, K, alpha, q, psi_q, p, psi_p);
    uint64_t N = 1ull << logN;
    int E = K + L, dnum = n_digits(L, alpha);
    uint64_t *S = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *Ej = (uint64_t *)malloc(N * sizeof(uint64_t));
    int64_t *e = (int64_t *)malloc(N * sizeof(int64_t));
    for (int j = 0; j < dnum; j++) {
        rng_t ra = rng_open(seed, ST_EVK_A + j), re = rng_open(seed, ST_EVK_E + j);
        for (uint64_t n = 0; n < N; n++) e[n] = rng_gauss(&re, sigma);
        uint64_t *bj = evk + ((size_t)j * 2 + 0) * E * N;
        uint64_t *aj = evk + ((size_t)j * 2 + 1) * E * N;
        for (int x = 0; x < E; x++) {
            uint64_t t = ext_mod(&M, x);
            uint64_t *a = aj + (size_t)x * N, *b = bj + (size_t)x * N;
            for (uint64_t n = 0; n < N; n++) a[n] = rng_below(&ra, t);
            small_to_ntt(s, S, logN, t, ext_psi(&M, x));
            small_to_ntt(e, Ej, logN, t, ext_psi(&M, x));
            int in_digit = (x >= K) && (x - K) >= digit_lo(j, alpha) && (x - K) < digit_hi(j, alpha, L);
            uint64_t Pmod = 1;
            if (in_digit)
                for (int k = 0; k < K; k++) Pmod = mulmod(Pmod, p[k] % t, t);
            for (uint64_t n = 0; n < N; n++) {
                uint64_t v = addmod(mulmod(a[n], S[n], t), Ej[n], t);
                if (in_digit) v = addmod(v, mulmod(Pmod, mulmod(S[n], S[n], t), t), t);
                b[n] = v;
            }
        }
    }
    free(S); free(Ej); free(e);
}

/* Encryption at level l (Sec. 3.1): c.ax = u*pk1 + e1, c.bx = u*pk0 + e0 + t.
 * pt: plaintext integer coefficients.  ct: uint64[2][l][N], b first. */
void or_encrypt(int logN, int L, const uint64_t *q, const uint64_t *psi_q, double sigma,
                const uint64_t *pk, const int64_t *pt, int l, uint64_t seed, uint64_t *ct)
{
    uint64_t N = 1ull << logN;
    int64_t *u = (int64_t *)malloc(N * sizeof(int64_t));
    int64_t *e0 = (int64_t *)malloc(N * sizeof(int64_t));
    int64_t *e1 = (int64_t *)malloc(N * sizeof(int64_t));
    rng_t ru = rng_open(seed, ST_ENC_U), r0 = rng_open(seed, ST_ENC_E0), r1 = rng_open(seed, ST_ENC_E1);
    for (uint64_t n = 0; n < N; n++) u[n] = rng_zo(&ru);
    for (uint64_t n = 0; n < N; n++) e0[n] = rng_gauss(&r0, sigma);
    for (uint64_t n = 0; n < N; n++) e1[n] = rng_gauss(&r1, sigma);
    uint64_t *U = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *E0 = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *E1 = (uint64_t *)malloc(N * sizeof(uint64_t));
    for (int i = 0; i < l; i++) {
        uint64_t qi = q[i];
        small_to_ntt(u, U, logN, qi, psi_q[i]);
        for (uint64_t n = 0; n < N; n++) E0[n] = addmod(to_res(e0[n], qi), to_res(pt[n], qi), qi);
        or_ntt(E0, logN, qi, psi_q[i]);
        small_to_ntt(e1, E1, logN, qi, psi_q[i]);
        const uint64_t *pk0 = pk + (size_t)i * N, *pk1 = pk + ((size_t)L + i) * N;
        uint64_t *cb = ct + (size_t)i * N, *ca = ct + ((size_t)l + i) * N;
        for (uint64_t n = 0; n < N; n++) {
            cb[n] = addmod(mulmod(U[n], pk0[n], qi), E0[n], qi);
            ca[n] = addmod(mulmod(U[n], pk1[n], qi), E1[n], qi);
        }
    }
    free(u); free(e0); free(e1); free(U); free(E0); free(E1);
}

/* Decryption relation (Sec. 3.1): t + e' = c.bx - c.ax * sk.  Output: the
 * coefficient-form residues m[l][N] (CRT reconstruction is done by the caller
 * with big integers). */
void or_decrypt(int logN, const uint64_t *q, const uint64_t *psi_q, const int64_t *s,
                const uint64_t *ct, int l, uint64_t *m)
{
    uint64_t N = 1ull << logN;
    uint64_t *S = (uint64_t *)malloc(N * sizeof(uint64_t));
    for (int i = 0; i < l; i++) {
        small_to_ntt(s, S, logN, q[i], psi_q[i]);
        const uint64_t *cb = ct + (size_t)i * N, *ca = ct + ((size_t)l + i) * N;
        uint64_t *mi = m + (size_t)i * N;
        for (uint64_t n = 0; n < N; n++) mi[n] = submod(cb[n], mulmod(ca[n], S[n], q[i]), q[i]);
        or_intt(mi, logN, q[i], psi_q[i]);
    }
    free(S);
}

/* ---------------------------------------------------------------------------
 * c-4. Tensor product (Region 1 of Fig. 2, RNS congruence relation of Sec. 3.3):
 *   d0 = b1*b2, d1 = a1*b2 + a2*b1, d2 = a1*a2 mod q_i, element-wise, NTT domain.
 * ct layout [2][l][N] (b first); d0, d1, d2 are [l][N].
 * ------------------------------------------------------------------------- */
void or_tensor(int logN, int l, const uint64_t *q, const uint64_t *ct1, const uint64_t *ct2,
               uint64_t *d0, uint64_t *d1, uint64_t *d2)
{
    uint64_t N = 1ull << logN;
    for (int i = 0; i < l; i++) {
        uint64_t qi = q[i];
        const uint64_t *b1 = ct1 + (size_t)i * N, *a1 = ct1 + ((size_t)l + i) * N;
        const uint64_t *b2 = ct2 + (size_t)i * N, *a2 = ct2 + ((size_t)l + i) * N;
        for (uint64_t n = 0; n < N; n++) {
            size_t o = (size_t)i * N + n;
            d0[o] = mulmod(b1[n], b2[n], qi);
            d1[o] = addmod(mulmod(a1[n], b2[n], qi), mulmod(a2[n], b1[n], qi), qi);
            d2[o] = mulmod(a1[n], a2[n], qi);
        }
    }
}

/* ---------------------------------------------------------------------------
 * c-5. ModUp of digit j at level l (full-RNS "mod up", Sec. 7 / Table 11; the
 * iCRT-then-CRT shape of Algo 5 and Algo 1).  Input x: coefficient-form limbs
 * of d2, [l][N], canonical.  Output U: [K+l][N] in ext order, coefficient form:
 *   y_i = x_i * [Qhat_{j,i}^-1]_{q_i} mod q_i,   Qhat_{j,i} = prod_{i' in I_j, i' != i} q_i'
 *   U[t] = sum_{i in I_j} y_i * [Qhat_{j,i}]_t  mod t       for t outside I_j
 *   U[t] = x_t                                               for t in I_j
 * ------------------------------------------------------------------------- */
void or_modup_digit(int logN, int l, int K, int alpha, const uint64_t *q, const uint64_t *p, int j,
                    const uint64_t *x, uint64_t *U)
{
    uint64_t N = 1ull << logN;
    int lo = digit_lo(j, alpha), hi = digit_hi(j, alpha, l), E = K + l;
    or_mod M = mk_mod(logN, l, K, alpha, q, NULL, p, NULL);
    /* y_i */
    uint64_t *y = (uint64_t *)malloc((size_t)(hi - lo) * N * sizeof(uint64_t));
    for (int i = lo; i < hi; i++) {
        uint64_t qhat = 1;
        for (int i2 = lo; i2 < hi; i2++)
            if (i2 != i) qhat = mulmod(qhat, q[i2] % q[i], q[i]);
        uint64_t qhat_inv = invmod(qhat, q[i]);
        for (uint64_t n = 0; n < N; n++)
            y[(size_t)(i - lo) * N + n] = mulmod(x[(size_t)i * N + n], qhat_inv, q[i]);
    }
    for (int e = 0; e < E; e++) {
        uint64_t *out = U + (size_t)e * N;
        int ci = e - K; /* ciphertext index, if e >= K */
        if (e >= K && ci >= lo && ci < hi) {
            memcpy(out, x + (size_t)ci * N, N * sizeof(uint64_t));
            continue;
        }
        uint64_t t = ext_mod(&M, e);
        /* [Qhat_{j,i}]_t */
        uint64_t *qh = (uint64_t *)malloc((size_t)(hi - lo) * sizeof(uint64_t));
        for (int i = lo; i < hi; i++) {
            uint64_t v = 1;
            for (int i2 = lo; i2 < hi; i2++)
                if (i2 != i) v = mulmod(v, q[i2] % t, t);
            qh[i - lo] = v;
        }
        for (uint64_t n = 0; n < N; n++) {
            uint64_t acc = 0;
            for (int i = lo; i < hi; i++) acc = addmod(acc, mulmod(y[(size_t)(i - lo) * N + n] % t, qh[i - lo], t), t);
            out[n] = acc;
        }
        free(qh);
    }
    free(y);
}

/* ---------------------------------------------------------------------------
 * c-7. Inner product with evk (Region 2 of Fig. 2): for every ext limb t < K+l,
 *   KS_b[t] = sum_j U_j[t] * evk_j.b[t],  KS_a[t] = sum_j U_j[t] * evk_j.a[t]  (mod t)
 * U: [beta][K+l][N] NTT domain; evk: [dnum][2][K+L][N]; KS: [2][K+l][N].
 * ------------------------------------------------------------------------- */
void or_inner_product(int logN, int l, int L, int K, int alpha, const uint64_t *q, const uint64_t *p,
                      const uint64_t *U, const uint64_t *evk, uint64_t *KS)
{
    uint64_t N = 1ull << logN;
    int E = K + l, EL = K + L, beta = n_digits(l, alpha);
    or_mod M = mk_mod(logN, l, K, alpha, q, NULL, p, NULL);
    for (int e = 0; e < E; e++) {
        uint64_t t = ext_mod(&M, e);
        for (uint64_t n = 0; n < N; n++) {
            uint64_t sb = 0, sa = 0;
            for (int j = 0; j < beta; j++) {
                uint64_t u = U[((size_t)j * E + e) * N + n];
                uint64_t eb = evk[(((size_t)j * 2 + 0) * EL + e) * N + n];
                uint64_t ea = evk[(((size_t)j * 2 + 1) * EL + e) * N + n];
                sb = addmod(sb, mulmod(u, eb, t), t);
                sa = addmod(sa, mulmod(u, ea, t), t);
            }
            KS[((size_t)0 * E + e) * N + n] = sb;
            KS[((size_t)1 * E + e) * N + n] = sa;
        }
    }
}

/* ---------------------------------------------------------------------------
 * c-8. ModDown of one polynomial (full-RNS "mod down ... with an additional
 * division", Sec. 7).  In: X [K+l][N] NTT domain, ext order.  Out: [l][N] NTT:
 *   x_k   = iNTT(X[k]) mod p_k
 *   y_k   = x_k * [Phat_k^-1]_{p_k}
 *   conv_i = sum_k y_k * [Phat_k]_{q_i} mod q_i,  then NTT(conv_i)
 *   out_i = (X[K+i] - NTT(conv_i)) * [P^-1]_{q_i}
 * ------------------------------------------------------------------------- */
void or_moddown(int logN, int l, int K, const uint64_t *q, const uint64_t *psi_q, const uint64_t *p,
                const uint64_t *psi_p, const uint64_t *X, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    uint64_t *y = (uint64_t *)malloc((size_t)K * N * sizeof(uint64_t));
    for (int k = 0; k < K; k++) {
        uint64_t *yk = y + (size_t)k * N;
        memcpy(yk, X + (size_t)k * N, N * sizeof(uint64_t));
        or_intt(yk, logN, p[k], psi_p[k]);
        uint64_t phat = 1;
        for (int k2 = 0; k2 < K; k2++)
            if (k2 != k) phat = mulmod(phat, p[k2] % p[k], p[k]);
        uint64_t phat_inv = invmod(phat, p[k]);
        for (uint64_t n = 0; n < N; n++) yk[n] = mulmod(yk[n], phat_inv, p[k]);
    }
    uint64_t *conv = (uint64_t *)malloc(N * sizeof(uint64_t));
    for (int i = 0; i < l; i++) {
        uint64_t qi = q[i];
        uint64_t *ph = (uint64_t *)malloc((size_t)K * sizeof(uint64_t));
        uint64_t Pm = 1;
        for (int k = 0; k < K; k++) {
            uint64_t v = 1;
            for (int k2 = 0; k2 < K; k2++)
                if (k2 != k) v = mulmod(v, p[k2] % qi, qi);
            ph[k] = v;
            Pm = mulmod(Pm, p[k] % qi, qi);
        }
        uint64_t Pinv = invmod(Pm, qi);
        for (uint64_t n = 0; n < N; n++) {
            uint64_t acc = 0;
            for (int k = 0; k < K; k++) acc = addmod(acc, mulmod(y[(size_t)k * N + n] % qi, ph[k], qi), qi);
            conv[n] = acc;
        }
        or_ntt(conv, logN, qi, psi_q[i]);
        const uint64_t *Xi = X + ((size_t)K + i) * N;
        for (uint64_t n = 0; n < N; n++) out[(size_t)i * N + n] = mulmod(submod(Xi[n], conv[n], qi), Pinv, qi);
        free(ph);
    }
    free(conv);
    free(y);
}

/* ---------------------------------------------------------------------------
 * Key switching of d2 at level l: c-5 (ModUp), NTT of every limb, c-7 (inner
 * product), c-8 (ModDown of both halves).  d2: [l][N] NTT domain.
 * Out ks: [2][l][N] NTT domain.  Optional intermediates: U_out [beta][K+l][N]
 * (NTT domain) and KS_out [2][K+l][N] if non-NULL.
 * ------------------------------------------------------------------------- */
void or_keyswitch(int logN, int l, int L, int K, int alpha, const uint64_t *q, const uint64_t *psi_q,
                  const uint64_t *p, const uint64_t *psi_p, const uint64_t *d2, const uint64_t *evk,
                  uint64_t *ks, uint64_t *U_out, uint64_t *KS_out)
{
    uint64_t N = 1ull << logN;
    int E = K + l, beta = n_digits(l, alpha);
    or_mod M = mk_mod(logN, l, K, alpha, q, psi_q, p, psi_p);
    uint64_t *x = (uint64_t *)malloc((size_t)l * N * sizeof(uint64_t));
    memcpy(x, d2, (size_t)l * N * sizeof(uint64_t));
    for (int i = 0; i < l; i++) or_intt(x + (size_t)i * N, logN, q[i], psi_q[i]);
    uint64_t *U = U_out ? U_out : (uint64_t *)malloc((size_t)beta * E * N * sizeof(uint64_t));
    for (int j = 0; j < beta; j++) {
        uint64_t *Uj = U + (size_t)j * E * N;
        or_modup_digit(logN, l, K, alpha, q, p, j, x, Uj);
        for (int e = 0; e < E; e++) or_ntt(Uj + (size_t)e * N, logN, ext_mod(&M, e), ext_psi(&M, e));
    }
    uint64_t *KS = KS_out ? KS_out : (uint64_t *)malloc((size_t)2 * E * N * sizeof(uint64_t));
    or_inner_product(logN, l, L, K, alpha, q, p, U, evk, KS);
    or_moddown(logN, l, K, q, psi_q, p, psi_p, KS, ks);
    or_moddown(logN, l, K, q, psi_q, p, psi_p, KS + (size_t)E * N, ks + (size_t)l * N);
    if (!U_out) free(U);
    if (!KS_out) free(KS);
    free(x);
}

/* ---------------------------------------------------------------------------
 * HE Mul at level l (Fig. 2, RNS form): tensor product, key switching of d2,
 * then the additions c3.b = d0 + ModDown(KS_b), c3.a = d1 + ModDown(KS_a).
 * ct1, ct2, out: [2][l][N].  L is the level the evk was generated at.
 * ------------------------------------------------------------------------- */
void or_he_mul(int logN, int l, int L, int K, int alpha, const uint64_t *q, const uint64_t *psi_q,
               const uint64_t *p, const uint64_t *psi_p, const uint64_t *ct1, const uint64_t *ct2,
               const uint64_t *evk, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    size_t LN = (size_t)l * N;
    uint64_t *d0 = (uint64_t *)malloc(LN * sizeof(uint64_t));
    uint64_t *d1 = (uint64_t *)malloc(LN * sizeof(uint64_t));
    uint64_t *d2 = (uint64_t *)malloc(LN * sizeof(uint64_t));
    uint64_t *ks = (uint64_t *)malloc(2 * LN * sizeof(uint64_t));
    or_tensor(logN, l, q, ct1, ct2, d0, d1, d2);
    or_keyswitch(logN, l, L, K, alpha, q, psi_q, p, psi_p, d2, evk, ks, NULL, NULL);
    for (int i = 0; i < l; i++)
        for (uint64_t n = 0; n < N; n++) {
            size_t o = (size_t)i * N + n;
            out[o] = addmod(d0[o], ks[o], q[i]);
            out[LN + o] = addmod(d1[o], ks[LN + o], q[i]);
        }
    free(d0); free(d1); free(d2); free(ks);
}

/* ---------------------------------------------------------------------------
 * c-9. Rescale (Sec. 3.1, "divide by p"): ct at level l -> level l-1.
 *   r     = iNTT(c_{l-1}) in [0, q_{l-1})
 *   r_i   = r mod q_i  (no centring: the result is the exact floor)
 *   out_i = (c_i - NTT_i(r_i)) * [q_{l-1}^-1]_{q_i}
 * ------------------------------------------------------------------------- */
void or_rescale(int logN, int l, const uint64_t *q, const uint64_t *psi_q, const uint64_t *ct, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    uint64_t ql = q[l - 1];
    uint64_t *r = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *ri = (uint64_t *)malloc(N * sizeof(uint64_t));
    for (int h = 0; h < 2; h++) {
        const uint64_t *c = ct + (size_t)h * l * N;
        uint64_t *o = out + (size_t)h * (l - 1) * N;
        memcpy(r, c + (size_t)(l - 1) * N, N * sizeof(uint64_t));
        or_intt(r, logN, ql, psi_q[l - 1]);
        for (int i = 0; i < l - 1; i++) {
            uint64_t qi = q[i];
            uint64_t qinv = invmod(ql % qi, qi);
            for (uint64_t n = 0; n < N; n++) ri[n] = r[n] % qi;
            or_ntt(ri, logN, qi, psi_q[i]);
            for (uint64_t n = 0; n < N; n++)
                o[(size_t)i * N + n] = mulmod(submod(c[(size_t)i * N + n], ri[n], qi), qinv, qi);
        }
    }
    free(r); free(ri);
}

/* ---------------------------------------------------------------------------
 * HE Mul followed by one division by M = P * q_{l-1}: ModDown and rescale
 * folded into a single fast base conversion (the single-division variant of
 * the key-switch tail; not in the paper, built on Fig. 2's flow and the
 * full-RNS "mod down ... with an additional division" of Sec. 7).
 * For each half h (b, a), over the basis Q_l and P, in the NTT domain:
 *   Y_h[p_k] = KS_h[p_k],   Y_h[q_i] = P d_h[i] + KS_h[q_i]  (mod q_i)
 * (the tensor products d0, d1 lifted by P, plus the inner product).  The
 * basis B = (p_0, ..., p_{K-1}, q_{l-1}) with product M is dropped by:
 *   x_j    = iNTT(Y_h[b_j]) in [0, b_j)
 *   y_j    = x_j [Mhat_j^-1]_{b_j},   Mhat_j = M / b_j
 *   conv_i = sum_j y_j [Mhat_j]_{q_i} mod q_i   (i < l-1), NTT(conv_i)
 *   out_i  = (Y_h[q_i] - NTT(conv_i)) [M^-1]_{q_i}
 * In coefficient form out = floor(Y / M) - floor(sum_j y_j / b_j) mod Q_{l-1},
 * Y the CRT value of Y_h over P Q_l (one floor, where HE Mul followed by a
 * rescale takes two).  ct1, ct2: [2][l][N]; out: [2][l-1][N]; 2 <= l.
 * ------------------------------------------------------------------------- */
void or_he_mul_rescale_pq(int logN, int l, int L, int K, int alpha, const uint64_t *q, const uint64_t *psi_q,
                          const uint64_t *p, const uint64_t *psi_p, const uint64_t *ct1, const uint64_t *ct2,
                          const uint64_t *evk, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    size_t LN = (size_t)l * N;
    int E = K + l, nb = K + 1;
    uint64_t *d = (uint64_t *)malloc(3 * LN * sizeof(uint64_t));
    uint64_t *ks = (uint64_t *)malloc(2 * LN * sizeof(uint64_t));
    uint64_t *KS = (uint64_t *)malloc((size_t)2 * E * N * sizeof(uint64_t));
    uint64_t *Y = (uint64_t *)malloc((size_t)E * N * sizeof(uint64_t));
    uint64_t *y = (uint64_t *)malloc((size_t)nb * N * sizeof(uint64_t));
    uint64_t *conv = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *b = (uint64_t *)malloc((size_t)nb * sizeof(uint64_t));
    uint64_t *bpsi = (uint64_t *)malloc((size_t)nb * sizeof(uint64_t));
    or_tensor(logN, l, q, ct1, ct2, d, d + LN, d + 2 * LN);
    or_keyswitch(logN, l, L, K, alpha, q, psi_q, p, psi_p, d + 2 * LN, evk, ks, NULL, KS);
    for (int k = 0; k < K; k++) { b[k] = p[k]; bpsi[k] = psi_p[k]; }
    b[K] = q[l - 1];
    bpsi[K] = psi_q[l - 1];
    for (int h = 0; h < 2; h++) {
        const uint64_t *dh = d + (size_t)h * LN, *KSh = KS + (size_t)h * E * N;
        /* Y_h = P d_h + KS_h */
        for (int k = 0; k < K; k++) memcpy(Y + (size_t)k * N, KSh + (size_t)k * N, N * sizeof(uint64_t));
        for (int i = 0; i < l; i++) {
            uint64_t Pm = 1;
            for (int k = 0; k < K; k++) Pm = mulmod(Pm, p[k] % q[i], q[i]);
            for (uint64_t n = 0; n < N; n++)
                Y[((size_t)K + i) * N + n] =
                    addmod(mulmod(Pm, dh[(size_t)i * N + n], q[i]), KSh[((size_t)K + i) * N + n], q[i]);
        }
        /* x_j, y_j over the dropped basis B */
        for (int j = 0; j < nb; j++) {
            uint64_t *yj = y + (size_t)j * N;
            size_t row = j < K ? (size_t)j : (size_t)K + l - 1;
            memcpy(yj, Y + row * N, N * sizeof(uint64_t));
            or_intt(yj, logN, b[j], bpsi[j]);
            uint64_t mhat = 1;
            for (int j2 = 0; j2 < nb; j2++)
                if (j2 != j) mhat = mulmod(mhat, b[j2] % b[j], b[j]);
            uint64_t mhat_inv = invmod(mhat, b[j]);
            for (uint64_t n = 0; n < N; n++) yj[n] = mulmod(yj[n], mhat_inv, b[j]);
        }
        for (int i = 0; i < l - 1; i++) {
            uint64_t qi = q[i], Mm = 1;
            uint64_t *mh = (uint64_t *)malloc((size_t)nb * sizeof(uint64_t));
            for (int j = 0; j < nb; j++) {
                uint64_t v = 1;
                for (int j2 = 0; j2 < nb; j2++)
                    if (j2 != j) v = mulmod(v, b[j2] % qi, qi);
                mh[j] = v;
                Mm = mulmod(Mm, b[j] % qi, qi);
            }
            uint64_t Minv = invmod(Mm, qi);
            for (uint64_t n = 0; n < N; n++) {
                uint64_t acc = 0;
                for (int j = 0; j < nb; j++) acc = addmod(acc, mulmod(y[(size_t)j * N + n] % qi, mh[j], qi), qi);
                conv[n] = acc;
            }
            or_ntt(conv, logN, qi, psi_q[i]);
            uint64_t *o = out + ((size_t)h * (l - 1) + i) * N;
            for (uint64_t n = 0; n < N; n++)
                o[n] = mulmod(submod(Y[((size_t)K + i) * N + n], conv[n], qi), Minv, qi);
            free(mh);
        }
    }
    free(d); free(ks); free(KS); free(Y); free(y); free(conv); free(b); free(bpsi);
}

/* ---------------------------------------------------------------------------
 * Galois automorphism kappa_g : a(X) -> a(X^g) on Z_q[X]/(X^N + 1), g odd in
 * [1, 2N).  Written from the definition: coefficient i goes to exponent
 * i*g mod 2N, and an exponent e >= N is X^(e-N) * X^N = -X^(e-N).  (Rotation
 * is not in the paper; it is the next operation built on the paper's key
 * switching, Fig. 2.)  a, out: [N] coefficient form, out != a.
 * ------------------------------------------------------------------------- */
void or_automorphism(const uint64_t *a, int logN, uint64_t q, uint64_t g, uint64_t *out)
{
    uint64_t N = 1ull << logN, twoN = 2 * N;
    for (uint64_t i = 0; i < N; i++) {
        uint64_t e = (uint64_t)(((u128)i * (g % twoN)) % twoN);
        if (e < N) out[e] = a[i] % q;
        else out[e - N] = submod(0, a[i], q);
    }
}

/* The same on a small signed polynomial (the secret key). */
static void small_automorphism(const int64_t *a, int logN, uint64_t g, int64_t *out)
{
    uint64_t N = 1ull << logN, twoN = 2 * N;
    for (uint64_t i = 0; i < N; i++) {
        uint64_t e = (uint64_t)(((u128)i * (g % twoN)) % twoN);
        if (e < N) out[e] = a[i];
        else out[e - N] = -a[i];
    }
}

/* ---------------------------------------------------------------------------
 * Key-switching key from kappa_g(s) to s (a "rotation key"): the evk of
 * or_keygen_evk with kappa_g(s) in place of s^2,
 *   b_j[t] = a_j[t] s + e_j + [t = q_i, i in I_j] (P mod q_i) kappa_g(s)  mod t,
 * a_j uniform (stream ST_ROT_A + j), e_j Gaussian (stream ST_ROT_E + j).
 * Layout as evk: [dnum][2][K+L][N], b first, ext order, NTT domain.
 * ------------------------------------------------------------------------- */
void or_keygen_rot(int logN, int L, int K, int alpha, const uint64_t *q, const uint64_t *psi_q,
                   const uint64_t *p, const uint64_t *psi_p, double sigma, const int64_t *s, uint64_t g,
                   uint64_t seed, uint64_t *rk)
{
    or_mod M = mk_mod(logN, L, K, alpha, q, psi_q, p, psi_p);
    uint64_t N = 1ull << logN;
    int E = K + L, dnum = n_digits(L, alpha);
    int64_t *ks = (int64_t *)malloc(N * sizeof(int64_t));
    small_automorphism(s, logN, g, ks);
    uint64_t *S = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *KSn = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *Ej = (uint64_t *)malloc(N * sizeof(uint64_t));
    int64_t *e = (int64_t *)malloc(N * sizeof(int64_t));
    for (int j = 0; j < dnum; j++) {
        rng_t ra = rng_open(seed, ST_ROT_A + j), re = rng_open(seed, ST_ROT_E + j);
        for (uint64_t n = 0; n < N; n++) e[n] = rng_gauss(&re, sigma);
        uint64_t *bj = rk + ((size_t)j * 2 + 0) * E * N;
        uint64_t *aj = rk + ((size_t)j * 2 + 1) * E * N;
        for (int x = 0; x < E; x++) {
            uint64_t t = ext_mod(&M, x);
            uint64_t *a = aj + (size_t)x * N, *b = bj + (size_t)x * N;
            for (uint64_t n = 0; n < N; n++) a[n] = rng_below(&ra, t);
            small_to_ntt(s, S, logN, t, ext_psi(&M, x));
            small_to_ntt(ks, KSn, logN, t, ext_psi(&M, x));
            small_to_ntt(e, Ej, logN, t, ext_psi(&M, x));
            int in_digit = (x >= K) && (x - K) >= digit_lo(j, alpha) && (x - K) < digit_hi(j, alpha, L);
            uint64_t Pmod = 1;
            if (in_digit)
                for (int k = 0; k < K; k++) Pmod = mulmod(Pmod, p[k] % t, t);
            for (uint64_t n = 0; n < N; n++) {
                uint64_t v = addmod(mulmod(a[n], S[n], t), Ej[n], t);
                if (in_digit) v = addmod(v, mulmod(Pmod, KSn[n], t), t);
                b[n] = v;
            }
        }
    }
    free(ks); free(S); free(KSn); free(Ej); free(e);
}

/* ---------------------------------------------------------------------------
 * HE rotation by the automorphism kappa_g at level l.  (kappa(b), kappa(a))
 * decrypts under kappa(s): kappa(b) - kappa(a) kappa(s) = kappa(m).  Key
 * switching x = -kappa(a) with the key for kappa(s) (Fig. 2's region 2 flow:
 * ModUp, NTT, inner product, ModDown) gives
 *   out = (kappa(b) + ModDown(KS_b), ModDown(KS_a)),
 * which decrypts to kappa(b) - kappa(a) kappa(s) + small.  kappa is applied
 * in coefficient form (iNTT, definition, NTT).  ct, out: [2][l][N].
 * ------------------------------------------------------------------------- */
void or_rotate(int logN, int l, int L, int K, int alpha, const uint64_t *q, const uint64_t *psi_q,
               const uint64_t *p, const uint64_t *psi_p, const uint64_t *ct, uint64_t g, const uint64_t *rk,
               uint64_t *out)
{
    uint64_t N = 1ull << logN;
    size_t LN = (size_t)l * N;
    uint64_t *kc = (uint64_t *)malloc(2 * LN * sizeof(uint64_t));
    uint64_t *tmp = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *ks = (uint64_t *)malloc(2 * LN * sizeof(uint64_t));
    for (int h = 0; h < 2; h++)
        for (int i = 0; i < l; i++) {
            const uint64_t *src = ct + (size_t)h * LN + (size_t)i * N;
            uint64_t *dst = kc + (size_t)h * LN + (size_t)i * N;
            memcpy(tmp, src, N * sizeof(uint64_t));
            or_intt(tmp, logN, q[i], psi_q[i]);
            or_automorphism(tmp, logN, q[i], g, dst);
            or_ntt(dst, logN, q[i], psi_q[i]);
        }
    uint64_t *x = kc + LN;  /* x = -kappa(a), in place */
    for (int i = 0; i < l; i++)
        for (uint64_t n = 0; n < N; n++) x[(size_t)i * N + n] = submod(0, x[(size_t)i * N + n], q[i]);
    or_keyswitch(logN, l, L, K, alpha, q, psi_q, p, psi_p, x, rk, ks, NULL, NULL);
    for (int i = 0; i < l; i++)
        for (uint64_t n = 0; n < N; n++) {
            size_t o = (size_t)i * N + n;
            out[o] = addmod(kc[o], ks[o], q[i]);
            out[LN + o] = ks[LN + o];
        }
    free(kc); free(tmp); free(ks);
}

/* ---------------------------------------------------------------------------
 * HE Add (Sec. 3.2, "HEAAN computation"): c3.ax = mod(c1.ax + c2.ax, q),
 * c3.bx = mod(c1.bx + c2.bx, q), element-wise per limb.  The difference is
 * the same with a subtraction.  ct1, ct2, out: [2][l][N].
 * ------------------------------------------------------------------------- */
void or_add(int logN, int l, const uint64_t *q, const uint64_t *ct1, const uint64_t *ct2, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    for (int h = 0; h < 2; h++)
        for (int i = 0; i < l; i++)
            for (uint64_t n = 0; n < N; n++) {
                size_t o = ((size_t)h * l + i) * N + n;
                out[o] = addmod(ct1[o], ct2[o], q[i]);
            }
}

void or_sub(int logN, int l, const uint64_t *q, const uint64_t *ct1, const uint64_t *ct2, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    for (int h = 0; h < 2; h++)
        for (int i = 0; i < l; i++)
            for (uint64_t n = 0; n < N; n++) {
                size_t o = ((size_t)h * l + i) * N + n;
                out[o] = submod(ct1[o], ct2[o], q[i]);
            }
}

/* ---------------------------------------------------------------------------
 * Plaintext operations.  A plaintext at level l is the integer polynomial of
 * the encoder (Sec. 3.1) reduced mod each q_i and transformed by Algo 3:
 * pt [l][N] NTT domain.  Multiplying a ciphertext by it multiplies both
 * halves (b - a s becomes (b - a s) pt, so the message is multiplied and the
 * scale is the product of the scales); adding it adds to the b half only.
 * ------------------------------------------------------------------------- */
void or_plain_ntt(int logN, int l, const uint64_t *q, const uint64_t *psi_q, const int64_t *coeffs, uint64_t *pt)
{
    uint64_t N = 1ull << logN;
    for (int i = 0; i < l; i++) {
        uint64_t *o = pt + (size_t)i * N;
        for (uint64_t n = 0; n < N; n++) {
            int64_t c = coeffs[n];
            o[n] = c >= 0 ? (uint64_t)c % q[i] : submod(0, (uint64_t)(-(c + 1)) + 1, q[i]);
        }
        or_ntt(o, logN, q[i], psi_q[i]);
    }
}

void or_mul_plain(int logN, int l, const uint64_t *q, const uint64_t *ct, const uint64_t *pt, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    for (int h = 0; h < 2; h++)
        for (int i = 0; i < l; i++)
            for (uint64_t n = 0; n < N; n++) {
                size_t o = ((size_t)h * l + i) * N + n;
                out[o] = mulmod(ct[o], pt[(size_t)i * N + n], q[i]);
            }
}

void or_add_plain(int logN, int l, const uint64_t *q, const uint64_t *ct, const uint64_t *pt, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    for (int i = 0; i < l; i++)
        for (uint64_t n = 0; n < N; n++) {
            size_t o = (size_t)i * N + n;
            out[o] = addmod(ct[o], pt[o], q[i]);
            out[(size_t)l * N + o] = ct[(size_t)l * N + o];
        }
}

/* ---------------------------------------------------------------------------
 * Seeded evaluation key (NEXT-3: halve the key's bytes).  The a halves come
 * from a counter-based sampler that can be evaluated for any single element:
 *   S_j            = mix64(seed + (ST_SEED_A + j + 1) gamma)   (stream state)
 *   w1, w2         = words 2*idx and 2*idx + 1 of that stream, idx = e*N + n
 *   a_j[e][n]      = floor((w1 * 2^64 + w2) * t / 2^128),  t = the e-th modulus
 * (uniform up to a bias below t / 2^128; no rejection loop).  The b halves
 * are those of or_keygen_evk with these a's:
 *   b_j = a_j s + e_j + [t in digit j] P s^2, e_j from stream ST_EVK_E + j.
 * Layout as evk: [dnum][2][K+L][N]; a device stores only the b halves.
 * ------------------------------------------------------------------------- */
enum { ST_SEED_A = 144 };

uint64_t or_seeded_a(uint64_t seed, int j, uint64_t idx, uint64_t t)
{
    uint64_t S = mix64(seed + ((uint64_t)(ST_SEED_A + j) + 1) * SM_GAMMA);
    uint64_t w1 = mix64(S + (2 * idx + 1) * SM_GAMMA), w2 = mix64(S + (2 * idx + 2) * SM_GAMMA);
    u128 hi = (u128)w1 * t, lo = (u128)w2 * t;
    return (uint64_t)((hi + (lo >> 64)) >> 64);
}

void or_keygen_evk_seeded(int logN, int L, int K, int alpha, const uint64_t *q, const uint64_t *psi_q,
                          const uint64_t *p, const uint64_t *psi_p, double sigma, const int64_t *s,
                          uint64_t seed, uint64_t *evk)
{
    or_mod M = mk_mod(logN, L, K, alpha, q, psi_q, p, psi_p);
    uint64_t N = 1ull << logN;
    int E = K + L, dnum = n_digits(L, alpha);
    uint64_t *S = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *Ej = (uint64_t *)malloc(N * sizeof(uint64_t));
    int64_t *e = (int64_t *)malloc(N * sizeof(int64_t));
    for (int j = 0; j < dnum; j++) {
        rng_t re = rng_open(seed, ST_EVK_E + j);
        for (uint64_t n = 0; n < N; n++) e[n] = rng_gauss(&re, sigma);
        uint64_t *bj = evk + ((size_t)j * 2 + 0) * E * N;
        uint64_t *aj = evk + ((size_t)j * 2 + 1) * E * N;
        for (int x = 0; x < E; x++) {
            uint64_t t = ext_mod(&M, x);
            uint64_t *a = aj + (size_t)x * N, *b = bj + (size_t)x * N;
            for (uint64_t n = 0; n < N; n++) a[n] = or_seeded_a(seed, j, (uint64_t)x * N + n, t);
            small_to_ntt(s, S, logN, t, ext_psi(&M, x));
            small_to_ntt(e, Ej, logN, t, ext_psi(&M, x));
            int in_digit = (x >= K) && (x - K) >= digit_lo(j, alpha) && (x - K) < digit_hi(j, alpha, L);
            uint64_t Pmod = 1;
            if (in_digit)
                for (int k = 0; k < K; k++) Pmod = mulmod(Pmod, p[k] % t, t);
            for (uint64_t n = 0; n < N; n++) {
                uint64_t v = addmod(mulmod(a[n], S[n], t), Ej[n], t);
                if (in_digit) v = addmod(v, mulmod(Pmod, mulmod(S[n], S[n], t), t), t);
                b[n] = v;
            }
        }
    }
    free(S); free(Ej); free(e);
}

/* ===========================================================================
 * NEXT-2: the paper's own (non-RNS) HEAAN HE Mul.
 *
 * Ciphertext and key coefficients are BigInts modulo powers of two (Sec. 3,
 * Table 3: q = 2^logq, Q = 2^logQ, p = 2^logp), stored word-major: word w of
 * coefficient n at a[w * N + n], W = ceil(k / 64) words for a k-bit modulus,
 * little-endian, the top word holding k - 64 (W - 1) bits.  A polynomial
 * product goes through the paper's five steps (Fig. 2, Sec. 4): CRT (BigInt
 * -> residues mod np primes p_i, P = prod p_i), NTT, element-wise products,
 * iNTT, iCRT (residues -> BigInt).  The iCRT here is exact: X = sum_i
 * [x_i Phat_i^-1]_{p_i} Phat_i as a multiword integer, reduced mod P by
 * subtraction, taken as the centred representative (P exceeds four times the
 * product's magnitude) and truncated to the output modulus.
 * ======================================================================== */
#define MW_MAX 96 /* words of a multiword integer in the iCRT */

static int nwords(int k) { return (k + 63) / 64; }

/* X mod p for the word-major coefficient n of a (w words) */
static uint64_t mw_mod(const uint64_t *a, int w, uint64_t N, uint64_t n, uint64_t p)
{
    u128 r = 0;
    for (int i = w - 1; i >= 0; i--) r = ((r << 64) | a[(size_t)i * N + n]) % p;
    return (uint64_t)r;
}

/* acc (len words) += v * b (nb words) */
static void mw_mac(uint64_t *acc, int len, uint64_t v, const uint64_t *b, int nb)
{
    u128 carry = 0;
    for (int i = 0; i < len; i++) {
        u128 t = (u128)acc[i] + carry + (i < nb ? (u128)v * b[i] : 0);
        acc[i] = (uint64_t)t;
        carry = t >> 64;
    }
}
static int mw_cmp(const uint64_t *a, const uint64_t *b, int len)
{
    for (int i = len - 1; i >= 0; i--)
        if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
    return 0;
}
static void mw_sub(uint64_t *a, const uint64_t *b, int len) /* a -= b (mod 2^(64 len)) */
{
    uint64_t borrow = 0;
    for (int i = 0; i < len; i++) {
        u128 t = (u128)a[i] - b[i] - borrow;
        a[i] = (uint64_t)t;
        borrow = (uint64_t)(t >> 64) ? 1 : 0;
    }
}
static void mw_shr1(uint64_t *a, int len)
{
    for (int i = 0; i < len; i++) a[i] = (a[i] >> 1) | (i + 1 < len ? a[i + 1] << 63 : 0);
}

/* The CRT tables of np primes: Phat_i (multiword), [Phat_i^-1]_{p_i}, P, P/2. */
typedef struct {
    int np, len;
    uint64_t p[MW_MAX], psi[MW_MAX], phinv[MW_MAX];
    uint64_t Phat[MW_MAX][MW_MAX], P[MW_MAX], Phalf[MW_MAX];
} crt_t;

static void crt_init(crt_t *T, int np, const uint64_t *p, const uint64_t *psi)
{
    memset(T, 0, sizeof(*T));
    T->np = np;
    T->len = np + 2;
    for (int i = 0; i < np; i++) {
        T->p[i] = p[i];
        T->psi[i] = psi[i];
    }
    T->P[0] = 1;
    for (int i = 0; i < np; i++) {
        uint64_t t[MW_MAX] = {0};
        mw_mac(t, T->len, p[i], T->P, T->len);
        memcpy(T->P, t, sizeof(t));
    }
    for (int i = 0; i < np; i++) {
        T->Phat[i][0] = 1;
        for (int j = 0; j < np; j++)
            if (j != i) {
                uint64_t t[MW_MAX] = {0};
                mw_mac(t, T->len, p[j], T->Phat[i], T->len);
                memcpy(T->Phat[i], t, sizeof(t));
            }
        uint64_t r = 0; /* Phat_i mod p_i */
        for (int w = T->len - 1; w >= 0; w--) r = (uint64_t)((((u128)r << 64) | T->Phat[i][w]) % p[i]);
        T->phinv[i] = invmod(r, p[i]);
    }
    memcpy(T->Phalf, T->P, sizeof(T->P));
    mw_shr1(T->Phalf, T->len);
}

/* C = A * B mod (X^N + 1, 2^kout).  A: wa words per coefficient (unsigned);
 * B: wb words (unsigned), or, when bs != NULL, the small signed polynomial bs.
 * The primes must satisfy P > 4 N max|A| max|B|. */
static void nr_polymul(int logN, const crt_t *T, const uint64_t *A, int wa, const uint64_t *B, int wb,
                       const int64_t *bs, int kout, uint64_t *C)
{
    uint64_t N = 1ull << logN;
    int np = T->np, wo = nwords(kout);
    uint64_t *ra = (uint64_t *)malloc(N * sizeof(uint64_t)), *rb = (uint64_t *)malloc(N * sizeof(uint64_t));
    uint64_t *Y = (uint64_t *)malloc((size_t)np * N * sizeof(uint64_t));
    for (int i = 0; i < np; i++) {
        uint64_t p = T->p[i];
        for (uint64_t n = 0; n < N; n++) {
            ra[n] = mw_mod(A, wa, N, n, p);
            rb[n] = bs ? (bs[n] >= 0 ? (uint64_t)bs[n] % p : submod(0, (uint64_t)(-bs[n]), p)) : mw_mod(B, wb, N, n, p);
        }
        or_ntt(ra, logN, p, T->psi[i]);
        or_ntt(rb, logN, p, T->psi[i]);
        for (uint64_t n = 0; n < N; n++) ra[n] = mulmod(ra[n], rb[n], p);
        or_intt(ra, logN, p, T->psi[i]);
        for (uint64_t n = 0; n < N; n++) Y[(size_t)i * N + n] = mulmod(ra[n], T->phinv[i], p);
    }
    for (uint64_t n = 0; n < N; n++) {
        uint64_t X[MW_MAX] = {0};
        for (int i = 0; i < np; i++) mw_mac(X, T->len, Y[(size_t)i * N + n], T->Phat[i], T->len);
        while (mw_cmp(X, T->P, T->len) >= 0) mw_sub(X, T->P, T->len);
        if (mw_cmp(X, T->Phalf, T->len) > 0) mw_sub(X, T->P, T->len); /* negative: two's complement */
        for (int w = 0; w < wo; w++) {
            uint64_t v = w < T->len ? X[w] : (X[T->len - 1] >> 63 ? ~0ull : 0);
            if (w == wo - 1 && (kout & 63)) v &= (1ull << (kout & 63)) - 1;
            C[(size_t)w * N + n] = v;
        }
    }
    free(ra); free(rb); free(Y);
}

/* out = (a + b) mod 2^k and out = (a - b) mod 2^k, word-major, w = nwords(k) */
static void nr_addsub(uint64_t N, int k, const uint64_t *a, const uint64_t *b, int sub, uint64_t *out)
{
    int w = nwords(k);
    for (uint64_t n = 0; n < N; n++) {
        uint64_t c = 0;
        for (int i = 0; i < w; i++) {
            size_t o = (size_t)i * N + n;
            u128 t = sub ? (u128)a[o] - b[o] - c : (u128)a[o] + b[o] + c;
            out[o] = (uint64_t)t;
            c = sub ? ((uint64_t)(t >> 64) ? 1 : 0) : (uint64_t)(t >> 64);
        }
        if (k & 63) out[(size_t)(w - 1) * N + n] &= (1ull << (k & 63)) - 1;
    }
}

/* out = floor((a + 2^(s-1)) / 2^s) mod 2^kout: the division by a power of
 * two with rounding (rescale by p = 2^logp, and the key switch's division by
 * Q = 2^logQ).  a: nwords(kin) words. */
static void nr_shift_round(uint64_t N, const uint64_t *a, int kin, int s, int kout, uint64_t *out)
{
    int wi = nwords(kin), wo = nwords(kout);
    uint64_t t[MW_MAX + 1];
    for (uint64_t n = 0; n < N; n++) {
        memset(t, 0, sizeof(t));
        for (int i = 0; i < wi; i++) t[i] = a[(size_t)i * N + n];
        uint64_t half[MW_MAX + 1] = {0};
        half[(s - 1) / 64] = 1ull << ((s - 1) & 63);
        uint64_t c = 0;
        for (int i = 0; i <= wi; i++) {
            u128 v = (u128)t[i] + half[i] + c;
            t[i] = (uint64_t)v;
            c = (uint64_t)(v >> 64);
        }
        for (int w = 0; w < wo; w++) {
            int bit = s + 64 * w, q = bit / 64, r = bit & 63;
            uint64_t v = (q <= wi ? t[q] >> r : 0);
            if (r && q + 1 <= wi) v |= t[q + 1] << (64 - r);
            if (w == wo - 1 && (kout & 63)) v &= (1ull << (kout & 63)) - 1;
            out[(size_t)w * N + n] = v;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Non-RNS HE Mul at logq (Fig. 2): region 1 multiplies the ciphertexts mod q,
 * d0 = b1 b2, d1 = a1 b2 + a2 b1, d2 = a1 a2; region 2 multiplies d2 by the
 * evaluation key (coefficients mod Q^2, encrypting Q s^2) mod qQ and divides
 * by Q with rounding; c3 = (d0 + ks_b, d1 + ks_a) mod q.  Decryption relation
 * of Sec. 3.1: b - a s = m + e.  ct: [2][W_q][N] word-major, b half first;
 * evk: [2][W_{2 logQ}][N].  np1 primes for region 1, np2 for region 2.
 * ------------------------------------------------------------------------- */
void or_nr_he_mul(int logN, int logq, int logQ, int np1, int np2, const uint64_t *primes, const uint64_t *psis,
                  const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    int wq = nwords(logq), wqQ = nwords(logq + logQ), wQQ = nwords(2 * logQ);
    size_t PQ = (size_t)wq * N, PQQ = (size_t)wqQ * N;
    crt_t *T1 = (crt_t *)malloc(sizeof(crt_t)), *T2 = (crt_t *)malloc(sizeof(crt_t));
    crt_init(T1, np1, primes, psis);
    crt_init(T2, np2, primes, psis);
    const uint64_t *b1 = ct1, *a1 = ct1 + PQ, *b2 = ct2, *a2 = ct2 + PQ;
    uint64_t *d0 = (uint64_t *)malloc(PQ * 8), *d1 = (uint64_t *)malloc(PQ * 8), *d2 = (uint64_t *)malloc(PQ * 8);
    uint64_t *t = (uint64_t *)malloc(PQ * 8);
    nr_polymul(logN, T1, b1, wq, b2, wq, NULL, logq, d0);
    nr_polymul(logN, T1, a1, wq, b2, wq, NULL, logq, d1);
    nr_polymul(logN, T1, a2, wq, b1, wq, NULL, logq, t);
    nr_addsub(N, logq, d1, t, 0, d1);
    nr_polymul(logN, T1, a1, wq, a2, wq, NULL, logq, d2);
    uint64_t *k = (uint64_t *)malloc(PQQ * 8), *ks = (uint64_t *)malloc(PQ * 8);
    for (int h = 0; h < 2; h++) {
        nr_polymul(logN, T2, d2, wq, evk + (size_t)h * wQQ * N, wQQ, NULL, logq + logQ, k);
        nr_shift_round(N, k, logq + logQ, logQ, logq, ks);
        nr_addsub(N, logq, h ? d1 : d0, ks, 0, out + (size_t)h * PQ);
    }
    free(T1); free(T2); free(d0); free(d1); free(d2); free(t); free(k); free(ks);
}

/* Rescale by p = 2^logp (Sec. 3.1): c' = round(c / p) mod q/p. */
void or_nr_rescale(int logN, int logq, int logp, const uint64_t *ct, uint64_t *out)
{
    uint64_t N = 1ull << logN;
    int wq = nwords(logq), wo = nwords(logq - logp);
    for (int h = 0; h < 2; h++)
        nr_shift_round(N, ct + (size_t)h * wq * N, logq, logp, logq - logp, out + (size_t)h * wo * N);
}

/* A product mod (X^N + 1, 2^kout), exposed for the schoolbook pins. */
void or_nr_polymul(int logN, int np, const uint64_t *primes, const uint64_t *psis, const uint64_t *A, int wa,
                   const uint64_t *B, int wb, const int64_t *bs, int kout, uint64_t *C)
{
    crt_t *T = (crt_t *)malloc(sizeof(crt_t));
    crt_init(T, np, primes, psis);
    nr_polymul(logN, T, A, wa, B, wb, bs, kout, C);
    free(T);
}

/* Uniform BigInt coefficients mod 2^k from a stream (word by word). */
static void nr_uniform(rng_t *r, uint64_t N, int k, uint64_t *a)
{
    int w = nwords(k);
    for (uint64_t n = 0; n < N; n++)
        for (int i = 0; i < w; i++) {
            uint64_t v = rng_next(r);
            if (i == w - 1 && (k & 63)) v &= (1ull << (k & 63)) - 1;
            a[(size_t)i * N + n] = v;
        }
}
static void nr_add_small(uint64_t N, int k, uint64_t *a, const int64_t *s) /* a += s mod 2^k */
{
    int w = nwords(k);
    for (uint64_t n = 0; n < N; n++) {
        uint64_t add = (uint64_t)s[n], ext = s[n] < 0 ? ~0ull : 0, c = 0;
        for (int i = 0; i < w; i++) {
            u128 t = (u128)a[(size_t)i * N + n] + (i == 0 ? add : ext) + c;
            a[(size_t)i * N + n] = (uint64_t)t;
            c = (uint64_t)(t >> 64);
        }
        if (k & 63) a[(size_t)(w - 1) * N + n] &= (1ull << (k & 63)) - 1;
    }
}

enum { ST_NR_PK_A = 200, ST_NR_PK_E = 201, ST_NR_EVK_A = 202, ST_NR_EVK_E = 203, ST_NR_U = 204,
       ST_NR_E0 = 205, ST_NR_E1 = 206 };

/* Keys (Sec. 3.1 with the non-RNS moduli): pk mod Q: a uniform, b = a s + e;
 * evk mod Q^2: a uniform, b = a s + e + Q s^2.  sk from or_keygen_sk. */
void or_nr_keygen(int logN, int logQ, int np, const uint64_t *primes, const uint64_t *psis, double sigma,
                  const int64_t *s, uint64_t seed, uint64_t *pk, uint64_t *evk)
{
    uint64_t N = 1ull << logN;
    int wQ = nwords(logQ), wQQ = nwords(2 * logQ);
    crt_t *T = (crt_t *)malloc(sizeof(crt_t));
    crt_init(T, np, primes, psis);
    int64_t *e = (int64_t *)malloc(N * sizeof(int64_t));
    /* pk */
    rng_t ra = rng_open(seed, ST_NR_PK_A), re = rng_open(seed, ST_NR_PK_E);
    nr_uniform(&ra, N, logQ, pk + (size_t)wQ * N);
    nr_polymul(logN, T, pk + (size_t)wQ * N, wQ, NULL, 0, s, logQ, pk);
    for (uint64_t n = 0; n < N; n++) e[n] = rng_gauss(&re, sigma);
    nr_add_small(N, logQ, pk, e);
    /* evk: b = a s + e + Q s^2 mod Q^2 */
    rng_t rea = rng_open(seed, ST_NR_EVK_A), ree = rng_open(seed, ST_NR_EVK_E);
    nr_uniform(&rea, N, 2 * logQ, evk + (size_t)wQQ * N);
    nr_polymul(logN, T, evk + (size_t)wQQ * N, wQQ, NULL, 0, s, 2 * logQ, evk);
    for (uint64_t n = 0; n < N; n++) e[n] = rng_gauss(&ree, sigma);
    nr_add_small(N, 2 * logQ, evk, e);
    int64_t *s2 = (int64_t *)calloc(N, sizeof(int64_t)); /* s^2 in Z[X]/(X^N+1), small */
    for (uint64_t i = 0; i < N; i++)
        if (s[i])
            for (uint64_t j = 0; j < N; j++)
                if (s[j]) {
                    uint64_t d = i + j;
                    if (d < N) s2[d] += s[i] * s[j];
                    else s2[d - N] -= s[i] * s[j];
                }
    /* + Q s^2: add s2 shifted left by logQ bits */
    for (uint64_t n = 0; n < N; n++) {
        uint64_t tmp[MW_MAX] = {0}, add[MW_MAX] = {0};
        for (int i = 0; i < wQQ; i++) tmp[i] = evk[(size_t)i * N + n];
        int64_t v = s2[n];
        uint64_t mag = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
        add[logQ / 64] = mag << (logQ & 63);
        if ((logQ & 63) && logQ / 64 + 1 < MW_MAX) add[logQ / 64 + 1] = mag >> (64 - (logQ & 63));
        if (v < 0) mw_sub(tmp, add, wQQ + 1);
        else {
            uint64_t c = 0;
            for (int i = 0; i <= wQQ; i++) {
                u128 t2 = (u128)tmp[i] + add[i] + c;
                tmp[i] = (uint64_t)t2;
                c = (uint64_t)(t2 >> 64);
            }
        }
        for (int i = 0; i < wQQ; i++) {
            uint64_t x = tmp[i];
            if (i == wQQ - 1 && ((2 * logQ) & 63)) x &= (1ull << ((2 * logQ) & 63)) - 1;
            evk[(size_t)i * N + n] = x;
        }
    }
    free(T); free(e); free(s2);
}

/* Encryption at logq of the integer plaintext pt (Sec. 3.1):
 * a = v pk.a + e1, b = v pk.b + e0 + pt (mod q), v ZO(1/2). */
void or_nr_encrypt(int logN, int logq, int logQ, int np, const uint64_t *primes, const uint64_t *psis,
                   double sigma, const uint64_t *pk, const int64_t *pt, uint64_t seed, uint64_t *ct)
{
    uint64_t N = 1ull << logN;
    int wQ = nwords(logQ), wq = nwords(logq);
    crt_t *T = (crt_t *)malloc(sizeof(crt_t));
    crt_init(T, np, primes, psis);
    int64_t *v = (int64_t *)malloc(N * sizeof(int64_t)), *e = (int64_t *)malloc(N * sizeof(int64_t));
    rng_t ru = rng_open(seed, ST_NR_U), r0 = rng_open(seed, ST_NR_E0), r1 = rng_open(seed, ST_NR_E1);
    for (uint64_t n = 0; n < N; n++) v[n] = rng_zo(&ru);
    nr_polymul(logN, T, pk, wQ, NULL, 0, v, logq, ct);
    nr_polymul(logN, T, pk + (size_t)wQ * N, wQ, NULL, 0, v, logq, ct + (size_t)wq * N);
    for (uint64_t n = 0; n < N; n++) e[n] = rng_gauss(&r0, sigma) + pt[n];
    nr_add_small(N, logq, ct, e);
    for (uint64_t n = 0; n < N; n++) e[n] = rng_gauss(&r1, sigma);
    nr_add_small(N, logq, ct + (size_t)wq * N, e);
    free(T); free(v); free(e);
}

/* m = b - a s mod q, centred, returned as doubles (|m| < 2^1023). */
void or_nr_decrypt(int logN, int logq, int np, const uint64_t *primes, const uint64_t *psis, const int64_t *s,
                   const uint64_t *ct, double *m)
{
    uint64_t N = 1ull << logN;
    int wq = nwords(logq);
    crt_t *T = (crt_t *)malloc(sizeof(crt_t));
    crt_init(T, np, primes, psis);
    uint64_t *as = (uint64_t *)malloc((size_t)wq * N * 8), *r = (uint64_t *)malloc((size_t)wq * N * 8);
    nr_polymul(logN, T, ct + (size_t)wq * N, wq, NULL, 0, s, logq, as);
    nr_addsub(N, logq, ct, as, 1, r);
    for (uint64_t n = 0; n < N; n++) {
        int neg = (r[(size_t)(wq - 1) * N + n] >> (((logq - 1) & 63))) & 1; /* top bit of the logq-bit value */
        double acc = 0, scale = 1;
        uint64_t c = 1;
        for (int i = 0; i < wq; i++) {
            uint64_t x = r[(size_t)i * N + n];
            if (neg) { /* value - q: negate the logq-bit two's complement */
                u128 t = (u128)(~x) + c;
                x = (uint64_t)t;
                c = (uint64_t)(t >> 64);
                if (i == wq - 1 && (logq & 63)) x &= (1ull << (logq & 63)) - 1;
            }
            acc += (double)x * scale;
            scale *= 18446744073709551616.0;
        }
        m[n] = neg ? -acc : acc;
    }
    free(T); free(as); free(r);
}
