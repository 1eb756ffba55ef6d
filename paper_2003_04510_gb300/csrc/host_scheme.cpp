// host_scheme.cpp -- host side of the scheme (Sec. 3.1 of the paper):
// sampling, key generation, encoding, encryption and decryption.  These run
// once per key / message and are not on the timed path; the HE Mul itself
// runs on the GPU.
//
// Random words: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a
// counter-based generator.  Stream (seed, id) starts at state
// S = mix64(seed + (id+1)*gamma); its k-th word (k = 1, 2, ...) is
// mix64(S + k*gamma).  Stream ids: 1 secret, 2/3 public-key a/e, 4/5/6
// encryption u/e0/e1, 16+j / 48+j evaluation-key digit j a/e.
// Distributions: secret HWT(h) by partial Fisher-Yates with one sign word per
// pick; u ZO(1/2) from the two low bits of one word; errors rounded Gaussian
// (Box-Muller, one sample per two words, rejected beyond floor(6 sigma));
// uniform residues by rejection on the low bitlen(t) bits.
#include <cmath>
#include <complex>
#include <cstring>

#include "he_internal.h"
#include "host_math.h"

namespace he {
using namespace hm;

namespace {

constexpr u64 kGamma = 0x9E3779B97F4A7C15ull;
inline u64 mix(u64 z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Stream {
    u64 s, k;
    Stream(u64 seed, u64 id) : s(mix(seed + (id + 1) * kGamma)), k(0) {}
    u64 next() { return mix(s + (++k) * kGamma); }
    u64 below(u64 t)
    {
        u64 mask = 1;
        while (mask < t) mask <<= 1;
        mask -= 1;  // 2^bitlen(t-1) - 1 ... covers [0, t)
        for (;;) {
            u64 v = next() & mask;
            if (v < t) return v;
        }
    }
    int64_t gauss(double sigma)
    {
        const int64_t bound = (int64_t)std::floor(6.0 * sigma);
        for (;;) {
            u64 a = next(), b = next();
            double u1 = (double)((a >> 11) + 1) * 0x1.0p-53;
            double u2 = (double)(b >> 11) * 0x1.0p-53;
            double rad = std::sqrt(-2.0 * std::log(u1));
            double cs = std::cos(6.283185307179586 * u2);
            int64_t v = std::llround(sigma * (rad * cs));
            if (v <= bound && v >= -bound) return v;
        }
    }
    int64_t zo()
    {
        u64 w = next();
        if (!(w & 1)) return 0;
        return (w & 2) ? -1 : 1;
    }
};

enum { kSk = 1, kPkA = 2, kPkE = 3, kEncU = 4, kEncE0 = 5, kEncE1 = 6, kEvkA = 16, kEvkE = 48,
       kRotA = 80, kRotE = 112, kSeedA = 144 };

inline u64 lift(int64_t v, u64 m)
{
    if (v >= 0) return (u64)v % m;
    u64 r = (0ull - (u64)v) % m;  // |v|, also for INT64_MIN
    return r ? m - r : 0;
}

// In-place forward NTT (Algo 3 order, bit-reversed output) with Shoup twiddles.
void host_ntt(const he_ctx *c, int e, u64 *a)
{
    const u64 q = c->ext[e];
    const u64 *W = c->w[e].data(), *Ws = c->wsh[e].data();
    const int N = c->N;
    for (int m = 1, t = N / 2; m < N; m <<= 1, t >>= 1) {
        for (int j = 0; j < m; j++) {
            u64 w = W[m + j], ws = Ws[m + j];
            u64 *x = a + 2 * (size_t)j * t, *y = x + t;
            for (int k = 0; k < t; k++) {
                u64 v = y[k] * w - (u64)(((u128)y[k] * ws) >> 64) * q;
                if (v >= q) v -= q;
                u64 u = x[k];
                x[k] = add(u, v, q);
                y[k] = sub(u, v, q);
            }
        }
    }
}

void host_intt(const he_ctx *c, int e, u64 *a)
{
    const u64 q = c->ext[e];
    const u64 *W = c->iw[e].data(), *Ws = c->iwsh[e].data();
    const int N = c->N;
    for (int m = N / 2, t = 1; m >= 1; m >>= 1, t <<= 1) {
        for (int j = 0; j < m; j++) {
            u64 w = W[m + j], ws = Ws[m + j];
            u64 *x = a + 2 * (size_t)j * t, *y = x + t;
            for (int k = 0; k < t; k++) {
                u64 u = x[k], v = y[k];
                x[k] = add(u, v, q);
                u64 d = sub(u, v, q);
                u64 r = d * w - (u64)(((u128)d * ws) >> 64) * q;
                y[k] = r >= q ? r - q : r;
            }
        }
    }
    const u64 ni = c->ninv[e], nis = c->ninv_sh[e];
    for (int k = 0; k < N; k++) {
        u64 r = a[k] * ni - (u64)(((u128)a[k] * nis) >> 64) * q;
        a[k] = r >= q ? r - q : r;
    }
}

void small_ntt(const he_ctx *c, int e, const int64_t *v, u64 *out)
{
    for (int k = 0; k < c->N; k++) out[k] = lift(v[k], c->ext[e]);
    host_ntt(c, e, out);
}

void sample_sk(const he_ctx *c, u64 seed, int64_t *s)
{
    const int N = c->N;
    std::vector<u64> perm(N);
    for (int i = 0; i < N; i++) { perm[i] = (u64)i; s[i] = 0; }
    Stream st(seed, kSk);
    for (int k = 0; k < c->prm.h; k++) {
        u64 r = (u64)k + st.below((u64)(N - k));
        std::swap(perm[k], perm[r]);
        s[perm[k]] = (st.next() & 1) ? -1 : 1;
    }
}

void make_pk(const he_ctx *c, u64 seed, const int64_t *s, u64 *pk)
{
    const int N = c->N, L = c->L, K = c->K;
    Stream sa(seed, kPkA), se(seed, kPkE);
    std::vector<int64_t> err(N);
    for (int k = 0; k < N; k++) err[k] = se.gauss(c->prm.sigma);
    std::vector<u64> S(N), Er(N);
    for (int i = 0; i < L; i++) {
        const int e = K + i;
        const u64 q = c->ext[e];
        u64 *b = pk + (size_t)i * N, *a = pk + (size_t)(L + i) * N;
        for (int k = 0; k < N; k++) a[k] = sa.below(q);
        small_ntt(c, e, s, S.data());
        small_ntt(c, e, err.data(), Er.data());
        for (int k = 0; k < N; k++) b[k] = add(mul(a[k], S[k], q), Er[k], q);
    }
}

// Key-switching key to s for the source key `from` (NTT domain per limb):
// b_j = a_j s + e_j + [t in digit j] P from.  The evaluation key has
// from = s^2 (streams kEvkA/kEvkE), a rotation key from = kappa_g(s)
// (streams kRotA/kRotE).
void make_switch_key(const he_ctx *c, u64 seed, const int64_t *s, const int64_t *from_small, bool square, int sa0,
                     int se0, u64 *key)
{
    const int N = c->N, L = c->L, K = c->K, E = c->E;
    std::vector<u64> S(N), F(N), Er(N);
    std::vector<int64_t> err(N);
    for (int j = 0; j < c->dnum; j++) {
        Stream sa(seed, sa0 + j), se(seed, se0 + j);
        for (int k = 0; k < N; k++) err[k] = se.gauss(c->prm.sigma);
        const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, L);
        u64 *B = key + (size_t)(2 * j) * E * N, *A = key + (size_t)(2 * j + 1) * E * N;
        for (int e = 0; e < E; e++) {
            const u64 t = c->ext[e];
            u64 *a = A + (size_t)e * N, *b = B + (size_t)e * N;
            for (int k = 0; k < N; k++) a[k] = sa.below(t);
            small_ntt(c, e, s, S.data());
            small_ntt(c, e, err.data(), Er.data());
            if (!square) small_ntt(c, e, from_small, F.data());
            const bool gadget = e >= K && (e - K) >= lo && (e - K) < hi;
            u64 Pm = 1;
            for (int k = 0; k < K && gadget; k++) Pm = mul(Pm, c->ext[k] % t, t);
            for (int k = 0; k < N; k++) {
                u64 v = add(mul(a[k], S[k], t), Er[k], t);
                if (gadget) v = add(v, mul(Pm, square ? mul(S[k], S[k], t) : F[k], t), t);
                b[k] = v;
            }
        }
    }
}

// Seeded evaluation key: b halves only, with a_j[e][n] = floor((w1 2^64 + w2)
// t / 2^128), w1 and w2 words 2(eN+n) and 2(eN+n)+1 of stream kSeedA + j.
void make_seeded_evk(const he_ctx *c, u64 seed, const int64_t *s, u64 *evk_b)
{
    const int N = c->N, L = c->L, K = c->K, E = c->E;
    std::vector<u64> S(N), Er(N);
    std::vector<int64_t> err(N);
    for (int j = 0; j < c->dnum; j++) {
        Stream se(seed, kEvkE + j), sa(seed, kSeedA + j);
        for (int k = 0; k < N; k++) err[k] = se.gauss(c->prm.sigma);
        const int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, L);
        for (int e = 0; e < E; e++) {
            const u64 t = c->ext[e];
            u64 *b = evk_b + ((size_t)j * E + e) * N;
            small_ntt(c, e, s, S.data());
            small_ntt(c, e, err.data(), Er.data());
            const bool gadget = e >= K && (e - K) >= lo && (e - K) < hi;
            u64 Pm = 1;
            for (int k = 0; k < K && gadget; k++) Pm = mul(Pm, c->ext[k] % t, t);
            for (int k = 0; k < N; k++) {
                const u64 idx = (u64)e * N + k;
                const u64 w1 = mix(sa.s + (2 * idx + 1) * kGamma), w2 = mix(sa.s + (2 * idx + 2) * kGamma);
                const u128 hiw = (u128)w1 * t, low = (u128)w2 * t;
                const u64 a = (u64)((hiw + (low >> 64)) >> 64);
                u64 v = add(mul(a, S[k], t), Er[k], t);
                if (gadget) v = add(v, mul(Pm, mul(S[k], S[k], t), t), t);
                b[k] = v;
            }
        }
    }
}

// a(X) -> a(X^g) mod X^N + 1 on a small signed polynomial
void small_automorphism(int N, const int64_t *a, u64 g, int64_t *out)
{
    const u64 twoN = 2 * (u64)N;
    for (int i = 0; i < N; i++) {
        const u64 e = (u64)i * (g % twoN) % twoN;
        if (e < (u64)N) out[e] = a[i];
        else out[e - N] = -a[i];
    }
}

void make_evk(const he_ctx *c, u64 seed, const int64_t *s, u64 *evk)
{
    make_switch_key(c, seed, s, nullptr, true, kEvkA, kEvkE, evk);
}

// ---- canonical embedding ---------------------------------------------------
typedef std::complex<double> cd;

// in-place iterative radix-2 FFT, sign -1: X_k = sum x_n e^{-2 pi i nk/N}
void fft(std::vector<cd> &x, int sign)
{
    const size_t n = x.size();
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(x[i], x[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1) {
        const double ang = sign * 2.0 * M_PI / (double)len;
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; k++) {
                cd w(std::cos(ang * (double)k), std::sin(ang * (double)k));
                cd u = x[i + k], v = x[i + k + len / 2] * w;
                x[i + k] = u + v;
                x[i + k + len / 2] = u - v;
            }
    }
}

void slot_index(int logN, std::vector<size_t> &rows, std::vector<size_t> &conj)
{
    const u64 N = 1ull << logN, twoN = 2 * N;
    rows.resize(N / 2);
    conj.resize(N / 2);
    u64 g = 1;
    for (u64 k = 0; k < N / 2; k++) {
        rows[k] = (size_t)((g - 1) / 2);
        conj[k] = (size_t)((twoN - g - 1) / 2);
        g = g * 5 % twoN;
    }
}

}  // namespace

}  // namespace he

using namespace he;
using namespace he::hm;

extern "C" {

int he_keygen_from_sk(he_ctx *c, uint64_t seed, const int64_t *sk, uint64_t *pk, uint64_t *evk)
{
    if (!c || !sk) return HE_EINVAL;
    if (pk) make_pk(c, seed, sk, pk);
    if (evk) make_evk(c, seed, sk, evk);
    return HE_OK;
}

int he_plain_ntt(he_ctx *c, const int64_t *coeffs, int level, uint64_t *pt)
{
    if (!c || !coeffs || !pt) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    for (int i = 0; i < level; i++) {
        u64 *o = pt + (size_t)i * c->N;
        const u64 q = c->ext[c->K + i];
        for (int k = 0; k < c->N; k++) o[k] = lift(coeffs[k], q);
        host_ntt(c, c->K + i, o);
    }
    return HE_OK;
}

uint64_t he_galois_elt(const he_ctx *c, int steps)
{
    if (!c) return 0;
    const u64 twoN = 2 * (u64)c->N, half = (u64)c->N / 2;
    const u64 e = (u64)(((long long)steps % (long long)half + (long long)half) % (long long)half);
    u64 g = 1;
    for (u64 k = 0; k < e; k++) g = g * 5 % twoN;
    return g;
}

uint64_t he_conj_elt(const he_ctx *c)
{
    if (!c) return 0;
    return 2 * (u64)c->N - 1;  // X -> X^(-1) = X^(2N-1) mod X^N + 1
}

int he_keygen_seeded(he_ctx *c, uint64_t seed, const int64_t *sk, uint64_t *evk_b)
{
    if (!c || !sk || !evk_b) return HE_EINVAL;
    make_seeded_evk(c, seed, sk, evk_b);
    return HE_OK;
}

int he_keygen_rot(he_ctx *c, uint64_t seed, const int64_t *sk, uint64_t galois, uint64_t *rk)
{
    if (!c || !sk || !rk) return HE_EINVAL;
    if (galois % 2 == 0 || galois >= 2 * (u64)c->N) return HE_EINVAL;
    std::vector<int64_t> ks(c->N);
    small_automorphism(c->N, sk, galois, ks.data());
    make_switch_key(c, seed, sk, ks.data(), false, kRotA, kRotE, rk);
    return HE_OK;
}

int he_keygen(he_ctx *c, uint64_t seed, int64_t *sk, uint64_t *pk, uint64_t *evk)
{
    if (!c) return HE_EINVAL;
    std::vector<int64_t> s(c->N);
    sample_sk(c, seed, s.data());
    if (sk) memcpy(sk, s.data(), sizeof(int64_t) * c->N);
    return he_keygen_from_sk(c, seed, s.data(), pk, evk);
}

int he_encode(he_ctx *c, const double *re, const double *im, size_t n, double scale, int64_t *coeffs)
{
    if (!c || !re || !im || !coeffs || n != (size_t)c->N / 2) return HE_EINVAL;
    const int N = c->N;
    std::vector<size_t> rows, conj;
    slot_index(c->logN, rows, conj);
    std::vector<cd> full(N, cd(0, 0));
    for (size_t k = 0; k < n; k++) {
        cd z(scale * re[k], scale * im[k]);
        full[rows[k]] = z;
        full[conj[k]] = std::conj(z);
    }
    fft(full, -1);  // sum_r full[r] e^{-2 pi i r j / N}
    for (int j = 0; j < N; j++) {
        cd zinv(std::cos(-M_PI * j / N), std::sin(-M_PI * j / N));
        double t = (full[j] * zinv).real() / N;
        coeffs[j] = (int64_t)std::llround(t);
    }
    return HE_OK;
}

int he_decode(he_ctx *c, const double *coeffs, double *re, double *im, size_t n)
{
    if (!c || !coeffs || !re || !im || n != (size_t)c->N / 2) return HE_EINVAL;
    const int N = c->N;
    std::vector<cd> v(N);
    for (int j = 0; j < N; j++) v[j] = coeffs[j] * cd(std::cos(M_PI * j / N), std::sin(M_PI * j / N));
    fft(v, +1);  // sum_j (t_j zeta^j) e^{+2 pi i r j / N}
    std::vector<size_t> rows, conj;
    slot_index(c->logN, rows, conj);
    for (size_t k = 0; k < n; k++) {
        re[k] = v[rows[k]].real();
        im[k] = v[rows[k]].imag();
    }
    return HE_OK;
}

int he_encrypt_poly(he_ctx *c, const uint64_t *pk, const int64_t *pt, int level, uint64_t seed, uint64_t *ct)
{
    if (!c || !pk || !pt || !ct) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    const int N = c->N, L = c->L, K = c->K;
    std::vector<int64_t> u(N), e0(N), e1(N);
    Stream su(seed, kEncU), s0(seed, kEncE0), s1(seed, kEncE1);
    for (int k = 0; k < N; k++) u[k] = su.zo();
    for (int k = 0; k < N; k++) e0[k] = s0.gauss(c->prm.sigma);
    for (int k = 0; k < N; k++) e1[k] = s1.gauss(c->prm.sigma);
    std::vector<u64> U(N), E0(N), E1(N);
    for (int i = 0; i < level; i++) {
        const int e = K + i;
        const u64 q = c->ext[e];
        small_ntt(c, e, u.data(), U.data());
        for (int k = 0; k < N; k++) E0[k] = add(lift(e0[k], q), lift(pt[k], q), q);
        host_ntt(c, e, E0.data());
        small_ntt(c, e, e1.data(), E1.data());
        const u64 *p0 = pk + (size_t)i * N, *p1 = pk + (size_t)(L + i) * N;
        u64 *cb = ct + (size_t)i * N, *ca = ct + (size_t)(level + i) * N;
        for (int k = 0; k < N; k++) {
            cb[k] = add(mul(U[k], p0[k], q), E0[k], q);
            ca[k] = add(mul(U[k], p1[k], q), E1[k], q);
        }
    }
    return HE_OK;
}

int he_encrypt(he_ctx *c, const uint64_t *pk, const double *re, const double *im, size_t n, double scale, int level,
               uint64_t seed, uint64_t *ct)
{
    if (!c) return HE_EINVAL;
    std::vector<int64_t> pt(c->N);
    int rc = he_encode(c, re, im, n, scale, pt.data());
    if (rc) return rc;
    return he_encrypt_poly(c, pk, pt.data(), level, seed, ct);
}

int he_decrypt_poly(he_ctx *c, const int64_t *sk, const uint64_t *ct, int level, uint64_t *m)
{
    if (!c || !sk || !ct || !m) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    const int N = c->N, K = c->K;
    std::vector<u64> S(N);
    for (int i = 0; i < level; i++) {
        const int e = K + i;
        const u64 q = c->ext[e];
        small_ntt(c, e, sk, S.data());
        const u64 *cb = ct + (size_t)i * N, *ca = ct + (size_t)(level + i) * N;
        u64 *mi = m + (size_t)i * N;
        for (int k = 0; k < N; k++) mi[k] = sub(cb[k], mul(ca[k], S[k], q), q);
        host_intt(c, e, mi);
    }
    return HE_OK;
}

int he_decrypt(he_ctx *c, const int64_t *sk, const uint64_t *ct, int level, double scale, double *re, double *im,
               size_t n)
{
    if (!c) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    const int N = c->N, K = c->K;
    std::vector<u64> m((size_t)level * N);
    int rc = he_decrypt_poly(c, sk, ct, level, m.data());
    if (rc) return rc;
    std::vector<double> coef(N);
    const u64 q0 = c->ext[K];
    if (level == 1) {
        for (int k = 0; k < N; k++) {
            u64 v = m[k];
            coef[k] = (v > q0 / 2 ? -(double)(q0 - v) : (double)v) / scale;
        }
    } else {
        const u64 q1 = c->ext[K + 1];
        const u64 q0inv = inv(q0 % q1, q1);
        const u128 Q = (u128)q0 * q1;
        for (int k = 0; k < N; k++) {
            u64 r0 = m[k], r1 = m[(size_t)N + k];
            u64 t = mul(sub(r1, r0 % q1, q1), q0inv, q1);
            u128 x = (u128)r0 + (u128)q0 * t;  // in [0, q0 q1)
            double v = x > Q / 2 ? -(double)(Q - x) : (double)x;
            coef[k] = v / scale;
        }
    }
    return he_decode(c, coef.data(), re, im, n);
}

}  // extern "C"
