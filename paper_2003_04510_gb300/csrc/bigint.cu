// bigint.cu -- the paper's own (non-RNS) HEAAN HE Mul on sm_103a.
//
// Ciphertext and key coefficients are BigInts modulo powers of two (the
// paper's Table 3: q = 2^logq, Q = 2^logQ, p = 2^logp), stored word-major:
// word w of coefficient n at a[w * N + n], little-endian, ceil(k / 64) words.
// Each polynomial product follows the paper's five steps (Fig. 2, Sec. 4):
//   CRT    BigInt -> residues mod np NTT primes (k_nr_crt: 28-bit chunks
//          times 2^(28k) mod p_i, lazy 32x32->64 multiply-adds, one Barrett
//          reduction -- Algo 1's accumulate-then-reduce, without BigInt carries)
//   NTT    the RNS path's k_ntt_pass over the context's primes
//   mul    element-wise (k_nr_tensor: d0 = b1 b2, d1 = a1 b2 + a2 b1,
//          d2 = a1 a2 mod p_i; k_nr_ks_mult: d2 times the evaluation key)
//   iNTT   with N^-1 [Phat_i^-1]_{p_i} folded into its scaling, so its
//          outputs are y_i = [x_i Phat_i^-1]_{p_i}
//   iCRT   (k_nr_icrt: Algo 6's matrix form) C = sum_i y_i Phat_i - u P with
//          u = round(sum_i y_i / p_i), which is exact because P exceeds four
//          times the product's magnitude (the fraction is never near 1/2);
//          C mod 2^(64 W) column by column, u P taken from a table of
//          (2^(64 W) - u P) rows.
// Region 2 (the evaluation key, coefficients mod Q^2) folds the division by
// Q with rounding and the final addition into its iCRT.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "he_internal.h"
#include "modarith.cuh"

struct he_nr_plan {
    he_ctx *c = nullptr;
    int logQ = 0, logp = 0, np1 = 0, np2 = 0, W1 = 0, W2 = 0;
    int chunks_ct = 0, chunks_evk = 0;
    void *dev = nullptr;  // one allocation: tables and NTT group lists
    const u64 *crt = nullptr;           // [np2][chunks_evk]: 2^(28k) mod p_i, split at bit 28
    const u64 *m1 = nullptr, *neg1 = nullptr, *m2 = nullptr, *neg2 = nullptr;
    const double *inv1 = nullptr, *inv2 = nullptr;
    const he::NttGroup *gF1 = nullptr, *gI1 = nullptr, *gF2 = nullptr, *gI2 = nullptr, *gFe = nullptr;
    int nF1 = 0, nI1 = 0, nF2 = 0, nI2 = 0, nFe = 0;
};

namespace he {

namespace {

constexpr int kT = 256;     // one coefficient per thread (CRT, products, rescale)
constexpr int kIT = 128;    // iCRT threads per CTA
constexpr int kCP = 8;      // primes per CTA in the CRT
constexpr int kMaxNp = 64;  // primes of a plan (the context's ciphertext primes)
constexpr int kChunkBlock = 40;  // 28-bit chunks accumulated before a reduction

__device__ __forceinline__ ulonglong2 ld2(const u64 *p) { return *reinterpret_cast<const ulonglong2 *>(p); }
__device__ __forceinline__ void st2(u64 *p, u64 x, u64 y) { *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(x, y); }

// bits [28k, 28k + 28) of the WI-word integer w
template <int WI>
__device__ __forceinline__ uint32_t chunk28(const u64 (&w)[WI], int k)
{
    const int bit = 28 * k, q = bit >> 6, o = bit & 63;
    u64 v = q < WI ? w[q] >> o : 0;
    if (o > 36 && q + 1 < WI) v |= w[q + 1] << (64 - o);
    return (uint32_t)(v & 0xFFFFFFFull);
}

// CRT of `polys` BigInt polynomials (wi <= WI words each, word-major, poly
// stride `stride` words) to residues out[poly][np][N].  grid: x over N / kT,
// y over polys, z over prime groups of kCP.
template <int WI>
__global__ void __launch_bounds__(kT)
k_nr_crt(const u64 *__restrict__ in, int wi, size_t stride, u64 *__restrict__ out, int np,
         const u64 *__restrict__ tab, int tab_stride, const DevPrime *__restrict__ primes, int K, int N)
{
    constexpr int CH = (64 * WI + 27) / 28;
    __shared__ u64 sc[kCP][CH];
    const int i0 = blockIdx.z * kCP, cnt = min(kCP, np - i0);
    for (int t = threadIdx.x; t < kCP * CH; t += kT) {
        const int r = t / CH, k = t % CH;
        sc[r][k] = r < cnt ? tab[(size_t)(i0 + r) * tab_stride + k] : 0;
    }
    const int n = blockIdx.x * kT + threadIdx.x;
    const u64 *src = in + (size_t)blockIdx.y * stride + n;
    griddep_wait();
    u64 w[WI];
#pragma unroll
    for (int q = 0; q < WI; q++) w[q] = q < wi ? src[(size_t)q * N] : 0;
    __syncthreads();
    for (int r = 0; r < cnt; r++) {
        const DevPrime pr = primes[K + i0 + r];
        u64 res = 0;
#pragma unroll
        for (int k0 = 0; k0 < CH; k0 += kChunkBlock) {
            u64 a0 = 0, a1 = 0;  // weights 1 and 2^28: each term below 2^57, 40 terms below 2^63
#pragma unroll
            for (int k = k0; k < min(CH, k0 + kChunkBlock); k++) {
                const uint32_t x = chunk28<WI>(w, k);
                const u64 b = sc[r][k];
                a0 = mad_wide(x, (uint32_t)b, a0);
                a1 = mad_wide(x, (uint32_t)(b >> 32), a1);
            }
            U128 v;
            v.lo = a0 + (a1 << 28);
            v.hi = (a1 >> 36) + (v.lo < a0 ? 1ull : 0ull);
            res = add_mod(res, barrett128(v, pr.q, pr.mu, pr.s), pr.q);
        }
        out[((size_t)blockIdx.y * np + i0 + r) * N + n] = res;
    }
}

// Region 1 products in place: slots [A1 | B1 | A2 | B2][np][N] become
// [D0 | D1 | D2 | -] with d0 = b1 b2, d1 = a1 b2 + a2 b1, d2 = a1 a2 mod p_i.
// grid: x over N / 2 / kT, y over primes.
__global__ void __launch_bounds__(kT)
k_nr_tensor(u64 *__restrict__ r, int np, const DevPrime *__restrict__ primes, int K, int N)
{
    const int i = blockIdx.y;
    const DevPrime pr = primes[K + i];
    const size_t n = 2 * ((size_t)blockIdx.x * kT + threadIdx.x);
    const size_t L = (size_t)np * N, o = (size_t)i * N + n;
    griddep_wait();
    const ulonglong2 a1 = ld2(r + o), b1 = ld2(r + L + o), a2 = ld2(r + 2 * L + o), b2 = ld2(r + 3 * L + o);
    U128 x = mul_wide(a1.x, b2.x), y = mul_wide(a1.y, b2.y);
    mac(x, a2.x, b1.x);
    mac(y, a2.y, b1.y);
    st2(r + o, mul_mod(b1.x, b2.x, pr.q, pr.mu, pr.s), mul_mod(b1.y, b2.y, pr.q, pr.mu, pr.s));
    st2(r + L + o, barrett128(x, pr.q, pr.mu, pr.s), barrett128(y, pr.q, pr.mu, pr.s));
    st2(r + 2 * L + o, mul_mod(a1.x, a2.x, pr.q, pr.mu, pr.s), mul_mod(a1.y, a2.y, pr.q, pr.mu, pr.s));
}

// Region 2 products: r[0] (d2 residues) -> KS_b in place, r[1] = KS_a, with
// the prepared key ek = [b | a][np][N].  grid: x over N / 2 / kT, y over primes.
__global__ void __launch_bounds__(kT)
k_nr_ks_mult(u64 *__restrict__ r, const u64 *__restrict__ ek, int np, const DevPrime *__restrict__ primes, int K,
             int N)
{
    const int i = blockIdx.y;
    const DevPrime pr = primes[K + i];
    const size_t n = 2 * ((size_t)blockIdx.x * kT + threadIdx.x);
    const size_t L = (size_t)np * N, o = (size_t)i * N + n;
    griddep_wait();
    const ulonglong2 d = ld2(r + o), kb = ld2(ek + o), ka = ld2(ek + L + o);
    st2(r + o, mul_mod(d.x, kb.x, pr.q, pr.mu, pr.s), mul_mod(d.y, kb.y, pr.q, pr.mu, pr.s));
    st2(r + L + o, mul_mod(d.x, ka.x, pr.q, pr.mu, pr.s), mul_mod(d.y, ka.y, pr.q, pr.mu, pr.s));
}

// iCRT of polys y[poly][np][N] (y_i = [x_i Phat_i^-1]_{p_i}) into BigInts.
// T = sum_i y_i M_i + NEG_u (mod 2^(64 W)), M_i = Phat_i mod 2^(64 W),
// NEG_u = (2^(64 W) - u P + rnd) mod 2^(64 W), u = round(sum_i y_i / p_i).
// Each thread keeps one accumulator per column in registers (column w
// collects the low words of y_i M_i[w] and the high words of y_i M_i[w-1]),
// in passes over at most 19 columns, reading the y_i once per pass; the
// carries run after each pass's sums.
// KS = false: out[poly] = T mod 2^kout (wo words; polys ostride * N words apart).
// KS = true: out[poly] = d[poly] + floor((T + 2^(s-1)) / 2^s) mod 2^kout, the
// rounding term being part of NEG_u (s = logQ).
// grid: x over N / kIT, y over polys; dynamic shared memory holds M
// ([np][W]) and NEG ([np + 1][W]).
template <int W, bool KS>
__global__ void __launch_bounds__(kIT)
k_nr_icrt(const u64 *__restrict__ y, int np, const u64 *__restrict__ M, const u64 *__restrict__ NEG,
          const double *__restrict__ inv, u64 *__restrict__ out, int ostride, int wo, int kout,
          const u64 *__restrict__ d, int s, int N)
{
    extern __shared__ __align__(16) u64 sh[];
    u64 *sM = sh;                         // [np][W]
    u64 *sN = sM + (size_t)np * W;        // [np + 1][W]
    for (int t = threadIdx.x; t < np * W; t += kIT) sM[t] = M[t];
    for (int t = threadIdx.x; t < (np + 1) * W; t += kIT) sN[t] = NEG[t];
    const int n = blockIdx.x * kIT + threadIdx.x;
    const u64 *yp = y + (size_t)blockIdx.y * np * N + n;
    __syncthreads();
    griddep_wait();
    // columns in passes of CW (one pass for W <= 24): fewer live accumulators;
    // the high words of a pass's last column seed the next pass's first one
    constexpr int CW = W > 24 ? (W + 1) / 2 : W;
    constexpr int NPASS = (W + CW - 1) / CW;
    u64 *o = out + (size_t)blockIdx.y * ostride * N + n;
    const u64 *dp = KS ? d + (size_t)blockIdx.y * ostride * N + n : nullptr;
    const int q0 = s >> 6, r = s & 63;
    u64 carry = 0, prev = 0, dc = 0, ov_lo = 0;
    uint32_t ov_hi = 0;
    int u = 0;
#pragma unroll
    for (int ps = 0; ps < NPASS; ps++) {
        const int w0 = ps * CW;
        u64 lo[CW + 1];
        uint32_t hi[CW + 1];  // carries out of the low words: at most 2 np per column
#pragma unroll
        for (int w = 0; w <= CW; w++) {
            lo[w] = 0;
            hi[w] = 0;
        }
        lo[0] = ov_lo;
        hi[0] = ov_hi;
        double f = 0;
        u64 ynext = yp[0];
        for (int i = 0; i < np; i++) {
            const u64 a = ynext;
            if (i + 1 < np) ynext = yp[(size_t)(i + 1) * N];
            if (ps == 0) f = fma((double)a, inv[i], f);
            const u64 *m = sM + (size_t)i * W + w0;
#pragma unroll
            for (int w = 0; w < CW; w++) {
                if (w0 + w < W) {
                    const u64 mw = m[w];
                    const u64 pl = a * mw, ph = __umul64hi(a, mw);
                    lo[w] += pl;
                    hi[w] += lo[w] < pl ? 1u : 0u;
                    lo[w + 1] += ph;
                    hi[w + 1] += lo[w + 1] < ph ? 1u : 0u;
                }
            }
        }
        if (ps == 0) u = (int)llrint(f);
        ov_lo = lo[CW];
        ov_hi = hi[CW];
        const u64 *neg = sN + (size_t)u * W;
#pragma unroll
        for (int k = 0; k < CW; k++) {
            const int w = w0 + k;
            if (w >= W) break;
            u64 col = lo[k] + carry;
            u64 c = (u64)hi[k] + (col < carry ? 1ull : 0ull);
            const u64 ng = neg[w];
            col += ng;
            c += col < ng ? 1ull : 0ull;
            carry = c;
            if (!KS) {
                if (w < wo) {
                    u64 v = col;
                    if (w == wo - 1 && (kout & 63)) v &= (1ull << (kout & 63)) - 1;
                    o[(size_t)w * N] = v;
                }
            } else {
                // output word j = bits [s + 64 j, s + 64 j + 64) of T: columns q0 + j and q0 + j + 1
                const int j = w - q0 - 1;
                if (j >= 0 && j < wo) {
                    const u64 v = r ? (prev >> r) | (col << (64 - r)) : prev;
                    const u64 dv = dp[(size_t)j * N];
                    u64 sum = v + dv;
                    const u64 c1 = sum < v ? 1ull : 0ull;
                    sum += dc;
                    dc = c1 + (sum < dc ? 1ull : 0ull);
                    if (j == wo - 1 && (kout & 63)) sum &= (1ull << (kout & 63)) - 1;
                    o[(size_t)j * N] = sum;
                }
                prev = col;
            }
        }
    }
}

// Rescale by 2^s with rounding: out = floor((a + 2^(s-1)) / 2^s) mod 2^kout.
// grid: x over N / kT, y over the two halves.
__global__ void __launch_bounds__(kT)
k_nr_rescale(const u64 *__restrict__ in, int wi, u64 *__restrict__ out, int wo, int kout, int s, int N)
{
    const int n = blockIdx.x * kT + threadIdx.x;
    const u64 *a = in + (size_t)blockIdx.y * wi * N + n;
    u64 *o = out + (size_t)blockIdx.y * wo * N + n;
    griddep_wait();
    const int q0 = s >> 6, r = s & 63;
    // add 2^(s-1) and shift right by s, word by word
    u64 carry = 0, prev = 0;
    for (int w = 0; w <= wi; w++) {
        u64 x = w < wi ? a[(size_t)w * N] : 0;
        const u64 add = (w == ((s - 1) >> 6)) ? (1ull << ((s - 1) & 63)) : 0;
        u64 t = x + add;
        u64 c = t < x ? 1ull : 0ull;
        t += carry;
        c += t < carry ? 1ull : 0ull;
        carry = c;
        const int j = w - q0 - 1;
        if (j >= 0 && j < wo) {
            u64 v = r ? (prev >> r) | (t << (64 - r)) : prev;
            if (j == wo - 1 && (kout & 63)) v &= (1ull << (kout & 63)) - 1;
            o[(size_t)j * N] = v;
        }
        prev = t;
    }
    // the last output word may need the column past the input
    const int j = wi - q0;
    if (j >= 0 && j < wo) {
        u64 v = r ? (prev >> r) | (carry << (64 - r)) : prev;
        if (j == wo - 1 && (kout & 63)) v &= (1ull << (kout & 63)) - 1;
        o[(size_t)j * N] = v;
    }
}

int nwords(int k) { return (k + 63) / 64; }

// ---- host-side multiword helpers for the plan's tables ----------------------
typedef std::vector<u64> MW;
void mw_mul_small(MW &a, u64 v)
{
    unsigned __int128 c = 0;
    for (auto &x : a) {
        c += (unsigned __int128)x * v;
        x = (u64)c;
        c >>= 64;
    }
}
void mw_add(MW &a, const MW &b)
{
    unsigned __int128 c = 0;
    for (size_t i = 0; i < a.size(); i++) {
        c += (unsigned __int128)a[i] + (i < b.size() ? b[i] : 0);
        a[i] = (u64)c;
        c >>= 64;
    }
}
u64 mw_mod(const MW &a, u64 p)
{
    unsigned __int128 r = 0;
    for (size_t i = a.size(); i-- > 0;) r = ((r << 64) | a[i]) % p;
    return (u64)r;
}
u64 powmod(u64 b, u64 e, u64 m)
{
    u64 r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = (u64)((unsigned __int128)r * b % m);
        b = (u64)((unsigned __int128)b * b % m);
        e >>= 1;
    }
    return r;
}
u64 invmod(u64 a, u64 p) { return powmod(a, p - 2, p); }
u64 shoup_c(u64 w, u64 p) { return (u64)(((unsigned __int128)w << 64) / p); }

// Phat_i mod 2^(64 W) for the first np primes, P mod 2^(64 W), Phat_i^-1 mod p_i
void crt_tables(const he_ctx *c, int np, int W, std::vector<u64> &M, std::vector<u64> &P, std::vector<u64> &phinv)
{
    const int len = np + 2;
    M.assign((size_t)np * W, 0);
    P.assign(W, 0);
    phinv.assign(np, 0);
    MW full(len, 0);
    full[0] = 1;
    for (int i = 0; i < np; i++) mw_mul_small(full, c->ext[c->K + i]);
    for (int w = 0; w < W && w < len; w++) P[w] = full[w];
    for (int i = 0; i < np; i++) {
        MW h(len, 0);
        h[0] = 1;
        for (int j = 0; j < np; j++)
            if (j != i) mw_mul_small(h, c->ext[c->K + j]);
        for (int w = 0; w < W && w < len; w++) M[(size_t)i * W + w] = h[w];
        phinv[i] = invmod(mw_mod(h, c->ext[c->K + i]), c->ext[c->K + i]);
    }
}

// (2^(64 W) - u P + add) mod 2^(64 W) for u = 0..np
std::vector<u64> neg_rows(const std::vector<u64> &P, int np, int W, int add_bit)
{
    std::vector<u64> out((size_t)(np + 1) * W, 0);
    for (int u = 0; u <= np; u++) {
        MW uP(W + 1, 0);
        for (int w = 0; w < W; w++) uP[w] = P[w];
        uP[W] = 0;
        mw_mul_small(uP, (u64)u);
        MW v(W, 0);  // 0 - uP mod 2^(64W)
        unsigned __int128 borrow = 0;
        for (int w = 0; w < W; w++) {
            unsigned __int128 t = (unsigned __int128)0 - uP[w] - borrow;
            v[w] = (u64)t;
            borrow = (t >> 64) ? 1 : 0;
        }
        if (add_bit >= 0) {
            MW a(W, 0);
            if (add_bit / 64 < W) a[add_bit / 64] = 1ull << (add_bit & 63);
            mw_add(v, a);
        }
        for (int w = 0; w < W; w++) out[(size_t)u * W + w] = v[w];
    }
    return out;
}

template <int WI>
void launch_crt(const he_nr_plan *pl, const u64 *in, int wi, int polys, u64 *out, int np, cudaStream_t st)
{
    const he_ctx *c = pl->c;
    dim3 g((unsigned)(c->N / kT), (unsigned)polys, (unsigned)((np + kCP - 1) / kCP));
    launch_k(c->pdl, k_nr_crt<WI>, g, dim3(kT), 0, st, in, wi, (size_t)wi * c->N, out, np, pl->crt, pl->chunks_evk,
             (const DevPrime *)c->d_primes, c->K, c->N);
}

template <int W, bool KS>
cudaError_t launch_icrt(const he_nr_plan *pl, const u64 *y, int np, const u64 *M, const u64 *NEG, const double *inv,
                        u64 *out, int ostride, int wo, int kout, const u64 *d, int s, int polys, cudaStream_t st)
{
    const he_ctx *c = pl->c;
    const size_t smem = sizeof(u64) * ((size_t)np * W + (size_t)(np + 1) * W);
    auto kern = k_nr_icrt<W, KS>;
    static bool configured = false;
    if (!configured) {
        const size_t most = sizeof(u64) * ((size_t)kMaxNp * W + (size_t)(kMaxNp + 1) * W);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 g((unsigned)(c->N / kIT), (unsigned)polys);
    launch_k(c->pdl, kern, g, dim3(kIT), smem, st, y, np, M, NEG, inv, out, ostride, wo, kout, d, s, c->N);
    return cudaGetLastError();
}

}  // namespace

}  // namespace he

using namespace he;

namespace {

// Supported: log Q with nwords(logQ) <= 19 and nwords(2 logQ) <= 38, the
// template widths of the kernels below.
constexpr int kW1 = 19, kW2 = 38;

size_t ws_words(const he_nr_plan *pl)
{
    const size_t N = (size_t)pl->c->N;
    return (size_t)4 * pl->np1 * N + (size_t)3 * pl->W1 * N + (size_t)2 * pl->np2 * N;
}

int dev_try(cudaError_t e) { return e == cudaSuccess ? HE_OK : HE_ECUDA; }

}  // namespace

extern "C" {

int he_nr_plan_create(he_ctx *c, int logQ, int logp, he_nr_plan **out)
{
    if (!c || !c->device || !out) return HE_EINVAL;
    if (logQ < 64 || nwords(logQ) > kW1 || nwords(2 * logQ) > kW2 || logp < 1 || logp >= logQ) return HE_EINVAL;
    // primes: the fewest leading context primes whose product exceeds
    // 2^(2 logQ + logN + 2) (region 1) and 2^(3 logQ + logN + 2) (region 2)
    auto count = [&](double bits) {
        double tot = 0;
        for (int i = 0; i < c->L; i++) {
            tot += std::log2((double)c->ext[c->K + i]);
            if (tot > bits) return i + 1;
        }
        return -1;
    };
    const int np1 = count(2.0 * logQ + c->logN + 2), np2 = count(3.0 * logQ + c->logN + 2);
    if (np1 < 0 || np2 < 0 || np2 > kMaxNp) return HE_EINVAL;
    for (int i = 0; i < np2; i++)
        if (c->ext[c->K + i] >= (1ull << 57) || c->ext[c->K + i] < (1ull << 40)) return HE_EINVAL;
    he_nr_plan *pl = new (std::nothrow) he_nr_plan();
    if (!pl) return HE_ENOMEM;
    pl->c = c;
    pl->logQ = logQ;
    pl->logp = logp;
    pl->np1 = np1;
    pl->np2 = np2;
    pl->W1 = kW1;
    pl->W2 = kW2;
    pl->chunks_ct = (64 * kW1 + 27) / 28;
    pl->chunks_evk = (64 * kW2 + 27) / 28;
    const int N = c->N, K = c->K;
    // host tables
    std::vector<u64> crt((size_t)np2 * pl->chunks_evk);
    for (int i = 0; i < np2; i++) {
        const u64 p = c->ext[K + i];
        for (int k = 0; k < pl->chunks_evk; k++) {
            const u64 v = powmod(2, 28ull * (u64)k, p);
            crt[(size_t)i * pl->chunks_evk + k] = (v & 0xFFFFFFFull) | ((v >> 28) << 32);
        }
    }
    std::vector<u64> M1, P1, phinv1, M2, P2, phinv2;
    crt_tables(c, np1, kW1, M1, P1, phinv1);
    crt_tables(c, np2, kW2, M2, P2, phinv2);
    std::vector<u64> neg1 = neg_rows(P1, np1, kW1, -1), neg2 = neg_rows(P2, np2, kW2, logQ - 1);
    std::vector<double> inv1(np1), inv2(np2);
    for (int i = 0; i < np1; i++) inv1[i] = 1.0 / (double)c->ext[K + i];
    for (int i = 0; i < np2; i++) inv2[i] = 1.0 / (double)c->ext[K + i];
    // NTT job lists (offsets in limbs from the workspace, or from the prepared key)
    const unsigned d_limbs = (unsigned)(3 * kW1);  // the d0, d1, d2 words, in units of N words
    const unsigned r2 = (unsigned)(4 * np1) + d_limbs;
    std::vector<NttJob> F1, I1, F2, I2, Fe;
    auto job = [&](unsigned src, unsigned dst, int i, u64 sc, u64 scs) {
        NttJob j;
        memset(&j, 0, sizeof(j));
        j.src = src;
        j.dst = dst;
        j.prime = (unsigned)(K + i);
        j.scale = sc;
        j.scale_sh = scs;
        return j;
    };
    for (int t = 0; t < 4; t++)
        for (int i = 0; i < np1; i++) F1.push_back(job(t * np1 + i, t * np1 + i, i, 0, 0));
    for (int t = 0; t < 3; t++)
        for (int i = 0; i < np1; i++) {
            const u64 p = c->ext[K + i];
            const u64 sc = (u64)((unsigned __int128)c->ninv[K + i] * phinv1[i] % p);
            I1.push_back(job(t * np1 + i, t * np1 + i, i, sc, shoup_c(sc, p)));
        }
    for (int i = 0; i < np2; i++) F2.push_back(job(r2 + i, r2 + i, i, 0, 0));
    for (int t = 0; t < 2; t++)
        for (int i = 0; i < np2; i++) {
            const u64 p = c->ext[K + i];
            const u64 sc = (u64)((unsigned __int128)c->ninv[K + i] * phinv2[i] % p);
            I2.push_back(job(r2 + t * np2 + i, r2 + t * np2 + i, i, sc, shoup_c(sc, p)));
        }
    for (int t = 0; t < 2; t++)
        for (int i = 0; i < np2; i++) Fe.push_back(job(t * np2 + i, t * np2 + i, i, 0, 0));
    std::vector<NttGroup> gF1 = group_jobs(F1), gI1 = group_jobs(I1), gF2 = group_jobs(F2), gI2 = group_jobs(I2),
                          gFe = group_jobs(Fe);
    // one device allocation for everything
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off += (b + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_crt = take(crt.size() * 8), o_m1 = take(M1.size() * 8), o_n1 = take(neg1.size() * 8),
                 o_i1 = take(inv1.size() * 8), o_m2 = take(M2.size() * 8), o_n2 = take(neg2.size() * 8),
                 o_i2 = take(inv2.size() * 8), o_g1 = take(gF1.size() * sizeof(NttGroup)),
                 o_g2 = take(gI1.size() * sizeof(NttGroup)), o_g3 = take(gF2.size() * sizeof(NttGroup)),
                 o_g4 = take(gI2.size() * sizeof(NttGroup)), o_g5 = take(gFe.size() * sizeof(NttGroup));
    if (cudaMalloc(&pl->dev, off) != cudaSuccess) {
        delete pl;
        return HE_ECUDA;
    }
    std::vector<unsigned char> img(off, 0);
    auto put = [&](size_t o, const void *p, size_t b) { memcpy(img.data() + o, p, b); };
    put(o_crt, crt.data(), crt.size() * 8);
    put(o_m1, M1.data(), M1.size() * 8);
    put(o_n1, neg1.data(), neg1.size() * 8);
    put(o_i1, inv1.data(), inv1.size() * 8);
    put(o_m2, M2.data(), M2.size() * 8);
    put(o_n2, neg2.data(), neg2.size() * 8);
    put(o_i2, inv2.data(), inv2.size() * 8);
    put(o_g1, gF1.data(), gF1.size() * sizeof(NttGroup));
    put(o_g2, gI1.data(), gI1.size() * sizeof(NttGroup));
    put(o_g3, gF2.data(), gF2.size() * sizeof(NttGroup));
    put(o_g4, gI2.data(), gI2.size() * sizeof(NttGroup));
    put(o_g5, gFe.data(), gFe.size() * sizeof(NttGroup));
    if (cudaMemcpy(pl->dev, img.data(), off, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(pl->dev);
        delete pl;
        return HE_ECUDA;
    }
    char *b = (char *)pl->dev;
    pl->crt = (const u64 *)(b + o_crt);
    pl->m1 = (const u64 *)(b + o_m1);
    pl->neg1 = (const u64 *)(b + o_n1);
    pl->inv1 = (const double *)(b + o_i1);
    pl->m2 = (const u64 *)(b + o_m2);
    pl->neg2 = (const u64 *)(b + o_n2);
    pl->inv2 = (const double *)(b + o_i2);
    pl->gF1 = (const NttGroup *)(b + o_g1);
    pl->gI1 = (const NttGroup *)(b + o_g2);
    pl->gF2 = (const NttGroup *)(b + o_g3);
    pl->gI2 = (const NttGroup *)(b + o_g4);
    pl->gFe = (const NttGroup *)(b + o_g5);
    pl->nF1 = (int)gF1.size();
    pl->nI1 = (int)gI1.size();
    pl->nF2 = (int)gF2.size();
    pl->nI2 = (int)gI2.size();
    pl->nFe = (int)gFe.size();
    (void)N;
    *out = pl;
    return HE_OK;
}

int he_nr_plan_destroy(he_nr_plan *pl)
{
    if (!pl) return HE_EINVAL;
    if (pl->dev) cudaFree(pl->dev);
    delete pl;
    return HE_OK;
}

int he_nr_plan_info(const he_nr_plan *pl, int *np1, int *np2)
{
    if (!pl) return HE_EINVAL;
    if (np1) *np1 = pl->np1;
    if (np2) *np2 = pl->np2;
    return HE_OK;
}

size_t he_nr_workspace_bytes(const he_nr_plan *pl) { return pl ? ws_words(pl) * sizeof(u64) : 0; }

size_t he_nr_evk_bytes(const he_nr_plan *pl) { return pl ? (size_t)2 * pl->np2 * pl->c->N * sizeof(u64) : 0; }

int he_nr_evk_prepare(he_nr_plan *pl, const uint64_t *evk, uint64_t *prep, void *stream)
{
    if (!pl || !evk || !prep) return HE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    launch_crt<kW2>(pl, evk, nwords(2 * pl->logQ), 2, prep, pl->np2, st);
    if (cudaGetLastError() != cudaSuccess) return HE_ECUDA;
    return dev_try(launch_ntt(pl->c, prep, pl->gFe, pl->nFe, false, st, "nr_evk"));
}

int he_nr_mul(he_nr_plan *pl, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *prep, int logq,
              uint64_t *out, void *ws, size_t ws_bytes, void *stream)
{
    if (!pl || !ct1 || !ct2 || !prep || !out || !ws) return HE_EINVAL;
    if (logq < pl->logp + 1 || logq > pl->logQ) return HE_ELEVEL;
    if (ws_bytes < ws_words(pl) * sizeof(u64)) return HE_ENOMEM;
    const he_ctx *c = pl->c;
    he_ctx *cm = pl->c;
    const size_t N = (size_t)c->N;
    const int wq = nwords(logq), np1 = pl->np1, np2 = pl->np2;
    cudaStream_t st = (cudaStream_t)stream;
    u64 *w = (u64 *)ws;
    u64 *R1 = w, *D = w + (size_t)4 * np1 * N, *R2 = D + (size_t)3 * kW1 * N;
    prof_mark(c, st, "");
    // region 1: CRT of a1, b1, a2, b2 (ct = [b | a], word-major)
    launch_crt<kW1>(pl, ct1 + (size_t)wq * N, wq, 1, R1, np1, st);
    launch_crt<kW1>(pl, ct1, wq, 1, R1 + (size_t)np1 * N, np1, st);
    launch_crt<kW1>(pl, ct2 + (size_t)wq * N, wq, 1, R1 + (size_t)2 * np1 * N, np1, st);
    launch_crt<kW1>(pl, ct2, wq, 1, R1 + (size_t)3 * np1 * N, np1, st);
    if (cudaGetLastError() != cudaSuccess) return HE_ECUDA;
    prof_mark(c, st, "nr_crt1");
    if (launch_ntt(cm, w, pl->gF1, pl->nF1, false, st, "nr_ntt1") != cudaSuccess) return HE_ECUDA;
    launch_k(c->pdl, k_nr_tensor, dim3((unsigned)(N / 2 / kT), (unsigned)np1), dim3(kT), 0, st, R1, np1,
             (const DevPrime *)c->d_primes, c->K, c->N);
    if (cudaGetLastError() != cudaSuccess) return HE_ECUDA;
    prof_mark(c, st, "nr_tensor");
    if (launch_ntt(cm, w, pl->gI1, pl->nI1, true, st, "nr_intt1") != cudaSuccess) return HE_ECUDA;
    // d0, d1, d2 mod q (word-major, wq words each, stride kW1 words)
    if (launch_icrt<kW1, false>(pl, R1, np1, pl->m1, pl->neg1, pl->inv1, D, kW1, wq, logq, nullptr, 0, 3, st) !=
        cudaSuccess)
        return HE_ECUDA;
    prof_mark(c, st, "nr_icrt1");
    // region 2: CRT of d2, NTT, products with the prepared key, iNTT, iCRT + shift + add
    launch_crt<kW1>(pl, D + (size_t)2 * kW1 * N, wq, 1, R2, np2, st);
    if (cudaGetLastError() != cudaSuccess) return HE_ECUDA;
    prof_mark(c, st, "nr_crt2");
    if (launch_ntt(cm, w, pl->gF2, pl->nF2, false, st, "nr_ntt2") != cudaSuccess) return HE_ECUDA;
    launch_k(c->pdl, k_nr_ks_mult, dim3((unsigned)(N / 2 / kT), (unsigned)np2), dim3(kT), 0, st, R2, prep, np2,
             (const DevPrime *)c->d_primes, c->K, c->N);
    if (cudaGetLastError() != cudaSuccess) return HE_ECUDA;
    prof_mark(c, st, "nr_ks_mult");
    if (launch_ntt(cm, w, pl->gI2, pl->nI2, true, st, "nr_intt2") != cudaSuccess) return HE_ECUDA;
    // out[h] = d_h + round(KS_h / Q) mod q; the d's sit kW1 words apart, out wq words apart
    for (int h = 0; h < 2; h++)
        if (launch_icrt<kW2, true>(pl, R2 + (size_t)h * np2 * N, np2, pl->m2, pl->neg2, pl->inv2,
                                   out + (size_t)h * wq * N, 0, wq, logq, D + (size_t)h * kW1 * N, pl->logQ, 1, st) !=
            cudaSuccess)
            return HE_ECUDA;
    prof_mark(c, st, "nr_icrt2");
    return HE_OK;
}

int he_nr_rescale(he_nr_plan *pl, const uint64_t *ct, int logq, uint64_t *out, void *stream)
{
    if (!pl || !ct || !out) return HE_EINVAL;
    if (logq <= pl->logp || logq > pl->logQ) return HE_ELEVEL;
    const he_ctx *c = pl->c;
    const int wi = nwords(logq), wo = nwords(logq - pl->logp);
    launch_k(c->pdl, k_nr_rescale, dim3((unsigned)(c->N / kT), 2u), dim3(kT), 0, (cudaStream_t)stream, ct, wi, out,
             wo, logq - pl->logp, pl->logp, c->N);
    return dev_try(cudaGetLastError());
}

}  // extern "C"
