// keyswitch.cu -- element-wise and base-conversion kernels of HE Mul on sm_103a.
//
//  k_tensor        Region 1 of Fig. 2 in RNS form (congruence relation,
//                  Sec. 3.3): d0 = b1 b2, d1 = a1 b2 + a2 b1, d2 = a1 a2 mod q_i.
//  k_modup         full-RNS mod up (Sec. 7, Table 11): the iCRT-then-CRT
//                  shape of Algo 5 / Algo 1 as a fast base conversion
//                  U_j[t] = sum_{i in I_j} y_i [Qhat_{j,i}]_t mod t, with the
//                  y_i = x_i Qhat^-1 factor already applied by the iNTT.
//                  Lazy accumulation (the paper's delayed-modulo idea for
//                  CRT, Sec. 5.3): operands split at bit 28, three 32x32->64
//                  multiply-adds per term (Karatsuba), one Barrett reduction
//                  per output.
//  k_inner_product Region 2 of Fig. 2: KS_{b,a}[t] = sum_j U_j[t] evk_j.{b,a}[t].
//  k_moddown_conv  mod down (Sec. 7): conv_i = sum_k y_k [Phat_k]_{q_i} mod q_i;
//                  the fused variant uses constants [Phat_k P^-1]_{q_i}, giving
//                  conv_i P^-1 directly, and folds in the rescale residue.
//  k_combine_plain the final additions (Fig. 2) after a plain ModDown; with
//                  rescale, the same combine runs in the last NTT pass of the
//                  ModDown limbs (ntt.cu).
//
// Every kernel handles two consecutive coefficients per thread with 16-byte
// loads and stores; the limb-major layouts keep all accesses coalesced.  A
// launch serves one HE Mul or a batch of them (grid.z = job), each job
// bringing its own operands, workspace and level (JobRef); blocks beyond a
// job's level exit at once.
#include <algorithm>
#include <cstring>

#include "he_internal.h"
#include "modarith.cuh"

namespace he {

namespace {

constexpr int kThreads = 256;
// Base conversions: two targets per loop trip, so one target's reduction
// overlaps the next target's multiply-adds.
constexpr int kConvUnroll = 2;

__device__ __forceinline__ ulonglong2 ld2(const u64 *p) { return *reinterpret_cast<const ulonglong2 *>(p); }
__device__ __forceinline__ void st2(u64 *p, u64 x, u64 y) { *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(x, y); }

__device__ __forceinline__ BatchItem job_of(const JobRef &R, int z) { return R.items ? R.items[z] : R.one; }

// grid: x over N/2/kThreads, y over limbs (up to the largest level), z over jobs
__global__ void __launch_bounds__(kThreads)
k_tensor(const JobRef R, const DevPrime *__restrict__ primes, const DevLevel *__restrict__ lv_arr, int K, int N)
{
    const BatchItem it = job_of(R, blockIdx.z);
    const int l = it.level, i = blockIdx.y;
    if (i >= l) return idle_exit();
    const DevLevel &lv = lv_arr[l];
    const size_t n = 2 * ((size_t)blockIdx.x * kThreads + threadIdx.x);
    const DevPrime pr = primes[K + i];
    const size_t ob = (size_t)i * N + n, oa = ((size_t)l + i) * N + n;
    griddep_wait(R.trigger);
    const u64 pol = l2_policy_stream();  // the inputs are read once
    const ulonglong2 b1 = ld2_hint(it.ct1 + ob, pol), a1 = ld2_hint(it.ct1 + oa, pol),
                     b2 = ld2_hint(it.ct2 + ob, pol), a2 = ld2_hint(it.ct2 + oa, pol);
    u64 *d0 = it.ws + (size_t)lv.o_d0 * N, *d1 = it.ws + (size_t)lv.o_d1 * N, *d2 = it.ws + (size_t)lv.o_d2 * N;
    st2(d0 + (size_t)i * N + n, mul_mod(b1.x, b2.x, pr.q, pr.mu, pr.s), mul_mod(b1.y, b2.y, pr.q, pr.mu, pr.s));
    U128 x = mul_wide(a1.x, b2.x), y = mul_wide(a1.y, b2.y);
    mac(x, a2.x, b1.x);
    mac(y, a2.y, b1.y);
    st2(d1 + (size_t)i * N + n, barrett128(x, pr.q, pr.mu, pr.s), barrett128(y, pr.q, pr.mu, pr.s));
    st2(d2 + (size_t)i * N + n, mul_mod(a1.x, a2.x, pr.q, pr.mu, pr.s), mul_mod(a1.y, a2.y, pr.q, pr.mu, pr.s));
}

// grid: x over N/2/kThreads, y over (digit, chunk of CH targets),
// z over jobs.  Input: the scaled iNTT of d2 (y region), output U: [beta][E][N],
// canonical with CANON, else lazily in [0, 3q) (the forward NTT that follows
// takes inputs below 4q; see acc3k_reduce_lazy).
// Target u of digit j (u < E - n_j) is ext limb u below the digit's own limbs,
// u + n_j above.  Digits are padded to A limbs with zero constants (the padding
// loads reread a real limb, whose value is multiplied by zero), so the MAC loop
// has no predicates; the chunk's constants and prime parameters sit in shared
// memory.
template <int A, int CH, bool CANON>
__global__ void __launch_bounds__(kThreads)
k_modup(const JobRef R, const DevLevel *__restrict__ lv_arr, const DevPrime *__restrict__ primes, int K, int N,
        int chunks)
{
    const BatchItem it = job_of(R, blockIdx.z);
    const DevLevel &lv = lv_arr[it.level];
    const int j = blockIdx.y / chunks;
    if (j >= lv.beta) return idle_exit();
    const int lo = lv.dig_lo[j], nj = lv.dig_n[j];
    const int E = lv.E;
    const int u0 = (blockIdx.y - j * chunks) * CH;
    const int cnt = min(CH, E - nj - u0);
    if (cnt <= 0) return idle_exit();
    __shared__ u64 sB[CH][A];
    __shared__ u64 sq[CH], smu[CH];
    __shared__ unsigned ss[CH];
    __shared__ int se[CH];
    const u64 *B = lv.modupB + (size_t)j * E * A;
    for (int t = threadIdx.x; t < cnt * A; t += kThreads) {
        const int u = u0 + t / A;
        const int e = u < K + lo ? u : u + nj;
        sB[t / A][t % A] = B[(size_t)e * A + t % A];
    }
    if (threadIdx.x < cnt) {
        const int u = u0 + threadIdx.x;
        const int e = u < K + lo ? u : u + nj;
        se[threadIdx.x] = e;
        sq[threadIdx.x] = primes[e].q;
        smu[threadIdx.x] = primes[e].mu;
        ss[threadIdx.x] = primes[e].s;
    }
    const u64 *y = it.ws + (size_t)lv.o_y * N;
    const size_t n = 2 * ((size_t)blockIdx.x * kThreads + threadIdx.x);
    griddep_wait(R.trigger);
    uint32_t x0[A], x1[A], z0[A], z1[A];
#pragma unroll
    for (int i = 0; i < A; i++) {
        const ulonglong2 v = ld2(y + (size_t)(lo + min(i, nj - 1)) * N + n);
        split28(v.x, x0[i], x1[i]);
        split28(v.y, z0[i], z1[i]);
    }
    __syncthreads();
    u64 *Uj = it.ws + ((size_t)lv.o_u + (size_t)j * E) * N;
#pragma unroll kConvUnroll
    for (int u = 0; u < cnt; u++) {
        Acc3 ax = {0, 0, 0}, ay = {0, 0, 0};
#pragma unroll
        for (int i = 0; i < A; i++) {
            const u64 c = sB[u][i];
            mac28k(ax, x0[i], x1[i], x0[i] + x1[i], c);
            mac28k(ay, z0[i], z1[i], z0[i] + z1[i], c);
        }
        const u64 q = sq[u], mu = smu[u];
        const unsigned sh = ss[u];
        if (CANON)
            st2(Uj + (size_t)se[u] * N + n, barrett128(acc3k_value(ax), q, mu, sh),
                barrett128(acc3k_value(ay), q, mu, sh));
        else
            st2(Uj + (size_t)se[u] * N + n, acc3k_reduce_lazy(ax, q, mu, sh), acc3k_reduce_lazy(ay, q, mu, sh));
    }
}

// grid: x over N/2/kThreads, y over ext limbs (up to K + lmax), z over jobs.
// Seeded evaluation key: a_j[e][n] = floor((w1 2^64 + w2) t / 2^128) with
// w1, w2 the SplitMix64 words 2(eN+n) and 2(eN+n)+1 of digit j's stream
// (state S_j): any element is computed on its own.
struct SeedStates {
    u64 s[kMaxDigits];
};

__device__ __forceinline__ u64 splitmix_word(u64 state, u64 i)
{
    u64 z = state + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ u64 seeded_a(u64 state, u64 idx, u64 t)
{
    const u64 w1 = splitmix_word(state, 2 * idx), w2 = splitmix_word(state, 2 * idx + 1);
    const u64 lo = w1 * t, hi = __umul64hi(w1, t), sum = lo + __umul64hi(w2, t);
    return hi + (sum < lo ? 1ull : 0ull);
}

// U: [beta][E][N] (own-digit rows read from d2), evk: [dnum][2][K+L][N]
// (SEEDED: [dnum][K+L][N], b halves only, a halves regenerated), KS: [2][E][N].
// The digit loop is unrolled to BM >= beta with guards, so every operand
// load of a thread is issued before the first product.
//
// Rows: the key-switch sum of ext limb e of one job.  Which limb a CTA takes
// (IpRows): every limb (grid.y over K + lmax); the special limbs and, for the
// rescaling tails, the last q limb (their iNTT comes next: grid.y = K + 1);
// or the q limbs (only the final combine reads them, so their sum can run
// beside the ModDown conversion: all l, or l - 1 for the rescaling tails).
enum IpRows { kIpAll = 0, kIpSpecialLast = 1, kIpSpecial = 2, kIpQButLast = 3, kIpQ = 4 };

__device__ __forceinline__ int ip_row(int rows, int y, int K, int l)
{
    switch (rows) {
    case kIpAll: return y < K + l ? y : -1;
    case kIpSpecialLast: return y < K ? y : y == K ? K + l - 1 : -1;
    case kIpSpecial: return y < K ? y : -1;
    case kIpQButLast: return y < l - 1 ? K + y : -1;
    default: return y < l ? K + y : -1;
    }
}

template <int BM, bool SEEDED>
__device__ __forceinline__ void ip_body(const JobRef &R, const BatchItem &it, const DevLevel &lv, int e,
                                        const u64 *__restrict__ evk, const DevPrime *__restrict__ primes, int K,
                                        int L, int N, const SeedStates &seeds)
{
    const int E = lv.E, EL = K + L, beta = lv.beta;
    const size_t n = 2 * ((size_t)blockIdx.x * kThreads + threadIdx.x);
    const DevPrime pr = primes[e];
    const u64 *U = it.ws + (size_t)lv.o_u * N, *d2 = it.ws + (size_t)lv.o_d2 * N;
    griddep_wait(R.trigger);
    // the key and the ModUp outputs are read once: evict-first keeps them from
    // displacing the twiddle tables in L2
    const u64 pol = l2_policy_stream();
    ulonglong2 u[BM], kb[BM], ka[BM];
#pragma unroll
    for (int j = 0; j < BM; j++) {
        if (j < beta) {
            const int lo = lv.dig_lo[j], nj = lv.dig_n[j];
            const bool own = e >= K && e - K >= lo && e - K < lo + nj;
            const u64 *up = own ? d2 + (size_t)(e - K) * N : U + ((size_t)j * E + e) * N;
            u[j] = own ? ld2(up + n) : ld2_hint(up + n, pol);
            if (SEEDED) {
                kb[j] = ld2_hint(evk + ((size_t)j * EL + e) * N + n, pol);
                const u64 idx = (u64)e * (u64)N + n;
                ka[j] = make_ulonglong2(seeded_a(seeds.s[j], idx, pr.q), seeded_a(seeds.s[j], idx + 1, pr.q));
            } else {
                kb[j] = ld2_hint(evk + ((size_t)(2 * j) * EL + e) * N + n, pol);
                ka[j] = ld2_hint(evk + ((size_t)(2 * j + 1) * EL + e) * N + n, pol);
            }
        }
    }
    U128 bx = {0, 0}, by = {0, 0}, ax = {0, 0}, ay = {0, 0};
#pragma unroll
    for (int j = 0; j < BM; j++) {
        if (j < beta) {
            mac(bx, u[j].x, kb[j].x);
            mac(by, u[j].y, kb[j].y);
            mac(ax, u[j].x, ka[j].x);
            mac(ay, u[j].y, ka[j].y);
        }
    }
    u64 *KS = it.ws + (size_t)lv.o_ks * N;
    st2(KS + (size_t)e * N + n, barrett128(bx, pr.q, pr.mu, pr.s), barrett128(by, pr.q, pr.mu, pr.s));
    st2(KS + ((size_t)E + e) * N + n, barrett128(ax, pr.q, pr.mu, pr.s), barrett128(ay, pr.q, pr.mu, pr.s));
}

// grid: x over N/2/kThreads, y over the rows selected (IpRows), z over jobs.
template <int BM, bool SEEDED>
__global__ void __launch_bounds__(kThreads)
k_inner_product(const JobRef R, const u64 *__restrict__ evk, const DevLevel *__restrict__ lv_arr,
                const DevPrime *__restrict__ primes, int K, int L, int N, const SeedStates seeds, int rows)
{
    const BatchItem it = job_of(R, blockIdx.z);
    const DevLevel &lv = lv_arr[it.level];
    const int e = ip_row(rows, blockIdx.y, K, it.level);
    if (e < 0) return idle_exit();
    ip_body<BM, SEEDED>(R, it, lv, e, evk, primes, K, L, N, seeds);
}

// Batched inner product with key words shared across jobs.  grid: x over
// N/2/kThreads, y over ext limbs (up to K + lmax), z over job groups
// (IpGroup: at most kIpJobsMax jobs, highest level first).  A CTA loads the
// key words of digits j < beta(group's highest level) at (e, n) once and
// forms KS of each job of its group that has limb e (the jobs whose level
// exceeds e - K: a prefix of the group).  Per job the words are those of
// k_inner_product: the key limbs and digits do not depend on the level (one
// full-level key serves every level), only U, d2, KS and beta do.  The jobs'
// row addresses are gathered into shared memory before the wait for the
// previous kernel (they come from host-written tables); after it, the U words
// of a chunk of jobs (four; two at four digits, for registers) are loaded
// together with the key words, so a thread has every load of a chunk in
// flight before its first product.

template <int BM, bool SEEDED>
__global__ void __launch_bounds__(kThreads)
k_inner_product_shared(const JobRef R, const IpGroup *__restrict__ groups, const int *count,
                       const u64 *__restrict__ evk, const DevLevel *__restrict__ lv_arr,
                       const DevPrime *__restrict__ primes, int K, int L, int N, const SeedStates seeds)
{
    __shared__ const u64 *s_row[kIpJobsMax][BM];  // U row of digit j at limb e (own digit: d2's row)
    __shared__ u64 *s_ks[kIpJobsMax][2];          // KS_b, KS_a rows of limb e
    __shared__ int s_beta[kIpJobsMax];            // the job's digits; 0: the job has no limb e
    const int gz = blockIdx.z;
    if (count && gz >= *count) return idle_exit();
    const IpGroup &gr = groups[gz];
    const int e = blockIdx.y;
    const DevLevel &lv0 = lv_arr[gr.level];
    if (gr.n < 1 || e >= lv0.E) return idle_exit();
    const int EL = K + L, beta0 = lv0.beta;
    if (threadIdx.x < kIpJobsMax) {
        const int g = threadIdx.x;
        int b = 0;
        if (g < gr.n) {
            const BatchItem it = job_item(R, gr.job[g]);
            if (e < K + it.level) {
                const DevLevel &lv = lv_arr[it.level];
                b = lv.beta;
                const u64 *U = it.ws + (size_t)lv.o_u * N, *d2 = it.ws + (size_t)lv.o_d2 * N;
                for (int j = 0; j < BM; j++) {
                    const int lo = lv.dig_lo[j], nj = lv.dig_n[j];
                    const bool own = j < b && e >= K && e - K >= lo && e - K < lo + nj;
                    s_row[g][j] = own ? d2 + (size_t)(e - K) * N : U + ((size_t)j * lv.E + e) * N;
                }
                u64 *KS = it.ws + (size_t)lv.o_ks * N;
                s_ks[g][0] = KS + (size_t)e * N;
                s_ks[g][1] = KS + ((size_t)lv.E + e) * N;
            }
        }
        s_beta[g] = b;
    }
    const size_t n = 2 * ((size_t)blockIdx.x * kThreads + threadIdx.x);
    const DevPrime pr = primes[e];
    __syncthreads();
    int njobs = 0;  // jobs sorted by level, highest first: those with limb e are a prefix
#pragma unroll
    for (int g = 0; g < kIpJobsMax; g++) njobs += s_beta[g] > 0 ? 1 : 0;
    griddep_wait(R.trigger);
    const u64 pol = l2_policy_stream();
    ulonglong2 kb[BM], ka[BM];
#pragma unroll
    for (int j = 0; j < BM; j++) {
        if (j < beta0) {
            if (SEEDED) {
                kb[j] = ld2_hint(evk + ((size_t)j * EL + e) * N + n, pol);
                const u64 idx = (u64)e * (u64)N + n;
                ka[j] = make_ulonglong2(seeded_a(seeds.s[j], idx, pr.q), seeded_a(seeds.s[j], idx + 1, pr.q));
            } else {
                kb[j] = ld2_hint(evk + ((size_t)(2 * j) * EL + e) * N + n, pol);
                ka[j] = ld2_hint(evk + ((size_t)(2 * j + 1) * EL + e) * N + n, pol);
            }
        }
    }
    constexpr int CJ = BM >= 4 ? 2 : 4;
    for (int c0 = 0; c0 < njobs; c0 += CJ) {
        ulonglong2 u[CJ][BM];
#pragma unroll
        for (int g = 0; g < CJ; g++) {
            const int gg = c0 + g;
            if (gg < njobs) {
#pragma unroll
                for (int j = 0; j < BM; j++)
                    if (j < s_beta[gg]) u[g][j] = ld2_hint(s_row[gg][j] + n, pol);
            }
        }
#pragma unroll
        for (int g = 0; g < CJ; g++) {
            const int gg = c0 + g;
            if (gg < njobs) {
                U128 bx = {0, 0}, by = {0, 0}, ax = {0, 0}, ay = {0, 0};
                const int b = s_beta[gg];
#pragma unroll
                for (int j = 0; j < BM; j++) {
                    if (j < b) {
                        mac(bx, u[g][j].x, kb[j].x);
                        mac(by, u[g][j].y, kb[j].y);
                        mac(ax, u[g][j].x, ka[j].x);
                        mac(ay, u[g][j].y, ka[j].y);
                    }
                }
                st2(s_ks[gg][0] + n, barrett128(bx, pr.q, pr.mu, pr.s), barrett128(by, pr.q, pr.mu, pr.s));
                st2(s_ks[gg][1] + n, barrett128(ax, pr.q, pr.mu, pr.s), barrett128(ay, pr.q, pr.mu, pr.s));
            }
        }
    }
}

// grid: x over N/2/kThreads, y over (h in {0,1}, chunk of kModdownChunk
// outputs), z over jobs.  ys: [2][K] coefficient form (already times
// Phat_k^-1).  PLAIN: z[h][i] = conv_i for i < l.
// FUSED: r = r0 + (r1 - conv_{l-1}) P^-1 mod q_{l-1} with r0 = iNTT(d_h)_{l-1},
// r1 = iNTT(KS_h)_{l-1}; z[h][i] = conv_i P^-1 + r mod q_i for i < l-1.
// PB rows are zero-padded to KM constants, so the MAC loop has no predicates.
constexpr int kModdownChunk = 8;

// LAZY: the conversion in [0, 3q) (acc3k_reduce_lazy), else canonical.
template <int KM, bool LAZY = false>
__device__ __forceinline__ void conv_one(const uint32_t *x0, const uint32_t *x1, const uint32_t *z0,
                                         const uint32_t *z1, const u64 *b, u64 q, u64 mu, unsigned sh, u64 &cx,
                                         u64 &cy)
{
    Acc3 ax = {0, 0, 0}, ay = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < KM; k++) {
        const u64 c = b[k];
        mac28k(ax, x0[k], x1[k], x0[k] + x1[k], c);
        mac28k(ay, z0[k], z1[k], z0[k] + z1[k], c);
    }
    if (LAZY) {
        cx = acc3k_reduce_lazy(ax, q, mu, sh);
        cy = acc3k_reduce_lazy(ay, q, mu, sh);
    } else {
        cx = barrett128(acc3k_value(ax), q, mu, sh);
        cy = barrett128(acc3k_value(ay), q, mu, sh);
    }
}

// MODE (TailMode): kTailPlain: z[h][i] = conv_i for i < l.  kTailRescale:
// z[h][i] = conv_i P^-1 + r (the fused ModDown + rescale above).
// kTailRescalePQ: one division by M = P q_{l-1} over the basis (p_0..p_{K-1},
// q_{l-1}): ys carry [Mhat_k^-1]_{p_k} (the special iNTT's scale), the last
// limb's term is y_last = x_last [P^-1]_{q_{l-1}} = r0 + r1 P^-1 mod q_{l-1}
// (x_last = P r0 + r1, the iNTT of P d_{l-1} + KS_{l-1}), and
// z[h][i] = sum_k y_k [Mhat_k P^-1]_{q_i} + y_last = conv_i P^-1 mod q_i with
// the per-level constants lv.pbpq: the combine pass then forms
// (P d + KS - NTT(conv)) / M exactly as for two floors.
template <int KM, int MODE>
__device__ __forceinline__ void moddown_body(const JobRef &R, const u64 *__restrict__ PB,
                                             const ulonglong2 *__restrict__ pinv, const DevLevel *__restrict__ lv_arr,
                                             const DevPrime *__restrict__ primes, int K, int N, int chunks, int y)
{
    constexpr bool FUSED = MODE == kTailRescale, PQ = MODE == kTailRescalePQ;
    const BatchItem it = job_of(R, blockIdx.z);
    const int l = it.level;
    const DevLevel &lv = lv_arr[l];
    const int h = y / chunks;
    const int nout = MODE != kTailPlain ? l - 1 : l;
    const int i0 = (y - h * chunks) * kModdownChunk;
    const int cnt = min(kModdownChunk, nout - i0);
    if (cnt <= 0) return idle_exit();
    const u64 *PBt = PQ ? lv.pbpq : PB;
    // rows 0..cnt-1: this chunk's outputs; row kModdownChunk: q_{l-1} (fused)
    __shared__ u64 sB[kModdownChunk + 1][KM];
    __shared__ u64 sq[kModdownChunk + 1], smu[kModdownChunk + 1];
    __shared__ unsigned ss[kModdownChunk + 1];
    __shared__ ulonglong2 spv[kModdownChunk + 1];
    for (int t = threadIdx.x; t < (kModdownChunk + 1) * KM; t += kThreads) {
        const int r = t / KM, k = t % KM;
        const int i = r < kModdownChunk ? i0 + r : l - 1;
        if (r < cnt || (FUSED && r == kModdownChunk)) sB[r][k] = PBt[(size_t)i * KM + k];
    }
    if (threadIdx.x <= kModdownChunk) {
        const int r = threadIdx.x;
        const int i = r < kModdownChunk ? i0 + r : l - 1;
        if (r < cnt || ((FUSED || PQ) && r == kModdownChunk)) {
            sq[r] = primes[K + i].q;
            smu[r] = primes[K + i].mu;
            ss[r] = primes[K + i].s;
            spv[r] = pinv[i];
        }
    }
    const u64 *ys = it.ws + (size_t)lv.o_ys * N, *rr = it.ws + (size_t)lv.o_r * N;
    u64 *z = it.ws + (size_t)lv.o_z * N;
    const size_t n = 2 * ((size_t)blockIdx.x * kThreads + threadIdx.x);
    griddep_wait(R.trigger);
    uint32_t x0[KM], x1[KM], z0[KM], z1[KM];
#pragma unroll
    for (int k = 0; k < KM; k++) {
        const ulonglong2 v = ld2(ys + ((size_t)h * K + min(k, K - 1)) * N + n);
        split28(v.x, x0[k], x1[k]);
        split28(v.y, z0[k], z1[k]);
    }
    __syncthreads();
    u64 rx = 0, ry = 0;
    if (FUSED) {
        // PB rows already carry the factor P^-1: the conversion yields
        // conv_{l-1} P^-1, and r = r0 + r1 P^-1 - conv_{l-1} P^-1
        const int r = kModdownChunk;
        const u64 q = sq[r];
        u64 cx, cy;
        conv_one<KM>(x0, x1, z0, z1, sB[r], q, smu[r], ss[r], cx, cy);
        const ulonglong2 r0 = ld2(rr + (size_t)h * N + n), r1 = ld2(rr + (size_t)(2 + h) * N + n);
        const ulonglong2 pv = spv[r];
        rx = add_mod(r0.x, sub_mod(shoup(r1.x, pv.x, pv.y, q), cx, q), q);
        ry = add_mod(r0.y, sub_mod(shoup(r1.y, pv.x, pv.y, q), cy, q), q);
    }
    if (PQ) {
        // y_last = r0 + r1 P^-1 mod q_{l-1}; no conversion row to q_{l-1}
        const int r = kModdownChunk;
        const u64 q = sq[r];
        const ulonglong2 r0 = ld2(rr + (size_t)h * N + n), r1 = ld2(rr + (size_t)(2 + h) * N + n);
        const ulonglong2 pv = spv[r];
        rx = add_mod(r0.x, shoup(r1.x, pv.x, pv.y, q), q);
        ry = add_mod(r0.y, shoup(r1.y, pv.x, pv.y, q), q);
    }
    // z feeds a forward NTT, which takes inputs below 4q: the conversion is
    // left lazily in [0, 3q) and r (or y_last, below q_{l-1} < q_i) added
    // without a reduction
#pragma unroll kConvUnroll
    for (int r = 0; r < cnt; r++) {
        const u64 q = sq[r];
        u64 cx, cy;
        conv_one<KM, true>(x0, x1, z0, z1, sB[r], q, smu[r], ss[r], cx, cy);
        if (FUSED || PQ) {
            cx += rx;
            cy += ry;
        }
        st2(z + ((size_t)h * nout + i0 + r) * N + n, cx, cy);
    }
}

template <int KM, int MODE>
__global__ void __launch_bounds__(kThreads, KM <= 8 ? 3 : 2)  // 85 / 128 registers
k_moddown_conv(const JobRef R, const u64 *__restrict__ PB, const ulonglong2 *__restrict__ pinv,
               const DevLevel *__restrict__ lv_arr, const DevPrime *__restrict__ primes, int K, int N, int chunks)
{
    moddown_body<KM, MODE>(R, PB, pinv, lv_arr, primes, K, N, chunks, blockIdx.y);
}

// The ModDown conversion and the key-switch sums of the q limbs in one
// launch: grid.y below 2 chunks runs the conversion (compute-bound), above it
// the sums of the q limbs (a stream of key and ModUp words), so the SMs run
// both kinds of CTA side by side.  The conversion reads only the special
// limbs' iNTT (and the rescale limbs), the q-limb sums only U, d2 and the
// key: the two parts touch disjoint data.
template <int KM, int MODE, int BM, bool SEEDED>
__global__ void __launch_bounds__(kThreads, KM <= 8 ? 3 : 2)
k_moddown_ipq(const JobRef R, const u64 *__restrict__ PB, const ulonglong2 *__restrict__ pinv,
              const DevLevel *__restrict__ lv_arr, const DevPrime *__restrict__ primes, int K, int N, int chunks,
              const u64 *__restrict__ evk, int L, const SeedStates seeds)
{
    const int y = blockIdx.y;
    if (y < 2 * chunks) {
        moddown_body<KM, MODE>(R, PB, pinv, lv_arr, primes, K, N, chunks, y);
        return;
    }
    const BatchItem it = job_of(R, blockIdx.z);
    const int e = ip_row(MODE == kTailPlain ? kIpQ : kIpQButLast, y - 2 * chunks, K, it.level);
    if (e < 0) return idle_exit();
    ip_body<BM, SEEDED>(R, it, lv_arr[it.level], e, evk, primes, K, L, N, seeds);
}

// grid: x over N/2/kThreads, y over limbs, z over 2 * jobs (h = z & 1).
// out[h][i] = d_h[i] + (KS_h[K+i] - C[h][i]) P^-1 mod q_i, i < l
__global__ void __launch_bounds__(kThreads)
k_combine_plain(const JobRef R, const ulonglong2 *__restrict__ pinv, const DevLevel *__restrict__ lv_arr,
                const DevPrime *__restrict__ primes, int K, int N)
{
    const BatchItem it = job_of(R, blockIdx.z >> 1);
    const int h = blockIdx.z & 1, l = it.level, i = blockIdx.y;
    if (i >= l) return idle_exit();
    const DevLevel &lv = lv_arr[l];
    const int E = K + l;
    const size_t n = 2 * ((size_t)blockIdx.x * kThreads + threadIdx.x);
    const DevPrime pr = primes[K + i];
    const ulonglong2 pv = pinv[i];
    const u64 *d = it.ws + (size_t)(h ? lv.o_d1 : lv.o_d0) * N;
    const u64 *KS = it.ws + (size_t)lv.o_ks * N, *C = it.ws + (size_t)lv.o_z * N;
    griddep_wait(R.trigger);
    const ulonglong2 dv = ld2(d + (size_t)i * N + n);
    const ulonglong2 ks = ld2(KS + ((size_t)h * E + K + i) * N + n);
    const ulonglong2 c = ld2(C + ((size_t)h * l + i) * N + n);
    const u64 x = add_mod(dv.x, shoup(sub_mod(ks.x, c.x, pr.q), pv.x, pv.y, pr.q), pr.q);
    const u64 y = add_mod(dv.y, shoup(sub_mod(ks.y, c.y, pr.q), pv.x, pv.y, pr.q), pr.q);
    st2(it.out + ((size_t)h * l + i) * N + n, x, y);
}

// Rescale on its own: out[h][i] = (c_h[i] - Z[h][i]) q_{l-1}^-1, i < l-1
__global__ void __launch_bounds__(kThreads)
k_rescale_combine(const u64 *__restrict__ ct, const u64 *__restrict__ Z, u64 *__restrict__ out,
                  const DevLevel *__restrict__ lv_arr, const DevPrime *__restrict__ primes, int K, int l, int N)
{
    const int i = blockIdx.y, h = blockIdx.z;
    const size_t n = 2 * ((size_t)blockIdx.x * kThreads + threadIdx.x);
    const DevPrime pr = primes[K + i];
    const ulonglong2 qv = lv_arr[l].qinv_last[i];
    griddep_wait();
    const ulonglong2 c = ld2(ct + ((size_t)h * l + i) * N + n);
    const ulonglong2 zz = ld2(Z + ((size_t)h * (l - 1) + i) * N + n);
    st2(out + ((size_t)h * (l - 1) + i) * N + n, shoup(sub_mod(c.x, zz.x, pr.q), qv.x, qv.y, pr.q),
        shoup(sub_mod(c.y, zz.y, pr.q), qv.x, qv.y, pr.q));
}

// Galois automorphism kappa_g in the NTT domain (bit-reversed evaluation
// order): entry i holds a(psi^(2 br(i) + 1)), so kappa_g(a) at entry i is
// a(psi^(g (2 br(i) + 1))), the entry j with 2 br(j) + 1 = g (2 br(i) + 1)
// mod 2N -- a gather, the same for every limb.  Writes the rotation's key
// switching inputs into the workspace: d0 = kappa(b), d1 = 0,
// d2 = -kappa(a) mod q_i.  grid: x over N/2/kThreads, y over limbs.
__global__ void __launch_bounds__(kThreads)
k_automorph(const u64 *__restrict__ ct, u64 *__restrict__ ws, const DevLevel *__restrict__ lv_arr,
            const DevPrime *__restrict__ primes, int K, int l, int N, int logN, unsigned long long g)
{
    const int i = blockIdx.y;
    const DevLevel &lv = lv_arr[l];
    const u64 q = primes[K + i].q;
    const unsigned n = 2 * (blockIdx.x * kThreads + threadIdx.x);
    const unsigned long long twoN = 2ull * (unsigned)N;
    const u64 *b = ct + (size_t)i * N, *a = ct + ((size_t)l + i) * N;
    unsigned src[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const unsigned br = __brev(n + k) >> (32 - logN);
        const unsigned long long e = (g * (2ull * br + 1)) % twoN;
        src[k] = __brev((unsigned)((e - 1) / 2)) >> (32 - logN);
    }
    griddep_wait();
    const u64 a0 = a[src[0]], a1 = a[src[1]];
    st2(ws + (size_t)lv.o_d0 * N + (size_t)i * N + n, b[src[0]], b[src[1]]);
    st2(ws + (size_t)lv.o_d1 * N + (size_t)i * N + n, 0, 0);
    st2(ws + (size_t)lv.o_d2 * N + (size_t)i * N + n, a0 ? q - a0 : 0, a1 ? q - a1 : 0);
}

// Element-wise ciphertext operations (HE Add of Sec. 3.2 and its relatives).
// OP 0: out = x + y (both halves); 1: out = x - y; 2: out = x * pt (both
// halves, pt [l][N]); 3: out.b = x.b + pt, out.a = x.a.  x, y, out:
// [2][l][N]; out may alias an input (each word is read, then written, by
// one thread).  grid: x over N/2/kThreads, y over limbs, z over the halves.
template <int OP>
__global__ void __launch_bounds__(kThreads)
k_elementwise(const u64 *x, const u64 *y, u64 *out, const DevPrime *__restrict__ primes, int K, int l, int N)
{
    const int i = blockIdx.y, h = blockIdx.z;
    const DevPrime pr = primes[K + i];
    const size_t n = 2 * ((size_t)blockIdx.x * kThreads + threadIdx.x);
    const size_t o = ((size_t)h * l + i) * N + n;
    griddep_wait();
    const ulonglong2 a = ld2(x + o);
    u64 r0, r1;
    if (OP == 0 || OP == 1) {
        const ulonglong2 b = ld2(y + o);
        r0 = OP == 0 ? add_mod(a.x, b.x, pr.q) : sub_mod(a.x, b.x, pr.q);
        r1 = OP == 0 ? add_mod(a.y, b.y, pr.q) : sub_mod(a.y, b.y, pr.q);
    } else if (OP == 2) {
        const ulonglong2 b = ld2(y + (size_t)i * N + n);
        r0 = mul_mod(a.x, b.x, pr.q, pr.mu, pr.s);
        r1 = mul_mod(a.y, b.y, pr.q, pr.mu, pr.s);
    } else {
        if (h == 0) {
            const ulonglong2 b = ld2(y + (size_t)i * N + n);
            r0 = add_mod(a.x, b.x, pr.q);
            r1 = add_mod(a.y, b.y, pr.q);
        } else {
            r0 = a.x;
            r1 = a.y;
        }
    }
    st2(out + o, r0, r1);
}

inline dim3 grid_x(int N) { return dim3((unsigned)(N / 2 / kThreads)); }

}  // namespace

cudaError_t run_tensor(const he_ctx *c, const JobRef &R, cudaStream_t st)
{
    dim3 g = grid_x(c->N);
    g.y = R.lmax;
    g.z = R.B;
    launch_k(c->pdl, k_tensor, g, dim3(kThreads), 0, st, R, c->d_primes, c->d_levels, c->K, c->N);
    return cudaGetLastError();
}

cudaError_t run_elementwise(const he_ctx *c, int op, const u64 *x, const u64 *y, u64 *out, int l, cudaStream_t st)
{
    dim3 grid = grid_x(c->N);
    grid.y = l;
    grid.z = 2;
    switch (op) {
    case 0: launch_k(c->pdl, k_elementwise<0>, grid, dim3(kThreads), 0, st, x, y, out, c->d_primes, c->K, l, c->N); break;
    case 1: launch_k(c->pdl, k_elementwise<1>, grid, dim3(kThreads), 0, st, x, y, out, c->d_primes, c->K, l, c->N); break;
    case 2: launch_k(c->pdl, k_elementwise<2>, grid, dim3(kThreads), 0, st, x, y, out, c->d_primes, c->K, l, c->N); break;
    default: launch_k(c->pdl, k_elementwise<3>, grid, dim3(kThreads), 0, st, x, y, out, c->d_primes, c->K, l, c->N); break;
    }
    return cudaGetLastError();
}

cudaError_t run_automorph(const he_ctx *c, const u64 *ct, u64 *ws, int l, u64 g, cudaStream_t st)
{
    dim3 grid = grid_x(c->N);
    grid.y = l;
    launch_k(c->pdl, k_automorph, grid, dim3(kThreads), 0, st, ct, ws, c->d_levels, c->d_primes, c->K, l, c->N, c->logN,
             (unsigned long long)g);
    return cudaGetLastError();
}

template <int CH, bool CANON>
cudaError_t launch_modup(const he_ctx *c, const JobRef &R, cudaStream_t st)
{
    // the most targets any digit of any level up to lmax has: K + (beta - 1) alpha
    const int beta = (R.lmax + c->alpha - 1) / c->alpha;
    const int chunks = (c->K + (beta - 1) * c->alpha + CH - 1) / CH;
    dim3 g = grid_x(c->N);
    g.y = beta * chunks;
    g.z = R.B;
    const int a = c->AP;
#define HE_MODUP(AA) \
    launch_k(c->pdl, k_modup<AA, CH, CANON>, g, dim3(kThreads), 0, st, R, c->d_levels, c->d_primes, c->K, c->N, chunks)
    if (a == 1) HE_MODUP(1);
    else if (a == 2) HE_MODUP(2);
    else if (a == 4) HE_MODUP(4);
    else if (a == 8) HE_MODUP(8);
    else if (a == 12) HE_MODUP(12);
    else HE_MODUP(16);
#undef HE_MODUP
    return cudaGetLastError();
}

cudaError_t run_modup(const he_ctx *c, const JobRef &R, cudaStream_t st, bool canonical)
{
    if (canonical) return launch_modup<8, true>(c, R, st);
    if (c->modup_chunk == 4) return launch_modup<4, false>(c, R, st);
    if (c->modup_chunk == 16) return launch_modup<16, false>(c, R, st);
    return launch_modup<8, false>(c, R, st);
}

SeedStates seed_states(const he_ctx *c, const u64 *evk, bool *seeded)
{
    SeedStates ss;
    memset(&ss, 0, sizeof(ss));
    *seeded = false;
    for (const auto &k : c->seeded)
        if (k.ptr == evk) {
            *seeded = true;
            memcpy(ss.s, k.state, sizeof(ss.s));
        }
    return ss;
}

cudaError_t run_inner_product(const he_ctx *c, const JobRef &R, const u64 *evk, cudaStream_t st, int rows)
{
    dim3 g = grid_x(c->N);
    g.y = rows == kIpAll ? c->K + R.lmax : rows == kIpSpecialLast ? c->K + 1 : rows == kIpSpecial ? c->K
        : rows == kIpQButLast ? R.lmax - 1 : R.lmax;
    g.z = R.B;
    const int bm = (c->L + c->alpha - 1) / c->alpha;  // the most digits any level has
    SeedStates ss;
    memset(&ss, 0, sizeof(ss));
    bool seeded = false;
    for (const auto &k : c->seeded)
        if (k.ptr == evk) {
            seeded = true;
            memcpy(ss.s, k.state, sizeof(ss.s));
        }
#define HE_IP(B)                                                                                                     \
    do {                                                                                                             \
        if (seeded)                                                                                                  \
            launch_k(c->pdl, k_inner_product<B, true>, g, dim3(kThreads), 0, st, R, evk, c->d_levels, c->d_primes,   \
                     c->K, c->L, c->N, ss, rows);                                                                    \
        else                                                                                                         \
            launch_k(c->pdl, k_inner_product<B, false>, g, dim3(kThreads), 0, st, R, evk, c->d_levels, c->d_primes,  \
                     c->K, c->L, c->N, ss, rows);                                                                    \
    } while (0)
    // three digits get their own width: 64 registers, four CTAs per SM
    // (the four-digit width takes 78 and fits three)
    if (bm <= 2) HE_IP(2);
    else if (bm == 3) HE_IP(3);
    else if (bm <= 4) HE_IP(4);
    else if (bm <= 8) HE_IP(8);
    else HE_IP(16);
#undef HE_IP
    return cudaGetLastError();
}

bool inner_product_shared_fits(const he_ctx *c) { return (c->L + c->alpha - 1) / c->alpha <= 4; }

cudaError_t run_inner_product_shared(const he_ctx *c, const JobRef &R, const IpGroup *groups, int ngroups,
                                     const int *dev_count, const u64 *evk, cudaStream_t st)
{
    if (!inner_product_shared_fits(c)) return cudaErrorInvalidValue;
    dim3 g = grid_x(c->N);
    g.y = c->K + R.lmax;
    g.z = ngroups;
    const int bm = (c->L + c->alpha - 1) / c->alpha;
    SeedStates ss;
    memset(&ss, 0, sizeof(ss));
    bool seeded = false;
    for (const auto &k : c->seeded)
        if (k.ptr == evk) {
            seeded = true;
            memcpy(ss.s, k.state, sizeof(ss.s));
        }
#define HE_IPS(B)                                                                                                  \
    do {                                                                                                           \
        if (seeded)                                                                                                \
            launch_k(c->pdl, k_inner_product_shared<B, true>, g, dim3(kThreads), 0, st, R, groups, dev_count, evk, \
                     c->d_levels, c->d_primes, c->K, c->L, c->N, ss);                                              \
        else                                                                                                       \
            launch_k(c->pdl, k_inner_product_shared<B, false>, g, dim3(kThreads), 0, st, R, groups, dev_count,     \
                     evk, c->d_levels, c->d_primes, c->K, c->L, c->N, ss);                                         \
    } while (0)
    if (bm <= 2) HE_IPS(2);
    else if (bm == 3) HE_IPS(3);
    else HE_IPS(4);
#undef HE_IPS
    return cudaGetLastError();
}

cudaError_t run_moddown_conv(const he_ctx *c, const JobRef &R, int mode, cudaStream_t st)
{
    const int chunks = (R.lmax + kModdownChunk - 1) / kModdownChunk;
    dim3 g = grid_x(c->N);
    g.y = 2 * chunks;
    g.z = R.B;
    const int K = c->K;
#define HE_MD(KK)                                                                                                   \
    do {                                                                                                            \
        if (mode == kTailRescale)                                                                                   \
            launch_k(c->pdl, k_moddown_conv<KK, kTailRescale>, g, dim3(kThreads), 0, st, R, c->d_PBP, c->d_pinv,    \
                     c->d_levels, c->d_primes, K, c->N, chunks);                                                    \
        else if (mode == kTailRescalePQ)                                                                            \
            launch_k(c->pdl, k_moddown_conv<KK, kTailRescalePQ>, g, dim3(kThreads), 0, st, R, c->d_PB, c->d_pinv,   \
                     c->d_levels, c->d_primes, K, c->N, chunks);                                                    \
        else                                                                                                        \
            launch_k(c->pdl, k_moddown_conv<KK, kTailPlain>, g, dim3(kThreads), 0, st, R, c->d_PB, c->d_pinv,       \
                     c->d_levels, c->d_primes, K, c->N, chunks);                                                    \
    } while (0)
    const int kp = c->KP;
    if (kp == 1) HE_MD(1);
    else if (kp == 2) HE_MD(2);
    else if (kp == 4) HE_MD(4);
    else if (kp == 8) HE_MD(8);
    else if (kp == 12) HE_MD(12);
    else HE_MD(16);
#undef HE_MD
    return cudaGetLastError();
}

bool moddown_ipq_fits(const he_ctx *c)
{
    return (c->L + c->alpha - 1) / c->alpha <= 4 && (c->KP == 1 || c->KP == 8 || c->KP == 12);
}

cudaError_t run_moddown_ipq(const he_ctx *c, const JobRef &R, int mode, const u64 *evk, cudaStream_t st)
{
    if (!moddown_ipq_fits(c)) return cudaErrorInvalidValue;
    const int chunks = (R.lmax + kModdownChunk - 1) / kModdownChunk;
    dim3 g = grid_x(c->N);
    g.y = 2 * chunks + (mode == kTailPlain ? R.lmax : R.lmax - 1);  // the q rows the final additions read
    g.z = R.B;
    const int K = c->K, bm = (c->L + c->alpha - 1) / c->alpha;
    bool seeded;
    const SeedStates ss = seed_states(c, evk, &seeded);
    const u64 *PB = mode == kTailRescale ? c->d_PBP : c->d_PB;
#define HE_MDQ(KK, MM, BB, SS)                                                                                       \
    launch_k(c->pdl, k_moddown_ipq<KK, MM, BB, SS>, g, dim3(kThreads), 0, st, R, PB, c->d_pinv, c->d_levels,         \
             c->d_primes, K, c->N, chunks, evk, c->L, ss)
#define HE_MDQ_B(KK, MM)                                                                                             \
    do {                                                                                                             \
        if (bm <= 2) { if (seeded) HE_MDQ(KK, MM, 2, true); else HE_MDQ(KK, MM, 2, false); }                         \
        else if (bm == 3) { if (seeded) HE_MDQ(KK, MM, 3, true); else HE_MDQ(KK, MM, 3, false); }                    \
        else { if (seeded) HE_MDQ(KK, MM, 4, true); else HE_MDQ(KK, MM, 4, false); }                                 \
    } while (0)
#define HE_MDQ_M(KK)                                                                                                 \
    do {                                                                                                             \
        if (mode == kTailRescale) HE_MDQ_B(KK, kTailRescale);                                                        \
        else if (mode == kTailPlain) HE_MDQ_B(KK, kTailPlain);                                                       \
        else HE_MDQ_B(KK, kTailRescalePQ);                                                                           \
    } while (0)
    if (c->KP == 1) HE_MDQ_M(1);
    else if (c->KP == 8) HE_MDQ_M(8);
    else HE_MDQ_M(12);
#undef HE_MDQ_M
#undef HE_MDQ_B
#undef HE_MDQ
    return cudaGetLastError();
}

cudaError_t run_combine_plain(const he_ctx *c, const JobRef &R, cudaStream_t st)
{
    dim3 g = grid_x(c->N);
    g.y = R.lmax;
    g.z = 2 * R.B;
    launch_k(c->pdl, k_combine_plain, g, dim3(kThreads), 0, st, R, c->d_pinv, c->d_levels, c->d_primes, c->K, c->N);
    return cudaGetLastError();
}

cudaError_t run_rescale_combine(const he_ctx *c, const u64 *ct, const u64 *Z, u64 *out, int l, cudaStream_t st)
{
    dim3 g = grid_x(c->N);
    g.y = l - 1;
    g.z = 2;
    launch_k(c->pdl, k_rescale_combine, g, dim3(kThreads), 0, st, ct, Z, out, c->d_levels, c->d_primes, c->K, l, c->N);
    return cudaGetLastError();
}

}  // namespace he
