// ntt.cu -- negacyclic NTT / iNTT of batches of limbs on sm_103a.
//
// The transform is the paper's Algo 3 (Cooley-Tukey, twiddles
// TB_W[m + j] = psi^bitrev(m + j), bit-reversed output) with Algo 4's
// butterfly, and its inverse (Gentleman-Sande with TB_invW, then N^-1).
// GPU mapping (the paper's high-radix idea, Sec. 5.3, rebuilt for 64-bit
// words): log N stages are split into two passes over HBM (one for N = 2^12);
// a pass works on 4096-element tiles held in shared memory and runs its
// stages as rounds of radix-2^r butterflies in registers, one shared-memory
// exchange per round.  Butterflies are Harvey's lazy forms: forward values
// stay in [0, 4q), inverse values in [0, 2q); the last pass reduces to
// [0, q) and, for the inverse, multiplies by N^-1 times a per-limb constant.
//
// Stage / twiddle indexing.  Global stage sigma (m = 2^sigma) pairs j and
// j + N/2^(sigma+1) and uses twiddle m + floor(j / 2^(logN - sigma)).  A pass
// covering stages [s0, s0 + M) sees element j = G * 2^(logN - s0) + k * C + c
// (k < 2^M the in-group index, c < C the column, G the group's high bits); at
// local stage l the twiddle index is 2^(s0+l) + (G << l) + (k >> (M - l)).
#include "he_internal.h"
#include "modarith.cuh"

namespace he {

namespace {

constexpr int kTE = 4096;                  // elements per tile
constexpr int kSmem = kTE + kTE / 16;      // one pad word every 16 elements

__device__ __forceinline__ int padi(int e) { return e + (e >> 4); }

struct NttArgs {
    const u64 *src;      // base of job.src offsets
    u64 *dst;            // base of job.dst offsets
    const NttJob *jobs;
    const DevPrime *primes;
    int logN;
    int tiles;           // tiles per job
};

__device__ __forceinline__ void ct_bfly(u64 &x, u64 &y, ulonglong2 w, u64 q, u64 q2)
{
    u64 a = x >= q2 ? x - q2 : x;
    u64 t = shoup_lazy(y, w.x, w.y, q);
    x = a + t;
    y = a - t + q2;
}

__device__ __forceinline__ void gs_bfly(u64 &x, u64 &y, ulonglong2 w, u64 q, u64 q2)
{
    u64 s = x + y;
    s = s >= q2 ? s - q2 : s;
    u64 d = x - y + q2;
    y = shoup_lazy(d, w.x, w.y, q);
    x = s;
}

// One round of R stages [l0, l0 + R) on every register set of the tile.
template <int LOGM, int R, bool STRIDED, bool INV, int NT>
__device__ __forceinline__ void ntt_round(u64 *sm, int l0, int s0, int gbase, const ulonglong2 *__restrict__ tw,
                                          u64 q, u64 q2)
{
    constexpr int M = 1 << LOGM;
    constexpr int NG = kTE / M;
    constexpr int SETS = kTE >> R;
    const int lo_bits = LOGM - l0 - R;
    for (int s = threadIdx.x; s < SETS; s += NT) {
        int grp, khi, klo;
        if (STRIDED) {
            grp = s % NG;
            int rest = s / NG;
            klo = rest & ((1 << lo_bits) - 1);
            khi = rest >> lo_bits;
        } else {
            klo = s & ((1 << lo_bits) - 1);
            int rest = s >> lo_bits;
            const int nhi = 1 << l0;
            khi = rest % nhi;
            grp = rest / nhi;
        }
        const int kbase = (khi << (LOGM - l0)) | klo;
        u64 a[1 << R];
#pragma unroll
        for (int v = 0; v < (1 << R); v++) {
            int k = kbase + (v << lo_bits);
            int e = STRIDED ? k * NG + grp : grp * M + k;
            a[v] = sm[padi(e)];
        }
        const int G = STRIDED ? 0 : gbase + grp;
        if (!INV) {
#pragma unroll
            for (int lp = 0; lp < R; lp++) {
                const int l = l0 + lp;
                const int tb = (1 << (s0 + l)) + (G << l) + (khi << lp);
                const int h = 1 << (R - 1 - lp);
#pragma unroll
                for (int v = 0; v < (1 << R); v++) {
                    if (v & h) continue;
                    ulonglong2 w = __ldg(&tw[tb + (v >> (R - lp))]);
                    ct_bfly(a[v], a[v + h], w, q, q2);
                }
            }
        } else {
#pragma unroll
            for (int lp = R - 1; lp >= 0; lp--) {
                const int l = l0 + lp;
                const int tb = (1 << (s0 + l)) + (G << l) + (khi << lp);
                const int h = 1 << (R - 1 - lp);
#pragma unroll
                for (int v = 0; v < (1 << R); v++) {
                    if (v & h) continue;
                    ulonglong2 w = __ldg(&tw[tb + (v >> (R - lp))]);
                    gs_bfly(a[v], a[v + h], w, q, q2);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < (1 << R); v++) {
            int k = kbase + (v << lo_bits);
            int e = STRIDED ? k * NG + grp : grp * M + k;
            sm[padi(e)] = a[v];
        }
    }
}

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// One pass of LOGM stages.  Rounds RA, RB, RC (RC may be 0) in forward order;
// the inverse runs them in reverse.  FIRST: read job.src (else job.dst);
// LAST: apply the output reduction / scaling.
template <int LOGM, int RA, int RB, int RC, bool STRIDED, bool INV, bool FIRST, bool LAST>
__global__ void __launch_bounds__(kTE >> cmax(RA, cmax(RB, RC)))
k_ntt_pass(const NttArgs P)
{
    constexpr int NT = kTE >> cmax(RA, cmax(RB, RC));
    constexpr int M = 1 << LOGM;
    constexpr int NG = kTE / M;
    static_assert(RA + RB + RC == LOGM, "rounds must cover the pass");
    __shared__ u64 sm[kSmem];

    const int job = blockIdx.x / P.tiles;
    const int tile = blockIdx.x - job * P.tiles;
    const NttJob J = P.jobs[job];
    const DevPrime pr = P.primes[J.prime];
    const int N = 1 << P.logN;
    const u64 *src = (FIRST ? P.src + (size_t)J.src * N : P.dst + (size_t)J.dst * N);
    u64 *dst = P.dst + (size_t)J.dst * N;
    const int stride = N >> LOGM;  // columns (strided) -- element k of column c at k*stride + c
    const int col0 = tile * NG;    // strided: first column of the tile
    const int g0 = tile * NG;      // contiguous: first group of the tile
    const int s0 = STRIDED ? 0 : P.logN - LOGM;

    // HBM -> shared memory, coalesced 16-byte loads
    for (int i = threadIdx.x; i < kTE / 2; i += NT) {
        const int e = 2 * i;
        size_t gi;
        if (STRIDED) gi = (size_t)(e / NG) * stride + col0 + (e % NG);
        else gi = (size_t)g0 * M + e;
        ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(src + gi);
        sm[padi(e)] = v.x;
        sm[padi(e + 1)] = v.y;
    }
    __syncthreads();

    const ulonglong2 *tw = INV ? pr.iw : pr.w;
    if (!INV) {
        ntt_round<LOGM, RA, STRIDED, false, NT>(sm, 0, s0, g0, tw, pr.q, pr.q2);
        __syncthreads();
        ntt_round<LOGM, RB, STRIDED, false, NT>(sm, RA, s0, g0, tw, pr.q, pr.q2);
        __syncthreads();
        if (RC) {
            ntt_round<LOGM, (RC ? RC : 1), STRIDED, false, NT>(sm, RA + RB, s0, g0, tw, pr.q, pr.q2);
            __syncthreads();
        }
    } else {
        if (RC) {
            ntt_round<LOGM, (RC ? RC : 1), STRIDED, true, NT>(sm, RA + RB, s0, g0, tw, pr.q, pr.q2);
            __syncthreads();
        }
        ntt_round<LOGM, RB, STRIDED, true, NT>(sm, RA, s0, g0, tw, pr.q, pr.q2);
        __syncthreads();
        ntt_round<LOGM, RA, STRIDED, true, NT>(sm, 0, s0, g0, tw, pr.q, pr.q2);
        __syncthreads();
    }

    // shared memory -> HBM, with the output reduction on the last pass
    for (int i = threadIdx.x; i < kTE / 2; i += NT) {
        const int e = 2 * i;
        u64 x = sm[padi(e)], y = sm[padi(e + 1)];
        if (LAST) {
            if (!INV) {
                x = csub(x >= pr.q2 ? x - pr.q2 : x, pr.q);
                y = csub(y >= pr.q2 ? y - pr.q2 : y, pr.q);
            } else {
                x = shoup(x, J.scale, J.scale_sh, pr.q);
                y = shoup(y, J.scale, J.scale_sh, pr.q);
            }
        }
        size_t gi;
        if (STRIDED) gi = (size_t)(e / NG) * stride + col0 + (e % NG);
        else gi = (size_t)g0 * M + e;
        *reinterpret_cast<ulonglong2 *>(dst + gi) = make_ulonglong2(x, y);
    }
}

template <int LOGM, int RA, int RB, int RC, bool STRIDED, bool INV, bool FIRST, bool LAST>
cudaError_t run_pass(const NttArgs &a, int njobs, cudaStream_t st)
{
    constexpr int NT = kTE >> cmax(RA, cmax(RB, RC));
    k_ntt_pass<LOGM, RA, RB, RC, STRIDED, INV, FIRST, LAST><<<njobs * a.tiles, NT, 0, st>>>(a);
    return cudaGetLastError();
}

// Two-pass transform: the strided pass covers the first S1 stages (forward
// order), the contiguous pass the last S2.
template <int S1, int A1, int B1, int C1, int S2, int A2, int B2, int C2>
cudaError_t two_pass(const he_ctx *c, NttArgs a, int njobs, bool inverse, cudaStream_t st, const char *tag)
{
    a.tiles = (1 << (S1 + S2)) / kTE;
    cudaError_t e;
    const char *t1 = inverse ? ".inv_pass1" : ".fwd_pass1";
    const char *t2 = inverse ? ".inv_pass2" : ".fwd_pass2";
    if (!inverse) {
        e = run_pass<S1, A1, B1, C1, true, false, true, false>(a, njobs, st);
        if (e != cudaSuccess) return e;
        prof_mark(c, st, tag, t1);
        e = run_pass<S2, A2, B2, C2, false, false, false, true>(a, njobs, st);
        prof_mark(c, st, tag, t2);
        return e;
    }
    e = run_pass<S2, A2, B2, C2, false, true, true, false>(a, njobs, st);
    if (e != cudaSuccess) return e;
    prof_mark(c, st, tag, t1);
    e = run_pass<S1, A1, B1, C1, true, true, false, true>(a, njobs, st);
    prof_mark(c, st, tag, t2);
    return e;
}

}  // namespace

cudaError_t launch_ntt2(const he_ctx *c, const u64 *src, u64 *dst, const NttJob *jobs, int njobs, bool inverse,
                        cudaStream_t st, const char *tag)
{
    if (njobs <= 0) return cudaSuccess;
    NttArgs a;
    a.src = src;
    a.dst = dst;
    a.jobs = jobs;
    a.primes = c->d_primes;
    a.logN = c->logN;
    a.tiles = 1;
    switch (c->logN) {
    case 12: {
        cudaError_t e = inverse ? run_pass<12, 4, 4, 4, false, true, true, true>(a, njobs, st)
                                : run_pass<12, 4, 4, 4, false, false, true, true>(a, njobs, st);
        prof_mark(c, st, tag, inverse ? ".inv" : ".fwd");
        return e;
    }
    case 13: return two_pass<7, 4, 3, 0, 6, 3, 3, 0>(c, a, njobs, inverse, st, tag);
    case 14: return two_pass<7, 4, 3, 0, 7, 4, 3, 0>(c, a, njobs, inverse, st, tag);
    case 15: return two_pass<8, 4, 4, 0, 7, 4, 3, 0>(c, a, njobs, inverse, st, tag);
    case 16: return two_pass<8, 4, 4, 0, 8, 4, 4, 0>(c, a, njobs, inverse, st, tag);
    case 17: return two_pass<9, 3, 3, 3, 8, 4, 4, 0>(c, a, njobs, inverse, st, tag);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ntt(const he_ctx *c, u64 *base, const NttJob *jobs, int njobs, bool inverse, cudaStream_t st,
                       const char *tag)
{
    return launch_ntt2(c, base, base, jobs, njobs, inverse, st, tag);
}

}  // namespace he
