// ntt.cu -- negacyclic NTT / iNTT of batches of limbs on sm_103a.
//
// The transform is the paper's Algo 3 (Cooley-Tukey, twiddles
// TB_W[m + j] = psi^bitrev(m + j), bit-reversed output) with Algo 4's
// butterfly, and its inverse (Gentleman-Sande with TB_invW, then N^-1).
// GPU mapping (the paper's high-radix idea, Sec. 5.3, rebuilt for 64-bit
// words): the log N stages are split into two passes over memory (one for
// N = 2^12).  A pass works on tiles of TE elements held in shared memory and
// runs its stages as rounds of radix-2^r butterflies in registers, one
// shared-memory exchange per round.  Butterflies are lazy: forward values
// grow by at most 4q per stage with no correction step, inverse values stay in
// [0, 4q); the paper's modified Shoup product (Sec. 5.2) supplies the twiddle
// multiplications.  The last pass reduces to [0, q) and, for the inverse,
// multiplies by N^-1 times a per-limb constant.
//
// Memory side: a CTA takes one tile position of a group of up to four limbs
// that share a prime.  The tile's twiddles are copied into shared memory once
// (cp.async) and reused for every limb of the group.  Strided passes (whose
// twiddles, TB_W[1, M), are few) double-buffer the limbs' data tiles so the
// next limb loads while this one computes; contiguous passes stage a 32 KB
// twiddle run per tile and keep a single data buffer, which holds occupancy
// at four CTAs per SM.
//
// Stage / twiddle indexing.  Global stage sigma (m = 2^sigma) pairs j and
// j + N/2^(sigma+1) and uses twiddle m + floor(j / 2^(logN - sigma)).  A pass
// covering stages [s0, s0 + M) sees element j = G * 2^(logN - s0) + k * C + c
// (k < 2^M the in-group index, c < C the column, G the group's high bits); at
// local stage l the twiddle index is 2^(s0+l) + (G << l) + (k >> (M - l)).
// In the strided (first forward / last inverse) pass s0 = 0 and G = 0, so
// every tile uses twiddles [1, 2^M); in the contiguous pass the tile's groups
// [g0, g0 + NG) use, per stage l, the run [2^(s0+l) + g0 2^l, + NG 2^l).
#include <cstring>
#include <type_traits>

#include <cuda_pipeline_primitives.h>

#include "he_internal.h"
#include "modarith.cuh"

namespace he {

namespace {

__device__ __forceinline__ int padi(int e) { return e + (e >> 4); }

struct NttArgs {
    const u64 *src;  // base of group.src offsets
    u64 *dst;        // base of group.dst offsets
    const NttGroup *groups;
    const DevPrime *primes;
    int logN;
    int ts;          // first stage whose twiddle runs the table stores transposed
    int tiles;       // tiles per limb
    const int *count;  // optional device-side group count (grids sized for a maximum)
    int pdl;           // programmatic dependent launch: 0 off, 1 on, 2 with early dependent launch
    // fused final combine (COMBINE passes only)
    JobRef R;
    const DevLevel *levels;
    const ulonglong2 *pinv;
    // fused key-switch sums (kFuseIp passes only): the evaluation key
    // [dnum][2][EL][N], EL = K + L
    const u64 *evk;
    int EL;
};

// 16-byte read-only load that does not allocate in L1 (twiddles read once).
// The table's lines are kept in L2 (evict-last): every HE Mul rereads them.
__device__ __forceinline__ ulonglong2 ld_tw(const ulonglong2 *p) { return ld2_hint(p, l2_policy_keep()); }

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Pass geometry.  RL is the pass's last round in forward order (the round
// whose sets are 2^RL consecutive elements).  In the contiguous pass each
// twiddle of that round is used by exactly one thread, so its twiddles are
// read straight into registers; only the earlier rounds' twiddles (stages
// l < LOGM - RL) are staged in shared memory.  The strided pass stages all of
// TB_W[1, M), which every tile shares.  Data tiles are double-buffered.
template <int LOGM, int TE, bool STRIDED, int RL>
struct Geometry {
    static constexpr int M = 1 << LOGM;
    static constexpr int NG = TE / M;                                   // groups (or columns) per tile
    static constexpr int LS = STRIDED ? LOGM : LOGM - RL;               // stages with shared-memory twiddles
    static constexpr int TWN = STRIDED ? M - 1 : NG * ((1 << LS) - 1);  // twiddle pairs staged per tile
    static constexpr int DATA = TE + TE / 16;                           // padded words per data buffer
    static constexpr int NBUF = 2;
    static constexpr size_t SMEM = sizeof(ulonglong2) * TWN + sizeof(u64) * NBUF * DATA;
};

// Shared-memory twiddle slot of local stage l, group grp, offset x.
template <int LOGM, int TE, bool STRIDED>
__device__ __forceinline__ int tw_slot(int l, int grp, int x)
{
    if (STRIDED) return (1 << l) - 1 + x;
    return (TE >> LOGM) * ((1 << l) - 1) + (grp << l) + x;
}

// Register twiddles of the direct round: for each of the thread's SPT sets,
// the 2^R - 1 twiddles of its stages, stage lp at offset 2^lp - 1.
template <int R, int SPT>
struct TwReg {
    ulonglong2 t[SPT][(1 << R) - 1];
};

// One round of R stages [l0, l0 + R) on every register set of the tile.
// The 2^R elements of a set sit at shared-memory word padi(e0) + c + (c >> 4)
// with c = v * 2^lo_bits * (STRIDED ? NG : 1): for every configuration used
// (R >= 3) the low four bits of e0 plus those of c never carry, so the
// padding of e0 + c splits into padi(e0) plus a compile-time offset.
// DIRECT: twiddles come from TR (the contiguous pass's last round).
template <int LOGM, int TE, int R, bool STRIDED, bool INV, int NT, bool DIRECT, class TRT>
__device__ __forceinline__ void ntt_round(u64 *sm, const ulonglong2 *tw, const TRT &TR, int l0, u64 nq, u64 q4)
{
    constexpr int M = 1 << LOGM;
    constexpr int NG = TE / M;
    constexpr int SETS = TE >> R;
    constexpr int SPT = SETS / NT;
    constexpr int CSTEP = STRIDED ? NG : 1;
    static_assert(SETS % NT == 0, "sets must divide evenly over the threads");
    const int lo_bits = LOGM - l0 - R;
#pragma unroll
    for (int si = 0; si < SPT; si++) {
        const int s = threadIdx.x + si * NT;
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
        u64 *base = sm + padi(STRIDED ? kbase * NG + grp : grp * M + kbase);
        u64 a[1 << R];
#pragma unroll
        for (int v = 0; v < (1 << R); v++) {
            const int c = (v << lo_bits) * CSTEP;
            a[v] = base[c + (c >> 4)];
        }
        if (!INV) {
#pragma unroll
            for (int lp = 0; lp < R; lp++) {
                const int l = l0 + lp;
                const ulonglong2 *t = tw + tw_slot<LOGM, TE, STRIDED>(l, grp, khi << lp);
                const int h = 1 << (R - 1 - lp);
#pragma unroll
                for (int v = 0; v < (1 << R); v++) {
                    if (v & h) continue;
                    const int j = v >> (R - lp);
                    ulonglong2 w;
                    if constexpr (DIRECT) w = TR.t[si][(1 << lp) - 1 + j];
                    else w = t[j];
                    ct_bfly(a[v], a[v + h], w, nq, q4);
                }
            }
        } else {
#pragma unroll
            for (int lp = R - 1; lp >= 0; lp--) {
                const int l = l0 + lp;
                const ulonglong2 *t = tw + tw_slot<LOGM, TE, STRIDED>(l, grp, khi << lp);
                const int h = 1 << (R - 1 - lp);
#pragma unroll
                for (int v = 0; v < (1 << R); v++) {
                    if (v & h) continue;
                    const int j = v >> (R - lp);
                    ulonglong2 w;
                    if constexpr (DIRECT) w = TR.t[si][(1 << lp) - 1 + j];
                    else w = t[j];
                    gs_bfly(a[v], a[v + h], w, nq, q4);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < (1 << R); v++) {
            const int c = (v << lo_bits) * CSTEP;
            base[c + (c >> 4)] = a[v];
        }
    }
}

// Table position of twiddle m + t of stage m = 2^sigma.  The table stores
// the runs of every stage sigma >= ts transposed: with d = sigma - ts, entry
// m + t sits at m + (t mod 2^d) 2^ts + floor(t / 2^d).
__host__ __device__ __forceinline__ size_t tw_pos(int sigma, int ts, size_t t)
{
    const int d = sigma - ts;
    if (d <= 0) return ((size_t)1 << sigma) + t;
    return ((size_t)1 << sigma) + ((t & (((size_t)1 << d) - 1)) << ts) + (t >> d);
}

// The direct round's twiddles of set Tn (its stages s0 + L0 + lp, lp < RL,
// all at or after ts): twiddle j of stage lp is entry Tn 2^lp + j of that
// stage, at base_lp + j 2^ts with base_lp = m + ((Tn mod 2^e) 2^lp) 2^ts +
// floor(Tn / 2^e), e = s0 + L0 - ts.  For consecutive sets a warp reads
// 2^e runs of consecutive entries per j.
__device__ __forceinline__ const ulonglong2 *direct_base(const ulonglong2 *twg, int sigma, int ts, int e, int lp, int Tn)
{
    return twg + ((size_t)1 << sigma) + ((size_t)((Tn & ((1 << e) - 1)) << lp) << ts) + (Tn >> e);
}

// L2 prefetch of the lines the direct round will read (one thread per
// 128-byte line of the transposed runs: the sets whose floor(Tn / 2^e) is a
// multiple of eight); issued when a CTA starts, so the round's loads hit L2
// instead of DRAM.
template <int LOGM, int TE, int RL, int NT>
__device__ __forceinline__ void prefetch_direct_tw(const ulonglong2 *twg, int tile, int s0, int ts)
{
    constexpr int L0 = LOGM - RL;
    constexpr int NG = TE >> LOGM;
    constexpr int SPT = (TE >> RL) / NT;
    const int e = s0 + L0 - ts;
#pragma unroll
    for (int si = 0; si < SPT; si++) {
        const int s = threadIdx.x + si * NT;
        const int Tn = ((tile * NG + (s >> L0)) << L0) + (s & ((1 << L0) - 1));
        if ((Tn >> e) & 7) continue;
#pragma unroll
        for (int lp = 0; lp < RL; lp++) {
            const ulonglong2 *g = direct_base(twg, s0 + L0 + lp, ts, e, lp, Tn);
#pragma unroll
            for (int j = 0; j < (1 << lp); j++)
                asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(g + ((size_t)j << ts)));
        }
    }
}

// The tensor product (Fig. 2 region 1 in RNS form: d0 = b1 b2, d1 = a1 b2 +
// a2 b1, d2 = a1 a2 mod q_i) of the contiguous tile `tile` of limb i, as the
// tile load of an inverse contiguous first pass.  The group's limb k carries
// the job (job[k]) and ci[k] = i | comp << 16 | keep << 18: the product comp
// (0: d0, 1: d1, 2: d2) goes to shared memory for the transform, and with
// keep all three are also stored to the job's workspace (d0, d1 for the final
// additions, d2 in the NTT domain for the inner product's own-digit rows).
// Without keep only the product needed is formed (the rescale limbs of d0,
// d1, whose d2 job stores them).
template <int TE, int NT>
__device__ __forceinline__ void tensor_tile(const NttArgs &P, const NttGroup &G, int k, int tile, const DevPrime &pr,
                                            u64 *b)
{
    const int lg = P.logN;
    const BatchItem it = job_item(P.R, (int)G.job[k]);
    const unsigned spec = G.ci[k];
    const int li = (int)(spec & 0xffffu), comp = (int)((spec >> 16) & 3u);
    const bool keep = ((spec >> 18) & 1u) != 0;
    const int l = it.level;
    const DevLevel &lv = P.levels[l];
    const size_t t0 = (size_t)tile * TE;
    const u64 *c1b = it.ct1 + ((size_t)li << lg) + t0, *c1a = it.ct1 + (((size_t)l + li) << lg) + t0;
    const u64 *c2b = it.ct2 + ((size_t)li << lg) + t0, *c2a = it.ct2 + (((size_t)l + li) << lg) + t0;
    u64 *w0 = it.ws + (((size_t)lv.o_d0 + li) << lg) + t0, *w1 = it.ws + (((size_t)lv.o_d1 + li) << lg) + t0;
    u64 *w2 = it.ws + (((size_t)lv.o_d2 + li) << lg) + t0;
    const u64 pol = l2_policy_stream();  // the ciphertexts are read once
    constexpr int PAIRS = TE / 2 / NT;
    static_assert(PAIRS % 2 == 0, "pairs per thread");
    constexpr int UNROLL = NT >= 256 ? 1 : 2;  // registers: the 256-thread tiles run at 64
#pragma unroll UNROLL
    for (int s = 0; s < PAIRS; s++) {
        const int e = 2 * (threadIdx.x + s * NT);
        const int gi = e;
        u64 x, y;
        if (keep) {
            const ulonglong2 b1 = ld2_hint(c1b + gi, pol), a1 = ld2_hint(c1a + gi, pol), b2 = ld2_hint(c2b + gi, pol),
                             a2 = ld2_hint(c2a + gi, pol);
            U128 sx = mul_wide(a1.x, b2.x), sy = mul_wide(a1.y, b2.y);
            mac(sx, a2.x, b1.x);
            mac(sy, a2.y, b1.y);
            const u64 d0x = mul_mod(b1.x, b2.x, pr.q, pr.mu, pr.s), d0y = mul_mod(b1.y, b2.y, pr.q, pr.mu, pr.s);
            const u64 d1x = barrett128(sx, pr.q, pr.mu, pr.s), d1y = barrett128(sy, pr.q, pr.mu, pr.s);
            const u64 d2x = mul_mod(a1.x, a2.x, pr.q, pr.mu, pr.s), d2y = mul_mod(a1.y, a2.y, pr.q, pr.mu, pr.s);
            *reinterpret_cast<ulonglong2 *>(w0 + gi) = make_ulonglong2(d0x, d0y);
            *reinterpret_cast<ulonglong2 *>(w1 + gi) = make_ulonglong2(d1x, d1y);
            *reinterpret_cast<ulonglong2 *>(w2 + gi) = make_ulonglong2(d2x, d2y);
            x = comp == 0 ? d0x : comp == 1 ? d1x : d2x;
            y = comp == 0 ? d0y : comp == 1 ? d1y : d2y;
        } else if (comp == 1) {
            const ulonglong2 b1 = ld2_hint(c1b + gi, pol), a1 = ld2_hint(c1a + gi, pol), b2 = ld2_hint(c2b + gi, pol),
                             a2 = ld2_hint(c2a + gi, pol);
            U128 sx = mul_wide(a1.x, b2.x), sy = mul_wide(a1.y, b2.y);
            mac(sx, a2.x, b1.x);
            mac(sy, a2.y, b1.y);
            x = barrett128(sx, pr.q, pr.mu, pr.s);
            y = barrett128(sy, pr.q, pr.mu, pr.s);
        } else {
            const u64 *u1 = comp == 0 ? c1b : c1a, *u2 = comp == 0 ? c2b : c2a;
            const ulonglong2 v1 = ld2_hint(u1 + gi, pol), v2 = ld2_hint(u2 + gi, pol);
            x = mul_mod(v1.x, v2.x, pr.q, pr.mu, pr.s);
            y = mul_mod(v1.y, v2.y, pr.q, pr.mu, pr.s);
        }
        b[padi(e)] = x;
        b[padi(e + 1)] = y;
    }
}

// The key-switch sum KS_h[e] = sum_j U_j[e] evk_{j,h}[e] mod q_e (Fig. 2
// region 2, the inner product with the evaluation key in the NTT domain) of
// the contiguous tile `tile` of one special limb (or q_{l-1}), as the tile
// load of the inverse contiguous first pass that takes it out of the NTT
// domain: the group's limb k carries the job (job[k]) and ci[k] = e | h << 16.
// U_j[e] is row e of digit j's ModUp output, or row e - K of d2 for the
// digit's own limbs; the products of up to kIpFuseDigits digits are summed in
// 128 bits and reduced once (below 4 q^2 < 2^112).  The sums are not stored:
// only this transform reads them.  At most kIpFuseDigits digits.

template <int TE, int NT>
__device__ __forceinline__ void ip_tile(const NttArgs &P, const NttGroup &G, int k, int tile, const DevPrime &pr,
                                        u64 *b)
{
    const int lg = P.logN;
    const BatchItem it = job_item(P.R, (int)G.job[k]);
    const unsigned spec = G.ci[k];
    const int e = (int)(spec & 0xffffu), h = (int)((spec >> 16) & 1u);
    const DevLevel &lv = P.levels[it.level];
    const int beta = lv.beta, E = lv.E, K = lv.E - it.level;
    // per digit: the limb of U_j[e] in the workspace (or of d2's row for the
    // digit's own limbs) and the key's limb, as limb indices
    unsigned uo[kIpFuseDigits], ko[kIpFuseDigits];
#pragma unroll
    for (int j = 0; j < kIpFuseDigits; j++) {
        const int jj = j < beta ? j : 0;
        const int lo = lv.dig_lo[jj], nj = lv.dig_n[jj];
        const bool own = e >= K && e - K >= lo && e - K < lo + nj;
        uo[j] = own ? lv.o_d2 + (unsigned)(e - K) : lv.o_u + (unsigned)(jj * E + e);
        ko[j] = (unsigned)((2 * jj + h) * P.EL + e);
    }
    const u64 *ws = it.ws + (size_t)tile * TE, *kb = P.evk + (size_t)tile * TE;
    const u64 pol = l2_policy_stream();  // U and the key are read once
    constexpr int PAIRS = TE / 2 / NT;
    constexpr int UNROLL = NT >= 256 ? 1 : 2;  // registers: the 256-thread tiles run at 64
#pragma unroll UNROLL
    for (int s = 0; s < PAIRS; s++) {
        const int x = 2 * (threadIdx.x + s * NT);
        ulonglong2 u[kIpFuseDigits], w[kIpFuseDigits];
#pragma unroll
        for (int j = 0; j < kIpFuseDigits; j++)
            if (j < beta) {
                u[j] = ld2_hint(ws + ((size_t)uo[j] << lg) + x, pol);
                w[j] = ld2_hint(kb + ((size_t)ko[j] << lg) + x, pol);
            }
        U128 ax = {0, 0}, ay = {0, 0};
#pragma unroll
        for (int j = 0; j < kIpFuseDigits; j++)
            if (j < beta) {
                mac(ax, u[j].x, w[j].x);
                mac(ay, u[j].y, w[j].y);
            }
        b[padi(x)] = barrett128(ax, pr.q, pr.mu, pr.s);
        b[padi(x + 1)] = barrett128(ay, pr.q, pr.mu, pr.s);
    }
}

// Final combine in place of a forward last pass's store: for limb i of the
// group (ModDown output (h, ci) of job G.job[i]),
// out[h][ci] = (d_h[ci] + KS_h[K+ci] P^-1 - z) q_{l-1}^-1 with z the
// transform in shared memory (thread pairs 2 t, +1 at g2 + k gs2 and shared
// word padi(2 t) + k (2 NT + NT / 8)).
template <int TE, int NT>
__device__ __forceinline__ void combine_store(const NttArgs &P, const NttGroup &G, int i, const u64 *sm, size_t g2,
                                              size_t gs2, const DevPrime &pr, u64 nq)
{
    const BatchItem it = job_item(P.R, (int)G.job[i]);
    const int ci = (int)(G.ci[i] & 0x7fffffffu), hh = (int)(G.ci[i] >> 31);
    const ulonglong2 pv = P.pinv[ci], qv = P.levels[it.level].qinv_last[ci];
    // above any forward-NTT output (values grow by < 4q per stage from
    // inputs below 4q): d + KS P^-1 (lazy, < 4q) + Cz - z stays in
    // (0, (9 + 4 log N) q), below 2^64, and one Shoup product by
    // q_{l-1}^-1 reduces it
    const u64 Cz = pr.q * (u64)(4 + 4 * P.logN);
    u64 *o = it.out + ((((size_t)hh * (it.level - 1) + ci)) << P.logN) + g2;
    const u64 *dd = P.dst + ((size_t)G.cd[i] << P.logN) + g2, *kk = P.dst + ((size_t)G.cks[i] << P.logN) + g2;
    const u64 *sp = sm + padi(2 * threadIdx.x);
    // four pairs per step: their d and KS loads are all in flight before the first product
    constexpr int PAIRS = TE / 2 / NT, B4 = PAIRS >= 4 ? 4 : PAIRS;
    static_assert(PAIRS % B4 == 0, "pairs per thread");
    for (int b0 = 0; b0 < PAIRS; b0 += B4) {
        ulonglong2 dv[B4], kv[B4];
#pragma unroll
        for (int k = 0; k < B4; k++) {
            dv[k] = __ldg(reinterpret_cast<const ulonglong2 *>(dd + (b0 + k) * gs2));
            kv[k] = __ldg(reinterpret_cast<const ulonglong2 *>(kk + (b0 + k) * gs2));
        }
#pragma unroll
        for (int k = 0; k < B4; k++) {
            // KS P^-1 lazily in [0, 4q): x < (6 + 4 log N) q < 2^64
            const u64 *z = sp + (b0 + k) * (2 * NT + NT / 8);
            const u64 x = dv[k].x + shoup_approx_nq(kv[k].x, pv.x, pv.y, nq) + Cz - z[0];
            const u64 y = dv[k].y + shoup_approx_nq(kv[k].y, pv.x, pv.y, nq) + Cz - z[1];
            *reinterpret_cast<ulonglong2 *>(o + (b0 + k) * gs2) =
                make_ulonglong2(shoup_canon(x, qv.x, qv.y, pr.q, nq), shoup_canon(y, qv.x, qv.y, pr.q, nq));
        }
    }
}

// Shared memory -> HBM for limb i of the group (same thread walk as
// combine_store), 16-byte stores; LAST: the output reduction (forward: from
// below (4 + 4 log N) q to [0, q); inverse: times the limb's scale).
template <int TE, int NT, bool LAST, bool INV>
__device__ __forceinline__ void final_store(const NttArgs &P, const NttGroup &G, int i, const u64 *sm, size_t g2,
                                            size_t gs2, const DevPrime &pr, u64 nq)
{
    u64 *dst = P.dst + ((size_t)G.dst[i] << P.logN) + g2;
    const u64 sc = G.scale[i], scs = G.scale_sh[i];
    const bool small_red = (pr.r64 >> 32) == 0;  // q > 2^32: reduce_small applies
    const u64 *sp = sm + padi(2 * threadIdx.x);
#pragma unroll
    for (int k = 0; k < TE / 2 / NT; k++) {
        u64 x = sp[0], y = sp[1];
        if (LAST) {
            if (!INV) {  // x < (4 + 4 log N) q
                if (small_red) {
                    x = reduce_small(x, pr.q, pr.r64);
                    y = reduce_small(y, pr.q, pr.r64);
                } else {
                    x = shoup(x, 1, pr.r64, pr.q);
                    y = shoup(y, 1, pr.r64, pr.q);
                }
            } else {
                x = shoup_canon(x, sc, scs, pr.q, nq);
                y = shoup_canon(y, sc, scs, pr.q, nq);
            }
        }
        *reinterpret_cast<ulonglong2 *>(dst) = make_ulonglong2(x, y);
        dst += gs2;
        sp += 2 * NT + NT / 8;
    }
}

// One pass of LOGM stages over a group of limbs.  Rounds RA, RB, RC (RC may
// be 0) in forward order; the inverse runs them in reverse.  FIRST: read
// group.src (else group.dst); LAST: apply the output reduction / scaling.
// Resident CTAs per SM the register allocation is bounded for (0: no bound):
// 256-thread tiles (radix-8 rounds) five (51 registers; inverse ones four, 64
// registers, as their first pass holds the direct round's twiddles from the
// start and the tensor-fused variant its products), forward 128-thread
// tiles six (85 registers, what their shared memory allows; measured faster
// than the compiler's own choice), inverse 128-thread tiles unbounded (their
// first pass holds the direct round's fifteen twiddles from the start and
// spills under a bound).
__host__ __device__ constexpr int ntt_min_blocks(int nt, int logm, bool inv)
{
    // 64-thread tiles (radix-16 rounds on 1024 elements): twelve forward (85
    // registers), inverse unbounded
    return logm >= 12 ? 0 : nt >= 256 ? (inv ? 4 : 5) : nt <= 64 ? (inv ? 0 : 12) : inv ? 0 : 6;
}

// FUSE: kFuseNone; kFuseCombine, the final combine in the store loop of the
// forward contiguous last pass (ModDown + rescale limbs); kFuseTensor, the
// tensor product computed in place of the inverse contiguous first pass's
// tile load (d2 limbs and the rescale limbs of d0, d1).
// kFuseIp, the key-switch sums of Fig. 2 region 2 computed in place of the
// tile load of the special limbs' inverse contiguous first pass.
enum { kFuseNone = 0, kFuseCombine = 1, kFuseTensor = 2, kFuseIp = 3 };

template <int LOGM, int RA, int RB, int RC, bool STRIDED, bool INV, bool FIRST, bool LAST, int TE, int FUSE = kFuseNone>
__global__ void __launch_bounds__(TE >> cmax(RA, cmax(RB, RC)), ntt_min_blocks(TE >> cmax(RA, cmax(RB, RC)), LOGM, INV))
k_ntt_pass(const NttArgs P)
{
    constexpr bool COMBINE = FUSE == kFuseCombine, TENSOR = FUSE == kFuseTensor, IPF = FUSE == kFuseIp;
    constexpr bool COMPUTED = TENSOR || IPF;  // the tile load computes its words
    static_assert(!COMBINE || (LAST && !INV && !STRIDED), "the combine follows a forward contiguous last pass");
    static_assert(!COMPUTED || (FIRST && INV && !STRIDED), "computed tiles feed an inverse contiguous first pass");
    constexpr int NT = TE >> cmax(RA, cmax(RB, RC));
    constexpr int RL = RC ? RC : RB;  // last round in forward order
    constexpr int L0 = LOGM - RL;     // its first stage
    constexpr bool DIRECT = !STRIDED;
    using Gm = Geometry<LOGM, TE, STRIDED, RL>;
    constexpr int NG = Gm::NG;
    static_assert(RA + RB + RC == LOGM, "rounds must cover the pass");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ulonglong2 *tw = reinterpret_cast<ulonglong2 *>(smem_raw);
    u64 *buf = reinterpret_cast<u64 *>(smem_raw + sizeof(ulonglong2) * Gm::TWN);

    const int gidx = blockIdx.x / P.tiles;
    const int tile = blockIdx.x - gidx * P.tiles;
    if (P.count && gidx >= *P.count) return idle_exit();
    const NttGroup &G = P.groups[gidx];
    const int nl = (int)G.nl;
    const DevPrime pr = P.primes[G.prime];
    const u64 nq = 0ull - pr.q;
    const int s0 = STRIDED ? 0 : P.logN - LOGM;

    // Thread walks over the tile: element threadIdx.x + k NT sits at global
    // index g1 + k gs1 and shared word padi(threadIdx.x) + k (NT + NT / 16)
    // (NT is a multiple of 16 and of NG); the pair 2 (threadIdx.x + k NT),
    // +1 at g2 + k gs2 and padi(2 threadIdx.x) + k (2 NT + NT / 8).  Index
    // arithmetic by shifts and additions only, which leaves the wide-multiply
    // pipe to the butterflies.
    const int lsh = P.logN - LOGM;  // log2 of the strided pass's row stride
    const size_t g1 = STRIDED ? (((size_t)(threadIdx.x / NG) << lsh) + (size_t)tile * NG + threadIdx.x % NG)
                              : (size_t)tile * TE + threadIdx.x;
    const size_t gs1 = STRIDED ? ((size_t)(NT / NG) << lsh) : (size_t)NT;
    const size_t g2 = STRIDED ? (((size_t)(2 * threadIdx.x / NG) << lsh) + (size_t)tile * NG + 2 * threadIdx.x % NG)
                              : (size_t)tile * TE + 2 * threadIdx.x;
    const size_t gs2 = STRIDED ? ((size_t)(2 * NT / NG) << lsh) : (size_t)(2 * NT);
    static_assert(NT % 16 == 0 && NT % NG == 0 && (2 * NT) % NG == 0, "tile walk");

    // data tile of limb i of the group -> shared memory (8-byte async copies)
    auto load_tile = [&](int i, u64 *b) {
        if constexpr (TENSOR) {
            tensor_tile<TE, NT>(P, G, i, tile, pr, b);
        } else if constexpr (IPF) {
            ip_tile<TE, NT>(P, G, i, tile, pr, b);
        } else {
            const u64 *src = (FIRST ? P.src + ((size_t)G.src[i] << P.logN) : P.dst + ((size_t)G.dst[i] << P.logN)) + g1;
            u64 *d = b + padi(threadIdx.x);
#pragma unroll
            for (int k = 0; k < TE / NT; k++) {
                __pipeline_memcpy_async(d, src, 8);
                d += NT + NT / 16;
                src += gs1;
            }
        }
    };
    // staged twiddles of this tile -> shared memory (16-byte async copies)
    const ulonglong2 *twg = INV ? pr.iw : pr.w;
    if (STRIDED) {
        for (int f = threadIdx.x; f < Gm::TWN; f += NT) __pipeline_memcpy_async(&tw[f], &twg[1 + f], 16);
    } else {
#pragma unroll
        for (int l = 0; l < Gm::LS; l++) {
            const int n = NG << l;
            if (s0 + l < P.ts) {
                const ulonglong2 *g = twg + (1 << (s0 + l)) + (size_t)tile * n;
                for (int f = threadIdx.x; f < n; f += NT)
                    __pipeline_memcpy_async(&tw[NG * ((1 << l) - 1) + f], &g[f], 16);
            } else {  // a stage of the transposed region (radix-8 plans)
                for (int f = threadIdx.x; f < n; f += NT)
                    __pipeline_memcpy_async(&tw[NG * ((1 << l) - 1) + f],
                                            &twg[tw_pos(s0 + l, P.ts, (size_t)tile * n + f)], 16);
            }
        }
    }
    if (DIRECT) prefetch_direct_tw<LOGM, TE, RL, NT>(twg, tile, s0, P.ts);
    // the limbs come from the previous kernels; the pass that streams the key
    // (kFuseIp) does not launch its successor early, whose waiting CTAs would
    // hold SM slots its last loads need (measured: 2^17 985 against 992 µs)
    griddep_wait(P.pdl >= 2 && FUSE != kFuseIp);
    load_tile(0, buf);
    __pipeline_commit();

    // the direct round's twiddles -> registers (reloaded for every limb from
    // L2 so that they are live only during that round), from the table's
    // transposed runs (direct_base).
    constexpr int SPT = (TE >> RL) / NT;
    const int te = s0 + L0 - P.ts;
    auto load_direct = [&](TwReg<RL, SPT> &T) {
#pragma unroll
        for (int si = 0; si < SPT; si++) {
            const int s = threadIdx.x + si * NT;
            const int khi = s & ((1 << L0) - 1);
            const int gg = tile * NG + (s >> L0);
            const int Tn = (gg << L0) + khi;
#pragma unroll
            for (int lp = 0; lp < RL; lp++) {
                const ulonglong2 *g = direct_base(twg, s0 + L0 + lp, P.ts, te, lp, Tn);
#pragma unroll
                for (int j = 0; j < (1 << lp); j++) T.t[si][(1 << lp) - 1 + j] = ld_tw(g + ((size_t)j << P.ts));
            }
        }
    };

    for (int i = 0; i < nl; i++) {
        u64 *sm = buf + (i & 1) * Gm::DATA;
        TwReg<RL, SPT> TR;
        // the inverse starts with the direct round (its twiddles are loaded
        // after the next limb's computed tile, which needs the registers)
        if (DIRECT && INV && !COMPUTED) load_direct(TR);
        if (i + 1 < nl) {
            load_tile(i + 1, buf + ((i + 1) & 1) * Gm::DATA);
            __pipeline_commit();
            __pipeline_wait_prior(1);
        } else {
            __pipeline_wait_prior(0);
        }
        if (DIRECT && INV && COMPUTED) load_direct(TR);
        __syncthreads();
        if (!INV) {
            ntt_round<LOGM, TE, RA, STRIDED, false, NT, false>(sm, tw, TR, 0, nq, pr.q4);
            if (DIRECT && RC == 0) load_direct(TR);
            __syncthreads();
            ntt_round<LOGM, TE, RB, STRIDED, false, NT, DIRECT && RC == 0>(sm, tw, TR, RA, nq, pr.q4);
            if (DIRECT && RC != 0) load_direct(TR);
            __syncthreads();
            if (RC) {
                ntt_round<LOGM, TE, (RC ? RC : 1), STRIDED, false, NT, DIRECT>(sm, tw, TR, RA + RB, nq, pr.q4);
                __syncthreads();
            }
        } else {
            if (RC) {
                ntt_round<LOGM, TE, (RC ? RC : 1), STRIDED, true, NT, DIRECT>(sm, tw, TR, RA + RB, nq, pr.q4);
                __syncthreads();
            }
            ntt_round<LOGM, TE, RB, STRIDED, true, NT, DIRECT && RC == 0>(sm, tw, TR, RA, nq, pr.q4);
            __syncthreads();
            ntt_round<LOGM, TE, RA, STRIDED, true, NT, false>(sm, tw, TR, 0, nq, pr.q4);
            __syncthreads();
        }
        if (COMBINE) {
            combine_store<TE, NT>(P, G, i, sm, g2, gs2, pr, nq);
            __syncthreads();  // the next prefetch reuses this buffer
            continue;
        }
        final_store<TE, NT, LAST, INV>(P, G, i, sm, g2, gs2, pr, nq);
        __syncthreads();  // the next prefetch reuses this buffer
    }
}

// ngroups == 0 only sets the kernel's shared-memory limit (no launch).
template <int LOGM, int RA, int RB, int RC, bool STRIDED, bool INV, bool FIRST, bool LAST, int TE, int FUSE = kFuseNone>
cudaError_t run_pass(const NttArgs &a, int ngroups, cudaStream_t st)
{
    constexpr int NT = TE >> cmax(RA, cmax(RB, RC));
    constexpr size_t smem = Geometry<LOGM, TE, STRIDED, (RC ? RC : RB)>::SMEM;
    auto kern = k_ntt_pass<LOGM, RA, RB, RC, STRIDED, INV, FIRST, LAST, TE, FUSE>;
    static bool configured = false;  // once per instantiation
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (ngroups == 0) return cudaSuccess;
    launch_k(a.pdl != 0, kern, dim3(ngroups * a.tiles), dim3(NT), smem, st, a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One-pass transform of N = 2^16 over a thread-block cluster.
//
// The limb is cut into kCl = 8 contiguous chunks of TE = N / 8 elements, one
// per CTA of a cluster, each held in its CTA's shared memory.  Stages 0-2
// pair elements of different chunks (stage sigma pairs j and
// j + N / 2^(sigma+1) with twiddle 2^sigma + floor(j / 2^(16 - sigma)), which
// depends only on the chunk of j): for every offset k of a chunk they form one
// radix-8 set {v TE + k : v < 8} with the twiddles of entries 1..7.  CTA r
// runs those sets for the offsets [r TE / 8, (r + 1) TE / 8) and moves the
// values between the CTAs through distributed shared memory; stages 3-15 are
// the contiguous pass of one group (s0 = 3, LOGM = 13, tile r of the limb).
// Forward: the cross round reads HBM and writes every chunk into its CTA's
// shared memory, then the local rounds, then the output reduction (or the
// final combine) and the store.  Inverse: the chunk is loaded (or formed by
// the tensor product), local rounds in reverse, then the cross round reads the
// chunks from the cluster's shared memory, scales and stores.  The limb makes
// one trip through HBM instead of two; every butterfly is the one the two-pass
// plans apply to the same operands, so every output word equals theirs.
constexpr int kCl = 8;                  // CTAs per cluster (portable size)
constexpr int kClLogN = 16;             // ring size of the plan
constexpr int kClTE = (1 << kClLogN) / kCl;
constexpr int kClLogM = kClLogN - 3;    // local stages 3 .. 15

__device__ __forceinline__ unsigned cl_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Barrier over every thread of the cluster; shared-memory writes before it
// (local or remote) are visible to every thread after it.
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address in the cluster's shared window of the word `p` of this CTA's
// shared memory as held by CTA `rank`.
__device__ __forceinline__ uint32_t cl_map(const void *p, unsigned rank)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void cl_st(uint32_t a, u64 v)
{
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

__device__ __forceinline__ u64 cl_ld(uint32_t a)
{
    u64 v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}

// Stages 0-2 on one radix-8 set (element v of the set in a[v]), twiddle
// entry 2^l + (v >> (3 - l)) of stage l at w[2^l - 1 + (v >> (3 - l))].
__device__ __forceinline__ void cross_fwd(u64 (&a)[8], const ulonglong2 (&w)[7], u64 nq, u64 q4)
{
#pragma unroll
    for (int l = 0; l < 3; l++) {
        const int h = 4 >> l;
#pragma unroll
        for (int v = 0; v < 8; v++)
            if (!(v & h)) ct_bfly(a[v], a[v + h], w[(1 << l) - 1 + (v >> (3 - l))], nq, q4);
    }
}

__device__ __forceinline__ void cross_inv(u64 (&a)[8], const ulonglong2 (&w)[7], u64 nq, u64 q4)
{
#pragma unroll
    for (int l = 2; l >= 0; l--) {
        const int h = 4 >> l;
#pragma unroll
        for (int v = 0; v < 8; v++)
            if (!(v & h)) gs_bfly(a[v], a[v + h], w[(1 << l) - 1 + (v >> (3 - l))], nq, q4);
    }
}

// Local rounds R0..R4 in forward order (R4 = 0: four rounds); the last one
// is the direct round.  NT threads: one set of the widest round each.
template <int R0, int R1, int R2, int R3, int R4>
struct ClGeom {
    static constexpr int RMAX = cmax(cmax(cmax(R0, R1), cmax(R2, R3)), R4);
    static constexpr int NT = kClTE >> RMAX;
    static constexpr int RL = R4 ? R4 : R3;
    using Gm = Geometry<kClLogM, kClTE, false, RL>;
    static constexpr size_t SMEM = sizeof(ulonglong2) * Gm::TWN + sizeof(u64) * Gm::DATA;  // one data buffer
};

template <int R0, int R1, int R2, int R3, int R4, bool INV, int FUSE>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(ClGeom<R0, R1, R2, R3, R4>::NT, 1)
k_ntt_cluster(const NttArgs P)
{
    constexpr bool COMBINE = FUSE == kFuseCombine, TENSOR = FUSE == kFuseTensor;
    static_assert(!COMBINE || !INV, "the combine follows a forward transform");
    static_assert(!TENSOR || INV, "the tensor product feeds an inverse transform");
    using CG = ClGeom<R0, R1, R2, R3, R4>;
    using Gm = typename CG::Gm;
    constexpr int LOGM = kClLogM, TE = kClTE, NT = CG::NT, RL = CG::RL, L0 = LOGM - RL;
    static_assert(R0 + R1 + R2 + R3 + R4 == LOGM, "rounds must cover the local stages");
    static_assert(Gm::NG == 1, "one group per chunk");
    constexpr int CK = TE / kCl;    // cross-round offsets per CTA
    constexpr int CPT = CK / NT;    // per thread: consecutive offsets k0 .. k0 + CPT - 1
    static_assert(CPT * NT == CK && (CPT == 1 || CPT == 2), "one or two offsets per thread in the cross round");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ulonglong2 *tw = reinterpret_cast<ulonglong2 *>(smem_raw);
    u64 *sm = reinterpret_cast<u64 *>(smem_raw + sizeof(ulonglong2) * Gm::TWN);

    const int tile = (int)cl_rank();  // the chunk this CTA holds
    const int gidx = blockIdx.x / kCl;
    if (P.count && gidx >= *P.count) return idle_exit();  // the whole cluster leaves
    const NttGroup &G = P.groups[gidx];
    const int nl = (int)G.nl;
    const DevPrime pr = P.primes[G.prime];
    const u64 nq = 0ull - pr.q;
    constexpr int s0 = 3;
    const ulonglong2 *twg = INV ? pr.iw : pr.w;
    // the local rounds' staged twiddles (stages s0 + l, l < LS, of this tile)
#pragma unroll
    for (int l = 0; l < Gm::LS; l++) {
        const int n = 1 << l;
        if (s0 + l < P.ts) {
            const ulonglong2 *g = twg + (1 << (s0 + l)) + (size_t)tile * n;
            for (int f = threadIdx.x; f < n; f += NT) __pipeline_memcpy_async(&tw[n - 1 + f], &g[f], 16);
        } else {
            for (int f = threadIdx.x; f < n; f += NT)
                __pipeline_memcpy_async(&tw[n - 1 + f], &twg[tw_pos(s0 + l, P.ts, (size_t)tile * n + f)], 16);
        }
    }
    __pipeline_commit();
    prefetch_direct_tw<LOGM, TE, RL, NT>(twg, tile, s0, P.ts);
    // this thread's cross-round offsets and their words in every CTA's shared memory
    const int k0 = tile * CK + CPT * threadIdx.x;
    uint32_t ko[CPT];
#pragma unroll
    for (int c = 0; c < CPT; c++) ko[c] = 8u * (uint32_t)padi(k0 + c);
    uint32_t rb[kCl];
#pragma unroll
    for (int v = 0; v < kCl; v++) rb[v] = cl_map(sm, (unsigned)v);
    // the chunk's thread walk (as the contiguous pass with one tile per limb)
    const size_t g2 = (size_t)tile * TE + 2 * threadIdx.x, gs2 = 2 * NT;

    constexpr int SPT = (TE >> RL) / NT;
    const int te = s0 + L0 - P.ts;
    auto load_direct = [&](TwReg<RL, SPT> &T) {
#pragma unroll
        for (int si = 0; si < SPT; si++) {
            const int s = threadIdx.x + si * NT;
            const int Tn = ((tile + (s >> L0)) << L0) + (s & ((1 << L0) - 1));
#pragma unroll
            for (int lp = 0; lp < RL; lp++) {
                const ulonglong2 *g = direct_base(twg, s0 + L0 + lp, P.ts, te, lp, Tn);
#pragma unroll
                for (int j = 0; j < (1 << lp); j++) T.t[si][(1 << lp) - 1 + j] = ld_tw(g + ((size_t)j << P.ts));
            }
        }
    };

    griddep_wait(P.pdl >= 2);  // the limbs come from the previous kernels
    for (int i = 0; i < nl; i++) {
        TwReg<RL, SPT> TR;
        ulonglong2 cw[7];
#pragma unroll
        for (int t = 0; t < 7; t++) cw[t] = ld_tw(twg + 1 + t);
        if (!INV) {
            const u64 *src = P.src + ((size_t)G.src[i] << P.logN);
            u64 a[CPT][8];
#pragma unroll
            for (int v = 0; v < 8; v++) {
                if constexpr (CPT == 2) {
                    const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(src + (size_t)v * TE + k0);
                    a[0][v] = x.x;
                    a[CPT - 1][v] = x.y;
                } else {
                    a[0][v] = src[(size_t)v * TE + k0];
                }
            }
#pragma unroll
            for (int c = 0; c < CPT; c++) cross_fwd(a[c], cw, nq, pr.q4);
            cl_sync();  // every CTA of the cluster runs and is done with its previous chunk
#pragma unroll
            for (int v = 0; v < 8; v++)
#pragma unroll
                for (int c = 0; c < CPT; c++) cl_st(rb[v] + ko[c], a[c][v]);
            __pipeline_wait_prior(0);  // this thread's staged twiddles
            cl_sync();                 // every chunk complete, the twiddles visible
            ntt_round<LOGM, TE, R0, false, false, NT, false>(sm, tw, TR, 0, nq, pr.q4);
            __syncthreads();
            ntt_round<LOGM, TE, R1, false, false, NT, false>(sm, tw, TR, R0, nq, pr.q4);
            __syncthreads();
            ntt_round<LOGM, TE, R2, false, false, NT, false>(sm, tw, TR, R0 + R1, nq, pr.q4);
            if constexpr (R4 != 0) {
                __syncthreads();
                ntt_round<LOGM, TE, R3, false, false, NT, false>(sm, tw, TR, R0 + R1 + R2, nq, pr.q4);
            }
            load_direct(TR);
            __syncthreads();
            ntt_round<LOGM, TE, RL, false, false, NT, true>(sm, tw, TR, L0, nq, pr.q4);
            __syncthreads();
            if (COMBINE) combine_store<TE, NT>(P, G, i, sm, g2, gs2, pr, nq);
            else final_store<TE, NT, true, false>(P, G, i, sm, g2, gs2, pr, nq);
        } else {
            if (i > 0) cl_sync();  // the peers are done reading this CTA's previous chunk
            if constexpr (TENSOR) {
                tensor_tile<TE, NT>(P, G, i, tile, pr, sm);
            } else {
                const u64 *src = P.src + ((size_t)G.src[i] << P.logN) + (size_t)tile * TE + threadIdx.x;
                u64 *d = sm + padi(threadIdx.x);
#pragma unroll
                for (int k = 0; k < TE / NT; k++) {
                    __pipeline_memcpy_async(d, src, 8);
                    d += NT + NT / 16;
                    src += NT;
                }
                __pipeline_commit();
            }
            load_direct(TR);
            __pipeline_wait_prior(0);
            __syncthreads();
            ntt_round<LOGM, TE, RL, false, true, NT, true>(sm, tw, TR, L0, nq, pr.q4);
            __syncthreads();
            if constexpr (R4 != 0) {
                ntt_round<LOGM, TE, R3, false, true, NT, false>(sm, tw, TR, R0 + R1 + R2, nq, pr.q4);
                __syncthreads();
            }
            ntt_round<LOGM, TE, R2, false, true, NT, false>(sm, tw, TR, R0 + R1, nq, pr.q4);
            __syncthreads();
            ntt_round<LOGM, TE, R1, false, true, NT, false>(sm, tw, TR, R0, nq, pr.q4);
            __syncthreads();
            ntt_round<LOGM, TE, R0, false, true, NT, false>(sm, tw, TR, 0, nq, pr.q4);
            cl_sync();  // every chunk transformed
            u64 a[CPT][8];
#pragma unroll
            for (int v = 0; v < 8; v++)
#pragma unroll
                for (int c = 0; c < CPT; c++) a[c][v] = cl_ld(rb[v] + ko[c]);
#pragma unroll
            for (int c = 0; c < CPT; c++) cross_inv(a[c], cw, nq, pr.q4);
            u64 *dst = P.dst + ((size_t)G.dst[i] << P.logN) + k0;
            const u64 sc = G.scale[i], scs = G.scale_sh[i];
#pragma unroll
            for (int v = 0; v < 8; v++) {
                if constexpr (CPT == 2)
                    *reinterpret_cast<ulonglong2 *>(dst + (size_t)v * TE) = make_ulonglong2(
                        shoup_canon(a[0][v], sc, scs, pr.q, nq), shoup_canon(a[CPT - 1][v], sc, scs, pr.q, nq));
                else
                    dst[(size_t)v * TE] = shoup_canon(a[0][v], sc, scs, pr.q, nq);
            }
        }
    }
    if (INV) cl_sync();  // no CTA leaves while a peer still reads its shared memory
}

// ngroups == 0 only sets the kernel's shared-memory limit (no launch).
template <int R0, int R1, int R2, int R3, int R4, bool INV, int FUSE = kFuseNone>
cudaError_t run_cluster(const NttArgs &a, int ngroups, cudaStream_t st)
{
    using CG = ClGeom<R0, R1, R2, R3, R4>;
    auto kern = k_ntt_cluster<R0, R1, R2, R3, R4, INV, FUSE>;
    static bool configured = false;  // once per instantiation
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CG::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    if (ngroups == 0) return cudaSuccess;
    launch_k(a.pdl != 0, kern, dim3(ngroups * kCl), dim3(CG::NT), CG::SMEM, st, a);
    return cudaGetLastError();
}

// Pass plans per ring size: the strided pass covers the first S1 stages
// (rounds A1, B1, C1), the contiguous pass the last S2 (rounds A2, B2, C2).
// N = 2^12 is one contiguous pass of rounds 4, 4, 4.
template <int LOGN> struct Plan;
template <> struct Plan<13> { static constexpr int S1 = 7, A1 = 4, B1 = 3, C1 = 0, S2 = 6, A2 = 3, B2 = 3, C2 = 0; };
template <> struct Plan<14> { static constexpr int S1 = 7, A1 = 4, B1 = 3, C1 = 0, S2 = 7, A2 = 4, B2 = 3, C2 = 0; };
template <> struct Plan<15> { static constexpr int S1 = 8, A1 = 4, B1 = 4, C1 = 0, S2 = 7, A2 = 4, B2 = 3, C2 = 0; };
template <> struct Plan<16> { static constexpr int S1 = 8, A1 = 4, B1 = 4, C1 = 0, S2 = 8, A2 = 4, B2 = 4, C2 = 0; };
template <> struct Plan<17> { static constexpr int S1 = 9, A1 = 3, B1 = 3, C1 = 3, S2 = 8, A2 = 4, B2 = 4, C2 = 0; };
template <int LOGN> constexpr int plan_direct() { return Plan<LOGN>::C2 ? Plan<LOGN>::C2 : Plan<LOGN>::B2; }

// Radix-8 plans: every round of at most three stages, so a tile has 256
// threads (twice the radix-16 plans' threads per limb: launches over few
// limbs fill more of the GPU).  The direct round (the contiguous pass's last
// two or three stages) lies inside the transposed region of the table the
// radix-16 plan lays out (plan_direct stages), so both plans share one table.
template <int LOGN> struct Plan8;
// The round orders are the ones whose shared-memory accesses are free of
// bank conflicts with the one-word-per-16 padding (a warp's 32 8-byte words
// in two wavefronts), checked exhaustively on the CPU.
template <> struct Plan8<13> { static constexpr int S1 = 7, A1 = 3, B1 = 2, C1 = 2, S2 = 6, A2 = 3, B2 = 3, C2 = 0; };
template <> struct Plan8<14> { static constexpr int S1 = 7, A1 = 3, B1 = 2, C1 = 2, S2 = 7, A2 = 2, B2 = 3, C2 = 2; };
template <> struct Plan8<15> { static constexpr int S1 = 8, A1 = 2, B1 = 3, C1 = 3, S2 = 7, A2 = 2, B2 = 3, C2 = 2; };
template <> struct Plan8<16> { static constexpr int S1 = 8, A1 = 2, B1 = 3, C1 = 3, S2 = 8, A2 = 2, B2 = 3, C2 = 3; };
template <> struct Plan8<17> { static constexpr int S1 = 9, A1 = 3, B1 = 3, C1 = 3, S2 = 8, A2 = 2, B2 = 3, C2 = 3; };
template <int LOGN> constexpr bool plan8_fits()
{
    return (Plan8<LOGN>::C2 ? Plan8<LOGN>::C2 : Plan8<LOGN>::B2) <= plan_direct<LOGN>();
}
static_assert(plan8_fits<13>() && plan8_fits<14>() && plan8_fits<15>() && plan8_fits<16>() && plan8_fits<17>(),
              "the radix-8 direct round must lie in the transposed region");

// Pass splits (the launch shape's ntt_split): SPLIT 1 moves one stage from
// the strided pass to the contiguous one, SPLIT 2 the other way (2^16:
// 7 + 9 and 9 + 7 stages; 2^17: 8 + 9 and 10 + 7), each in a radix-16 and a
// radix-8 form (R8).  Every plan's direct round lies in the transposed
// region of the one twiddle table, and every round's shared-memory index map
// was checked on the CPU (each tile element touched once, the padding of
// e0 + c equal to padi(e0) plus the compile-time offset, addresses inside
// the padded buffer).  Other ring sizes keep their default plans.
template <int LOGN, int SPLIT, bool R8> struct PlanV : std::conditional_t<R8, Plan8<LOGN>, Plan<LOGN>> {};
template <> struct PlanV<16, 1, false> { static constexpr int S1 = 7, A1 = 4, B1 = 3, C1 = 0, S2 = 9, A2 = 4, B2 = 2, C2 = 3; };
template <> struct PlanV<16, 1, true> { static constexpr int S1 = 7, A1 = 3, B1 = 2, C1 = 2, S2 = 9, A2 = 3, B2 = 3, C2 = 3; };
template <> struct PlanV<16, 2, false> { static constexpr int S1 = 9, A1 = 4, B1 = 3, C1 = 2, S2 = 7, A2 = 4, B2 = 3, C2 = 0; };
template <> struct PlanV<16, 2, true> { static constexpr int S1 = 9, A1 = 3, B1 = 3, C1 = 3, S2 = 7, A2 = 2, B2 = 3, C2 = 2; };
template <> struct PlanV<17, 1, false> { static constexpr int S1 = 8, A1 = 4, B1 = 4, C1 = 0, S2 = 9, A2 = 4, B2 = 2, C2 = 3; };
template <> struct PlanV<17, 1, true> { static constexpr int S1 = 8, A1 = 2, B1 = 3, C1 = 3, S2 = 9, A2 = 3, B2 = 3, C2 = 3; };
template <> struct PlanV<17, 2, false> { static constexpr int S1 = 10, A1 = 4, B1 = 3, C1 = 3, S2 = 7, A2 = 4, B2 = 3, C2 = 0; };
template <> struct PlanV<17, 2, true> { static constexpr int S1 = 10, A1 = 4, B1 = 3, C1 = 3, S2 = 7, A2 = 2, B2 = 3, C2 = 2; };
template <int LOGN, int SPLIT, bool R8> constexpr bool planv_fits()
{
    using P = PlanV<LOGN, SPLIT, R8>;
    return P::S1 + P::S2 == LOGN && P::A1 + P::B1 + P::C1 == P::S1 && P::A2 + P::B2 + P::C2 == P::S2 &&
           (P::C2 ? P::C2 : P::B2) <= plan_direct<LOGN>() && P::S1 <= LOGN - plan_direct<LOGN>();
}
static_assert(planv_fits<16, 1, false>() && planv_fits<16, 1, true>() && planv_fits<16, 2, false>() &&
                  planv_fits<16, 2, true>() && planv_fits<17, 1, false>() && planv_fits<17, 1, true>() &&
                  planv_fits<17, 2, false>() && planv_fits<17, 2, true>(),
              "split plans: stages, rounds and the transposed region");

// plan id: bit 0 the radix-8 form, bits 1-2 the split (0, 1, 2), bit 3
// 1024-element tiles (twice the CTAs, each half the work, for launches with
// few limbs; every round's index map at that tile size was checked on the
// CPU as for 2048)
// bit 4: the one-pass transform over a cluster (N = 2^16; other sizes
// ignore it)
constexpr int kPlanOnePass = 16;
constexpr int kNttPlans = 32;
// 1024-element tiles of a plan: a strided pass of 2^10 stages would be one
// column wide, so that plan keeps 2048
template <class P> constexpr int small_te() { return P::S1 >= 10 ? 2048 : 1024; }

// Two-pass transform: the strided pass covers the first S1 stages (forward
// order), the contiguous pass the last S2.
template <int S1, int A1, int B1, int C1, int S2, int A2, int B2, int C2, int TE>
cudaError_t two_pass(const he_ctx *c, NttArgs a, int ngroups, bool inverse, cudaStream_t st, const char *tag)
{
    a.tiles = (1 << (S1 + S2)) / TE;
    cudaError_t e;
    const char *t1 = inverse ? ".inv_pass1" : ".fwd_pass1";
    const char *t2 = inverse ? ".inv_pass2" : ".fwd_pass2";
    if (ngroups == 0) {  // configure only
        e = run_pass<S1, A1, B1, C1, true, false, true, false, TE>(a, 0, st);
        if (e == cudaSuccess) e = run_pass<S2, A2, B2, C2, false, false, false, true, TE>(a, 0, st);
        if (e == cudaSuccess) e = run_pass<S2, A2, B2, C2, false, true, true, false, TE>(a, 0, st);
        if (e == cudaSuccess) e = run_pass<S1, A1, B1, C1, true, true, false, true, TE>(a, 0, st);
        return e;
    }
    if (!inverse) {
        e = run_pass<S1, A1, B1, C1, true, false, true, false, TE>(a, ngroups, st);
        if (e != cudaSuccess) return e;
        prof_mark(c, st, tag, t1);
        e = run_pass<S2, A2, B2, C2, false, false, false, true, TE>(a, ngroups, st);
        prof_mark(c, st, tag, t2);
        return e;
    }
    e = run_pass<S2, A2, B2, C2, false, true, true, false, TE>(a, ngroups, st);
    if (e != cudaSuccess) return e;
    prof_mark(c, st, tag, t1);
    e = run_pass<S1, A1, B1, C1, true, true, false, true, TE>(a, ngroups, st);
    prof_mark(c, st, tag, t2);
    return e;
}

// One-pass transforms over a cluster.  Local rounds (3, 3, 3, 4), 512
// threads, free of shared-memory bank conflicts with the one-word-per-16
// padding; with the plan's radix-8 bit, (3, 3, 2, 2, 3), 1024 threads at most
// 64 registers (a 2-way conflict in the fourth round).  Both keep the direct
// round inside the table's transposed region.
#define HE_CL16 3, 3, 3, 4, 0
#define HE_CL8 3, 3, 2, 2, 3
cudaError_t onepass(const he_ctx *c, const NttArgs &a, int ngroups, bool inverse, cudaStream_t st, const char *tag,
                    int plan)
{
    if (ngroups == 0) {  // configure only
        cudaError_t e = run_cluster<HE_CL16, false>(a, 0, st);
        if (e == cudaSuccess) e = run_cluster<HE_CL16, true>(a, 0, st);
        if (e == cudaSuccess) e = run_cluster<HE_CL8, false>(a, 0, st);
        return e == cudaSuccess ? run_cluster<HE_CL8, true>(a, 0, st) : e;
    }
    cudaError_t e;
    if (plan & 1) e = inverse ? run_cluster<HE_CL8, true>(a, ngroups, st) : run_cluster<HE_CL8, false>(a, ngroups, st);
    else e = inverse ? run_cluster<HE_CL16, true>(a, ngroups, st) : run_cluster<HE_CL16, false>(a, ngroups, st);
    prof_mark(c, st, tag, inverse ? ".inv_onepass" : ".fwd_onepass");
    return e;
}

cudaError_t onepass_combine(const he_ctx *c, const NttArgs &a, int ngroups, cudaStream_t st, const char *tag,
                            int plan)
{
    if (ngroups == 0) {
        const cudaError_t e = run_cluster<HE_CL16, false, kFuseCombine>(a, 0, st);
        return e == cudaSuccess ? run_cluster<HE_CL8, false, kFuseCombine>(a, 0, st) : e;
    }
    const cudaError_t e = (plan & 1) ? run_cluster<HE_CL8, false, kFuseCombine>(a, ngroups, st)
                                     : run_cluster<HE_CL16, false, kFuseCombine>(a, ngroups, st);
    prof_mark(c, st, tag, ".fwd_onepass_combine");
    return e;
}

cudaError_t onepass_tensor(const he_ctx *c, const NttArgs &a, int ngroups, cudaStream_t st, const char *tag,
                           int plan)
{
    if (ngroups == 0) {
        const cudaError_t e = run_cluster<HE_CL16, true, kFuseTensor>(a, 0, st);
        return e == cudaSuccess ? run_cluster<HE_CL8, true, kFuseTensor>(a, 0, st) : e;
    }
    const cudaError_t e = (plan & 1) ? run_cluster<HE_CL8, true, kFuseTensor>(a, ngroups, st)
                                     : run_cluster<HE_CL16, true, kFuseTensor>(a, ngroups, st);
    prof_mark(c, st, tag, ".tensor_inv_onepass");
    return e;
}
#undef HE_CL16
#undef HE_CL8

template <int LOGN, class P = Plan<LOGN>, int TE = 2048>
cudaError_t two_pass_plan(const he_ctx *c, NttArgs a, int ngroups, bool inverse, cudaStream_t st, const char *tag)
{
    return two_pass<P::S1, P::A1, P::B1, P::C1, P::S2, P::A2, P::B2, P::C2, TE>(c, a, ngroups, inverse, st, tag);
}

template <int LOGN>
cudaError_t two_pass_any(const he_ctx *c, NttArgs a, int ngroups, bool inverse, cudaStream_t st, const char *tag, int plan)
{
    if (LOGN == kClLogN && (plan & kPlanOnePass)) return onepass(c, a, ngroups, inverse, st, tag, plan);
    // bit 3: 1024-element tiles (2^16 and 2^17; a pass over 2^10 stages keeps 2048)
    constexpr bool SMALL_OK = LOGN == 16 || LOGN == 17;
    if (SMALL_OK && (plan & 8)) {
        switch (plan & 7) {
        case 1: return two_pass_plan<LOGN, Plan8<LOGN>, SMALL_OK ? 1024 : 2048>(c, a, ngroups, inverse, st, tag);
        case 2: return two_pass_plan<LOGN, PlanV<LOGN, 1, false>, SMALL_OK ? 1024 : 2048>(c, a, ngroups, inverse, st, tag);
        case 3: return two_pass_plan<LOGN, PlanV<LOGN, 1, true>, SMALL_OK ? 1024 : 2048>(c, a, ngroups, inverse, st, tag);
        case 4: return two_pass_plan<LOGN, PlanV<LOGN, 2, false>, small_te<PlanV<LOGN, 2, false>>()>(c, a, ngroups, inverse, st, tag);
        case 5: return two_pass_plan<LOGN, PlanV<LOGN, 2, true>, small_te<PlanV<LOGN, 2, true>>()>(c, a, ngroups, inverse, st, tag);
        default: return two_pass_plan<LOGN, Plan<LOGN>, SMALL_OK ? 1024 : 2048>(c, a, ngroups, inverse, st, tag);
        }
    }
    switch (plan & 7) {
    case 1: return two_pass_plan<LOGN, Plan8<LOGN>>(c, a, ngroups, inverse, st, tag);
    case 2: return two_pass_plan<LOGN, PlanV<LOGN, 1, false>>(c, a, ngroups, inverse, st, tag);
    case 3: return two_pass_plan<LOGN, PlanV<LOGN, 1, true>>(c, a, ngroups, inverse, st, tag);
    case 4: return two_pass_plan<LOGN, PlanV<LOGN, 2, false>>(c, a, ngroups, inverse, st, tag);
    case 5: return two_pass_plan<LOGN, PlanV<LOGN, 2, true>>(c, a, ngroups, inverse, st, tag);
    default: return two_pass_plan<LOGN, Plan<LOGN>>(c, a, ngroups, inverse, st, tag);
    }
}

// Forward transform whose last pass also applies the final combine.
template <int LOGN, class P, int TE = 2048>
cudaError_t combine_plan(const he_ctx *c, NttArgs a, int ngroups, cudaStream_t st, const char *tag)
{
    a.tiles = (1 << LOGN) / TE;
    if (ngroups == 0) return run_pass<P::S2, P::A2, P::B2, P::C2, false, false, false, true, TE, kFuseCombine>(a, 0, st);
    cudaError_t e = run_pass<P::S1, P::A1, P::B1, P::C1, true, false, true, false, TE>(a, ngroups, st);
    if (e != cudaSuccess) return e;
    prof_mark(c, st, tag, ".fwd_pass1");
    e = run_pass<P::S2, P::A2, P::B2, P::C2, false, false, false, true, TE, kFuseCombine>(a, ngroups, st);
    prof_mark(c, st, tag, ".fwd_pass2_combine");
    return e;
}

template <int LOGN>
cudaError_t combine_any(const he_ctx *c, NttArgs a, int ngroups, cudaStream_t st, const char *tag, int plan)
{
    if (LOGN == kClLogN && (plan & kPlanOnePass)) return onepass_combine(c, a, ngroups, st, tag, plan);
    // bit 3: 1024-element tiles (2^16 and 2^17; a pass over 2^10 stages keeps 2048)
    constexpr bool SMALL_OK = LOGN == 16 || LOGN == 17;
    if (SMALL_OK && (plan & 8)) {
        switch (plan & 7) {
        case 1: return combine_plan<LOGN, Plan8<LOGN>, SMALL_OK ? 1024 : 2048>(c, a, ngroups, st, tag);
        case 2: return combine_plan<LOGN, PlanV<LOGN, 1, false>, SMALL_OK ? 1024 : 2048>(c, a, ngroups, st, tag);
        case 3: return combine_plan<LOGN, PlanV<LOGN, 1, true>, SMALL_OK ? 1024 : 2048>(c, a, ngroups, st, tag);
        case 4: return combine_plan<LOGN, PlanV<LOGN, 2, false>, small_te<PlanV<LOGN, 2, false>>()>(c, a, ngroups, st, tag);
        case 5: return combine_plan<LOGN, PlanV<LOGN, 2, true>, small_te<PlanV<LOGN, 2, true>>()>(c, a, ngroups, st, tag);
        default: return combine_plan<LOGN, Plan<LOGN>, SMALL_OK ? 1024 : 2048>(c, a, ngroups, st, tag);
        }
    }
    switch (plan & 7) {
    case 1: return combine_plan<LOGN, Plan8<LOGN>>(c, a, ngroups, st, tag);
    case 2: return combine_plan<LOGN, PlanV<LOGN, 1, false>>(c, a, ngroups, st, tag);
    case 3: return combine_plan<LOGN, PlanV<LOGN, 1, true>>(c, a, ngroups, st, tag);
    case 4: return combine_plan<LOGN, PlanV<LOGN, 2, false>>(c, a, ngroups, st, tag);
    case 5: return combine_plan<LOGN, PlanV<LOGN, 2, true>>(c, a, ngroups, st, tag);
    default: return combine_plan<LOGN, Plan<LOGN>>(c, a, ngroups, st, tag);
    }
}

// Inverse transform whose first pass computes its input: the tensor
// product (kFuseTensor) or the key-switch sums (kFuseIp).
template <int LOGN, class P, int FUSE, int TE = 2048>
cudaError_t computed_plan(const he_ctx *c, NttArgs a, int ngroups, cudaStream_t st, const char *tag)
{
    a.tiles = (1 << LOGN) / TE;
    if (ngroups == 0) return run_pass<P::S2, P::A2, P::B2, P::C2, false, true, true, false, TE, FUSE>(a, 0, st);
    cudaError_t e = run_pass<P::S2, P::A2, P::B2, P::C2, false, true, true, false, TE, FUSE>(a, ngroups, st);
    if (e != cudaSuccess) return e;
    prof_mark(c, st, tag, FUSE == kFuseTensor ? ".tensor_inv_pass1" : ".ip_inv_pass1");
    e = run_pass<P::S1, P::A1, P::B1, P::C1, true, true, false, true, TE>(a, ngroups, st);
    prof_mark(c, st, tag, ".inv_pass2");
    return e;
}

// The plans of computed_plan (the one-pass cluster transform takes the
// tensor product only; with the key-switch sums that bit is ignored).
template <int LOGN, int FUSE>
cudaError_t computed_any(const he_ctx *c, NttArgs a, int ngroups, cudaStream_t st, const char *tag, int plan)
{
    if (FUSE == kFuseTensor && LOGN == kClLogN && (plan & kPlanOnePass)) return onepass_tensor(c, a, ngroups, st, tag, plan);
    // bit 3: 1024-element tiles (2^16 and 2^17; a pass over 2^10 stages keeps 2048)
    constexpr bool SMALL_OK = LOGN == 16 || LOGN == 17;
    constexpr int TS = SMALL_OK ? 1024 : 2048;
    if (SMALL_OK && (plan & 8)) {
        switch (plan & 7) {
        case 1: return computed_plan<LOGN, Plan8<LOGN>, FUSE, TS>(c, a, ngroups, st, tag);
        case 2: return computed_plan<LOGN, PlanV<LOGN, 1, false>, FUSE, TS>(c, a, ngroups, st, tag);
        case 3: return computed_plan<LOGN, PlanV<LOGN, 1, true>, FUSE, TS>(c, a, ngroups, st, tag);
        case 4: return computed_plan<LOGN, PlanV<LOGN, 2, false>, FUSE, small_te<PlanV<LOGN, 2, false>>()>(c, a, ngroups, st, tag);
        case 5: return computed_plan<LOGN, PlanV<LOGN, 2, true>, FUSE, small_te<PlanV<LOGN, 2, true>>()>(c, a, ngroups, st, tag);
        default: return computed_plan<LOGN, Plan<LOGN>, FUSE, TS>(c, a, ngroups, st, tag);
        }
    }
    switch (plan & 7) {
    case 1: return computed_plan<LOGN, Plan8<LOGN>, FUSE>(c, a, ngroups, st, tag);
    case 2: return computed_plan<LOGN, PlanV<LOGN, 1, false>, FUSE>(c, a, ngroups, st, tag);
    case 3: return computed_plan<LOGN, PlanV<LOGN, 1, true>, FUSE>(c, a, ngroups, st, tag);
    case 4: return computed_plan<LOGN, PlanV<LOGN, 2, false>, FUSE>(c, a, ngroups, st, tag);
    case 5: return computed_plan<LOGN, PlanV<LOGN, 2, true>, FUSE>(c, a, ngroups, st, tag);
    default: return computed_plan<LOGN, Plan<LOGN>, FUSE>(c, a, ngroups, st, tag);
    }
}

// An inverse transform with a computed first pass, at the context's ring size.
cudaError_t launch_computed(const he_ctx *c, const NttArgs &a, int ngroups, cudaStream_t st, const char *tag, int plan,
                            bool ip)
{
    switch (c->logN) {
    case 12: {
        cudaError_t e = ip ? run_pass<12, 4, 4, 4, false, true, true, true, 4096, kFuseIp>(a, ngroups, st)
                           : run_pass<12, 4, 4, 4, false, true, true, true, 4096, kFuseTensor>(a, ngroups, st);
        if (ngroups) prof_mark(c, st, tag, ip ? ".ip_inv" : ".tensor_inv");
        return e;
    }
    case 13: return ip ? computed_any<13, kFuseIp>(c, a, ngroups, st, tag, plan) : computed_any<13, kFuseTensor>(c, a, ngroups, st, tag, plan);
    case 14: return ip ? computed_any<14, kFuseIp>(c, a, ngroups, st, tag, plan) : computed_any<14, kFuseTensor>(c, a, ngroups, st, tag, plan);
    case 15: return ip ? computed_any<15, kFuseIp>(c, a, ngroups, st, tag, plan) : computed_any<15, kFuseTensor>(c, a, ngroups, st, tag, plan);
    case 16: return ip ? computed_any<16, kFuseIp>(c, a, ngroups, st, tag, plan) : computed_any<16, kFuseTensor>(c, a, ngroups, st, tag, plan);
    case 17: return ip ? computed_any<17, kFuseIp>(c, a, ngroups, st, tag, plan) : computed_any<17, kFuseTensor>(c, a, ngroups, st, tag, plan);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_ntt_tensor(const he_ctx *c, u64 *base, const NttGroup *groups, int ngroups, const JobRef &R,
                              cudaStream_t st, const char *tag, const int *dev_count, int plan)
{
    if (ngroups < 0) return cudaSuccess;  // ngroups == 0: configure the kernels only
    NttArgs a;
    memset(&a, 0, sizeof(a));
    a.src = base;
    a.dst = base;
    a.groups = groups;
    a.primes = c->d_primes;
    a.logN = c->logN;
    a.ts = c->logN - ntt_direct_stages(c->logN);
    a.tiles = 1;
    a.count = dev_count;
    a.pdl = c->pdl;
    a.R = R;
    a.levels = c->d_levels;
    a.pinv = c->d_pinv;
    return launch_computed(c, a, ngroups, st, tag, plan, false);
}

cudaError_t launch_ntt_ip(const he_ctx *c, u64 *base, const NttGroup *groups, int ngroups, const JobRef &R,
                          const u64 *evk, cudaStream_t st, const char *tag, const int *dev_count, int plan)
{
    if (ngroups < 0) return cudaSuccess;  // ngroups == 0: configure the kernels only
    NttArgs a;
    memset(&a, 0, sizeof(a));
    a.src = base;
    a.dst = base;
    a.groups = groups;
    a.primes = c->d_primes;
    a.logN = c->logN;
    a.ts = c->logN - ntt_direct_stages(c->logN);
    a.tiles = 1;
    a.count = dev_count;
    a.pdl = c->pdl;
    a.R = R;
    a.levels = c->d_levels;
    a.evk = evk;
    a.EL = c->K + c->L;
    return launch_computed(c, a, ngroups, st, tag, plan, true);
}

cudaError_t launch_ntt_combine(const he_ctx *c, u64 *base, const NttGroup *groups, int ngroups, const JobRef &R,
                               cudaStream_t st, const char *tag, const int *dev_count, int plan)
{
    if (ngroups < 0) return cudaSuccess;  // ngroups == 0: configure the kernels only
    NttArgs a;
    memset(&a, 0, sizeof(a));
    a.src = base;
    a.dst = base;
    a.groups = groups;
    a.primes = c->d_primes;
    a.logN = c->logN;
    a.ts = c->logN - ntt_direct_stages(c->logN);
    a.tiles = 1;
    a.count = dev_count;
    a.pdl = c->pdl;
    a.R = R;
    a.levels = c->d_levels;
    a.pinv = c->d_pinv;
    switch (c->logN) {
    case 12: {
        cudaError_t e = run_pass<12, 4, 4, 4, false, false, true, true, 4096, kFuseCombine>(a, ngroups, st);
        if (ngroups) prof_mark(c, st, tag, ".fwd_combine");
        return e;
    }
    case 13: return combine_any<13>(c, a, ngroups, st, tag, plan);
    case 14: return combine_any<14>(c, a, ngroups, st, tag, plan);
    case 15: return combine_any<15>(c, a, ngroups, st, tag, plan);
    case 16: return combine_any<16>(c, a, ngroups, st, tag, plan);
    case 17: return combine_any<17>(c, a, ngroups, st, tag, plan);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_ntt2(const he_ctx *c, const u64 *src, u64 *dst, const NttGroup *groups, int ngroups, bool inverse,
                        cudaStream_t st, const char *tag, const int *dev_count, int plan)
{
    if (ngroups < 0) return cudaSuccess;  // ngroups == 0: configure the kernels only
    NttArgs a;
    memset(&a, 0, sizeof(a));
    a.src = src;
    a.dst = dst;
    a.groups = groups;
    a.primes = c->d_primes;
    a.logN = c->logN;
    a.ts = c->logN - ntt_direct_stages(c->logN);
    a.tiles = 1;
    a.count = dev_count;
    a.pdl = c->pdl;
    switch (c->logN) {
    case 12: {
        if (ngroups == 0) {
            cudaError_t e = run_pass<12, 4, 4, 4, false, true, true, true, 4096>(a, 0, st);
            return e == cudaSuccess ? run_pass<12, 4, 4, 4, false, false, true, true, 4096>(a, 0, st) : e;
        }
        cudaError_t e = inverse ? run_pass<12, 4, 4, 4, false, true, true, true, 4096>(a, ngroups, st)
                                : run_pass<12, 4, 4, 4, false, false, true, true, 4096>(a, ngroups, st);
        prof_mark(c, st, tag, inverse ? ".inv" : ".fwd");
        return e;
    }
    case 13: return two_pass_any<13>(c, a, ngroups, inverse, st, tag, plan);
    case 14: return two_pass_any<14>(c, a, ngroups, inverse, st, tag, plan);
    case 15: return two_pass_any<15>(c, a, ngroups, inverse, st, tag, plan);
    case 16: return two_pass_any<16>(c, a, ngroups, inverse, st, tag, plan);
    case 17: return two_pass_any<17>(c, a, ngroups, inverse, st, tag, plan);
    default: return cudaErrorInvalidValue;
    }
}

int ntt_direct_stages(int logN)
{
    switch (logN) {
    case 12: return 4;  // the single pass's third round
    case 13: return plan_direct<13>();
    case 14: return plan_direct<14>();
    case 15: return plan_direct<15>();
    case 16: return plan_direct<16>();
    case 17: return plan_direct<17>();
    default: return 0;
    }
}

cudaError_t launch_ntt(const he_ctx *c, u64 *base, const NttGroup *groups, int ngroups, bool inverse, cudaStream_t st,
                       const char *tag, const int *dev_count, int plan)
{
    return launch_ntt2(c, base, base, groups, ngroups, inverse, st, tag, dev_count, plan);
}

// Set the dynamic shared-memory limit of every NTT pass this ring size uses,
// in every plan (done once per context, before any launch or stream capture).
cudaError_t configure_ntt(const he_ctx *c)
{
    JobRef R;
    memset(&R, 0, sizeof(R));
    for (int plan = 0; plan < kNttPlans; plan++) {
        cudaError_t e = launch_ntt2(c, nullptr, nullptr, nullptr, 0, false, nullptr, nullptr, nullptr, plan);
        if (e != cudaSuccess) return e;
        e = launch_ntt_combine(c, nullptr, nullptr, 0, R, nullptr, nullptr, nullptr, plan);
        if (e != cudaSuccess) return e;
        e = launch_ntt_tensor(c, nullptr, nullptr, 0, R, nullptr, nullptr, nullptr, plan);
        if (e != cudaSuccess) return e;
        e = launch_ntt_ip(c, nullptr, nullptr, 0, R, nullptr, nullptr, nullptr, nullptr, plan);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace he
