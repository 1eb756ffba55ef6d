// host_params.cpp -- context construction: primes, roots, twiddle tables,
// base-conversion constants, per-level workspace layouts and NTT job lists,
// and the upload of every device table into one arena.
//
// Parameter rules (the paper is silent on the RNS choices):
//   * q_0 > q_1 > ... : the L largest primes below 2^q_bits with q = 1 mod 2N
//   * p_0 > p_1 > ... : the K largest primes below 2^p_bits with p = 1 mod 2N
//                       that are not ciphertext primes
//   * psi             : the smallest primitive 2N-th root of unity mod each prime
//   * digits          : I_j = {j*alpha, ..., min((j+1)*alpha, l) - 1}
// Twiddles follow Algo 3's table TB_W[m + j] = psi^bitrev(m + j) and the iNTT's
// TB_invW; every constant carries its Shoup companion (Algo 2).
#include <algorithm>
#include <cstring>

#include "he_internal.h"
#include "host_math.h"

namespace he {

using namespace hm;

static std::vector<u64> find_primes(int logN, int bits, int count, const std::vector<u64> &skip)
{
    std::vector<u64> out;
    const u64 step = 2ull << logN;
    u64 top = (1ull << bits) - 1;
    u64 c = top - (top - 1) % step;  // largest c <= top with c = 1 mod 2N
    while ((int)out.size() < count && c > step) {
        if (std::find(skip.begin(), skip.end(), c) == skip.end() && is_prime(c)) out.push_back(c);
        c -= step;
    }
    return out;
}

// Smallest primitive 2N-th root: take a generator g of Z_q^*, psi0 = g^((q-1)/2N);
// the primitive 2N-th roots are psi0^k for odd k.
static u64 smallest_psi(u64 q, int logN)
{
    const u64 twoN = 2ull << logN;
    std::vector<u64> f = prime_factors(q - 1);
    u64 g = 2;
    for (;; g++) {
        bool gen = true;
        for (u64 p : f)
            if (pw(g, (q - 1) / p, q) == 1) { gen = false; break; }
        if (gen) break;
    }
    u64 psi0 = pw(g, (q - 1) / twoN, q);
    u64 sq = mul(psi0, psi0, q), best = psi0, cur = psi0;
    for (u64 k = 1; k < twoN / 2; k++) {
        cur = mul(cur, sq, q);
        best = std::min(best, cur);
    }
    return best;
}

static ulonglong2 pair(u64 v, u64 m) { return make_ulonglong2(v, shoup(v, m)); }

// base-conversion constant stored split at bit 28 for the kernels' lazy MACs
static u64 split28(u64 b) { return (b & 0xFFFFFFFull) | ((b >> 28) << 32); }

std::vector<NttGroup> group_jobs(const std::vector<NttJob> &jobs, int cap)
{
    cap = std::max(1, std::min(cap, kGroupMax));
    std::vector<NttGroup> out;
    std::vector<int> open_for_prime;  // index into out of the group being filled, per prime
    for (const NttJob &j : jobs) {
        if (j.prime >= open_for_prime.size()) open_for_prime.resize(j.prime + 1, -1);
        int g = open_for_prime[j.prime];
        if (g < 0 || out[g].nl == (unsigned)cap) {
            NttGroup ng;
            memset(&ng, 0, sizeof(ng));
            ng.prime = j.prime;
            out.push_back(ng);
            g = (int)out.size() - 1;
            open_for_prime[j.prime] = g;
        }
        NttGroup &G = out[g];
        G.src[G.nl] = j.src;
        G.dst[G.nl] = j.dst;
        G.scale[G.nl] = j.scale;
        G.scale_sh[G.nl] = j.scale_sh;
        G.job[G.nl] = j.job;
        G.ci[G.nl] = j.ci;
        G.cd[G.nl] = j.cd;
        G.cks[G.nl] = j.cks;
        G.nl++;
    }
    // groups of one prime next to each other: their CTAs run at the same time
    // and read that prime's twiddle runs from L2 instead of each from DRAM
    std::stable_sort(out.begin(), out.end(), [](const NttGroup &a, const NttGroup &b) { return a.prime < b.prime; });
    return out;
}

static WsLayout layout_for(int l, int K, int alpha)
{
    int beta = (l + alpha - 1) / alpha;
    int E = K + l;
    WsLayout w;
    w.d0 = 0;
    w.d1 = (size_t)l;
    w.d2 = 2 * (size_t)l;
    w.y = 3 * (size_t)l;
    w.u = 4 * (size_t)l;
    w.ks = w.u + (size_t)beta * E;
    w.ys = w.ks + 2 * (size_t)E;
    w.r = w.ys + 2 * (size_t)K;
    w.z = w.r + 4;
    w.total = w.z + 2 * (size_t)l;
    return w;
}

int build_context(he_ctx *c, const he_params *p, bool device)
{
    // q_bits, p_bits <= 57 keep every base-conversion accumulator (at most 16
    // products of a residue and a constant) below barrett128's 2^(b+61) bound.
    if (p->logN < 12 || p->logN > 17 || p->L < 1 || p->L > kMaxL || p->K < 1 || p->K > kMaxK ||
        p->alpha < 1 || p->alpha > 16 || p->q_bits < 30 || p->q_bits > 57 || p->p_bits < 30 ||
        p->p_bits > 57 || p->h < 1 || p->h > (1 << p->logN) || !(p->sigma > 0))
        return HE_EINVAL;
    c->prm = *p;
    c->logN = p->logN;
    c->N = 1 << p->logN;
    c->L = p->L;
    c->K = p->K;
    c->alpha = p->alpha;
    c->dnum = (p->L + p->alpha - 1) / p->alpha;
    c->E = p->K + p->L;
    c->device = device;
    if (c->dnum > kMaxDigits) return HE_EINVAL;
    auto pad_width = [](int v) { return v <= 2 ? v : v <= 4 ? 4 : v <= 8 ? 8 : v <= 12 ? 12 : 16; };
    c->AP = pad_width(p->alpha);
    c->KP = pad_width(p->K);

    std::vector<u64> q = find_primes(p->logN, p->q_bits, p->L, {});
    if ((int)q.size() != p->L) return HE_EINVAL;
    std::vector<u64> sp = find_primes(p->logN, p->p_bits, p->K, q);
    if ((int)sp.size() != p->K) return HE_EINVAL;
    c->ext = sp;
    c->ext.insert(c->ext.end(), q.begin(), q.end());
    const int N = c->N, K = c->K, L = c->L, E = c->E, logN = c->logN;

    // the ciphertext primes descend, so a rescale residue r < q_{l-1} is
    // already reduced mod every q_i with i < l-1.

    c->psi.resize(E);
    c->w.assign(E, {});
    c->wsh.assign(E, {});
    c->iw.assign(E, {});
    c->iwsh.assign(E, {});
    c->ninv.resize(E);
    c->ninv_sh.resize(E);
    for (int e = 0; e < E; e++) {
        u64 m = c->ext[e];
        u64 psi = smallest_psi(m, logN);
        c->psi[e] = psi;
        u64 ipsi = inv(psi, m);
        std::vector<u64> pow_f(N), pow_i(N);
        pow_f[0] = pow_i[0] = 1;
        for (int k = 1; k < N; k++) {
            pow_f[k] = mul(pow_f[k - 1], psi, m);
            pow_i[k] = mul(pow_i[k - 1], ipsi, m);
        }
        auto &W = c->w[e], &Ws = c->wsh[e], &IW = c->iw[e], &IWs = c->iwsh[e];
        W.resize(N); Ws.resize(N); IW.resize(N); IWs.resize(N);
        for (int k = 0; k < N; k++) {
            u64 br = bitrev((u64)k, logN);
            W[k] = pow_f[br];
            Ws[k] = shoup(W[k], m);
            IW[k] = pow_i[br];
            IWs[k] = shoup(IW[k], m);
        }
        c->ninv[e] = inv((u64)N % m, m);
        c->ninv_sh[e] = shoup(c->ninv[e], m);
    }

    // ModDown constants
    c->PB.assign((size_t)L * c->KP, 0);
    c->PBP.assign((size_t)L * c->KP, 0);
    c->pinv.resize(L);
    c->phat_inv.resize(K);
    for (int k = 0; k < K; k++) {
        u64 pk = c->ext[k], v = 1;
        for (int k2 = 0; k2 < K; k2++)
            if (k2 != k) v = mul(v, c->ext[k2] % pk, pk);
        c->phat_inv[k] = pair(inv(v, pk), pk);
    }
    for (int i = 0; i < L; i++) {
        u64 qi = c->ext[K + i], P = 1;
        for (int k = 0; k < K; k++) {
            u64 v = 1;
            for (int k2 = 0; k2 < K; k2++)
                if (k2 != k) v = mul(v, c->ext[k2] % qi, qi);
            c->PB[(size_t)i * c->KP + k] = split28(v);
            P = mul(P, c->ext[k] % qi, qi);
        }
        c->pinv[i] = pair(inv(P, qi), qi);
        for (int k = 0; k < K; k++) {
            u64 v = 1;
            for (int k2 = 0; k2 < K; k2++)
                if (k2 != k) v = mul(v, c->ext[k2] % qi, qi);
            c->PBP[(size_t)i * c->KP + k] = split28(mul(v, c->pinv[i].x, qi));
        }
    }

    // per level
    c->host_levels.assign(L + 1, HostLevel());
    for (int l = 1; l <= L; l++) {
        HostLevel &H = c->host_levels[l];
        const int beta = (l + c->alpha - 1) / c->alpha, El = K + l;
        const int A = c->AP;
        H.ws = layout_for(l, K, c->alpha);
        const WsLayout &W = H.ws;
        // ModUp tables and the iNTT scale N^-1 * Qhat_{j,i}^-1
        H.modupB.assign((size_t)beta * El * A, 0);
        for (int j = 0; j < beta; j++) {
            int lo = j * c->alpha, hi = std::min((j + 1) * c->alpha, l);
            for (int i = lo; i < hi; i++) {
                u64 qi = c->ext[K + i], qh = 1;
                for (int i2 = lo; i2 < hi; i2++)
                    if (i2 != i) qh = mul(qh, c->ext[K + i2] % qi, qi);
                u64 sc = mul(c->ninv[K + i], inv(qh, qi), qi);
                // tensor fields (the fused first pass): limb i, product d2, keep d0..d2
                H.intt1.push_back(NttJob{(unsigned)(W.d2 + i), (unsigned)(W.y + i), (unsigned)(K + i), 0, sc,
                                         shoup(sc, qi), 0, (unsigned)i | (2u << 16) | (1u << 18), 0, 0});
            }
            for (int e = 0; e < El; e++) {
                bool own = e >= K && (e - K) >= lo && (e - K) < hi;
                if (own) continue;
                u64 t = c->ext[e];
                for (int i = lo; i < hi; i++) {
                    u64 v = 1;
                    for (int i2 = lo; i2 < hi; i2++)
                        if (i2 != i) v = mul(v, c->ext[K + i2] % t, t);
                    H.modupB[((size_t)j * El + e) * A + (i - lo)] = split28(v);
                }
                H.ntt_up.push_back(NttJob{(unsigned)(W.u + (size_t)j * El + e), (unsigned)(W.u + (size_t)j * El + e),
                                          (unsigned)e, 0, 0, 0});
            }
        }
        const u64 ql = c->ext[K + l - 1];
        H.intt1f = H.intt1;
        for (int h = 0; h < 2; h++)
            H.intt1f.push_back(NttJob{(unsigned)((h ? W.d1 : W.d0) + l - 1), (unsigned)(W.r + h), (unsigned)(K + l - 1),
                                      0, c->ninv[K + l - 1], c->ninv_sh[K + l - 1], 0,
                                      (unsigned)(l - 1) | ((unsigned)h << 16), 0, 0});
        for (int h = 0; h < 2; h++)
            for (int k = 0; k < K; k++) {
                u64 pk = c->ext[k];
                u64 sc = mul(c->ninv[k], c->phat_inv[k].x, pk);
                // ci: the key-switch row and half (the first pass that computes the sums itself)
                H.intt2.push_back(NttJob{(unsigned)(W.ks + (size_t)h * El + k), (unsigned)(W.ys + (size_t)h * K + k),
                                         (unsigned)k, 0, sc, shoup(sc, pk), 0, (unsigned)k | ((unsigned)h << 16), 0, 0});
            }
        H.intt2f = H.intt2;
        for (int h = 0; h < 2; h++)
            H.intt2f.push_back(NttJob{(unsigned)(W.ks + (size_t)h * El + K + l - 1), (unsigned)(W.r + 2 + h),
                                      (unsigned)(K + l - 1), 0, c->ninv[K + l - 1], c->ninv_sh[K + l - 1], 0,
                                      (unsigned)(K + l - 1) | ((unsigned)h << 16), 0, 0});
        // one division by M = P q_{l-1}: y_k = x_k [Mhat_k^-1]_{p_k}, Mhat_k = Phat_k q_{l-1};
        // the conversion constants [Mhat_k P^-1]_{q_i} = [Phat_k P^-1 q_{l-1}]_{q_i}
        for (int h = 0; h < 2; h++)
            for (int k = 0; k < K; k++) {
                u64 pk = c->ext[k];
                u64 sc = mul(mul(c->ninv[k], c->phat_inv[k].x, pk), inv(ql % pk, pk), pk);
                H.intt2pq.push_back(NttJob{(unsigned)(W.ks + (size_t)h * El + k),
                                           (unsigned)(W.ys + (size_t)h * K + k), (unsigned)k, 0, sc, shoup(sc, pk), 0,
                                           (unsigned)k | ((unsigned)h << 16), 0, 0});
            }
        for (int h = 0; h < 2; h++) H.intt2pq.push_back(H.intt2f[(size_t)2 * K + h]);
        H.pbpq.assign((size_t)std::max(l - 1, 1) * c->KP, 0);
        for (int i = 0; i + 1 < l; i++) {
            u64 qi = c->ext[K + i];
            for (int k = 0; k < K; k++) {
                u64 v = 1;
                for (int k2 = 0; k2 < K; k2++)
                    if (k2 != k) v = mul(v, c->ext[k2] % qi, qi);
                H.pbpq[(size_t)i * c->KP + k] = split28(mul(mul(v, c->pinv[i].x, qi), ql % qi, qi));
            }
        }
        for (int h = 0; h < 2; h++)
            for (int i = 0; i < l; i++)
                H.ntt_conv.push_back(NttJob{(unsigned)(W.z + (size_t)h * l + i), (unsigned)(W.z + (size_t)h * l + i),
                                            (unsigned)(K + i), 0, 0, 0});
        for (int h = 0; h < 2; h++)
            for (int i = 0; i + 1 < l; i++)
                H.ntt_z.push_back(NttJob{(unsigned)(W.z + (size_t)h * (l - 1) + i),
                                         (unsigned)(W.z + (size_t)h * (l - 1) + i), (unsigned)(K + i), 0, 0, 0, 0,
                                         ((unsigned)h << 31) | (unsigned)i, (unsigned)((h ? W.d1 : W.d0) + i),
                                         (unsigned)(W.ks + (size_t)h * El + K + i)});
        // rescale on its own: src offsets are relative to the input ciphertext
        for (int h = 0; h < 2; h++)
            H.rs_intt.push_back(NttJob{(unsigned)((size_t)h * l + l - 1), (unsigned)(W.r + h), (unsigned)(K + l - 1), 0,
                                       c->ninv[K + l - 1], c->ninv_sh[K + l - 1]});
        for (int h = 0; h < 2; h++)
            for (int i = 0; i + 1 < l; i++)
                H.rs_ntt.push_back(NttJob{(unsigned)(W.r + h), (unsigned)(W.z + (size_t)h * (l - 1) + i), (unsigned)(K + i),
                                          0, 0, 0});
        H.qinv_last.resize(l > 1 ? l - 1 : 1);
        H.pinv_qinv.resize(l > 1 ? l - 1 : 1);
        for (int i = 0; i + 1 < l; i++) {
            u64 qi = c->ext[K + i];
            u64 qinv = inv(ql % qi, qi);
            H.qinv_last[i] = pair(qinv, qi);
            H.pinv_qinv[i] = pair(mul(qinv, c->pinv[i].x, qi), qi);
        }
    }
    if (!device) return HE_OK;

    // ---- device arena -------------------------------------------------------
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_primes = take(sizeof(DevPrime) * E);
    std::vector<size_t> o_w(E), o_iw(E);
    for (int e = 0; e < E; e++) {
        o_w[e] = take(sizeof(ulonglong2) * N);
        o_iw[e] = take(sizeof(ulonglong2) * N);
    }
    const size_t o_PB = take(sizeof(u64) * c->PB.size());
    const size_t o_PBP = take(sizeof(u64) * c->PBP.size());
    const size_t o_pinv = take(sizeof(ulonglong2) * L);
    const size_t o_levels = take(sizeof(DevLevel) * (L + 1));
    // per level and group cap: the nine NTT group lists
    constexpr int NL = 10;  // job lists per level
    struct LvlOff { size_t modupB, qinv, pq, pbpq, j[kGroupMax][NL]; };
    std::vector<LvlOff> lo(L + 1);
    std::vector<std::vector<std::vector<std::vector<NttGroup>>>> gl(
        L + 1, std::vector<std::vector<std::vector<NttGroup>>>(kGroupMax, std::vector<std::vector<NttGroup>>(NL)));
    for (int l = 1; l <= L; l++) {
        HostLevel &H = c->host_levels[l];
        lo[l].modupB = take(sizeof(u64) * H.modupB.size());
        lo[l].qinv = take(sizeof(ulonglong2) * H.qinv_last.size());
        lo[l].pq = take(sizeof(ulonglong2) * H.pinv_qinv.size());
        lo[l].pbpq = take(sizeof(u64) * H.pbpq.size());
        const std::vector<NttJob> *lists[NL] = {&H.intt1, &H.intt1f, &H.ntt_up, &H.intt2, &H.intt2f,
                                                &H.ntt_conv, &H.ntt_z, &H.rs_intt, &H.rs_ntt, &H.intt2pq};
        for (int cap = 1; cap <= kGroupMax; cap++)
            for (int t = 0; t < NL; t++) {
                gl[l][cap - 1][t] = group_jobs(*lists[t], cap);
                lo[l].j[cap - 1][t] = take(sizeof(NttGroup) * std::max<size_t>(1, gl[l][cap - 1][t].size()));
            }
    }
    c->arena_bytes = off;
    if (cudaGetDevice(&c->device_id) != cudaSuccess) return HE_ECUDA;
    if (cudaMalloc(&c->arena, off) != cudaSuccess) return HE_ECUDA;
    std::vector<unsigned char> img(off, 0);
    char *base = (char *)c->arena;
    std::vector<DevPrime> dp(E);
    const int direct = ntt_direct_stages(logN);
    if (direct <= 0) return HE_EINVAL;
    const int sd = logN - direct;  // first stage with transposed runs
    for (int e = 0; e < E; e++) {
        u64 m = c->ext[e];
        int b = bitlen(m);
        dp[e].q = m;
        dp[e].q2 = 2 * m;
        dp[e].q4 = 4 * m;
        dp[e].r64 = (u64)((((u128)1) << 64) / m);
        dp[e].s = (unsigned)(b - 2);
        dp[e].mu = (u64)(((u128)1 << (64 + b - 2)) / m);
        dp[e].pad = 0;
        dp[e].w = (const ulonglong2 *)(base + o_w[e]);
        dp[e].iw = (const ulonglong2 *)(base + o_iw[e]);
        ulonglong2 *W = (ulonglong2 *)(img.data() + o_w[e]);
        ulonglong2 *IW = (ulonglong2 *)(img.data() + o_iw[e]);
        for (int k = 0; k < N; k++) {
            W[k] = make_ulonglong2(c->w[e][k], c->wsh[e][k]);
            IW[k] = make_ulonglong2(c->iw[e][k], c->iwsh[e][k]);
        }
        // The last `direct` stages' runs are stored transposed (the NTT's
        // contiguous pass reads them one entry per thread): stage m = 2^sigma,
        // lp = sigma - sd, entry m + T 2^lp + j moves to m + j 2^sd + T.
        for (int sigma = sd; sigma < logN; sigma++) {
            const int lp = sigma - sd;
            const size_t m = (size_t)1 << sigma;
            for (size_t T = 0; T < ((size_t)1 << sd); T++)
                for (size_t j = 0; j < ((size_t)1 << lp); j++) {
                    const size_t from = m + (T << lp) + j, to = m + (j << sd) + T;
                    W[to] = make_ulonglong2(c->w[e][from], c->wsh[e][from]);
                    IW[to] = make_ulonglong2(c->iw[e][from], c->iwsh[e][from]);
                }
        }
    }
    memcpy(img.data() + o_primes, dp.data(), sizeof(DevPrime) * E);
    memcpy(img.data() + o_PB, c->PB.data(), sizeof(u64) * c->PB.size());
    memcpy(img.data() + o_PBP, c->PBP.data(), sizeof(u64) * c->PBP.size());
    memcpy(img.data() + o_pinv, c->pinv.data(), sizeof(ulonglong2) * L);
    c->dev_levels.assign(L + 1, DevLevel());
    c->jobs.assign(L + 1, LevelJobs());
    for (int cap = 0; cap < kGroupMax; cap++) c->jobs_cap[cap].assign(L + 1, LevelJobs());
    for (int l = 1; l <= L; l++) {
        HostLevel &H = c->host_levels[l];
        DevLevel &D = c->dev_levels[l];
        memset(&D, 0, sizeof(D));
        D.l = l;
        D.beta = (l + c->alpha - 1) / c->alpha;
        D.E = K + l;
        D.A = c->AP;
        const WsLayout &Wl = H.ws;
        D.o_d0 = (unsigned)Wl.d0; D.o_d1 = (unsigned)Wl.d1; D.o_d2 = (unsigned)Wl.d2; D.o_y = (unsigned)Wl.y;
        D.o_u = (unsigned)Wl.u; D.o_ks = (unsigned)Wl.ks; D.o_ys = (unsigned)Wl.ys; D.o_r = (unsigned)Wl.r;
        D.o_z = (unsigned)Wl.z; D.o_total = (unsigned)Wl.total;
        for (int j = 0; j < D.beta; j++) {
            D.dig_lo[j] = j * c->alpha;
            D.dig_n[j] = std::min((j + 1) * c->alpha, l) - j * c->alpha;
        }
        memcpy(img.data() + lo[l].modupB, H.modupB.data(), sizeof(u64) * H.modupB.size());
        memcpy(img.data() + lo[l].qinv, H.qinv_last.data(), sizeof(ulonglong2) * H.qinv_last.size());
        memcpy(img.data() + lo[l].pq, H.pinv_qinv.data(), sizeof(ulonglong2) * H.pinv_qinv.size());
        memcpy(img.data() + lo[l].pbpq, H.pbpq.data(), sizeof(u64) * H.pbpq.size());
        D.modupB = (const u64 *)(base + lo[l].modupB);
        D.qinv_last = (const ulonglong2 *)(base + lo[l].qinv);
        D.pinv_qinv = (const ulonglong2 *)(base + lo[l].pq);
        D.pbpq = (const u64 *)(base + lo[l].pbpq);
        for (int cap = 1; cap <= kGroupMax; cap++) {
            const NttGroup *dptr[NL];
            int cnt[NL];
            for (int t = 0; t < NL; t++) {
                const std::vector<NttGroup> &G = gl[l][cap - 1][t];
                if (!G.empty()) memcpy(img.data() + lo[l].j[cap - 1][t], G.data(), sizeof(NttGroup) * G.size());
                dptr[t] = (const NttGroup *)(base + lo[l].j[cap - 1][t]);
                cnt[t] = (int)G.size();
            }
            LevelJobs &J = c->jobs_cap[cap - 1][l];
            J.intt1 = dptr[0];    J.n_intt1 = cnt[0];
            J.intt1f = dptr[1];   J.n_intt1f = cnt[1];
            J.ntt_up = dptr[2];   J.n_ntt_up = cnt[2];
            J.intt2 = dptr[3];    J.n_intt2 = cnt[3];
            J.intt2f = dptr[4];   J.n_intt2f = cnt[4];
            J.ntt_conv = dptr[5]; J.n_ntt_conv = cnt[5];
            J.ntt_z = dptr[6];    J.n_ntt_z = cnt[6];
            J.rs_intt = dptr[7];  J.n_rs_intt = cnt[7];
            J.rs_ntt = dptr[8];   J.n_rs_ntt = cnt[8];
            J.intt2pq = dptr[9];  J.n_intt2pq = cnt[9];
        }
    }
    c->jobs = c->jobs_cap[c->group_cap - 1];
    memcpy(img.data() + o_levels, c->dev_levels.data(), sizeof(DevLevel) * (L + 1));
    if (cudaMemcpy(c->arena, img.data(), off, cudaMemcpyHostToDevice) != cudaSuccess) return HE_ECUDA;
    c->d_primes = (DevPrime *)(base + o_primes);
    c->d_PB = (const u64 *)(base + o_PB);
    c->d_PBP = (const u64 *)(base + o_PBP);
    c->d_pinv = (const ulonglong2 *)(base + o_pinv);
    c->d_levels = (DevLevel *)(base + o_levels);
    if (configure_ntt(c) != cudaSuccess) return HE_ECUDA;
    return HE_OK;
}

}  // namespace he
