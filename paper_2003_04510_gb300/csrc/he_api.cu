// he_api.cu -- the C ABI entry points: context lifetime, workspace sizing,
// and the orchestration of HE Mul / rescale as a sequence of kernels on the
// caller's stream.  No entry point allocates device memory on the hot path:
// the caller passes the workspace.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "he_internal.h"

using namespace he;

namespace he {

thread_local std::vector<int> *capture_log = nullptr;
thread_local int capture_tag = kTagFixed;

void prof_mark(const he_ctx *c, cudaStream_t st, const char *tag, const char *suffix)
{
    if (!c->prof || c->prof_used >= c->prof_pool.size()) return;
    std::string name = tag ? tag : "";
    if (suffix) name += suffix;
    c->prof_names[c->prof_used] = name;
    cudaEventRecord(c->prof_pool[c->prof_used], st);
    c->prof_used++;
}

std::vector<IpGroup> ip_groups(const int *levels, int count, int per)
{
    per = std::max(1, std::min(per, kIpJobsMax));
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return levels[a] > levels[b]; });
    std::vector<IpGroup> out;
    for (int i = 0; i < count; i += per) {
        IpGroup g;
        memset(&g, 0, sizeof(g));
        g.n = std::min(per, count - i);
        g.level = levels[order[i]];
        for (int k = 0; k < g.n; k++) g.job[k] = order[i + k];
        out.push_back(g);
    }
    return out;
}

}  // namespace he

namespace {

inline cudaStream_t S(void *s) { return (cudaStream_t)s; }

thread_local const char *g_last_cuda_error = "no error";

#define HE_TRY(x)                                           \
    do {                                                    \
        cudaError_t e_ = (x);                               \
        if (e_ != cudaSuccess) {                            \
            g_last_cuda_error = cudaGetErrorName(e_);       \
            return HE_ECUDA;                                \
        }                                                   \
    } while (0)

bool aligned(const void *p) { return ((uintptr_t)p & 255) == 0; }

size_t ws_bytes_for(const he_ctx *c, int l) { return c->host_levels[l].ws.total * (size_t)c->N * sizeof(u64); }

int check_dev(const he_ctx *c) { return (c && c->device) ? HE_OK : HE_EINVAL; }

// Upload a small job list for the per-step entry points (test helpers).
int with_jobs(const std::vector<NttGroup> &jobs, cudaStream_t st, NttGroup **out)
{
    void *p = nullptr;
    if (cudaMallocAsync(&p, sizeof(NttGroup) * jobs.size(), st) != cudaSuccess) return HE_ECUDA;
    if (cudaMemcpyAsync(p, jobs.data(), sizeof(NttGroup) * jobs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return HE_ECUDA;
    *out = (NttGroup *)p;
    return HE_OK;
}

// NTT job lists of one launch sequence.
struct Stages {
    const NttGroup *intt1;    int n_intt1;     // iNTT of d2 (+ d0/d1 last limb when fused)
    const NttGroup *ntt_up;   int n_ntt_up;    // NTT of the ModUp outputs
    const NttGroup *intt2;    int n_intt2;     // iNTT of the special limbs (+ KS last limb when fused)
    const NttGroup *ntt_last; int n_ntt_last;  // NTT of the ModDown (fused: ModDown + rescale) limbs
    const int *counts = nullptr;               // optional device-side counts of the four lists (+ ipg's)
    const IpGroup *ipg = nullptr;  int n_ipg = 0;  // batches: inner product with shared key words
};

// The HE Mul pipeline for one job or a batch (JobRef).  mode (TailMode):
// kTailPlain, out is the level-l product; kTailRescale, ModDown and rescale
// merged with two floors (out is [2][l-1][N], bit-identical to he_mul then
// he_rescale); kTailRescalePQ, one division by P q_{l-1} (out [2][l-1][N]).
// NTT group offsets are relative to ntt_base.
int run_keyswitch(he_ctx *c, const JobRef &R, u64 *ntt_base, const Stages &S, const u64 *evk, int mode,
                  cudaStream_t st, bool tensor_fused = false);

int run_pipeline(he_ctx *c, const JobRef &R, u64 *ntt_base, const Stages &S, const u64 *evk, int mode,
                 cudaStream_t st)
{
    prof_mark(c, st, "");
    // Region 1: tensor product, on its own or inside the first iNTT pass of d2
    const bool fused = (c->fuse & 1) != 0;
    if (!fused) {
        capture_tag = kTagJobs;
        HE_TRY(run_tensor(c, R, st));
        prof_mark(c, st, "tensor");
    }
    return run_keyswitch(c, R, ntt_base, S, evk, mode, st, fused);
}

// Region 2 and the final additions, on d0, d1, d2 already in the workspace
// (tensor_fused: the first iNTT pass forms d0, d1, d2 itself).
int run_keyswitch(he_ctx *c, const JobRef &R, u64 *ntt_base, const Stages &S, const u64 *evk, int mode,
                  cudaStream_t st, bool tensor_fused)
{
    // key switching: iNTT(d2) (times N^-1 Qhat^-1), ModUp, NTT, inner product
    const int *cnt = S.counts;
    auto r8 = [c](int site) {  // NTT plan of a site
        return ((c->ntt_r8 >> site) & 1) | (c->ntt_split << 1) | (((c->ntt_small >> site) & 1) << 3) |
               (((c->ntt_onepass >> site) & 1) << 4);
    };
    capture_tag = kTagNtt0 + 0;
    if (tensor_fused)
        HE_TRY(launch_ntt_tensor(c, ntt_base, S.intt1, S.n_intt1, R, st, "intt_d2", cnt ? cnt + 0 : nullptr, r8(0)));
    else
        HE_TRY(launch_ntt(c, ntt_base, S.intt1, S.n_intt1, true, st, "intt_d2", cnt ? cnt + 0 : nullptr, r8(0)));
    capture_tag = kTagJobs;
    HE_TRY(run_modup(c, R, st));
    prof_mark(c, st, "modup");
    capture_tag = kTagNtt0 + 1;
    HE_TRY(launch_ntt(c, ntt_base, S.ntt_up, S.n_ntt_up, false, st, "ntt_modup", cnt ? cnt + 1 : nullptr, r8(1)));
    // a single job's q-limb sums (read only by the final combine) may run
    // beside the ModDown conversion: the sums of the special limbs and the
    // last q limb (the next iNTT's inputs) come first
    const bool split = (c->fuse & 2) && !S.ipg && !R.items && moddown_ipq_fits(c);
    // with the split, the sums of the special limbs and the last q limb may
    // instead be formed by the first pass of their own iNTT (unseeded keys)
    bool seeded = false;
    for (const auto &k : c->seeded) seeded = seeded || k.ptr == evk;
    const bool ip_in_ntt = split && (c->fuse & 4) && !seeded && c->dnum <= kIpFuseDigits;
    if (S.ipg) {
        capture_tag = kTagIpGroups;
        HE_TRY(run_inner_product_shared(c, R, S.ipg, S.n_ipg, cnt ? cnt + 4 : nullptr, evk, st));
        prof_mark(c, st, "inner_product");
    } else if (!ip_in_ntt) {
        capture_tag = kTagJobs;
        HE_TRY(run_inner_product(c, R, evk, st,
                                 !split ? kIpAllRows : mode == kTailPlain ? kIpSpecialRows : kIpSpecialLastRows));
        prof_mark(c, st, split ? "inner_product_special" : "inner_product");
    }
    // ModDown: iNTT of the special limbs (times N^-1 Phat^-1), conversion, NTT
    capture_tag = kTagNtt0 + 2;
    if (ip_in_ntt)
        HE_TRY(launch_ntt_ip(c, ntt_base, S.intt2, S.n_intt2, R, evk, st, "intt_special", cnt ? cnt + 2 : nullptr,
                             r8(2)));
    else
        HE_TRY(launch_ntt(c, ntt_base, S.intt2, S.n_intt2, true, st, "intt_special", cnt ? cnt + 2 : nullptr, r8(2)));
    capture_tag = kTagJobs;
    if (split) {
        HE_TRY(run_moddown_ipq(c, R, mode, evk, st));
        prof_mark(c, st, "moddown_conv_ipq");
    } else {
        HE_TRY(run_moddown_conv(c, R, mode, st));
        prof_mark(c, st, "moddown_conv");
    }
    capture_tag = kTagNtt0 + 3;
    if (mode != kTailPlain) {
        // the final combine runs in the last NTT pass (writes each job's output)
        HE_TRY(launch_ntt_combine(c, ntt_base, S.ntt_last, S.n_ntt_last, R, st, "ntt_moddown", cnt ? cnt + 3 : nullptr,
                                  r8(3)));
    } else {
        HE_TRY(launch_ntt(c, ntt_base, S.ntt_last, S.n_ntt_last, false, st, "ntt_moddown", cnt ? cnt + 3 : nullptr,
                          r8(3)));
        capture_tag = kTagFixed;
        HE_TRY(run_combine_plain(c, R, st));
        prof_mark(c, st, "combine");
    }
    capture_tag = kTagFixed;
    return HE_OK;
}

JobRef single_job(const he_ctx *c, const u64 *ct1, const u64 *ct2, u64 *out, u64 *ws, int l)
{
    JobRef R;
    R.trigger = c->pdl >= 2;
    R.items = nullptr;
    R.one.ct1 = ct1;
    R.one.ct2 = ct2;
    R.one.out = out;
    R.one.ws = ws;
    R.one.level = l;
    R.one.pad = 0;
    R.B = 1;
    R.lmax = l;
    return R;
}

Stages level_stages(const he_ctx *c, int l, int mode)
{
    const LevelJobs &J = c->jobs[l];
    const bool fused = mode != kTailPlain;
    Stages S;
    S.intt1 = fused ? J.intt1f : J.intt1;
    S.n_intt1 = fused ? J.n_intt1f : J.n_intt1;
    S.ntt_up = J.ntt_up;
    S.n_ntt_up = J.n_ntt_up;
    S.intt2 = mode == kTailRescalePQ ? J.intt2pq : fused ? J.intt2f : J.intt2;
    S.n_intt2 = mode == kTailRescalePQ ? J.n_intt2pq : fused ? J.n_intt2f : J.n_intt2;
    S.ntt_last = fused ? J.ntt_z : J.ntt_conv;
    S.n_ntt_last = fused ? J.n_ntt_z : J.n_ntt_conv;
    return S;
}

int hemul_pipeline(he_ctx *c, const u64 *ct1, const u64 *ct2, const u64 *evk, int l, u64 *out, u64 *ws,
                   int mode, cudaStream_t st)
{
    return run_pipeline(c, single_job(c, ct1, ct2, out, ws, l), ws, level_stages(c, l, mode), evk, mode, st);
}

// ---- batches -------------------------------------------------------------
// Batch workspace: [header: items | four NTT group lists | inner-product job
// groups] [job 0 ws] [job 1 ws] ...  Group offsets are relative to the first
// job's ws.
size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t batch_header_bytes(const he_ctx *c, int count, const int *levels)
{
    size_t limbs = 0;
    for (int i = 0; i < count; i++) {
        const HostLevel &H = c->host_levels[levels[i]];
        limbs += H.intt1f.size() + H.ntt_up.size() + H.intt2f.size() + H.ntt_z.size();
    }
    return round_up(sizeof(BatchItem) * count) + round_up(sizeof(NttGroup) * limbs) +
           round_up(sizeof(IpGroup) * count);
}

// Whether a batch of `count` jobs runs the inner product with shared key words.
bool use_shared_ip(const he_ctx *c, int count) { return count > 1 && c->ip_jobs > 1 && inner_product_shared_fits(c); }

size_t batch_bytes(const he_ctx *c, int count, const int *levels)
{
    size_t total = batch_header_bytes(c, count, levels);
    for (int i = 0; i < count; i++) total += ws_bytes_for(c, levels[i]);
    return total;
}

}  // namespace

extern "C" {

const char *he_last_cuda_error(void) { return g_last_cuda_error; }

const char *he_strerror(int code)
{
    switch (code) {
    case HE_OK: return "ok";
    case HE_EINVAL: return "invalid argument";
    case HE_ELEVEL: return "unsupported or mismatched level";
    case HE_ENOMEM: return "workspace too small or admission refused";
    case HE_ECUDA: return "CUDA runtime error";
    case HE_ETIMEOUT: return "bounded device wait gave up";
    case HE_EBUSY: return "resource busy";
    default: return "unknown error";
    }
}

static int create(he_ctx **out, const he_params *p, bool device)
{
    if (!out || !p) return HE_EINVAL;
    he_ctx *c = new (std::nothrow) he_ctx();
    if (!c) return HE_ENOMEM;
    int rc = build_context(c, p, device);
    if (rc != HE_OK) {
        if (c->arena) cudaFree(c->arena);
        delete c;
        return rc;
    }
    *out = c;
    return HE_OK;
}

int he_ctx_create(he_ctx **out, const he_params *p) { return create(out, p, true); }
int he_ctx_create_host(he_ctx **out, const he_params *p) { return create(out, p, false); }

int he_ctx_destroy(he_ctx *c)
{
    if (!c) return HE_EINVAL;
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    for (auto &slot : c->io_ev)
        for (cudaEvent_t e : slot)
            if (e) cudaEventDestroy(e);
    if (c->io_h2d) cudaStreamDestroy(c->io_h2d);
    if (c->io_h2d2) cudaStreamDestroy(c->io_h2d2);
    if (c->io_d2h) cudaStreamDestroy(c->io_d2h);
    if (c->arena) cudaFree(c->arena);
    delete c;
    return HE_OK;
}

int he_ctx_info(const he_ctx *c, int *N, int *dnum, uint64_t *moduli)
{
    if (!c) return HE_EINVAL;
    if (N) *N = c->N;
    if (dnum) *dnum = c->dnum;
    if (moduli) memcpy(moduli, c->ext.data(), sizeof(u64) * c->E);
    return HE_OK;
}

int he_evk_upload(he_ctx *c, const uint64_t *evk_host, uint64_t *evk_dev, void *stream)
{
    if (check_dev(c) || !evk_host || !evk_dev) return HE_EINVAL;
    size_t bytes = (size_t)c->dnum * 2 * c->E * c->N * sizeof(u64);
    HE_TRY(cudaMemcpyAsync(evk_dev, evk_host, bytes, cudaMemcpyHostToDevice, S(stream)));
    return HE_OK;
}

size_t he_workspace_bytes(const he_ctx *c, int level)
{
    if (!c || level < 1 || level > c->L) return 0;
    return ws_bytes_for(c, level);
}

int he_mul(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk, int level, uint64_t *out,
           void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !ct1 || !ct2 || !evk || !out || !ws) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    if (!aligned(ct1) || !aligned(ct2) || !aligned(out) || !aligned(ws) || !aligned(evk)) return HE_EINVAL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    return hemul_pipeline(c, ct1, ct2, evk, level, out, (u64 *)ws, kTailPlain, S(stream));
}

int he_mul_rescale(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk, int level,
                   uint64_t *out, void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !ct1 || !ct2 || !evk || !out || !ws) return HE_EINVAL;
    if (level < 2 || level > c->L) return HE_ELEVEL;
    if (!aligned(ct1) || !aligned(ct2) || !aligned(out) || !aligned(ws) || !aligned(evk)) return HE_EINVAL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    return hemul_pipeline(c, ct1, ct2, evk, level, out, (u64 *)ws, kTailRescale, S(stream));
}

int he_mul_rescale_pq(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk, int level,
                      uint64_t *out, void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !ct1 || !ct2 || !evk || !out || !ws) return HE_EINVAL;
    if (level < 2 || level > c->L) return HE_ELEVEL;
    if (!aligned(ct1) || !aligned(ct2) || !aligned(out) || !aligned(ws) || !aligned(evk)) return HE_EINVAL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    return hemul_pipeline(c, ct1, ct2, evk, level, out, (u64 *)ws, kTailRescalePQ, S(stream));
}

namespace {
int elementwise(he_ctx *c, int op, const uint64_t *x, const uint64_t *y, int level, uint64_t *out, void *stream)
{
    if (check_dev(c) || !x || !y || !out) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    if (!aligned(x) || !aligned(y) || !aligned(out)) return HE_EINVAL;
    HE_TRY(run_elementwise(c, op, x, y, out, level, S(stream)));
    return HE_OK;
}
}  // namespace

int he_add(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, int level, uint64_t *out, void *stream)
{
    return elementwise(c, 0, ct1, ct2, level, out, stream);
}

int he_sub(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, int level, uint64_t *out, void *stream)
{
    return elementwise(c, 1, ct1, ct2, level, out, stream);
}

int he_mul_plain(he_ctx *c, const uint64_t *ct, const uint64_t *pt, int level, uint64_t *out, void *stream)
{
    return elementwise(c, 2, ct, pt, level, out, stream);
}

int he_add_plain(he_ctx *c, const uint64_t *ct, const uint64_t *pt, int level, uint64_t *out, void *stream)
{
    return elementwise(c, 3, ct, pt, level, out, stream);
}

int he_rotate(he_ctx *c, const uint64_t *ct, const uint64_t *rk, int level, uint64_t galois, uint64_t *out, void *ws,
              size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !ct || !rk || !out || !ws) return HE_EINVAL;
    if (galois % 2 == 0 || galois >= 2 * (uint64_t)c->N) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    if (!aligned(ct) || !aligned(out) || !aligned(ws) || !aligned(rk)) return HE_EINVAL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    cudaStream_t st = S(stream);
    u64 *w = (u64 *)ws;
    prof_mark(c, st, "");
    HE_TRY(run_automorph(c, ct, w, level, galois, st));
    prof_mark(c, st, "automorph");
    return run_keyswitch(c, single_job(c, nullptr, nullptr, out, w, level), w, level_stages(c, level, kTailPlain), rk, kTailPlain,
                         st);
}

int he_rescale(he_ctx *c, const uint64_t *ct, int level, uint64_t *out, void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !ct || !out || !ws) return HE_EINVAL;
    if (level < 2 || level > c->L) return HE_ELEVEL;
    if (!aligned(ct) || !aligned(out) || !aligned(ws)) return HE_EINVAL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    const WsLayout &W = c->host_levels[level].ws;
    const LevelJobs &J = c->jobs[level];
    const size_t N = (size_t)c->N;
    u64 *w = (u64 *)ws;
    cudaStream_t st = S(stream);
    HE_TRY(launch_ntt2(c, ct, w, J.rs_intt, J.n_rs_intt, true, st));
    HE_TRY(launch_ntt(c, w, J.rs_ntt, J.n_rs_ntt, false, st));
    HE_TRY(run_rescale_combine(c, ct, w + W.z * N, out, level, st));
    return HE_OK;
}

int he_step_ntt(he_ctx *c, uint64_t *data, const int *prime_idx, int count, int inverse, void *stream)
{
    if (check_dev(c) || !data || !prime_idx || count < 1 || !aligned(data)) return HE_EINVAL;
    std::vector<NttJob> jobs(count);
    for (int i = 0; i < count; i++) {
        if (prime_idx[i] < 0 || prime_idx[i] >= c->E) return HE_EINVAL;
        int e = prime_idx[i];
        jobs[i] = NttJob{(unsigned)i, (unsigned)i, (unsigned)e, 0, c->ninv[e], c->ninv_sh[e]};
    }
    cudaStream_t st = S(stream);
    std::vector<NttGroup> groups = group_jobs(jobs);
    NttGroup *dj = nullptr;
    int rc = with_jobs(groups, st, &dj);
    if (rc) return rc;
    cudaError_t e = launch_ntt(c, (u64 *)data, dj, (int)groups.size(), inverse != 0, st, nullptr, nullptr,
                               (c->ntt_r8 & 1) | (c->ntt_split << 1) | ((c->ntt_small & 1) << 3) |
                                   ((c->ntt_onepass & 1) << 4));
    cudaFreeAsync(dj, st);
    return e == cudaSuccess ? HE_OK : HE_ECUDA;
}

int he_step_tensor(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, int level, uint64_t *d, void *stream)
{
    if (check_dev(c) || !ct1 || !ct2 || !d) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    // d0, d1, d2 sit at limb offsets 0, l, 2l of a workspace: d serves as one
    HE_TRY(run_tensor(c, single_job(c, ct1, ct2, nullptr, (u64 *)d, level), S(stream)));
    return HE_OK;
}

int he_step_modup(he_ctx *c, const uint64_t *d2, int level, uint64_t *U, void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !d2 || !U || !ws) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    const WsLayout &W = c->host_levels[level].ws;
    const LevelJobs &J = c->jobs[level];
    const size_t N = (size_t)c->N;
    const size_t E = (size_t)c->K + level, beta = (size_t)(level + c->alpha - 1) / c->alpha;
    u64 *w = (u64 *)ws;
    cudaStream_t st = S(stream);
    HE_TRY(cudaMemcpyAsync(w + W.d2 * N, d2, (size_t)level * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    HE_TRY(cudaMemcpyAsync(w + W.u * N, U, beta * E * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    HE_TRY(launch_ntt(c, w, J.intt1, J.n_intt1, true, st));
    HE_TRY(run_modup(c, single_job(c, nullptr, nullptr, nullptr, w, level), st, true));
    HE_TRY(cudaMemcpyAsync(U, w + W.u * N, beta * E * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    return HE_OK;
}

int he_step_inner_product(he_ctx *c, const uint64_t *U, const uint64_t *d2, const uint64_t *evk, int level,
                          uint64_t *KS, void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !U || !d2 || !evk || !KS || !ws) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    const WsLayout &W = c->host_levels[level].ws;
    const size_t N = (size_t)c->N;
    const size_t E = (size_t)c->K + level, beta = (size_t)(level + c->alpha - 1) / c->alpha;
    u64 *w = (u64 *)ws;
    cudaStream_t st = S(stream);
    HE_TRY(cudaMemcpyAsync(w + W.d2 * N, d2, (size_t)level * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    HE_TRY(cudaMemcpyAsync(w + W.u * N, U, beta * E * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    HE_TRY(run_inner_product(c, single_job(c, nullptr, nullptr, nullptr, w, level), evk, st));
    HE_TRY(cudaMemcpyAsync(KS, w + W.ks * N, 2 * E * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    return HE_OK;
}

int he_step_moddown(he_ctx *c, const uint64_t *X, int level, uint64_t *out, void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !X || !out || !ws) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    const WsLayout &W = c->host_levels[level].ws;
    const LevelJobs &J = c->jobs[level];
    const size_t N = (size_t)c->N;
    const int E = c->K + level;
    u64 *w = (u64 *)ws;
    cudaStream_t st = S(stream);
    // X goes where KS_b sits; KS_a is zero, d0/d1 are zero
    HE_TRY(cudaMemcpyAsync(w + W.ks * N, X, (size_t)E * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    HE_TRY(cudaMemsetAsync(w + (W.ks + E) * N, 0, (size_t)E * N * sizeof(u64), st));
    HE_TRY(cudaMemsetAsync(w + W.d0 * N, 0, 2 * (size_t)level * N * sizeof(u64), st));
    HE_TRY(launch_ntt(c, w, J.intt2, J.n_intt2, true, st));
    const JobRef R = single_job(c, nullptr, nullptr, w + W.y * N, w, level);  // both halves land at y, u
    HE_TRY(run_moddown_conv(c, R, false, st));
    HE_TRY(launch_ntt(c, w, J.ntt_conv, J.n_ntt_conv, false, st));
    HE_TRY(run_combine_plain(c, R, st));
    HE_TRY(cudaMemcpyAsync(out, w + W.y * N, (size_t)level * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    return HE_OK;
}

}  // extern "C"

extern "C" {

size_t he_batch_workspace_bytes(const he_ctx *c, int count, const int *levels)
{
    if (!c || count < 1 || !levels) return 0;
    for (int i = 0; i < count; i++)
        if (levels[i] < 2 || levels[i] > c->L) return 0;
    return batch_bytes(c, count, levels);
}

int he_mul_batch(he_ctx *c, int count, const he_job *jobs, const uint64_t *evk, void *ws, size_t ws_bytes,
                 void *stream)
{
    if (check_dev(c) || count < 1 || count > 65535 || !jobs || !evk || !ws || !aligned(ws) || !aligned(evk))
        return HE_EINVAL;
    std::vector<int> levels(count);
    int lmax = 0;
    for (int i = 0; i < count; i++) {
        const he_job &j = jobs[i];
        if (!j.ct1 || !j.ct2 || !j.out) return HE_EINVAL;
        if (!aligned(j.ct1) || !aligned(j.ct2) || !aligned(j.out)) return HE_EINVAL;
        if (j.level < 2 || j.level > c->L) return HE_ELEVEL;
        levels[i] = j.level;
        lmax = std::max(lmax, j.level);
    }
    if (ws_bytes < batch_bytes(c, count, levels.data())) return HE_ENOMEM;
    const size_t N = (size_t)c->N;
    const size_t hdr = batch_header_bytes(c, count, levels.data());
    char *wsb = (char *)ws;
    u64 *data = (u64 *)(wsb + hdr);
    // items, and every job's single-limb NTT jobs shifted to its ws slice
    std::vector<BatchItem> items(count);
    std::vector<NttJob> l1, l2, l3, l4;
    size_t off = 0;  // limbs
    for (int i = 0; i < count; i++) {
        const HostLevel &H = c->host_levels[levels[i]];
        items[i].ct1 = jobs[i].ct1;
        items[i].ct2 = jobs[i].ct2;
        items[i].out = jobs[i].out;
        items[i].ws = data + off * N;
        items[i].level = levels[i];
        items[i].pad = 0;
        auto add = [&](const std::vector<NttJob> &src, std::vector<NttJob> &dst) {
            for (NttJob j : src) {
                j.src += (unsigned)off;
                j.dst += (unsigned)off;
                j.cd += (unsigned)off;
                j.cks += (unsigned)off;
                j.job = (unsigned)i;
                dst.push_back(j);
            }
        };
        add(H.intt1f, l1);
        add(H.ntt_up, l2);
        add(H.intt2f, l3);
        add(H.ntt_z, l4);
        off += H.ws.total;
    }
    if (off * N >= ((size_t)1 << 32) * N) return HE_EINVAL;  // offsets are 32-bit limb counts
    // regroup by prime across jobs: limbs of different jobs share a twiddle tile
    const int cap = c->group_cap;
    std::vector<NttGroup> g1 = group_jobs(l1, cap), g2 = group_jobs(l2, cap), g3 = group_jobs(l3, cap),
                          g4 = group_jobs(l4, cap);
    std::vector<unsigned char> head(hdr, 0);
    const size_t items_bytes = round_up(sizeof(BatchItem) * count);
    memcpy(head.data(), items.data(), sizeof(BatchItem) * count);
    NttGroup *gdst = (NttGroup *)(head.data() + items_bytes);
    const NttGroup *gdev = (const NttGroup *)(wsb + items_bytes);
    size_t gi = 0;
    Stages Sg;
    auto put = [&](const std::vector<NttGroup> &g, const NttGroup *&p, int &n) {
        memcpy(gdst + gi, g.data(), sizeof(NttGroup) * g.size());
        p = gdev + gi;
        n = (int)g.size();
        gi += g.size();
    };
    put(g1, Sg.intt1, Sg.n_intt1);
    put(g2, Sg.ntt_up, Sg.n_ntt_up);
    put(g3, Sg.intt2, Sg.n_intt2);
    put(g4, Sg.ntt_last, Sg.n_ntt_last);
    if (use_shared_ip(c, count)) {
        const std::vector<IpGroup> ipg = ip_groups(levels.data(), count, c->ip_jobs);
        const size_t ip_off = items_bytes + round_up(sizeof(NttGroup) * gi);
        memcpy(head.data() + ip_off, ipg.data(), sizeof(IpGroup) * ipg.size());
        Sg.ipg = (const IpGroup *)(wsb + ip_off);
        Sg.n_ipg = (int)ipg.size();
    }
    cudaStream_t st = S(stream);
    // the header is staged from this call's own host memory, which a captured
    // copy would read after it is gone: batches are captured with
    // he_batch_graph_create instead
    cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
    HE_TRY(cudaStreamIsCapturing(st, &capturing));
    if (capturing != cudaStreamCaptureStatusNone) return HE_EINVAL;
    HE_TRY(cudaMemcpyAsync(ws, head.data(), hdr, cudaMemcpyHostToDevice, st));
    JobRef R;
    R.items = (const BatchItem *)ws;
    memset(&R.one, 0, sizeof(R.one));
    R.B = count;
    R.lmax = lmax;
    R.trigger = c->pdl >= 2;
    return run_pipeline(c, R, data, Sg, evk, kTailRescale, st);
}

}  // extern "C"

extern "C" {

int he_profile(he_ctx *c, int enable)
{
    if (check_dev(c)) return HE_EINVAL;
    if (enable && c->prof_pool.empty()) {
        c->prof_pool.resize(8192);
        c->prof_names.resize(8192);
        for (auto &e : c->prof_pool)
            if (cudaEventCreate(&e) != cudaSuccess) return HE_ECUDA;
    }
    c->prof = enable != 0;
    c->prof_used = 0;
    return HE_OK;
}

int he_evk_register_seeded(he_ctx *c, const uint64_t *evk_b, uint64_t seed)
{
    if (check_dev(c) || !evk_b || !aligned(evk_b)) return HE_EINVAL;
    he_evk_unregister(c, evk_b);
    if (c->seeded.size() >= 64) return HE_ENOMEM;
    he_ctx::SeededKey k;
    k.ptr = evk_b;
    // stream state of digit j: word (144 + j) of the seed's SplitMix64 generator
    for (int j = 0; j < kMaxDigits; j++) {
        u64 z = seed + (u64)(144 + j + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        k.state[j] = z ^ (z >> 31);
    }
    c->seeded.push_back(k);
    return HE_OK;
}

int he_evk_unregister(he_ctx *c, const uint64_t *evk)
{
    if (!c || !evk) return HE_EINVAL;
    for (size_t i = 0; i < c->seeded.size(); i++)
        if (c->seeded[i].ptr == evk) {
            c->seeded.erase(c->seeded.begin() + (long)i);
            return HE_OK;
        }
    return HE_OK;
}

int he_set_shape(he_ctx *c, const he_shape *sh)
{
    if (!c || !sh) return HE_EINVAL;
    if (sh->group_cap < 1 || sh->group_cap > kGroupMax) return HE_EINVAL;
    if (sh->modup_chunk != 4 && sh->modup_chunk != 8 && sh->modup_chunk != 16) return HE_EINVAL;
    if (sh->pdl < 0 || sh->pdl > 2) return HE_EINVAL;
    if (sh->ntt_r8 < 0 || sh->ntt_r8 > 15) return HE_EINVAL;
    if (sh->ip_jobs != 1 && sh->ip_jobs != 4 && sh->ip_jobs != 8) return HE_EINVAL;
    if (sh->fuse < 0 || sh->fuse > 7) return HE_EINVAL;
    if (sh->ntt_split < 0 || sh->ntt_split > 2) return HE_EINVAL;
    if (sh->ntt_small < 0 || sh->ntt_small > 15) return HE_EINVAL;
    if (sh->ntt_onepass < 0 || sh->ntt_onepass > 15) return HE_EINVAL;
    c->group_cap = sh->group_cap;
    c->modup_chunk = sh->modup_chunk;
    c->pdl = sh->pdl;
    c->ntt_r8 = sh->ntt_r8;
    c->ip_jobs = sh->ip_jobs;
    c->fuse = sh->fuse;
    c->ntt_split = sh->ntt_split;
    c->ntt_small = sh->ntt_small;
    c->ntt_onepass = sh->ntt_onepass;
    if (c->device) c->jobs = c->jobs_cap[c->group_cap - 1];
    return HE_OK;
}

int he_get_shape(const he_ctx *c, he_shape *sh)
{
    if (!c || !sh) return HE_EINVAL;
    sh->group_cap = c->group_cap;
    sh->modup_chunk = c->modup_chunk;
    sh->pdl = c->pdl;
    sh->ntt_r8 = c->ntt_r8;
    sh->ip_jobs = c->ip_jobs;
    sh->fuse = c->fuse;
    sh->ntt_split = c->ntt_split;
    sh->ntt_small = c->ntt_small;
    sh->ntt_onepass = c->ntt_onepass;
    sh->ms = 0;
    return HE_OK;
}

int he_autotune(he_ctx *c, const he_job *jobs, int count, const uint64_t *evk, void *ws, size_t ws_bytes, int reps,
                void *stream, he_shape *best, he_shape *tried, int max_tried, int *n_tried)
{
    if (check_dev(c) || !jobs || count < 1 || !evk || !ws || !best || reps < 1) return HE_EINVAL;
    he_shape keep;
    he_get_shape(c, &keep);
    auto call = [&]() -> int {
        if (count == 1)
            return he_mul_rescale(c, jobs[0].ct1, jobs[0].ct2, evk, jobs[0].level, jobs[0].out, ws, ws_bytes, stream);
        return he_mul_batch(c, count, jobs, evk, ws, ws_bytes, stream);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return HE_ECUDA;
    }
    const bool prof = c->prof;
    c->prof = false;
    int rc = HE_OK, n = 0;
    he_shape top = keep;
    top.ms = -1;
    std::vector<he_shape> timed;  // every shape timed, with its time
    auto time_shape = [&](he_shape sh) -> int {
        he_set_shape(c, &sh);
        int r = call();  // warm-up (and argument check)
        if (r != HE_OK) return r;
        cudaEventRecord(e0, S(stream));
        for (int k = 0; k < reps && r == HE_OK; k++) r = call();
        cudaEventRecord(e1, S(stream));
        if (r != HE_OK) return r;
        float ms = 0;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            return HE_ECUDA;
        sh.ms = ms / reps;
        if (tried && n < max_tried) tried[n] = sh;
        n++;
        timed.push_back(sh);
        if (top.ms < 0 || sh.ms < top.ms) top = sh;
        return HE_OK;
    };
    // coordinate descent over the knobs, from the context's shape: each knob
    // in turn takes every value with the others held at the best so far,
    // until a full sweep changes nothing (at most four sweeps); shapes
    // already timed are not timed again
    std::vector<he_shape> seen;
    auto same = [](const he_shape &a, const he_shape &b) {
        return a.group_cap == b.group_cap && a.modup_chunk == b.modup_chunk && a.pdl == b.pdl &&
               a.ntt_r8 == b.ntt_r8 && a.ip_jobs == b.ip_jobs && a.fuse == b.fuse && a.ntt_split == b.ntt_split &&
               a.ntt_small == b.ntt_small && a.ntt_onepass == b.ntt_onepass;
    };
    auto try_shape = [&](he_shape sh) -> int {
        if ((sh.fuse & 4) && !(sh.fuse & 2)) return HE_OK;  // bit 2 acts with bit 1 only
        // with the special rows' sums in their iNTT, that site keeps two passes
        if (count == 1 && (sh.fuse & 6) == 6 && (sh.ntt_onepass & 4)) return HE_OK;
        for (const he_shape &t : seen)
            if (same(t, sh)) return HE_OK;
        seen.push_back(sh);
        return time_shape(sh);
    };
    rc = try_shape(keep);
    const bool batch = count > 1 && inner_product_shared_fits(c);
    const int nsplit = (c->logN == 16 || c->logN == 17) ? 3 : 1;
    // knobs whose best values depend on each other move together: the PDL
    // mode with the fusions, the NTT radix mask with the pass split
    constexpr int kKnobs = 7;
    auto knob_values = [&](int knob) {
        switch (knob) {
        case 0: return kGroupMax;
        case 1: return 3;
        case 2: return 3 * 8;
        case 3: return 16 * nsplit;
        case 4: return batch ? 3 : 0;
        case 5: return nsplit > 1 ? 16 : 0;           // 1024-element tiles: 2^16 and 2^17
        default: return c->logN == 16 ? 16 : 0;       // one-pass cluster transforms: 2^16
        }
    };
    auto descent = [&]() {
        for (int sweep = 0; sweep < 4 && rc == HE_OK; sweep++) {
            const he_shape before = top;
            for (int knob = 0; knob < kKnobs && rc == HE_OK; knob++) {
                const he_shape base = top;
                const int nv = knob_values(knob);
                for (int v = 0; v < nv && rc == HE_OK; v++) {
                    he_shape sh = base;
                    switch (knob) {
                    case 0: sh.group_cap = v + 1; break;
                    case 1: sh.modup_chunk = v == 0 ? 4 : v == 1 ? 8 : 16; break;
                    case 2: sh.pdl = v / 8; sh.fuse = v % 8; break;
                    case 3: sh.ntt_r8 = v % 16; sh.ntt_split = v / 16; break;
                    case 4: sh.ip_jobs = v == 0 ? 1 : v == 1 ? 4 : 8; break;
                    case 5: sh.ntt_small = v; break;
                    default: sh.ntt_onepass = v; break;
                    }
                    rc = try_shape(sh);
                }
            }
            if (same(before, top)) break;
        }
    };
    descent();
    // the knobs whose best values interact most, exhaustively: every PDL
    // mode, fusion set and pass split with the radix masks {best, none, all},
    // then descent sweeps again from the best
    if (rc == HE_OK) {
        const he_shape base = top;
        const int masks[3] = {base.ntt_r8, 0, 15};
        for (int m = 0; m < 3 && rc == HE_OK; m++)
            for (int pdl = 0; pdl < 3 && rc == HE_OK; pdl++)
                for (int fz = 0; fz < 8 && rc == HE_OK; fz++)
                    for (int sp = 0; sp < nsplit && rc == HE_OK; sp++) {
                        he_shape sh = base;
                        sh.ntt_r8 = masks[m];
                        sh.pdl = pdl;
                        sh.fuse = fz;
                        sh.ntt_split = sp;
                        rc = try_shape(sh);
                    }
    }
    descent();
    // the fastest few are timed again, interleaved, three rounds of 2 reps
    // calls each, and the best median is kept: the differences between them
    // are of the size of one timing's noise
    if (rc == HE_OK && timed.size() > 1) {
        std::vector<he_shape> cand = timed;
        std::sort(cand.begin(), cand.end(), [](const he_shape &a, const he_shape &b) { return a.ms < b.ms; });
        cand.resize(std::min<size_t>(cand.size(), 4));
        std::vector<std::vector<float>> t(cand.size());
        for (int round = 0; round < 3 && rc == HE_OK; round++)
            for (size_t k = 0; k < cand.size() && rc == HE_OK; k++) {
                he_set_shape(c, &cand[k]);
                rc = call();
                cudaEventRecord(e0, S(stream));
                for (int r = 0; r < 2 * reps && rc == HE_OK; r++) rc = call();
                cudaEventRecord(e1, S(stream));
                float ms = 0;
                if (rc == HE_OK &&
                    (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                    rc = HE_ECUDA;
                t[k].push_back(ms / (2 * reps));
            }
        if (rc == HE_OK) {
            for (size_t k = 0; k < cand.size(); k++) {
                std::sort(t[k].begin(), t[k].end());
                cand[k].ms = t[k][t[k].size() / 2];
            }
            top = *std::min_element(cand.begin(), cand.end(),
                                    [](const he_shape &a, const he_shape &b) { return a.ms < b.ms; });
        }
    }
    c->prof = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_tried) *n_tried = std::min(n, max_tried);
    if (rc != HE_OK) {
        he_set_shape(c, &keep);
        return rc;
    }
    he_set_shape(c, &top);
    *best = top;
    return HE_OK;
}

int he_profile_read(he_ctx *c, int max, char *names, double *total_ms, int *calls, int *count)
{
    if (check_dev(c) || max < 1 || !names || !total_ms || !calls || !count) return HE_EINVAL;
    if (c->prof_used > 0 && cudaEventSynchronize(c->prof_pool[c->prof_used - 1]) != cudaSuccess) return HE_ECUDA;
    std::vector<std::string> keys;
    std::vector<double> ms;
    std::vector<int> n;
    for (size_t i = 1; i < c->prof_used; i++) {
        const std::string &k = c->prof_names[i];
        if (k.empty()) continue;
        float t = 0;
        if (cudaEventElapsedTime(&t, c->prof_pool[i - 1], c->prof_pool[i]) != cudaSuccess) return HE_ECUDA;
        size_t j = 0;
        while (j < keys.size() && keys[j] != k) j++;
        if (j == keys.size()) { keys.push_back(k); ms.push_back(0); n.push_back(0); }
        ms[j] += t;
        n[j] += 1;
    }
    int m = (int)std::min<size_t>(keys.size(), (size_t)max);
    for (int j = 0; j < m; j++) {
        strncpy(names + 48 * j, keys[j].c_str(), 47);
        names[48 * j + 47] = 0;
        total_ms[j] = ms[j];
        calls[j] = n[j];
    }
    *count = m;
    c->prof_used = 0;
    return HE_OK;
}

size_t he_host_workspace_bytes(const he_ctx *c, int level)
{
    if (!c || level < 2 || level > c->L) return 0;
    const size_t limb = (size_t)c->N * sizeof(u64);
    return ws_bytes_for(c, level) + (4 * (size_t)level + 2 * (size_t)(level - 1)) * limb;
}

int he_mul_rescale_host(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk, int level,
                        uint64_t *out, void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !ct1 || !ct2 || !evk || !out || !ws) return HE_EINVAL;
    if (level < 2 || level > c->L) return HE_ELEVEL;
    if (!aligned(ws) || !aligned(evk)) return HE_EINVAL;
    if (ws_bytes < he_host_workspace_bytes(c, level)) return HE_ENOMEM;
    const size_t limb = (size_t)c->N * sizeof(u64);
    char *base = (char *)ws;
    u64 *w = (u64 *)base;
    u64 *d1 = (u64 *)(base + ws_bytes_for(c, level));
    u64 *d2 = (u64 *)((char *)d1 + 2 * (size_t)level * limb);
    u64 *dout = (u64 *)((char *)d2 + 2 * (size_t)level * limb);
    cudaStream_t st = S(stream);
    HE_TRY(cudaMemcpyAsync(d1, ct1, 2 * (size_t)level * limb, cudaMemcpyHostToDevice, st));
    HE_TRY(cudaMemcpyAsync(d2, ct2, 2 * (size_t)level * limb, cudaMemcpyHostToDevice, st));
    int rc = hemul_pipeline(c, d1, d2, evk, level, dout, w, kTailRescale, st);
    if (rc) return rc;
    HE_TRY(cudaMemcpyAsync(out, dout, 2 * (size_t)(level - 1) * limb, cudaMemcpyDeviceToHost, st));
    HE_TRY(cudaStreamSynchronize(st));
    return HE_OK;
}

size_t he_host_stream_workspace_bytes(const he_ctx *c, int max_level, int slots)
{
    if (!c || max_level < 2 || max_level > c->L || slots < 2 || slots > 4) return 0;
    size_t path = 0;
    for (int l = 2; l <= max_level; l++) path = std::max(path, ws_bytes_for(c, l));
    const size_t limb = (size_t)c->N * sizeof(u64);
    return path + (size_t)slots * (6 * (size_t)max_level - 2) * limb;
}

int he_mul_rescale_host_stream(he_ctx *c, int count, const uint64_t *const *ct1, const uint64_t *const *ct2,
                               const int *levels, uint64_t *const *out, const uint64_t *evk, void *ws,
                               size_t ws_bytes, int slots, void *stream)
{
    if (check_dev(c) || count < 0 || !evk || !ws || slots < 2 || slots > 4) return HE_EINVAL;
    if (count == 0) return HE_OK;
    if (!ct1 || !ct2 || !levels || !out) return HE_EINVAL;
    if (!aligned(ws) || !aligned(evk)) return HE_EINVAL;
    int ml = 0;
    for (int k = 0; k < count; k++) {
        if (!ct1[k] || !ct2[k] || !out[k]) return HE_EINVAL;
        if (levels[k] < 2 || levels[k] > c->L) return HE_ELEVEL;
        ml = std::max(ml, levels[k]);
    }
    if (ws_bytes < he_host_stream_workspace_bytes(c, ml, slots)) return HE_ENOMEM;
    {
        std::lock_guard<std::mutex> lk(c->io_mu);
        if (!c->io_h2d && cudaStreamCreateWithFlags(&c->io_h2d, cudaStreamNonBlocking) != cudaSuccess) return HE_ECUDA;
        if (!c->io_h2d2 && cudaStreamCreateWithFlags(&c->io_h2d2, cudaStreamNonBlocking) != cudaSuccess)
            return HE_ECUDA;
        if (!c->io_d2h && cudaStreamCreateWithFlags(&c->io_d2h, cudaStreamNonBlocking) != cudaSuccess) return HE_ECUDA;
        for (auto &slot : c->io_ev)
            for (cudaEvent_t &e : slot)
                if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return HE_ECUDA;
    }
    size_t path = 0;
    for (int l = 2; l <= ml; l++) path = std::max(path, ws_bytes_for(c, l));
    const size_t limb = (size_t)c->N * sizeof(u64);
    const size_t slot_bytes = (6 * (size_t)ml - 2) * limb;
    u64 *w = (u64 *)ws;
    cudaStream_t st = S(stream), up = c->io_h2d, up2 = c->io_h2d2, down = c->io_d2h;
    for (int k = 0; k < count; k++) {
        const int s = k % slots, l = levels[k];
        // 0: ct1 copied, 3: ct2 copied, 1: path done, 2: result copied
        cudaEvent_t *ev = c->io_ev[s];
        char *sb = (char *)ws + path + (size_t)s * slot_bytes;
        u64 *a = (u64 *)sb, *b = (u64 *)(sb + 2 * (size_t)ml * limb), *o = (u64 *)(sb + 4 * (size_t)ml * limb);
        // the slot's inputs are free once the path of job k - slots has run;
        // the two operands travel on two streams, side by side
        if (k >= slots) {
            HE_TRY(cudaStreamWaitEvent(up, ev[1], 0));
            HE_TRY(cudaStreamWaitEvent(up2, ev[1], 0));
        }
        HE_TRY(cudaMemcpyAsync(a, ct1[k], 2 * (size_t)l * limb, cudaMemcpyHostToDevice, up));
        HE_TRY(cudaMemcpyAsync(b, ct2[k], 2 * (size_t)l * limb, cudaMemcpyHostToDevice, up2));
        HE_TRY(cudaEventRecord(ev[0], up));
        HE_TRY(cudaEventRecord(ev[3], up2));
        // the path waits for its inputs and for the slot's previous result to be read back
        HE_TRY(cudaStreamWaitEvent(st, ev[0], 0));
        HE_TRY(cudaStreamWaitEvent(st, ev[3], 0));
        if (k >= slots) HE_TRY(cudaStreamWaitEvent(st, ev[2], 0));
        int rc = hemul_pipeline(c, a, b, evk, l, o, w, kTailRescale, st);
        if (rc) return rc;
        HE_TRY(cudaEventRecord(ev[1], st));
        HE_TRY(cudaStreamWaitEvent(down, ev[1], 0));
        HE_TRY(cudaMemcpyAsync(out[k], o, 2 * (size_t)(l - 1) * limb, cudaMemcpyDeviceToHost, down));
        HE_TRY(cudaEventRecord(ev[2], down));
    }
    HE_TRY(cudaStreamSynchronize(down));
    HE_TRY(cudaStreamSynchronize(st));
    return HE_OK;
}

}  // extern "C"

// ---- batch graphs ----------------------------------------------------------
// The batched pipeline captured once in a CUDA graph for up to max_jobs jobs:
// the per-job grids are sized for max_jobs jobs at level L, the NTT grids for
// the most groups max_jobs jobs can form at the limb-group cap in effect at
// capture (at least that cap is used at every launch), the job table and NTT
// group lists (and their counts) live at the head of the workspace and are
// refreshed from a pinned host copy by the graph's first node, so a replay
// with a different batch (count, levels, operands) is one graph launch.
// Unused job slots carry level 0, for which every kernel block exits.
struct he_batch_graph {
    he_ctx *c = nullptr;
    int max_jobs = 0;
    const u64 *evk = nullptr;
    char *ws = nullptr;
    size_t hdr = 0, slot_limbs = 0;
    size_t items_bytes = 0, counts_off = 0, lists_off[4] = {0, 0, 0, 0}, ipg_off = 0;
    size_t hdr_copy = 0;  // header bytes the graph's first node copies (up to the last list's end)
    int list_max[4] = {0, 0, 0, 0};  // groups each NTT list may hold (and its launch's grid) at `cap`
    int cap = 1;                     // limb-group cap at capture
    int ip_jobs = 0;  // jobs per inner-product group captured (0: one job per CTA)
    // kernel nodes resized at every launch to the batch it runs (NTT nodes to
    // its limb groups, per-job nodes to its jobs); empty if the captured
    // launches could not be matched to the graph's nodes
    struct NodeFix {
        cudaGraphNode_t node;
        cudaKernelNodeParams p;
        int tag;
        unsigned tiles;
    };
    std::vector<NodeFix> fixes;
    // the graph's first node copies the header from pinned[b]; with its node
    // found, launches alternate between two pinned headers, so the host fills
    // one while the previous launch (which read the other) may still run
    cudaGraphNode_t memcpy_node = nullptr;
    unsigned char *pinned[2] = {nullptr, nullptr};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool launched[2] = {false, false};
    unsigned nlaunch = 0;
};

namespace {

// Most groups NTT list t (0..3: the four sites) can hold for max_jobs jobs
// at limb-group cap `cap`: per prime, the most limbs one job of any level has
// in that list, times max_jobs, in groups of cap (group_jobs never mixes
// primes).
int graph_list_bound(const he_ctx *c, int max_jobs, int t, int cap)
{
    std::vector<int> most(c->E, 0), cnt(c->E, 0);
    for (int l = 2; l <= c->L; l++) {
        const HostLevel &H = c->host_levels[l];
        const std::vector<NttJob> *lists[4] = {&H.intt1f, &H.ntt_up, &H.intt2f, &H.ntt_z};
        std::fill(cnt.begin(), cnt.end(), 0);
        for (const NttJob &j : *lists[t]) cnt[j.prime]++;
        for (int p = 0; p < c->E; p++) most[p] = std::max(most[p], cnt[p]);
    }
    long long groups = 0;
    for (int p = 0; p < c->E; p++) groups += ((long long)most[p] * max_jobs + cap - 1) / cap;
    return (int)groups;
}

// Header layout: [items | counts | inner-product groups | four NTT lists at
// the capture cap's bounds | room up to the bounds at cap 1], then the jobs'
// workspaces; the workspace size does not depend on the cap.
void graph_layout(const he_ctx *c, int max_jobs, he_batch_graph *g, int cap)
{
    g->cap = cap;
    g->items_bytes = round_up(sizeof(BatchItem) * max_jobs);
    g->counts_off = g->items_bytes;
    size_t off = g->counts_off + 256;
    g->ipg_off = off;
    off += round_up(sizeof(IpGroup) * (size_t)max_jobs);
    size_t room = off;
    for (int t = 0; t < 4; t++) {
        g->list_max[t] = graph_list_bound(c, max_jobs, t, cap);
        g->lists_off[t] = off;
        off += round_up(sizeof(NttGroup) * (size_t)g->list_max[t]);
        room += round_up(sizeof(NttGroup) * (size_t)graph_list_bound(c, max_jobs, t, 1));
    }
    g->hdr_copy = off;
    g->hdr = std::max(off, room);
    size_t slot = 0;
    for (int l = 2; l <= c->L; l++) slot = std::max(slot, c->host_levels[l].ws.total);
    g->slot_limbs = slot;
}

// The graph's kernel nodes in launch order (a topological walk of the
// captured chain), matched one to one with the tags logged at capture.
void graph_match_nodes(he_batch_graph *g, const std::vector<int> &log, const Stages &S)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g->graph, nullptr, &n) != cudaSuccess || n == 0) {
        (void)cudaGetLastError();
        return;
    }
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g->graph, nodes.data(), &n) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    // Kahn's order over the dependency edges (programmatic edges carry edge
    // data, so the query passes room for it; a failed query leaves the nodes
    // as captured and clears the error it raised)
    std::vector<size_t> indeg(n, 0);
    std::vector<std::vector<size_t>> out(n);
    std::vector<cudaGraphNode_t> dep(n);
    std::vector<cudaGraphEdgeData> edata(n);
    for (size_t i = 0; i < n; i++) {
        size_t nd = n;
        if (cudaGraphNodeGetDependentNodes(nodes[i], dep.data(), edata.data(), &nd) != cudaSuccess || nd > n) {
            (void)cudaGetLastError();
            return;
        }
        for (size_t k = 0; k < nd; k++) {
            const cudaGraphNode_t d = dep[k];
            for (size_t j = 0; j < n; j++)
                if (nodes[j] == d) {
                    out[i].push_back(j);
                    indeg[j]++;
                }
        }
    }
    std::vector<size_t> order, ready;
    for (size_t i = 0; i < n; i++)
        if (!indeg[i]) ready.push_back(i);
    while (!ready.empty()) {
        if (ready.size() != 1) return;  // not a chain: leave the nodes as captured
        const size_t i = ready.back();
        ready.pop_back();
        order.push_back(i);
        for (size_t j : out[i])
            if (--indeg[j] == 0) ready.push_back(j);
    }
    std::vector<he_batch_graph::NodeFix> fixes;
    cudaGraphNode_t copy = nullptr;
    const int lists[4] = {S.n_intt1, S.n_ntt_up, S.n_intt2, S.n_ntt_last};
    for (size_t i : order) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        if (ty == cudaGraphNodeTypeMemcpy && i == order[0]) copy = nodes[i];
        if (ty != cudaGraphNodeTypeKernel) continue;
        he_batch_graph::NodeFix f;
        f.node = nodes[i];
        if (cudaGraphKernelNodeGetParams(nodes[i], &f.p) != cudaSuccess) {
            (void)cudaGetLastError();
            return;
        }
        if (fixes.size() >= log.size()) return;
        f.tag = log[fixes.size()];
        f.tiles = 1;
        if (f.tag >= kTagNtt0 && f.tag < kTagNtt0 + 4) {
            const int t = f.tag - kTagNtt0;
            if (lists[t] < 1 || f.p.gridDim.x % (unsigned)lists[t]) return;
            f.tiles = f.p.gridDim.x / (unsigned)lists[t];
        }
        fixes.push_back(f);
    }
    if (fixes.size() == log.size()) {
        g->fixes = fixes;
        g->memcpy_node = copy;
    }
}

}  // namespace

extern "C" {

size_t he_batch_graph_workspace_bytes(const he_ctx *c, int max_jobs)
{
    if (!c || max_jobs < 1 || max_jobs > 65535 || c->L < 2) return 0;
    he_batch_graph g;
    graph_layout(c, max_jobs, &g, 1);
    return g.hdr + (size_t)max_jobs * g.slot_limbs * c->N * sizeof(u64);
}

int he_batch_graph_create(he_ctx *c, int max_jobs, const uint64_t *evk, void *ws, size_t ws_bytes, void *stream,
                          he_batch_graph **out)
{
    if (check_dev(c) || !evk || !ws || !out || !aligned(ws) || !aligned(evk)) return HE_EINVAL;
    if (max_jobs < 1 || max_jobs > 65535 || c->L < 2) return HE_EINVAL;
    if (ws_bytes < he_batch_graph_workspace_bytes(c, max_jobs)) return HE_ENOMEM;
    he_batch_graph *g = new (std::nothrow) he_batch_graph();
    if (!g) return HE_ENOMEM;
    g->c = c;
    g->max_jobs = max_jobs;
    g->evk = evk;
    g->ws = (char *)ws;
    graph_layout(c, max_jobs, g, c->group_cap);
    // capture runs nothing, so it uses a private stream: capture is not
    // permitted on the legacy default stream the caller may be using
    (void)stream;
    cudaStream_t st = nullptr;
    auto fail = [&](int rc) {
        if (st) cudaStreamDestroy(st);
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        for (int b = 0; b < 2; b++) {
            if (g->done[b]) cudaEventDestroy(g->done[b]);
            if (g->pinned[b]) cudaFreeHost(g->pinned[b]);
        }
        delete g;
        return rc;
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fail(HE_ECUDA);
    for (int b = 0; b < 2; b++) {
        if (cudaMallocHost((void **)&g->pinned[b], g->hdr) != cudaSuccess) return fail(HE_ENOMEM);
        memset(g->pinned[b], 0, g->hdr);  // level-0 items: every block exits
        if (cudaEventCreateWithFlags(&g->done[b], cudaEventDisableTiming) != cudaSuccess) return fail(HE_ECUDA);
    }
    const bool prof = c->prof;
    c->prof = false;
    JobRef R;
    R.items = (const BatchItem *)g->ws;
    memset(&R.one, 0, sizeof(R.one));
    R.B = max_jobs;
    R.lmax = c->L;
    R.trigger = c->pdl >= 2;
    Stages Sg;
    const NttGroup **lp[4] = {&Sg.intt1, &Sg.ntt_up, &Sg.intt2, &Sg.ntt_last};
    int *np[4] = {&Sg.n_intt1, &Sg.n_ntt_up, &Sg.n_intt2, &Sg.n_ntt_last};
    for (int t = 0; t < 4; t++) {
        *lp[t] = (const NttGroup *)(g->ws + g->lists_off[t]);
        *np[t] = g->list_max[t];
    }
    Sg.counts = (const int *)(g->ws + g->counts_off);
    if (use_shared_ip(c, max_jobs)) {
        g->ip_jobs = c->ip_jobs;
        Sg.ipg = (const IpGroup *)(g->ws + g->ipg_off);
        Sg.n_ipg = (max_jobs + g->ip_jobs - 1) / g->ip_jobs;
    }
    u64 *data = (u64 *)(g->ws + g->hdr);
    int rc = HE_OK;
    cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) {
        c->prof = prof;
        g_last_cuda_error = cudaGetErrorName(ce);
        return fail(HE_ECUDA);
    }
    ce = cudaMemcpyAsync(g->ws, g->pinned[0], g->hdr_copy, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) {
        g_last_cuda_error = cudaGetErrorName(ce);
        rc = HE_ECUDA;
    }
    std::vector<int> log;
    capture_log = &log;
    if (rc == HE_OK) rc = run_pipeline(c, R, data, Sg, evk, kTailRescale, st);
    capture_log = nullptr;
    capture_tag = kTagFixed;
    ce = cudaStreamEndCapture(st, &g->graph);
    c->prof = prof;
    if (ce != cudaSuccess) g_last_cuda_error = cudaGetErrorName(ce);
    if (rc != HE_OK || ce != cudaSuccess) return fail(rc != HE_OK ? rc : HE_ECUDA);
    ce = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (ce != cudaSuccess) {
        g_last_cuda_error = cudaGetErrorName(ce);
        return fail(HE_ECUDA);
    }
    graph_match_nodes(g, log, Sg);
    cudaStreamDestroy(st);
    *out = g;
    return HE_OK;
}

int he_batch_graph_launch(he_batch_graph *g, int count, const he_job *jobs, void *stream)
{
    if (!g || !jobs || count < 1 || count > g->max_jobs) return HE_EINVAL;
    he_ctx *c = g->c;
    for (int i = 0; i < count; i++) {
        const he_job &j = jobs[i];
        if (!j.ct1 || !j.ct2 || !j.out || !aligned(j.ct1) || !aligned(j.ct2) || !aligned(j.out)) return HE_EINVAL;
        if (j.level < 2 || j.level > c->L) return HE_ELEVEL;
    }
    // the launch that last read this pinned header must have finished
    const int b = g->memcpy_node ? (int)(g->nlaunch & 1u) : 0;
    if (g->launched[b] && cudaEventSynchronize(g->done[b]) != cudaSuccess) return HE_ECUDA;
    unsigned char *pin = g->pinned[b];
    const size_t N = (size_t)c->N;
    u64 *data = (u64 *)(g->ws + g->hdr);
    BatchItem *items = (BatchItem *)pin;
    memset(items, 0, sizeof(BatchItem) * g->max_jobs);
    std::vector<NttJob> lists[4];
    for (int i = 0; i < count; i++) {
        const HostLevel &H = c->host_levels[jobs[i].level];
        const size_t off = (size_t)i * g->slot_limbs;
        items[i].ct1 = jobs[i].ct1;
        items[i].ct2 = jobs[i].ct2;
        items[i].out = jobs[i].out;
        items[i].ws = data + off * N;
        items[i].level = jobs[i].level;
        const std::vector<NttJob> *src[4] = {&H.intt1f, &H.ntt_up, &H.intt2f, &H.ntt_z};
        for (int t = 0; t < 4; t++)
            for (NttJob j : *src[t]) {
                j.src += (unsigned)off;
                j.dst += (unsigned)off;
                j.cd += (unsigned)off;
                j.cks += (unsigned)off;
                j.job = (unsigned)i;
                lists[t].push_back(j);
            }
    }
    int *counts = (int *)(pin + g->counts_off);
    for (int t = 0; t < 4; t++) {
        std::vector<NttGroup> grp = group_jobs(lists[t], std::max(c->group_cap, g->cap));
        if ((int)grp.size() > g->list_max[t]) return HE_EINVAL;  // cannot happen: bounded at capture
        memcpy(pin + g->lists_off[t], grp.data(), sizeof(NttGroup) * grp.size());
        counts[t] = (int)grp.size();
    }
    if (g->ip_jobs) {
        std::vector<int> lv(count);
        for (int i = 0; i < count; i++) lv[i] = jobs[i].level;
        const std::vector<IpGroup> ipg = ip_groups(lv.data(), count, g->ip_jobs);
        memcpy(pin + g->ipg_off, ipg.data(), sizeof(IpGroup) * ipg.size());
        counts[4] = (int)ipg.size();
    }
    // the header copy reads this launch's pinned buffer; every kernel node is
    // sized to this batch (the updates apply to this launch, not to one that
    // is still running)
    if (g->memcpy_node &&
        cudaGraphExecMemcpyNodeSetParams1D(g->exec, g->memcpy_node, g->ws, pin, g->hdr_copy,
                                           cudaMemcpyHostToDevice) != cudaSuccess)
        return HE_ECUDA;
    for (const he_batch_graph::NodeFix &f : g->fixes) {
        cudaKernelNodeParams p = f.p;
        if (f.tag >= kTagNtt0 && f.tag < kTagNtt0 + 4)
            p.gridDim.x = (unsigned)std::max(1, counts[f.tag - kTagNtt0]) * f.tiles;
        else if (f.tag == kTagJobs)
            p.gridDim.z = (unsigned)count;
        else if (f.tag == kTagIpGroups)
            p.gridDim.z = (unsigned)std::max(1, counts[4]);
        else
            continue;
        if (cudaGraphExecKernelNodeSetParams(g->exec, f.node, &p) != cudaSuccess) return HE_ECUDA;
    }
    cudaStream_t st = S(stream);
    if (cudaGraphLaunch(g->exec, st) != cudaSuccess) return HE_ECUDA;
    if (cudaEventRecord(g->done[b], st) != cudaSuccess) return HE_ECUDA;
    g->launched[b] = true;
    g->nlaunch++;
    return HE_OK;
}

int he_batch_graph_destroy(he_batch_graph *g)
{
    if (!g) return HE_EINVAL;
    for (int b = 0; b < 2; b++)
        if (g->launched[b]) cudaEventSynchronize(g->done[b]);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    for (int b = 0; b < 2; b++) {
        if (g->done[b]) cudaEventDestroy(g->done[b]);
        if (g->pinned[b]) cudaFreeHost(g->pinned[b]);
    }
    delete g;
    return HE_OK;
}

}  // extern "C"
