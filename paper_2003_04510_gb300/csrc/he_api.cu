// he_api.cu -- the C ABI entry points: context lifetime, workspace sizing,
// and the orchestration of HE Mul / rescale as a sequence of kernels on the
// caller's stream.  No entry point allocates device memory on the hot path:
// the caller passes the workspace.
#include <algorithm>
#include <cstring>
#include <new>

#include "he_internal.h"

using namespace he;

namespace he {

void prof_mark(const he_ctx *c, cudaStream_t st, const char *tag, const char *suffix)
{
    if (!c->prof || c->prof_used >= c->prof_pool.size()) return;
    std::string name = tag ? tag : "";
    if (suffix) name += suffix;
    c->prof_names[c->prof_used] = name;
    cudaEventRecord(c->prof_pool[c->prof_used], st);
    c->prof_used++;
}

}  // namespace he

namespace {

inline cudaStream_t S(void *s) { return (cudaStream_t)s; }

#define HE_TRY(x)                                  \
    do {                                           \
        cudaError_t e_ = (x);                      \
        if (e_ != cudaSuccess) return HE_ECUDA;    \
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

// The HE Mul pipeline at level l.  fused = ModDown and rescale merged (out is
// [2][l-1][N]); otherwise out is the level-l product ([2][l][N]).
int hemul_pipeline(he_ctx *c, const u64 *ct1, const u64 *ct2, const u64 *evk, int l, u64 *out, u64 *ws,
                   bool fused, cudaStream_t st)
{
    const WsLayout &W = c->host_levels[l].ws;
    const LevelJobs &J = c->jobs[l];
    const size_t N = (size_t)c->N;
    u64 *d0 = ws + W.d0 * N, *d1 = ws + W.d1 * N, *d2 = ws + W.d2 * N;
    prof_mark(c, st, "");
    // Region 1: tensor product
    HE_TRY(run_tensor(c, ct1, ct2, d0, d1, d2, l, st));
    prof_mark(c, st, "tensor");
    // key switching: iNTT(d2) (times N^-1 Qhat^-1), ModUp, NTT, inner product
    HE_TRY(launch_ntt(c, ws, fused ? J.intt1f : J.intt1, fused ? J.n_intt1f : J.n_intt1, true, st, "intt_d2"));
    HE_TRY(run_modup(c, ws + W.y * N, ws + W.u * N, l, st));
    prof_mark(c, st, "modup");
    HE_TRY(launch_ntt(c, ws, J.ntt_up, J.n_ntt_up, false, st, "ntt_modup"));
    HE_TRY(run_inner_product(c, ws + W.u * N, d2, evk, ws + W.ks * N, l, st));
    prof_mark(c, st, "inner_product");
    // ModDown: iNTT of the special limbs (times N^-1 Phat^-1), conversion, NTT
    HE_TRY(launch_ntt(c, ws, fused ? J.intt2f : J.intt2, fused ? J.n_intt2f : J.n_intt2, true, st, "intt_special"));
    HE_TRY(run_moddown_conv(c, ws + W.ys * N, ws + W.r * N, ws + W.z * N, l, fused, st));
    prof_mark(c, st, "moddown_conv");
    if (fused) {
        HE_TRY(launch_ntt(c, ws, J.ntt_z, J.n_ntt_z, false, st, "ntt_moddown"));
        HE_TRY(run_combine_rescale(c, d0, d1, ws + W.ks * N, ws + W.z * N, out, l, st));
        prof_mark(c, st, "combine_rescale");
    } else {
        HE_TRY(launch_ntt(c, ws, J.ntt_conv, J.n_ntt_conv, false, st, "ntt_moddown"));
        HE_TRY(run_combine_plain(c, d0, d1, ws + W.ks * N, ws + W.z * N, out, l, st));
        prof_mark(c, st, "combine");
    }
    return HE_OK;
}

}  // namespace

extern "C" {

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
    return hemul_pipeline(c, ct1, ct2, evk, level, out, (u64 *)ws, false, S(stream));
}

int he_mul_rescale(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk, int level,
                   uint64_t *out, void *ws, size_t ws_bytes, void *stream)
{
    if (check_dev(c) || !ct1 || !ct2 || !evk || !out || !ws) return HE_EINVAL;
    if (level < 2 || level > c->L) return HE_ELEVEL;
    if (!aligned(ct1) || !aligned(ct2) || !aligned(out) || !aligned(ws) || !aligned(evk)) return HE_EINVAL;
    if (ws_bytes < ws_bytes_for(c, level)) return HE_ENOMEM;
    return hemul_pipeline(c, ct1, ct2, evk, level, out, (u64 *)ws, true, S(stream));
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
    cudaError_t e = launch_ntt(c, (u64 *)data, dj, (int)groups.size(), inverse != 0, st);
    cudaFreeAsync(dj, st);
    return e == cudaSuccess ? HE_OK : HE_ECUDA;
}

int he_step_tensor(he_ctx *c, const uint64_t *ct1, const uint64_t *ct2, int level, uint64_t *d, void *stream)
{
    if (check_dev(c) || !ct1 || !ct2 || !d) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    const size_t lN = (size_t)level * c->N;
    HE_TRY(run_tensor(c, ct1, ct2, d, d + lN, d + 2 * lN, level, S(stream)));
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
    u64 *w = (u64 *)ws;
    cudaStream_t st = S(stream);
    HE_TRY(cudaMemcpyAsync(w + W.d2 * N, d2, (size_t)level * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    HE_TRY(launch_ntt(c, w, J.intt1, J.n_intt1, true, st));
    HE_TRY(run_modup(c, w + W.y * N, (u64 *)U, level, st));
    return HE_OK;
}

int he_step_inner_product(he_ctx *c, const uint64_t *U, const uint64_t *d2, const uint64_t *evk, int level,
                          uint64_t *KS, void *stream)
{
    if (check_dev(c) || !U || !d2 || !evk || !KS) return HE_EINVAL;
    if (level < 1 || level > c->L) return HE_ELEVEL;
    HE_TRY(run_inner_product(c, U, d2, evk, KS, level, S(stream)));
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
    HE_TRY(run_moddown_conv(c, w + W.ys * N, w + W.r * N, w + W.z * N, level, false, st));
    HE_TRY(launch_ntt(c, w, J.ntt_conv, J.n_ntt_conv, false, st));
    // the combine writes both halves; the b half is the answer
    HE_TRY(run_combine_plain(c, w + W.d0 * N, w + W.d1 * N, w + W.ks * N, w + W.z * N, w + W.y * N, level, st));
    HE_TRY(cudaMemcpyAsync(out, w + W.y * N, (size_t)level * N * sizeof(u64), cudaMemcpyDeviceToDevice, st));
    return HE_OK;
}

}  // extern "C"

extern "C" {

size_t he_batch_workspace_bytes(const he_ctx *c, int count, const int *levels)
{
    if (!c || count < 1 || !levels) return 0;
    size_t total = 0;
    for (int i = 0; i < count; i++) {
        if (levels[i] < 2 || levels[i] > c->L) return 0;
        total += (ws_bytes_for(c, levels[i]) + 255) & ~(size_t)255;
    }
    return total;
}

int he_mul_batch(he_ctx *c, int count, const he_job *jobs, const uint64_t *evk, void *ws, size_t ws_bytes,
                 void *stream)
{
    if (check_dev(c) || count < 1 || !jobs || !evk || !ws) return HE_EINVAL;
    size_t need = 0;
    for (int i = 0; i < count; i++) {
        const he_job &j = jobs[i];
        if (!j.ct1 || !j.ct2 || !j.out) return HE_EINVAL;
        if (j.level < 2 || j.level > c->L) return HE_ELEVEL;
        need += (ws_bytes_for(c, j.level) + 255) & ~(size_t)255;
    }
    if (ws_bytes < need) return HE_ENOMEM;
    char *w = (char *)ws;
    for (int i = 0; i < count; i++) {
        const he_job &j = jobs[i];
        int rc = hemul_pipeline(c, j.ct1, j.ct2, evk, j.level, j.out, (u64 *)w, true, S(stream));
        if (rc) return rc;
        w += (ws_bytes_for(c, j.level) + 255) & ~(size_t)255;
    }
    return HE_OK;
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
    int rc = hemul_pipeline(c, d1, d2, evk, level, dout, w, true, st);
    if (rc) return rc;
    HE_TRY(cudaMemcpyAsync(out, dout, 2 * (size_t)(level - 1) * limb, cudaMemcpyDeviceToHost, st));
    HE_TRY(cudaStreamSynchronize(st));
    return HE_OK;
}

}  // extern "C"
