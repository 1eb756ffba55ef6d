// he_internal.h -- internal types shared by the host and device translation
// units of the library (not part of the public ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "he.h"

typedef uint64_t u64;

namespace he {

constexpr int kMaxDigits = 16;
// digits the fused key-switch sums of an NTT pass's tile load take (ip_tile)
constexpr int kIpFuseDigits = 4;
constexpr int kMaxK = 16;
constexpr int kMaxL = 64;

// One prime as the kernels see it (ext order: specials first, then q_0..).
struct DevPrime {
    u64 q, q2, q4;          // q, 2q, 4q
    u64 r64;                // floor(2^64 / q): Shoup companion of 1, for final reductions
    u64 mu;                 // Barrett: floor(2^(64+s) / q)
    unsigned s, pad;        // s = bitlen(q) - 2
    const ulonglong2 *w;    // forward twiddles: w[m+j] = psi^bitrev(m+j), (value, Shoup)
    const ulonglong2 *iw;   // inverse twiddles: psi^-bitrev(m+j)
};

// One limb transform of an NTT launch.  Offsets are in limbs (units of N
// words) from the launch's base pointer.  scale (with its Shoup companion) is
// applied to inverse-transform outputs together with N^-1.
struct NttJob {
    unsigned src, dst, prime, pad;
    u64 scale, scale_sh;
    // fused final combine (forward NTT of the ModDown + rescale limbs): job
    // index in the launch, h << 31 | i, and the limbs d_h[i] and KS_h[K+i]
    unsigned job, ci, cd, cks;
};

// What the NTT kernels consume: up to kGroupMax limb transforms that share a
// prime, so one CTA stages that prime's twiddles once and reuses them.
constexpr int kGroupMax = 4;
struct NttGroup {
    unsigned prime, nl, pad0, pad1;
    unsigned src[kGroupMax], dst[kGroupMax];
    u64 scale[kGroupMax], scale_sh[kGroupMax];
    unsigned job[kGroupMax], ci[kGroupMax], cd[kGroupMax], cks[kGroupMax];  // NttJob's combine fields
};

// Group single-limb jobs by prime, at most `cap` limbs per group (order
// within a prime is kept); the groups come out sorted by prime.
std::vector<NttGroup> group_jobs(const std::vector<NttJob> &jobs, int cap = kGroupMax);

// Per-level constants on the device.
struct DevLevel {
    int l, beta, E, A;             // level, digits, K+l, alpha padded for the kernels
    int dig_lo[kMaxDigits], dig_n[kMaxDigits];
    // workspace layout of one HE Mul at this level (limb offsets from the job's ws)
    unsigned o_d0, o_d1, o_d2, o_y, o_u, o_ks, o_ys, o_r, o_z, o_total;
    const u64 *modupB;             // [beta][E][A]: [Qhat_{j,i}]_t split at bit 28, zero-padded
    const ulonglong2 *qinv_last;   // [l-1]: q_{l-1}^-1 mod q_i (value, Shoup)
    const ulonglong2 *pinv_qinv;   // [l-1]: P^-1 * q_{l-1}^-1 mod q_i
    const u64 *pbpq;               // [l-1][KP]: [Phat_k P^-1 q_{l-1}]_{q_i} (one division by P q_{l-1})
};

// One HE Mul of a launch: its operands, output, workspace base and level.
// Kernels take a JobRef: either a device array of items (batched execution,
// item = blockIdx.z) or one item by value (a single HE Mul).
struct BatchItem {
    const u64 *ct1, *ct2;
    u64 *out, *ws;
    int level, pad;
};
struct JobRef {
    const BatchItem *items;  // device array, or nullptr to use `one`
    BatchItem one;
    int B;                   // number of jobs
    int lmax;                // largest level among them
    int trigger;             // early dependent launch (the shape's pdl = 2): see griddep_wait
};
#ifdef __CUDACC__
__device__ __forceinline__ BatchItem job_item(const JobRef &R, int z) { return R.items ? R.items[z] : R.one; }
#endif

// Batched inner product with shared key tiles: the jobs of a batch, sorted by
// level (highest first), are cut into groups of at most kIpJobsMax; one CTA
// loads the evaluation-key words of its (limb, coefficients) once and forms
// the products of every job of its group with them.  `level` is the group's
// highest level (its first job's).
constexpr int kIpJobsMax = 8;
struct IpGroup {
    int n, level, pad0, pad1;
    int job[kIpJobsMax];
};
// Groups of at most `per` jobs (1..kIpJobsMax) over jobs sorted by level,
// highest first (ties keep the batch order).
std::vector<IpGroup> ip_groups(const int *levels, int count, int per);

// Workspace layout of one HE Mul at level l (offsets in limbs).
struct WsLayout {
    size_t d0, d1, d2, y, u, ks, ys, r, z, total;
};

// Job lists of one level, stored in the context's device arena (one set
// per group cap 1..kGroupMax; jobs[l] is the set of the context's cap).
struct LevelJobs {
    const NttGroup *intt1;    int n_intt1;     // d2 -> y          (+2 fused: d0,d1 last limb -> r[0..1])
    const NttGroup *intt1f;   int n_intt1f;    // fused variant
    const NttGroup *ntt_up;   int n_ntt_up;    // ModUp outputs, in place
    const NttGroup *intt2;    int n_intt2;     // KS specials -> ys (scaled by N^-1 Phat^-1)
    const NttGroup *intt2f;   int n_intt2f;    // + KS last limb -> r[2..3]
    const NttGroup *intt2pq;  int n_intt2pq;   // intt2f with Phat^-1 q_{l-1}^-1 scales (one division by P q_{l-1})
    const NttGroup *ntt_conv; int n_ntt_conv;  // 2l conv limbs (plain ModDown)
    const NttGroup *ntt_z;    int n_ntt_z;     // 2(l-1) z limbs (fused ModDown + rescale)
    const NttGroup *rs_intt;  int n_rs_intt;   // rescale: last limb of b, a -> r
    const NttGroup *rs_ntt;   int n_rs_ntt;    // rescale: r -> z_i
};

struct HostLevel {
    WsLayout ws;
    std::vector<NttJob> intt1, intt1f, ntt_up, intt2, intt2f, ntt_conv, ntt_z, rs_intt, rs_ntt, intt2pq;
    std::vector<u64> modupB;
    std::vector<u64> pbpq;  // [l-1][KP]: [Phat_k P^-1 q_{l-1}]_{q_i}, split at bit 28 (one division by P q_{l-1})
    std::vector<ulonglong2> qinv_last, pinv_qinv;
};

}  // namespace he

struct he_ctx {
    he_params prm;
    int N, logN, L, K, alpha, dnum, E;  // E = K + L
    int AP, KP;                          // alpha and K padded to a kernel width (1,2,4,8,12,16)
    bool device;
    // launch shapes (speed only; he_autotune / he_set_shape): NTT limbs per
    // group (1..kGroupMax) and ModUp targets per CTA (4, 8 or 16)
    int group_cap = he::kGroupMax;
    int modup_chunk = 8;
    int pdl = 1;                         // programmatic dependent launch between the path's kernels:
                                         // 0 off, 1 on, 2 on with early dependent launch (griddep_wait)
    int ntt_r8 = 0;                      // bit s: the radix-8 NTT plan at pipeline NTT site s (0..3)
    int ntt_split = 0;                   // NTT pass split of every site (0 default, 1, 2: see launch_ntt)
    int ntt_small = 0;                   // bit s: 1024-element NTT tiles at pipeline NTT site s (2^16, 2^17)
    int ntt_onepass = 0;                 // bit s: one-pass cluster transform at pipeline NTT site s (2^16)
    int ip_jobs = he::kIpJobsMax;        // batches: jobs sharing one CTA's key words in the inner product (1: none)
    int fuse = 7;                        // bit 0: the tensor product inside the first inverse NTT pass of d2;
                                         // bit 1: the q limbs' key-switch sums beside the ModDown conversion;
                                         // bit 2: the special limbs' sums inside their iNTT's first pass
    std::vector<u64> ext;                // moduli, ext order
    std::vector<u64> psi;                // smallest primitive 2N-th roots, ext order
    // host tables (for the host NTT used by keygen / encrypt / decrypt)
    std::vector<std::vector<u64>> w, wsh, iw, iwsh;  // [E][N]
    std::vector<u64> ninv, ninv_sh;                  // [E]
    // level-independent ModDown constants
    std::vector<u64> PB;                 // [L][KP]: [Phat_k]_{q_i} split at bit 28, zero-padded
    std::vector<u64> PBP;                // [L][KP]: [Phat_k P^-1]_{q_i}, same format (fused ModDown)
    std::vector<ulonglong2> pinv;        // [L]: P^-1 mod q_i
    std::vector<ulonglong2> phat_inv;    // [K]: Phat_k^-1 mod p_k
    std::vector<he::HostLevel> host_levels;  // index l (1..L)
    // device
    int device_id = -1;
    void *arena = nullptr;               // one allocation holding every device table
    size_t arena_bytes = 0;
    he::DevPrime *d_primes = nullptr;    // [E]
    const u64 *d_PB = nullptr;
    const u64 *d_PBP = nullptr;
    const ulonglong2 *d_pinv = nullptr;
    std::vector<he::DevLevel> dev_levels;  // index l (host copy of the device structs)
    he::DevLevel *d_levels = nullptr;      // [L+1]
    // evaluation keys stored as b halves only (he_evk_register_seeded): the
    // device pointer and the SplitMix64 stream state of each digit's a halves
    struct SeededKey {
        const u64 *ptr;
        u64 state[he::kMaxDigits];
    };
    std::vector<SeededKey> seeded;
    std::vector<he::LevelJobs> jobs;       // index l: the lists of group_cap
    std::vector<he::LevelJobs> jobs_cap[he::kGroupMax];  // [cap-1][l]: every cap's lists
    // optional per-kernel event marks (he_profile); consecutive marks on one
    // stream bracket one kernel each
    mutable bool prof = false;
    mutable std::vector<cudaEvent_t> prof_pool;
    mutable std::vector<std::string> prof_names;  // prof_names[i] = kernel ended by event i ("" = a start mark)
    mutable size_t prof_used = 0;
    // host-stream entry point: two upload streams (one per operand, so both
    // copies run at once) and a download stream and, per staging slot, the
    // events ordering a job's uploads, path and download
    // (created on first use, under io_mu)
    std::mutex io_mu;
    cudaStream_t io_h2d = nullptr, io_h2d2 = nullptr, io_d2h = nullptr;
    cudaEvent_t io_ev[4][4] = {};
};

namespace he {
// host_params.cpp
int build_context(he_ctx *ctx, const he_params *p, bool device);
// kernels (ntt.cu, keyswitch.cu); return cudaError_t
// Record a profiling mark named after the kernel that just finished (no-op
// unless profiling is enabled on the context).
void prof_mark(const he_ctx *ctx, cudaStream_t st, const char *tag, const char *suffix = nullptr);
// ngroups > 0 launches; dev_count (optional) bounds the groups on the device.
// Kernel launch with programmatic dependent launch allowed when `dep` is
// set: the kernel's CTAs may be scheduled while the previous kernel on the
// stream drains, so every such kernel executes griddep_wait() before it
// touches memory that earlier work on the stream produces or reads (static
// tables may be read before).  Errors are left for cudaGetLastError().
//
// While a batch graph is being captured (capture_log set on this thread),
// every launch appends capture_tag, the kind of grid the caller set before
// it, so that the graph can resize each kernel node to the batch it runs.
enum LaunchTag {
    kTagNtt0 = 0,   // NTT launches over group list t (0..3): grid.x = groups x tiles
    kTagJobs = 8,   // per-job kernels: grid.z = jobs
    kTagIpGroups,   // the shared-key inner product: grid.z = its job groups
    kTagFixed       // not resized
};
extern thread_local std::vector<int> *capture_log;
extern thread_local int capture_tag;

template <typename... KArgs, typename... Args>
inline void launch_k(bool dep, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args)
{
    if (capture_log) capture_log->push_back(capture_tag);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = dep ? at : nullptr;
    cfg.numAttrs = dep ? 1 : 0;
    (void)cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

#ifdef __CUDACC__
// Wait for the previous kernel on the stream (a no-op without a programmatic
// dependency).  With `trigger`, then allow the next kernel to be launched:
// once every CTA of this grid has passed this point (the grid's last wave is
// running), the next kernel's CTAs may occupy the SMs this grid's tail leaves
// idle and run their prologue; they wait in their own griddep_wait for this
// grid's completion and memory flush before touching its data.  Without it
// the next kernel is launched as this grid's CTAs exit.
__device__ __forceinline__ void griddep_wait(bool trigger = false)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (trigger) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Exit of a CTA with no work.  It still waits for the previous kernel first:
// a kernel launched after this one waits only for this kernel's completion,
// so this kernel must not complete before its own predecessor has, even when
// none of its CTAs has work (ordering is then transitive along the stream).
// Tables that only the host writes (job items, NTT group lists and their
// counts, copied before a launch sequence's first kernel) may be read before
// the wait; nothing a kernel writes is.
__device__ __forceinline__ void idle_exit() { griddep_wait(); }

// L2 eviction policies.  Streams read once per HE Mul (the evaluation key,
// the input ciphertexts, ModUp outputs) are marked evict-first, so they pass
// through L2 without displacing the NTT twiddle tables, which every HE Mul
// rereads and which are marked evict-last.
__device__ __forceinline__ u64 l2_policy_stream()
{
    u64 p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ u64 l2_policy_keep()
{
    u64 p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// 16-byte read-only load with an L2 policy, no L1 allocation.
__device__ __forceinline__ ulonglong2 ld2_hint(const void *p, u64 pol)
{
    ulonglong2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
                 : "=l"(v.x), "=l"(v.y) : "l"(p), "l"(pol));
    return v;
}
#endif

// plan: bit 0 the radix-8 plan (256 threads per tile) instead of the
// radix-16 one; bits 1-2 the pass split (0 default, 1 one stage from the
// strided pass to the contiguous one, 2 the other way; 2^16 and 2^17 only);
// bit 3 tiles of 1024 elements instead of 2048 (2^16 and 2^17 only).  Every
// plan gives the same words.
cudaError_t launch_ntt(const he_ctx *ctx, u64 *base, const NttGroup *groups, int ngroups, bool inverse,
                       cudaStream_t st, const char *tag = nullptr, const int *dev_count = nullptr, int plan = 0);
cudaError_t launch_ntt2(const he_ctx *ctx, const u64 *src, u64 *dst, const NttGroup *groups, int ngroups,
                        bool inverse, cudaStream_t st, const char *tag = nullptr, const int *dev_count = nullptr,
                        int plan = 0);
cudaError_t configure_ntt(const he_ctx *ctx);
// Forward NTT of the fused ModDown + rescale limbs with the final combine in
// its last pass: out[h][i] = (d_h[i] + KS_h[K+i] P^-1 - NTT(z)) q_{l-1}^-1,
// written to each job's output (groups carry the combine fields).
cudaError_t launch_ntt_combine(const he_ctx *ctx, u64 *base, const NttGroup *groups, int ngroups, const JobRef &R,
                               cudaStream_t st, const char *tag = nullptr, const int *dev_count = nullptr,
                               int plan = 0);
// Inverse NTT of d2 (and the rescale limbs of d0, d1) whose first pass forms
// its input tiles with the tensor product from each job's ciphertexts and
// stores d0, d1, d2 to the job's workspace (groups carry job and ci = limb |
// product << 16 | keep << 18).
cudaError_t launch_ntt_tensor(const he_ctx *ctx, u64 *base, const NttGroup *groups, int ngroups, const JobRef &R,
                              cudaStream_t st, const char *tag = nullptr, const int *dev_count = nullptr,
                              int plan = 0);
// The special limbs' inverse NTT whose first pass computes its input, the
// key-switch sums KS_h[e] of the group limbs (ci = e | h << 16) from U, d2
// and the (unseeded) evaluation key, instead of loading it.
cudaError_t launch_ntt_ip(const he_ctx *ctx, u64 *base, const NttGroup *groups, int ngroups, const JobRef &R,
                          const u64 *evk, cudaStream_t st, const char *tag, const int *dev_count, int plan);
// Number of final stages (the contiguous pass's last round) whose twiddle
// runs the device table stores transposed; 0 for an unsupported logN.
int ntt_direct_stages(int logN);
cudaError_t run_tensor(const he_ctx *c, const JobRef &R, cudaStream_t st);
// ModUp outputs lazily in [0, 3q) (the forward NTT that follows reduces them),
// or canonical residues (the per-step entry point).
cudaError_t run_modup(const he_ctx *c, const JobRef &R, cudaStream_t st, bool canonical = false);
// Element-wise ops: 0 add, 1 sub, 2 times plaintext, 3 plus plaintext (b half).
cudaError_t run_elementwise(const he_ctx *c, int op, const u64 *x, const u64 *y, u64 *out, int l, cudaStream_t st);
// Rotation's first step: d0 = kappa_g(b), d1 = 0, d2 = -kappa_g(a) into ws (level l).
cudaError_t run_automorph(const he_ctx *c, const u64 *ct, u64 *ws, int l, u64 g, cudaStream_t st);
// rows (IpRows in keyswitch.cu): 0 every ext limb; 1 the special limbs and the
// last q limb; 2 the special limbs; 3 the q limbs but the last; 4 the q limbs.
enum { kIpAllRows = 0, kIpSpecialLastRows = 1, kIpSpecialRows = 2 };
cudaError_t run_inner_product(const he_ctx *c, const JobRef &R, const u64 *evk, cudaStream_t st,
                              int rows = kIpAllRows);
// The ModDown conversion (rescaling tails) and the key-switch sums of the q
// limbs but the last in one launch (after run_inner_product of the special
// limbs and the last q limb).  Single jobs; moddown_ipq_fits says whether the
// context's sizes have an instantiation.
bool moddown_ipq_fits(const he_ctx *c);
cudaError_t run_moddown_ipq(const he_ctx *c, const JobRef &R, int mode, const u64 *evk, cudaStream_t st);
// The batched inner product with key words shared by the jobs of each group
// (ngroups launched; dev_count, optional, bounds the groups on the device).
bool inner_product_shared_fits(const he_ctx *c);  // the shared kernel covers at most four digits
cudaError_t run_inner_product_shared(const he_ctx *c, const JobRef &R, const IpGroup *groups, int ngroups,
                                     const int *dev_count, const u64 *evk, cudaStream_t st);
// The key switch's tail: ModDown alone, ModDown then rescale (two floors,
// bit-identical to he_mul then he_rescale), or one division by P q_{l-1}.
enum TailMode { kTailPlain = 0, kTailRescale = 1, kTailRescalePQ = 2 };
cudaError_t run_moddown_conv(const he_ctx *c, const JobRef &R, int mode, cudaStream_t st);
cudaError_t run_combine_plain(const he_ctx *c, const JobRef &R, cudaStream_t st);
cudaError_t run_rescale_combine(const he_ctx *c, const u64 *ct, const u64 *Z, u64 *out, int l, cudaStream_t st);
}  // namespace he
