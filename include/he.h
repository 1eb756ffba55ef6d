/*
 * he.h -- C ABI of the GB300 (sm_103a) full-RNS CKKS HE Mul library.
 *
 * The operations follow "HEAAN Demystified" (arXiv 2003.04510):
 *   - encryption c.ax = u*pk1 + e1, c.bx = u*pk0 + e0 + t, and the decryption
 *     relation c.bx = c.ax*sk + t + e'                     (Sec. 3.1)
 *   - rescale after each multiplication, q -> q/p         (Sec. 3.1)
 *   - HE Mul of two ciphertexts under the same modulus: the tensor product,
 *     then key switching of c1.ax*c2.ax with the evaluation key (Sec. 3.2,
 *     Fig. 2), in its full-RNS form with mod up / mod down (Sec. 7, Table 11)
 *   - NTT / iNTT (Algo 3, Algo 4)
 *
 * Data model (every array is uint64 residues in [0, q), limb-major):
 *   ciphertext at level l : [2][l][N], b (= c.bx) part first, then a (= c.ax);
 *                           NTT domain, bit-reversed evaluation order (the
 *                           output order of Algo 3).
 *   public key            : [2][L][N] (pk0 first, then pk1), NTT domain.
 *   evaluation key        : [dnum][2][K+L][N], b part first; limb order is
 *                           "ext": the K special primes first, then the L
 *                           ciphertext primes.  One key serves every level.
 *   secret key            : int64[N], coefficients in {-1, 0, 1}.
 * Level l means the ciphertext primes q_0..q_{l-1}; rescale drops q_{l-1}.
 *
 * Ownership: the caller owns every buffer (host arrays and device memory).
 * The library never frees caller memory.  A context owns only its parameter
 * tables (host and device copies).
 *
 * Device calls are asynchronous on the stream given (a cudaStream_t passed as
 * void*; NULL is the legacy default stream).  Device pointers must be
 * 256-byte aligned and must not overlap unless a function says otherwise.
 *
 * Errors: every call returns an int status (HE_OK on success).  Argument
 * errors are detected on the host before anything is enqueued.  A CUDA launch
 * failure returns HE_ECUDA.  Bounded device waits (batched and served
 * execution) that give up surface as HE_ETIMEOUT at the next synchronising
 * call.  he_strerror() names a code.
 */
#ifndef HE_GB300_H
#define HE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HE_OK = 0,
    HE_EINVAL = 1,   /* bad argument: NULL pointer, level out of range, bad size */
    HE_ELEVEL = 2,   /* operands at different or unsupported levels */
    HE_ENOMEM = 3,   /* workspace too small, or admission refused */
    HE_ECUDA = 4,    /* a CUDA runtime call failed */
    HE_ETIMEOUT = 5, /* a bounded device wait gave up */
    HE_EBUSY = 6     /* resource in use (e.g. serving slot pool exhausted) */
};

typedef struct he_ctx he_ctx;

/* Parameters of one ring / modulus chain (the paper's Table 3 and Table 6
 * list the non-RNS analogues).  Primes: q_0 > ... > q_{L-1} are the L largest
 * primes below 2^q_bits that are 1 mod 2N; p_0 > ... > p_{K-1} the K largest
 * below 2^p_bits that are 1 mod 2N and not ciphertext primes.  alpha = limbs
 * per key-switching digit; dnum = ceil(L/alpha).  h = Hamming weight of the
 * secret; sigma = error standard deviation (3.2 in the paper, Sec. 3.1). */
typedef struct {
    int logN;    /* 12 .. 17 */
    int L;       /* ciphertext primes, 1 .. 64 */
    int K;       /* special primes, 1 .. 16 */
    int alpha;   /* limbs per digit, 1 .. 16 */
    int q_bits;  /* 30 .. 57 */
    int p_bits;  /* 30 .. 57 */
    int h;       /* secret Hamming weight, 1 .. N */
    double sigma;
} he_params;

/* Create a context: generates the primes, roots and every table on the host
 * and uploads the device tables to the current CUDA device.  *out is set only
 * on success.  Returns HE_EINVAL for out-of-range parameters, HE_ECUDA if the
 * device upload fails (no device is needed when only host functions are
 * used: pass a context created with he_ctx_create_host). */
int he_ctx_create(he_ctx **out, const he_params *p);
/* Host-only context (no CUDA calls are made); device entry points return
 * HE_EINVAL on it. */
int he_ctx_create_host(he_ctx **out, const he_params *p);
int he_ctx_destroy(he_ctx *ctx);

/* Query: N, dnum, and the moduli in ext order (K specials then L ciphertext
 * primes; `moduli` must hold K+L words). */
int he_ctx_info(const he_ctx *ctx, int *N, int *dnum, uint64_t *moduli);

/* ---- host side (plain C buffers, caller-owned) --------------------------- */

/* Key generation from a seed (counter-based SplitMix64 streams).  Any output
 * pointer may be NULL to skip that key; pk and evk need sk's values, so sk is
 * always generated internally.  sk: int64[N]; pk: [2][L][N]; evk:
 * [dnum][2][K+L][N].  The evaluation key of digit j encrypts P*Qtilde_j*s^2,
 * Qtilde_j = 1 mod the primes of digit j and 0 mod the others (Fig. 2's evk,
 * full-RNS gadget). */
int he_keygen(he_ctx *ctx, uint64_t seed, int64_t *sk, uint64_t *pk, uint64_t *evk);
/* The same, from a given secret key. */
int he_keygen_from_sk(he_ctx *ctx, uint64_t seed, const int64_t *sk, uint64_t *pk, uint64_t *evk);

/* Encoding (Sec. 3.1): n = N/2 complex numbers, scaled by `scale` and rounded
 * to the nearest integer, into int64[N] coefficients via the canonical
 * embedding at the roots zeta^(5^k).  Decoding is the inverse evaluation
 * (coefficients are given as doubles already divided by the scale). */
int he_encode(he_ctx *ctx, const double *re, const double *im, size_t n, double scale, int64_t *coeffs);
int he_decode(he_ctx *ctx, const double *coeffs, double *re, double *im, size_t n);

/* Encryption at `level` of an integer plaintext (Sec. 3.1): u ZO(1/2), e0 and
 * e1 rounded Gaussians, drawn from `seed`.  ct: [2][level][N]. */
int he_encrypt_poly(he_ctx *ctx, const uint64_t *pk, const int64_t *pt, int level, uint64_t seed,
                    uint64_t *ct);
/* Encode + encrypt. */
int he_encrypt(he_ctx *ctx, const uint64_t *pk, const double *re, const double *im, size_t n, double scale,
               int level, uint64_t seed, uint64_t *ct);
/* Decryption relation (Sec. 3.1): returns the coefficient-form residues of
 * c.bx - c.ax*sk, m: [level][N]. */
int he_decrypt_poly(he_ctx *ctx, const int64_t *sk, const uint64_t *ct, int level, uint64_t *m);
/* Decrypt + decode.  Centres each coefficient using CRT over the first
 * min(level, 2) primes, which is exact while |coefficient| < q_0*q_1/2. */
int he_decrypt(he_ctx *ctx, const int64_t *sk, const uint64_t *ct, int level, double scale, double *re,
               double *im, size_t n);

/* ---- device side: caller-owned device memory, caller's stream ------------ */

/* Copy an evaluation key (Fig. 2, region 2: the key switch's evk, as
 * he_keygen writes it) from host to device memory; evk_dev holds
 * dnum*2*(K+L)*N words.  Asynchronous on `stream`.  HE_EINVAL for a NULL
 * pointer or a host-only context, HE_ECUDA if the copy cannot be queued. */
int he_evk_upload(he_ctx *ctx, const uint64_t *evk_host, uint64_t *evk_dev, void *stream);

/* Bytes of device workspace one he_mul / he_rescale / he_mul_rescale call at
 * `level` needs (the largest of the three): the intermediates of Fig. 2 in
 * RNS form (region 1's d0, d1, d2; region 2's ModUp limbs of every digit,
 * key-switch sums and special limbs' iNTT) and the rescale's (Sec. 3.1).  0
 * for a level outside 1..L. */
size_t he_workspace_bytes(const he_ctx *ctx, int level);

/* HE Mul (Fig. 2, full-RNS form): out = (d0 + ModDown(KS_b), d1 + ModDown(KS_a))
 * where d0 = b1*b2, d1 = a1*b2 + a2*b1, d2 = a1*a2 and KS = sum_j
 * ModUp_j(d2) * evk_j.  ct1, ct2, out: [2][level][N] device; out may not alias
 * the inputs.  Result scale is scale1*scale2 (host metadata).  Returns
 * HE_ELEVEL if level is outside 1..L, HE_ENOMEM if ws_bytes is too small. */
int he_mul(he_ctx *ctx, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk_dev, int level,
           uint64_t *out, void *ws, size_t ws_bytes, void *stream);

/* Rescale (Sec. 3.1, "divide by p"): out = floor(ct / q_{level-1}) in RNS form,
 * [2][level-1][N].  level >= 2. */
int he_rescale(he_ctx *ctx, const uint64_t *ct, int level, uint64_t *out, void *ws, size_t ws_bytes,
               void *stream);

/* he_mul followed by he_rescale, fused: bit-identical to the two calls, with
 * the ModDown and rescale NTTs merged (out: [2][level-1][N]).  level >= 2. */
int he_mul_rescale(he_ctx *ctx, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk_dev, int level,
                   uint64_t *out, void *ws, size_t ws_bytes, void *stream);

/* HE Mul with ModDown and rescale as one division by M = P * q_{level-1}
 * (Sec. 7's mod down "with an additional division", applied once for both
 * divisions): with Y = P*(d0, d1) + KS over Q_level and P, the basis
 * (p_0, ..., p_{K-1}, q_{level-1}) is dropped by one fast base conversion, so
 * out = floor(Y / M) - floor(sum_j y_j / b_j) in coefficient form: one floor
 * where he_mul_rescale takes two, hence different words (decrypting to the
 * same product within the same error bound) and one fewer conversion row.
 * out: [2][level-1][N], scale1*scale2/q_{level-1}.  level >= 2; errors as
 * he_mul_rescale. */
int he_mul_rescale_pq(he_ctx *ctx, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk_dev, int level,
                      uint64_t *out, void *ws, size_t ws_bytes, void *stream);

/* he_mul_rescale with no workspace argument.  The paper has no counterpart:
 * this is a library convenience for callers that cannot allocate device
 * memory or keep a workspace between calls (for example a host application
 * whose device memory is owned entirely by another allocator, or a binding
 * with no device allocator of its own).  The workspace is a scratch array of
 * HE_STATIC_SCRATCH_BYTES inside the library's own device memory, one per
 * device; nothing is allocated by the call.
 *  - Limit: levels whose he_workspace_bytes exceeds HE_STATIC_SCRATCH_BYTES
 *    (64 MiB: every level of logN <= 15 parameter sets of this size, logN 16
 *    up to level 8) return HE_ENOMEM; use he_mul_rescale for those.
 *  - Every call looks up the current device's scratch address
 *    (cudaGetSymbolAddress); the first lookup on a device may load the
 *    library's device code, so make the first call outside any stream
 *    capture.
 *  - HE_ELEVEL for a level outside 2..L, as he_mul_rescale.
 *  - The current device must be the context's (HE_EINVAL otherwise).
 *  - Nothing in the scratch needs to start at zero.
 *  - All calls on one device share the scratch: calls whose executions
 *    overlap (different streams, or threads without ordering between their
 *    streams) race and give wrong results.  Calls on one stream are safe.
 * Results are bit-identical to he_mul_rescale. */
#define HE_STATIC_SCRATCH_BYTES (64u << 20)
int he_mul_rescale_static(he_ctx *ctx, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk_dev,
                          int level, uint64_t *out, void *stream);

/* he_mul_rescale on HOST buffers: copies ct1, ct2 ([2][level][N], host) to the
 * device, runs the path and copies the result ([2][level-1][N]) back to `out`
 * (host), then waits for the stream.  ws is device memory of at least
 * he_host_workspace_bytes(level) (the path's workspace plus staging for the
 * operands and the result).  Pinned host buffers give asynchronous copies. */
size_t he_host_workspace_bytes(const he_ctx *ctx, int level);
int he_mul_rescale_host(he_ctx *ctx, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk_dev, int level,
                        uint64_t *out, void *ws, size_t ws_bytes, void *stream);

/* A stream of HE Mul + rescale jobs from host buffers: job k's operands
 * ct1[k], ct2[k] (host, [2][levels[k]][N]) are copied to the device, run
 * through the path (he_mul_rescale) and the result copied to out[k] (host,
 * [2][levels[k]-1][N]).  Uploads (one stream per operand) and downloads run
 * on three copy streams the context owns, the path on `stream`, and `slots`
 * (2..4) device staging slots
 * let job k+1's upload and job k-1's download overlap job k's kernels (the
 * host buffers should be pinned for that).  ws: device memory of at least
 * he_host_stream_workspace_bytes(max level, slots) (one path workspace plus
 * the slots).  Returns once every result is in host memory.  HE_ELEVEL for a
 * level outside 2..L, HE_ENOMEM for a short workspace, HE_EINVAL otherwise.
 * Calls on one context must not overlap (the copy streams are shared). */
size_t he_host_stream_workspace_bytes(const he_ctx *ctx, int max_level, int slots);
int he_mul_rescale_host_stream(he_ctx *ctx, int count, const uint64_t *const *ct1, const uint64_t *const *ct2,
                               const int *levels, uint64_t *const *out, const uint64_t *evk_dev, void *ws,
                               size_t ws_bytes, int slots, void *stream);

/* ---- individual steps of the path (per-kernel parity) -------------------- */

/* Forward / inverse NTT (Algo 3 / its inverse) of `count` limbs in place:
 * limb c of `data` (device, [count][N]) is taken mod the ext prime
 * prime_idx[c] (host array; ext order, 0..K+L-1). */
int he_step_ntt(he_ctx *ctx, uint64_t *data, const int *prime_idx, int count, int inverse, void *stream);
/* Tensor product at level l: d = [3][l][N] (d0, d1, d2) from ct1, ct2. */
int he_step_tensor(he_ctx *ctx, const uint64_t *ct1, const uint64_t *ct2, int level, uint64_t *d, void *stream);
/* iNTT of d2 ([level][N], NTT domain) followed by ModUp of every digit:
 * U [beta][K+level][N] in ext order, coefficient form.  Rows of a digit's own
 * limbs are not written (the path reuses d2 for them).  ws must hold
 * he_workspace_bytes(level). */
int he_step_modup(he_ctx *ctx, const uint64_t *d2, int level, uint64_t *U, void *ws, size_t ws_bytes,
                  void *stream);
/* Inner product of NTT-domain U ([beta][K+level][N], own-digit rows taken
 * from d2 [level][N]) with the device evk: KS [2][K+level][N].  ws must hold
 * he_workspace_bytes(level). */
int he_step_inner_product(he_ctx *ctx, const uint64_t *U, const uint64_t *d2, const uint64_t *evk_dev, int level,
                          uint64_t *KS, void *ws, size_t ws_bytes, void *stream);
/* ModDown of one NTT-domain polynomial X ([K+level][N], ext order) to
 * out [level][N]; ws must hold he_workspace_bytes(level). */
int he_step_moddown(he_ctx *ctx, const uint64_t *X, int level, uint64_t *out, void *ws, size_t ws_bytes,
                    void *stream);

/* ---- batched execution ---------------------------------------------------- */

typedef struct {
    const uint64_t *ct1; /* [2][level][N] device */
    const uint64_t *ct2;
    uint64_t *out;       /* [2][level-1][N] device (rescaled) */
    int level;           /* 2 .. L */
} he_job;

/* Batches have no counterpart in the paper, which times one HE Mul at a
 * time; each job is the HE Mul of Fig. 2 followed by Sec. 3.1's rescale.
 * Workspace bytes for a batch of `count` jobs at the given levels (0 for a
 * level outside 2..L). */
size_t he_batch_workspace_bytes(const he_ctx *ctx, int count, const int *levels);
/* Run B independent HE Mul + rescale jobs (uneven levels allowed) as one
 * batch: each stage is one launch over every job's work (grid.z = job), and
 * each NTT launch groups the limbs of all jobs by prime so that one staged
 * twiddle tile serves limbs of several jobs.  The first bytes of ws receive
 * the batch's job table and NTT job lists (one host-to-device copy on the
 * stream); the rest holds the jobs' workspaces.  Results are bit-identical
 * to he_mul_rescale on each job.  count <= 65535.  HE_EINVAL while `stream`
 * is being captured into a CUDA graph (the header copy reads this call's host
 * memory; capture batches with he_batch_graph_create). */
int he_mul_batch(he_ctx *ctx, int count, const he_job *jobs, const uint64_t *evk_dev, void *ws,
                 size_t ws_bytes, void *stream);

/* The batched path (each job Fig. 2 + Sec. 3.1's rescale; no counterpart in
 * the paper) captured once in a CUDA graph for up to max_jobs jobs:
 * every launch is sized for max_jobs jobs at level L (the NTT launches for
 * the most limb groups they can form at the limb-group cap in effect at
 * creation; launches group at that cap or the context's current one,
 * whichever is larger) and reads the job table and NTT job lists (and their
 * counts) that the graph's first node copies from a pinned host buffer, so
 * he_batch_graph_launch with any batch of at most max_jobs jobs (levels
 * 2..L) is one graph launch.  ws (device, at least
 * he_batch_graph_workspace_bytes(max_jobs)) and evk_dev are bound at
 * creation and must outlive the graph.  Creation captures `stream` (no work
 * runs).  Launches alternate between two pinned tables: a launch waits on the
 * host only for the launch before the previous one (which read the table it
 * rewrites), so the host prepares a batch while the previous one runs.
 * Launches of one graph share its workspace: issue them on one stream (or
 * order their streams), as overlapping launches would race on it.  Results
 * are bit-identical to he_mul_rescale per job. */
typedef struct he_batch_graph he_batch_graph;
size_t he_batch_graph_workspace_bytes(const he_ctx *ctx, int max_jobs);
int he_batch_graph_create(he_ctx *ctx, int max_jobs, const uint64_t *evk_dev, void *ws, size_t ws_bytes,
                          void *stream, he_batch_graph **out);
int he_batch_graph_launch(he_batch_graph *g, int count, const he_job *jobs, void *stream);
int he_batch_graph_destroy(he_batch_graph *g);

/* ---- serving (continuous batching) ------------------------------------------ */

/* A served request: HE Mul + rescale of device-resident operands on ring
 * ctx_index of the server (ct1, ct2: [2][level][N]; out: [2][level-1][N]).
 * The server runs batches on streams of its own: operands written on another
 * stream must either be complete before he_server_submit (synchronise that
 * stream) or come with `ready`, a cudaEvent_t (passed as void*) recorded after
 * the writes, which the batch waits for on the device before its first
 * kernel; NULL means the operands are already complete.  The event must stay
 * valid until the request completes. */
typedef struct {
    int ctx_index;
    int level;
    const uint64_t *ct1;
    const uint64_t *ct2;
    uint64_t *out;
    void *ready;
} he_request;

typedef struct {
    uint64_t completed, pending, batches;
    double mean_batch;   /* requests per launched batch */
    double p50_ms, p99_ms, max_ms;  /* submit -> completion observed */
    double throughput;   /* completed requests per second, first submit to last completion */
} he_server_report;

typedef struct he_server he_server;

/* Serving has no counterpart in the paper; every request is the HE Mul of
 * Fig. 2 followed by Sec. 3.1's rescale.  Create a server over nctx rings
 * (contexts) with their device-resident evaluation keys.  It allocates one device arena of hbm_budget bytes for
 * request workspaces and `streams` CUDA streams, and starts a scheduler
 * thread.  The scheduler admits queued requests in arrival order as arena
 * space and streams free up, groups admitted requests of one ring into a
 * batch of at most max_batch (one launch per stage, as he_mul_batch) and runs
 * it on a free stream, so batches formed while others run overlap on the
 * device.  Completion is detected by polling CUDA events on the host.
 * Results are bit-identical to he_mul_rescale per request.  The operand and
 * output buffers of a request must stay valid until it completes. */
int he_server_create(he_server **out, he_ctx *const *ctxs, const uint64_t *const *evk_devs, int nctx,
                     size_t hbm_budget, int max_batch, int streams);
/* Queue a request (non-blocking).  HE_ENOMEM if its workspace exceeds the
 * whole budget (it could never be admitted), HE_ELEVEL / HE_EINVAL for bad
 * arguments. */
int he_server_submit(he_server *s, const he_request *r, uint64_t *ticket);
/* done = 1 once the request completed; returns its error code if it failed.
 * The status of finished tickets is kept for the 2^20 most recent tickets;
 * an older or unknown ticket gives HE_EINVAL. */
int he_server_poll(he_server *s, uint64_t ticket, int *done);
/* Wait up to timeout_ms (0: do not wait) for a request; HE_ETIMEOUT if it has
 * not completed by then, its error code if it failed. */
int he_server_wait(he_server *s, uint64_t ticket, int timeout_ms);
/* Counters since creation; latency percentiles over the last 65536
 * completions. */
int he_server_stats(he_server *s, he_server_report *stats);
/* Stops the scheduler after the batches in flight finish; queued requests
 * that were never launched are dropped. */
int he_server_destroy(he_server *s);

/* ---- seeded evaluation keys (no paper counterpart: halve the key's bytes) -- */

/* Evaluation key whose a halves are a function of a seed: a_j[e][n] =
 * floor((w1 2^64 + w2) t_e / 2^128), w1 and w2 the SplitMix64 words 2(eN+n)
 * and 2(eN+n)+1 of stream 144+j of `seed` (t_e the e-th modulus, ext order);
 * b_j = a_j s + e_j + [t_e in digit j] P s^2 as for he_keygen.  Writes only
 * the b halves, evk_b [dnum][K+L][N] (host).  A seeded key is a different key
 * from he_keygen's (other a halves), equally valid. */
int he_keygen_seeded(he_ctx *ctx, uint64_t seed, const int64_t *sk, uint64_t *evk_b);
/* Declare that the device buffer evk_b_dev holds the b halves of the seeded
 * key of `seed` ([dnum][K+L][N]): every call of this context that receives
 * this pointer as its evaluation key regenerates the a halves inside the
 * inner product instead of reading them (half the key's HBM traffic and
 * footprint).  At most 64 registered keys; registering a pointer again
 * replaces its seed.  he_evk_unregister forgets a pointer (HE_OK if it was
 * not registered).  Batch graphs keep the choice made when they were
 * captured. */
int he_evk_register_seeded(he_ctx *ctx, const uint64_t *evk_b_dev, uint64_t seed);
int he_evk_unregister(he_ctx *ctx, const uint64_t *evk_dev);

/* ---- HE Add and plaintext operations --------------------------------------- */

/* HE Add (Sec. 3.2): out.b = c1.b + c2.b, out.a = c1.a + c2.a mod q_i, element
 * by element with one conditional subtraction.  he_sub: the difference (no
 * paper counterpart; same shape).  ct1, ct2, out: [2][level][N] device, same
 * level and scale; out may alias an input.  HE_ELEVEL for level outside 1..L. */
int he_add(he_ctx *ctx, const uint64_t *ct1, const uint64_t *ct2, int level, uint64_t *out, void *stream);
int he_sub(he_ctx *ctx, const uint64_t *ct1, const uint64_t *ct2, int level, uint64_t *out, void *stream);
/* A plaintext at `level` in the NTT domain (host): the integer polynomial
 * `coeffs` (int64[N], e.g. from he_encode) reduced mod q_0..q_{level-1} and
 * transformed by Algo 3; pt: [level][N]. */
int he_plain_ntt(he_ctx *ctx, const int64_t *coeffs, int level, uint64_t *pt);
/* Plaintext product (both halves times pt, element-wise in the NTT domain;
 * the message is multiplied, scales multiply: rescale afterwards) and
 * plaintext sum (pt added to the b half).  ct, out: [2][level][N], pt:
 * [level][N], device; out may alias ct. */
int he_mul_plain(he_ctx *ctx, const uint64_t *ct, const uint64_t *pt, int level, uint64_t *out, void *stream);
int he_add_plain(he_ctx *ctx, const uint64_t *ct, const uint64_t *pt, int level, uint64_t *out, void *stream);

/* ---- rotation ---------------------------------------------------------------
 * HE rotation is not in the paper; it is the next operation built on the
 * paper's key switching (Fig. 2, region 2), reusing every kernel of it.
 * kappa_g : a(X) -> a(X^g) (g odd, 1 <= g < 2N) maps a ciphertext of m under
 * s to one of kappa_g(m) under kappa_g(s); key switching back to s uses a
 * rotation key, the evaluation key with kappa_g(s) in place of s^2. */

/* g = 5^steps mod 2N: kappa_g moves slot k+steps to slot k (left rotation by
 * `steps`, which may be negative).  2N - 1 conjugates every slot.  0 if ctx
 * is NULL. */
uint64_t he_galois_elt(const he_ctx *ctx, int steps);
/* g = 2N - 1: kappa_g = X -> X^(-1) takes every slot to its complex conjugate
 * (the canonical embedding's roots zeta^(5^k) map to their inverses, i.e.
 * their conjugates).  Used with he_keygen_rot / he_rotate like a rotation.
 * 0 if ctx is NULL. */
uint64_t he_conj_elt(const he_ctx *ctx);
/* Rotation key for kappa_g: rk [dnum][2][K+L][N] host, same layout as evk;
 * b_j = a_j s + e_j + [t in digit j] P kappa_g(s), a_j and e_j drawn from
 * `seed` (streams distinct from the evaluation key's).  HE_EINVAL for an even
 * or out-of-range g. */
int he_keygen_rot(he_ctx *ctx, uint64_t seed, const int64_t *sk, uint64_t galois, uint64_t *rk);
/* HE rotation at `level` (device): out = (kappa(b) + ModDown(KS_b),
 * ModDown(KS_a)) with KS = sum_j ModUp_j(-kappa(a)) rk_j; out decrypts under
 * s to kappa_g(m) at the same level and scale.  ct, out: [2][level][N] device,
 * out may not alias ct; ws as for he_mul (he_workspace_bytes(level)).
 * HE_EINVAL for an even or out-of-range g, HE_ELEVEL for level outside 1..L,
 * HE_ENOMEM if ws_bytes is too small. */
int he_rotate(he_ctx *ctx, const uint64_t *ct, const uint64_t *rk_dev, int level, uint64_t galois, uint64_t *out,
              void *ws, size_t ws_bytes, void *stream);

/* ---- the paper's own non-RNS HE Mul (Sec. 3-4, Fig. 2) ---------------------
 * HEAAN as the paper measures it: ciphertext coefficients are BigInts modulo
 * q = 2^logq (fresh: q = Q = 2^logQ), the evaluation key's modulo Q^2 and
 * encrypting Q s^2; rescale divides by p = 2^logp with rounding.  BigInt
 * polynomials are word-major: word w of coefficient n at a[w * N + n],
 * little-endian, ceil(k / 64) words for modulus 2^k; ciphertexts [2][Wq][N]
 * (b half first), keys [2][W_{2 logQ}][N].  Each polynomial product is the
 * paper's CRT -> NTT -> element-wise product -> iNTT -> iCRT over the context's
 * ciphertext primes: create the context with q_bits = 57 and L >= the plan's
 * np2 (64 at logQ = 1200, N = 2^16); region 1 uses np1 of them (43 there).
 * Decryption relation as above: b - a s = m + e (mod q).  Supported: logQ <=
 * 1216, 1 <= logp < logQ. */
typedef struct he_nr_plan he_nr_plan;
/* Tables (CRT constants, iCRT multiword constants) and NTT job lists for
 * (logQ, logp) on the context's device; HE_EINVAL if the context has too few
 * primes for P > 4 N 2^(3 logQ) or unsupported sizes. */
int he_nr_plan_create(he_ctx *ctx, int logQ, int logp, he_nr_plan **out);
int he_nr_plan_destroy(he_nr_plan *plan);
int he_nr_plan_info(const he_nr_plan *plan, int *np1, int *np2);
size_t he_nr_workspace_bytes(const he_nr_plan *plan);
/* The evaluation key in the NTT-RNS form region 2 uses: CRT and NTT of its
 * two halves over np2 primes, once per key.  evk: [2][W_{2 logQ}][N] device;
 * prep: he_nr_evk_bytes(plan) bytes of device memory. */
size_t he_nr_evk_bytes(const he_nr_plan *plan);
int he_nr_evk_prepare(he_nr_plan *plan, const uint64_t *evk, uint64_t *prep, void *stream);
/* out = HE Mul of ct1, ct2 at logq (Fig. 2): region 1 d0 = b1 b2, d1 = a1 b2 +
 * a2 b1, d2 = a1 a2 mod q; region 2 KS = d2 * evk mod qQ, divided by Q with
 * rounding; out = (d0 + KS_b, d1 + KS_a) mod q.  HE_ELEVEL for logq outside
 * (logp, logQ]; HE_ENOMEM for a short workspace. */
int he_nr_mul(he_nr_plan *plan, const uint64_t *ct1, const uint64_t *ct2, const uint64_t *evk_prep, int logq,
              uint64_t *out, void *ws, size_t ws_bytes, void *stream);
/* Rescale (Sec. 3.1): out = round(ct / 2^logp) mod 2^(logq - logp), [2][W][N]. */
int he_nr_rescale(he_nr_plan *plan, const uint64_t *ct, int logq, uint64_t *out, void *stream);

/* ---- launch shapes and autotuning (no paper counterpart) ------------------ */

/* Launch shape of the path: NTT limbs that share a CTA (they share the
 * staged twiddles; 1..4), ModUp targets per CTA (4, 8 or 16), whether the
 * path's kernels use programmatic dependent launch (1: a kernel's CTAs may be
 * scheduled while its predecessor drains; each waits for it in hardware
 * before touching its data; 2: as 1, and a kernel allows its successor to be
 * launched as soon as its own last wave runs, so the successor's CTAs fill
 * the SMs its tail leaves idle; 0: off), and which of the four NTT sites of the key
 * switch (bit 0 the iNTT of d2, 1 the NTT of the ModUp outputs, 2 the iNTT of
 * the special limbs, 3 the NTT of the ModDown limbs) use the radix-8 plan
 * (rounds of at most three stages, 256 threads per tile) instead of the
 * radix-16 one (128 threads per tile).  Speed only: every shape gives
 * bit-identical results.  Default {4, 8, 1, 0, 8, 7, 0, 0, 0}.  A batch graph keeps the
 * shape it was captured with, except the limb-group cap. */
typedef struct {
    int group_cap;
    int modup_chunk;
    int pdl;     /* 0..2 */
    int ntt_r8;  /* 0..15 */
    int ip_jobs; /* batches of 2 or more jobs: 4 or 8 jobs of similar level share each CTA of the inner
                    product, which reads the evaluation key's words once for all of them (Fig. 2 region 2's
                    key stream, read once per group instead of once per job); 1 = one job per CTA.  Used
                    while the context has at most four digits (dnum <= 4), else 1. */
    int fuse;    /* bit 0: the tensor product (Fig. 2 region 1) is formed inside the first inverse-NTT pass
                    of d2, which loads the ciphertexts instead of d2 and also stores d0, d1, d2 (one launch
                    and one read of d2 fewer); else its own kernel.  bit 1 (single HE Mul with rescale):
                    the key-switch sums of Fig. 2 region 2 are split: those of the special primes and of
                    q_{level-1} (the next iNTT's inputs) first, those of the other q primes (read only by
                    the final additions) in the same launch as the ModDown conversion, so the key stream
                    overlaps the conversion's arithmetic.  bit 2 (with bit 1, unseeded keys): the sums of
                    the special primes and of q_{level-1} are formed by the first pass of their own
                    inverse NTT, which computes its tile from U, d2 and the key instead of loading it (one
                    launch and one write and read of those limbs fewer).  0..7 */
    int ntt_split; /* the stages each pass of every NTT covers (Algo 3 split into a strided pass over the
                    first stages and a contiguous pass over the last ones): 0 the default (2^16: 8 + 8;
                    2^17: 9 + 8), 1 one stage more in the contiguous pass (7 + 9; 8 + 9), 2 one more in the
                    strided pass (9 + 7; 10 + 7); ring sizes other than 2^16 and 2^17 keep the default.
                    0..2 */
    int ntt_small; /* bit s (the sites of ntt_r8): that site's NTT passes work on tiles of 1024 elements
                    instead of 2048 (twice the CTAs, each with half the work: launches over few limbs
                    then end sooner); 2^16 and 2^17 only (a 10-stage strided pass keeps 2048).  0..15 */
    int ntt_onepass; /* bit s (the sites of ntt_r8), N = 2^16 only: that site's transform runs in one pass
                    over memory (Algo 3 whole), each limb on a cluster of 8 CTAs that hold one eighth of it
                    each in shared memory and exchange the first three stages through the cluster's
                    distributed shared memory; else the two passes of ntt_split.  The site's ntt_r8 bit
                    picks the local rounds: radix-8 and radix-4 on 1024 threads, else radix-16 on 512.
                    Site 2 keeps two
                    passes when fuse bits 1 and 2 put the key-switch sums into its first pass.
                    0..15 */
    double ms;   /* he_autotune: measured milliseconds per call; else 0 */
} he_shape;

/* HE_EINVAL for a NULL context or an unsupported value. */
int he_set_shape(he_ctx *ctx, const he_shape *shape);
int he_get_shape(const he_ctx *ctx, he_shape *shape);
/* Time shapes on the caller's own work and keep the fastest in ctx, by
 * coordinate descent from the context's current shape: each knob in turn
 * (group_cap; modup_chunk; pdl and fuse together; ntt_r8 and ntt_split
 * together; ip_jobs for a batch; ntt_small; ntt_onepass) takes every value with the others held at
 * the best shape so far, sweep after sweep until one changes nothing (at
 * most four); then every (pdl, fuse, ntt_split) with the radix masks {best,
 * 0, 15}, and descent sweeps again from the best (no shape is timed twice);
 * count == 1 times he_mul_rescale on jobs[0] (ws of he_workspace_bytes),
 * count > 1 times he_mul_batch on the jobs (ws of he_batch_workspace_bytes),
 * `reps` calls per shape after one warm-up call, CUDA events on `stream`.
 * The four fastest are then timed again, interleaved, in three rounds of
 * 2 x `reps` calls, and the best median is kept.  The jobs' outputs are
 * overwritten.  best: the shape kept, with that median; tried (optional,
 * max_tried entries): every shape of the search with its time, *n_tried set. */
int he_autotune(he_ctx *ctx, const he_job *jobs, int count, const uint64_t *evk_dev, void *ws, size_t ws_bytes,
                int reps, void *stream, he_shape *best, he_shape *tried, int max_tried, int *n_tried);

/* ---- profiling ------------------------------------------------------------ */

/* Enable (1) or disable (0) per-kernel CUDA-event marks on this context's
 * device calls.  While enabled, every kernel of the path is followed by an
 * event on the stream it was launched on; he_profile_read waits for the last
 * mark and returns, per kernel name, the summed time between each kernel's
 * mark and the previous mark (names: 48-byte slots), then clears the marks.
 * Use a single stream while profiling. */
int he_profile(he_ctx *ctx, int enable);
int he_profile_read(he_ctx *ctx, int max, char *names, double *total_ms, int *calls, int *count);

/* Measurement helper: rate (butterflies per second) of the NTT's own lazy
 * Cooley-Tukey butterfly (Algo 4 with the modified Shoup product of Sec. 5.2;
 * the same device function the NTT passes call) on register-resident data,
 * `blocks` x 256 threads x 8 chains x `iters`.  The ALU ceiling the NTT
 * kernels are compared against.  Allocates a small output buffer with
 * cudaMallocAsync on `stream`; HE_EINVAL for a non-positive count. */
int he_probe_butterfly_rate(int blocks, int iters, double *bfly_per_s, void *stream);
/* Measurement helper: rate (multiply-accumulates per second) of the base
 * conversion's inner loop (Sec. 7's mod up / mod down as fast base conversion
 * with Sec. 5.3's delayed-modulo accumulation): per output, `width` terms
 * (1, 2, 4, 8, 12 or 16: the kernels' padded digit or special-prime count)
 * of the split-28 Karatsuba multiply-accumulate with the constant read from
 * shared memory, then one reduction straight from the accumulators, on two
 * coefficients per thread held in registers; `blocks` x 256 threads x 16
 * outputs x `iters`.  The ALU ceiling the ModUp and ModDown conversions are
 * compared against.  HE_EINVAL for another width or a non-positive count. */
int he_probe_conversion_rate(int width, int blocks, int iters, double *mac_per_s, void *stream);
/* Measurement helper: rate (outputs per second) of the work a byte-split
 * tensor-core base conversion would still leave on the CUDA cores per output
 * (the conversion's matrix product, Sec. 7's base conversion, cut into 8-bit
 * pieces exact in bf16 and summed in fp32): the MMA's 13 byte-diagonal planes,
 * each an exact integer below 2^23, turned into integers, shifted and added
 * into 128 bits, then one lazy Barrett reduction; register-resident, MMA not
 * counted; `blocks` x 256 threads x 16 outputs x `iters`.  Compare with
 * he_probe_conversion_rate / width, the outputs per second of the CUDA-core
 * conversion itself.  HE_EINVAL for a non-positive count or iters above
 * 2^18. */
int he_probe_recombine_rate(int blocks, int iters, double *out_per_s, void *stream);

const char *he_strerror(int code);
/* Name of the CUDA error behind the calling thread's last HE_ECUDA. */
const char *he_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HE_GB300_H */
