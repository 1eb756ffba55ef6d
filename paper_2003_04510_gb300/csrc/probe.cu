// probe.cu -- throughput probes for the ALU rooflines of the path's
// compute-bound kernels.
//
// The NTT kernels and the base conversions are bound by integer multiply
// work, not by HBM.  Each probe runs the kernels' own device functions on
// register-resident data with no global-memory traffic inside the timed loop,
// so its rate is the practical ceiling of that instruction sequence on this
// GPU at the clocks of the run:
//
//  * butterflies: ct_bfly (modarith.cuh), the forward butterfly every NTT
//    pass issues (the paper's modified Shoup product of Sec. 5.2 plus the
//    lazy additions of Algo 4), eight independent chains per thread.  The
//    values are not kept reduced (they wrap), which changes no instruction.
//  * base conversion: the inner loop of k_modup / k_moddown_conv (Sec. 7's
//    mod up / mod down as fast base conversion, with the delayed-modulo
//    accumulation of Sec. 5.3): per output, A terms of mac28k on two
//    coefficients with the constant read from shared memory, then the lazy
//    reduction straight from the accumulators (acc3k_reduce_lazy) per
//    coefficient.  A thread keeps its A split
//    inputs in registers, as the kernels do, and walks a table of constant
//    rows; the outputs are folded into a checksum instead of stored.
#include "he_internal.h"
#include "modarith.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_probe_bfly(u64 *out, u64 q, u64 w, u64 wp, int iters)
{
    const u64 q4 = 4 * q, nq = 0ull - q;
    const ulonglong2 tw = make_ulonglong2(w, wp);
    u64 x[kChains], y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        x[c] = (threadIdx.x * 7919ull + c * 104729ull + blockIdx.x) % q;
        y[c] = (threadIdx.x * 15485863ull + c * 32452843ull + blockIdx.x) % q;
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) ct_bfly(x[c], y[c], tw, nq, q4);
    }
    u64 acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc ^= x[c] ^ y[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// Constant rows staged in shared memory (a conversion CTA's chunk of targets).
constexpr int kRows = 16;

template <int A>
__global__ void __launch_bounds__(256) k_probe_conv(u64 *out, const u64 *rows, u64 q, u64 mu, unsigned sh, int iters)
{
    __shared__ u64 sB[kRows][A];
    for (int t = threadIdx.x; t < kRows * A; t += blockDim.x) sB[t / A][t % A] = rows[t];
    uint32_t x0[A], x1[A], z0[A], z1[A];
#pragma unroll
    for (int i = 0; i < A; i++) {
        const u64 vx = (threadIdx.x * 7919ull + i * 104729ull + blockIdx.x) % q;
        const u64 vy = (threadIdx.x * 15485863ull + i * 32452843ull + blockIdx.x) % q;
        split28(vx, x0[i], x1[i]);
        split28(vy, z0[i], z1[i]);
    }
    __syncthreads();
    u64 acc = 0;
    for (int it = 0; it < iters; it++) {
#pragma unroll 2
        for (int u = 0; u < kRows; u++) {
            Acc3 ax = {0, 0, 0}, ay = {0, 0, 0};
#pragma unroll
            for (int i = 0; i < A; i++) {
                const u64 c = sB[u][i];
                mac28k(ax, x0[i], x1[i], x0[i] + x1[i], c);
                mac28k(ay, z0[i], z1[i], z0[i] + z1[i], c);
            }
            acc ^= acc3k_reduce_lazy(ax, q, mu, sh) + acc3k_reduce_lazy(ay, q, mu, sh);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// The recombination a byte-split tensor-core base conversion would need per
// output.  Such a conversion (residues and constants cut into 8-bit pieces,
// exact in bf16, products summed in fp32 by the MMA) leaves, per output, 13
// fp32 planes S_d = sum over byte pairs (a, b) with a + b = d, each an exact
// integer below 2^23 for up to 16 terms; the output is
// (sum_d S_d 2^(8 d)) mod q.  Here each plane is turned into an integer by
// the cheapest exact route (adding 2^23 and masking the significand), the
// shifted planes are added into a 128-bit value and reduced lazily into
// [0, 2q) (no final subtraction): the least a tensor-core conversion must
// still execute on the CUDA cores per output, MMA not counted.  Every output
// shifts every plane by a loop-carried count (folded into the magic 2^23), so
// nothing is hoisted out of the loop.
constexpr int kPlanes = 13;

__global__ void __launch_bounds__(256) k_probe_recombine(u64 *out, u64 q, u64 mu, unsigned sh, int iters)
{
    float S[kPlanes];
#pragma unroll
    for (int d = 0; d < kPlanes; d++)
        S[d] = (float)((threadIdx.x * 2654435761u + d * 40503u + blockIdx.x * 977u) & 0x3FFFFFu);  // < 2^22
    u64 acc = 0;
    float t = 8388608.0f;  // 2^23 + the output count (below 2^22)
    for (int it = 0; it < iters; it++) {
#pragma unroll 2
        for (int o = 0; o < kRows; o++) {
            U128 v = {0, 0};
#pragma unroll
            for (int d = 0; d < kPlanes; d++) {
                const u64 p = (u64)(__float_as_uint(S[d] + t) & 0x7FFFFFu);  // exact: S_d + count < 2^23
                const int shl = 8 * d;
                const u64 lo = shl < 64 ? p << shl : 0ull;
                const u64 hi = shl == 0 ? 0ull : shl < 64 ? p >> (64 - shl) : p << (shl - 64);
                v.lo += lo;
                v.hi += hi + (v.lo < lo ? 1ull : 0ull);
            }
            const uint32_t l0 = (uint32_t)v.lo, l1 = (uint32_t)(v.lo >> 32), h0 = (uint32_t)v.hi,
                           h1 = (uint32_t)(v.hi >> 32);
            const bool up = sh >= 32;
            const uint32_t w0 = up ? l1 : l0, w1 = up ? h0 : l1, w2 = up ? h1 : h0;
            const u64 u = ((u64)__funnelshift_r(w1, w2, sh) << 32) | __funnelshift_r(w0, w1, sh);
            acc ^= v.lo - __umul64hi(u, mu) * q;
            t += 1.0f;
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// q_0 of the N = 2^16 chain (54 bits) and its Barrett constants as the
// context computes them (s = bitlen(q) - 2, mu = floor(2^(64+s) / q)).
constexpr u64 kProbeQ = 18014398506729473ull;

template <class Launch>
int time_launch(cudaStream_t st, Launch launch, float *ms)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return HE_ECUDA;
    }
    launch(true);  // warm-up
    cudaEventRecord(a, st);
    launch(false);
    cudaEventRecord(b, st);
    const cudaError_t e = cudaEventSynchronize(b);
    *ms = 0;
    cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return (e != cudaSuccess || cudaGetLastError() != cudaSuccess) ? HE_ECUDA : HE_OK;
}

}  // namespace

extern "C" int he_probe_butterfly_rate(int blocks, int iters, double *bfly_per_s, void *stream)
{
    if (blocks < 1 || iters < 1 || !bfly_per_s) return HE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    u64 *out = nullptr;
    if (cudaMallocAsync((void **)&out, sizeof(u64) * blocks * 256, st) != cudaSuccess) return HE_ECUDA;
    const u64 q = kProbeQ;
    const u64 w = 1234567890123ull % q;
    const u64 wp = (u64)(((unsigned __int128)w << 64) / q);
    float ms = 0;
    const int rc = time_launch(st, [&](bool warm) {
        k_probe_bfly<<<blocks, 256, 0, st>>>(out, q, w, wp, warm ? iters / 10 + 1 : iters);
    }, &ms);
    cudaFreeAsync(out, st);
    if (rc != HE_OK) return rc;
    *bfly_per_s = (double)blocks * 256.0 * kChains * (double)iters / (ms * 1e-3);
    return HE_OK;
}

extern "C" int he_probe_conversion_rate(int width, int blocks, int iters, double *mac_per_s, void *stream)
{
    if (blocks < 1 || iters < 1 || !mac_per_s) return HE_EINVAL;
    if (width != 1 && width != 2 && width != 4 && width != 8 && width != 12 && width != 16) return HE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const u64 q = kProbeQ;
    const unsigned sh = 64 - __builtin_clzll(q) - 2;
    const u64 mu = (u64)(((unsigned __int128)1 << (64 + sh)) / q);
    // constant rows: residues below 2^55 pre-split at bit 28 (b0 | b1 << 32),
    // as the contexts store them
    u64 rows[kRows * 16];
    u64 z = 0x243F6A8885A308D3ull;
    for (int t = 0; t < kRows * 16; t++) {
        z = z * 6364136223846793005ull + 1442695040888963407ull;
        const u64 b = (z >> 9) % q;
        rows[t] = (b & 0xFFFFFFFull) | ((b >> 28) << 32);
    }
    u64 *buf = nullptr;
    const size_t out_words = (size_t)blocks * 256;
    if (cudaMallocAsync((void **)&buf, sizeof(u64) * (out_words + kRows * 16), st) != cudaSuccess) return HE_ECUDA;
    u64 *d_rows = buf + out_words;
    if (cudaMemcpyAsync(d_rows, rows, sizeof(rows), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaFreeAsync(buf, st);
        return HE_ECUDA;
    }
    float ms = 0;
    const int rc = time_launch(st, [&](bool warm) {
        const int n = warm ? iters / 10 + 1 : iters;
        switch (width) {
        case 1: k_probe_conv<1><<<blocks, 256, 0, st>>>(buf, d_rows, q, mu, sh, n); break;
        case 2: k_probe_conv<2><<<blocks, 256, 0, st>>>(buf, d_rows, q, mu, sh, n); break;
        case 4: k_probe_conv<4><<<blocks, 256, 0, st>>>(buf, d_rows, q, mu, sh, n); break;
        case 8: k_probe_conv<8><<<blocks, 256, 0, st>>>(buf, d_rows, q, mu, sh, n); break;
        case 12: k_probe_conv<12><<<blocks, 256, 0, st>>>(buf, d_rows, q, mu, sh, n); break;
        default: k_probe_conv<16><<<blocks, 256, 0, st>>>(buf, d_rows, q, mu, sh, n); break;
        }
    }, &ms);
    cudaFreeAsync(buf, st);
    if (rc != HE_OK) return rc;
    // per thread and trip: kRows outputs on two coefficients, `width` terms each
    *mac_per_s = (double)blocks * 256.0 * kRows * 2.0 * width * (double)iters / (ms * 1e-3);
    return HE_OK;
}

extern "C" int he_probe_recombine_rate(int blocks, int iters, double *out_per_s, void *stream)
{
    // the count folded into the planes stays below 2^22 (exact in fp32)
    if (blocks < 1 || iters < 1 || iters > (1 << 22) / kRows || !out_per_s) return HE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const u64 q = kProbeQ;
    const unsigned sh = 64 - __builtin_clzll(q) - 2;
    const u64 mu = (u64)(((unsigned __int128)1 << (64 + sh)) / q);
    u64 *out = nullptr;
    if (cudaMallocAsync((void **)&out, sizeof(u64) * blocks * 256, st) != cudaSuccess) return HE_ECUDA;
    float ms = 0;
    const int rc = time_launch(st, [&](bool warm) {
        k_probe_recombine<<<blocks, 256, 0, st>>>(out, q, mu, sh, warm ? iters / 10 + 1 : iters);
    }, &ms);
    cudaFreeAsync(out, st);
    if (rc != HE_OK) return rc;
    *out_per_s = (double)blocks * 256.0 * kRows * (double)iters / (ms * 1e-3);
    return HE_OK;
}
