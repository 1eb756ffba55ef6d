// probe.cu -- throughput probe for the ALU roofline of the NTT kernels.
//
// The NTT kernels are bound by 64-bit integer multiply work, not by HBM: each
// butterfly is one Shoup product (the paper's modified Shoup of Sec. 5.2)
// plus adds.  This kernel issues exactly the forward butterfly of ntt.cu
// (ct_bfly: no correction step) on register-resident data with no memory
// traffic and eight independent chains per thread, so its rate is the
// practical ceiling for butterflies per second on this GPU.  The values are
// not kept reduced (they wrap), which changes no instruction.
#include "he_internal.h"
#include "modarith.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_probe_bfly(u64 *out, u64 q, u64 w, u64 wp, int iters)
{
    const u64 q2 = 2 * q;
    u64 x[kChains], y[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        x[c] = (threadIdx.x * 7919ull + c * 104729ull + blockIdx.x) % q;
        y[c] = (threadIdx.x * 15485863ull + c * 32452843ull + blockIdx.x) % q;
    }
    const u64 q4 = 2 * q2;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) {
            const u64 t = shoup_approx(y[c], w, wp, q);
            y[c] = x[c] + q4 - t;
            x[c] = x[c] + t;
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc ^= x[c] ^ y[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

extern "C" int he_probe_butterfly_rate(int blocks, int iters, double *bfly_per_s, void *stream)
{
    if (blocks < 1 || iters < 1 || !bfly_per_s) return HE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    u64 *out = nullptr;
    if (cudaMallocAsync((void **)&out, sizeof(u64) * blocks * 256, st) != cudaSuccess) return HE_ECUDA;
    // q_0 of the N = 2^16 chain (54 bits) and a twiddle with its Shoup companion
    const u64 q = 18014398506729473ull;
    const u64 w = 1234567890123ull % q;
    const u64 wp = (u64)(((unsigned __int128)w << 64) / q);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_probe_bfly<<<blocks, 256, 0, st>>>(out, q, w, wp, iters / 10 + 1);  // warm-up
    cudaEventRecord(a, st);
    k_probe_bfly<<<blocks, 256, 0, st>>>(out, q, w, wp, iters);
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFreeAsync(out, st);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return HE_ECUDA;
    *bfly_per_s = (double)blocks * 256.0 * kChains * (double)iters / (ms * 1e-3);
    return HE_OK;
}
