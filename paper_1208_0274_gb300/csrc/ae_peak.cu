// Integer-ALU throughput of the current GPU (include/ae_peak.h): the roofline
// denominator of the search's row and sweep kernels, measured rather than
// derived from unit counts.
//
// Each thread keeps `chains` values x[0..chains) and, per step, updates
// x[i] = op(x[i], x[i+1 mod chains]) (with a runtime constant b for the
// add-max kinds).  Steps of different chains are independent, so with 2+
// chains per thread and 8 resident blocks per SM every scheduler has a ready
// instruction each cycle; the value of every step feeds the next, so none can
// be dropped, and the runtime constant keeps the compiler from folding steps.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ae_peak.h"

namespace {

template <int KIND, int CH>
__device__ __forceinline__ void step(int32_t (&x)[8], int32_t b) {
#pragma unroll
    for (int i = 0; i < CH; ++i) {
        const int32_t y = x[(i + 1) % CH];
        if (KIND == AE_PEAK_IADD) {
            asm volatile("add.s32 %0, %0, %1;" : "+r"(x[i]) : "r"(y));
        } else if (KIND == AE_PEAK_IMAX) {
            asm volatile("max.s32 %0, %0, %1;" : "+r"(x[i]) : "r"(y));
        } else if (KIND == AE_PEAK_ADDMAX32) {
            x[i] = __viaddmax_s32(x[i], b, y);
        } else {
            x[i] = (int32_t)__viaddmax_s16x2((uint32_t)x[i], (uint32_t)b, (uint32_t)y);
        }
    }
}

template <int KIND, int CH>
__global__ void __launch_bounds__(256) k_int_peak(int32_t *out, int iters, int32_t seed, int32_t b) {
    const int32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    int32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = seed ^ (tid * (2 * i + 1));
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) step<KIND, CH>(x, b);
    }
    int32_t acc = 0;
#pragma unroll
    for (int i = 0; i < CH; ++i) acc ^= x[i];
    out[tid] = acc;
}

template <int KIND>
void launch(int chains, unsigned blocks, int32_t *out, int iters, int32_t seed, int32_t b, cudaStream_t st) {
    switch (chains) {
        case 1: k_int_peak<KIND, 1><<<blocks, 256, 0, st>>>(out, iters, seed, b); break;
        case 2: k_int_peak<KIND, 2><<<blocks, 256, 0, st>>>(out, iters, seed, b); break;
        case 3: k_int_peak<KIND, 3><<<blocks, 256, 0, st>>>(out, iters, seed, b); break;
        case 4: k_int_peak<KIND, 4><<<blocks, 256, 0, st>>>(out, iters, seed, b); break;
        case 5: k_int_peak<KIND, 5><<<blocks, 256, 0, st>>>(out, iters, seed, b); break;
        case 6: k_int_peak<KIND, 6><<<blocks, 256, 0, st>>>(out, iters, seed, b); break;
        case 7: k_int_peak<KIND, 7><<<blocks, 256, 0, st>>>(out, iters, seed, b); break;
        default: k_int_peak<KIND, 8><<<blocks, 256, 0, st>>>(out, iters, seed, b); break;
    }
}

}  // namespace

extern "C" ae_status ae_int_peak(int32_t kind, int32_t chains, int32_t iters, int32_t blocks_per_sm, void *stream,
                                 double *ops_per_s, double *insts_per_s, double *ms) {
    if (kind < AE_PEAK_IADD || kind > AE_PEAK_ADDMAX16X2 || chains < 1 || chains > 8 || iters < 1 ||
        blocks_per_sm < 1 || blocks_per_sm > 64)
        return AE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return AE_ECUDA;
    }
    const unsigned blocks = (unsigned)(sms * blocks_per_sm);
    int32_t *out = nullptr;
    if (cudaMalloc(&out, sizeof(int32_t) * (size_t)blocks * 256) != cudaSuccess) {
        cudaGetLastError();
        return AE_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ae_status res = AE_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) res = AE_ECUDA;
    float t = 0.f;
    if (res == AE_OK) {
        const int32_t seed = 0x2545F491, b = -3;
        auto run = [&]() {
            switch (kind) {
                case AE_PEAK_IADD: launch<AE_PEAK_IADD>(chains, blocks, out, iters, seed, b, st); break;
                case AE_PEAK_IMAX: launch<AE_PEAK_IMAX>(chains, blocks, out, iters, seed, b, st); break;
                case AE_PEAK_ADDMAX32: launch<AE_PEAK_ADDMAX32>(chains, blocks, out, iters, seed, b, st); break;
                default: launch<AE_PEAK_ADDMAX16X2>(chains, blocks, out, iters, seed, b, st); break;
            }
        };
        run();   // warm-up
        if (cudaEventRecord(e0, st) != cudaSuccess) res = AE_ECUDA;
        run();
        if (res == AE_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
            res = AE_ECUDA;
    }
    if (res == AE_OK && cudaGetLastError() != cudaSuccess) res = AE_ECUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(st);
    cudaFree(out);
    cudaGetLastError();
    if (res != AE_OK) return res;
    const double insts = (double)blocks * 256.0 * (double)iters * 16.0 * (double)chains;
    const double per = kind == AE_PEAK_ADDMAX32 ? 2.0 : (kind == AE_PEAK_ADDMAX16X2 ? 4.0 : 1.0);
    const double sec = (double)t / 1000.0;
    if (ms) *ms = t;
    if (insts_per_s) *insts_per_s = sec > 0 ? insts / sec : 0.0;
    if (ops_per_s) *ops_per_s = sec > 0 ? insts * per / sec : 0.0;
    return AE_OK;
}
