// probe.cu -- throughput probes: random gathers (the denominator of the
// marcher's gather roofline) and random non-returning vector reductions (the
// backward's scatter).
//
// Every thread issues `iters` loads of `bytes` (16 or 32) bytes at
// pseudo-random, aligned offsets of a device buffer of `buffer_bytes`, the
// access pattern of the marcher's texel gathers when neighbouring lanes read
// unrelated texels.  With a buffer that fits L1 (tens of KB, every SM reads
// the same one) the probe measures the L1 scattered-sector rate; with one of
// tens of MB the L2 rate; with one of GBs the HBM rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cow.h"
#include "cow_common.cuh"

namespace cow {

namespace {

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int BYTES>
__global__ void __launch_bounds__(256) k_gather_probe(const uint4 *__restrict__ buf, uint32_t n_elems_mask, int iters,
                                                      uint32_t *sink) {
    uint32_t h = mix32((uint32_t)(blockIdx.x * blockDim.x + threadIdx.x) * 0x9e3779b9u + 1u);
    uint32_t acc = 0;
#pragma unroll 4
    for (int it = 0; it < iters; it++) {
        h = mix32(h + (uint32_t)it);
        const uint32_t e = h & n_elems_mask;
        if (BYTES == 32) {
            uint32_t r[8];
            ld256(buf + 2 * (size_t)e, r);
            acc ^= r[0] ^ r[1] ^ r[2] ^ r[3] ^ r[4] ^ r[5] ^ r[6] ^ r[7];
        } else {
            const uint4 q = __ldg(buf + e);
            acc ^= q.x ^ q.y ^ q.z ^ q.w;
        }
    }
    if (acc == 0x12345678u) sink[0] = acc;  // keeps the loads alive
}

// Every thread issues `iters` non-returning 4-float reductions
// (red.global.add.v4.f32, the backward's scatter instruction) at
// pseudo-random 16-byte-aligned offsets of a buffer of n_vec4 float4s.
__global__ void __launch_bounds__(256) k_reduce_probe(float *__restrict__ buf, uint32_t n_vec4_mask, int iters) {
    uint32_t h = mix32((uint32_t)(blockIdx.x * blockDim.x + threadIdx.x) * 0x9e3779b9u + 7u);
#pragma unroll 4
    for (int it = 0; it < iters; it++) {
        h = mix32(h + (uint32_t)it);
        float *dst = buf + 4 * (size_t)(h & n_vec4_mask);
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(dst), "f"(1.0f), "f"(2.0f), "f"(3.0f),
                     "f"(4.0f)
                     : "memory");
    }
}

}  // namespace

}  // namespace cow

extern "C" cow_status cow_gather_peak(int32_t bytes_per_load, int64_t buffer_bytes, int32_t iters, double *out_gbs,
                                      void *stream) {
    if (!out_gbs || (bytes_per_load != 16 && bytes_per_load != 32) || iters < 1 || buffer_bytes < 1024 ||
        (buffer_bytes & (buffer_bytes - 1)) || buffer_bytes > ((int64_t)1 << 36))
        return COW_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    void *buf = nullptr;
    uint32_t *sink = nullptr;
    if (cudaMalloc(&buf, (size_t)buffer_bytes) != cudaSuccess) return COW_ERR_OOM;
    if (cudaMalloc((void **)&sink, 4) != cudaSuccess) {
        cudaFree(buf);
        return COW_ERR_OOM;
    }
    cudaMemsetAsync(buf, 1, (size_t)buffer_bytes, st);
    const int64_t n_elems = buffer_bytes / bytes_per_load;
    const uint32_t mask = (uint32_t)(n_elems - 1 > 0xffffffffLL ? 0xffffffffu : (uint32_t)(n_elems - 1));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = sms * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto launch = [&]() {
        if (bytes_per_load == 32)
            cow::k_gather_probe<32><<<blocks, 256, 0, st>>>((const uint4 *)buf, mask, iters, sink);
        else
            cow::k_gather_probe<16><<<blocks, 256, 0, st>>>((const uint4 *)buf, mask, iters, sink);
    };
    launch();  // warm-up
    cudaEventRecord(a, st);
    const int reps = 5;
    for (int r = 0; r < reps; r++) launch();
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) return COW_ERR_CUDA;
    const double bytes = (double)reps * blocks * 256.0 * iters * bytes_per_load;
    *out_gbs = bytes / (ms * 1e-3) / 1e9;
    return COW_OK;
}

extern "C" cow_status cow_reduce_peak(int64_t buffer_bytes, int32_t iters, double *out_gred_per_s, void *stream) {
    if (!out_gred_per_s || iters < 1 || buffer_bytes < 1024 || (buffer_bytes & (buffer_bytes - 1)) ||
        buffer_bytes > ((int64_t)1 << 36))
        return COW_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float *buf = nullptr;
    if (cudaMalloc((void **)&buf, (size_t)buffer_bytes) != cudaSuccess) return COW_ERR_OOM;
    cudaMemsetAsync(buf, 0, (size_t)buffer_bytes, st);
    const int64_t n_vec4 = buffer_bytes / 16;
    const uint32_t mask = (uint32_t)(n_vec4 - 1 > 0xffffffffLL ? 0xffffffffu : (uint32_t)(n_vec4 - 1));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const int blocks = sms * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cow::k_reduce_probe<<<blocks, 256, 0, st>>>(buf, mask, iters);  // warm-up
    cudaEventRecord(a, st);
    const int reps = 5;
    for (int r = 0; r < reps; r++) cow::k_reduce_probe<<<blocks, 256, 0, st>>>(buf, mask, iters);
    cudaEventRecord(b, st);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    if (e != cudaSuccess || ms <= 0.f) return COW_ERR_CUDA;
    *out_gred_per_s = (double)reps * blocks * 256.0 * iters / (ms * 1e-3) / 1e9;
    return COW_OK;
}
