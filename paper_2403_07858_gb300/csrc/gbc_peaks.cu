// gbc_measure_int_peaks: two microbenchmarks that put the enumeration kernel's
// work on a scale.  The enumeration spends its time on bitmap words (one AND,
// one POPC and one ADD per word) whose operands come from shared memory, L1 or
// L2, so its ceilings are the integer pipe and the cache that serves the rows:
//
//   * a register-only loop of s += popc(s & y): the rate at which the SMs
//     retire the AND + POPC + ADD triple with no memory operand at all;
//   * an AND + popcount stream over two 16 MiB word arrays that stay in L2
//     (loads bypass L1), the rate at which L2 can feed such a loop.
//
// Both launch 8 CTAs of 256 threads per SM, time each launch with CUDA events,
// drop the first (warm-up) launch and report the best of the next three.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "gbc.h"
#include "gbc_internal.cuh"

namespace gbc {
namespace {

constexpr int kPkThreads = 256;
constexpr int kPkChains = 8;          // independent dependency chains per thread
constexpr int kPkIters = 1 << 14;     // loop trips per thread (x kPkChains words)
constexpr size_t kPkWords = 4u << 20; // 16 MiB per array, two arrays: L2-resident

__global__ void __launch_bounds__(kPkThreads) k_peak_and_popc(uint32_t seed, int iters, uint32_t *sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t s[kPkChains], y[kPkChains];
#pragma unroll
    for (int j = 0; j < kPkChains; ++j) {
        s[j] = (t + 1u) * 2654435761u + (uint32_t)j * 40503u + seed;
        y[j] = (s[j] ^ 0x9e3779b9u) * 2246822519u;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kPkChains; ++j) s[j] += __popc(s[j] & y[j]);  // AND, POPC, ADD
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < kPkChains; ++j) r ^= s[j];
    if (r == 0x5bd1e995u) sink[0] = r;  // keeps the chains live; practically never taken
}

__global__ void __launch_bounds__(kPkThreads) k_peak_l2_stream(const uint4 *a, const uint4 *b, size_t n4, int passes,
                                                             uint32_t *sink) {
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int p = 0; p < passes; ++p) {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
            const uint4 x = __ldcg(a + i), z = __ldcg(b + i);
            acc += __popc(x.x & z.x) + __popc(x.y & z.y) + __popc(x.z & z.z) + __popc(x.w & z.w);
        }
    }
    if (acc == 0xffffffffu) sink[1] = acc;
}

__global__ void k_peak_fill(uint32_t *w, size_t n, uint32_t seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        w[i] = ((uint32_t)i + seed) * 2654435761u;
}

gbc_status pk_fail(const char *what, cudaError_t e) {
    char msg[256];
    snprintf(msg, sizeof msg, "gbc_measure_int_peaks: %s: %s", what, cudaGetErrorString(e));
    set_last_error(msg);
    return GBC_ERR_CUDA;
}

}  // namespace
}  // namespace gbc

using namespace gbc;

extern "C" gbc_status gbc_measure_int_peaks(int device, double *and_popc_words_per_s, double *l2_bytes_per_s) {
    if (!and_popc_words_per_s || !l2_bytes_per_s) {
        set_last_error("gbc_measure_int_peaks: null output pointer");
        return GBC_ERR_ARG;
    }
    cudaError_t e;
    if ((e = cudaSetDevice(device)) != cudaSuccess) return pk_fail("cudaSetDevice", e);
    int n_sms = 0;
    if ((e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return pk_fail("cudaDeviceGetAttribute", e);
    uint32_t *buf = nullptr;
    if ((e = cudaMalloc(&buf, 2 * kPkWords * sizeof(uint32_t) + 64)) != cudaSuccess) return pk_fail("cudaMalloc", e);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gbc_status rc = GBC_OK;
    double best_alu = 0.0, best_l2 = 0.0;
    do {
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
            rc = pk_fail("stream/event", e);
            break;
        }
        uint32_t *sink = buf + 2 * kPkWords;
        k_peak_fill<<<4 * n_sms, 256, 0, st>>>(buf, 2 * kPkWords, 12345u);
        const int grid = 8 * n_sms;  // 8 CTAs of 256 threads per SM: 64 warps
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            k_peak_and_popc<<<grid, kPkThreads, 0, st>>>((uint32_t)rep, kPkIters, sink);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = pk_fail("and/popc loop", e); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double words = (double)grid * kPkThreads * kPkIters * kPkChains;
            if (rep > 0 && ms > 0.f) best_alu = std::max(best_alu, words / (ms * 1e-3));
        }
        if (rc != GBC_OK) break;
        const size_t n4 = kPkWords / 4;
        const uint4 *a = reinterpret_cast<const uint4 *>(buf);
        const uint4 *b = reinterpret_cast<const uint4 *>(buf + kPkWords);
        const int passes = 16;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            k_peak_l2_stream<<<grid, kPkThreads, 0, st>>>(a, b, n4, passes, sink);
            cudaEventRecord(e1, st);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = pk_fail("L2 stream", e); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double bytes = 2.0 * kPkWords * sizeof(uint32_t) * passes;
            if (rep > 0 && ms > 0.f) best_l2 = std::max(best_l2, bytes / (ms * 1e-3));
        }
        if (rc != GBC_OK) break;
        if ((e = cudaGetLastError()) != cudaSuccess) rc = pk_fail("launch", e);
    } while (false);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(buf);
    if (rc != GBC_OK) return rc;
    *and_popc_words_per_s = best_alu;
    *l2_bytes_per_s = best_l2;
    return GBC_OK;
}
