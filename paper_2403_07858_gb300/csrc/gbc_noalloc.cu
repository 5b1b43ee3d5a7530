// gbc_count_p2_noalloc: the (2,q)-biclique count for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another framework's
// memory pool, plug-ins that may only touch buffers handed to them, or a
// process whose allocator is reserved for something else.  They hand over the
// graph's CSR arrays in device memory and read the count back; every scratch
// byte the count needs lives in one file-scope device array of fixed size,
// so the call allocates nothing (no cudaMalloc, cudaFree or allocating library
// routine).
//
// It is a variant of the global-table candidate kernel: one CTA per root at a
// time counts the root's higher-ranked 2-hop neighbours in an open-addressing
// hash table, here a fixed slab of the static array, and adds C(count, q) for
// each neighbour sharing at least q vertices with the root.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "gbc.h"
#include "gbc_internal.cuh"

namespace gbc {
namespace {

constexpr int kNaCtas = 256;                 // CTAs of one launch, one table slab each
constexpr int kNaSlots = 2 * GBC_NOALLOC_MAX_2HOP;  // table slots per slab (load factor <= 1/2)
constexpr size_t kNaHeader = 256;            // acc (2 x u64) and status (u32), padded
constexpr size_t kNaBytes = kNaHeader + (size_t)kNaCtas * kNaSlots * 2 * sizeof(int32_t);
constexpr uint32_t kNaTooLarge = 1u << 8;    // a root has more than GBC_NOALLOC_MAX_2HOP 2-hop neighbours
constexpr int kNaThreads = 256;

// The only scratch of this entry point: every call shares it and it keeps the
// last call's contents.  In host code this name is a host-side stand-in, not a
// device address; the kernel gets the address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

__device__ __forceinline__ bool above(const int32_t *offU, int32_t w, int32_t u) {
    const int32_t dw = offU[w + 1] - offU[w], du = offU[u + 1] - offU[u];
    return dw > du || (dw == du && w > u);
}

// C(n, q) in 128 bits by the exact multiplicative recurrence; ovf if larger.
__device__ __forceinline__ u128 binom_exact(int32_t n, int q, bool &ovf) {
    if (q > n) return 0;
    uint64_t lo = 1, hi = 0;
    for (int j = 1; j <= q; ++j) {
        if (mul_div_small(lo, hi, (uint32_t)(n - j + 1), (uint32_t)j)) { ovf = true; return 0; }
    }
    return ((u128)hi << 64) | lo;
}

__global__ void __launch_bounds__(kNaThreads)
k_p2_noalloc(int32_t nU, const int32_t *offU, const int32_t *adjU, const int32_t *offV, const int32_t *adjV,
             int q, unsigned char *scratch) {
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(scratch);
    uint32_t *status = reinterpret_cast<uint32_t *>(scratch + 16);
    int32_t *keys = reinterpret_cast<int32_t *>(scratch + kNaHeader) + (size_t)blockIdx.x * 2 * kNaSlots;
    int32_t *vals = keys + kNaSlots;
    volatile int32_t *vkeys = keys, *vvals = vals;
    __shared__ int s_distinct;
    __shared__ int s_stop;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t mask = kNaSlots - 1;
    const volatile int *vdistinct = &s_distinct;
    u128 sum = 0;
    bool ovf = false;
    for (int32_t u = blockIdx.x; u < nU; u += gridDim.x) {
        if (offU[u + 1] - offU[u] < q) continue;  // uniform: fewer than q neighbours
        // once any root has overflowed the fixed table the call fails: skip the rest
        if (threadIdx.x == 0) s_stop = (*(volatile uint32_t *)status & kNaTooLarge) != 0u;
        // the slab keeps the previous root's entries: clear it first
        for (int s = threadIdx.x; s < kNaSlots; s += blockDim.x) { keys[s] = -1; vals[s] = 0; }
        if (threadIdx.x == 0) s_distinct = 0;
        __syncthreads();
        if (s_stop) break;  // block-uniform
        // wedges u - v - w with w ranked above u: a warp per v, lanes over N(v).
        // A thread stops as soon as the root has more distinct 2-hop neighbours
        // than the table holds: at most GBC_NOALLOC_MAX_2HOP + kNaThreads keys
        // are ever inserted, so every probe sequence finds a free slot within
        // the table's 2 * GBC_NOALLOC_MAX_2HOP slots.
        for (int32_t e = offU[u] + warp; e < offU[u + 1] && *vdistinct <= GBC_NOALLOC_MAX_2HOP;
             e += kNaThreads / 32) {
            const int32_t v = adjU[e];
            for (int32_t f = offV[v] + lane; f < offV[v + 1]; f += 32) {
                if (*vdistinct > GBC_NOALLOC_MAX_2HOP) break;
                const int32_t w = adjV[f];
                if (!above(offU, w, u)) continue;
                uint32_t h = ((uint32_t)w * 2654435761u) & mask;
                for (uint32_t probes = 0; probes <= mask; ++probes) {
                    int32_t k = vkeys[h];
                    if (k == -1) {
                        k = atomicCAS(&keys[h], -1, w);
                        if (k == -1) {
                            if (atomicAdd(&s_distinct, 1) >= GBC_NOALLOC_MAX_2HOP) atomicOr(status, kNaTooLarge);
                            k = w;
                        }
                    }
                    if (k == w) { atomicAdd(&vals[h], 1); break; }
                    h = (h + 1) & mask;
                }
            }
        }
        __syncthreads();
        if (*vdistinct <= GBC_NOALLOC_MAX_2HOP) {
            for (int s = threadIdx.x; s < kNaSlots; s += blockDim.x) {
                const int32_t k = vkeys[s], cnt = vvals[s];
                if (k >= 0 && cnt >= q) add_u128(sum, binom_exact(cnt, q, ovf), ovf);
            }
        }
        __syncthreads();
    }
    sum = warp_sum_u128(sum, ovf);
    if (lane == 0) {
        if (ovf) atomicOr(status, kStOverflow);
        atomic_add_u128(acc, sum, status);
    }
}

std::mutex g_mu;
void *g_addr[64] = {nullptr};  // device address of the scratch array, per device

gbc_status na_fail(gbc_status s, const char *fmt, ...) {
    char msg[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    set_last_error(msg);
    return s;
}

}  // namespace
}  // namespace gbc

using namespace gbc;

extern "C" gbc_status gbc_count_p2_noalloc(int32_t nU, int32_t nV, const int32_t *offU_d, const int32_t *adjU_d,
                                           const int32_t *offV_d, const int32_t *adjV_d, int q, void *stream,
                                           gbc_u128 *out) {
    if (!offU_d || !offV_d || !out || nU < 0 || nV < 0)
        return na_fail(GBC_ERR_ARG, "gbc_count_p2_noalloc: null pointer or negative size");
    if (q < 1 || q > GBC_MAX_PQ) return na_fail(GBC_ERR_ARG, "gbc_count_p2_noalloc: q=%d outside [1, %d]", q, GBC_MAX_PQ);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64)
        return na_fail(GBC_ERR_CUDA, "gbc_count_p2_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    unsigned char *scratch = nullptr;
    {
        // set-up, once per device, with that device current
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr)
                return na_fail(GBC_ERR_CUDA, "gbc_count_p2_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_addr[dev] = ptr;
        }
        scratch = static_cast<unsigned char *>(g_addr[dev]);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    struct { unsigned long long acc[2]; uint32_t status; } h{};
    if ((e = cudaMemsetAsync(scratch, 0, 32, st)) != cudaSuccess)  // acc and status start at zero
        return na_fail(GBC_ERR_CUDA, "gbc_count_p2_noalloc: %s", cudaGetErrorString(e));
    if (nU > 0 && nV > 0 && adjU_d && adjV_d) {
        const int grid = (int)std::min<int64_t>(kNaCtas, nU);
        k_p2_noalloc<<<grid, kNaThreads, 0, st>>>(nU, offU_d, adjU_d, offV_d, adjV_d, q, scratch);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return na_fail(GBC_ERR_CUDA, "gbc_count_p2_noalloc: launch: %s", cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(&h, scratch, 20, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return na_fail(GBC_ERR_CUDA, "gbc_count_p2_noalloc: %s", cudaGetErrorString(e));
    if (h.status & kNaTooLarge)
        return na_fail(GBC_ERR_OOM, "gbc_count_p2_noalloc: a vertex of U has more than %d higher-ranked 2-hop "
                                    "neighbours, beyond the fixed scratch of this entry point",
                       GBC_NOALLOC_MAX_2HOP);
    if (h.status & kStOverflow) return na_fail(GBC_ERR_OVERFLOW, "gbc_count_p2_noalloc: count exceeds 2^128-1");
    out->lo = h.acc[0];
    out->hi = h.acc[1];
    return GBC_OK;
}
