// Load-time kernels: CSR validation, degrees, neighbour lists re-sorted by the
// anchor side's priority (Def. 2), mirror positions, and the binomial table.
#include <algorithm>

#include "gbc_internal.cuh"

namespace gbc {

// ---------------------------------------------------------------------------
// Validation.  Offsets are checked before any adjacency read, so a malformed
// CSR is reported without out-of-range accesses.
__global__ void k_validate_offsets(const int32_t *off, int32_t n, int64_t nE, uint32_t *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = off[i];
        bool bad = (o < 0) || (o > nE);
        if (i == 0 && o != 0) bad = true;
        if (i == n && o != nE) bad = true;
        if (i < n && off[i + 1] < o) bad = true;
        if (bad) atomicOr(status, kStBadOffsets);
    }
}

// Warp per row: every neighbour in [0, n_other), rows strictly increasing.
__global__ void k_validate_rows(const int32_t *off, const int32_t *adj, int32_t n, int32_t n_other,
                                uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; r < n; r += nwarps) {
        int32_t b = off[r], e = off[r + 1];
        for (int32_t i = b + lane; i < e; i += 32) {
            int32_t x = adj[i];
            if (x < 0 || x >= n_other) atomicOr(status, kStBadRange);
            if (i + 1 < e && adj[i + 1] <= x) atomicOr(status, kStUnsorted);
        }
    }
}

// Every U-edge (u, v) must appear in v's row of the V-CSR.  With both CSRs
// sorted, duplicate-free and holding the same number of edges, this makes the
// V-CSR exactly the transpose of the U-CSR.
__global__ void k_validate_transpose(const int32_t *offU, const int32_t *adjU, int32_t nU,
                                     const int32_t *offV, const int32_t *adjV, uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; u < nU; u += nwarps) {
        for (int32_t i = offU[u] + lane; i < offU[u + 1]; i += 32) {
            int32_t v = adjU[i];
            int32_t lo = offV[v], hi = offV[v + 1] - 1;
            bool found = false;
            while (lo <= hi) {
                int32_t m = lo + ((hi - lo) >> 1);
                int32_t x = adjV[m];
                if (x == u) { found = true; break; }
                if (x < u) lo = m + 1; else hi = m - 1;
            }
            if (!found) atomicOr(status, kStNotTranspose);
        }
    }
}

cudaError_t launch_validate_offsets(const int32_t *off, int32_t n, int64_t nE, uint32_t *status, cudaStream_t st) {
    int grid = (int)std::min<int64_t>(((int64_t)n + 256) / 256 + 1, 4096);
    k_validate_offsets<<<grid, 256, 0, st>>>(off, n, nE, status);
    return cudaGetLastError();
}

cudaError_t launch_validate_rows(const int32_t *off, const int32_t *adj, int32_t n, int32_t n_other,
                                 uint32_t *status, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>(((int64_t)n * 32 + 255) / 256, 8192);
    k_validate_rows<<<grid, 256, 0, st>>>(off, adj, n, n_other, status);
    return cudaGetLastError();
}

cudaError_t launch_validate_transpose(const int32_t *offU, const int32_t *adjU, int32_t nU,
                                      const int32_t *offV, const int32_t *adjV, uint32_t *status,
                                      cudaStream_t st) {
    if (nU == 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>(((int64_t)nU * 32 + 255) / 256, 8192);
    k_validate_transpose<<<grid, 256, 0, st>>>(offU, adjU, nU, offV, adjV, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Degrees, maximum degree and the wedge count sum_x C(deg x, 2) of one side.
__global__ void k_degrees(const int32_t *off, int32_t n, int32_t *deg, int32_t *maxdeg,
                          unsigned long long *wedges) {
    int32_t mx = 0;
    unsigned long long w = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = off[i + 1] - off[i];
        deg[i] = d;
        mx = max(mx, d);
        w += (unsigned long long)d * (unsigned long long)(d > 0 ? d - 1 : 0) / 2ull;
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(kFull, mx, o));
        w += __shfl_xor_sync(kFull, w, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(maxdeg, mx);
        atomicAdd(wedges, w);
    }
}

cudaError_t launch_degrees(const int32_t *off, int32_t n, int32_t *deg, int32_t *maxdeg,
                           unsigned long long *wedges, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>(((int64_t)n + 255) / 256, 4096);
    k_degrees<<<grid, 256, 0, st>>>(off, n, deg, maxdeg, wedges);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Re-sort every row of a CSR by the rank key (deg_target[x], x) of its entries.
// After this, the entries of a row ranked above a given vertex form a suffix.
// One CTA per row; bitonic sort of the padded row in shared memory, or in a
// per-CTA global buffer for rows longer than kSortSmem.
constexpr int kSortSmem = 4096;
constexpr int kSortThreads = 256;

template <typename Ptr>
__device__ void bitonic_sort_u64(Ptr keys, int P) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t a = keys[i], b = keys[ixj];
                    bool asc = (i & k) == 0;
                    if ((a > b) == asc) { keys[i] = b; keys[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kSortThreads)
k_rank_sort_rows(const int32_t *off, const int32_t *adj, int32_t n_rows, const int32_t *deg,
                 int32_t *out, bool long_rows, uint64_t *gtmp, int64_t gtmp_per_cta) {
    __shared__ uint64_t skeys[kSortSmem];
    for (int64_t r = blockIdx.x; r < n_rows; r += gridDim.x) {
        const int32_t b = off[r], e = off[r + 1], len = e - b;
        const bool is_long = len > kSortSmem;
        if (is_long != long_rows) continue;
        if (len <= 1) {
            if (len == 1 && threadIdx.x == 0) out[b] = adj[b];
            continue;
        }
        int P = 1;
        while (P < len) P <<= 1;
        uint64_t *keys = is_long ? gtmp + (int64_t)blockIdx.x * gtmp_per_cta : skeys;
        for (int i = threadIdx.x; i < P; i += blockDim.x)
            keys[i] = (i < len) ? rank_key(deg, adj[b + i]) : ~0ull;
        __syncthreads();
        bitonic_sort_u64(keys, P);
        for (int i = threadIdx.x; i < len; i += blockDim.x) out[b + i] = (int32_t)(uint32_t)keys[i];
        __syncthreads();
    }
}

cudaError_t launch_rank_sort_rows(const int32_t *off, const int32_t *adj, int32_t n_rows,
                                  const int32_t *deg_target, int32_t *out, int32_t max_row,
                                  int64_t *gtmp, cudaStream_t st) {
    if (n_rows == 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>(n_rows, 152 * 16);
    k_rank_sort_rows<<<grid, kSortThreads, 0, st>>>(off, adj, n_rows, deg_target, out, false, nullptr, 0);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || max_row <= kSortSmem) return err;
    int64_t P = 1;
    while (P < max_row) P <<= 1;
    k_rank_sort_rows<<<64, kSortThreads, 0, st>>>(off, adj, n_rows, deg_target, out, true,
                                                  reinterpret_cast<uint64_t *>(gtmp), P);
    return cudaGetLastError();
}

// mirror[e] for the A-edge e = (a, o): index of a inside o's rank-sorted row.
__global__ void k_mirror(const int32_t *offA, const int32_t *adjA, int32_t nA, const int32_t *offO,
                         const int32_t *adjO_rank, const int32_t *degA, int32_t *mirror) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * blockDim.x / 32;
    for (int64_t a = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; a < nA; a += nwarps) {
        const uint64_t ka = rank_key(degA, (int32_t)a);
        for (int32_t e = offA[a] + lane; e < offA[a + 1]; e += 32) {
            const int32_t o = adjA[e];
            int32_t lo = offO[o], hi = offO[o + 1] - 1, pos = -1;
            while (lo <= hi) {
                int32_t m = lo + ((hi - lo) >> 1);
                uint64_t km = rank_key(degA, adjO_rank[m]);
                if (km == ka) { pos = m; break; }
                if (km < ka) lo = m + 1; else hi = m - 1;
            }
            mirror[e] = pos - offO[o];
        }
    }
}

cudaError_t launch_mirror(const int32_t *offA, const int32_t *adjA, int32_t nA, const int32_t *offO,
                          const int32_t *adjO_rank, const int32_t *degA, int32_t *mirror, cudaStream_t st) {
    if (nA == 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>(((int64_t)nA * 32 + 255) / 256, 8192);
    k_mirror<<<grid, 256, 0, st>>>(offA, adjA, nA, offO, adjO_rank, degA, mirror);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Binomial table C(n, j), 0 <= j <= 16, by the multiplicative recurrence
// C(n, j) = C(n, j-1) * (n - j + 1) / j, which is exact in integers: the
// 160-bit product is divided by j with 64-bit limbs.  The first j whose value
// leaves 128 bits marks this n, and every larger j, as overflowing.
__global__ void k_binomial(ulonglong2 *c, int32_t *n_ovf, int32_t nmax) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= nmax; n += (int64_t)gridDim.x * blockDim.x) {
        uint64_t lo = 1, hi = 0;
        bool ovf = false;
        c[n] = make_ulonglong2(1, 0);  // C(n, 0)
        for (int j = 1; j <= kMaxPQ; ++j) {
            if (!ovf) {
                if ((int64_t)j > n) { lo = 0; hi = 0; }
                else ovf = mul_div_small(lo, hi, (uint32_t)(n - j + 1), (uint32_t)j);
            }
            if (ovf) {
                c[(size_t)j * (nmax + 1) + n] = make_ulonglong2(~0ull, ~0ull);
                atomicMin(&n_ovf[j], (int32_t)n);
            } else {
                c[(size_t)j * (nmax + 1) + n] = make_ulonglong2(lo, hi);
            }
        }
    }
}

__global__ void k_fill_i32(int32_t *p, int32_t n, int32_t v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// ---------------------------------------------------------------------------
// Per-side sums behind the scratch-footprint bound of a count (serving
// admission): with omega(u) the oriented wedges of root u (wedges u - o - w
// with w ranked above u), a root keeps at most omega(u) / kq candidates, each
// with an R row of row_stride(deg u) words and an S row of about c / 32 words.
// out: [0] sum omega, [1] sum omega * row_stride(deg), [2] max omega,
// [3] roots with omega > 0, [4] sum omega^2 (as the bits of a double).
__global__ void k_footprint_sums(const int32_t *offA, int32_t nA, const int32_t *adjA, const int32_t *offO,
                                 const int32_t *mirror, unsigned long long *out) {
    unsigned long long s0 = 0, s1 = 0, mx = 0, npos = 0;
    double sq = 0.0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nA; u += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long om = 0;
        for (int32_t e = offA[u]; e < offA[u + 1]; ++e) {
            const int32_t o = adjA[e];
            om += (unsigned long long)(offO[o + 1] - offO[o] - mirror[e] - 1);
        }
        s0 += om;
        s1 += om * (unsigned long long)row_stride(offA[u + 1] - offA[u]);
        mx = om > mx ? om : mx;
        npos += om > 0;
        sq += (double)om * (double)om;
    }
    for (int o = 16; o >= 1; o >>= 1) {
        s0 += __shfl_xor_sync(kFull, s0, o);
        s1 += __shfl_xor_sync(kFull, s1, o);
        const unsigned long long m2 = __shfl_xor_sync(kFull, mx, o);
        mx = m2 > mx ? m2 : mx;
        npos += __shfl_xor_sync(kFull, npos, o);
        sq += __shfl_xor_sync(kFull, sq, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], s0);
        atomicAdd(&out[1], s1);
        atomicMax(&out[2], mx);
        atomicAdd(&out[3], npos);
        atomicAdd(reinterpret_cast<double *>(&out[4]), sq);
    }
}

cudaError_t launch_footprint_sums(const int32_t *offA, int32_t nA, const int32_t *adjA, const int32_t *offO,
                                  const int32_t *mirror, unsigned long long *out, cudaStream_t st) {
    if (nA == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(((int64_t)nA + 255) / 256, 2048);
    k_footprint_sums<<<grid, 256, 0, st>>>(offA, nA, adjA, offO, mirror, out);
    return cudaGetLastError();
}

cudaError_t launch_binomial(ulonglong2 *c, int32_t *n_ovf, int32_t nmax, cudaStream_t st) {
    k_fill_i32<<<1, 32, 0, st>>>(n_ovf, kMaxPQ + 1, INT32_MAX);
    int grid = (int)std::min<int64_t>(((int64_t)nmax + 256) / 256, 4096);
    k_binomial<<<grid, 256, 0, st>>>(c, n_ovf, nmax);
    return cudaGetLastError();
}

}  // namespace gbc
