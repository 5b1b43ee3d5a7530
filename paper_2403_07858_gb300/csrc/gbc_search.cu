// Per-count kernels: 2-hop candidates and their C_R bitmap rows, pairwise C_L
// rows, the enumeration of the search trees, and the u128 reduction.
//
// Notation (Sec. III-A, Alg. 1): anchor side A, other side O; k = |L| on A,
// kq = |R| on O.  Root u (an A vertex) with d = |N(u)| keeps
//   C_L(u) = { w in A ranked above u : |N(u) & N(w)| >= kq }   (c = |C_L(u)|)
// in rank order, and for each candidate j the row R_j, a d-bit bitmap over the
// positions of N(u) (bit i set when N(u)[i] is a neighbour of candidate j).
// For k >= 4 it also keeps S_j, a c-bit bitmap with bit x (x > j) set when
// candidates j and x share >= kq neighbours inside N(u) (the q-strength 2-hop
// relation of Sec. II, taken inside the root's neighbourhood).
#include <algorithm>

#include "gbc_internal.cuh"

namespace gbc {

thread_local int t_launches = 0;

// For |L| >= 4 each root also keeps T, the transpose of its R block: for each
// position i of N(u) (P = row_stride(d) * 32 rows, the width of an R row in
// bits), the bitmap T_i of the candidates whose R row holds i, placed after the
// root's S block.  T is stored word-interleaved: word w of the P rows sits
// together (P words), so the lanes of a warp that read word w of different rows
// share cache sectors.
__host__ __device__ __forceinline__ int64_t t_rows(int32_t d) { return (int64_t)row_stride(d) * 32; }


// ---------------------------------------------------------------------------
// k == 1: every anchor vertex alone is L; it contributes C(deg, kq).
__global__ void k_single_vertex_sets(CountArgs a) {
    u128 acc = 0;
    bool ovf = false;
    const int64_t n = a.g.nA;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ((n + 31) / 32) * 32;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ic = i < n ? a.g.callerA[i] : -1;  // root ranges are in the caller's ids
        if (i < n && ic >= a.root_begin && ic < a.root_end) {
            bool o = false;
            ulonglong2 v = binom_lookup(a.binom, a.kq, a.g.degA[i], o);
            if (a.per_root) {
                a.per_root[2 * i] = v.x;
                a.per_root[2 * i + 1] = v.y;
            }
            ovf |= o;
            add_u128(acc, v, ovf);
        }
    }
    acc = warp_sum_u128(acc, ovf);
    if ((threadIdx.x & 31) == 0) {
        if (ovf) atomicOr(a.status, kStOverflow);
        atomic_add_u128(a.acc, acc, a.status);
    }
    if (a.stats && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(&a.stats->roots, (unsigned long long)((n < a.root_end ? n : a.root_end) - max(0, a.root_begin)));
}

__global__ void k_set_deadline(unsigned long long *deadline, unsigned long long limit_ns) {
    *deadline = limit_ns ? global_ns() + limit_ns : 0ull;
}

cudaError_t launch_set_deadline(unsigned long long *deadline, unsigned long long limit_ns, cudaStream_t st) {
    k_set_deadline<<<1, 1, 0, st>>>(deadline, limit_ns);
    return cudaGetLastError();
}

cudaError_t launch_single_vertex_sets(const CountArgs &a, cudaStream_t st) {
    int grid = (int)std::min<int64_t>(((int64_t)a.g.nA + 255) / 256 + 1, 2048);
    k_single_vertex_sets<<<grid, 256, 0, st>>>(a);
    ++t_launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Oriented wedge count of each root and its tier.  omega(u) counts wedges
// u - v - w with w ranked above u; a root can hold at most omega/kq candidates,
// so roots with omega < (k-1)*kq cannot reach |L| = k and are dropped
// (Alg. 1 root filter, applied before the candidates are even formed).
__global__ void k_root_omega(CountArgs a) {
    const SideView &g = a.g;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < g.nA; u += (int64_t)gridDim.x * blockDim.x) {
        int64_t om = 0;
        const int32_t d = g.degA[u];
        a.cand_count[u] = 0;
        if (d >= a.kq) {
            for (int32_t e = g.offA[u]; e < g.offA[u + 1]; ++e) {
                const int32_t o = g.adjA[e];
                om += (int64_t)(g.offO[o + 1] - g.offO[o] - g.mirror[e] - 1);
            }
        }
        a.omega[u] = (int32_t)om;
        const int32_t uc = g.callerA[u];  // root ranges are in the caller's ids
        const bool mine = uc >= a.root_begin && uc < a.root_end;
        if (mine && om >= (int64_t)(a.k - 1) * a.kq && om > 0) {
            const int tier = om <= kWarpTierOmega ? 0 : (om <= kCtaTierOmega ? 1 : 2);
            const int slot = atomicAdd(&a.tier_count[tier], 1);
            a.tier_list[(int64_t)tier * g.nA + slot] = (int32_t)u;
            atomicMax(&a.omega_max[tier], (int32_t)om);
        }
    }
}

cudaError_t launch_root_omega(const CountArgs &a, cudaStream_t st) {
    int grid = (int)std::min<int64_t>(((int64_t)a.g.nA + 255) / 256, 4096);
    if (grid == 0) return cudaSuccess;
    k_root_omega<<<grid, 256, 0, st>>>(a);
    ++t_launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Candidate generation for one root by a group of NW warps (NW = 1: a warp;
// otherwise the whole CTA).  The wedges u - N(u)[i] - w (w ranked above u) are
// the suffixes of the rank-sorted rows of N(u)'s members; they are counted in
// an open-addressing hash table keyed by w.
template <int NW>
struct Group {
    __device__ static int tid() { return NW == 1 ? (threadIdx.x & 31) : threadIdx.x; }
    __device__ static int size() { return 32 * NW; }
    __device__ static int warp() { return NW == 1 ? 0 : (threadIdx.x >> 5); }
    __device__ static void sync() {
        if (NW == 1) __syncwarp(); else __syncthreads();
    }
};

__device__ __forceinline__ uint32_t hash_slot(int32_t w, int log2slots) {
    return ((uint32_t)w * 2654435761u) >> (32 - log2slots);
}

// Linear probing; a table is sized to at least twice the number of wedges of
// its root, so a probe sequence never wraps.  The probe count is bounded all
// the same: running past it flags kStScratch instead of spinning.
__device__ __forceinline__ void table_insert(int32_t *keys, int32_t *vals, int log2slots, int32_t w,
                                             uint32_t *status) {
    const uint32_t mask = (1u << log2slots) - 1;
    uint32_t h = hash_slot(w, log2slots);
    for (uint32_t probes = 0; probes <= mask; ++probes) {
        int32_t k = ((volatile int32_t *)keys)[h];
        if (k == -1) {
            k = atomicCAS(&keys[h], -1, w);
            if (k == -1) k = w;
        }
        if (k == w) { atomicAdd(&vals[h], 1); return; }
        h = (h + 1) & mask;
    }
    atomicOr(status, kStScratch);
}

// Slot of w (present by construction); returns -1 and flags kStScratch if not found.
__device__ __forceinline__ int32_t table_find(const int32_t *keys, int log2slots, int32_t w, uint32_t *status) {
    const uint32_t mask = (1u << log2slots) - 1;
    uint32_t h = hash_slot(w, log2slots);
    for (uint32_t probes = 0; probes <= mask; ++probes) {
        if (((volatile const int32_t *)keys)[h] == w) return (int32_t)h;
        h = (h + 1) & mask;
    }
    atomicOr(status, kStScratch);
    return -1;
}

// Visit every oriented wedge (w, i) of root u: i = position in N(u), w in the
// part of N(N(u)[i]) ranked above u.  Each warp of the group takes chunks of 32
// positions; the warp's lanes share the chunk's wedges evenly through a scan.
template <int NW, typename F>
__device__ __forceinline__ void for_each_wedge(const SideView &g, int32_t u, F fn) {
    const int lane = threadIdx.x & 31;
    const int32_t d = g.degA[u];
    const int32_t eA = g.offA[u];
    for (int32_t base = Group<NW>::warp() * 32; base < d; base += 32 * NW) {
        const int32_t i = base + lane;
        int32_t len = 0, s0 = 0;
        if (i < d) {
            const int32_t e = eA + i;
            const int32_t o = g.adjA[e];
            s0 = g.offO[o] + g.mirror[e] + 1;
            len = g.offO[o + 1] - s0;
        }
        const int32_t incl = warp_incl_scan(len);
        const int32_t total = __shfl_sync(kFull, incl, 31);
        for (int32_t f0 = 0; f0 < total; f0 += 32) {
            const int32_t f = f0 + lane;
            int owner = 0;
#pragma unroll
            for (int b = 16; b >= 1; b >>= 1) {
                const int32_t v = __shfl_sync(kFull, incl, owner + b - 1);
                if (v <= f) owner += b;
            }
            owner = min(owner, 31);
            const int32_t o_incl = __shfl_sync(kFull, incl, owner);
            const int32_t o_len = __shfl_sync(kFull, len, owner);
            const int32_t o_s0 = __shfl_sync(kFull, s0, owner);
            if (f < total) fn(g.adjO_rank[o_s0 + (f - (o_incl - o_len))], base + owner);
        }
    }
}

template <typename Ptr>
__device__ void group_bitonic_u64(Ptr keys, int P, int tid, int gsize, bool cta) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += gsize) {
                int ixj = i ^ j;
                if (ixj > i) {
                    uint64_t x = keys[i], y = keys[ixj];
                    bool asc = (i & k) == 0;
                    if ((x > y) == asc) { keys[i] = y; keys[ixj] = x; }
                }
            }
            if (cta) __syncthreads(); else __syncwarp();
        }
    }
}

// One root, pass A (BUILD = false): count candidates; for k == 2 the leaves
// are the candidates themselves and their C(common, kq) are summed here.
// Pass B (BUILD = true): list the candidates in rank order and set their R rows.
template <int NW, bool BUILD>
__device__ void process_root(const CountArgs &a, int32_t u, int32_t *keys, int32_t *vals,
                             uint64_t *sortbuf, int32_t *shared_int, u128 &acc, bool &ovf) {
    typedef Group<NW> G;
    const SideView &g = a.g;
    const int tid = G::tid(), gs = G::size();
    const int32_t om = a.omega[u];
    int log2slots = 5;
    while ((1 << log2slots) < 2 * om) ++log2slots;
    const int slots = 1 << log2slots;
    for (int s = tid; s < slots; s += gs) { keys[s] = -1; vals[s] = 0; }
    G::sync();
    for_each_wedge<NW>(g, u, [&](int32_t w, int32_t) { table_insert(keys, vals, log2slots, w, a.status); });
    G::sync();
    const int32_t d = g.degA[u];
    const int32_t WR = (d + 31) >> 5;
    if (!BUILD) {
        int c = 0;
        u128 leaf = 0;
        bool o = false;
        const volatile int32_t *vk = keys, *vv = vals;
        for (int s = tid; s < slots; s += gs) {
            const int32_t key = vk[s], cnt = vv[s];
            if (key >= 0 && cnt >= a.kq) {
                ++c;
                if (a.k == 2) add_u128(leaf, binom_lookup(a.binom, a.kq, cnt, o), o);
            }
        }
        // group reductions through the warp sums and (for CTAs) shared memory
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(kFull, c, off);
        if (a.k == 2) leaf = warp_sum_u128(leaf, o);
        if (NW > 1) {
            if (tid == 0) shared_int[0] = 0;
            __syncthreads();
            if ((tid & 31) == 0) atomicAdd(&shared_int[0], c);
            __syncthreads();
            c = shared_int[0];
            __syncthreads();
        }
        if (tid == 0) {
            a.cand_count[u] = c;
            if (c >= a.k - 1) {
                atomicMax(a.cand_max, c);
                if (a.stats) {
                    atomicAdd(&a.stats->roots, 1ull);
                    atomicAdd(&a.stats->cands, (unsigned long long)c);
                    if (a.k == 2) {
                        atomicAdd(&a.stats->evals[2], (unsigned long long)c);
                        atomicAdd(&a.stats->passed[2], (unsigned long long)c);
                        atomicAdd(&a.stats->words_r, (unsigned long long)c * WR);
                    }
                }
            }
        }
        if (a.k == 2 && (tid & 31) == 0) {
            // each warp adds its own part (a warp group has one warp)
            if (o) atomicOr(a.status, kStOverflow);
            if (a.per_root) atomic_add_u128(a.per_root + 2 * (int64_t)u, leaf, a.status);
            add_u128(acc, leaf, ovf);
        }
        G::sync();
        return;
    }
    // ---- pass B
    const int32_t c = a.cand_count[u];
    if (tid == 0) { shared_int[0] = 0; shared_int[1] = 0; }
    G::sync();
    {
        const volatile int32_t *vk = keys, *vv = vals;
        for (int s = tid; s < slots; s += gs) {
            const int32_t key = vk[s], cnt = vv[s];
            if (key >= 0 && cnt >= a.kq) {
                int idx = atomicAdd(&shared_int[0], 1);
                sortbuf[idx] = rank_key(g.degA, key);
            }
        }
    }
    G::sync();
    int P = 1;
    while (P < c) P <<= 1;
    for (int i = c + tid; i < P; i += gs) sortbuf[i] = ~0ull;
    G::sync();
    group_bitonic_u64(sortbuf, P, tid, gs, NW > 1);
    const int64_t coff = a.cand_off[u];
    for (int i = tid; i < c; i += gs) {
        const int32_t w = (int32_t)(uint32_t)sortbuf[i];
        a.cand[coff + i] = w;
        a.cand_root[coff + i] = u;
        const int32_t slot = table_find(keys, log2slots, w, a.status);
        if (slot >= 0) vals[slot] = -1 - i;
    }
    G::sync();
    // Position order (the bitmap analogue of Sec. V-B's reordering, per root):
    // the positions of N(u) sorted by how many candidates contain them, most
    // shared first, so the common neighbourhoods deep in the tree gather in the
    // first words of C_R.  Positions no candidate contains get no bit at all.
    int32_t *pc = a.poscnt + g.offA[u];
    int32_t *pm = a.posmap + g.offA[u];
    const volatile int32_t *vvals = vals;
    for_each_wedge<NW>(g, u, [&](int32_t w, int32_t i) {
        const int32_t slot = table_find(keys, log2slots, w, a.status);
        if (slot >= 0 && vvals[slot] < 0) atomicAdd(&pc[i], 1);
    });
    G::sync();
    for (int i = tid; i < d; i += gs) {
        const int32_t cnt = __ldcg(&pc[i]);
        if (cnt > 0) {
            const int t = atomicAdd(&shared_int[1], 1);
            // most shared first; or, on request, the other side's id order (N(u)'s order)
            sortbuf[t] = a.position_order ? (uint64_t)(uint32_t)i
                                          : ((uint64_t)(0xffffffffu - (uint32_t)cnt) << 32) | (uint32_t)i;
        }
    }
    G::sync();
    const int dn = ((volatile int32_t *)shared_int)[1];
    P = 1;
    while (P < dn) P <<= 1;
    for (int i = dn + tid; i < P; i += gs) sortbuf[i] = ~0ull;
    G::sync();
    group_bitonic_u64(sortbuf, P, tid, gs, NW > 1);
    for (int t = tid; t < dn; t += gs) pm[(uint32_t)sortbuf[t]] = t;
    G::sync();
    // R block of the root, word-major in pairs: words 2*pw and 2*pw+1 of row x
    // sit at pair pw * c + x, so the first pair of every row forms one
    // contiguous c * 8 B block (deep C_R spans rarely go past it).
    uint32_t *Rb = a.R + a.r_off[u];
    const int32_t WLc = (c + 31) >> 5;
    uint32_t *Tb = a.k >= 4 && a.S ? a.S + a.s_off[u] + (int64_t)c * WLc : nullptr;  // no S in listing mode
    for_each_wedge<NW>(g, u, [&](int32_t w, int32_t i) {
        const int32_t slot = table_find(keys, log2slots, w, a.status);
        const int32_t v = slot >= 0 ? vvals[slot] : 0;
        if (v < 0) {
            const int32_t np = __ldcg(&pm[i]);
            const int64_t x = -1 - v;
            atomicOr(&Rb[2 * ((int64_t)(np >> 6) * c + x) + ((np >> 5) & 1)], 1u << (np & 31));
            if (Tb) atomicOr(&Tb[(int64_t)(x >> 5) * t_rows(d) + np], 1u << (x & 31));
        }
    });
    G::sync();
}

// Tier 0: one warp per root; each warp owns a 512-slot table in shared memory.
template <bool BUILD>
__global__ void __launch_bounds__(32 * kWarpTierWarps)
k_cand_warp(CountArgs a) {
    // per warp: keys[512] | vals[512] | sort[256] (u64); plus 2 ints per warp
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ int32_t s_int[kWarpTierWarps][2];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *mine = dyn + (size_t)w * kWarpTierBytes;
    int32_t *my_keys = reinterpret_cast<int32_t *>(mine);
    int32_t *my_vals = my_keys + kWarpTierSlots;
    uint64_t *my_sort = reinterpret_cast<uint64_t *>(my_vals + kWarpTierSlots);
    u128 acc = 0;
    bool ovf = false;
    const int n = a.tier_count[0];
    int32_t *queue = a.queues + (BUILD ? 3 : 0);
    while (true) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(queue, 1);
        idx = __shfl_sync(kFull, idx, 0);
        if (idx >= n || __shfl_sync(kFull, (int)past_deadline(a), 0)) break;
        const int32_t u = a.tier_list[idx];
        if (BUILD && (a.cand_count[u] < a.k - 1 || u < a.lib_begin || u >= a.lib_end)) continue;
        process_root<1, BUILD>(a, u, my_keys, my_vals, my_sort, s_int[w], acc, ovf);
    }
    if (!BUILD && a.k == 2 && lane == 0) {
        if (ovf) atomicOr(a.status, kStOverflow);
        atomic_add_u128(a.acc, acc, a.status);
    }
}

// Tiers 1 and 2: one CTA per root, table in dynamic shared memory (tier 1) or
// in the CTA's global slab (tier 2).
template <bool BUILD, bool GLOBAL_TABLE>
__global__ void __launch_bounds__(kCtaThreads)
k_cand_cta(CountArgs a) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ int32_t s_int[2];
    __shared__ int32_t s_idx;
    const int tier = GLOBAL_TABLE ? 2 : 1;
    int32_t *keys, *vals;
    uint64_t *sortbuf;
    if (GLOBAL_TABLE) {
        int32_t *slab = a.slab + (int64_t)blockIdx.x * a.slab_words;
        int slots = 32;
        while (slots < 2 * a.omega_max[2]) slots <<= 1;
        keys = slab;
        vals = slab + slots;
        sortbuf = reinterpret_cast<uint64_t *>(slab + 2 * (int64_t)slots);
    } else {
        keys = reinterpret_cast<int32_t *>(dyn);
        vals = keys + kCtaTierSlots;
        sortbuf = reinterpret_cast<uint64_t *>(vals + kCtaTierSlots);
    }
    u128 acc = 0;
    bool ovf = false;
    const int n = a.tier_count[tier];
    int32_t *queue = a.queues + (BUILD ? 3 : 0) + tier;
    while (true) {
        if (threadIdx.x == 0) s_idx = past_deadline(a) ? n : atomicAdd(queue, 1);
        __syncthreads();
        const int idx = s_idx;
        __syncthreads();
        if (idx >= n) break;
        const int32_t u = a.tier_list[(int64_t)tier * a.g.nA + idx];
        if (BUILD && (a.cand_count[u] < a.k - 1 || u < a.lib_begin || u >= a.lib_end)) continue;
        process_root<kCtaThreads / 32, BUILD>(a, u, keys, vals, sortbuf, s_int, acc, ovf);
    }
    if (!BUILD && a.k == 2 && (threadIdx.x & 31) == 0) {
        if (ovf) atomicOr(a.status, kStOverflow);
        atomic_add_u128(a.acc, acc, a.status);
    }
}

constexpr size_t kCtaTierSmem = 2 * kCtaTierSlots * sizeof(int32_t) + kCtaTierOmega * sizeof(uint64_t);

cudaError_t launch_candidates(const CountArgs &a, bool build, const int32_t *tier_counts_host,
                              int n_sms, cudaStream_t st) {
    constexpr int warp_smem = kWarpTierWarps * kWarpTierBytes;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_cand_cta<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCtaTierSmem);
        cudaFuncSetAttribute(k_cand_cta<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCtaTierSmem);
        cudaFuncSetAttribute(k_cand_warp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, warp_smem);
        cudaFuncSetAttribute(k_cand_warp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, warp_smem);
        attr_set = true;
    }
    if (tier_counts_host[0] > 0) {
        int grid = std::min(n_sms * 4, (tier_counts_host[0] + kWarpTierWarps - 1) / kWarpTierWarps);
        if (build) k_cand_warp<true><<<grid, 32 * kWarpTierWarps, warp_smem, st>>>(a);
        else k_cand_warp<false><<<grid, 32 * kWarpTierWarps, warp_smem, st>>>(a);
        ++t_launches;
    }
    if (tier_counts_host[1] > 0) {
        int grid = std::min(n_sms * 2, tier_counts_host[1]);
        if (build) k_cand_cta<true, false><<<grid, kCtaThreads, kCtaTierSmem, st>>>(a);
        else k_cand_cta<false, false><<<grid, kCtaThreads, kCtaTierSmem, st>>>(a);
        ++t_launches;
    }
    if (tier_counts_host[2] > 0) {
        const int grid = a.slab_ctas;  // one global table slab per CTA
        if (build) k_cand_cta<true, true><<<grid, kCtaThreads, 0, st>>>(a);
        else k_cand_cta<false, true><<<grid, kCtaThreads, 0, st>>>(a);
        ++t_launches;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-root offsets: exclusive scans of c', c'*W_R and c'*W_L, where c' = c for
// roots that keep >= k-1 candidates and 0 otherwise.  Three-phase block scan.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ void root_sizes(const CountArgs &a, int64_t r, int64_t &c, int64_t &wr, int64_t &wl) {
    c = 0; wr = 0; wl = 0;
    if (r >= a.g.nA) return;
    const int32_t cc = a.cand_count[r];
    if (cc < a.k - 1 || cc == 0) return;
    c = cc;
    wr = (int64_t)cc * row_stride(a.g.degA[r]);
    wl = a.k >= 4 ? (cc + t_rows(a.g.degA[r])) * ((cc + 31) >> 5) : 0;
}

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T *tmp, T &total) {
    // tmp: kScanThreads/32 entries
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) tmp[w] = incl;
    __syncthreads();
    if (w == 0) {
        T x = lane < kScanThreads / 32 ? tmp[lane] : 0;
        T xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(kFull, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < kScanThreads / 32) tmp[lane] = xi - x;
        if (lane == kScanThreads / 32 - 1) tmp[kScanThreads / 32] = xi;
    }
    __syncthreads();
    T res = incl - v + tmp[w];
    total = tmp[kScanThreads / 32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(CountArgs a, int64_t *tile_sums) {
    __shared__ int64_t tmp[3][kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int64_t s[3] = {0, 0, 0};
    for (int t = 0; t < kScanItems; ++t) {
        int64_t c, wr, wl;
        root_sizes(a, base + t, c, wr, wl);
        s[0] += c; s[1] += wr; s[2] += wl;
    }
    for (int m = 0; m < 3; ++m) {
        int64_t tot;
        block_excl_scan(s[m], tmp[m], tot);
        if (threadIdx.x == 0) tile_sums[(int64_t)m * gridDim.x + blockIdx.x] = tot;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int64_t *tile_sums, int n_tiles, int64_t *totals) {
    __shared__ int64_t tmp[kScanThreads / 32 + 1];
    for (int m = 0; m < 3; ++m) {
        int64_t carry = 0;
        for (int b0 = 0; b0 < n_tiles; b0 += kScanThreads) {
            const int b = b0 + threadIdx.x;
            int64_t v = b < n_tiles ? tile_sums[(int64_t)m * n_tiles + b] : 0;
            int64_t tot;
            int64_t ex = block_excl_scan(v, tmp, tot);
            if (b < n_tiles) tile_sums[(int64_t)m * n_tiles + b] = carry + ex;
            carry += tot;
        }
        if (threadIdx.x == 0) totals[m] = carry;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(CountArgs a, const int64_t *tile_sums, int64_t *cand_off, int64_t *r_off, int64_t *s_off) {
    __shared__ int64_t tmp[3][kScanThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int64_t v[3][kScanItems];
    int64_t s[3] = {0, 0, 0};
    for (int t = 0; t < kScanItems; ++t) {
        root_sizes(a, base + t, v[0][t], v[1][t], v[2][t]);
        s[0] += v[0][t]; s[1] += v[1][t]; s[2] += v[2][t];
    }
    int64_t *outs[3] = {cand_off, r_off, s_off};
    for (int m = 0; m < 3; ++m) {
        int64_t tot;
        int64_t ex = block_excl_scan(s[m], tmp[m], tot) + tile_sums[(int64_t)m * gridDim.x + blockIdx.x];
        for (int t = 0; t < kScanItems; ++t) {
            const int64_t r = base + t;
            if (r <= a.g.nA) outs[m][r] = ex;
            ex += v[m][t];
        }
    }
}

cudaError_t launch_root_offsets(const CountArgs &a, int64_t *cand_off, int64_t *r_off, int64_t *s_off,
                                int64_t *tmp, int64_t *totals, cudaStream_t st) {
    // covers r in [0, nA] (the entry nA receives the total)
    const int n_tiles = (int)(((int64_t)a.g.nA + 1 + kScanTile - 1) / kScanTile);
    k_scan_reduce<<<n_tiles, kScanThreads, 0, st>>>(a, tmp);
    k_scan_tiles<<<1, kScanThreads, 0, st>>>(tmp, n_tiles, totals);
    k_scan_apply<<<n_tiles, kScanThreads, 0, st>>>(a, tmp, cand_off, r_off, s_off);
    t_launches += 3;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Root blocks (written in pass B and by k_pairs), for a root with d neighbours
// and c candidates, np = row_stride(d) / 2 word pairs per R row, WL = ceil(c/32):
//   R: pair pw of candidate x at ((uint2*)Rb)[pw * c + x]   (word-major)
//   S: word w of candidate y at Sb[w * c + y]               (word-major)
// Lanes holding neighbouring candidates therefore read neighbouring addresses.

__device__ __forceinline__ int popc2(uint2 a, uint2 b) { return __popc(a.x & b.x) + __popc(a.y & b.y); }
__device__ __forceinline__ uint2 and2(uint2 a, uint2 b) { return make_uint2(a.x & b.x, a.y & b.y); }

// Pairs of row x holding all of its set bits (its span).  Warp-wide.
__device__ __forceinline__ int row_span_pairs(const uint2 *Rp, int64_t c, int64_t x, int npairs) {
    const int lane = threadIdx.x & 31;
    int span = 0;
    for (int base = 0; base < npairs; base += 32) {
        const int pw = base + lane;
        bool nz = false;
        if (pw < npairs) {
            const uint2 v = Rp[pw * c + x];
            nz = (v.x | v.y) != 0u;
        }
        const unsigned m = __ballot_sync(kFull, nz);
        if (m) span = base + 32 - __clz(m);
    }
    return span;
}

// ---------------------------------------------------------------------------
// Level-2 rows.  Warp per candidate j of a root: for every later candidate x,
// n = popc(R_j & R_x) over the span of R_j.  k == 3: (u, j, x) is a leaf and
// adds C(n, kq) when n >= kq.  k >= 4: the ballot of (n >= kq) over 32
// consecutive x is word x/32 of S_j; units with |S_j| >= k-2 go to the
// enumeration list.
template <bool STATS>
__global__ void __launch_bounds__(256) k_pairs(CountArgs a) {
    const int lane = threadIdx.x & 31;
    u128 acc = 0;
    bool ovf = false;
    while (true) {
        int64_t gidx = 0;
        if (lane == 0) gidx = atomicAdd(a.queues + 6, 1);
        gidx = __shfl_sync(kFull, gidx, 0);
        if (gidx >= a.n_cand || __shfl_sync(kFull, (int)past_deadline(a), 0)) break;
        gidx += a.cand_base;  // the piece's first candidate (0 when the count runs whole)
        const int32_t r = a.cand_root[gidx];
        const int32_t j = (int32_t)(gidx - a.cand_off[r]);
        const int64_t c = a.cand_count[r];
        const int32_t d = a.g.degA[r];
        const int32_t WRm = (d + 31) >> 5;  // words of the full-width model (statistics)
        const int npairs = row_stride(d) >> 1;
        const int32_t WL = (int32_t)((c + 31) >> 5);
        const uint2 *Rp = reinterpret_cast<const uint2 *>(a.R + a.r_off[r]);
        const int s2 = row_span_pairs(Rp, c, j, npairs);
        uint2 rj0 = make_uint2(0, 0), rj1 = make_uint2(0, 0);
        if (s2 > 0) rj0 = Rp[j];
        if (s2 > 1) rj1 = Rp[c + j];
        u128 row_acc = 0;
        int passes = 0;
        for (int32_t t = (j + 1) >> 5; t < WL; ++t) {
            const int32_t x = (t << 5) + lane;
            const bool valid = x > j && x < c;
            int n = 0;
            if (valid) {
                if (s2 <= 2) {
                    n = popc2(rj0, Rp[x]);
                    if (s2 > 1) n += popc2(rj1, Rp[c + x]);
                } else {
                    for (int pw = 0; pw < s2; ++pw) n += popc2(Rp[pw * c + j], Rp[pw * c + x]);
                }
            }
            const bool pass = valid && n >= a.kq;
            const unsigned m = __ballot_sync(kFull, pass);
            passes += __popc(m);
            if (a.k == 3) {
                if (pass) add_u128(row_acc, binom_lookup(a.binom, a.kq, n, ovf), ovf);
            } else if (lane == 0) {
                a.S[a.s_off[r] + (int64_t)t * c + j] = m;
            }
        }
        if (a.k >= 4 && lane == 0 && passes >= a.k - 2) {
            // live unit: tag it with the size class of its subtree (its number of
            // children) so the enumeration can start the largest subtrees first
            atomicAdd(a.n_units, 1);
            const int slot = atomicAdd(a.n_units_all, 1);
            const int b = min(15, 31 - __clz(passes));
            a.units_all[slot] = make_int2(a.job_id, (int)gidx);
            a.units_bucket[slot] = (uint8_t)b;
            atomicAdd(&a.bucket_count[b], 1);
        }
        if (a.per_root && a.k == 3) {
            row_acc = warp_sum_u128(row_acc, ovf);
            if (lane == 0) atomic_add_u128(a.per_root + 2 * (int64_t)r, row_acc, a.status);
            if (lane != 0) row_acc = 0;
        }
        add_u128(acc, row_acc, ovf);
        if (STATS && lane == 0) {
            atomicAdd(&a.stats->evals[2], 1ull);
            atomicAdd(&a.stats->passed[2], 1ull);
            atomicAdd(&a.stats->words_r, (unsigned long long)WRm);
            atomicAdd(&a.stats->words_l, (unsigned long long)WL);
            if (a.k == 3) {
                atomicAdd(&a.stats->evals[3], (unsigned long long)passes);
                atomicAdd(&a.stats->passed[3], (unsigned long long)passes);
                atomicAdd(&a.stats->words_r, (unsigned long long)passes * WRm);
            } else if (passes >= a.k - 2) {
                atomicAdd(&a.stats->units, 1ull);
            }
        }
    }
    if (a.k == 3) {
        acc = warp_sum_u128(acc, ovf);
        if (lane == 0) {
            if (ovf) atomicOr(a.status, kStOverflow);
            atomic_add_u128(a.acc, acc, a.status);
        }
    }
    // The last warp to leave publishes the count when nothing is left for the
    // enumeration: every |L| = 3 count, and larger ones with no live unit.
    if (a.done && lane == 0) {
        __threadfence();
        const int warps = (int)(gridDim.x * (blockDim.x >> 5));
        if (atomicAdd(a.fin, 1) == warps - 1) {
            __threadfence();
            if (a.k == 3 || *(volatile int32_t *)a.n_units == 0) publish_done(a);
        }
    }
}

cudaError_t launch_pairs(const CountArgs &a, int n_sms, cudaStream_t st) {
    if (a.n_cand == 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>((a.n_cand + 7) / 8, (int64_t)n_sms * 8);
    if (a.stats) k_pairs<true><<<grid, 256, 0, st>>>(a);
    else k_pairs<false><<<grid, 256, 0, st>>>(a);
    ++t_launches;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Enumeration of the subtrees below the live level-2 units (k >= 4).
//
// A warp owns one unit at a time and walks its subtree depth-first.  At each
// node the warp takes the node's children 32 at a time (the next 32 set bits of
// C_L) and evaluates them side by side, one child per lane, against the
// parent's C_R and C_L, which sit in shared memory and are read by every lane
// at once (the siblings-share-the-parent idea of Sec. IV's hybrid search).
//
// At a node two levels above the leaves (|L| = k - 2) the warp does not enter
// its children y (the leaf parents).  Each lane forms C_R(y) = C_R & R_y; a
// child that reaches kq takes a slot in the warp's parent list and stages the
// nonzero words of its leaves C_L & S_y (after y) in the warp's leaf-word list.
// The staged words are expanded 32 at a time (count_leaves): for each word,
// the counts |C_R(y) & R_x| of its up to 32 leaves x are summed bit-sliced from
// the root's T block and C(count, kq) is added per leaf (Alg. 1's last two
// levels).  Internal children that pass both pruning tests (|C_R'| >= kq,
// |C_L'| >= k - |L'|) are entered one by one, their C_R' and C_L' rebuilt
// cooperatively.
//
// C_R is read only up to its span (word pairs holding its set bits); thanks to
// the per-root position order, spans are one pair deep in most of the tree.
//
// Per warp: the parent list (kParents C_R(y) as uint4), the leaf-word list
// (kLeafList words and their tags) and, for each level lv = |L| - 2 in
// [0, k-3): CR[lv] : wr words, CL[lv] : wl words, xs[lv] : 32 child ids;
// cursor[lv] (next C_L position to take), dmask[lv] (children still to
// enter), span[lv] (pair span of CR[lv]).
constexpr int kLeafList = 128;  // nonzero leaf words staged per warp before they are expanded
constexpr int kParents = 64;    // leaf parents per warp (their C_R) whose words may be staged
constexpr int kTagShift = 24;   // a staged word's tag: parent slot << 24 | word index (< 2^24)

constexpr int kPhases = 10;  // phases whose SM cycles the executed-traversal statistics add up

struct EnumLayout {
    int wr, wl;     // row capacities in words (both even)
    int levels;     // k - 3 (levels with a node whose children are not all leaf parents)
    int collapse;   // >= 0: count the subtree of a node with |C_R| <= kq + collapse in closed form; -1: off
    // per warp: parents (kParents x uint4) | their word indices (kParents) | leaf masks | leaf tags |
    // levels x (CR | CL | xs) | scalars
    __host__ __device__ int staging_words() const { return kParents * 5 + 2 * kLeafList; }
    __host__ __device__ int level_words() const { return wr + wl + 32; }
    __host__ __device__ int warp_words() const {
        return (staging_words() + levels * level_words() + 3 * kMaxPQ + 2 + 2 * kPhases + 3) & ~3;
    }
};

// Position of the n-th (from 0) set bit of w (n < popc(w)).
__device__ __forceinline__ int select_bit(uint32_t w, int n) {
    int pos = 0, c;
    c = __popc(w & 0xffffu); if (n >= c) { n -= c; w >>= 16; pos += 16; }
    c = __popc(w & 0xffu);   if (n >= c) { n -= c; w >>= 8;  pos += 8; }
    c = __popc(w & 0xfu);    if (n >= c) { n -= c; w >>= 4;  pos += 4; }
    c = __popc(w & 0x3u);    if (n >= c) { n -= c; w >>= 2;  pos += 2; }
    if (n >= (int)(w & 1u)) pos += 1;
    return pos;
}

// The next <= 32 set bits of CL at or after cursor, in order, into xs: lane t
// finds the t-th bit of the round by a shuffle search over the word counts.
__device__ __forceinline__ int gather_children(const uint32_t *CL, int WL, int c, int &cursor, int32_t *xs) {
    const int lane = threadIdx.x & 31;
    int got = 0;
    int pos = cursor;
    while (got < 32 && pos < c) {
        const int w0 = pos >> 5;
        const int wi = w0 + lane;
        uint32_t word = wi < WL ? CL[wi] : 0u;
        if (lane == 0) word &= ~0u << (pos & 31);
        const int cnt = __popc(word);
        const int incl = warp_incl_scan(cnt);
        const int total = __shfl_sync(kFull, incl, 31);
        const int room = 32 - got;
        int src = 0;
#pragma unroll
        for (int b = 16; b >= 1; b >>= 1) {
            const int v = __shfl_sync(kFull, incl, src + b - 1);
            if (v <= lane) src += b;
        }
        src = min(src, 31);
        const uint32_t ws = __shfl_sync(kFull, word, src);
        const int ex = __shfl_sync(kFull, incl - cnt, src);
        const int x = ((w0 + src) << 5) + select_bit(ws, lane - ex);
        if (lane < min(total, room)) xs[got + lane] = x;
        if (total <= room) {
            got += total;
            pos = (w0 + 32) << 5;
        } else {
            pos = __shfl_sync(kFull, x, room - 1) + 1;
            got = 32;
        }
    }
    cursor = pos;
    __syncwarp();
    return got;
}

constexpr int kSmemBinom = 256;  // C(n, kq) for n < 256 in shared memory (never above 2^128)

// Skip sets of the subtree collapse: every s-subset of {0, ..., 15} for s = 2..4
// as a bit mask, in increasing order of the mask (colexicographic order), so
// the first C(m, s) entries of row s are exactly the s-subsets of {0..m-1}.
constexpr int kColexMaxM = 16;
constexpr int kColexMaxS = 4;
constexpr int kColexEntries = 120 + 560 + 1820;
__device__ uint16_t g_colex[kColexEntries];
__device__ __forceinline__ int colex_row(int s) { return s == 2 ? 0 : (s == 3 ? 120 : 680); }
constexpr int kCollapseRounds = 8;  // at most 8 x 32 kq-subsets per collapsed node

__host__ __device__ __forceinline__ int binom_small(int m, int s) {
    return s == 0 ? 1 : s == 1 ? m : s == 2 ? m * (m - 1) / 2
         : s == 3 ? m * (m - 1) * (m - 2) / 6 : m * (m - 1) * (m - 2) * (m - 3) / 24;
}

// Which subtrees collapse: those whose C_R exceeds kq by at most max_skip
// positions; lane t of a round takes C_R minus the t-th skip set of s = m - kq
// positions, at most kCollapseRounds rounds of 32.
__device__ __forceinline__ bool collapsible(int m, int kq, int max_skip) {
    const int s = m - kq;
    if (s > max_skip) return false;
    if (s <= 1) return m <= 32;
    return s <= kColexMaxS && m <= kColexMaxM && binom_small(m, s) <= 32 * kCollapseRounds;
}

cudaError_t init_enumerate_tables() {
    static uint16_t h[kColexEntries];
    static bool made = false;
    if (!made) {
        int at = 0;
        for (int s = 2; s <= kColexMaxS; ++s) {
            // Gosper's successor: the next larger mask with the same popcount
            for (uint32_t v = (1u << s) - 1; v < (1u << kColexMaxM);) {
                if (at == kColexEntries) return cudaErrorInvalidValue;  // cannot happen: C(16, 2..4) entries
                h[at++] = (uint16_t)v;
                const uint32_t lo = v & (0u - v), r = v + lo;
                v = (((r ^ v) >> 2) / lo) | r;
            }
        }
        made = true;
    }
    return cudaMemcpyToSymbol(g_colex, h, sizeof h);
}

// MODE 0: the count.  MODE 1: the count with the search-tree statistics of the
// full traversal (every node evaluated, no collapse), which equal the oracle's.
// MODE 2: the count with the words of the traversal this kernel executes
// (collapsed subtrees included), for the roofline.
template <int MODE>
__global__ void __launch_bounds__(256, 4)
k_enumerate(const CountArgs *jobs, const int2 *units, const int32_t *n_units, int32_t *queue, EnumLayout lay,
            uint32_t *gstack) {
    constexpr bool STATS = MODE == 1;
    constexpr bool WORK = MODE == 2;
    extern __shared__ __align__(16) uint32_t smem_stack[];
    __shared__ ulonglong2 s_binom[kSmemBinom];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    // C(n, kq0) for n < 256 in shared memory, for the first job's kq (any job
    // with another kq reads its own table); binomials do not depend on the graph
    const int kq0 = jobs[0].kq;
    for (int n = threadIdx.x; n < kSmemBinom; n += blockDim.x) {
        bool o = false;
        uint64_t lo = 1, hi = 0;
        for (int jj = 1; jj <= kq0 && !o; ++jj) {
            if (jj > n) { lo = 0; hi = 0; break; }
            o = mul_div_small(lo, hi, (uint32_t)(n - jj + 1), (uint32_t)jj);
        }
        s_binom[n] = make_ulonglong2(lo, hi);
    }
    __syncthreads();
    const CountArgs &a0 = jobs[0];  // holds the batch-wide deadline and status
    uint32_t *wbase = gstack ? gstack + ((int64_t)blockIdx.x * (blockDim.x >> 5) + wib) * lay.warp_words()
                             : smem_stack + (int64_t)wib * lay.warp_words();
    uint4 *PAR = reinterpret_cast<uint4 *>(wbase);              // C_R of the staged leaf parents: up to
    uint32_t *PARI = wbase + kParents * 4;                      // four nonzero words, and their word indices
    uint32_t *LM = PARI + kParents;                             // staged nonzero leaf words
    uint32_t *LT = LM + kLeafList;                              // their tags: slot << kTagShift | word
    uint32_t *base = wbase + lay.staging_words();
    int32_t *cursor = reinterpret_cast<int32_t *>(base + lay.levels * lay.level_words());
    uint32_t *dmask = reinterpret_cast<uint32_t *>(cursor + kMaxPQ);
    int32_t *spanp = reinterpret_cast<int32_t *>(dmask + kMaxPQ);
    auto CR = [&](int lv) { return reinterpret_cast<uint2 *>(base + (int64_t)lv * lay.level_words()); };
    auto CL = [&](int lv) { return base + (int64_t)lv * lay.level_words() + lay.wr; };
    auto XS = [&](int lv) { return reinterpret_cast<int32_t *>(base + (int64_t)lv * lay.level_words() + lay.wr + lay.wl); };

    bool ovf = false;
    unsigned long long st_evals[2] = {0, 0}, st_passed[2] = {0, 0}, st_wr = 0, st_wl = 0;
    unsigned long long wk_words = 0, wk_nodes = 0;  // executed words and collapsed nodes (WORK)
    const int total_units = *n_units;
    // the launch's start: the first warp to get here sets it
    if (lane == 0) atomicCAS(a0.tail, 0ull, global_ns());
    // each unit's start time, kept in the warp's shared scalars (no register)
    unsigned long long *t_unit = reinterpret_cast<unsigned long long *>(spanp + kMaxPQ);
    // SM cycles this warp spends per phase (WORK): 0 unit set-up, 1 collapse,
    // 2 child gather, 3 internal-child tests, 4 descent, 5 leaf-parent nodes
    // (gross), 6 leaf counting, 7 leaf counting inside 5, 8 lane-serial leaf walks,
    // 9 children with |C_R| = kq counted by their own lane (inside 3; lane 0's)
    unsigned long long *ph = t_unit + 1;
    if (WORK && lane == 0)
        for (int i = 0; i < kPhases; ++i) ph[i] = 0;
    auto ph_now = [&]() -> long long { return WORK ? clock64() : 0ll; };
    auto ph_add = [&](int i, long long t0) {
        if (WORK && lane == 0) ph[i] += (unsigned long long)(clock64() - t0);
    };
    while (true) {
        int guidx = 0;
        if (lane == 0) guidx = atomicAdd(queue, 1);
        guidx = __shfl_sync(kFull, guidx, 0);
        if (guidx >= total_units) break;
        const int2 unit = units[guidx];  // (job, global candidate index), largest subtrees first
        const CountArgs &a = jobs[unit.x];
        // the warp that finishes a count's last unit publishes the count
        auto unit_done = [&]() {
            if (a.done && lane == 0) {
                __threadfence();
                if (atomicAdd(a.fin + 1, 1) + 1 == *(volatile int32_t *)a.n_units) {
                    __threadfence();
                    publish_done(a);
                }
            }
        };
        if (__shfl_sync(kFull, (int)past_deadline(a), 0)) {  // this job ran out of time: drop its units
            unit_done();
            continue;
        }
        const int k = a.k, kq = a.kq;
        const bool smem_binom = kq == kq0;
        unsigned long long words = 0;  // words this lane loaded for children (span-truncated; statistics only)
        const int64_t gidx = unit.y;
        const int32_t r = a.cand_root[gidx];
        const int32_t j = (int32_t)(gidx - a.cand_off[r]);
        const int64_t c = a.cand_count[r];
        const int32_t d = a.g.degA[r];
        const int32_t WRm = (d + 31) >> 5;
        const int npairs = row_stride(d) >> 1;
        const int32_t WL = (int32_t)((c + 31) >> 5);
        const uint2 *Rp = reinterpret_cast<const uint2 *>(a.R + a.r_off[r]);
        const uint32_t *St = a.S + a.s_off[r];
        const uint32_t *Tb = St + (int64_t)c * WL;  // T: candidates per position
        const int64_t P = t_rows(d);                // T rows of the root
        const uint32_t *Rw = reinterpret_cast<const uint32_t *>(Rp);
        // word wi of R row x (rows are stored word-major in pairs)
        auto r_word = [&](int32_t x, uint32_t wi) { return Rw[2 * ((int64_t)(wi >> 1) * c + x) + (wi & 1u)]; };
        u128 unit_acc = 0;
        if (lane == 0) *t_unit = global_ns();
        const long long t_setup = ph_now();
        // Collapse of a node's subtree (C_R = cr over nsp pairs holding m
        // positions, C_L = cl from word lo, jrem vertices still to add).  The
        // subtree adds C(|C_R & R_Z|, kq) for every jrem-subset Z of C_L (its
        // pruning only skips zero terms), and summing over the kq-subsets Q of
        // C_R instead gives  sum_Q C(n_Q, jrem),  n_Q = |C_L & T_Q|  where T_Q
        // is the AND of the T rows (candidates containing a position) of Q:
        // the same (L, R) pairs counted from the other side (Def. 1).  Lane t
        // takes the t-th Q, i.e. C_R without its skip set of m - kq positions.
        auto collapse = [&](const uint2 *cr, int nsp, int m, const uint32_t *cl, int lo, int jrem, int32_t *posbuf) {
            const long long tc = ph_now();
            int cur = 0;
            gather_children(reinterpret_cast<const uint32_t *>(cr), 2 * nsp, 64 * nsp, cur, posbuf);
            const int s = m - kq;
            const int pos = lane < m ? posbuf[lane] : 0;
            const int nsub = binom_small(m, s);
            int nzw = 0;
            for (int r0 = 0; r0 < nsub; r0 += 32) {
                const int t = r0 + lane;  // this lane's Q: C_R without skip set t
                uint32_t skip = 0;
                if (s == 1) skip = 1u << t;
                else if (s >= 2 && t < nsub) skip = g_colex[colex_row(s) + t];
                int n = 0;
                for (int w0 = lo; w0 < WL; w0 += 32) {
                    const uint32_t cwl = w0 + lane < WL ? cl[w0 + lane] : 0u;
                    uint32_t nz = __ballot_sync(kFull, cwl != 0u);
                    if (WORK && r0 == 0) nzw += __popc(nz);
                    while (nz) {
                        const int b = __ffs(nz) - 1;
                        nz &= nz - 1;
                        const uint32_t cw = __shfl_sync(kFull, cwl, b);
                        const uint32_t tv = lane < m ? Tb[(int64_t)(w0 + b) * P + pos] : ~0u;
                        if (s == 0) {
                            n += __popc(cw & __reduce_and_sync(kFull, tv));
                        } else {
                            uint32_t acc = cw;
                            for (int l = 0; l < m; ++l) {
                                const uint32_t v = __shfl_sync(kFull, tv, l);
                                if (!((skip >> l) & 1u)) acc &= v;
                            }
                            n += __popc(acc);
                        }
                    }
                }
                if (t < nsub && n >= jrem) {
                    if (jrem == kq && smem_binom && n < kSmemBinom) add_u128(unit_acc, s_binom[n], ovf);
                    else add_u128(unit_acc, binom_lookup(a.binom, jrem, n, ovf), ovf);
                }
            }
            if (WORK && lane == 0) { wk_words += (unsigned long long)(WL - lo) + (unsigned long long)m * nzw; wk_nodes += 1; }
            __syncwarp();
            ph_add(1, tc);
        };
        const bool may_collapse = !STATS && lay.collapse >= 0 && k >= 4;
        // level 2 node {u, j}: C_R = R_j, C_L = S_j (bits after j only)
        bool unit_collapsed = false;
        {
            int mc = 0;
            for (int pw = lane; pw < npairs; pw += 32) {
                const uint2 v = Rp[pw * c + j];
                CR(0)[pw] = v;
                mc += __popc(v.x) + __popc(v.y);
            }
            const int lo = (j + 1) >> 5;
            for (int w = lo + lane; w < WL; w += 32) CL(0)[w] = St[(int64_t)w * c + j];
            const int sp = row_span_pairs(Rp, c, j, npairs);
            if (lane == 0) { cursor[0] = j + 1; dmask[0] = 0; spanp[0] = sp; }
            mc = __reduce_add_sync(kFull, mc);
            __syncwarp();
            ph_add(0, t_setup);
            if (may_collapse && collapsible(mc, kq, lay.collapse)) {
                collapse(CR(0), sp, mc, CL(0), lo, k - 2, XS(0));
                unit_collapsed = true;
            }
        }
        __syncwarp();
        int nl = 0, npar = 0;  // staged leaf words and their parents (warp-uniform)
        // Phase B over LM[0, n_staged): one staged word (parent y, word w, leaves
        // M) per lane.  The leaves' counts |C_R(y) & R_x| for all x of the word
        // are summed bit-sliced: for each position i of C_R(y) the word T_i[w]
        // of candidates containing i is added into 4-bit vertical counters, and
        // the word's leaves add sum_v C(v, kq) * |{x : count = v}|.  A parent's
        // C_R(y) is kept as its (at most four) nonzero words with their word
        // indices in N(u)'s position order, so it may lie anywhere in the row.
        auto count_leaves = [&](int n_staged, bool inside) {
            const long long tl = ph_now();
            for (int e0 = 0; e0 < n_staged; e0 += 32) {
                const int e = e0 + lane;
                if (e < n_staged) {
                    const uint32_t M = LM[e], tg = LT[e];
                    const int w = (int)(tg & ((1u << kTagShift) - 1u));
                    const uint4 cy = PAR[tg >> kTagShift];
                    const uint32_t ix = PARI[tg >> kTagShift];      // word index of cy.x .. cy.w, 8 bits each
                    const uint32_t *Tw = Tb + (int64_t)w * P;       // word w of every T row
                    const int m = __popc(cy.x) + __popc(cy.y) + __popc(cy.z) + __popc(cy.w);
                    if (STATS) st_evals[1] += __popc(M), st_wr += (unsigned long long)__popc(M) * WRm;
                    if (WORK) wk_words += (unsigned long long)__popc(M) * WRm;
                    if (m < 16) {
                        uint32_t b0 = 0u, b1 = 0u, b2 = 0u, b3 = 0u;
#pragma unroll
                        for (int qw = 0; qw < 4; ++qw) {
                            uint32_t bits = qw == 0 ? cy.x : (qw == 1 ? cy.y : (qw == 2 ? cy.z : cy.w));
                            const int wb = (int)((ix >> (8 * qw)) & 0xffu) << 5;  // first position of the word
                            // two positions per step: a carry-save add of both T words
                            // (sum into b0, majority carry into b1..b3); the leaf mask M
                            // is applied once, when the counts are read
                            while (bits) {
                                const int i1 = wb + __ffs(bits) - 1;
                                bits &= bits - 1;
                                const uint32_t t1 = Tw[i1];
                                uint32_t t2 = 0u;
                                if (bits) {
                                    const int i2 = wb + __ffs(bits) - 1;
                                    bits &= bits - 1;
                                    t2 = Tw[i2];
                                }
                                const uint32_t cy2 = (b0 & t1) | (b0 & t2) | (t1 & t2);
                                b0 ^= t1 ^ t2;
                                const uint32_t c1 = b1 & cy2;
                                b1 ^= cy2;
                                const uint32_t c2 = b2 & c1;
                                b2 ^= c1;
                                b3 ^= c2;
                            }
                        }
                        if (STATS) words += m + 1;
                        for (int v = kq; v <= m; ++v) {
                            const uint32_t eq = M & ((v & 1) ? b0 : ~b0) & ((v & 2) ? b1 : ~b1) &
                                                ((v & 4) ? b2 : ~b2) & ((v & 8) ? b3 : ~b3);
                            const int cnt = __popc(eq);
                            if (cnt) {
                                if (STATS) st_passed[1] += cnt;
                                const ulonglong2 bc = (smem_binom && v < kSmemBinom)
                                                          ? s_binom[v] : binom_lookup(a.binom, kq, v, ovf);
                                add_u128(unit_acc, (u128)bc.x * (unsigned)cnt, ovf);
                            }
                        }
                    } else {
                        // |C_R(y)| >= 16 (beyond the 4-bit counters): the leaves one by one
                        uint32_t bits = M;
                        while (bits) {
                            const int32_t x = (w << 5) + __ffs(bits) - 1;
                            bits &= bits - 1;
                            int nx = 0;
#pragma unroll
                            for (int qw = 0; qw < 4; ++qw) {
                                const uint32_t cw = qw == 0 ? cy.x : (qw == 1 ? cy.y : (qw == 2 ? cy.z : cy.w));
                                if (cw) {
                                    nx += __popc(cw & r_word(x, (ix >> (8 * qw)) & 0xffu));
                                    if (STATS) words += 1;
                                }
                            }
                            if (nx >= kq) {
                                if (STATS) st_passed[1] += 1;
                                if (smem_binom && nx < kSmemBinom) add_u128(unit_acc, s_binom[nx], ovf);
                                else add_u128(unit_acc, binom_lookup(a.binom, kq, nx, ovf), ovf);
                            }
                        }
                    }
                }
            }
            ph_add(inside ? 7 : 6, tl);
        };
        int lv = 0;
        unsigned batches = 0;
        while (!unit_collapsed) {
            if ((++batches & 1023u) == 0 && __shfl_sync(kFull, (int)past_deadline(a), 0)) break;
            const uint32_t dm = dmask[lv];
            if (dm != 0) {
                const long long td = ph_now();
                const int t = __ffs(dm) - 1;
                const int32_t x = XS(lv)[t];
                const int sp = spanp[lv];
                __syncwarp();
                if (lane == 0) dmask[lv] = dm & (dm - 1);
                const uint2 *cr = CR(lv);
                uint2 *cr2 = CR(lv + 1);
                const uint32_t *cl = CL(lv);
                uint32_t *cl2 = CL(lv + 1);
                int nsp = 0, mc = 0;
                for (int b = 0; b < sp; b += 32) {
                    const int pw = b + lane;
                    uint2 v = make_uint2(0, 0);
                    if (pw < sp) {
                        v = and2(cr[pw], Rp[pw * c + x]);
                        cr2[pw] = v;
                        mc += __popc(v.x) + __popc(v.y);
                    }
                    const unsigned m = __ballot_sync(kFull, (v.x | v.y) != 0u);
                    if (m) nsp = b + 32 - __clz(m);
                }
                const int lo = (x + 1) >> 5;
                for (int w = lo + lane; w < WL; w += 32) cl2[w] = cl[w] & St[(int64_t)w * c + x];
                if (may_collapse) mc = __reduce_add_sync(kFull, mc);
                __syncwarp();
                ph_add(4, td);
                if (may_collapse && collapsible(mc, kq, lay.collapse)) {
                    // the child (|L| = lv + 3) is counted whole, not entered
                    collapse(cr2, nsp, mc, cl2, lo, k - (lv + 3), XS(lv + 1));
                    continue;
                }
                if (lane == 0) { cursor[lv + 1] = x + 1; dmask[lv + 1] = 0; spanp[lv + 1] = nsp; }
                __syncwarp();
                ++lv;
                continue;
            }
            int cur = cursor[lv];
            const long long tg = ph_now();
            const int got = gather_children(CL(lv), WL, (int)c, cur, XS(lv));
            if (lane == 0) cursor[lv] = cur;
            ph_add(2, tg);
            if (got == 0) {
                __syncwarp();
                if (lv == 0) break;
                --lv;
                continue;
            }
            const int ell = lv + 2;  // |L| of the node
            const int sp = spanp[lv];
            const uint2 *cr = CR(lv);
            const uint32_t *cl = CL(lv);
            if (ell + 2 == k) {
                const long long tp = ph_now();
                // Children y are leaf parents.  Phase A: each lane forms C_R(y) =
                // C_R & R_y; a child that passes puts it in the warp's parent list
                // and stages the nonzero words of its leaf set C_L & S_y (after y)
                // in the warp's leaf-word list.  Phase B (count_leaves) deals the
                // staged words out 32 at a time, whatever parent, node or batch
                // they come from, so every lane evaluates leaves on every step.
                // The lists carry over from batch to batch and node to node of
                // the unit and are expanded when full or when the unit ends.
                // C_R(y) is staged as its nonzero words with their indices, so a
                // node whose C_R spans more than two word pairs stages like the
                // others; a C_R(y) with more than four nonzero words (or one past
                // word 255) has its leaves walked by its own lane instead.
                int32_t y = 0;
                bool py = false, narrow = true;
                uint4 cy = make_uint4(0, 0, 0, 0);
                uint32_t ix = 0x03020100u;  // word indices of cy.x .. cy.w
                if (lane < got) {
                    y = XS(lv)[lane];
                    int ny = 0;
                    if (sp <= 2) {
                        if (sp > 0) { const uint2 v = and2(cr[0], Rp[y]); cy.x = v.x; cy.y = v.y; }
                        if (sp > 1) { const uint2 v = and2(cr[1], Rp[c + y]); cy.z = v.x; cy.w = v.y; }
                        ny = __popc(cy.x) + __popc(cy.y) + __popc(cy.z) + __popc(cy.w);
                    } else {
                        int nw = 0;
                        for (int pw = 0; pw < sp; ++pw) {
                            const uint2 v = and2(cr[pw], Rp[pw * c + y]);
                            ny += __popc(v.x) + __popc(v.y);
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const uint32_t wv = h ? v.y : v.x;
                                if (wv) {
                                    const uint32_t wi = 2u * (uint32_t)pw + (uint32_t)h;
                                    if (nw < 4 && wi < 256u) {
                                        if (nw == 0) cy.x = wv;
                                        else if (nw == 1) cy.y = wv;
                                        else if (nw == 2) cy.z = wv;
                                        else cy.w = wv;
                                        ix = (ix & ~(0xffu << (8 * nw))) | (wi << (8 * nw));
                                    } else {
                                        narrow = false;
                                    }
                                    ++nw;
                                }
                            }
                        }
                    }
                    py = ny >= kq;
                    if (STATS) words += 2 * sp;
                }
                const bool ps = py && narrow;  // staged for phase B
                if (STATS || WORK) {
                    const unsigned pm = __ballot_sync(kFull, py);
                    if (lane == 0) {
                        if (STATS) {
                            st_evals[0] += got;
                            st_passed[0] += __popc(pm);
                            st_wr += (unsigned long long)got * WRm;
                            st_wl += (unsigned long long)__popc(pm) * WL;
                        } else {
                            wk_words += (unsigned long long)got * WRm + (unsigned long long)__popc(pm) * WL;
                        }
                    }
                }
                const int lo_y = (y + 1) >> 5;
                const int lo_min = __reduce_min_sync(kFull, ps ? lo_y : (int)WL);  // first word any staged child stages
                {
                    if (lo_min < WL) {  // else no staged child has a leaf after it
                        const unsigned pm = __ballot_sync(kFull, ps);
                        const int slot = npar + __popc(pm & ((1u << lane) - 1u));
                        if (ps) { PAR[slot] = cy; PARI[slot] = ix; }
                        npar += __popc(pm);  // <= kParents: at most kParents - 32 before the batch
                        for (int w = lo_min; w < WL; ++w) {
                            uint32_t mk = 0;
                            if (ps && w >= lo_y) { mk = cl[w] & St[(int64_t)w * c + y]; if (STATS) words += 1; }
                            const unsigned nz = __ballot_sync(kFull, mk != 0u);
                            if (mk) {
                                const int at = nl + __popc(nz & ((1u << lane) - 1u));
                                LM[at] = mk;
                                LT[at] = ((uint32_t)slot << kTagShift) | (uint32_t)w;
                            }
                            nl += __popc(nz);
                            const bool last = w + 1 == WL;
                            if (nl > kLeafList - 32 || (last && npar > kParents - 32)) {
                                __syncwarp();
                                count_leaves(nl, true);
                                nl = 0;
                                if (last) npar = 0;  // every parent's words are staged and counted
                                __syncwarp();
                            }
                        }
                    }
                }
                const long long tw = ph_now();
                if (py && !narrow) {
                    // C_R(y) spread over more than four words (rare): the lane walks its
                    // own leaves, C_R(y) & R_x re-read per leaf
                    for (int w = lo_y; w < WL; ++w) {
                        uint32_t bits = cl[w] & St[(int64_t)w * c + y];
                        if (STATS) words += 1;
                        while (bits) {
                            const int32_t x = (w << 5) + __ffs(bits) - 1;
                            bits &= bits - 1;
                            int n = 0;
                            for (int pw = 0; pw < sp; ++pw) n += popc2(and2(cr[pw], Rp[pw * c + y]), Rp[pw * c + x]);
                            if (STATS) words += 2 * sp;
                            if (STATS) { st_evals[1] += 1; st_wr += WRm; }
                            if (WORK) wk_words += WRm;
                            if (n >= kq) {
                                if (STATS) st_passed[1] += 1;
                                if (smem_binom && n < kSmemBinom) add_u128(unit_acc, s_binom[n], ovf);
                                else add_u128(unit_acc, binom_lookup(a.binom, kq, n, ovf), ovf);
                            }
                        }
                    }
                }
                __syncwarp();
                ph_add(8, tw);
                ph_add(5, tp);
                if (cur >= c) {  // every child taken: back to the parent at once
                    if (lv == 0) break;
                    --lv;
                }
                continue;  // no child to enter: the next batch of this node
            }
            // internal children: evaluate both pruning tests, flag those to enter
            const long long ti = ph_now();
            int n = 0;
            int32_t x = 0;
            if (lane < got) {
                x = XS(lv)[lane];
                for (int pw = 0; pw < sp; ++pw) n += popc2(cr[pw], Rp[pw * c + x]);
                if (STATS) words += 2 * sp;
            }
            const bool pass = lane < got && n >= kq;
            bool desc = false;
            if (pass) {
                const int lo = (x + 1) >> 5;
                int m = 0;
                for (int w = lo; w < WL; ++w) m += __popc(cl[w] & St[(int64_t)w * c + x]);
                if (STATS) words += WL - lo;
                const int jrem = k - (ell + 1);  // vertices the child still has to add
                desc = m >= jrem;
                if (desc && may_collapse && n == kq) {
                    // |C_R(x)| = kq: the child's subtree is C(n_Q, jrem) for the one
                    // Q = C_R(x), n_Q = |C_L(x) & T_Q|; this lane counts it alone
                    const long long tq = ph_now();
                    int nq = 0, loads = 0;
                    for (int w = lo; w < WL; ++w) {
                        uint32_t acc = cl[w] & St[(int64_t)w * c + x];
                        const uint32_t *Tw = Tb + (int64_t)w * P;
                        for (int pw = 0; pw < sp && acc; ++pw) {
                            const uint2 v = and2(cr[pw], Rp[pw * c + x]);
                            for (uint32_t b = v.x; b && acc; b &= b - 1) acc &= Tw[pw * 64 + __ffs(b) - 1], ++loads;
                            for (uint32_t b = v.y; b && acc; b &= b - 1) acc &= Tw[pw * 64 + 32 + __ffs(b) - 1], ++loads;
                        }
                        nq += __popc(acc);
                    }
                    if (nq >= jrem) add_u128(unit_acc, binom_lookup(a.binom, jrem, nq, ovf), ovf);
                    if (WORK) { wk_words += (unsigned long long)(WL - lo) + loads; wk_nodes += 1; }
                    desc = false;
                    ph_add(9, tq);
                }
            }
            const unsigned dmb = __ballot_sync(kFull, desc);
            if (WORK) {
                const unsigned pm = __ballot_sync(kFull, pass);
                if (lane == 0) wk_words += (unsigned long long)got * WRm + (unsigned long long)__popc(pm) * WL;
            }
            if (STATS) {
                const unsigned pm = __ballot_sync(kFull, pass);
                if (lane == 0) {
                    atomicAdd(&a.stats->evals[ell + 1], (unsigned long long)got);
                    atomicAdd(&a.stats->passed[ell + 1], (unsigned long long)__popc(pm));
                    atomicAdd(&a.stats->words_r, (unsigned long long)got * WRm);
                    atomicAdd(&a.stats->words_l, (unsigned long long)__popc(pm) * WL);
                    atomicAdd(&a.stats->words_enum, (unsigned long long)got * WRm + (unsigned long long)__popc(pm) * WL);
                }
            }
            __syncwarp();
            if (lane == 0) dmask[lv] = dmb;
            __syncwarp();
            ph_add(3, ti);
        }
        if (nl > 0) count_leaves(nl, false);  // the unit's last staged words
        __syncwarp();
        // the unit's sum goes to its job (and to its root when split by root)
        const u128 s = warp_sum_u128(unit_acc, ovf);
#pragma unroll
        if (STATS) for (int o = 16; o >= 1; o >>= 1) words += __shfl_xor_sync(kFull, words, o);
        if (lane == 0) {
            if (ovf) atomicOr(a.status, kStOverflow);
            atomic_add_u128(a.acc, s, a.status);
            if (a.per_root) atomic_add_u128(a.per_root + 2 * (int64_t)r, s, a.status);
            if (STATS) atomicAdd(a.enum_words, words);
        }
        unit_done();
        if (lane == 0) atomicMax(a0.tail + 3, global_ns() - *t_unit);  // longest unit of the launch
        ovf = false;
    }
    if (lane == 0) {
        // this warp's exit: how long after the launch's start the warps leave
        const unsigned long long te = global_ns();
        const unsigned long long t0 = *(volatile unsigned long long *)a0.tail;
        atomicMax(a0.tail + 1, te);
        atomicAdd(a0.tail + 2, te > t0 ? (te - t0) / 1000ull : 0ull);
        atomicAdd(a0.tail + 4, 1ull);
    }
    if (WORK) {
        atomicAdd(&a0.stats->words_exec, wk_words);
        atomicAdd(&a0.stats->collapsed, wk_nodes);
        if (lane == 0)
            for (int i = 0; i < kPhases; ++i) atomicAdd(&a0.stats->phase_cycles[i], ph[i]);
    }
    if (STATS) {
        const CountArgs &a = a0;  // statistics are kept for single-job launches
        const int k = a.k;
        // the last two levels were counted per lane
        atomicAdd(&a.stats->evals[k - 1], st_evals[0]);
        atomicAdd(&a.stats->evals[k], st_evals[1]);
        atomicAdd(&a.stats->passed[k - 1], st_passed[0]);
        atomicAdd(&a.stats->passed[k], st_passed[1]);
        atomicAdd(&a.stats->words_r, st_wr);
        atomicAdd(&a.stats->words_l, st_wl);
        atomicAdd(&a.stats->words_enum, st_wr + st_wl);
    }
}

__global__ void k_sort_units(const int2 *units_all, const uint8_t *bucket, const int32_t *n_all,
                             const int32_t *bucket_count, int32_t *cursor, int2 *sorted) {
    __shared__ int32_t base[16];
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int b = 15; b >= 0; --b) {  // the largest size class first
            base[b] = t;
            t += bucket_count[b];
        }
    }
    __syncthreads();
    const int n = *n_all;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int b = bucket[i];
        sorted[base[b] + atomicAdd(&cursor[b], 1)] = units_all[i];
    }
}

cudaError_t launch_sort_units(const int2 *units_all, const uint8_t *bucket, const int32_t *n_all,
                              const int32_t *bucket_count, int32_t *cursor, int2 *sorted, int64_t capacity,
                              cudaStream_t st) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((capacity + 255) / 256, 4096));
    k_sort_units<<<grid, 256, 0, st>>>(units_all, bucket, n_all, bucket_count, cursor, sorted);
    ++t_launches;
    return cudaGetLastError();
}

cudaError_t launch_enumerate(const CountArgs *d_jobs, const int2 *units, const int32_t *n_units, int32_t *d_queue,
                             int mode, int collapse, int n_warps_hint, int max_wr, int max_wl, int max_k, int n_sms,
                             cudaStream_t st) {
    EnumLayout lay{(max_wr + 1) & ~1, (max_wl + 1) & ~1, std::max(1, max_k - 3), collapse};
    if (max_wl >= (1 << kTagShift)) return cudaErrorInvalidValue;  // staged-word tags hold the word index in 24 bits
    const size_t per_warp = (size_t)lay.warp_words() * 4;
    const int warps_per_cta = 8;
    const size_t smem = per_warp * warps_per_cta;
    const bool use_smem = smem <= 160 * 1024;
    int grid = n_sms * 4;
    if (n_warps_hint > 0) grid = std::max(1, n_warps_hint / warps_per_cta);
    uint32_t *gstack = nullptr;
    cudaError_t err;
    if (use_smem) {
        auto kern = mode == 1 ? k_enumerate<1> : (mode == 2 ? k_enumerate<2> : k_enumerate<0>);
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps_per_cta, smem);
        if (n_warps_hint <= 0) grid = n_sms * std::max(1, per_sm);
        kern<<<grid, 32 * warps_per_cta, smem, st>>>(d_jobs, units, n_units, d_queue, lay, nullptr);
        ++t_launches;
    } else {
        err = cudaMallocAsync(reinterpret_cast<void **>(&gstack), per_warp * warps_per_cta * grid, st);
        if (err != cudaSuccess) return err;
        auto kern = mode == 1 ? k_enumerate<1> : (mode == 2 ? k_enumerate<2> : k_enumerate<0>);
        kern<<<grid, 32 * warps_per_cta, 0, st>>>(d_jobs, units, n_units, d_queue, lay, gstack);
        ++t_launches;
        err = cudaGetLastError();
        cudaFreeAsync(gstack, st);
        return err;
    }
    return cudaGetLastError();
}

}  // namespace gbc
