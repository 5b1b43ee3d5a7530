// Ablation: the same search trees with sorted-list (CSR) sets instead of
// bitmaps -- the representation of the GPU baseline that Sec. III-B describes
// (neighbour lists in CSR, intersections by binary search), against which the
// paper measures its bitmap design (the HTB ablation of its experiments).
//
// One warp walks one level-2 unit's subtree depth-first (root u and one of its
// candidates, the bitmap path's units, taken from a global queue).  C_R is a
// sorted list of other-side ids (N(u) is a CSR row, sorted by id) and C_L a
// list of the root's candidates in rank order (pass A/B's lists, as in the
// bitmap path).  A child x keeps C_R' = C_R & N(x): each lane takes elements
// of C_R and binary-searches them in the CSR row of x.  The tree, its order
// and its pruning are exactly those of the bitmap kernels (|C_R'| >= kq to
// keep a child; C_L' = the later candidates y with |N(u) & N(x) & N(y)| >= kq,
// the pairwise relation the S rows hold; entered when |C_L'| >= k - |L'|), so
// every count and every search-tree statistic is the same; only the set
// representation differs.
#include <algorithm>

#include "gbc_internal.cuh"

namespace gbc {

namespace {

// Is v in the sorted row [row, row + n)?
__device__ __forceinline__ bool in_row(const int32_t *row, int32_t n, int32_t v) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        const int32_t x = row[mid];
        if (x < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && row[lo] == v;
}

}  // namespace

template <bool STATS>
__global__ void __launch_bounds__(256) k_enumerate_csr(CountArgs a, CsrArgs C) {
    const int lane = threadIdx.x & 31;
    const int warp_g = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const SideView &g = a.g;
    const int k = a.k, kq = a.kq;
    int32_t *stack = C.stack + (int64_t)warp_g * C.stack_words;
    bool ovf = false;
    u128 acc = 0;
    unsigned long long st_ev[kMaxPQ + 1], st_pa[kMaxPQ + 1];
    if (STATS)
        for (int l = 0; l <= kMaxPQ; ++l) st_ev[l] = st_pa[l] = 0;
    // per-warp stack: NU[dmax] | CR[k][dmax] | CL[k][cmax] | nCR[k] | nCL[k] | pos[k] | RX[dmax]
    int32_t *NU = stack;
    int32_t *CRb = NU + C.dmax;
    int32_t *CLb = CRb + (int64_t)k * C.dmax;
    int32_t *nCR = CLb + (int64_t)k * C.cmax;
    int32_t *nCL = nCR + k;
    int32_t *pos = nCL + k;
    int32_t *RX = pos + k;  // R_x = N(u) & N(x) of the child being entered
    bool stop = false;
    while (!stop) {
        // a level-2 unit: root u and its candidate j (the same units as the bitmap path)
        int64_t gidx = 0;
        if (lane == 0) gidx = atomicAdd(C.queue, 1);
        gidx = __shfl_sync(kFull, gidx, 0);
        if (gidx >= a.n_cand || __shfl_sync(kFull, (int)past_deadline(a), 0)) break;
        const int32_t u = a.cand_root[gidx];
        const int32_t c = a.cand_count[u];
        const int32_t j = (int32_t)(gidx - a.cand_off[u]);
        const int32_t d = g.degA[u];
        const int32_t *cand = a.cand + a.cand_off[u];
        // N(u), then level 1 = {u, x_j}: C_R = N(u) & N(x_j) = R_j, C_L = the later
        // candidates y with |R_j & N(y)| >= kq
        for (int32_t i = lane; i < d; i += 32) NU[i] = g.adjA[g.offA[u] + i];
        __syncwarp();
        {
            const int32_t x = cand[j];
            const int32_t *row = g.adjA + g.offA[x];
            const int32_t dx = g.degA[x];
            int m = 0;
            for (int32_t i0 = 0; i0 < d; i0 += 32) {
                const int32_t i = i0 + lane;
                const bool in = i < d && in_row(row, dx, NU[i]);
                const unsigned bal = __ballot_sync(kFull, in);
                if (in) CRb[m + __popc(bal & ((1u << lane) - 1u))] = NU[i];
                m += __popc(bal);
            }
            __syncwarp();
            if (STATS && lane == 0) { st_ev[2] += 1; st_pa[2] += m >= kq; }
            int n2 = 0;
            for (int32_t t0 = j + 1; t0 < c; t0 += 32) {
                const int32_t t = t0 + lane;
                bool keep = false;
                int32_t y = 0;
                if (t < c) {
                    y = cand[t];
                    const int32_t *ry = g.adjA + g.offA[y];
                    const int32_t dy = g.degA[y];
                    int cnt = 0;
                    for (int32_t i = 0; i < m && cnt < kq; ++i) cnt += in_row(ry, dy, CRb[i]);
                    keep = cnt >= kq;
                }
                const unsigned bal = __ballot_sync(kFull, keep);
                if (keep) CLb[n2 + __popc(bal & ((1u << lane) - 1u))] = y;
                n2 += __popc(bal);
            }
            if (lane == 0) { nCR[0] = m; nCL[0] = n2; pos[0] = 0; }
            __syncwarp();
            if (m < kq || n2 < k - 2) continue;  // as the pairwise rows' unit test
        }
        u128 unit_acc = 0;
        unsigned steps = 0;
        int lv = 0;  // node at level lv has |L| = lv + 2
        while (lv >= 0) {
            if ((++steps & 255u) == 0 && __shfl_sync(kFull, (int)past_deadline(a), 0)) { stop = true; break; }
            if (pos[lv] >= nCL[lv]) { --lv; continue; }
            const int ell = lv + 2;
            const int32_t *cr = CRb + (int64_t)lv * C.dmax;
            const int32_t *cl = CLb + (int64_t)lv * C.cmax;
            const int32_t ncr = nCR[lv], ncl = nCL[lv];
            if (ell + 1 == k) {
                // the children are leaves: one per lane, |C_R & N(x)| by binary searches
                const int t0 = pos[lv];
                const int t = t0 + lane;
                int n = 0;
                if (t < ncl) {
                    const int32_t x = cl[t];
                    const int32_t *row = g.adjA + g.offA[x];
                    const int32_t dx = g.degA[x];
                    for (int32_t i = 0; i < ncr; ++i) n += in_row(row, dx, cr[i]);
                    if (n >= kq) add_u128(unit_acc, binom_lookup(a.binom, kq, n, ovf), ovf);
                }
                if (STATS) {
                    const unsigned pm = __ballot_sync(kFull, t < ncl && n >= kq);
                    if (lane == 0) {
                        st_ev[ell + 1] += min(32, ncl - t0);
                        st_pa[ell + 1] += __popc(pm);
                    }
                }
                __syncwarp();
                if (lane == 0) pos[lv] = t0 + 32;
                __syncwarp();
                continue;
            }
            // one internal child at a time: C_R' cooperatively, then C_L'
            const int32_t x = cl[pos[lv]];
            const int next = pos[lv] + 1;
            __syncwarp();
            if (lane == 0) pos[lv] = next;
            const int32_t *row = g.adjA + g.offA[x];
            const int32_t dx = g.degA[x];
            int32_t *cr2 = CRb + (int64_t)(lv + 1) * C.dmax;
            int m = 0;
            for (int32_t i0 = 0; i0 < ncr; i0 += 32) {
                const int32_t i = i0 + lane;
                const bool in = i < ncr && in_row(row, dx, cr[i]);
                const unsigned bal = __ballot_sync(kFull, in);
                if (in) cr2[m + __popc(bal & ((1u << lane) - 1u))] = cr[i];
                m += __popc(bal);
            }
            if (STATS && lane == 0) {
                st_ev[ell + 1] += 1;
                st_pa[ell + 1] += m >= kq;
            }
            __syncwarp();
            if (m < kq) continue;
            // R_x = N(u) & N(x)
            int nrx = 0;
            for (int32_t i0 = 0; i0 < d; i0 += 32) {
                const int32_t i = i0 + lane;
                const bool in = i < d && in_row(row, dx, NU[i]);
                const unsigned bal = __ballot_sync(kFull, in);
                if (in) RX[nrx + __popc(bal & ((1u << lane) - 1u))] = NU[i];
                nrx += __popc(bal);
            }
            __syncwarp();
            int32_t *cl2 = CLb + (int64_t)(lv + 1) * C.cmax;
            int n2 = 0;
            for (int t0 = next; t0 < ncl; t0 += 32) {
                const int t = t0 + lane;
                bool keep = false;
                int32_t y = 0;
                if (t < ncl) {
                    y = cl[t];
                    const int32_t *ry = g.adjA + g.offA[y];
                    const int32_t dy = g.degA[y];
                    int cnt = 0;
                    for (int32_t i = 0; i < nrx && cnt < kq; ++i) cnt += in_row(ry, dy, RX[i]);
                    keep = cnt >= kq;
                }
                const unsigned bal = __ballot_sync(kFull, keep);
                if (keep) cl2[n2 + __popc(bal & ((1u << lane) - 1u))] = y;
                n2 += __popc(bal);
            }
            __syncwarp();
            if (n2 >= k - (ell + 1)) {
                if (lane == 0) {
                    nCR[lv + 1] = m;
                    nCL[lv + 1] = n2;
                    pos[lv + 1] = 0;
                }
                __syncwarp();
                ++lv;
            }
        }
        const u128 us = warp_sum_u128(unit_acc, ovf);
        if (lane == 0) {
            if (a.per_root) atomic_add_u128(a.per_root + 2 * (int64_t)u, us, a.status);
            add_u128(acc, us, ovf);
        }
    }
    if (lane == 0) {
        if (ovf) atomicOr(a.status, kStOverflow);
        atomic_add_u128(a.acc, acc, a.status);
        if (STATS)
            for (int l = 2; l <= kMaxPQ; ++l) {
                if (st_ev[l]) atomicAdd(&a.stats->evals[l], st_ev[l]);
                if (st_pa[l]) atomicAdd(&a.stats->passed[l], st_pa[l]);
            }
    }
}

int64_t csr_stack_words(int k, int32_t dmax, int64_t cmax) {
    return (int64_t)(k + 2) * std::max<int32_t>(dmax, 1) + (int64_t)k * std::max<int64_t>(cmax, 1) + 3 * k + 4;
}

cudaError_t launch_enumerate_csr(const CountArgs &a, const CsrArgs &C, int warps, bool stats, cudaStream_t st) {
    const int blocks = std::max(1, (warps + 7) / 8);
    if (stats) k_enumerate_csr<true><<<blocks, 256, 0, st>>>(a, C);
    else k_enumerate_csr<false><<<blocks, 256, 0, st>>>(a, C);
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace gbc
