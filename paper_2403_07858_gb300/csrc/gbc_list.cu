// Listing mode: the bicliques themselves, not only their number (Alg. 1
// outputs the set of bicliques; Sec. IV).
//
// A record is one leaf of a root's search tree: the k anchor-side vertices of
// L, then m = |C_R|, then the m other-side vertices of C_R, all as the
// caller's ids (int32).  Every (k,kq)-biclique (L, R) is (L, any kq-subset of
// C_R) for exactly one record, because each L is built by exactly one tree
// (its lowest-ranked member's, Def. 2) and its C_R is its whole common
// neighbourhood.
//
// One warp walks one root's tree depth-first over the R rows of pass B: a
// child x of a node with common neighbourhood C_R gives C_R' = C_R & R_x; it
// is a leaf when |L'| = k and |C_R'| >= kq; otherwise its candidates are the
// later candidates y of the node with |C_R' & R_y| >= kq (exact pruning: any
// other y cannot extend L' to a biclique), and it is entered when at least
// k - |L'| remain.  Mode 1 only sizes each root's records (words and
// records); mode 2 writes them at the root's offset, which the host computed
// from mode 1, so a call never writes past the caller's buffer.
#include <algorithm>

#include "gbc_internal.cuh"

namespace gbc {

namespace {

// Word w of R row x of a root block (rows stored word-major in pairs).
__device__ __forceinline__ uint32_t r_word(const uint32_t *Rb, int64_t c, int32_t x, int w) {
    return Rb[2 * ((int64_t)(w >> 1) * c + x) + (w & 1)];
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

}  // namespace

__global__ void __launch_bounds__(256) k_list(CountArgs a, ListArgs L) {
    const int lane = threadIdx.x & 31;
    const int warp_g = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const SideView &g = a.g;
    const int k = a.k, kq = a.kq;
    uint32_t *stack = L.stack + (int64_t)warp_g * L.stack_words;
    while (true) {
        int32_t u = 0;
        if (lane == 0) u = L.begin + atomicAdd(L.queue, 1);
        u = __shfl_sync(kFull, u, 0);
        if (u >= L.end) break;
        const int32_t d = g.degA[u];
        const int64_t eA = g.offA[u];
        int64_t words = 0, recs = 0;
        int64_t out = L.mode == 2 ? L.offsets[u - L.begin] : 0;
        if (k == 1) {
            // L = {u}: C_R is all of N(u)
            if (d >= kq) {
                words = 2 + d;
                recs = 1;
                if (L.mode == 2) {
                    if (lane == 0) {
                        L.out[out] = g.callerA[u];
                        L.out[out + 1] = d;
                    }
                    for (int32_t i = lane; i < d; i += 32) L.out[out + 2 + i] = L.callerO[g.adjA[eA + i]];
                }
            }
        } else if (a.cand_count[u] >= k - 1 && a.cand_count[u] > 0) {
            const int64_t c = a.cand_count[u];
            const int WR = row_stride(d);
            const uint32_t *Rb = a.R + a.r_off[u];
            const int32_t *cand = a.cand + a.cand_off[u];
            const int32_t *pc = a.poscnt + eA;
            const int32_t *pm = a.posmap + eA;
            // per-warp stack: inv[d] | CR[k][WR] | CL[k][c] | nCL[k] | pos[k] | chosen[k]
            int32_t *inv = reinterpret_cast<int32_t *>(stack);
            uint32_t *CRb = stack + d;
            int32_t *CLb = reinterpret_cast<int32_t *>(CRb + (int64_t)k * WR);
            int32_t *nCL = CLb + (int64_t)k * c;
            int32_t *pos = nCL + k;
            int32_t *chosen = pos + k;
            // bit position -> position in N(u) (positions no candidate holds have no bit)
            for (int32_t i = lane; i < d; i += 32)
                if (__ldcg(&pc[i]) > 0) inv[__ldcg(&pm[i])] = i;
            for (int w = lane; w < WR; w += 32) CRb[w] = 0xffffffffu;
            for (int64_t t = lane; t < c; t += 32) CLb[t] = (int32_t)t;
            if (lane == 0) { nCL[0] = (int32_t)c; pos[0] = 0; }
            __syncwarp();
            int lv = 0;
            while (lv >= 0) {
                if (pos[lv] >= nCL[lv]) { --lv; continue; }
                const int32_t x = CLb[(int64_t)lv * c + pos[lv]];
                const int next = pos[lv] + 1;
                __syncwarp();
                if (lane == 0) pos[lv] = next;
                const uint32_t *cr = CRb + (int64_t)lv * WR;
                uint32_t *cr2 = CRb + (int64_t)(lv + 1) * WR;  // lv + 1 <= k - 1: the child's row
                // C_R' = C_R & R_x
                const bool leaf = lv + 2 == k;
                int m = 0;
                for (int w = lane; w < WR; w += 32) {
                    const uint32_t v = cr[w] & r_word(Rb, c, x, w);
                    m += __popc(v);
                    cr2[w] = v;
                }
                m = warp_sum_int(m);
                __syncwarp();
                if (m < kq) continue;
                if (leaf) {
                    words += k + 1 + m;
                    recs += 1;
                    if (L.mode == 2) {
                        // L: the root, the chosen children of the path, then x
                        if (lane < k) {
                            int32_t cidx = lane == 0 ? -1 : (lane < k - 1 ? chosen[lane] : x);
                            const int32_t lib = lane == 0 ? u : cand[cidx];
                            L.out[out + lane] = g.callerA[lib];
                        }
                        if (lane == 0) L.out[out + k] = m;
                        // C_R: each lane writes the vertices of its words, after the
                        // vertices of the words before them
                        int base = 0;
                        for (int w0 = 0; w0 < WR; w0 += 32) {
                            const int w = w0 + lane;
                            uint32_t v = w < WR ? cr2[w] : 0u;
                            const int cnt = __popc(v);
                            int incl = warp_incl_scan(cnt);
                            int at = base + incl - cnt;
                            while (v) {
                                const int b = __ffs(v) - 1;
                                v &= v - 1;
                                const int32_t i = inv[(w << 5) + b];
                                L.out[out + k + 1 + at] = L.callerO[g.adjA[eA + i]];
                                ++at;
                            }
                            base += __shfl_sync(kFull, incl, 31);
                        }
                        out += k + 1 + m;
                    }
                    __syncwarp();
                    continue;
                }
                // the child's candidates: later candidates y with |C_R' & R_y| >= kq
                const int ell = lv + 2;  // |L'|
                const int32_t *cl = CLb + (int64_t)lv * c;
                int32_t *cl2 = CLb + (int64_t)(lv + 1) * c;
                int n = 0;
                for (int t0 = next; t0 < nCL[lv]; t0 += 32) {
                    const int t = t0 + lane;
                    bool keep = false;
                    int32_t y = 0;
                    if (t < nCL[lv]) {
                        y = cl[t];
                        int cnt = 0;
                        for (int w = 0; w < WR && cnt < kq; ++w) cnt += __popc(cr2[w] & r_word(Rb, c, y, w));
                        keep = cnt >= kq;
                    }
                    const unsigned bal = __ballot_sync(kFull, keep);
                    if (keep) cl2[n + __popc(bal & ((1u << lane) - 1u))] = y;
                    n += __popc(bal);
                }
                __syncwarp();
                if (n >= k - ell) {
                    if (lane == 0) {
                        chosen[lv + 1] = x;
                        nCL[lv + 1] = n;
                        pos[lv + 1] = 0;
                    }
                    __syncwarp();
                    ++lv;
                }
            }
        }
        if (lane == 0 && L.mode == 1) {
            L.sizes[2 * (int64_t)u] = words;
            L.sizes[2 * (int64_t)u + 1] = recs;
        }
        __syncwarp();
    }
}

int64_t list_stack_words(int k, int32_t maxdeg, int64_t cand_max) {
    return (int64_t)maxdeg + (int64_t)k * row_stride(maxdeg) + (int64_t)k * std::max<int64_t>(cand_max, 1) + 3 * k + 4;
}

cudaError_t launch_list(const CountArgs &a, const ListArgs &L, int warps, cudaStream_t st) {
    const int blocks = std::max(1, (warps + 7) / 8);
    k_list<<<blocks, 256, 0, st>>>(a, L);
    ++t_launches;
    return cudaGetLastError();
}

}  // namespace gbc
