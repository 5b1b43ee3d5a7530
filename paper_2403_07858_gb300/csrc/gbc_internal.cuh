// Internal declarations shared by the library's CUDA translation units.
// Nothing here is part of the C ABI (see include/gbc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gbc {

constexpr int kMaxPQ = 16;
constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

typedef unsigned __int128 u128;

// Error bits of the device status word.
enum : uint32_t {
    kStOverflow = 1u << 0,      // a binomial term or the sum exceeded 2^128-1
    kStScratch = 1u << 1,       // a scratch capacity bound was hit (host sizing bug)
    kStBadOffsets = 1u << 2,    // validation: offsets not monotone / wrong ends
    kStBadRange = 1u << 3,      // validation: neighbour id out of range
    kStUnsorted = 1u << 4,      // validation: row not strictly increasing
    kStNotTranspose = 1u << 5,  // validation: the two CSRs are not transposes
    kStTimeout = 1u << 6,       // a bounded device wait ran out
};

// The graph seen from one anchor side A (the side whose vertices root the
// search trees); O is the other side.  Vertex ids are the library's: each side
// renumbered by descending degree at load time, ties in the caller's order, so
// the rank order (degree, id) is the caller's; callerA maps back.
struct SideView {
    int32_t nA, nO;
    const int32_t *offA, *adjA;   // A -> O, rows sorted by O id
    const int32_t *offO;          // O row offsets
    const int32_t *adjO_rank;     // O -> A, rows sorted by A's rank key (deg, id)
    const int32_t *mirror;        // per A-edge e = (a, o): index of a in adjO_rank row of o
    const int32_t *degA;          // degree of every A vertex
    int32_t maxdegA;
    const int32_t *callerA;       // the caller's id of every A vertex
};

// Rank key of Def. 2 (reading: degree first, ties by id), ascending.
__device__ __forceinline__ uint64_t rank_key(const int32_t *deg, int32_t a) {
    return ((uint64_t)(uint32_t)deg[a] << 32) | (uint32_t)a;
}

// Binomial table of one graph: C(n, j) for 0 <= n <= nmax, 0 <= j <= 16, as
// (lo, hi) pairs at [j * (nmax + 1) + n]; n_ovf[j] = least n with C(n, j) >
// 2^128 - 1 (INT32_MAX if none up to nmax).  C(n, j) grows with n for j >= 1,
// so the overflow test of a lookup is n >= n_ovf[j].
struct BinomTable {
    const ulonglong2 *c;
    const int32_t *n_ovf;
    int32_t nmax;
};

__device__ __forceinline__ ulonglong2 binom_lookup(const BinomTable &t, int j, int n, bool &ovf) {
    if (n >= t.n_ovf[j]) { ovf = true; return make_ulonglong2(0, 0); }
    return t.c[(size_t)j * (t.nmax + 1) + n];
}

__device__ __forceinline__ void add_u128(u128 &acc, ulonglong2 v, bool &ovf) {
    u128 x = ((u128)v.y << 64) | v.x;
    u128 s = acc + x;
    if (s < acc) ovf = true;
    acc = s;
}

__device__ __forceinline__ void add_u128(u128 &acc, u128 x, bool &ovf) {
    u128 s = acc + x;
    if (s < acc) ovf = true;
    acc = s;
}

// Warp sum of a u128 with overflow detection; result valid in every lane.
__device__ __forceinline__ u128 warp_sum_u128(u128 v, bool &ovf) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        uint64_t lo = __shfl_xor_sync(kFull, (uint64_t)v, o);
        uint64_t hi = __shfl_xor_sync(kFull, (uint64_t)(v >> 64), o);
        add_u128(v, ((u128)hi << 64) | lo, ovf);
    }
    ovf = __any_sync(kFull, ovf);
    return v;
}

// Atomic 128-bit add into (lo, hi) with exact carry; sets kStOverflow in
// *status when the running total passes 2^128 - 1.  All adds are non-negative,
// so the total wraps exactly when some add carries out of hi.
__device__ __forceinline__ void atomic_add_u128(unsigned long long *dst, u128 v, uint32_t *status) {
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    bool ovf = false;
    if (lo) {
        unsigned long long old = atomicAdd(dst, lo);
        if (old + lo < old) { hi += 1; if (hi == 0) ovf = true; }
    }
    if (hi) {
        unsigned long long old = atomicAdd(dst + 1, hi);
        if (old + hi < old) ovf = true;
    }
    if (ovf) atomicOr(status, kStOverflow);
}

// Inclusive warp scan of an int.
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// (hi, lo) <- (hi, lo) * m / j, exact when j divides the 160-bit product (as it
// does in C(n, j) = C(n, j-1) * (n - j + 1) / j); returns true when the
// quotient does not fit in 128 bits.
__device__ __forceinline__ bool mul_div_small(uint64_t &lo, uint64_t &hi, uint32_t m, uint32_t j) {
    // (hi, lo) * m  ->  (r2, r1, r0)
    uint64_t p0_lo = lo * (uint64_t)m, p0_hi = __umul64hi(lo, (uint64_t)m);
    uint64_t p1_lo = hi * (uint64_t)m, p1_hi = __umul64hi(hi, (uint64_t)m);
    uint64_t r0 = p0_lo;
    uint64_t r1 = p0_hi + p1_lo;
    uint64_t r2 = p1_hi + (r1 < p0_hi ? 1ull : 0ull);
    // divide (r2, r1, r0) by j (<= 16), most significant limb first
    uint64_t q2 = r2 / j, rem = r2 % j;
    uint64_t limbs[2] = {r1, r0}, q[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        uint64_t a = (rem << 32) | (limbs[t] >> 32);
        uint64_t qa = a / j;
        rem = a % j;
        uint64_t b = (rem << 32) | (limbs[t] & 0xffffffffull);
        uint64_t qb = b / j;
        rem = b % j;
        q[t] = (qa << 32) | qb;
    }
    hi = q[0];
    lo = q[1];
    return q2 != 0;
}

// Per-count search statistics (filled only when stats are requested).
struct SearchStats {
    unsigned long long roots;
    unsigned long long cands;
    unsigned long long units;
    unsigned long long evals[kMaxPQ + 1];
    unsigned long long passed[kMaxPQ + 1];
    unsigned long long words_r;
    unsigned long long words_l;
    unsigned long long words_enum;  // the part of words_r + words_l of nodes k_enumerate evaluates
    unsigned long long words_exec;  // words of the traversal k_enumerate executes (collapsed subtrees
                                    // as their C_L and T words)
    unsigned long long collapsed;   // subtrees k_enumerate counted in closed form
    unsigned long long phase_cycles[10];  // SM cycles of k_enumerate's warps per phase (executed traversal)
};

// Sets the text gbc_last_error() returns on the calling thread.
void set_last_error(const char *msg);

// Kernels launched by the calling thread since the last reset (a count runs on
// the calling thread, serialised per context).
extern thread_local int t_launches;

// Completion record of one count in host-mapped memory: the device writes the
// result and then sets flag, so a waiting host thread can release the count as
// soon as its last kernel work is done, before the rest of its batch finishes.
struct DoneRec {
    unsigned long long acc[2];
    uint32_t status;
    uint32_t flag;
};

// Everything one count's kernels share (device pointers).
struct CountArgs {
    SideView g;
    BinomTable binom;
    int k;          // |L| on the anchor side
    int kq;         // |R| on the other side
    int32_t root_begin, root_end;  // roots taken: [root_begin, root_end) (caller's ids)
    // A count whose search scratch exceeds the budget runs in pieces, each a
    // contiguous range of roots in the library's ids (independent search trees,
    // the closure partitioning of Sec. VI); pass B and the pairwise rows then
    // take only roots in [lib_begin, lib_end), whose candidates are the global
    // candidate indices [cand_base, cand_base + n_cand).  R, S, cand and
    // cand_root point so that the piece's global offsets land in its buffers.
    int32_t lib_begin, lib_end;
    int64_t cand_base;
    int32_t position_order;  // 0: a root's positions most shared first; 1: in N(u)'s (id) order
    // root classification
    int32_t *omega;          // [nA] oriented wedge count of each root
    int32_t *tier_list;      // 3 lists of roots, each of capacity nA
    int32_t *tier_count;     // [3]
    int32_t *omega_max;      // [3] max omega per tier
    int32_t *queues;         // [8] persistent-grid work counters
    // pass A / B outputs
    int32_t *cand_count;     // [nA] |C_L| at each root (0 if filtered)
    const int64_t *cand_off; // [nA+1] offsets into cand / cand_root
    const int64_t *r_off;    // [nA+1] word offsets of each root's R block
    const int64_t *s_off;    // [nA+1] word offsets of each root's S block
    int32_t *cand;           // [sum c] candidate ids in rank order
    int32_t *cand_root;      // [sum c] root of each candidate slot
    uint32_t *R;             // R rows: row j of root r is W_R(r) words at R + r_off[r] + j*W_R
    uint32_t *S;             // S rows: row j of root r is W_L(r) words at S + s_off[r] + j*W_L
    int64_t n_cand;          // sum c
    int32_t *n_units;        // [1] live level-2 units of this count
    // live units of every count in the enumeration launch, tagged for ordering
    int32_t job_id;          // this count's index in the launch's job table
    int2 *units_all;         // (job, global candidate index) of each live unit
    uint8_t *units_bucket;   // floor(log2(children)) of each live unit, capped at 15
    int32_t *n_units_all;    // [1]
    int32_t *bucket_count;   // [16]
    int32_t *cand_max;       // [1] largest |C_L| of a kept root
    // global-tier hash slabs
    int32_t *slab;           // per-CTA slabs for roots with large omega
    int64_t slab_words;      // int32 words per CTA slab
    int32_t slab_ctas;       // CTAs (and slabs) of the global-table tier
    // results
    unsigned long long *acc;        // [2] (lo, hi)
    unsigned long long *per_root;   // [2*nA] or null
    uint32_t *status;
    SearchStats *stats;             // or null
    unsigned long long *deadline;   // [1] globaltimer (ns) past which kernels stop; 0 = none
    unsigned long long *enum_words; // [1] C_R + C_L words read by the enumeration kernel
    unsigned long long *tail;       // [5] enumeration launch (globaltimer): start (ns), last warp
                                    // exit (ns), sum of warp exits after the start (us), longest
                                    // unit (ns), warps
    int32_t *poscnt;                // [|E|] per anchor edge slot: candidates containing that position
    int32_t *posmap;                // [|E|] per anchor edge slot: its bit position in the R rows
    DoneRec *done;                  // host-mapped completion record, or null (no early release)
    int32_t *fin;                   // [2] exited k_pairs warps, finished enumeration units
};

// Writes the count's final sum and status to its completion record (called by
// the one thread that finishes the count's last piece of work, after a fence).
__device__ __forceinline__ void publish_done(const CountArgs &a) {
    volatile DoneRec *d = a.done;
    const unsigned long long lo = atomicAdd(a.acc, 0ull), hi = atomicAdd(a.acc + 1, 0ull);
    const uint32_t st = atomicOr(a.status, 0u);
    d->acc[0] = lo;
    d->acc[1] = hi;
    d->status = st;
    __threadfence_system();
    d->flag = 1u;
}

// R rows of a root with d neighbours take ceil(d/32) words, stored with an even
// stride so that two words load at once.
__host__ __device__ __forceinline__ int32_t row_stride(int32_t d) { return (((d + 31) >> 5) + 1) & ~1; }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// True when the count's deadline has passed (then kStTimeout is set) or another
// warp already flagged a timeout.
__device__ __forceinline__ bool past_deadline(const CountArgs &a) {
    if (*(volatile uint32_t *)a.status & kStTimeout) return true;
    const unsigned long long d = *(volatile unsigned long long *)a.deadline;
    if (d != 0ull && global_ns() > d) {
        atomicOr(a.status, kStTimeout);
        return true;
    }
    return false;
}

// Tier bounds on omega (exact number of oriented wedges of a root).
constexpr int kWarpTierOmega = 256;    // warp per root, shared-memory table of 512 slots
constexpr int kWarpTierSlots = 512;
constexpr int kCtaTierOmega = 4096;    // CTA per root, shared-memory table of 8192 slots
constexpr int kCtaTierSlots = 8192;
constexpr int kCtaThreads = 256;
constexpr int kWarpTierWarps = 8;
constexpr int kWarpTierBytes = 2 * kWarpTierSlots * 4 + kWarpTierOmega * 8;

// Listing mode (gbc_list.cu): mode 1 writes each root's record words and
// records to sizes[2u], sizes[2u+1]; mode 2 writes the records of roots
// [begin, end) at out + offsets[u - begin].
struct ListArgs {
    int32_t mode;
    int32_t begin, end;           // roots, library ids
    int32_t *queue;               // zeroed work counter
    int64_t *sizes;               // mode 1: [2 * nA]
    const int64_t *offsets;       // mode 2: [end - begin]
    int32_t *out;                 // mode 2: the caller's buffer
    const int32_t *callerO;       // the caller's id of every other-side vertex
    uint32_t *stack;              // per-warp depth-first stacks
    int64_t stack_words;          // words of one warp's stack
};
int64_t list_stack_words(int k, int32_t maxdeg, int64_t cand_max);
cudaError_t launch_list(const CountArgs &a, const ListArgs &L, int warps, cudaStream_t st);

// The sorted-list (CSR) ablation of the enumeration (gbc_csr.cu): warp per
// root over [lib_begin, lib_end), per-warp stacks of k * (dmax + cmax) ints.
struct CsrArgs {
    int32_t *queue;          // zeroed work counter
    int32_t *stack;          // per-warp depth-first stacks
    int64_t stack_words;     // ints of one warp's stack
    int32_t dmax;            // largest anchor degree (C_R capacity per level)
    int64_t cmax;            // largest candidate list (C_L capacity per level)
};
int64_t csr_stack_words(int k, int32_t dmax, int64_t cmax);
cudaError_t launch_enumerate_csr(const CountArgs &a, const CsrArgs &C, int warps, bool stats, cudaStream_t st);

// Launchers (gbc_kernels.cu).  All run on `st`; none synchronises.
cudaError_t launch_validate_offsets(const int32_t *off, int32_t n, int64_t nE, uint32_t *status, cudaStream_t st);
cudaError_t launch_validate_rows(const int32_t *off, const int32_t *adj, int32_t n, int32_t n_other,
                                 uint32_t *status, cudaStream_t st);
cudaError_t launch_validate_transpose(const int32_t *offU, const int32_t *adjU, int32_t nU,
                                      const int32_t *offV, const int32_t *adjV, uint32_t *status,
                                      cudaStream_t st);
cudaError_t launch_degrees(const int32_t *off, int32_t n, int32_t *deg, int32_t *maxdeg,
                           unsigned long long *wedges, cudaStream_t st);
cudaError_t launch_rank_sort_rows(const int32_t *off, const int32_t *adj, int32_t n_rows,
                                  const int32_t *deg_target, int32_t *out, int32_t max_row,
                                  int64_t *gtmp, cudaStream_t st);
cudaError_t launch_mirror(const int32_t *offA, const int32_t *adjA, int32_t nA, const int32_t *offO,
                          const int32_t *adjO_rank, const int32_t *degA, int32_t *mirror, cudaStream_t st);
cudaError_t launch_binomial(ulonglong2 *c, int32_t *n_ovf, int32_t nmax, cudaStream_t st);
// out[5] (zeroed): sum omega, sum omega * row_stride(deg), max omega, roots with
// omega > 0, sum omega^2 (double bits) over the anchor side A.
cudaError_t launch_footprint_sums(const int32_t *offA, int32_t nA, const int32_t *adjA, const int32_t *offO,
                                  const int32_t *mirror, unsigned long long *out, cudaStream_t st);

cudaError_t launch_single_vertex_sets(const CountArgs &a, cudaStream_t st);
cudaError_t launch_set_deadline(unsigned long long *deadline, unsigned long long limit_ns, cudaStream_t st);
cudaError_t launch_root_omega(const CountArgs &a, cudaStream_t st);
cudaError_t launch_candidates(const CountArgs &a, bool build, const int32_t *tier_counts_host,
                              int n_sms, cudaStream_t st);
cudaError_t launch_root_offsets(const CountArgs &a, int64_t *cand_off, int64_t *r_off, int64_t *s_off,
                                int64_t *tmp, int64_t *totals, cudaStream_t st);
cudaError_t launch_pairs(const CountArgs &a, int n_sms, cudaStream_t st);
// Orders the live units of a launch by their bucket, largest first, into
// sorted (capacity entries); cursor: 16 zeroed ints.
cudaError_t launch_sort_units(const int2 *units_all, const uint8_t *bucket, const int32_t *n_all,
                              const int32_t *bucket_count, int32_t *cursor, int2 *sorted, int64_t capacity,
                              cudaStream_t st);
// One persistent launch over the sorted level-2 units of several counts
// (d_jobs: a device array of their CountArgs, indexed by the units' job id).
// d_queue: a zeroed int32 work counter.
// mode: 0 the count, 1 with the full traversal's statistics, 2 with the words of
// the executed traversal.  collapse >= 0: count the subtrees of nodes with
// |C_R| <= kq + collapse in closed form (never in mode 1); -1: enter every node.
cudaError_t launch_enumerate(const CountArgs *d_jobs, const int2 *units, const int32_t *n_units, int32_t *d_queue,
                             int mode, int collapse, int n_warps_hint, int max_wr, int max_wl, int max_k, int n_sms,
                             cudaStream_t st);
// The enumeration's constant tables on the current device (once per context).
cudaError_t init_enumerate_tables();
// Default of gbc_count_options.collapse_skip.
constexpr int kCollapseSkipDefault = 4;

}  // namespace gbc
