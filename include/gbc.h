/*
 * gbc.h -- C ABI of the GB300 (sm_103a) exact (p,q)-biclique counter.
 *
 * Problem (Sec. II, Def. 1 and the problem statement): given a bipartite graph
 * G = (U, V, E) and integers p, q, return the number of bicliques B(L, R) with
 * L a subset of U, R a subset of V, |L| = p, |R| = q and every (u, v) in L x R an
 * edge.  The count is exact, as an unsigned 128-bit integer.
 *
 * Method (Sec. III-A Basic model, Sec. IV Alg. 1, Def. 2): one side is the
 * anchor; every anchor vertex u roots a search tree that grows the sets L whose
 * lowest-ranked member is u from u's higher-ranked q-strength 2-hop neighbours
 * (Sec. II, N_2^q), keeps the common neighbourhood C_R as a bitmap over the
 * positions of N(u) and the candidates C_L as a bitmap over the root's
 * candidate list, intersects by word-wise AND plus popcount, and at |L| = p adds
 * C(|C_R|, q).  Every step runs in CUDA kernels on one GPU.
 *
 * Conventions for every call:
 *   - every call returns a gbc_status; outputs are written only on GBC_OK;
 *     gbc_last_error() then describes the last failure of the calling thread;
 *   - no call throws, aborts or exits the process;
 *   - pointers documented as "host" are ordinary CPU memory, borrowed for the
 *     duration of the call only; "device" pointers are CUDA global memory of
 *     the context's device, also borrowed for the call only;
 *   - CSR arrays are int32: off[n+1] with off[0] = 0 and off[n] = |E|,
 *     adj[|E|] with each row strictly increasing (sorted, no duplicates) and in
 *     range; the V-side CSR must be the exact transpose of the U-side CSR;
 *   - 1 <= p, q <= GBC_MAX_PQ, else GBC_ERR_ARG; p > |U| or q > |V| is not an
 *     error and gives 0;
 *   - calls on one context are serialised internally (thread-safe).
 */
#ifndef GBC_H
#define GBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GBC_MAX_PQ 16

/* Unsigned 128-bit count: value = hi * 2^64 + lo. */
typedef struct { uint64_t lo, hi; } gbc_u128;

typedef struct gbc_ctx_s   *gbc_ctx_t;
typedef struct gbc_graph_s *gbc_graph_t;

typedef enum {
    GBC_OK = 0,
    GBC_ERR_ARG = 1,            /* bad argument (null pointer, p or q out of range, ...) */
    GBC_ERR_INVALID_GRAPH = 2,  /* CSR not sorted / not in range / not transposes      */
    GBC_ERR_OOM = 3,            /* device memory or the context's budget exhausted     */
    GBC_ERR_OVERFLOW = 4,       /* the count, or one binomial term, exceeds 2^128 - 1   */
    GBC_ERR_TIMEOUT = 5,        /* a bounded device wait or gbc_poll timed out           */
    GBC_ERR_CUDA = 6,           /* a CUDA runtime call failed                           */
    GBC_PENDING = 7,            /* gbc_poll: the request has not finished yet           */
    GBC_ERR_REJECTED = 8        /* admission refused (queue full / over budget)         */
} gbc_status;

/* Anchor side: which side's vertices root the search trees (the count does not
 * depend on it; Sec. III-A footnote, layer selection deferred to the cost model). */
typedef enum { GBC_ANCHOR_AUTO = 0, GBC_ANCHOR_U = 1, GBC_ANCHOR_V = 2 } gbc_anchor;

/*
 * gbc_ctx_create -- bind a context to CUDA device `device` with a device-memory
 * budget for search scratch (bytes; 0 = 80% of the device's free memory).
 * The context owns one CUDA stream.  Errors: GBC_ERR_ARG (bad device / null
 * out), GBC_ERR_CUDA.
 */
gbc_status gbc_ctx_create(int device, size_t mem_budget_bytes, gbc_ctx_t *out);

/* Use the caller's CUDA stream (a cudaStream_t passed as void*; NULL = the
 * context's own stream) for every later call on this context. */
gbc_status gbc_ctx_set_stream(gbc_ctx_t ctx, void *stream);

/* Release the context (its graphs must be freed first). */
void gbc_ctx_destroy(gbc_ctx_t ctx);

/*
 * gbc_load_graph -- copy a bipartite graph given as CSR on both sides (host
 * arrays) to the device, validate it there and build the per-side index the
 * search uses (Sec. V: neighbour lists re-sorted by the anchor-side priority
 * of Def. 2, with the mirror position of every edge).
 *   nU, nV            vertex counts (>= 0)
 *   offU [nU+1], adjU [|E|]   U -> V adjacency (host)
 *   offV [nV+1], adjV [|E|]   V -> U adjacency (host), the transpose of U's
 * After validation the library renumbers each side by descending degree (ties
 * in the caller's order) for memory locality; the priority order (degree, id)
 * and so every count, per-root split and root range are the caller's, and every
 * vertex id this interface takes or returns is the caller's.  The renumbering
 * runs on the host, O(|U| + |V| + |E|).
 * The graph handle owns its device memory until gbc_free_graph.
 * Errors: GBC_ERR_ARG, GBC_ERR_INVALID_GRAPH, GBC_ERR_OOM, GBC_ERR_CUDA.
 */
gbc_status gbc_load_graph(gbc_ctx_t ctx, int32_t nU, int32_t nV,
                          const int32_t *offU, const int32_t *adjU,
                          const int32_t *offV, const int32_t *adjV,
                          gbc_graph_t *out);

/* As gbc_load_graph (host arrays), with flags: GBC_LOAD_KEEP_IDS keeps the
 * caller's vertex ids on the device instead of renumbering each side by degree
 * (the counts are the same; the other side's id order is then the caller's,
 * e.g. an order from gbc_border_order). */
#define GBC_LOAD_KEEP_IDS 1
gbc_status gbc_load_graph_ex(gbc_ctx_t ctx, int32_t nU, int32_t nV,
                             const int32_t *offU, const int32_t *adjU,
                             const int32_t *offV, const int32_t *adjV,
                             int32_t flags, gbc_graph_t *out);

/* As gbc_load_graph, but the four arrays are device pointers (borrowed; the
 * graph keeps its own copy).  The renumbering copies the U side's arrays and
 * V's offsets to the host once. */
gbc_status gbc_load_graph_device(gbc_ctx_t ctx, int32_t nU, int32_t nV,
                                 const int32_t *offU_d, const int32_t *adjU_d,
                                 const int32_t *offV_d, const int32_t *adjV_d,
                                 gbc_graph_t *out);

/* Release a graph's device memory. */
void gbc_free_graph(gbc_graph_t g);

/* Basic facts of a loaded graph (host outputs; any may be NULL). */
gbc_status gbc_graph_info(gbc_graph_t g, int32_t *nU, int32_t *nV, int64_t *nE,
                          int32_t *max_deg_u, int32_t *max_deg_v);

/*
 * gbc_count -- exact number of (p,q)-bicliques of g (blocking).
 * out: host.  Errors: GBC_ERR_ARG, GBC_ERR_OVERFLOW (count >= 2^128),
 * GBC_ERR_OOM (scratch over the context budget), GBC_ERR_CUDA.
 */
gbc_status gbc_count(gbc_graph_t g, int p, int q, gbc_u128 *out);

/* Options of gbc_count_ex; zero-initialise for the defaults. */
typedef struct {
    int32_t anchor;      /* gbc_anchor; GBC_ANCHOR_AUTO = cost model picks */
    int32_t collect_stats; /* 1: fill gbc_count_info's search-tree counters (slower); 2: fill
                              words_exec and collapsed instead (the executed traversal) */
    int32_t enum_warps;  /* warps of the persistent enumeration launch; 0 = auto */
    int32_t time_limit_ms; /* > 0: device-side deadline; past it the kernels stop and the
                              call returns GBC_ERR_TIMEOUT (the count is then not valid) */
    int32_t root_begin;  /* root_end > root_begin: only anchor vertices in [root_begin, root_end)
                            root search trees, i.e. the count of the bicliques whose lowest-ranked
                            anchor vertex lies there (Def. 2 reading); disjoint ranges that cover
                            the anchor side add up to the count (the split used across GPUs) */
    int32_t root_end;
    int32_t kernel;      /* GBC_KERNEL_BITMAP (0, the default) or GBC_KERNEL_CSR: the same search trees
                            with sorted neighbour lists intersected by binary search instead of
                            bitmaps (the CSR representation Sec. III-B describes; an ablation, counts
                            with |L| >= 3 on the anchor side only) */
    int32_t position_order; /* bit order of a root's C_R bitmaps over the positions of N(u):
                               0 = most shared position first (the default), 1 = the other side's
                               id order (on a graph relabelled by gbc_border_order: Border's order,
                               Sec. V-B); the count does not depend on it */
    int32_t collapse_skip; /* subtree collapse of the bitmap enumeration: a node whose C_R holds at
                              most q' + s positions (q' the set size on the other side) adds its
                              whole subtree in closed form instead of being entered: the sum over
                              the q'-subsets Q of C_R of C(|C_L with every vertex of Q|, vertices
                              still to add) -- the subtree's leaves counted from the other side
                              (Def. 1).  0 = the default s (4); -1 = enter every node; 1..4 = that
                              s (nodes needing more than 256 subsets Q are entered).  The count does
                              not depend on it; collect_stats = 1 always enters every node. */
} gbc_count_options;

/* Set representation of the enumeration (gbc_count_options.kernel). */
enum { GBC_KERNEL_BITMAP = 0, GBC_KERNEL_CSR = 1 };

/* Facts about one count (host output of gbc_count_ex). */
typedef struct {
    int32_t anchor_used;        /* GBC_ANCHOR_U or GBC_ANCHOR_V */
    int32_t set_size;           /* |L| enumerated on the anchor side */
    int64_t roots;              /* anchor vertices with >= set_size-1 candidates */
    int64_t candidates;         /* sum over roots of |C_L| at the root */
    int64_t units;              /* level-2 work units handed to the enumeration */
    int64_t evals[GBC_MAX_PQ + 1];  /* children evaluated, by |L| of the child (stats) */
    int64_t passed[GBC_MAX_PQ + 1]; /* children with |C_R| >= q, by |L| (stats)       */
    int64_t words_r;            /* C_R words of the tree (stats) */
    int64_t words_l;            /* C_L words of the tree (stats) */
    int64_t scratch_bytes;      /* device scratch used by this count */
    float ms_candidates;        /* device time: 2-hop candidates + bitmap rows */
    float ms_pairs;             /* device time: pairwise rows (C_L bitmaps) */
    float ms_enumerate;         /* device time: enumeration kernel */
    float ms_total;             /* device time of the whole count */
    int64_t enum_words;         /* words the enumeration kernel actually loaded for the
                                   children it evaluated (C_R read up to its span; stats) */
    int32_t launches;           /* CUDA kernels this count launched */
    int32_t pieces;             /* root ranges the count ran in: > 1 when its search scratch exceeded
                                   the context's budget and it ran in independent pieces (Sec. VI) */
    int64_t words_enum;         /* the part of words_r + words_l that belongs to the nodes the
                                   enumeration kernel evaluates (|L| >= 3; stats) */
    float enum_span_ms;         /* the enumeration launch, first warp start to last warp exit */
    float enum_longest_unit_ms; /* its longest level-2 unit */
    float enum_exit_spread_ms;  /* how long before the launch's end its warps left, on average
                                   (the launch's tail) */
    int32_t reserved_t;
    int64_t words_exec;         /* words of the traversal the enumeration kernel executes: the
                                   C_R / C_L words of every node it evaluates (as in words_enum),
                                   plus, per collapsed subtree, its C_L words and |C_R| T words per
                                   nonzero C_L word (collect_stats = 2) */
    int64_t collapsed;          /* subtrees the enumeration counted in closed form (collect_stats = 2) */
    int64_t enum_phase_cycles[10]; /* SM clock cycles the enumeration's warps spent per phase
                                      (collect_stats = 2): 0 unit set-up, 1 collapsed subtrees,
                                      2 child gathers, 3 internal-child tests, 4 descents, 5 nodes
                                      whose children are leaf parents (gross: includes 7 and 8),
                                      6 leaf counting at unit ends, 7 leaf counting inside 5,
                                      8 lane-serial leaf walks inside 5, 9 children with
                                      |C_R| = q' counted whole by one lane (inside 3, lane 0's) */
} gbc_count_info;

/* gbc_count with options and facts (either pointer may be NULL). */
gbc_status gbc_count_ex(gbc_graph_t g, int p, int q, const gbc_count_options *opt,
                        gbc_u128 *out, gbc_count_info *info);

/*
 * gbc_count_per_root -- the count split by search-tree root: per_root[a] is the
 * number of (p,q)-bicliques whose lowest-ranked anchor-side vertex (rank key
 * (degree, id), Def. 2 reading) is a.  anchor must be GBC_ANCHOR_U or _V;
 * per_root: host array of |anchor side| entries.  The sum equals gbc_count.
 */
gbc_status gbc_count_per_root(gbc_graph_t g, int p, int q, int anchor,
                              gbc_u128 *per_root, gbc_u128 *total);

/* Most higher-ranked 2-hop neighbours a vertex of U may have in
 * gbc_count_p2_noalloc (its fixed scratch holds one hash table per CTA). */
#define GBC_NOALLOC_MAX_2HOP 4096

/*
 * gbc_count_p2_noalloc -- the number of (2,q)-bicliques (|L| = 2 on U, |R| = q
 * on V) for callers that cannot allocate device memory.  The paper has no
 * counterpart of this entry point.
 *
 * Some callers cannot call cudaMalloc: code living inside another framework's
 * memory pool, plug-ins allowed to touch only the buffers handed to them, or
 * processes whose allocator is reserved.  They pass the graph's CSR arrays in
 * device memory and get the count back; the call itself allocates nothing (no
 * cudaMalloc, cudaFree or allocating library routine).  Its only scratch is one
 * static device array of this library, 16 MiB + 256 B, which every GPU that
 * loads the library holds until the process exits.
 *   nU, nV, offU_d, adjU_d, offV_d, adjV_d: device CSR arrays on the current
 *     device, with the layout rules of gbc_load_graph (not validated here);
 *   q: 1..GBC_MAX_PQ;  stream: a cudaStream_t passed as void* (NULL = the
 *     legacy default stream);  out: host, written on GBC_OK.
 * The first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress) with that device current and keeps it for the life of
 * the process; make that first call before any stream capture.  After
 * cudaDeviceReset, or any other teardown of the device's primary context, the
 * kept address is stale: do not call this entry point on that device again.  Every call shares the array and it keeps the last
 * call's contents (the call clears what must start at zero), so calls that
 * overlap on the GPU -- from other streams or threads -- race and give wrong
 * results: serialise them.
 * Errors: GBC_ERR_ARG; GBC_ERR_OOM when a vertex of U has more than
 * GBC_NOALLOC_MAX_2HOP higher-ranked (by (degree, id)) 2-hop neighbours, the
 * size its fixed scratch holds (the kernel stops at the first such vertex, so
 * this error comes back quickly); GBC_ERR_OVERFLOW; GBC_ERR_CUDA.
 */
gbc_status gbc_count_p2_noalloc(int32_t nU, int32_t nV, const int32_t *offU_d, const int32_t *adjU_d,
                                const int32_t *offV_d, const int32_t *adjV_d, int q, void *stream,
                                gbc_u128 *out);

/*
 * Listing mode: the bicliques themselves (Alg. 1 outputs them; Sec. IV).
 *
 * Records, int32 words in the caller's device buffer, one per leaf of a search
 * tree: the anchor-side set L (|L| = p with anchor U, q with anchor V; the
 * caller's ids, the tree's root first), then m = |C_R|, then the m vertices of
 * C_R (the common neighbourhood of L on the other side, caller's ids), with
 * m >= q (anchor U) or m >= p (anchor V).  Every biclique (L, R) of the count
 * is (L, a subset of C_R) of exactly one record, so the number of bicliques is
 * the sum over records of C(m, q) (anchor U).
 *
 * gbc_list_begin prepares a listing of (g, p, q) from `anchor` (GBC_ANCHOR_AUTO
 * = U): it runs the search once to size every root's records and returns the
 * totals and the words of the largest root's records, the least buffer that
 * drains the listing (host outputs, may be NULL).  Each gbc_list_next call writes the
 * records of the next roots that fit entirely in buf_d (device, capacity_words
 * int32 words, caller-owned): *words and *records (host) say how much it wrote,
 * *done (host) becomes 1 when every record has been written.  The caller
 * consumes the buffer between calls (back-pressure: the listing waits for the
 * caller, nothing is dropped).  A root whose records alone exceed the buffer
 * gives GBC_ERR_OOM (the message states the words it needs).  gbc_list_end
 * releases the listing.  Errors: GBC_ERR_ARG, GBC_ERR_OOM, GBC_ERR_CUDA.
 */
typedef struct gbc_lister_s *gbc_lister_t;
gbc_status gbc_list_begin(gbc_graph_t g, int p, int q, int anchor, gbc_lister_t *out,
                          int64_t *total_words, int64_t *total_records, int64_t *max_root_words);
gbc_status gbc_list_next(gbc_lister_t l, int32_t *buf_d, int64_t capacity_words, int64_t *words,
                         int64_t *records, int *done);
void gbc_list_end(gbc_lister_t l);

/*
 * gbc_count_batch -- many counts, possibly on different graphs of this context,
 * in one pipeline: every stage runs for all jobs before the host waits, and the
 * enumeration (Alg. 1's search below the roots' children, Sec. IV) of all jobs
 * is one persistent launch per set size |L| over the concatenated level-2 work
 * units of the jobs with that size (each launch laid out for its own jobs).
 *   graphs[n], p[n], q[n]: host arrays; graphs must belong to ctx;
 *   out[n]: host, the count of job i when per_job[i] == GBC_OK;
 *   per_job[n]: host, each job's status (GBC_ERR_ARG, _OOM, _OVERFLOW, ...).
 * Returns GBC_OK when the batch ran (check per_job), GBC_ERR_ARG for null
 * arrays, GBC_ERR_CUDA if the device failed.  Scratch is granted in waves that
 * fit the context's budget.
 */
gbc_status gbc_count_batch(gbc_ctx_t ctx, int n, const gbc_graph_t *graphs, const int *p, const int *q,
                           gbc_u128 *out, gbc_status *per_job);

/*
 * gbc_autotune -- for each job (graphs[i], p[i], q[i]) with p, q >= 2, count it
 * from both anchor sides (each run bounded by time_limit_ms, the second also by
 * 1.2x the first's time), check that both agree, and remember the faster side
 * in the context; for |L| >= 4 it then times the enumeration with fewer warps
 * (gbc_tuned_warps).  Later gbc_count / gbc_count_batch calls on the same
 * (graph, p, q) use both (explicit options still win).  The layer choice is a
 * cost question the paper leaves to its CPU predecessor (Sec. IV); this
 * measures it instead.  Entries are dropped when their graph is freed.
 * Errors: GBC_ERR_ARG, and the errors of gbc_count except GBC_ERR_TIMEOUT.
 */
gbc_status gbc_autotune(gbc_ctx_t ctx, int n, const gbc_graph_t *graphs, const int *p, const int *q,
                        int time_limit_ms);

/* The anchor gbc_autotune chose for (g, p, q): GBC_ANCHOR_U, GBC_ANCHOR_V, or 0 if untuned. */
int gbc_tuned_anchor(gbc_graph_t g, int p, int q);

/* The enumeration warps gbc_autotune kept for (g, p, q), or 0 (the default:
 * every SM filled to its occupancy; the autotuner also times a half and a
 * quarter of the SMs' 32 warps each and keeps one only if it is >= 3% faster).
 * A launch over several counts uses the tuned warps only when all of them
 * have some (their largest). */
int gbc_tuned_warps(gbc_graph_t g, int p, int q);

/*
 * Serving (continuous batching).  gbc_serve_start starts `workers` threads
 * (0 = 4), each with its own CUDA streams.  Waiting requests are admitted by
 * their scratch footprint (gbc_footprint): a free worker takes requests from
 * the queue, up to max_batch (0 = 256), while their footprints fit in the part
 * of the context's scratch budget that no running batch holds, and runs them
 * as one batched pipeline (gbc_count_batch's).  Requests that arrive while
 * others are on the GPU are admitted as workers and memory free up, so the
 * pipelines of successive batches overlap on the device.  A request larger
 * than the whole budget runs alone.  Each request completes as soon as its own
 * count is done, not when its batch ends.  max_queue (0 = 4096) bounds the
 * waiting requests; time_limit_ms > 0 gives every request a device deadline
 * (its poll then returns GBC_ERR_TIMEOUT).  The paper has no serving layer;
 * each served count is the count of gbc_count.
 */
gbc_status gbc_serve_start(gbc_ctx_t ctx, int workers, int max_batch, int max_queue, int time_limit_ms);

/* Stop serving: waiting requests are still run; results not yet polled are dropped. */
gbc_status gbc_serve_stop(gbc_ctx_t ctx);

/* Counters of the running server (host output of gbc_serve_stats_get). */
typedef struct {
    int64_t submitted;            /* requests accepted by gbc_submit */
    int64_t rejected;             /* requests refused (queue full) */
    int64_t admitted;             /* requests taken into a batch */
    int64_t batches;              /* batches run */
    int64_t peak_in_flight_bytes; /* most scratch reserved by running batches at once */
    int64_t budget_bytes;         /* the scratch budget the batches share */
    int32_t peak_running_batches; /* most batches on the device at once */
    int32_t reserved_i;
} gbc_serve_stats;

/* The server's counters since gbc_serve_start.  Errors: GBC_ERR_ARG (null, not serving). */
gbc_status gbc_serve_stats_get(gbc_ctx_t ctx, gbc_serve_stats *out);

/*
 * gbc_footprint -- device scratch bytes that the count of (g, p, q) holds (host
 * output), the figure serving admission reserves for it.  *exact (host, may be
 * NULL) is 1 when the same count already ran on this context and the figure is
 * its measured scratch, 0 when it is an upper bound from load-time sums: root u
 * keeps at most omega(u) / q' candidates (omega = its oriented wedges, q' the
 * size on the other side), each with a C_R row of ceil(deg u / 32) words and a
 * C_L row of at most |C_L| / 32 + 5 words (the truncated bitmaps of Sec. V-A
 * sized per root).  Errors: GBC_ERR_ARG.
 */
gbc_status gbc_footprint(gbc_graph_t g, int p, int q, size_t *bytes, int *exact);

/*
 * gbc_submit -- queue the count of (g, p, q) and return its ticket at once
 * (host output).  Starts the server with defaults if needed.  g must stay
 * loaded until the request is polled.  Errors: GBC_ERR_ARG, GBC_ERR_REJECTED
 * (max_queue requests already waiting).
 */
gbc_status gbc_submit(gbc_ctx_t ctx, gbc_graph_t g, int p, int q, uint64_t *ticket);

/*
 * gbc_poll -- the result of a ticket: waits up to timeout_ms (0 = do not wait,
 * < 0 = wait until done).  Returns GBC_PENDING if not finished; otherwise the
 * request's status (its count in *out when GBC_OK), after which the ticket is
 * retired.  Errors: GBC_ERR_ARG (unknown ticket, not serving) and the count's.
 */
gbc_status gbc_poll(gbc_ctx_t ctx, uint64_t ticket, int timeout_ms, gbc_u128 *out);

/*
 * gbc_border_order -- Border (Sec. V-B, Alg. 2), host preprocessing: a new id
 * order of side O that lowers the number of 1-blocks (32-id blocks holding a
 * single neighbour) in the adjacency rows of side A, starting from the order
 * by descending degree and taking at most `iterations` greedy exchanges.
 *   nA, offA [nA+1], adjA [|E|]: A -> O CSR (host, borrowed), nO columns;
 *   max_cand: candidates whose exchange profit each iteration evaluates (the
 *     least-overlapping columns in the blocks v_m's rows fill most; >= 1);
 *   new_id [nO] (host output): the new id of every O vertex (a permutation);
 *   one_blocks_before / _after (host, may be NULL): 1-blocks of the degree
 *     order and of the result.
 * The library's bitmaps are per root over positions of N(u), so Border's order
 * reaches them only through gbc_count_options.position_order = 1 on a graph
 * relabelled with it.  Errors: GBC_ERR_ARG.
 */
gbc_status gbc_border_order(int32_t nA, int32_t nO, const int32_t *offA, const int32_t *adjA,
                            int32_t iterations, int32_t max_cand, int32_t *new_id,
                            int64_t *one_blocks_before, int64_t *one_blocks_after);

/*
 * gbc_measure_int_peaks -- two microbenchmarks on `device` that scale the
 * enumeration's roofline (the paper has no counterpart; the benchmark reports
 * them beside its derived integer peak).  and_popc_words_per_s (host output):
 * words per second of a register-only loop doing one AND, one POPC and one ADD
 * per 32-bit word.  l2_bytes_per_s (host output): bytes per second of an
 * AND + popcount stream over two 16 MiB arrays held in L2 (L1 bypassed).
 * Allocates 32 MiB of device memory for the duration of the call; takes tens
 * of milliseconds.  Errors: GBC_ERR_ARG (null output), GBC_ERR_CUDA.
 */
gbc_status gbc_measure_int_peaks(int device, double *and_popc_words_per_s, double *l2_bytes_per_s);

/* Human-readable text of a status, and the calling thread's last error. */
const char *gbc_status_string(gbc_status s);
const char *gbc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GBC_H */
