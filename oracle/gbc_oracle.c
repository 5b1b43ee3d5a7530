/*
 * Oracle for exact (p,q)-biclique counting -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-purpose CPU code used by the tests, by smoke() and by
 * the benchmark's CPU-baseline leg.  It shares no code, header, table or
 * helper with the CUDA library; the product path never loads it.
 *
 * What it computes (Def. 1 and the problem statement of Sec. II): the number of
 * pairs (L, R), L a p-subset of the anchor side, R a q-subset of the other
 * side, with every vertex of L adjacent to every vertex of R.  Equivalently
 * sum over p-subsets L of C(|common neighbourhood of L|, q).
 *
 * How (Sec. III-A, the Basic model, with the vertex priority of Def. 2 and the
 * pruning rules stated with Alg. 1):
 *   - every anchor vertex u is the root of one search tree; the tree of u only
 *     builds sets L whose lowest-priority member is u, so every L is found once;
 *   - priority: vertices are ordered by (degree, id) ascending and a root keeps
 *     only candidates ranked above itself (Def. 2 uses |N_2^q| as the key; any
 *     strict total order counts each L exactly once, degree is the key used
 *     on both sides of every parity test);
 *   - C_R starts as N(u), C_L as the q-strength 2-hop neighbours of u ranked
 *     above u (Sec. II, N_2^k), kept in rank order;
 *   - roots with fewer than p-1 candidates are dropped (Alg. 1, root filter);
 *   - adding x to L: C_R' = C_R with N(x);  C_L' = the later candidates y of
 *     C_L that are q-strength 2-hop neighbours of x, where common neighbours
 *     are counted inside N(u) (every R of this tree lies in N(u), so two
 *     vertices sharing fewer than q neighbours there cannot both be in L);
 *   - a child x is kept only if |C_R'| >= q, and is descended into only if
 *     |C_L'| >= p - |L'| (the pruning conditions of Alg. 1);
 *   - when |L| = p the leaf adds C(|C_R|, q) (choose q of C_R, Sec. III-A).
 * All counts are unsigned 128-bit; any binomial or sum beyond 2^128-1 makes the
 * call return ORC_OVERFLOW.
 *
 * Instrumentation: for each search node the oracle records the number of
 * 32-bit words a word-bitmap implementation of the same tree reads, with
 * C_R held over the root's d = |N(u)| positions (ceil(d/32) words) and C_L
 * over the root's c = |C_L| candidates (ceil(c/32) words): one C_R row per
 * evaluated child, one C_L row per child that passes the C_R test and is not
 * a leaf.  These are the algorithmic words of the tree.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_OVERFLOW = 2, ORC_NOMEM = 3 };

#define ORC_MAXK 16

typedef struct {
    int64_t roots_expanded;           /* roots with >= p-1 candidates (or p == 1) */
    int64_t evals[ORC_MAXK + 1];      /* children evaluated, by |L| of the child  */
    int64_t passed[ORC_MAXK + 1];     /* children with |C_R'| >= q, by |L|         */
    int64_t words_r;                  /* C_R words read                           */
    int64_t words_l;                  /* C_L words read                           */
    int64_t cand_total;               /* sum over roots of |C_L| at the root      */
    int64_t words_lvl2;               /* the part of words_r + words_l read by the
                                         children of the roots (|L| = 2)          */
} orc_stats;

/* ---- binomial coefficients by Pascal's rule, checked ---------------------- */
typedef struct { u128 v; int ovf; } bin_t;

static bin_t *binom_table(int nmax, int k)
{
    /* T[n*(k+1)+j] = C(n, j), n in [0,nmax], j in [0,k]; ovf marks > 2^128-1 */
    bin_t *t = (bin_t *)calloc((size_t)(nmax + 1) * (size_t)(k + 1), sizeof(bin_t));
    if (!t) return NULL;
    for (int n = 0; n <= nmax; ++n) {
        bin_t *row = t + (size_t)n * (k + 1);
        row[0].v = 1;
        if (n == 0) continue;
        bin_t *up = t + (size_t)(n - 1) * (k + 1);
        for (int j = 1; j <= k; ++j) {
            u128 a = up[j - 1].v, b = up[j].v;
            row[j].v = a + b;
            row[j].ovf = up[j - 1].ovf || up[j].ovf || (row[j].v < a);
        }
    }
    return t;
}

/* ---- sorted-set helpers ---------------------------------------------------- */
static int intersect(const int32_t *a, int na, const int32_t *b, int nb, int32_t *out)
{
    int i = 0, j = 0, n = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { if (out) out[n] = a[i]; ++n; ++i; ++j; }
    }
    return n;
}

static int cmp_i32(const void *x, const void *y)
{
    int32_t a = *(const int32_t *)x, b = *(const int32_t *)y;
    return (a > b) - (a < b);
}

/* ---- one graph viewed from the anchor side -------------------------------- */
typedef struct {
    int32_t nA, nO;
    const int32_t *offA, *adjA;   /* anchor -> other */
    const int32_t *offO, *adjO;   /* other -> anchor */
    int p, q;
    bin_t *binom;                 /* C(n, j), n <= max anchor degree, j <= q */
} view_t;

static inline int deg(const view_t *g, int32_t a) { return g->offA[a + 1] - g->offA[a]; }

/* Def. 2 reading: rank key (degree, id), ascending */
static inline int ranked_above(const view_t *g, int32_t w, int32_t u)
{
    int dw = deg(g, w), du = deg(g, u);
    return dw > du || (dw == du && w > u);
}

static void sort_by_rank(const view_t *g, int32_t *x, int n)
{
    /* insertion sort on (degree, id): plain, the lists are root-local */
    for (int i = 1; i < n; ++i) {
        int32_t v = x[i];
        int j = i - 1;
        while (j >= 0 && ranked_above(g, x[j], v)) { x[j + 1] = x[j]; --j; }
        x[j + 1] = v;
    }
}

typedef struct {
    const view_t *g;
    int32_t root;
    int d, c;                     /* |N(root)|, |C_L at root| */
    int wr, wl;                   /* ceil(d/32), ceil(c/32) */
    int32_t *cand;                /* C_L at the root, rank order */
    int32_t **rsets;              /* rsets[i] = N(cand[i]) within N(root), sorted */
    int *rlen;
    unsigned char *compat;        /* compat[i*c+j]: |R_i with R_j| >= q */
    u128 acc;
    int ovf;
    orc_stats st;
    int32_t *scratch;             /* C_R storage: p levels of d entries */
    int32_t *clbuf;               /* C_L storage: p levels of c entries */
} tree_t;

static void add_checked(tree_t *t, u128 x, int xovf)
{
    u128 s = t->acc + x;
    if (xovf || s < t->acc) t->ovf = 1;
    t->acc = s;
}

/* Node with |L| = ell; its C_R (cr, ncr) and C_L as candidate indices (cl, ncl). */
static void expand(tree_t *t, int ell, const int32_t *cr, int ncr, const int32_t *cl, int ncl)
{
    const view_t *g = t->g;
    int32_t *cr_next = t->scratch + (size_t)ell * t->d;
    int32_t *cl_next = t->clbuf + (size_t)ell * t->c;
    for (int a = 0; a < ncl; ++a) {
        int x = cl[a];
        int n_cr = intersect(cr, ncr, t->rsets[x], t->rlen[x], cr_next);
        t->st.evals[ell + 1] += 1;
        t->st.words_r += t->wr;
        if (ell == 1) t->st.words_lvl2 += t->wr;
        if (n_cr < g->q) continue;
        t->st.passed[ell + 1] += 1;
        if (ell + 1 == g->p) {
            const bin_t *b = g->binom + (size_t)n_cr * (g->q + 1) + g->q;
            add_checked(t, b->v, b->ovf);
            continue;
        }
        int n_cl = 0;
        for (int b2 = a + 1; b2 < ncl; ++b2) {
            int y = cl[b2];
            if (t->compat[(size_t)x * t->c + y]) cl_next[n_cl++] = y;
        }
        t->st.words_l += t->wl;
        if (ell == 1) t->st.words_lvl2 += t->wl;
        if (n_cl < g->p - (ell + 1)) continue;
        expand(t, ell + 1, cr_next, n_cr, cl_next, n_cl);
    }
}

static int count_root(const view_t *g, int32_t u, u128 *out, int *ovf, orc_stats *st)
{
    const int32_t *nu = g->adjA + g->offA[u];
    int d = deg(g, u);
    *out = 0;
    *ovf = 0;
    if (g->p == 1) {
        const bin_t *b = g->binom + (size_t)d * (g->q + 1) + g->q;
        *out = b->v;
        *ovf = b->ovf;
        st->roots_expanded += 1;
        return ORC_OK;
    }
    if (d < g->q) return ORC_OK;

    /* wedges u -> v -> w with w ranked above u; keep w reached >= q times */
    size_t nw = 0;
    for (int i = 0; i < d; ++i) nw += (size_t)(g->offO[nu[i] + 1] - g->offO[nu[i]]);
    int32_t *wed = (int32_t *)malloc((nw ? nw : 1) * sizeof(int32_t));
    if (!wed) return ORC_NOMEM;
    size_t m = 0;
    for (int i = 0; i < d; ++i) {
        int32_t v = nu[i];
        for (int32_t e = g->offO[v]; e < g->offO[v + 1]; ++e) {
            int32_t w = g->adjO[e];
            if (ranked_above(g, w, u)) wed[m++] = w;
        }
    }
    qsort(wed, m, sizeof(int32_t), cmp_i32);
    int c = 0;
    for (size_t i = 0; i < m;) {
        size_t j = i;
        while (j < m && wed[j] == wed[i]) ++j;
        if ((int)(j - i) >= g->q) wed[c++] = wed[i];
        i = j;
    }
    st->cand_total += c;
    if (c < g->p - 1) { free(wed); return ORC_OK; }
    st->roots_expanded += 1;
    sort_by_rank(g, wed, c);

    tree_t t;
    memset(&t, 0, sizeof t);
    t.g = g; t.root = u; t.d = d; t.c = c;
    t.wr = (d + 31) / 32; t.wl = (c + 31) / 32;
    t.cand = wed;
    t.rsets = (int32_t **)calloc((size_t)c, sizeof(int32_t *));
    t.rlen = (int *)calloc((size_t)c, sizeof(int));
    t.compat = (unsigned char *)calloc((size_t)c * (size_t)c, 1);
    t.scratch = (int32_t *)malloc((size_t)(g->p + 1) * (size_t)d * sizeof(int32_t));
    t.clbuf = (int32_t *)malloc((size_t)(g->p + 1) * (size_t)c * sizeof(int32_t));
    int32_t *cl0 = (int32_t *)malloc((size_t)c * sizeof(int32_t));
    int rc = ORC_OK;
    if (!t.rsets || !t.rlen || !t.compat || !t.scratch || !t.clbuf || !cl0) { rc = ORC_NOMEM; goto done; }
    for (int i = 0; i < c; ++i) {
        int32_t w = wed[i];
        int dw = deg(g, w);
        t.rsets[i] = (int32_t *)malloc((size_t)(dw ? dw : 1) * sizeof(int32_t));
        if (!t.rsets[i]) { rc = ORC_NOMEM; goto done; }
        t.rlen[i] = intersect(g->adjA + g->offA[w], dw, nu, d, t.rsets[i]);
    }
    if (g->p >= 3)  /* the 2-hop relation among candidates is only read below level 2 */
        for (int i = 0; i < c; ++i)
            for (int j = i + 1; j < c; ++j)
                t.compat[(size_t)i * c + j] = t.compat[(size_t)j * c + i] =
                    intersect(t.rsets[i], t.rlen[i], t.rsets[j], t.rlen[j], NULL) >= g->q;
    for (int i = 0; i < c; ++i) cl0[i] = i;
    expand(&t, 1, nu, d, cl0, c);
    *out = t.acc;
    *ovf = t.ovf;
    for (int l = 0; l <= ORC_MAXK; ++l) { st->evals[l] += t.st.evals[l]; st->passed[l] += t.st.passed[l]; }
    st->words_r += t.st.words_r;
    st->words_l += t.st.words_l;
    st->words_lvl2 += t.st.words_lvl2;
done:
    if (t.rsets) for (int i = 0; i < c; ++i) free(t.rsets[i]);
    free(t.rsets); free(t.rlen); free(t.compat); free(t.scratch); free(t.clbuf); free(cl0);
    free(wed);
    return rc;
}

/*
 * Count over anchor vertices [root_begin, root_end).  anchor = 0: L on U
 * (size p), R on V (size q); anchor = 1: the roles of the two CSRs swap, L on V
 * has size p and R on U has size q -- callers wanting count(p,q) with V as the
 * anchor pass (q, p) and anchor = 1.
 * per_root (optional): 2 uint64 (lo, hi) per root in the range.
 * total: lo, hi.  Returns ORC_OK / ORC_ERR_ARG / ORC_OVERFLOW / ORC_NOMEM.
 */
int orc_count(int32_t nU, int32_t nV, const int32_t *offU, const int32_t *adjU,
              const int32_t *offV, const int32_t *adjV, int p, int q, int anchor,
              int32_t root_begin, int32_t root_end, uint64_t *per_root,
              uint64_t *total, orc_stats *stats)
{
    if (p < 1 || q < 1 || p > ORC_MAXK || q > ORC_MAXK || nU < 0 || nV < 0) return ORC_ERR_ARG;
    view_t g;
    memset(&g, 0, sizeof g);
    if (anchor == 0) { g.nA = nU; g.nO = nV; g.offA = offU; g.adjA = adjU; g.offO = offV; g.adjO = adjV; }
    else             { g.nA = nV; g.nO = nU; g.offA = offV; g.adjA = adjV; g.offO = offU; g.adjO = adjU; }
    g.p = p; g.q = q;
    if (root_begin < 0) root_begin = 0;
    if (root_end > g.nA) root_end = g.nA;
    orc_stats st;
    memset(&st, 0, sizeof st);
    u128 acc = 0;
    int ovf = 0, rc = ORC_OK;
    int maxd = 0;
    for (int32_t a = 0; a < g.nA; ++a) if (deg(&g, a) > maxd) maxd = deg(&g, a);
    g.binom = binom_table(maxd, q);
    if (!g.binom) return ORC_NOMEM;
    for (int32_t u = root_begin; u < root_end; ++u) {
        u128 r;
        int o;
        rc = count_root(&g, u, &r, &o, &st);
        if (rc != ORC_OK) break;
        if (per_root) {
            per_root[2 * (size_t)(u - root_begin)] = (uint64_t)r;
            per_root[2 * (size_t)(u - root_begin) + 1] = (uint64_t)(r >> 64);
        }
        u128 s = acc + r;
        if (o || s < acc) ovf = 1;
        acc = s;
    }
    free(g.binom);
    if (stats) *stats = st;
    if (rc != ORC_OK) return rc;
    total[0] = (uint64_t)acc;
    total[1] = (uint64_t)(acc >> 64);
    return ovf ? ORC_OVERFLOW : ORC_OK;
}

/* C(n, k) from the oracle's Pascal table; returns 1 if it exceeds 2^128-1. */
int orc_binomial(int n, int k, uint64_t *out)
{
    if (n < 0 || k < 0 || k > 64) return -1;
    bin_t *t = binom_table(n, k);
    if (!t) return -1;
    bin_t b = t[(size_t)n * (k + 1) + k];
    free(t);
    out[0] = (uint64_t)b.v;
    out[1] = (uint64_t)(b.v >> 64);
    return b.ovf;
}
