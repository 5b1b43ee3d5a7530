// Border (Sec. V-B, Alg. 2): a greedy reordering of one side's ids that lowers
// the number of 1-blocks -- 32-id blocks of an adjacency row holding a single
// neighbour -- in the bitmaps of the other side's adjacency rows.  Host code:
// the paper runs it as preprocessing, once per graph.
//
// Rows are the vertices of side A, columns the vertices of side O (the side
// being reordered); column v sits at id pos[v], and block B of row r holds the
// row's neighbours with ids in [32B, 32B + 32).  Each iteration:
//   1. takes the column v_m that is alone in its block in the most rows;
//   2. takes candidates v sharing the fewest rows with v_m (Alg. 2 finds them
//      with a matrix product; here the overlaps are counted from v_m's rows,
//      so every column outside them shares none);
//   3. computes the profit of exchanging the ids of v_m and v -- the 1-blocks
//      removed minus the 1-blocks created, x_m + x_n - y_m - y_n -- and keeps
//      the best;
//   4. exchanges the two ids and updates the block counts.
// Reading (the paper leaves the candidate set unbounded; on a sparse graph it
// is almost every column): the profits are evaluated for at most max_cand of
// the least-overlapping columns, taken from the blocks that v_m's rows fill
// most (only there can moving v_m remove a 1-block), and a column whose best
// exchange gains nothing is not taken again.  Each row keeps, per occupied
// block, its count and the XOR of its columns' ids, so a block that drops to
// one neighbour names that neighbour at once.
#include <algorithm>
#include <cstdint>
#include <queue>
#include <unordered_map>
#include <vector>

#include "gbc.h"
#include "gbc_internal.cuh"

namespace gbc {
namespace {

struct BlockCell {
    int32_t count;
    int32_t xr;  // XOR of the column ids (vertex ids, not positions) in the block
};

struct Border {
    int32_t nA, nO;
    const int32_t *offA, *adjA;
    std::vector<int32_t> offO, adjO;               // column -> rows
    std::vector<int32_t> pos;                      // column -> id
    std::vector<int32_t> at;                       // id -> column
    std::vector<std::unordered_map<int32_t, BlockCell>> cells;  // per row: block -> cell
    std::vector<int32_t> ones;                     // column -> rows where it is alone in its block
    int64_t total_ones = 0;

    void build() {
        offO.assign((size_t)nO + 1, 0);
        for (int64_t e = 0; e < offA[nA]; ++e) offO[(size_t)adjA[e] + 1]++;
        for (int32_t v = 0; v < nO; ++v) offO[(size_t)v + 1] += offO[v];
        adjO.resize((size_t)offA[nA]);
        std::vector<int32_t> cur(offO.begin(), offO.end() - 1);
        for (int32_t r = 0; r < nA; ++r)
            for (int32_t e = offA[r]; e < offA[r + 1]; ++e) adjO[(size_t)cur[adjA[e]]++] = r;
        cells.assign((size_t)nA, {});
        for (int32_t r = 0; r < nA; ++r) {
            auto &m = cells[r];
            m.reserve((size_t)(offA[r + 1] - offA[r]));
            for (int32_t e = offA[r]; e < offA[r + 1]; ++e) {
                BlockCell &c = m[pos[adjA[e]] >> 5];
                c.count += 1;
                c.xr ^= adjA[e];
            }
        }
        ones.assign((size_t)nO, 0);
        total_ones = 0;
        for (int32_t r = 0; r < nA; ++r)
            for (auto &kv : cells[r])
                if (kv.second.count == 1) { ones[kv.second.xr]++; total_ones++; }
    }

    static int one(int c) { return c == 1 ? 1 : 0; }

    // 1-blocks removed by exchanging the ids of columns a and b (negative:
    // created); in_a marks a's rows, in_b is zeroed scratch of nA entries
    int64_t profit(int32_t a, int32_t b, const std::vector<char> &in_a, std::vector<char> &in_b) const {
        const int32_t Ba = pos[a] >> 5, Bb = pos[b] >> 5;
        if (Ba == Bb) return 0;
        for (int32_t e = offO[b]; e < offO[b + 1]; ++e) in_b[adjO[e]] = 1;
        int64_t gain = 0;
        auto delta = [&](int32_t r, int32_t from, int32_t to) {
            const auto &m = cells[r];
            auto f = m.find(from);
            auto t = m.find(to);
            const int cf = f == m.end() ? 0 : f->second.count;
            const int ct = t == m.end() ? 0 : t->second.count;
            // before: blocks from (cf) and to (ct); after: cf - 1 and ct + 1
            return (int64_t)(one(cf) + one(ct)) - (int64_t)(one(cf - 1) + one(ct + 1));
        };
        for (int32_t e = offO[a]; e < offO[a + 1]; ++e) {
            const int32_t r = adjO[e];
            if (!in_b[r]) gain += delta(r, Ba, Bb);
        }
        for (int32_t e = offO[b]; e < offO[b + 1]; ++e) {
            const int32_t r = adjO[e];
            if (!in_a[r]) gain += delta(r, Bb, Ba);
        }
        for (int32_t e = offO[b]; e < offO[b + 1]; ++e) in_b[adjO[e]] = 0;
        return gain;
    }

    // move column v of row r from block `from` to block `to`, keeping the counts
    void move(int32_t r, int32_t v, int32_t from, int32_t to) {
        auto &m = cells[r];
        BlockCell &f = m[from];
        if (f.count == 1) { ones[v]--; total_ones--; }
        f.count -= 1;
        f.xr ^= v;
        if (f.count == 1) { ones[f.xr]++; total_ones++; }
        if (f.count == 0) m.erase(from);
        BlockCell &t = m[to];
        if (t.count == 1) { ones[t.xr]--; total_ones--; }
        t.count += 1;
        t.xr ^= v;
        if (t.count == 1) { ones[v]++; total_ones++; }
    }

    void exchange(int32_t a, int32_t b, const std::vector<char> &in_a, std::vector<char> &in_b) {
        const int32_t Ba = pos[a] >> 5, Bb = pos[b] >> 5;
        if (Ba != Bb) {
            for (int32_t e = offO[b]; e < offO[b + 1]; ++e) in_b[adjO[e]] = 1;
            for (int32_t e = offO[a]; e < offO[a + 1]; ++e) {
                const int32_t r = adjO[e];
                if (!in_b[r]) move(r, a, Ba, Bb);
            }
            for (int32_t e = offO[b]; e < offO[b + 1]; ++e) {
                const int32_t r = adjO[e];
                if (!in_a[r]) move(r, b, Bb, Ba);
            }
            for (int32_t e = offO[b]; e < offO[b + 1]; ++e) in_b[adjO[e]] = 0;
        }
        std::swap(pos[a], pos[b]);
        at[pos[a]] = a;
        at[pos[b]] = b;
    }
};

}  // namespace
}  // namespace gbc

using namespace gbc;

extern "C" gbc_status gbc_border_order(int32_t nA, int32_t nO, const int32_t *offA, const int32_t *adjA,
                                       int32_t iterations, int32_t max_cand, int32_t *new_id,
                                       int64_t *one_blocks_before, int64_t *one_blocks_after) {
    if (nA < 0 || nO < 0 || !offA || (offA[nA] > 0 && !adjA) || !new_id || iterations < 0 || max_cand < 1) {
        set_last_error("gbc_border_order: bad argument");
        return GBC_ERR_ARG;
    }
    Border b;
    b.nA = nA;
    b.nO = nO;
    b.offA = offA;
    b.adjA = adjA;
    // start from the degree order (descending degree, ties by id), as the paper does
    std::vector<int32_t> deg((size_t)nO, 0);
    for (int64_t e = 0; e < offA[nA]; ++e) deg[(size_t)adjA[e]]++;
    b.at.resize((size_t)nO);
    for (int32_t v = 0; v < nO; ++v) b.at[v] = v;
    std::stable_sort(b.at.begin(), b.at.end(), [&](int32_t x, int32_t y) { return deg[x] > deg[y]; });
    b.pos.assign((size_t)nO, 0);
    for (int32_t i = 0; i < nO; ++i) b.pos[b.at[i]] = i;
    b.build();
    if (one_blocks_before) *one_blocks_before = b.total_ones;
    // columns by their 1-block count, largest first (lazy entries)
    std::priority_queue<std::pair<int32_t, int32_t>> heap;
    for (int32_t v = 0; v < nO; ++v)
        if (b.ones[v] > 0) heap.push({b.ones[v], v});
    std::vector<char> in_m((size_t)nA, 0), in_b((size_t)nA, 0);
    std::vector<int32_t> overlap((size_t)nO, 0);
    std::vector<char> tried((size_t)nO, 0);
    for (int32_t it = 0; it < iterations && !heap.empty(); ++it) {
        const auto top = heap.top();
        heap.pop();
        const int32_t vm = top.second;
        if (b.ones[vm] != top.first) {  // stale entry
            if (b.ones[vm] > 0) heap.push({b.ones[vm], vm});
            --it;
            continue;
        }
        if (tried[vm]) continue;  // no exchange helped this column before
        // rows of v_m; overlaps of the columns found in them; blocks they fill
        std::vector<int32_t> touched;
        std::unordered_map<int32_t, int32_t> fill;  // block -> rows of v_m with neighbours there
        for (int32_t e = b.offO[vm]; e < b.offO[vm + 1]; ++e) {
            const int32_t r = b.adjO[e];
            in_m[r] = 1;
            for (int32_t f = offA[r]; f < offA[r + 1]; ++f) {
                const int32_t v = adjA[f];
                if (v == vm) continue;
                if (overlap[v]++ == 0) touched.push_back(v);
            }
            for (auto &kv : b.cells[r])
                if (kv.first != (b.pos[vm] >> 5)) fill[kv.first] += 1;
        }
        // candidate blocks: most filled by v_m's rows; candidates there with the least overlap
        std::vector<std::pair<int32_t, int32_t>> blocks(fill.begin(), fill.end());
        std::sort(blocks.begin(), blocks.end(), [](const std::pair<int32_t, int32_t> &x,
                                                   const std::pair<int32_t, int32_t> &y) {
            return x.second != y.second ? x.second > y.second : x.first < y.first;
        });
        std::vector<int32_t> cand;
        int32_t best_ov = INT32_MAX;
        for (size_t bi = 0; bi < blocks.size() && bi < 16; ++bi) {
            for (int32_t id = blocks[bi].first * 32; id < std::min(nO, blocks[bi].first * 32 + 32); ++id) {
                const int32_t v = b.at[id];
                if (v == vm) continue;
                const int32_t ov = overlap[v];
                if (ov < best_ov) { best_ov = ov; cand.clear(); }
                if (ov == best_ov && (int32_t)cand.size() < max_cand) cand.push_back(v);
            }
        }
        int64_t best = 0;
        int32_t vn = -1;
        for (int32_t v : cand) {
            const int64_t pf = b.profit(vm, v, in_m, in_b);
            if (pf > best) { best = pf; vn = v; }
        }
        if (vn >= 0) {
            b.exchange(vm, vn, in_m, in_b);
            // every column whose 1-block count may have changed gets a fresh entry
            heap.push({b.ones[vm], vm});
            heap.push({b.ones[vn], vn});
            for (int32_t v : touched)
                if (b.ones[v] > 0) heap.push({b.ones[v], v});
            for (int32_t e = b.offO[vn]; e < b.offO[vn + 1]; ++e) {
                const int32_t r = b.adjO[e];
                for (int32_t f = offA[r]; f < offA[r + 1]; ++f)
                    if (b.ones[adjA[f]] > 0) heap.push({b.ones[adjA[f]], adjA[f]});
            }
        } else {
            tried[vm] = 1;
        }
        for (int32_t e = b.offO[vm]; e < b.offO[vm + 1]; ++e) in_m[b.adjO[e]] = 0;
        for (int32_t v : touched) overlap[v] = 0;
    }
    for (int32_t v = 0; v < nO; ++v) new_id[v] = b.pos[v];
    if (one_blocks_after) *one_blocks_after = b.total_ones;
    return GBC_OK;
}
