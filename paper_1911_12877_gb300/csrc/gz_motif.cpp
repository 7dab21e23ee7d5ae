// gz_motif.cpp - motif counting: the counts of every connected k-vertex pattern
// (Sec. 7.1-7.2 count the motifs of 3 to 5 vertices: 2 patterns on 3 vertices,
// 21 on 5; Sec. 1 quotes 112 size-6 and 853 size-7 patterns). The patterns are enumerated on the
// host, each is planned like any other pattern, and all of them are counted in
// one batched call.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <set>
#include <vector>

#include "gz_internal.h"

namespace gz {

namespace {

// Edge (i, j), i < j, of a k-vertex graph as a bit index.
inline int ebit(int i, int j, int k) {
    int b = 0;
    for (int r = 0; r < i; ++r) b += k - 1 - r;
    return b + (j - i - 1);
}

// Canonical code of an edge set: the smallest edge bitmask over the relabellings
// that list the vertices by colour, where the colours come from refining the
// degrees (a vertex's new colour ranks its colour together with the sorted
// colours of its neighbours) until the number of colours stops growing. The
// refinement commutes with relabelling, so an isomorphism maps each colour class
// onto itself and the minimum over the permutations inside the classes is the
// same for every graph of an isomorphism class; the classes are permuted
// independently, odometer style.
uint32_t canonical(int k, uint32_t edges) {
    bool adj[GZ_MAX_K][GZ_MAX_K] = {};
    int color[GZ_MAX_K] = {0};
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j)
            if (edges >> ebit(i, j, k) & 1) { adj[i][j] = adj[j][i] = true; ++color[i]; ++color[j]; }
    int ncolors = 0;
    for (;;) {
        std::vector<std::vector<int>> sig(k);
        for (int v = 0; v < k; ++v) {
            sig[v].push_back(color[v]);
            std::vector<int> nb;
            for (int u = 0; u < k; ++u)
                if (adj[v][u]) nb.push_back(color[u]);
            std::sort(nb.begin(), nb.end());
            sig[v].insert(sig[v].end(), nb.begin(), nb.end());
        }
        std::vector<std::vector<int>> dist(sig);
        std::sort(dist.begin(), dist.end());
        dist.erase(std::unique(dist.begin(), dist.end()), dist.end());
        for (int v = 0; v < k; ++v)
            color[v] = (int)(std::lower_bound(dist.begin(), dist.end(), sig[v]) - dist.begin());
        if ((int)dist.size() == ncolors) break;
        ncolors = (int)dist.size();
    }
    int perm[GZ_MAX_K];
    for (int i = 0; i < k; ++i) perm[i] = i;
    std::sort(perm, perm + k, [&](int a, int b) { return color[a] != color[b] ? color[a] < color[b] : a < b; });
    int start[GZ_MAX_K + 1], ng = 0;  // class boundaries in perm
    for (int i = 0; i < k; ++i)
        if (i == 0 || color[perm[i]] != color[perm[i - 1]]) start[ng++] = i;
    start[ng] = k;
    uint32_t best = UINT32_MAX;
    for (;;) {
        uint32_t code = 0;
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j)
                if (adj[perm[i]][perm[j]]) code |= 1u << ebit(i, j, k);
        best = std::min(best, code);
        int g = ng - 1;  // advance the last class; on wrap-around carry into the previous one
        while (g >= 0 && !std::next_permutation(perm + start[g], perm + start[g + 1])) --g;
        if (g < 0) break;
    }
    return best;
}

}  // namespace

const std::vector<uint32_t>& motif_codes(int k);

// Every connected graph on k labelled vertices up to isomorphism, as canonical
// edge sets, ordered by edge count and then by code. Removing a leaf of a
// spanning tree leaves a connected graph connected, so every k-vertex one is a
// connected (k-1)-vertex graph plus a vertex joined to a non-empty subset of it.
std::vector<uint32_t> motif_codes_uncached(int k) {
    if (k == 2) return {1u};
    std::set<std::pair<int, uint32_t>> found;
    for (const uint32_t c : motif_codes(k - 1)) {
        uint32_t base = 0;
        for (int i = 0; i < k - 1; ++i)
            for (int j = i + 1; j < k - 1; ++j)
                if (c >> ebit(i, j, k - 1) & 1) base |= 1u << ebit(i, j, k);
        for (uint32_t sub = 1; sub < (1u << (k - 1)); ++sub) {
            uint32_t e = base;
            for (int i = 0; i < k - 1; ++i)
                if (sub >> i & 1) e |= 1u << ebit(i, k - 1, k);
            const uint32_t cc = canonical(k, e);
            found.insert({__builtin_popcount(cc), cc});
        }
    }
    std::vector<uint32_t> out;
    for (const auto& f : found) out.push_back(f.second);
    return out;
}

// The same, computed once per k and process.
const std::vector<uint32_t>& motif_codes(int k) {
    static std::recursive_mutex mu;  // the k list is built from the k-1 list
    static std::vector<uint32_t> cache[GZ_MOTIF_MAX_K + 1];
    static bool done[GZ_MOTIF_MAX_K + 1] = {};
    std::lock_guard<std::recursive_mutex> lk(mu);
    if (!done[k]) {
        cache[k] = motif_codes_uncached(k);
        done[k] = true;
    }
    return cache[k];
}

}  // namespace gz

using namespace gz;

extern "C" {

gz_status gz_motif_patterns(int k, uint8_t* adjs, int cap, int* count) {
    if (k < 2 || k > GZ_MOTIF_MAX_K || !count) {
        set_error("gz_motif_patterns: k = %d out of range [2, %d]", k, GZ_MOTIF_MAX_K);
        return GZ_EINVAL;
    }
    const std::vector<uint32_t>& codes = motif_codes(k);
    *count = (int)codes.size();
    for (int p = 0; p < (int)codes.size() && p < cap && adjs; ++p) {
        uint8_t* a = adjs + (size_t)p * k * k;
        memset(a, 0, (size_t)k * k);
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j)
                if (codes[p] >> ebit(i, j, k) & 1) a[i * k + j] = a[j * k + i] = 1;
    }
    return GZ_OK;
}

gz_status gz_count_motifs(const gz_graph* g, int k, int use_orientation, void* stream,
                          uint64_t* counts, int cap, int* count) {
    GZ_RANGE("gz_count_motifs");
    if (!g || !count) {
        set_error("gz_count_motifs: NULL argument");
        return GZ_EINVAL;
    }
    int np = 0;
    gz_status st = gz_motif_patterns(k, nullptr, 0, &np);
    if (st != GZ_OK) return st;
    *count = np;
    if (!counts || cap < np) {
        if (counts) {
            set_error("gz_count_motifs: %d patterns of size %d, room for %d", np, k, cap);
            return GZ_EINVAL;
        }
        return GZ_OK;
    }
    std::vector<uint8_t> adj((size_t)np * k * k);
    gz_motif_patterns(k, adj.data(), np, &np);
    std::vector<gz_plan*> plans(np, nullptr);
    for (int p = 0; p < np && st == GZ_OK; ++p) st = gz_plan_create(k, adj.data() + (size_t)p * k * k, 0, &plans[p]);
    if (st == GZ_OK) st = gz_count_merged(plans.data(), np, g, use_orientation, stream, counts);
    for (gz_plan* p : plans) gz_plan_destroy(p);
    return st;
}

}  // extern "C"
