// gz_motif.cpp - motif counting: the counts of every connected k-vertex pattern
// (Sec. 7.1-7.2 count the motifs of 3 to 5 vertices: 2 patterns on 3 vertices,
// 21 on 5; Sec. 1 quotes 112 size-6 patterns). The patterns are enumerated on the
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

bool connected(int k, uint32_t edges) {
    uint32_t seen = 1, frontier = 1;
    while (frontier) {
        uint32_t next = 0;
        for (int v = 0; v < k; ++v) {
            if (!(frontier >> v & 1)) continue;
            for (int u = 0; u < k; ++u)
                if (u != v && (edges >> ebit(std::min(u, v), std::max(u, v), k) & 1) && !(seen >> u & 1))
                    next |= 1u << u;
        }
        seen |= next;
        frontier = next;
    }
    return seen == (1u << k) - 1;
}

// Canonical code of an edge set: the smallest edge bitmask over the relabellings
// that list the vertices by decreasing degree (an isomorphism maps each degree
// class onto itself, so the minimum over these is the same for the whole
// class); the classes are permuted independently, odometer style.
uint32_t canonical(int k, uint32_t edges) {
    int deg[GZ_MAX_K] = {0};
    for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j)
            if (edges >> ebit(i, j, k) & 1) { ++deg[i]; ++deg[j]; }
    int perm[GZ_MAX_K];
    for (int i = 0; i < k; ++i) perm[i] = i;
    std::sort(perm, perm + k, [&](int a, int b) { return deg[a] != deg[b] ? deg[a] > deg[b] : a < b; });
    int start[GZ_MAX_K + 1], ng = 0;  // class boundaries in perm
    for (int i = 0; i < k; ++i)
        if (i == 0 || deg[perm[i]] != deg[perm[i - 1]]) start[ng++] = i;
    start[ng] = k;
    uint32_t best = UINT32_MAX;
    for (;;) {
        uint32_t code = 0;
        for (int i = 0; i < k; ++i)
            for (int j = i + 1; j < k; ++j) {
                const int a = std::min(perm[i], perm[j]), b = std::max(perm[i], perm[j]);
                if (edges >> ebit(a, b, k) & 1) code |= 1u << ebit(i, j, k);
            }
        best = std::min(best, code);
        int g = ng - 1;  // advance the last class; on wrap-around carry into the previous one
        while (g >= 0 && !std::next_permutation(perm + start[g], perm + start[g + 1])) --g;
        if (g < 0) break;
    }
    return best;
}

}  // namespace

// Every connected graph on k labelled vertices up to isomorphism, as canonical
// edge sets, ordered by edge count and then by code.
std::vector<uint32_t> motif_codes_uncached(int k) {
    const int ne = k * (k - 1) / 2;
    std::set<std::pair<int, uint32_t>> found;
    std::set<uint32_t> seen;
    for (uint32_t e = 0; e < (1u << ne); ++e) {
        if (__builtin_popcount(e) < k - 1 || !connected(k, e)) continue;
        const uint32_t c = canonical(k, e);
        if (seen.insert(c).second) found.insert({__builtin_popcount(c), c});
    }
    std::vector<uint32_t> out;
    for (const auto& f : found) out.push_back(f.second);
    return out;
}

// The same, computed once per k and process.
const std::vector<uint32_t>& motif_codes(int k) {
    static std::mutex mu;
    static std::vector<uint32_t> cache[GZ_MOTIF_MAX_K + 1];
    static bool done[GZ_MOTIF_MAX_K + 1] = {};
    std::lock_guard<std::mutex> lk(mu);
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
    if (st == GZ_OK) {
        std::vector<const gz_graph*> gs(np, g);
        std::vector<int> ori(np, use_orientation);
        st = gz_count_batch(plans.data(), gs.data(), ori.data(), np, stream, counts);
    }
    for (gz_plan* p : plans) gz_plan_destroy(p);
    return st;
}

}  // extern "C"
