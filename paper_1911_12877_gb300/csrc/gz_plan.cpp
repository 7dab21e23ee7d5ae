// gz_plan.cpp - the host planner: automorphisms (Sec. 4.2), distinct schedules
// (Algorithm 4, Sec. 5.3), restrictions (Algorithm 1 with the Theorem 2
// reduction), the performance model (Sec. 5.4, Appendix) and the compilation of
// the chosen schedule into the per-loop set-operation program the kernels run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "gz_internal.h"

namespace gz {

namespace {

using Perm = std::vector<int>;

struct Pattern {
    int k;
    bool a[GZ_MAX_K][GZ_MAX_K];
};

bool load_pattern(int k, const uint8_t* adj, Pattern& p) {
    if (k < 2 || k > GZ_MAX_K || !adj) {
        set_error("pattern: k = %d out of range [2, %d]", k, GZ_MAX_K);
        return false;
    }
    p.k = k;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            p.a[i][j] = adj[i * k + j] != 0;
            if ((adj[i * k + j] != 0) != (adj[j * k + i] != 0)) {
                set_error("pattern: adjacency not symmetric at (%d, %d)", i, j);
                return false;
            }
        }
    for (int i = 0; i < k; ++i)
        if (p.a[i][i]) {
            set_error("pattern: self-loop at %d", i);
            return false;
        }
    unsigned seen = 1, frontier = 1;
    while (frontier) {
        unsigned next = 0;
        for (int v = 0; v < k; ++v)
            if (frontier >> v & 1)
                for (int u = 0; u < k; ++u)
                    if (p.a[v][u] && !(seen >> u & 1)) next |= 1u << u;
        seen |= next;
        frontier = next;
    }
    if (seen != (1u << k) - 1) {
        set_error("pattern: not connected");
        return false;
    }
    return true;
}

// Sec. 4.2: every label permutation that preserves adjacency and non-adjacency.
std::vector<Perm> automorphisms(const Pattern& p) {
    std::vector<Perm> out;
    Perm x(p.k);
    for (int i = 0; i < p.k; ++i) x[i] = i;
    do {
        bool ok = true;
        for (int i = 0; i < p.k && ok; ++i)
            for (int j = i + 1; j < p.k && ok; ++j) ok = p.a[i][j] == p.a[x[i]][x[j]];
        if (ok) out.push_back(x);
    } while (std::next_permutation(x.begin(), x.end()));
    return out;
}

bool valid_schedule(const Pattern& p, const int32_t* order) {
    unsigned used = 0;
    for (int i = 0; i < p.k; ++i) {
        int v = order[i];
        if (v < 0 || v >= p.k || (used >> v & 1)) return false;
        if (i > 0) {
            bool conn = false;
            for (int j = 0; j < i; ++j) conn = conn || p.a[v][order[j]];
            if (!conn) return false;
        }
        used |= 1u << v;
    }
    return true;
}

// Algorithm 4. `aut` holds the automorphisms fixing every scheduled label;
// candidates equivalent under them are marked processed and skipped.
void explore(const Pattern& p, std::vector<int>& sched, const std::vector<Perm>& aut,
             unsigned valid_next, std::vector<std::vector<int>>& out) {
    const int k = p.k;
    if ((int)sched.size() == k) {
        out.push_back(sched);
        return;
    }
    unsigned iterate = sched.empty() ? (1u << k) - 1 : valid_next;
    unsigned processed = 0;
    for (int v = 0; v < k; ++v) {
        if (!(iterate >> v & 1) || (processed >> v & 1)) continue;
        std::vector<Perm> stab;
        for (const Perm& x : aut) {
            if (x[v] == v) stab.push_back(x);
            else processed |= 1u << x[v];
        }
        unsigned in_sched = 1u << v;
        for (int s : sched) in_sched |= 1u << s;
        unsigned nb = 0;
        for (int u = 0; u < k; ++u)
            if (p.a[v][u]) nb |= 1u << u;
        sched.push_back(v);
        explore(p, sched, stab, (valid_next | nb) & ~in_sched, out);
        sched.pop_back();
    }
}

// Algorithm 1 + Theorem 2: bp[i] = schedule position that bounds position i.
void restrictions(const Pattern& p, const std::vector<Perm>& aut_all, const int32_t* order,
                  int32_t* bp) {
    const int k = p.k;
    int pos[GZ_MAX_K];
    for (int i = 0; i < k; ++i) pos[order[i]] = i;
    int parent_label[GZ_MAX_K];
    for (int i = 0; i < k; ++i) parent_label[i] = -1;
    std::vector<Perm> aut = aut_all;
    for (int s = 0; s < k; ++s) {
        const int v = order[s];
        std::vector<Perm> stab;
        for (const Perm& x : aut) {
            if (x[v] == v) stab.push_back(x);
            else parent_label[x[v]] = v;  // later v overwrite: the largest z survives
        }
        aut.swap(stab);
    }
    for (int i = 0; i < k; ++i)
        bp[i] = parent_label[order[i]] < 0 ? -1 : pos[parent_label[order[i]]];
}

// Sec. 5.4 / Appendix with n = 1000 and average degree 5 (Sec. 7.3).
double model_cost(const Pattern& p, const int32_t* order, const int32_t* bp) {
    const int k = p.k;
    const double n = 1000.0, pr = 5.0 / 999.0;
    double prod = 1.0, cost = 0.0;
    for (int d = 0; d < k; ++d) {
        double iters = n;
        if (d > 0) {
            int nb = 0, nr = 0;
            for (int j = 0; j < d; ++j) (p.a[order[d]][order[j]] ? nb : nr)++;
            iters = n * std::pow(pr, (double)nb) * std::pow(1.0 - pr, (double)nr);
        }
        prod *= iters;
        // restriction pass probability of loops 0..d: prod_i 1/z_i, z_i = size of
        // i's subtree in the bound-parent forest restricted to loops <= d
        double pass = 1.0;
        for (int i = 0; i <= d; ++i) {
            int z = 0;
            for (int j = 0; j <= d; ++j) {
                int a = j;
                while (a >= 0 && a != i) a = bp[a];
                if (a == i) ++z;
            }
            pass /= (double)z;
        }
        cost += prod * pass;
    }
    return cost;
}

// ------------------------------------------------------------ compilation

struct Compiler {
    int k;
    bool black[GZ_MAX_K][GZ_MAX_K];  // schedule positions
    int bp[GZ_MAX_K];
    GzProg prog;

    bool is_anc_or_self(int a, int x) const {  // a on x's bound-parent chain (or a == x)
        while (x >= 0 && x != a) x = bp[x];
        return x == a;
    }
    // deepest bound ancestor of d with position <= t (tightest bound known at t)
    int astar(int d, int t) const {
        for (int a = bp[d]; a >= 0; a = bp[a])
            if (a <= t) return a;
        return -1;
    }
    int j0(int d) const {
        for (int j = 0; j < d; ++j)
            if (black[d][j]) return j;
        return -1;
    }
    // DAG class of N(e_owner)[<e_bound]: 2 whole out-list, 1 inside it, 0 no
    int dag_class(int owner, int bound) const {
        if (bound < 0) return 0;
        if (bound == owner) return 2;
        return is_anc_or_self(owner, bound) ? 1 : 0;
    }

    // What holds T_{d,t}: a scratch buffer, or a view of one list.
    struct Src {
        int buf = -1;
        int pos = -1, bound = -1;
    };

    bool compile(GzProg& out) {
        memset(&prog, 0, sizeof(prog));
        prog.k = k;
        prog.unit_dag = (k >= 2 && bp[1] == 0) ? 1 : 0;
        for (int d = 0; d < GZ_MAX_K; ++d) {
            prog.cand_buf[d] = -1;
            prog.cand_pos[d] = -1;
            prog.cand_bound[d] = -1;
        }
        // T_{d,t} for every d > t: key -> source at level t
        std::vector<std::vector<Src>> T(k, std::vector<Src>(k));
        for (int t = 0; t <= k - 2; ++t) {
            if (t >= 2) set_cands(t, T[t][t - 1]);
            prog.level_begin[t] = (int8_t)prog.nops;
            std::map<std::string, Src> level_keys;
            for (int d = t + 1; d < k; ++d) {
                const int jz = j0(d);
                if (jz < 0) return false;  // invalid schedule
                if (jz > t) continue;
                const int a = astar(d, t);
                const bool last = (d == k - 1) && (t == k - 2);
                // key: black / red membership of positions <= t, plus the bound
                std::string key;
                for (int j = 0; j <= t; ++j) key += black[d][j] ? 'B' : 'R';
                key += ':' + std::to_string(a);
                if (!last) {
                    auto it = level_keys.find(key);
                    if (it != level_keys.end()) {
                        T[d][t] = it->second;
                        continue;
                    }
                }
                Src src;
                if (jz == t) {
                    std::vector<int> reds;
                    for (int j = 0; j < t; ++j)
                        if (!black[d][j]) reds.push_back(j);
                    if (reds.empty() && !last) {
                        src.pos = t;  // a view of N(e_t)[<e_a]
                        src.bound = a;
                    } else if (!emit(t, -1, t, a, reds, std::vector<int>(reds.size(), 1), last, d, src))
                        return false;
                } else {
                    const Src& prev = T[d][t - 1];
                    std::vector<int> rp{t};
                    std::vector<int> rs{black[d][t] ? 0 : 1};
                    if (prev.buf >= 0) {
                        if (!emit(t, prev.buf, -1, a, rp, rs, last, d, src)) return false;
                    } else {
                        if (!emit(t, -1, prev.pos, a, rp, rs, last, d, src)) return false;
                    }
                }
                T[d][t] = src;
                if (!last) level_keys[key] = src;
            }
            prog.level_end[t] = (int8_t)prog.nops;
        }
        // shape of loop k-2's single count operation (see the kernel's flattened last loop)
        prog.flat = 0;
        if (k >= 4 && prog.level_end[k - 2] - prog.level_begin[k - 2] == 1) {
            const GzOp& op = prog.ops[prog.level_begin[k - 2]];
            if (op.dst < 0) {
                if (op.left_buf < 0 && op.left_pos == k - 2) {
                    bool fixed = true;
                    for (int r = 0; r < op.nright; ++r) fixed = fixed && op.right_pos[r] < k - 2;
                    if (fixed) prog.flat = 2;
                } else if (op.nright == 1 && op.right_pos[0] == k - 2) {
                    prog.flat = 1;
                }
            }
        }
        out = prog;
        return true;
    }

    // Candidates of loop d (2 <= d <= k-2) are T_{d,d-1}, minus the vertices of
    // red predecessors (already matched vertices are skipped).
    void set_cands(int d, const Src& s) {
        prog.cand_buf[d] = (int8_t)s.buf;
        if (s.buf < 0) {
            prog.cand_pos[d] = (int8_t)s.pos;
            prog.cand_bound[d] = (int8_t)s.bound;
            prog.cand_dag[d] = (int8_t)dag_class(s.pos, s.bound);
        }
        uint8_t ex = 0;
        for (int j = 0; j < d; ++j)
            if (!black[d][j]) ex |= (uint8_t)(1u << j);
        prog.cand_excl[d] = ex;
    }

    // left: buffer lb, or (lb < 0) the list of position lpos, truncated at e_a.
    bool emit(int t, int lb, int lpos, int a, const std::vector<int>& rpos,
              const std::vector<int>& rsub, bool last, int d, Src& src) {
        if (prog.nops >= GZ_MAXOPS || (int)rpos.size() > GZ_MAXRIGHT) {
            set_error("plan: program too large");
            return false;
        }
        GzOp& op = prog.ops[prog.nops++];
        memset(&op, 0, sizeof(op));
        op.level = (int8_t)t;
        op.left_buf = (int8_t)lb;
        op.left_pos = (int8_t)lpos;
        op.bound_pos = (int8_t)a;
        op.nright = (int8_t)rpos.size();
        for (size_t i = 0; i < rpos.size(); ++i) {
            op.right_pos[i] = (int8_t)rpos[i];
            op.right_sub[i] = (int8_t)rsub[i];
            op.right_dag[i] = (int8_t)dag_class(rpos[i], a);
        }
        if (lb < 0) op.left_dag = (int8_t)dag_class(lpos, a);
        // left[<e_t] is a prefix of loop t's candidate list ending just before e_t
        if (a == t && t >= 1) {
            if (t == 1) {
                // loop-1 candidates: N(e_0)[<e_{bp[1]}] from the work unit
                if (lb < 0 && lpos == 0) op.left_iter = 1;
            } else if (lb >= 0 && prog.cand_buf[t] == lb) {
                op.left_iter = 1;
            } else if (lb < 0 && prog.cand_buf[t] < 0 && prog.cand_pos[t] == lpos) {
                op.left_iter = 1;
            }
        }
        if (op.left_iter && lb < 0) {
            // the prefix lives in whatever list loop t iterates (out-list or full)
            op.left_dag = (int8_t)(t == 1 ? prog.unit_dag : prog.cand_dag[t]);
        }
        if (last) {
            op.dst = -1;
            uint8_t ex = 0;
            for (int j = 0; j < d; ++j)
                if (!black[d][j]) ex |= (uint8_t)(1u << j);
            op.excl_mask = ex;
            return true;
        }
        if (prog.nbuf >= GZ_MAXBUF) {
            set_error("plan: too many scratch buffers");
            return false;
        }
        const int b = prog.nbuf++;
        op.dst = (int8_t)b;
        // contents lie in an out-list when the bound is e_j or below it for a
        // black j <= t (T is a subset of N(e_j))
        int dag = 0;
        if (a >= 0)
            for (int j = 0; j <= t; ++j)
                if (black[d][j] && is_anc_or_self(j, a)) dag = 1;
        prog.buf_dag[b] = (int8_t)dag;
        src.buf = b;
        return true;
    }
};

}  // namespace

// Shared by gz_plan_create*.
gz_status make_plan(int k, const uint8_t* adj, const int32_t* forced_order, gz_plan** out) {
    if (!out) {
        set_error("plan: out is NULL");
        return GZ_EINVAL;
    }
    *out = nullptr;
    Pattern p;
    if (!load_pattern(k, adj, p)) return GZ_EINVAL;
    std::vector<Perm> aut = automorphisms(p);
    int32_t order[GZ_MAX_K], bp[GZ_MAX_K];
    double cost = 0.0;
    if (forced_order) {
        if (!valid_schedule(p, forced_order)) {
            set_error("plan: order is not a valid schedule (a vertex has no earlier neighbour)");
            return GZ_EINVAL;
        }
        memcpy(order, forced_order, sizeof(int32_t) * k);
        restrictions(p, aut, order, bp);
        cost = model_cost(p, order, bp);
    } else {
        std::vector<std::vector<int>> scheds;
        std::vector<int> cur;
        explore(p, cur, aut, 0u, scheds);
        double best = 0.0;
        int besti = -1;
        for (size_t i = 0; i < scheds.size(); ++i) {
            int32_t o[GZ_MAX_K], b[GZ_MAX_K];
            for (int j = 0; j < k; ++j) o[j] = scheds[i][j];
            restrictions(p, aut, o, b);
            double c = model_cost(p, o, b);
            if (besti < 0 || c < best * (1.0 - 1e-12)) {
                best = c;
                besti = (int)i;
            }
        }
        for (int j = 0; j < k; ++j) order[j] = scheds[besti][j];
        restrictions(p, aut, order, bp);
        cost = best;
    }
    Compiler c;
    c.k = k;
    for (int d = 0; d < k; ++d)
        for (int j = 0; j < k; ++j) c.black[d][j] = p.a[order[d]][order[j]];
    for (int i = 0; i < k; ++i) c.bp[i] = bp[i];
    gz_plan* pl = new (std::nothrow) gz_plan;
    if (!pl) {
        set_error("plan: out of host memory");
        return GZ_ENOMEM;
    }
    memset(pl, 0, sizeof(*pl));
    pl->k = k;
    for (int i = 0; i < k * k; ++i) pl->adj[i] = adj[i] ? 1 : 0;
    memcpy(pl->order, order, sizeof(int32_t) * k);
    memcpy(pl->bp, bp, sizeof(int32_t) * k);
    pl->aut_size = aut.size();
    pl->est_cost = cost;
    uint64_t h = 1469598103934665603ull;  // FNV-1a over k, adjacency and schedule
    auto mix = [&h](uint64_t x) { h = (h ^ x) * 1099511628211ull; };
    mix((uint64_t)k);
    for (int i = 0; i < k * k; ++i) mix(pl->adj[i]);
    for (int i = 0; i < k; ++i) mix((uint64_t)(uint32_t)pl->order[i]);
    pl->hash = h;
    if (!c.compile(pl->prog)) {
        delete pl;
        return GZ_EINVAL;
    }
    *out = pl;
    return GZ_OK;
}

gz_status list_schedules(int k, const uint8_t* adj, int32_t* orders, int cap, int* count) {
    Pattern p;
    if (!load_pattern(k, adj, p)) return GZ_EINVAL;
    std::vector<Perm> aut = automorphisms(p);
    std::vector<std::vector<int>> scheds;
    std::vector<int> cur;
    explore(p, cur, aut, 0u, scheds);
    if (count) *count = (int)scheds.size();
    for (int i = 0; i < (int)scheds.size() && i < cap && orders; ++i)
        for (int j = 0; j < k; ++j) orders[i * k + j] = scheds[i][j];
    return GZ_OK;
}

}  // namespace gz

// ------------------------------------------------------------ merged programs

namespace gz {

namespace {

// Key of a level-1 operation that writes a buffer: every field except the
// destination, with the left buffer in the merged numbering, and the capacity
// class of the destination.
struct OpKey {
    int8_t v[8 + 3 * GZ_MAXRIGHT + 2];
    bool operator<(const OpKey& o) const { return memcmp(v, o.v, sizeof(v)) < 0; }
};

OpKey op_key(const GzOp& op, int left_merged, int dst_dag) {
    OpKey k;
    memset(&k, 0, sizeof(k));
    int i = 0;
    k.v[i++] = op.level;
    k.v[i++] = (int8_t)left_merged;
    k.v[i++] = op.left_pos;
    k.v[i++] = op.left_dag;
    k.v[i++] = op.left_iter;
    k.v[i++] = op.nright;
    k.v[i++] = op.bound_pos;
    k.v[i++] = (int8_t)op.excl_mask;
    for (int r = 0; r < GZ_MAXRIGHT; ++r) {
        k.v[i++] = r < op.nright ? op.right_pos[r] : 0;
        k.v[i++] = r < op.nright ? op.right_sub[r] : 0;
        k.v[i++] = r < op.nright ? op.right_dag[r] : 0;
    }
    k.v[i++] = (int8_t)dst_dag;
    return k;
}

// One group under construction.
struct MergeState {
    GzMerged m;
    std::map<OpKey, int> shared;  // key -> merged buffer
};

// Tries to add plan p to the group: its level-1 buffer-writing operations are
// matched against the group's or added to them, and its program is rewritten
// without them. Returns false (the group unchanged) when the merged program
// would outgrow the kernel's operation or buffer limits.
bool add_to_group(MergeState& st, const gz_plan* p, int caller_index) {
    const GzProg& src = p->prog;
    MergeState trial = st;  // committed only on success
    GzProg& sh = trial.m.shared;
    std::vector<int> map(src.nbuf, -1);  // plan buffer -> shared buffer
    for (int i = src.level_begin[1]; i < src.level_end[1]; ++i) {
        const GzOp& op = src.ops[i];
        if (op.dst < 0) continue;
        const int left = op.left_buf >= 0 ? map[op.left_buf] : -1;
        if (op.left_buf >= 0 && left < 0) return false;  // reads a buffer no shared op writes
        const OpKey key = op_key(op, left, src.buf_dag[op.dst]);
        auto it = trial.shared.find(key);
        if (it != trial.shared.end()) {
            map[op.dst] = it->second;
            continue;
        }
        if (sh.nops >= GZ_MAXOPS || sh.nbuf >= GZ_MAXBUF) return false;
        const int b = sh.nbuf++;
        sh.buf_dag[b] = src.buf_dag[op.dst];
        GzOp m = op;
        m.dst = (int8_t)b;
        m.left_buf = (int8_t)left;
        sh.ops[sh.nops++] = m;
        trial.shared[key] = b;
        map[op.dst] = b;
    }
    // the plan's own buffers keep a provisional numbering, -(2 + own index),
    // until the group is complete (then they follow the shared ones)
    GzProg q;
    memset(&q, 0, sizeof(q));
    q.k = src.k;
    q.unit_dag = src.unit_dag;
    q.flat = src.flat;
    int own = 0;
    std::vector<int> own_index(src.nbuf, -1);
    for (int b = 0; b < src.nbuf; ++b)
        if (map[b] < 0) own_index[b] = own++;
    auto remap = [&](int b) -> int { return b < 0 ? b : (map[b] >= 0 ? map[b] : -(2 + own_index[b])); };
    for (int t = 0; t < GZ_MAX_K; ++t) {
        q.level_begin[t] = (int8_t)q.nops;
        if (t < src.k)
            for (int i = src.level_begin[t]; i < src.level_end[t]; ++i) {
                const GzOp& op = src.ops[i];
                if (t == 1 && op.dst >= 0) continue;  // computed by the shared operations
                GzOp o = op;
                o.dst = (int8_t)remap(op.dst);
                o.left_buf = (int8_t)remap(op.left_buf);
                q.ops[q.nops++] = o;
            }
        q.level_end[t] = (int8_t)q.nops;
    }
    for (int d = 0; d < GZ_MAX_K; ++d) {
        q.cand_buf[d] = (int8_t)remap(src.cand_buf[d]);
        q.cand_pos[d] = src.cand_pos[d];
        q.cand_bound[d] = src.cand_bound[d];
        q.cand_dag[d] = src.cand_dag[d];
        q.cand_excl[d] = src.cand_excl[d];
    }
    q.nbuf = own;  // own buffers only, until the group is finished
    for (int b = 0; b < src.nbuf; ++b)
        if (own_index[b] >= 0) q.buf_dag[own_index[b]] = src.buf_dag[b];
    int own_max = own;
    for (const GzProg& o : trial.m.progs) own_max = std::max(own_max, o.nbuf);
    if (sh.nbuf + own_max > GZ_MAXBUF) return false;
    trial.m.progs.push_back(q);
    trial.m.plans.push_back(p);
    trial.m.plan_index.push_back(caller_index);
    st = std::move(trial);
    return true;
}

// Final numbering: each plan's own buffers after the group's shared ones.
void finish_group(GzMerged& m) {
    const int ns = m.shared.nbuf;
    m.shared.k = 2;
    m.shared.unit_dag = m.unit_dag;
    for (int t = 0; t < GZ_MAX_K; ++t) {
        m.shared.level_begin[t] = t <= 1 ? 0 : (int8_t)m.shared.nops;
        m.shared.level_end[t] = t == 1 ? (int8_t)m.shared.nops : m.shared.level_begin[t];
    }
    for (GzProg& q : m.progs) {
        auto fin = [&](int8_t b) -> int8_t { return b <= -2 ? (int8_t)(ns + (-b - 2)) : b; };
        for (int i = 0; i < q.nops; ++i) {
            q.ops[i].dst = fin(q.ops[i].dst);
            q.ops[i].left_buf = fin(q.ops[i].left_buf);
        }
        for (int d = 0; d < GZ_MAX_K; ++d) q.cand_buf[d] = fin(q.cand_buf[d]);
        int8_t dag[GZ_MAXBUF] = {};
        for (int b = 0; b < ns; ++b) dag[b] = m.shared.buf_dag[b];
        for (int b = 0; b < q.nbuf; ++b) dag[ns + b] = q.buf_dag[b];
        q.nbuf += ns;
        memcpy(q.buf_dag, dag, sizeof(dag));
    }
}

}  // namespace

gz_status merge_plans(const gz_plan* const* plans, const int* idx, int n, std::vector<GzMerged>& out) {
    out.clear();
    for (int dag = 0; dag <= 1; ++dag) {
        std::vector<MergeState> groups;
        for (int i = 0; i < n; ++i) {
            const gz_plan* p = plans[idx[i]];
            if (p->prog.unit_dag != dag) continue;
            bool placed = false;
            for (MergeState& g : groups)
                if (add_to_group(g, p, idx[i])) { placed = true; break; }
            if (!placed) {
                groups.emplace_back();
                memset(&groups.back().m.shared, 0, sizeof(GzProg));
                groups.back().m.unit_dag = dag;
                if (!add_to_group(groups.back(), p, idx[i])) {
                    set_error("merge: a plan does not fit the merged program's limits");
                    return GZ_EOVERFLOW;
                }
            }
        }
        for (MergeState& g : groups) {
            finish_group(g.m);
            out.push_back(std::move(g.m));
        }
    }
    return GZ_OK;
}

}  // namespace gz
