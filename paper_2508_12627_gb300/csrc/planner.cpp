// Planner: partitions, Moebius coefficients, quotient factor multigraphs,
// elimination orders and the lowered program of device operations.
//
// Paper (arXiv 2508.12627) passages implemented here:
//   - partitions of [m] (Section 2.3, Definition "Partition"), as restricted
//     growth strings in lexicographic order;
//   - mu_pi = (-1)^(m-|pi|) prod_C (|C|-1)! (Section 3.3, Lemma "Decomposition of
//     U-Statistic into V-Statistics");
//   - the induced notation A_pi (Algorithm 3): every index replaced by its block,
//     kept here as a factor multigraph on the blocks (quotient graph, Definition
//     "Quotient Graph", with parallel factors kept as Hadamard products and
//     intra-block pairwise factors kept as their diagonal);
//   - the sparsification filter Pi_m^A (Lemma "sparsification_trick" and
//     equation "quotient_set");
//   - Einsum by summing out one index at a time along an elimination order
//     (Section 3.2, Proposition "complexity_einsum"; Appendix D): eliminating a
//     vertex with s live neighbours costs 2 n^(s+1) and yields a factor on those
//     neighbours;
//   - treewidth (Definitions "Vertex Elimination" and "Treewidth"), computed
//     exactly by dynamic programming over vertex subsets.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <tuple>
#include <vector>

#include "ustat_internal.h"

namespace ustat {

const char *op_name(int k) {
    static const char *names[] = {"kbuild", "loadmat", "unary",  "loadvec", "diag",
                                  "vmul",   "hadamard", "gemv",  "vsum",    "gemm",
                                  "gemm_red", "freduce", "gemm3", "split",  "prep", "mhb",
                                  "vdot"};
    return (k >= 0 && k < OP_COUNT) ? names[k] : "?";
}

namespace {

bool kind_pair(int k) {
    return k == USTAT_RBF || k == USTAT_LINEAR || k == USTAT_MATRIX || k == USTAT_DIST || k == USTAT_LOWRANK ||
           k == USTAT_COMPLEMENT || k == USTAT_GRAM;
}
bool kind_unary(int k) { return k == USTAT_TANH_DOT || k == USTAT_VECTOR; }
bool kind_symmetric(int k) { return k == USTAT_RBF || k == USTAT_LINEAR || k == USTAT_DIST || k == USTAT_GRAM; }
bool kind_unit_diag(int k) { return k == USTAT_RBF; }

int popc(uint32_t x) { return __builtin_popcount(x); }

void enum_partitions(int m, std::vector<std::vector<int>> &out) {
    std::vector<int> a(m, 0);
    // iterative restricted-growth-string enumeration in lexicographic order
    std::function<void(int, int)> rec = [&](int i, int top) {
        if (i == m) {
            out.push_back(a);
            return;
        }
        for (int b = 0; b <= top + 1; ++b) {
            a[i] = b;
            rec(i + 1, std::max(top, b));
        }
    };
    if (m == 0) return;
    a[0] = 0;
    rec(1, 0);
}

int mu_of(const std::vector<int> &rgs) {
    int k = *std::max_element(rgs.begin(), rgs.end()) + 1;
    std::vector<int> size(k, 0);
    for (int b : rgs) size[b]++;
    long long v = 1;
    for (int s : size)
        for (int t = 2; t < s; ++t) v *= t;
    int sign = ((int)rgs.size() - k) % 2 ? -1 : 1;
    return (int)(sign * v);
}

uint32_t component(int v, uint32_t alive, const uint32_t *adj) {
    uint32_t seen = 1u << v, frontier = 1u << v;
    while (frontier) {
        int u = __builtin_ctz(frontier);
        frontier &= frontier - 1;
        uint32_t nb = adj[u] & alive & ~seen;
        seen |= nb;
        frontier |= nb;
    }
    return seen;
}

// Cost of an elimination order as counts of steps per power of n (index p means
// n^(p+1)); compared from the highest power down, then by stored intermediates.
struct Cost {
    int c[5] = {0, 0, 0, 0, 0};
    int stores = 0;
    bool ok = true;
    bool operator<(const Cost &o) const {
        if (ok != o.ok) return ok;
        for (int p = 4; p >= 0; --p)
            if (c[p] != o.c[p]) return c[p] < o.c[p];
        return stores < o.stores;
    }
};

// Structural simulation.  A step with s neighbours is executable when s <= 2, or
// when s == 3 and the step ends its connected component (the n^3 intermediate is
// then consumed inside the same kernel).  A step that ends its component
// ("terminal") eliminates the whole component: the remaining 1..3 vertices are
// summed in the fused reduction.
Cost simulate(int k, const uint32_t *adj0, const int *order) {
    uint32_t adj[32];
    std::memcpy(adj, adj0, sizeof(uint32_t) * k);
    uint32_t alive = (k == 32) ? 0xffffffffu : ((1u << k) - 1);
    Cost c;
    for (int t = 0; t < k; ++t) {
        int v = order[t];
        if (!((alive >> v) & 1)) continue;
        uint32_t nb = adj[v] & alive & ~(1u << v);
        int s = popc(nb);
        uint32_t comp = component(v, alive, adj);
        bool terminal = popc(comp) == s + 1;
        if (s >= 4 || (s == 3 && !terminal)) {
            c.ok = false;
            return c;
        }
        c.c[s]++;
        if (s == 2 && !terminal) c.stores++;
        if (terminal) {
            alive &= ~comp;
        } else {
            alive &= ~(1u << v);
            for (uint32_t r = nb; r; r &= r - 1) {
                int w = __builtin_ctz(r);
                adj[w] |= nb & ~(1u << w);
            }
        }
    }
    return c;
}

std::vector<int> exhaustive_order(int k, const uint32_t *adj, Cost *best_cost) {
    std::vector<int> perm(k), best;
    for (int i = 0; i < k; ++i) perm[i] = i;
    Cost bc;
    bc.ok = false;
    do {
        Cost c = simulate(k, adj, perm.data());
        if (best.empty() || c < bc) {
            bc = c;
            best = perm;
        }
    } while (std::next_permutation(perm.begin(), perm.end()));
    *best_cost = bc;
    return best;
}

std::vector<int> minfill_order(int k, const uint32_t *adj0) {
    uint32_t adj[32];
    std::memcpy(adj, adj0, sizeof(uint32_t) * k);
    uint32_t alive = (1u << k) - 1;
    std::vector<int> order;
    while (alive) {
        int best = -1, bf = 1 << 30, bd = 1 << 30;
        for (uint32_t r = alive; r; r &= r - 1) {
            int v = __builtin_ctz(r);
            uint32_t nb = adj[v] & alive & ~(1u << v);
            int fill = 0;
            for (uint32_t q = nb; q; q &= q - 1) {
                int w = __builtin_ctz(q);
                fill += popc(nb & ~adj[w] & ~(1u << w));
            }
            fill /= 2;
            int deg = popc(nb);
            if (fill < bf || (fill == bf && deg < bd)) {
                best = v;
                bf = fill;
                bd = deg;
            }
        }
        uint32_t nb = adj[best] & alive & ~(1u << best);
        for (uint32_t r = nb; r; r &= r - 1) {
            int w = __builtin_ctz(r);
            adj[w] |= nb & ~(1u << w);
        }
        alive &= ~(1u << best);
        order.push_back(best);
    }
    return order;
}

// ---------------------------------------------------------------- lowering

struct Lowerer {
    Plan &P;
    std::map<std::vector<long long>, int> memo;   // op signature -> out slot
    explicit Lowerer(Plan &p) : P(p) {}

    int new_slot(int kind, int sym = 0) {
        Slot s;
        s.kind = kind;
        s.symmetric = sym;
        P.slots.push_back(s);
        return (int)P.slots.size() - 1;
    }
    bool sym(int mat) const { return mat >= 0 && P.slots[mat].symmetric; }
    Term canon(Term t) const {
        if (t.mat >= 0 && sym(t.mat)) t.trans = 0;
        return t;
    }
    Term flip(Term t) const {
        if (t.mat < 0) return t;
        t.trans ^= 1;
        return canon(t);
    }

    static void put_term(std::vector<long long> &k, Term t) {
        k.push_back(t.mat);
        k.push_back(t.trans);
    }

    std::vector<long long> key_of(const Op &o) const {
        std::vector<long long> k = {o.kind, o.factor, o.nt};
        for (int i = 0; i < o.nt; ++i) put_term(k, o.t[i]);
        k.push_back(o.u);
        k.push_back(o.a);
        k.push_back(o.b);
        put_term(k, o.A);
        put_term(k, o.B);
        put_term(k, o.W);
        put_term(k, o.Ab);
        put_term(k, o.Wbc);
        put_term(k, o.Wbd);
        k.push_back(o.ub);
        return k;
    }

    int out_kind(int opk) const {
        switch (opk) {
            case OP_KBUILD: case OP_LOADMAT: case OP_HADAMARD: case OP_GEMM: return S_MAT;
            case OP_UNARY: case OP_LOADVEC: case OP_DIAG: case OP_VMUL: case OP_GEMV: return S_VEC;
            case OP_SPLIT: return S_SLICES;
            case OP_PREP: return S_PREP;
            default: return S_SCAL;
        }
    }

    int emit(Op o, int symmetric_out = 0) {
        auto key = key_of(o);
        if (P.cse) {
            auto it = memo.find(key);
            if (it != memo.end()) return it->second;
        }
        o.out = new_slot(out_kind(o.kind), symmetric_out);
        P.ops.push_back(o);
        if (!memo.count(key)) {
            memo[key] = o.out;
            if (trial_log) trial_log->push_back(key);
        }
        return o.out;
    }

    // Trial lowering: everything emitted after begin_trial() is undone by rollback().
    std::vector<std::vector<long long>> *trial_log = nullptr;
    size_t trial_ops = 0, trial_slots = 0;
    std::vector<std::vector<long long>> log_store;
    void begin_trial() {
        trial_ops = P.ops.size();
        trial_slots = P.slots.size();
        log_store.clear();
        trial_log = &log_store;
    }
    void rollback() {
        P.ops.resize(trial_ops);
        P.slots.resize(trial_slots);
        for (auto &k : log_store) memo.erase(k);
        log_store.clear();
        trial_log = nullptr;
    }

    int vmul(std::vector<int> v) {
        std::sort(v.begin(), v.end());
        if (v.empty()) return -1;
        int acc = v[0];
        for (size_t i = 1; i < v.size(); ++i) {
            Op o;
            o.kind = OP_VMUL;
            o.u = std::min(acc, v[i]);
            o.a = std::max(acc, v[i]);
            acc = emit(o);
        }
        return acc;
    }

    Term hadamard(std::vector<Term> ts) {
        for (auto &t : ts) t = canon(t);
        std::sort(ts.begin(), ts.end());
        if (ts.empty()) return Term{};
        if (ts.size() == 1) return ts[0];
        while (ts.size() > 1) {
            Op o;
            o.kind = OP_HADAMARD;
            int take = std::min((int)ts.size(), kMaxTerms);
            bool all_sym = true;
            for (int i = 0; i < take; ++i) {
                o.t[i] = ts[i];
                all_sym = all_sym && sym(ts[i].mat);
            }
            o.nt = take;
            o.coef = take - 1;
            o.npow = 2;
            int out = emit(o, all_sym ? 1 : 0);
            std::vector<Term> rest(ts.begin() + take, ts.end());
            rest.push_back(Term{out, 0});
            std::sort(rest.begin(), rest.end());
            ts = rest;
        }
        return ts[0];
    }

    // reduce a term list to at most kMaxTerms - reserve entries
    std::vector<Term> fit(std::vector<Term> ts, int reserve = 0) {
        for (auto &t : ts) t = canon(t);
        std::sort(ts.begin(), ts.end());
        int cap = kMaxTerms - reserve;
        if ((int)ts.size() <= cap) return ts;
        std::vector<Term> head(ts.begin(), ts.begin() + (ts.size() - cap + 1));
        std::vector<Term> out(ts.begin() + (ts.size() - cap + 1), ts.end());
        out.push_back(hadamard(head));
        std::sort(out.begin(), out.end());
        return out;
    }
};

struct QState {
    int k = 0;
    std::vector<std::vector<int>> vecs;
    std::map<std::pair<int, int>, std::vector<Term>> E;   // key p < q; terms value(i_p, i_q)
    uint32_t adj[32] = {0};
};

}  // namespace

int exact_treewidth(int k, const std::vector<uint32_t> &adj) {
    if (k <= 1) return 0;
    // TW(S) = min_{v in S} max(TW(S \ v), |Q(S \ v, v)|), Q(S, v) = vertices outside
    // S + v reachable from v through S.
    std::vector<int> tw(1u << k, 0);
    for (uint32_t S = 1; S < (1u << k); ++S) {
        int best = 1 << 20;
        for (uint32_t r = S; r; r &= r - 1) {
            int v = __builtin_ctz(r);
            uint32_t Sv = S & ~(1u << v);
            uint32_t seen = 1u << v, fr = 1u << v, q = 0;
            while (fr) {
                int u = __builtin_ctz(fr);
                fr &= fr - 1;
                uint32_t nb = adj[u] & ~seen;
                seen |= nb;
                q |= nb & ~Sv;
                fr |= nb & Sv;
            }
            q &= ~(1u << v);
            int val = std::max(tw[Sv], popc(q));
            best = std::min(best, val);
        }
        tw[S] = best;
    }
    return tw[(1u << k) - 1];
}

// Features of the program one elimination sequence lowers to, in isolation
// (no sharing with other partitions): log2 n (and its square); counts of each
// step kind, of the n^3 products of an operand with itself (symmetric: half
// the tiles), of all steps and of stored n x n intermediates; the Hadamard
// terms read; the flop count of the whole sequence and of its n^3 and n^4
// steps (log2); the quotient's size.  Scaled to O(1).
void order_features(const std::vector<Op> &ops, size_t first, int k, int n_edges, int n_vecs, int64_t n,
                    float *f) {
    for (int i = 0; i < kRankFeatures; ++i) f[i] = 0.f;
    const double dn = (double)(n < 2 ? 2 : n);
    double fl = 0.0, fl3 = 0.0, fl4 = 0.0;
    int cnt[OP_COUNT + 1] = {0};
    int terms = 0, sym = 0, stored = 0;
    for (size_t i = first; i < ops.size(); ++i) {
        const Op &o = ops[i];
        cnt[o.kind]++;
        if ((o.kind == OP_GEMM || o.kind == OP_GEMM_RED) && o.A == o.B && o.u < 0) ++sym;
        if (o.kind == OP_GEMM || o.kind == OP_HADAMARD) ++stored;
        const double c = o.coef * std::pow(dn, o.npow);
        fl += c;
        if (o.npow == 3) fl3 += c;
        if (o.npow == 4) fl4 += c;
        if (o.kind == OP_HADAMARD || o.kind == OP_GEMV || o.kind == OP_FREDUCE) terms += o.nt;
    }
    f[0] = (float)(std::log2(dn) / 12.0);
    f[1] = cnt[OP_GEMM] / 4.f;
    f[2] = cnt[OP_GEMM_RED] / 4.f;
    f[3] = cnt[OP_GEMM3] / 4.f;
    f[4] = cnt[OP_GEMV] / 4.f;
    f[5] = cnt[OP_FREDUCE] / 4.f;
    f[6] = cnt[OP_HADAMARD] / 4.f;
    f[7] = cnt[OP_VSUM] / 4.f;
    f[8] = cnt[OP_VMUL] / 8.f;
    f[9] = terms / 16.f;
    f[10] = (float)(std::log2(1.0 + fl) / 48.0);
    f[11] = (float)(std::log2(1.0 + fl3) / 48.0);
    f[12] = (float)(std::log2(1.0 + fl4) / 48.0);
    f[13] = k / 8.f;
    f[14] = n_edges / 16.f;
    f[15] = n_vecs / 8.f;
    f[16] = sym / 4.f;
    f[17] = (float)(ops.size() - first) / 16.f;
    f[18] = stored / 8.f;
    f[19] = f[0] * f[0];
}

int build_plan(const ustat_graph *g, const ustat_options *o, Plan *plan, const PlanRequest *req) {
    if (!g || !o || !plan) return USTAT_ERR_INVALID_ARG;
    const int m = g->m;
    if (m < 1) return USTAT_ERR_INVALID_ARG;
    if (m > kMaxM) return USTAT_ERR_UNSUPPORTED;
    if (g->n_factors < 1 || !g->factor_kind) return USTAT_ERR_INVALID_ARG;
    if (g->n_edges < 0 || g->n_unary < 0) return USTAT_ERR_INVALID_ARG;
    if (g->n_edges > 0 && (!g->edge_src || !g->edge_dst || !g->edge_factor)) return USTAT_ERR_INVALID_ARG;
    if (g->n_unary > 0 && (!g->unary_vertex || !g->unary_factor)) return USTAT_ERR_INVALID_ARG;
    if (o->precision < USTAT_FP64 || o->precision > USTAT_BF16X5) return USTAT_ERR_INVALID_ARG;
    if (o->planner != USTAT_PLAN_EXHAUSTIVE && o->planner != USTAT_PLAN_MINFILL) return USTAT_ERR_INVALID_ARG;
    Plan &P = *plan;
    P = Plan();
    P.m = m;
    P.precision = o->precision;
    P.sparsify = o->sparsify ? 1 : 0;
    P.planner = o->planner;
    P.cse = o->cse ? 1 : 0;
    P.factor_kind.assign(g->factor_kind, g->factor_kind + g->n_factors);
    // split modes above n = 1024: 128 x 128 tiles with 64-byte k-blocks and a
    // deeper pipeline by default (measured on the n = 16384 products: 0.99 / 1.04
    // of the bf16x3 / bf16x4 ceilings against 0.92 / 0.67 with 128-byte k-blocks;
    // equal on the symmetric 4096 product); up to n = 1024 (short k loops, where
    // 128-byte k-blocks measured 5 % faster on the batched bf16x3 s = 3 steps)
    // 128-byte k-blocks, except in the float64-storage modes (bf16x5 has only the
    // 64-byte form; the bf16x4 s = 3 steps at n = 1024 measured 292 ms per K4 +
    // cycle evaluation with 128 x 128 tiles against 400 ms with 128 x 64 tiles)
    // the CUDA-core RBF build, when chosen, on 64 x 64 tiles above n = 1024
    // (measured at n = 4096: 75 us against 82 us for 128 x 128 tiles)
    for (int c = 0; c < 4; ++c) {
        int v = 0;
        if (is_split_mode(P.precision) && (c > 0 || wide_storage(P.precision))) v |= 2 << 2;
        if (!wide_storage(P.precision) && c > 0) v |= 1 << 4;
        P.tc_variant[c] = v;
    }
    for (int f = 0; f < g->n_factors; ++f)
        if (P.factor_kind[f] < USTAT_RBF || P.factor_kind[f] > USTAT_GRAM) return USTAT_ERR_INVALID_ARG;
    std::vector<int> covered(m, 0);
    for (int e = 0; e < g->n_edges; ++e) {
        int a = g->edge_src[e], b = g->edge_dst[e], f = g->edge_factor[e];
        if (a < 0 || a >= m || b < 0 || b >= m || f < 0 || f >= g->n_factors) return USTAT_ERR_INVALID_ARG;
        if (!kind_pair(P.factor_kind[f])) return USTAT_ERR_INVALID_ARG;
        if (a == b) return USTAT_ERR_INVALID_ARG;   // a signature tuple (a, a): not a graph edge
        covered[a] = covered[b] = 1;
    }
    for (int e = 0; e < g->n_unary; ++e) {
        int v = g->unary_vertex[e], f = g->unary_factor[e];
        if (v < 0 || v >= m || f < 0 || f >= g->n_factors) return USTAT_ERR_INVALID_ARG;
        if (!kind_unary(P.factor_kind[f])) return USTAT_ERR_INVALID_ARG;
        covered[v] = 1;
    }
    // Definition "Multiplicative Decomposition": the tuples cover [m]
    for (int v = 0; v < m; ++v)
        if (!covered[v]) return USTAT_ERR_INVALID_ARG;

    Lowerer L(P);
    const bool tc = is_tc_mode(P.precision);

    // base tensors (Algorithm 1): one per factor id, created lazily
    std::vector<int> base(g->n_factors, -1), diag(g->n_factors, -1);
    auto base_of = [&](int f) {
        if (base[f] >= 0) return base[f];
        Op op;
        op.factor = f;
        int k = P.factor_kind[f];
        if (k == USTAT_RBF || k == USTAT_LINEAR) op.kind = OP_KBUILD;
        else if (k == USTAT_MATRIX || k == USTAT_DIST || k == USTAT_LOWRANK || k == USTAT_COMPLEMENT ||
                 k == USTAT_GRAM)
            op.kind = OP_LOADMAT;   // matrices from the caller's data
        else if (k == USTAT_TANH_DOT) op.kind = OP_UNARY;
        else op.kind = OP_LOADVEC;
        op.npow = 2;
        op.coef = 0;
        base[f] = L.emit(op, kind_symmetric(k) ? 1 : 0);
        return base[f];
    };
    auto diag_of = [&](int f) {
        if (diag[f] >= 0) return diag[f];
        Op op;
        op.kind = OP_DIAG;
        op.t[0] = Term{base_of(f), 0};
        op.nt = 1;
        op.factor = f;   // the diagonal is taken from the factor's own data, in float64
        diag[f] = L.emit(op);
        return diag[f];
    };

    std::vector<std::vector<int>> parts;
    enum_partitions(m, parts);
    if (req && req->forced && req->forced->size() != parts.size()) return USTAT_ERR_INVALID_ARG;
    if (req && req->keep && req->keep->size() != parts.size()) return USTAT_ERR_INVALID_ARG;
    if (req && req->collect) req->collect->assign(parts.size(), {});
    std::set<std::tuple<int, int, int, int, int>> products;   // n^3 products in the program
    // partitions are lowered in restricted-growth-string order, or (req->reverse)
    // from the finest down; the plan keeps them in restricted-growth-string order
    std::vector<PartRec> parts_out(parts.size());
    for (size_t step = 0; step < parts.size(); ++step) {
        const size_t pi = (req && req->reverse) ? parts.size() - 1 - step : step;
        const std::vector<int> &rgs = parts[pi];
        PartRec pr;
        for (int i = 0; i < m; ++i) pr.rgs[i] = rgs[i];
        int k = *std::max_element(rgs.begin(), rgs.end()) + 1;
        pr.nblocks = k;
        pr.mu = mu_of(rgs);
        // exact treewidth of the simple quotient graph
        std::vector<uint32_t> qadj(k, 0);
        for (int e = 0; e < g->n_edges; ++e) {
            int p = rgs[g->edge_src[e]], q = rgs[g->edge_dst[e]];
            if (p != q) {
                qadj[p] |= 1u << q;
                qadj[q] |= 1u << p;
            }
        }
        pr.tw = exact_treewidth(k, qadj);
        if (req && ((req->finest_only && k != m) || (req->keep && !(*req->keep)[pi]))) {
            pr.evaluated = 0;
            parts_out[pi] = pr;
            continue;
        }
        // sparsification filter: no block holds both ends of a pairwise factor
        if (P.sparsify) {
            bool surv = true;
            for (int e = 0; e < g->n_edges; ++e)
                if (rgs[g->edge_src[e]] == rgs[g->edge_dst[e]]) surv = false;
            if (!surv) {
                pr.evaluated = 0;
                parts_out[pi] = pr;
                continue;
            }
        }
        // quotient factor multigraph
        QState Q;
        Q.k = k;
        Q.vecs.assign(k, {});
        for (int e = 0; e < g->n_edges; ++e) {
            int a = g->edge_src[e], b = g->edge_dst[e], f = g->edge_factor[e];
            int p = rgs[a], q = rgs[b];
            if (p == q) {
                // intra-block pairwise factor: F(x_i, x_i) (Definition "Restricted
                // V-Statistic"); an RBF factor has F(x, x) = 1 and drops out
                if (!kind_unit_diag(P.factor_kind[f])) Q.vecs[p].push_back(diag_of(f));
                continue;
            }
            Term t{base_of(f), 0};
            if (p > q) {
                std::swap(p, q);
                t = L.flip(t);
            }
            Q.E[{p, q}].push_back(L.canon(t));
            Q.adj[p] |= 1u << q;
            Q.adj[q] |= 1u << p;
        }
        for (int e = 0; e < g->n_unary; ++e) Q.vecs[rgs[g->unary_vertex[e]]].push_back(base_of(g->unary_factor[e]));

        // lower the partition along an order (Q is taken by value)
        auto lower = [&](QState Q, const std::vector<int> &order, PartRec &pr) -> int {
        auto oriented = [&](int p, int q) {
            std::vector<Term> ts;
            if (p < q) {
                auto it = Q.E.find({p, q});
                if (it != Q.E.end()) ts = it->second;
            } else {
                auto it = Q.E.find({q, p});
                if (it != Q.E.end())
                    for (auto t : it->second) ts.push_back(L.flip(t));
            }
            return ts;
        };
        auto add_scal = [&](int s) -> int {
            if (pr.nscal >= kMaxScal) return USTAT_ERR_UNSUPPORTED;
            pr.scal[pr.nscal++] = s;
            return USTAT_OK;
        };
        uint32_t alive = (1u << k) - 1;
        for (int v : order) {
            if (!((alive >> v) & 1)) continue;
            uint32_t nb = Q.adj[v] & alive & ~(1u << v);
            int s = popc(nb);
            uint32_t comp = component(v, alive, Q.adj);
            bool terminal = popc(comp) == s + 1;
            std::vector<int> nbs;
            for (uint32_t r = nb; r; r &= r - 1) nbs.push_back(__builtin_ctz(r));
            int rc = USTAT_OK;
            if (s == 0) {
                int u = L.vmul(Q.vecs[v]);
                if (u < 0) {
                    pr.nfree++;
                } else {
                    Op op;
                    op.kind = OP_VSUM;
                    op.u = u;
                    op.coef = 1;
                    op.npow = 1;
                    rc = add_scal(L.emit(op));
                }
            } else if (s == 1) {
                int w = nbs[0];
                if (terminal) {
                    Op op;
                    op.kind = OP_FREDUCE;
                    auto ts = L.fit(oriented(v, w));
                    for (size_t i = 0; i < ts.size(); ++i) op.t[i] = ts[i];
                    op.nt = (int)ts.size();
                    op.a = L.vmul(Q.vecs[v]);
                    op.b = L.vmul(Q.vecs[w]);
                    op.coef = 2;
                    op.npow = 2;
                    rc = add_scal(L.emit(op));
                } else {
                    Op op;
                    op.kind = OP_GEMV;
                    auto ts = L.fit(oriented(v, w));
                    for (size_t i = 0; i < ts.size(); ++i) op.t[i] = ts[i];
                    op.nt = (int)ts.size();
                    op.u = L.vmul(Q.vecs[v]);
                    op.coef = 2;
                    op.npow = 2;
                    Q.vecs[w].push_back(L.emit(op));
                }
            } else if (s == 2) {
                int w = nbs[0], x = nbs[1];
                Term A = L.hadamard(oriented(v, w));
                Term B = L.hadamard(oriented(v, x));
                int u = L.vmul(Q.vecs[v]);
                if (terminal) {
                    Op op;
                    op.kind = OP_GEMM_RED;
                    op.A = A;
                    op.B = B;
                    op.u = u;
                    op.W = L.hadamard(oriented(w, x));
                    op.a = L.vmul(Q.vecs[w]);
                    op.b = L.vmul(Q.vecs[x]);
                    // canonical operand order: (A,B,W,a,b) ~ (B,A,W^T,b,a)
                    if (B < A) {
                        std::swap(op.A, op.B);
                        op.W = L.flip(op.W);
                        std::swap(op.a, op.b);
                    }
                    op.coef = 2;
                    op.npow = 3;
                    rc = add_scal(L.emit(op));
                } else {
                    Op op;
                    op.kind = OP_GEMM;
                    op.A = A;
                    op.B = B;
                    op.u = u;
                    bool swapped = false;
                    if (B < A) {
                        std::swap(op.A, op.B);
                        swapped = true;
                    }
                    op.coef = 2;
                    op.npow = 3;
                    int out = L.emit(op, (op.A == op.B) ? 1 : 0);
                    Term T{out, swapped ? 1 : 0};
                    T = L.canon(T);   // T(i_w, i_x) with w < x
                    Q.E[{w, x}].push_back(T);
                    Q.adj[w] |= 1u << x;
                    Q.adj[x] |= 1u << w;
                }
            } else if (s == 3) {
                int b = nbs[0], cc = nbs[1], d = nbs[2];
                Op op;
                op.kind = OP_GEMM3;
                op.Ab = L.hadamard(oriented(v, b));
                op.A = L.hadamard(oriented(v, cc));
                op.B = L.hadamard(oriented(v, d));
                op.u = L.vmul(Q.vecs[v]);
                op.Wbc = L.hadamard(oriented(b, cc));
                op.Wbd = L.hadamard(oriented(b, d));
                op.W = L.hadamard(oriented(cc, d));
                op.ub = L.vmul(Q.vecs[b]);
                op.a = L.vmul(Q.vecs[cc]);
                op.b = L.vmul(Q.vecs[d]);
                op.coef = 2;
                op.npow = 4;
                rc = add_scal(L.emit(op));
            } else {
                return USTAT_ERR_TW_TOO_LARGE;
            }
            if (rc != USTAT_OK) return rc;
            if (terminal) {
                alive &= ~comp;
            } else {
                alive &= ~(1u << v);
                for (int w : nbs) Q.adj[w] &= ~(1u << v);
            }
            // edges incident to v are consumed
            for (auto it = Q.E.begin(); it != Q.E.end();) {
                if (it->first.first == v || it->first.second == v) it = Q.E.erase(it);
                else ++it;
            }
        }
        return USTAT_OK;
        };

        // candidates for the learned ranker: every distinct feasible elimination
        // sequence, lowered on trial in isolation (an empty memo: no sharing with
        // other partitions) and described by its features
        if (req && req->collect && (req->collect_part < 0 || req->collect_part == (int)pi)) {
            int n_edges_q = 0, n_vecs_q = 0;
            for (auto &kv : Q.E) n_edges_q += (int)kv.second.size();
            for (auto &v : Q.vecs) n_vecs_q += (int)v.size();
            if (req->feature_order) {
                const std::vector<int> &fo = *req->feature_order;
                if ((int)fo.size() != k) return USTAT_ERR_INVALID_ARG;
                std::vector<int> chk = fo;
                std::sort(chk.begin(), chk.end());
                for (int i = 0; i < k; ++i)
                    if (chk[i] != i) return USTAT_ERR_INVALID_ARG;
                if (!simulate(k, Q.adj, fo.data()).ok) return USTAT_ERR_TW_TOO_LARGE;
                auto saved = L.memo;
                PartRec tr = pr;
                L.memo.clear();
                L.begin_trial();
                const size_t first = P.ops.size();
                int rc = lower(Q, fo, tr);
                Candidate cd;
                cd.order = fo;
                order_features(P.ops, first, k, n_edges_q, n_vecs_q, req->n, cd.feat);
                L.rollback();
                L.memo = saved;
                if (rc != USTAT_OK) return rc;
                (*req->collect)[pi].push_back(cd);
                return USTAT_OK;
            }
            std::vector<int> perm(k);
            for (int i = 0; i < k; ++i) perm[i] = i;
            std::set<std::vector<int>> seen;
            auto saved = L.memo;
            do {
                Cost cc = simulate(k, Q.adj, perm.data());
                if (!cc.ok) continue;
                std::vector<int> eff;
                {
                    uint32_t adj2[32];
                    std::memcpy(adj2, Q.adj, sizeof(uint32_t) * k);
                    uint32_t al = (1u << k) - 1;
                    for (int v : perm) {
                        if (!((al >> v) & 1)) continue;
                        eff.push_back(v);
                        uint32_t nb = adj2[v] & al & ~(1u << v);
                        uint32_t comp = component(v, al, adj2);
                        if (popc(comp) == popc(nb) + 1) {
                            al &= ~comp;
                        } else {
                            al &= ~(1u << v);
                            for (uint32_t r = nb; r; r &= r - 1)
                                adj2[__builtin_ctz(r)] |= nb & ~(1u << __builtin_ctz(r));
                        }
                    }
                }
                if (!seen.insert(eff).second) continue;
                PartRec tr = pr;
                L.memo.clear();
                L.begin_trial();
                const size_t first = P.ops.size();
                int rc = lower(Q, perm, tr);
                Candidate cd;
                cd.order = perm;
                order_features(P.ops, first, k, n_edges_q, n_vecs_q, req->n, cd.feat);
                L.rollback();
                if (rc == USTAT_OK) (*req->collect)[pi].push_back(cd);
            } while (std::next_permutation(perm.begin(), perm.end()));
            L.memo = saved;
            if (req->collect_only && req->collect_part >= 0) return USTAT_OK;
        }

        // elimination order
        std::vector<int> order;
        Cost c;
        if (req && req->forced && !(*req->forced)[pi].empty()) {
            order = (*req->forced)[pi];
            if ((int)order.size() != k) return USTAT_ERR_INVALID_ARG;
            std::vector<int> chk = order;
            std::sort(chk.begin(), chk.end());
            for (int i = 0; i < k; ++i)
                if (chk[i] != i) return USTAT_ERR_INVALID_ARG;
            c = simulate(k, Q.adj, order.data());
            if (!c.ok) return USTAT_ERR_TW_TOO_LARGE;
        } else if (P.planner == USTAT_PLAN_MINFILL) {
            order = minfill_order(k, Q.adj);
            c = simulate(k, Q.adj, order.data());
            if (!c.ok) order = exhaustive_order(k, Q.adj, &c);
        } else if (!P.cse) {
            order = exhaustive_order(k, Q.adj, &c);
        } else {
            // Sharing-aware exhaustive search: every distinct feasible elimination
            // sequence is lowered on trial against the program built so far and
            // rolled back; the winner adds the fewest new n^4 steps, then the
            // fewest new n^3 products (a product already in the program costs an
            // n^2 pass), then the fewest new operations.
            std::vector<int> perm(k);
            for (int i = 0; i < k; ++i) perm[i] = i;
            std::set<std::vector<int>> seen;
            std::tuple<int, int, int, int> best_cost{1 << 30, 1 << 30, 1 << 30, 1 << 30};
            do {
                Cost cc = simulate(k, Q.adj, perm.data());
                if (!cc.ok) continue;
                // effective sequence: vertices at which a step happens
                std::vector<int> eff;
                {
                    uint32_t adj2[32];
                    std::memcpy(adj2, Q.adj, sizeof(uint32_t) * k);
                    uint32_t al = (1u << k) - 1;
                    for (int v : perm) {
                        if (!((al >> v) & 1)) continue;
                        eff.push_back(v);
                        uint32_t nb = adj2[v] & al & ~(1u << v);
                        uint32_t comp = component(v, al, adj2);
                        if (popc(comp) == popc(nb) + 1) {
                            al &= ~comp;
                        } else {
                            al &= ~(1u << v);
                            for (uint32_t r = nb; r; r &= r - 1) adj2[__builtin_ctz(r)] |= nb & ~(1u << __builtin_ctz(r));
                        }
                    }
                }
                if (!seen.insert(eff).second) continue;
                PartRec tr = pr;
                L.begin_trial();
                const size_t first = P.ops.size();
                int rc = lower(Q, perm, tr);
                int n4 = 0, n3 = 0, nother = 0;
                std::set<std::tuple<int, int, int, int, int>> fresh;
                for (size_t i = first; i < P.ops.size(); ++i) {
                    const Op &op = P.ops[i];
                    if (op.kind == OP_GEMM3) ++n4;
                    else if (op.kind == OP_GEMM || op.kind == OP_GEMM_RED) {
                        auto key = std::make_tuple(op.A.mat, op.A.trans, op.B.mat, op.B.trans, op.u);
                        if (!products.count(key) && fresh.insert(key).second) ++n3;
                        else ++nother;
                    } else ++nother;
                }
                L.rollback();
                if (rc != USTAT_OK) continue;
                auto tc = std::make_tuple(n4, n3, cc.c[1] + cc.c[0], nother);
                if (order.empty() || tc < best_cost) {
                    best_cost = tc;
                    order = perm;
                    c = cc;
                }
            } while (std::next_permutation(perm.begin(), perm.end()));
            if (order.empty()) c.ok = false;
        }
        if (!c.ok) return USTAT_ERR_TW_TOO_LARGE;
        for (int i = 0; i < k; ++i) pr.order[i] = order[i];
        pr.naive_coef[0] = c.c[0];
        for (int p = 1; p < 5; ++p) pr.naive_coef[p] = 2.0 * c.c[p];
        {
            const size_t first = P.ops.size();
            int rc = lower(Q, order, pr);
            if (rc != USTAT_OK) return rc;
            for (size_t i = first; i < P.ops.size(); ++i) {
                const Op &op = P.ops[i];
                if (op.kind == OP_GEMM || op.kind == OP_GEMM_RED)
                    products.insert(std::make_tuple(op.A.mat, op.A.trans, op.B.mat, op.B.trans, op.u));
            }
        }
        parts_out[pi] = pr;
    }
    P.parts = std::move(parts_out);

    // ---- share n^3 products across partitions
    if (P.cse) {
        using Key = std::tuple<int, int, int, int, int>;
        auto pkey = [](const Op &op) { return Key(op.A.mat, op.A.trans, op.B.mat, op.B.trans, op.u); };
        std::map<Key, int> first_use, store_idx;
        std::map<Key, int> red_count;
        for (int i = 0; i < (int)P.ops.size(); ++i) {
            const Op &op = P.ops[i];
            if (op.kind != OP_GEMM && op.kind != OP_GEMM_RED) continue;
            Key kk = pkey(op);
            if (!first_use.count(kk)) first_use[kk] = i;
            if (op.kind == OP_GEMM) store_idx[kk] = i;
            else red_count[kk]++;
        }
        std::map<Key, int> stored_slot;
        std::vector<Op> out;
        for (int i = 0; i < (int)P.ops.size(); ++i) {
            Op op = P.ops[i];
            if (op.kind == OP_GEMM || op.kind == OP_GEMM_RED) {
                Key kk = pkey(op);
                bool shared = store_idx.count(kk) || red_count[kk] >= 2;
                if (shared && first_use[kk] == i) {
                    // the stored product goes where it is first needed
                    if (store_idx.count(kk)) {
                        Op st = P.ops[store_idx[kk]];
                        out.push_back(st);
                        stored_slot[kk] = st.out;
                    } else {
                        Op st = op;
                        st.kind = OP_GEMM;
                        st.W = Term{};
                        st.a = st.b = -1;
                        Slot sl;
                        sl.kind = S_MAT;
                        sl.symmetric = (st.A == st.B) ? 1 : 0;
                        P.slots.push_back(sl);
                        st.out = (int)P.slots.size() - 1;
                        out.push_back(st);
                        stored_slot[kk] = st.out;
                    }
                }
                if (op.kind == OP_GEMM) {
                    if (shared) continue;   // already placed
                    out.push_back(op);
                    continue;
                }
                if (shared) {
                    Op fr;
                    fr.kind = OP_FREDUCE;
                    fr.out = op.out;
                    fr.t[0] = Term{stored_slot[kk], 0};
                    fr.nt = 1;
                    if (op.W.mat >= 0) fr.t[fr.nt++] = op.W;
                    fr.a = op.a;
                    fr.b = op.b;
                    fr.coef = 2;
                    fr.npow = 2;
                    out.push_back(fr);
                    continue;
                }
            }
            out.push_back(op);
        }
        P.ops.swap(out);
    }

    // ---- execution form of the n^3 steps: a terminal GEMM_RED is a GEMM that
    //      stores nothing and carries one fused reduction
    for (auto &op : P.ops) {
        if (op.kind != OP_GEMM_RED) continue;
        Red r;
        r.W = op.W;
        r.a = op.a;
        r.b = op.b;
        r.pow = 1;
        r.out = op.out;
        op.kind = OP_GEMM;
        op.store = 0;
        op.nred = 1;
        op.red[0] = r;
        op.out = -1;
    }

    // ---- fuse reductions of a stored product into its GEMM: a product read only
    //      by reductions sum_jk prod_t F_t(j,k) a(j) b(k) in which it appears once
    //      or twice (with at most one other factor) is reduced in the GEMM's
    //      epilogue and never written
    if (P.cse) {
        auto uses_slot = [](const Op &o, int s) {
            for (int t = 0; t < o.nt; ++t)
                if (o.t[t].mat == s) return true;
            const Term *ts[] = {&o.A, &o.B, &o.W, &o.Ab, &o.Wbc, &o.Wbd};
            for (auto *t : ts)
                if (t->mat == s) return true;
            for (int r = 0; r < o.nred; ++r)
                if (o.red[r].W.mat == s) return true;
            return false;
        };
        std::vector<char> dead(P.ops.size(), 0);
        std::vector<size_t> place(P.ops.size());   // where each op is emitted
        for (size_t i = 0; i < P.ops.size(); ++i) place[i] = i;
        for (size_t gi = 0; gi < P.ops.size(); ++gi) {
            Op &g = P.ops[gi];
            if (g.kind != OP_GEMM || !g.store || g.out < 0) continue;
            const int s = g.out;
            const bool psym = P.slots[s].symmetric != 0;
            std::vector<size_t> cons;
            bool ok = true;
            for (size_t j = 0; j < P.ops.size() && ok; ++j) {
                if (j == gi || dead[j] || !uses_slot(P.ops[j], s)) continue;
                const Op &c = P.ops[j];
                if (c.kind != OP_FREDUCE) {
                    ok = false;
                    break;
                }
                int np = 0, trans0 = -1, ntrans = 0;
                for (int t = 0; t < c.nt; ++t)
                    if (c.t[t].mat == s) {
                        ++np;
                        trans0 = c.t[t].trans;
                        ntrans += c.t[t].trans;
                    }
                if (np > 2 || c.nt - np > 1) ok = false;
                if (np == 2 && ntrans == 1 && !psym) ok = false;
                (void)trans0;
                cons.push_back(j);
            }
            if (!ok || cons.empty() || g.nred + (int)cons.size() > kMaxRed) continue;
            for (size_t j : cons) {
                const Op &c = P.ops[j];
                Red r;
                int np = 0, tr = 0;
                Term other;
                for (int t = 0; t < c.nt; ++t) {
                    if (c.t[t].mat == s) {
                        ++np;
                        tr = psym ? 0 : c.t[t].trans;
                    } else {
                        other = c.t[t];
                    }
                }
                r.pow = np;
                r.out = c.out;
                if (!tr) {
                    r.W = other;
                    r.a = c.a;
                    r.b = c.b;
                } else {
                    // sum_jk P(k,j) W(j,k) a(j) b(k) = sum_jk P(j,k) W(k,j) a(k) b(j)
                    r.W = L.flip(other);
                    r.a = c.b;
                    r.b = c.a;
                }
                g.red[g.nred++] = r;
                dead[j] = 1;
                // the reductions' other inputs may be produced after the GEMM: it
                // runs where its last absorbed reduction stood (nothing reads the
                // unstored product, so moving it later is safe)
                place[gi] = std::max(place[gi], j);
            }
            g.store = 0;
        }
        std::vector<std::vector<size_t>> at(P.ops.size());
        for (size_t i = 0; i < P.ops.size(); ++i)
            if (!dead[i]) at[place[i]].push_back(i);
        std::vector<Op> out;
        for (size_t p = 0; p < P.ops.size(); ++p)
            for (size_t i : at[p]) out.push_back(P.ops[i]);
        P.ops.swap(out);
    }
    // symmetric products with symmetric reductions only need tiles on or above
    // the diagonal
    for (auto &op : P.ops) {
        if (op.kind != OP_GEMM || op.store || !(op.A == op.B)) continue;
        bool sym = op.nred > 0;
        for (int r = 0; r < op.nred; ++r) {
            const Red &R = op.red[r];
            if (R.a != R.b) sym = false;
            if (R.W.mat >= 0 && !P.slots[R.W.mat].symmetric) sym = false;
        }
        op.symmetric = sym ? 1 : 0;
    }

    // ---- operands for the tensor-core GEMMs: K-major copies with the diagonal
    //      scaling of the contracted index folded into A
    if (tc) {
        std::vector<Op> out;
        std::map<std::tuple<int, int, int>, int> opmemo;
        const bool split = is_split_mode(P.precision);
        auto operand = [&](Term t, int u, std::vector<Op> &dst) {
            auto key = std::make_tuple(t.mat, t.trans, u);
            auto it = opmemo.find(key);
            if (it != opmemo.end()) return it->second;
            Op op;
            op.kind = split ? OP_SPLIT : OP_PREP;
            op.t[0] = t;
            op.nt = 1;
            op.u = u;
            op.npow = 2;
            Slot sl;
            sl.kind = split ? S_SLICES : S_PREP;
            P.slots.push_back(sl);
            op.out = (int)P.slots.size() - 1;
            dst.push_back(op);
            opmemo[key] = op.out;
            return op.out;
        };
        for (auto op : P.ops) {
            if (op.kind == OP_GEMM) {
                op.opA = operand(op.A, op.u, out);
                op.opB = (op.A == op.B && op.u < 0) ? op.opA : operand(op.B, -1, out);
            }
            // the s = 3 step on the tensor cores (split modes): B is an ordinary
            // operand; the A operands, scaled by Ab(., bb), are split per bb at run time
            if (op.kind == OP_GEMM3 && split) op.opB = operand(op.B, -1, out);
            out.push_back(op);
        }
        P.ops.swap(out);
        // an RBF kernel matrix has entries in (0, 1]: its unscaled split (row scale 1)
        // is written by the kernel-matrix build itself
        if (split && !wide_storage(P.precision)) {
            std::vector<char> fused(P.ops.size(), 0);
            for (size_t i = 0; i < P.ops.size(); ++i) {
                const Op &op = P.ops[i];
                if (op.kind != OP_SPLIT || op.u >= 0) continue;
                for (auto &kb : P.ops)
                    if (kb.kind == OP_KBUILD && kb.out == op.t[0].mat && kb.opA < 0 &&
                        P.factor_kind[kb.factor] == USTAT_RBF) {
                        kb.opA = op.out;
                        fused[i] = 1;
                        break;
                    }
            }
            std::vector<Op> kept;
            for (size_t i = 0; i < P.ops.size(); ++i)
                if (!fused[i]) kept.push_back(P.ops[i]);
            P.ops.swap(kept);
        }
    }
    for (auto &op : P.ops) {
        if (op.kind == OP_GEMM) {
            P.n_gemm++;
            if (op.symmetric) op.coef = 1.0;   // half the tiles: n^3 flops instead of 2 n^3
        }
        if (op.kind == OP_GEMM3) P.n_gemm3++;
    }

    // ---- a reduction weighted by a vector on one index and by ones on the other
    //      is a dot product with the one-sided sums of the same Hadamard product:
    //      sum_jk T(j,k) a(j) = sum_j a(j) [sum_k T(j,k)], and a GEMV that forms
    //      those sums may already exist.  Terms of symmetric slots are compared
    //      without orientation.
    {
        auto canon = [&](const Op &o, bool flip) {
            std::vector<std::pair<int, int>> v;
            for (int t = 0; t < o.nt; ++t) {
                const int tr = P.slots[o.t[t].mat].symmetric ? 0 : (o.t[t].trans ^ (flip ? 1 : 0));
                v.emplace_back(o.t[t].mat, tr);
            }
            std::sort(v.begin(), v.end());
            return v;
        };
        for (size_t i = 0; i < P.ops.size(); ++i) {
            Op &fr = P.ops[i];
            if (fr.kind != OP_FREDUCE || (fr.a >= 0) == (fr.b >= 0)) continue;
            // b(k) weights the second index: GEMV sums over the first, out(k)
            // a(j) weights the first index: GEMV of the transposed product
            const auto want = canon(fr, fr.a >= 0);
            for (size_t j = 0; j < i; ++j) {
                const Op &gv = P.ops[j];
                if (gv.kind != OP_GEMV || gv.u >= 0 || canon(gv, false) != want) continue;
                Op vd;
                vd.kind = OP_VDOT;
                vd.out = fr.out;
                vd.u = gv.out;
                vd.a = fr.a >= 0 ? fr.a : fr.b;
                vd.npow = 1;
                vd.coef = 2;
                fr = vd;
                break;
            }
        }
    }

    // ---- entrywise-power reductions of an RBF kernel matrix (full sums, and the
    //      row sums a GEMV with unit weights forms) are taken by the float32
    //      kernel-matrix build while the entries are in registers
    if (!wide_storage(P.precision)) {
        std::vector<char> dead(P.ops.size(), 0);
        for (size_t i = 0; i < P.ops.size(); ++i) {
            const Op &r = P.ops[i];
            const bool full = r.kind == OP_FREDUCE && r.a < 0 && r.b < 0;
            const bool rows = r.kind == OP_GEMV && r.u < 0;
            if ((!full && !rows) || r.nt < 1 || r.nt > 4) continue;
            const int s = r.t[0].mat;
            bool same = true;
            for (int t = 1; t < r.nt; ++t) same = same && r.t[t].mat == s;
            if (!same) continue;
            for (size_t k = 0; k < i; ++k) {
                Op &kb = P.ops[k];
                if (kb.kind != OP_KBUILD || kb.out != s || P.factor_kind[kb.factor] != USTAT_RBF ||
                    kb.nred >= kMaxRed)
                    continue;
                Red rd;
                rd.pow = r.nt;
                rd.out = r.out;
                kb.red[kb.nred++] = rd;
                dead[i] = 1;
                break;
            }
        }
        std::vector<Op> kept;
        for (size_t i = 0; i < P.ops.size(); ++i)
            if (!dead[i]) kept.push_back(P.ops[i]);
        P.ops.swap(kept);
    }

    // an RBF kernel matrix whose only readers are symmetric tensor-core GEMMs (which
    // read it as the weight of their upper-triangle tiles; their operands are the
    // digit planes the build writes) needs no stores below the diagonal
    if (is_split_mode(P.precision) && !wide_storage(P.precision)) {
        for (auto &kb : P.ops) {
            if (kb.kind != OP_KBUILD || kb.opA < 0 || P.factor_kind[kb.factor] != USTAT_RBF) continue;
            const int s = kb.out;
            bool ok = true;
            for (const Op &o : P.ops) {
                if (&o == &kb) continue;
                bool reads = false, as_weight = false;
                for (int t = 0; t < o.nt; ++t) reads |= o.t[t].mat == s;
                const Term *ts[] = {&o.W, &o.Ab, &o.Wbc, &o.Wbd};
                for (auto *t : ts) reads |= t->mat == s;
                for (int r = 0; r < o.nred; ++r) as_weight |= o.red[r].W.mat == s;
                const bool operand = o.A.mat == s || o.B.mat == s;
                if (o.kind == OP_GEMM) {
                    // a GEMM reads its weights through red[] (o.W is the pre-fusion copy)
                    if ((as_weight || operand) && !o.symmetric) ok = false;
                } else if (reads || operand || as_weight || o.kind == OP_MHB || o.kind == OP_SPLIT ||
                           o.kind == OP_PREP) {
                    if (o.kind == OP_MHB) {
                        for (const Op &m : P.groups[o.group])
                            for (int t = 0; t < m.nt; ++t)
                                if (m.t[t].mat == s) ok = false;
                    } else if (reads || operand || as_weight || (o.nt > 0 && o.t[0].mat == s)) {
                        ok = false;
                    }
                }
            }
            kb.upper_only = ok ? 1 : 0;
        }
    }
    // ---- schedule by dependency level and merge the n^2 reductions / GEMVs of
    //      one level that read the same few matrices into single passes
    {
        auto ins = [&](const Op &o) {
            std::vector<int> v;
            auto add = [&](int s) {
                if (s >= 0) v.push_back(s);
            };
            for (int t = 0; t < o.nt; ++t) add(o.t[t].mat);
            add(o.u), add(o.a), add(o.b), add(o.A.mat), add(o.B.mat), add(o.W.mat), add(o.Ab.mat);
            add(o.Wbc.mat), add(o.Wbd.mat), add(o.ub);
            if (o.kind == OP_GEMM) add(o.opA), add(o.opB);
            if (o.kind == OP_GEMM3) add(o.opB);
            for (int r = 0; r < o.nred; ++r) add(o.red[r].W.mat), add(o.red[r].a), add(o.red[r].b);
            return v;
        };
        auto outs = [&](const Op &o) {
            std::vector<int> v;
            if (o.out >= 0 && (o.kind != OP_GEMM || o.store)) v.push_back(o.out);
            if (o.kind == OP_KBUILD && o.opA >= 0) v.push_back(o.opA);
            for (int r = 0; r < o.nred; ++r) v.push_back(o.red[r].out);
            return v;
        };
        std::map<int, int> producer;
        std::vector<int> level(P.ops.size(), 0);
        for (size_t i = 0; i < P.ops.size(); ++i) {
            for (int s : ins(P.ops[i])) {
                auto it = producer.find(s);
                if (it != producer.end()) level[i] = std::max(level[i], level[it->second] + 1);
            }
            for (int s : outs(P.ops[i])) producer[s] = (int)i;
        }
        const bool can_group = true;
        auto eligible = [&](const Op &o) {
            if (!can_group || (o.kind != OP_FREDUCE && o.kind != OP_GEMV)) return false;
            for (int t = 0; t < o.nt; ++t)
                if (o.t[t].trans && !P.slots[o.t[t].mat].symmetric) return false;
            return true;
        };
        const int maxlev = level.empty() ? 0 : *std::max_element(level.begin(), level.end());
        std::vector<Op> out;
        for (int L = 0; L <= maxlev; ++L) {
            std::vector<Op> hb;
            for (size_t i = 0; i < P.ops.size(); ++i) {
                if (level[i] != L) continue;
                if (eligible(P.ops[i])) hb.push_back(P.ops[i]);
                else out.push_back(P.ops[i]);
            }
            // greedy packing: up to kMhbOps ops, 4 matrices, 2 GEMVs per pass
            std::vector<char> used(hb.size(), 0);
            for (size_t s = 0; s < hb.size(); ++s) {
                if (used[s]) continue;
                std::vector<Op> grp;
                std::set<int> mats;
                int ngemv = 0;
                for (size_t t = s; t < hb.size(); ++t) {
                    if (used[t] || grp.size() >= 6) continue;
                    std::set<int> m2 = mats;
                    for (int q = 0; q < hb[t].nt; ++q) m2.insert(hb[t].t[q].mat);
                    const int g2 = ngemv + (hb[t].kind == OP_GEMV);
                    if (m2.size() > 4 || g2 > 2) continue;
                    mats = m2;
                    ngemv = g2;
                    grp.push_back(hb[t]);
                    used[t] = 1;
                }
                Op m;
                m.kind = OP_MHB;
                m.group = (int)P.groups.size();
                for (auto &g : grp) {
                    m.coef += g.coef;
                    m.npow = 2;
                }
                P.groups.push_back(grp);
                out.push_back(m);
            }
        }
        P.ops.swap(out);

        // every slot an operation reads is written by an earlier operation, and
        // every scalar a partition multiplies is produced
        std::vector<char> made(P.slots.size(), 0);
        auto check_and_make = [&](const Op &o) {
            for (int s : ins(o))
                if (!made[s]) return false;
            for (int s : outs(o)) made[s] = 1;
            return true;
        };
        for (const Op &o : P.ops) {
            if (o.kind == OP_MHB) {
                for (const Op &m : P.groups[o.group])
                    for (int s : ins(m))
                        if (!made[s]) return USTAT_ERR_UNSUPPORTED;
                for (const Op &m : P.groups[o.group])
                    for (int s : outs(m)) made[s] = 1;
            } else if (!check_and_make(o)) {
                return USTAT_ERR_UNSUPPORTED;
            }
        }
        for (const PartRec &pr : P.parts)
            for (int q = 0; q < pr.nscal; ++q)
                if (!made[pr.scal[q]]) return USTAT_ERR_UNSUPPORTED;
    }
    return USTAT_OK;
}

}  // namespace ustat
