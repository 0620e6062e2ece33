// Gate DAG and the Nat / DFS / dagP part builders (Sec. IV of the paper).
//
// Readings of details the paper leaves open (Sec. IV-B defers the builders' details to
// external work; each reading below is this library's and the oracle's alike):
//  * Nat (Sec. IV-B): gate g joins the open part iff L(part + g) <= k; else
//    the part is closed and g opens the next one.
//  * DFS (Sec. IV-B): trial r draws from SplitMix64(seed ^ r*0x9E3779B97F4A7C15);
//    the order is a LIFO Kahn traversal: source gates shuffled (Fisher-Yates)
//    onto a stack, each popped gate emitted, its successors that become ready
//    (operand order) shuffled and pushed. Fewest parts wins, ties to lowest r.
//  * dagP (Sec. IV-B): (1) acyclic agglomerative clustering from single gates
//    over pairs that share a qubit; (2) recursive bisection of the clusters,
//    taken in Kahn order keyed by smallest gate, by the prefix cut minimising
//    L(V1) + L(V2) with the larger side at most floor(3W/4) gates (imbalance
//    ratio 1.5), refined by single-cluster moves of positive gain that keep V1
//    a down-set, until every piece has L <= k; (3) merge phase on the part
//    graph over all pairs. A merge takes the valid pair (L(a u b) <= k and no
//    path of length >= 2 between a and b, so the part graph stays acyclic)
//    with the most shared qubits, ties to the smaller (min gate, max gate) key.
//  * Schedule: Kahn order of the part graph, ties to the part holding the
//    smallest gate index (parts run in topological order, Sec. IV-A).
#include "partition.hpp"

#include <algorithm>
#include <array>
#include <functional>
#include <map>
#include <queue>
#include <set>
#include <tuple>

namespace hisv {

static inline int popc(uint64_t x) { return __builtin_popcountll(x); }

bool build_dag(const std::vector<GateRef> &gates, int n, Dag &dag, std::string &err) {
    dag.n = n;
    dag.G = (int)gates.size();
    dag.qmask.assign(dag.G, 0);
    dag.preds.assign(dag.G, {});
    dag.succs.assign(dag.G, {});
    dag.qubits.assign(dag.G, {});
    std::vector<int> last(n, -1);
    // next[g][j]: gate after g on its j-th operand wire
    std::vector<std::vector<int>> next(dag.G);
    for (int g = 0; g < dag.G; g++) {
        const GateRef &gr = gates[g];
        uint64_t m = 0;
        next[g].assign(gr.arity, -1);
        for (int j = 0; j < gr.arity; j++) {
            int q = gr.q[j];
            if (q < 0 || q >= n) {
                err = "gate " + std::to_string(g) + ": qubit " + std::to_string(q) + " out of range";
                return false;
            }
            if ((m >> q) & 1) {
                err = "gate " + std::to_string(g) + ": repeated qubit " + std::to_string(q);
                return false;
            }
            m |= 1ull << q;
            dag.qubits[g].push_back(q);
            int p = last[q];
            if (p >= 0) {
                if (std::find(dag.preds[g].begin(), dag.preds[g].end(), p) == dag.preds[g].end())
                    dag.preds[g].push_back(p);
                for (int jj = 0; jj < (int)dag.qubits[p].size(); jj++)
                    if (dag.qubits[p][jj] == q) next[p][jj] = g;
            }
        }
        for (int j = 0; j < gr.arity; j++) last[gr.q[j]] = g;
        dag.qmask[g] = m;
    }
    for (int p = 0; p < dag.G; p++)
        for (int s : next[p])
            if (s >= 0 && std::find(dag.succs[p].begin(), dag.succs[p].end(), s) == dag.succs[p].end())
                dag.succs[p].push_back(s);
    return true;
}

// ------------------------------------------------------------ schedule ---
std::vector<uint32_t> schedule_parts(const Dag &dag, const std::vector<uint32_t> &pog) {
    if (dag.G == 0) return {};
    uint32_t P = 0;
    for (uint32_t p : pog) P = std::max(P, p + 1);
    std::vector<int> mg(P, -1);
    for (int g = 0; g < dag.G; g++)
        if (mg[pog[g]] < 0) mg[pog[g]] = g;
    std::vector<std::set<uint32_t>> succ(P);
    for (int g = 0; g < dag.G; g++)
        for (int s : dag.succs[g])
            if (pog[s] != pog[g]) succ[pog[g]].insert(pog[s]);
    std::vector<int> indeg(P, 0);
    for (uint32_t a = 0; a < P; a++)
        for (uint32_t b : succ[a]) indeg[b]++;
    typedef std::pair<int, uint32_t> E;
    std::priority_queue<E, std::vector<E>, std::greater<E>> h;
    for (uint32_t a = 0; a < P; a++)
        if (indeg[a] == 0) h.push({mg[a], a});
    std::vector<uint32_t> newid(P, UINT32_MAX);
    uint32_t nxt = 0;
    while (!h.empty()) {
        uint32_t a = h.top().second;
        h.pop();
        newid[a] = nxt++;
        for (uint32_t b : succ[a])
            if (--indeg[b] == 0) h.push({mg[b], b});
    }
    std::vector<uint32_t> out(dag.G);
    for (int g = 0; g < dag.G; g++) out[g] = newid[pog[g]];
    return out;
}

static std::vector<std::vector<int>> cut_order(const Dag &dag, const std::vector<int> &order, int k) {
    std::vector<std::vector<int>> parts;
    std::vector<int> cur;
    uint64_t m = 0;
    for (int g : order) {
        uint64_t gm = dag.qmask[g];
        if (!cur.empty() && popc(m | gm) > k) {
            parts.push_back(cur);
            cur.clear();
            m = 0;
        }
        cur.push_back(g);
        m |= gm;
    }
    if (!cur.empty()) parts.push_back(cur);
    return parts;
}

static std::vector<uint32_t> parts_to_pog(int G, const std::vector<std::vector<int>> &parts) {
    std::vector<uint32_t> pog(G, 0);
    for (size_t i = 0; i < parts.size(); i++)
        for (int g : parts[i]) pog[g] = (uint32_t)i;
    return pog;
}

std::vector<uint32_t> part_nat(const Dag &dag, int k) {
    std::vector<int> order(dag.G);
    for (int i = 0; i < dag.G; i++) order[i] = i;
    return schedule_parts(dag, parts_to_pog(dag.G, cut_order(dag, order, k)));
}

// ----------------------------------------------------------------- DFS ---
namespace {
struct SplitMix64 {  // Steele, Lea, Flood (2014)
    uint64_t s;
    explicit SplitMix64(uint64_t seed) : s(seed) {}
    uint64_t next() {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    void shuffle(std::vector<int> &a) {
        for (int i = (int)a.size() - 1; i > 0; i--) {
            int j = (int)(next() % (uint64_t)(i + 1));
            std::swap(a[i], a[j]);
        }
    }
};
}  // namespace

std::vector<uint32_t> part_dfs(const Dag &dag, int k, uint64_t seed, int trials) {
    if (trials <= 0) trials = 16;
    std::vector<std::vector<int>> best;
    bool have = false;
    for (int r = 0; r < trials; r++) {
        SplitMix64 rng(seed ^ ((uint64_t)r * 0x9E3779B97F4A7C15ull));
        std::vector<int> indeg(dag.G);
        for (int g = 0; g < dag.G; g++) indeg[g] = (int)dag.preds[g].size();
        std::vector<int> stack;
        for (int g = 0; g < dag.G; g++)
            if (indeg[g] == 0) stack.push_back(g);
        rng.shuffle(stack);
        std::vector<int> order;
        order.reserve(dag.G);
        while (!stack.empty()) {
            int g = stack.back();
            stack.pop_back();
            order.push_back(g);
            std::vector<int> newly;
            for (int s : dag.succs[g])
                if (--indeg[s] == 0) newly.push_back(s);
            rng.shuffle(newly);
            stack.insert(stack.end(), newly.begin(), newly.end());
        }
        auto parts = cut_order(dag, order, k);
        if (!have || parts.size() < best.size()) {
            best = parts;
            have = true;
        }
    }
    return schedule_parts(dag, parts_to_pog(dag.G, best));
}

// ---------------------------------------------------------------- dagP ---
namespace {

// Units: groups of gates with their part graph and reachability bitsets.
struct Units {
    const Dag *dag;
    int words = 0;
    std::vector<char> alive;
    std::vector<std::vector<int>> gates;
    std::vector<uint64_t> qm;
    std::vector<int> mg;
    std::vector<std::set<int>> succ, pred;
    std::vector<std::vector<uint64_t>> reach;  // units reachable by >= 1 edge
    std::vector<int> wprev, wnext;             // [unit * n + q]: neighbouring unit on wire q, or -1
    int next_id = 0;

    bool bit(const std::vector<uint64_t> &r, int i) const { return (r[i >> 6] >> (i & 63)) & 1; }

    Units(const Dag &d, const std::vector<std::vector<int>> &groups) : dag(&d) {
        int U = (int)groups.size();
        int cap = 2 * U + 2;
        words = (cap + 63) / 64;
        alive.assign(cap, 0);
        gates.assign(cap, {});
        qm.assign(cap, 0);
        mg.assign(cap, 0);
        succ.assign(cap, {});
        pred.assign(cap, {});
        reach.assign(cap, std::vector<uint64_t>());
        std::vector<int> unit_of(d.G, 0);
        for (int i = 0; i < U; i++) {
            gates[i] = groups[i];
            std::sort(gates[i].begin(), gates[i].end());
            uint64_t m = 0;
            for (int g : gates[i]) {
                m |= d.qmask[g];
                unit_of[g] = i;
            }
            qm[i] = m;
            mg[i] = gates[i][0];
            alive[i] = 1;
        }
        next_id = U;
        for (int g = 0; g < d.G; g++)
            for (int t : d.succs[g]) {
                int a = unit_of[g], b = unit_of[t];
                if (a != b) {
                    succ[a].insert(b);
                    pred[b].insert(a);
                }
            }
        // wire order: a unit's gates on a wire are contiguous (the part graph
        // is acyclic), so units follow each other on every wire
        const int n = d.n;
        wprev.assign((size_t)cap * n, -1);
        wnext.assign((size_t)cap * n, -1);
        for (int q = 0; q < n; q++) {
            std::vector<std::pair<int, int>> on;   // (first gate on q, unit)
            for (int i = 0; i < U; i++) {
                if (!((qm[i] >> q) & 1)) continue;
                for (int g : gates[i])
                    if ((d.qmask[g] >> q) & 1) {
                        on.push_back({g, i});
                        break;
                    }
            }
            std::sort(on.begin(), on.end());
            for (size_t j = 1; j < on.size(); j++) {
                wnext[(size_t)on[j - 1].second * n + q] = on[j].second;
                wprev[(size_t)on[j].second * n + q] = on[j - 1].second;
            }
        }
        std::vector<int> order = topo();
        for (int i = (int)order.size() - 1; i >= 0; i--) {
            int u = order[i];
            reach[u].assign(words, 0);
            for (int v : succ[u]) {
                reach[u][v >> 6] |= 1ull << (v & 63);
                for (int w = 0; w < words; w++) reach[u][w] |= reach[v][w];
            }
        }
    }

    std::vector<int> live() const {
        std::vector<int> out;
        for (int i = 0; i < next_id; i++)
            if (alive[i]) out.push_back(i);
        return out;
    }

    // Kahn order keyed by each unit's smallest gate.
    std::vector<int> topo() const {
        std::vector<int> L = live();
        std::map<int, int> indeg;
        for (int u : L) indeg[u] = 0;
        for (int u : L)
            for (int v : succ[u]) indeg[v]++;
        typedef std::pair<int, int> E;
        std::priority_queue<E, std::vector<E>, std::greater<E>> h;
        for (int u : L)
            if (indeg[u] == 0) h.push({mg[u], u});
        std::vector<int> out;
        while (!h.empty()) {
            int u = h.top().second;
            h.pop();
            out.push_back(u);
            for (int v : succ[u])
                if (--indeg[v] == 0) h.push({mg[v], v});
        }
        return out;
    }

    bool long_path(int a, int b) const {
        for (int c : succ[a])
            if (bit(reach[c], b)) return true;
        for (int c : succ[b])
            if (bit(reach[c], a)) return true;
        return false;
    }

    int merge(int a, int b) {
        int c = next_id++;
        std::vector<int> g;
        std::merge(gates[a].begin(), gates[a].end(), gates[b].begin(), gates[b].end(), std::back_inserter(g));
        gates[c] = std::move(g);
        gates[a].clear();
        gates[b].clear();
        qm[c] = qm[a] | qm[b];
        mg[c] = std::min(mg[a], mg[b]);
        alive[a] = alive[b] = 0;
        alive[c] = 1;
        std::set<int> sc, pc;
        for (int x : succ[a]) if (x != a && x != b) sc.insert(x);
        for (int x : succ[b]) if (x != a && x != b) sc.insert(x);
        for (int x : pred[a]) if (x != a && x != b) pc.insert(x);
        for (int x : pred[b]) if (x != a && x != b) pc.insert(x);
        succ[a].clear(); succ[b].clear(); pred[a].clear(); pred[b].clear();
        for (int x : sc) { pred[x].erase(a); pred[x].erase(b); pred[x].insert(c); }
        for (int x : pc) { succ[x].erase(a); succ[x].erase(b); succ[x].insert(c); }
        succ[c] = std::move(sc);
        pred[c] = std::move(pc);
        const int n = dag->n;
        for (int q = 0; q < n; q++) {
            const bool ia = (qm[a] >> q) & 1, ib = (qm[b] >> q) & 1;
            if (!ia && !ib) continue;
            int p, nx;
            if (ia && ib) {   // adjacent on q (no unit between them: no long path)
                const bool ab = wnext[(size_t)a * n + q] == b;
                p = wprev[(size_t)(ab ? a : b) * n + q];
                nx = wnext[(size_t)(ab ? b : a) * n + q];
            } else {
                const int u = ia ? a : b;
                p = wprev[(size_t)u * n + q];
                nx = wnext[(size_t)u * n + q];
            }
            wprev[(size_t)c * n + q] = p;
            wnext[(size_t)c * n + q] = nx;
            if (p >= 0) wnext[(size_t)p * n + q] = c;
            if (nx >= 0) wprev[(size_t)nx * n + q] = c;
        }
        std::vector<uint64_t> rc(words, 0);
        for (int w = 0; w < words; w++) rc[w] = reach[a][w] | reach[b][w];
        rc[a >> 6] &= ~(1ull << (a & 63));
        rc[b >> 6] &= ~(1ull << (b & 63));
        for (int x = 0; x < next_id; x++) {
            if (!alive[x] || x == c) continue;
            std::vector<uint64_t> &r = reach[x];
            const bool ra = bit(r, a), rb = bit(r, b);
            if (!ra && !rb) continue;
            // x already holds the reach of the side it reached; only the
            // other side's reach can be new to it
            if (ra != rb) {
                const std::vector<uint64_t> &o = ra ? reach[b] : reach[a];
                for (int w = 0; w < words; w++) r[w] |= o[w];
            }
            r[a >> 6] &= ~(1ull << (a & 63));
            r[b >> 6] &= ~(1ull << (b & 63));
            r[c >> 6] |= 1ull << (c & 63);
        }
        reach[a].clear();
        reach[b].clear();
        reach[c] = std::move(rc);
        return c;
    }

    // Merge rule: smallest key (-shared, min mg, max mg) among valid pairs.
    // Two units that share a qubit can only be valid when no unit lies
    // between them on that wire (else a path of length 2 runs through it,
    // and it stays there while both live), so the candidates that share
    // qubits are the wire neighbours: the same merges as over all sharing
    // pairs, with far fewer heap entries.
    void merge_loop(int k, bool zero_shared) {
        typedef std::tuple<int, int, int, int, int> Key;
        std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
        int n = dag->n;
        auto push = [&](int a, int b) {
            if (popc(qm[a] | qm[b]) > k) return;
            int m1 = std::min(mg[a], mg[b]), m2 = std::max(mg[a], mg[b]);
            heap.push(Key(-popc(qm[a] & qm[b]), m1, m2, a, b));
        };
        auto push_neighbours = [&](int u) {
            for (int q = 0; q < n; q++)
                if ((qm[u] >> q) & 1) {
                    const int p = wprev[(size_t)u * n + q], nx = wnext[(size_t)u * n + q];
                    if (p >= 0) push(p, u);
                    if (nx >= 0) push(u, nx);
                }
        };
        for (int u : live()) {
            for (int q = 0; q < n; q++)
                if ((qm[u] >> q) & 1) {
                    const int nx = wnext[(size_t)u * n + q];
                    if (nx >= 0) push(std::min(u, nx), std::max(u, nx));
                }
        }
        bool zero_done = false;
        while (true) {
            if (heap.empty()) {
                if (!zero_shared || zero_done) break;
                zero_done = true;
                std::vector<int> L = live();
                for (size_t i = 0; i < L.size(); i++)
                    for (size_t j = i + 1; j < L.size(); j++)
                        if (!(qm[L[i]] & qm[L[j]])) push(L[i], L[j]);
                if (heap.empty()) break;
                continue;
            }
            Key top = heap.top();
            heap.pop();
            int a = std::get<3>(top), b = std::get<4>(top);
            if (!alive[a] || !alive[b]) continue;
            if (long_path(a, b)) continue;
            int c = merge(a, b);
            if (zero_done) {
                for (int v : live())
                    if (v != c) push(v, c);
            } else {
                push_neighbours(c);
            }
        }
    }
};

// Prefix cut of a unit sequence (see the file header).
static void bisect_units(const Units &U, const std::vector<int> &seq, std::vector<int> &V1,
                         std::vector<int> &V2, long &cap) {
    int m = (int)seq.size();
    std::vector<long> w(m), prew(m + 1, 0);
    std::vector<int> pre(m + 1, 0), suf(m + 1, 0);
    long W = 0;
    uint64_t mask = 0;
    for (int i = 0; i < m; i++) {
        w[i] = (long)U.gates[seq[i]].size();
        W += w[i];
        mask |= U.qm[seq[i]];
        pre[i + 1] = popc(mask);
        prew[i + 1] = prew[i] + w[i];
    }
    mask = 0;
    for (int i = m - 1; i >= 0; i--) {
        mask |= U.qm[seq[i]];
        suf[i] = popc(mask);
    }
    cap = (3 * W) / 4;
    bool have = false;
    std::tuple<long, long, int> best;
    for (int pass = 0; pass < 2 && !have; pass++) {
        for (int c = 1; c < m; c++) {
            if (pass == 0 && std::max(prew[c], W - prew[c]) > cap) continue;
            std::tuple<long, long, int> key((long)pre[c] + suf[c], std::labs(2 * prew[c] - W), c);
            if (!have || key < best) {
                best = key;
                have = true;
            }
        }
    }
    int c = std::get<2>(best);
    cap = std::max(cap, std::max(prew[c], W - prew[c]));
    V1.assign(seq.begin(), seq.begin() + c);
    V2.assign(seq.begin() + c, seq.end());
}

static void refine_units(const Units &U, const std::vector<int> &seq, std::vector<int> &V1,
                         std::vector<int> &V2, long cap) {
    int n = U.dag->n;
    std::map<int, int> side;
    std::set<int> inP(seq.begin(), seq.end());
    for (int u : V1) side[u] = 1;
    for (int u : V2) side[u] = 2;
    std::vector<long> cnt[3];
    cnt[1].assign(n, 0);
    cnt[2].assign(n, 0);
    std::map<int, std::vector<std::pair<int, long>>> use;  // unit -> (qubit, gate count)
    for (int u : seq) {
        std::vector<long> uq(n, 0);
        for (int g : U.gates[u])
            for (int q : U.dag->qubits[g]) uq[q]++;
        for (int q = 0; q < n; q++)
            if (uq[q]) {
                use[u].push_back({q, uq[q]});
                cnt[side[u]][q] += uq[q];
            }
    }
    long size[3] = {0, (long)V1.size(), (long)V2.size()};
    long wt[3] = {0, 0, 0};
    for (int u : V1) wt[1] += (long)U.gates[u].size();
    for (int u : V2) wt[2] += (long)U.gates[u].size();
    std::vector<int> order(seq);
    std::sort(order.begin(), order.end(), [&](int a, int b) { return U.mg[a] < U.mg[b]; });
    long moves = 0, limit = 4 * (long)seq.size();
    while (moves < limit) {
        int bestg = 0, bestu = -1;
        for (int u : order) {
            int s = side[u], o = 3 - s;
            if (size[s] == 1 || wt[o] + (long)U.gates[u].size() > cap) continue;
            bool blocked = false;
            if (s == 1) {
                for (int x : U.succ[u])
                    if (inP.count(x) && side[x] == 1) { blocked = true; break; }
            } else {
                for (int x : U.pred[u])
                    if (inP.count(x) && side[x] == 2) { blocked = true; break; }
            }
            if (blocked) continue;
            int gain = 0;
            for (auto &qc : use[u]) {
                if (cnt[s][qc.first] == qc.second) gain++;
                if (cnt[o][qc.first] == 0) gain--;
            }
            if (gain > 0 && (bestu < 0 || gain > bestg)) {
                bestg = gain;
                bestu = u;
            }
        }
        if (bestu < 0) break;
        int u = bestu, s = side[u], o = 3 - s;
        for (auto &qc : use[u]) {
            cnt[s][qc.first] -= qc.second;
            cnt[o][qc.first] += qc.second;
        }
        side[u] = o;
        size[s]--;
        size[o]++;
        wt[s] -= (long)U.gates[u].size();
        wt[o] += (long)U.gates[u].size();
        moves++;
    }
    V1.clear();
    V2.clear();
    for (int u : seq) (side[u] == 1 ? V1 : V2).push_back(u);
}

}  // namespace

std::vector<uint32_t> part_dagp(const Dag &dag, int k) {
    if (dag.G == 0) return {};
    std::vector<std::vector<int>> singles(dag.G);
    for (int g = 0; g < dag.G; g++) singles[g] = {g};
    Units U(dag, singles);
    U.merge_loop(k, false);                       // (1) coarsening
    std::vector<std::vector<int>> leaves;         // (2) recursive bisection
    std::vector<std::vector<int>> stack;
    stack.push_back(U.topo());
    while (!stack.empty()) {
        std::vector<int> seq = std::move(stack.back());
        stack.pop_back();
        uint64_t m = 0;
        for (int u : seq) m |= U.qm[u];
        if (popc(m) <= k) {
            std::vector<int> leaf;
            for (int u : seq) leaf.insert(leaf.end(), U.gates[u].begin(), U.gates[u].end());
            leaves.push_back(leaf);
            continue;
        }
        std::vector<int> V1, V2;
        long cap = 0;
        bisect_units(U, seq, V1, V2, cap);
        refine_units(U, seq, V1, V2, cap);
        stack.push_back(V2);
        stack.push_back(V1);
    }
    Units M(dag, leaves);                         // (3) merge phase
    M.merge_loop(k, true);
    std::vector<std::vector<int>> parts;
    for (int u : M.live()) parts.push_back(M.gates[u]);
    return schedule_parts(dag, parts_to_pog(dag.G, parts));
}

// ---------------------------------------------------------------- exact ---
// Minimum number of parts over all acyclic partitions with L <= k (the
// optimum the paper's ILP comparison measures dagP against, Sec. V-A). The
// parts of an acyclic partition, listed in a topological order of the part
// graph, have down-set prefixes, so a partition is a chain of down-sets and
// the optimum is a shortest path in the lattice of down-sets. Moving a gate
// that could join an earlier part into it never adds a part, so some optimal
// chain has every part inclusion-maximal given its prefix; such a part is
// fixed by its qubit set Q (|Q| = min(k, qubits used)): all gates on Q whose
// predecessors are in the prefix or the part. Breadth-first search over the
// down-sets with those steps; gates are in circuit order, a topological
// order, so one ascending sweep builds a part. Circuits of at most
// EXACT_MAX_GATES gates; the search is bounded and fails beyond it.
namespace {
constexpr int EXACT_MAX_GATES = 256;
using GateSet = std::array<uint64_t, EXACT_MAX_GATES / 64>;
inline bool has(const GateSet &s, int g) { return (s[g >> 6] >> (g & 63)) & 1; }
inline void put(GateSet &s, int g) { s[g >> 6] |= 1ull << (g & 63); }
}  // namespace

bool part_exact(const Dag &dag, int k, std::vector<uint32_t> &pog, std::string &err) {
    const int G = dag.G, n = dag.n;
    if (G > EXACT_MAX_GATES) {
        err = "exact part builder: at most " + std::to_string(EXACT_MAX_GATES) + " gates";
        return false;
    }
    pog.assign(G, 0);
    if (G == 0) return true;
    GateSet all{};
    for (int g = 0; g < G; g++) put(all, g);
    // the qubit sets Q: every subset of the circuit's qubits of size min(k, used)
    uint64_t used = 0;
    for (int g = 0; g < G; g++) used |= dag.qmask[g];
    std::vector<int> uq;
    for (int q = 0; q < n; q++)
        if ((used >> q) & 1) uq.push_back(q);
    const int r = std::min<int>(k, (int)uq.size());
    std::vector<uint64_t> qsets;
    std::vector<int> pick(r);
    for (int i = 0; i < r; i++) pick[i] = i;
    while (true) {
        uint64_t m = 0;
        for (int i = 0; i < r; i++) m |= 1ull << uq[pick[i]];
        qsets.push_back(m);
        if (qsets.size() > (1u << 20)) {
            err = "exact part builder: too many qubit sets";
            return false;
        }
        int i = r - 1;
        while (i >= 0 && pick[i] == (int)uq.size() - r + i) i--;
        if (i < 0) break;
        pick[i]++;
        for (int j = i + 1; j < r; j++) pick[j] = pick[j - 1] + 1;
    }
    std::map<GateSet, GateSet> parent;   // down-set -> its predecessor on a shortest chain
    parent[GateSet{}] = GateSet{};
    std::vector<GateSet> level{GateSet{}};
    uint64_t work = 0;
    while (!level.empty() && !parent.count(all)) {
        std::vector<GateSet> next;
        for (const GateSet &D : level) {
            for (uint64_t Q : qsets) {
                work += (uint64_t)G;
                if (work > (1ull << 30)) {   // about a second of host time
                    err = "exact part builder: search too large for this circuit";
                    return false;
                }
                GateSet E = D;
                bool grew = false;
                for (int g = 0; g < G; g++) {
                    if (has(E, g) || (dag.qmask[g] & ~Q) != 0) continue;
                    bool ready = true;
                    for (int p : dag.preds[g])
                        if (!has(E, p)) {
                            ready = false;
                            break;
                        }
                    if (ready) {
                        put(E, g);
                        grew = true;
                    }
                }
                if (!grew || parent.count(E)) continue;
                parent[E] = D;
                next.push_back(E);
                if (parent.size() > (1u << 22)) {
                    err = "exact part builder: search too large for this circuit";
                    return false;
                }
            }
        }
        level.swap(next);
    }
    if (!parent.count(all)) {
        err = "exact part builder: no partition found";
        return false;
    }
    std::vector<std::vector<int>> parts;
    for (GateSet E = all; E != GateSet{};) {
        const GateSet D = parent[E];
        std::vector<int> part;
        for (int g = 0; g < G; g++)
            if (has(E, g) && !has(D, g)) part.push_back(g);
        parts.push_back(part);
        E = D;
    }
    std::reverse(parts.begin(), parts.end());
    pog = schedule_parts(dag, parts_to_pog(G, parts));
    return true;
}

// ----------------------------------------------------------------- beam ---
// Beam search over the same lattice of down-sets as the exact builder, for
// circuits of any size: from each kept down-set D, candidate parts are grown
// from every available gate g0: start with Q = qubits(g0) and the closure of
// D on Q (all gates on Q whose predecessors are in D or the closure), then
// add, while |Q| < k, the qubit of a gate blocked only by Q that makes the
// closure largest (ties: the smaller qubit; widths of 32 and more rank a
// qubit by the largest closure one more qubit can reach, then by its own
// closure). Each level keeps the `width`
// down-sets covering the most gates (ties: the lexicographically smaller
// gate set); the first level that covers every gate gives the partition.
// A greedy width of 1 already picks each part's qubit set by its gate count,
// where dagP bisects; wider beams recover from early choices.
std::vector<uint32_t> part_beam(const Dag &dag, int k, int width) {
    const int G = dag.G, W = (G + 63) / 64;
    if (G == 0) return {};
    if (width < 1) width = 16;
    using Bits = std::vector<uint64_t>;
    auto in = [](const Bits &b, int g) { return (b[g >> 6] >> (g & 63)) & 1; };
    struct Node {
        Bits D;
        int count;
        int parent;
    };
    std::vector<Node> nodes;
    nodes.push_back({Bits(W, 0), 0, -1});
    std::vector<int> beam{0};
    std::vector<uint32_t> mark(G, 0);
    uint32_t gen = 0;
    std::vector<int> stack, added, trial, avail;
    // closure of D on Q, grown from the available gates: the added gates
    // (marked with the current generation)
    auto closure = [&](const Bits &D, uint64_t Q, std::vector<int> &out) {
        ++gen;
        out.clear();
        stack.clear();
        for (int g : avail)
            if ((dag.qmask[g] & ~Q) == 0) stack.push_back(g);
        while (!stack.empty()) {
            const int g = stack.back();
            stack.pop_back();
            if (mark[g] == gen || (dag.qmask[g] & ~Q) != 0) continue;
            bool ok = true;
            for (int p : dag.preds[g])
                if (!in(D, p) && mark[p] != gen) {
                    ok = false;
                    break;
                }
            if (!ok) continue;
            mark[g] = gen;
            out.push_back(g);
            for (int t : dag.succs[g])
                if (!in(D, t) && mark[t] != gen) stack.push_back(t);
        }
    };
    int done = -1;
    while (done < 0) {
        // next level: candidate down-set -> (count, parent); ordered for determinism
        std::map<Bits, std::pair<int, int>> next;
        for (int ni : beam) {
            const Bits D = nodes[ni].D;
            avail.clear();
            for (int g = 0; g < G; g++) {
                if (in(D, g)) continue;
                bool ok = true;
                for (int p : dag.preds[g])
                    if (!in(D, p)) {
                        ok = false;
                        break;
                    }
                if (ok) avail.push_back(g);
            }
            for (int g0 : avail) {
                uint64_t Q = dag.qmask[g0];
                closure(D, Q, added);
                while (popc(Q) < k) {
                    // qubits of the gates that only Q keeps out of the closure
                    uint64_t cq = 0;
                    auto consider = [&](int h) {
                        if (in(D, h) || mark[h] == gen) return;
                        for (int p : dag.preds[h])
                            if (!in(D, p) && mark[p] != gen) return;
                        cq |= dag.qmask[h];
                    };
                    for (int h : avail) consider(h);
                    for (int a : added)
                        for (int h : dag.succs[a]) consider(h);
                    cq &= ~Q;
                    if (!cq) break;
                    int best_q = -1;
                    size_t best_n = 0;
                    const bool look = width >= 32 && popc(Q) + 2 <= k;
                    for (uint64_t m = cq; m; m &= m - 1) {
                        const int q = __builtin_ctzll(m);
                        closure(D, Q | (1ull << q), trial);
                        size_t score = trial.size();
                        if (look) {
                            // wide beams look one qubit further: the score is the
                            // largest closure after the best follow-up qubit
                            uint64_t cq2 = 0;
                            const uint32_t g1 = gen;
                            auto consider2 = [&](int h) {
                                if (in(D, h) || mark[h] == g1) return;
                                for (int p : dag.preds[h])
                                    if (!in(D, p) && mark[p] != g1) return;
                                cq2 |= dag.qmask[h];
                            };
                            for (int h : avail) consider2(h);
                            for (int a : trial)
                                for (int h : dag.succs[a]) consider2(h);
                            cq2 &= ~(Q | (1ull << q));
                            std::vector<int> t2;
                            size_t best2 = trial.size();
                            for (uint64_t m2 = cq2; m2; m2 &= m2 - 1) {
                                const int q2 = __builtin_ctzll(m2);
                                closure(D, Q | (1ull << q) | (1ull << q2), t2);
                                best2 = std::max(best2, t2.size());
                            }
                            score = best2 * 1024 + trial.size();
                        }
                        if (best_q < 0 || score > best_n) {
                            best_q = q;
                            best_n = score;
                        }
                    }
                    Q |= 1ull << best_q;
                    closure(D, Q, added);
                }
                if (added.empty()) continue;
                Bits E = D;
                for (int g : added) E[g >> 6] |= 1ull << (g & 63);
                const int cnt = nodes[ni].count + (int)added.size();
                auto it = next.find(E);
                if (it == next.end()) next.emplace(std::move(E), std::make_pair(cnt, ni));
            }
        }
        // keep the `width` best: most gates, then the smaller gate set (map order)
        std::vector<std::pair<int, const Bits *>> order;
        for (auto &kv : next) order.push_back({kv.second.first, &kv.first});
        std::stable_sort(order.begin(), order.end(),
                         [](const std::pair<int, const Bits *> &a, const std::pair<int, const Bits *> &b) {
                             return a.first > b.first;
                         });
        beam.clear();
        for (size_t i = 0; i < order.size() && (int)i < width; i++) {
            const auto &val = next[*order[i].second];
            nodes.push_back({*order[i].second, val.first, val.second});
            beam.push_back((int)nodes.size() - 1);
            if (val.first == G && done < 0) done = (int)nodes.size() - 1;
        }
        if (beam.empty()) break;   // unreachable: some gate is always available
    }
    std::vector<std::vector<int>> parts;
    for (int ni = done; ni > 0; ni = nodes[ni].parent) {
        const Bits &E = nodes[ni].D, &D = nodes[nodes[ni].parent].D;
        std::vector<int> part;
        for (int g = 0; g < G; g++)
            if (in(E, g) && !in(D, g)) part.push_back(g);
        parts.push_back(part);
    }
    std::reverse(parts.begin(), parts.end());
    return schedule_parts(dag, parts_to_pog(G, parts));
}

// One builder by its method code (1 Nat, 2 DFS, 3 dagP, 4 exact, 5 beam).
bool run_builder(const Dag &dag, int method, int k, uint64_t seed, int trials, std::vector<uint32_t> &pog,
                 std::string &err) {
    switch (method) {
    case 1: pog = part_nat(dag, k); return true;
    case 2: pog = part_dfs(dag, k, seed, trials); return true;
    case 3: pog = part_dagp(dag, k); return true;
    case 4: return part_exact(dag, k, pog, err);
    case 5: pog = part_beam(dag, k, trials); return true;
    default: err = "bad builder"; return false;
    }
}

// Multi-level partitioning (Sec. IV-B): the circuit is partitioned under the
// first-level limit k1; then every first-level part, as a circuit of its own
// (its gates in their original order, which its sub-DAG respects), is
// partitioned again under the second-level limit k2. Inner parts are
// numbered globally: the first-level parts in schedule order, and inside
// each the inner parts in their own schedule order.
bool part_multilevel(const std::vector<GateRef> &gates, int n, int m1, int k1, int m2, int k2, uint64_t seed,
                     int trials, std::vector<uint32_t> &outer, std::vector<uint32_t> &inner, std::string &err) {
    Dag dag;
    if (!build_dag(gates, n, dag, err)) return false;
    if (!run_builder(dag, m1, k1, seed, trials, outer, err)) return false;
    uint32_t P = 0;
    for (uint32_t x : outer) P = std::max(P, x + 1);
    std::vector<std::vector<int>> members(P);
    for (size_t g = 0; g < gates.size(); g++) members[outer[g]].push_back((int)g);
    inner.assign(gates.size(), 0);
    uint32_t base = 0;
    for (uint32_t p = 0; p < P; p++) {
        std::vector<GateRef> sub;
        for (int g : members[p]) sub.push_back(gates[g]);
        Dag sd;
        if (!build_dag(sub, n, sd, err)) return false;
        std::vector<uint32_t> sp;
        if (!run_builder(sd, m2, k2, seed, trials, sp, err)) return false;
        uint32_t q = 0;
        for (size_t j = 0; j < sub.size(); j++) {
            inner[members[p][j]] = base + sp[j];
            q = std::max(q, sp[j] + 1);
        }
        base += q;
    }
    return true;
}

}  // namespace hisv
