// Part planner (host): for each part of the partition, fix its tile, split
// its gates into register phases and emit the kernel's op stream.
//
//  * Tile: the part's qubits S (|S| <= k) padded with the lowest qubits not
//    in S up to t (Sec. IV-B, multi-level partitioning: a part smaller than
//    the limit takes extra qubits for spatial locality). Slot p of the tile
//    holds the p-th smallest tile qubit; the n - t others are the outer
//    qubits of Algorithm 1, one CTA per binary assignment of them.
//  * Phases: a second partitioning level inside the part, with limit R on
//    the qubits that need register residency (targets of non-diagonal
//    gates). Gates are taken greedily along the part's gate order; a gate
//    that does not fit blocks its qubits for the rest of the phase, so every
//    qubit keeps its gate order (the schedule rule of Sec. IV-A).
//    Diagonal gates and CX controls need no residency: on a thread bit they
//    become per-thread conditions or a per-thread phase.
//  * SWAP gates cost nothing: they exchange the slots of their two qubits
//    for the rest of the part, and the store uses the final slot map.
#include "planner.hpp"

#include <algorithm>
#include <cstdint>
#include <cmath>
#include <cstring>

#include "../../include/hisvsim.h"

namespace hisv {

static inline int popc(uint64_t x) { return __builtin_popcountll(x); }

bool gate_is_two_qubit(int kind) {
    return kind == SV_GATE_CX || kind == SV_GATE_CZ || kind == SV_GATE_CP || kind == SV_GATE_SWAP;
}

void gate_matrix_1q(int kind, double th, double m[8]) {
    for (int i = 0; i < 8; i++) m[i] = 0.0;
    const double c = std::cos(th / 2), s = std::sin(th / 2), r = std::sqrt(0.5);
    switch (kind) {
    case SV_GATE_H: m[0] = r; m[2] = r; m[4] = r; m[6] = -r; break;
    case SV_GATE_X: m[2] = 1; m[4] = 1; break;
    case SV_GATE_Y: m[3] = -1; m[5] = 1; break;          // [[0,-i],[i,0]]
    case SV_GATE_Z: m[0] = 1; m[6] = -1; break;
    case SV_GATE_S: m[0] = 1; m[7] = 1; break;
    case SV_GATE_T: m[0] = 1; m[6] = r; m[7] = r; break;
    case SV_GATE_RX: m[0] = c; m[3] = -s; m[5] = -s; m[6] = c; break;
    case SV_GATE_RY: m[0] = c; m[2] = -s; m[4] = s; m[6] = c; break;
    case SV_GATE_RZ: m[0] = c; m[1] = -s; m[6] = c; m[7] = s; break;
    case SV_GATE_P: m[0] = 1; m[6] = std::cos(th); m[7] = std::sin(th); break;
    default: break;
    }
}

void gate_matrix_2q(int kind, double th, double m[32]) {
    for (int i = 0; i < 32; i++) m[i] = 0.0;
    auto set = [&](int r, int c, double re, double im) { m[2 * (4 * r + c)] = re; m[2 * (4 * r + c) + 1] = im; };
    switch (kind) {
    case SV_GATE_CX:   // l = b_c + 2 b_t: l=1 <-> l=3
        set(0, 0, 1, 0); set(2, 2, 1, 0); set(1, 3, 1, 0); set(3, 1, 1, 0); break;
    case SV_GATE_CZ:
        set(0, 0, 1, 0); set(1, 1, 1, 0); set(2, 2, 1, 0); set(3, 3, -1, 0); break;
    case SV_GATE_CP:
        set(0, 0, 1, 0); set(1, 1, 1, 0); set(2, 2, 1, 0); set(3, 3, std::cos(th), std::sin(th)); break;
    case SV_GATE_SWAP:
        set(0, 0, 1, 0); set(1, 2, 1, 0); set(2, 1, 1, 0); set(3, 3, 1, 0); break;
    default: break;
    }
}

// slots that must be register bits for this gate
static uint32_t needed_slots(const GateRef &g, const int *slot_of) {
    switch (g.kind) {
    case SV_GATE_H: case SV_GATE_X: case SV_GATE_Y: case SV_GATE_RX: case SV_GATE_RY:
        return 1u << slot_of[g.q[0]];
    case SV_GATE_CX:
        return 1u << slot_of[g.q[1]];
    default:
        return 0u;
    }
}

// Thread-bit order of a phase: lane bits first. The first lanes cover
// distinct slot residues (mod 4 for 8-byte, mod 3 for 16-byte amplitudes) so
// the swizzled shared-memory accesses are conflict free; otherwise slots
// follow the preference key (lowest global qubit first for the phases that
// load or store, for coalescing).
static std::vector<int> order_thread_slots(std::vector<int> cand, const std::vector<int> &key, bool fp64) {
    std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) { return key[a] < key[b]; });
    const int mod = fp64 ? 3 : 4;
    std::vector<int> lanes, rest;
    std::vector<char> used(cand.size(), 0);
    uint32_t covered = 0;
    for (size_t i = 0; i < cand.size() && (int)lanes.size() < mod; i++) {
        int r = cand[i] % mod;
        if (!((covered >> r) & 1)) {
            covered |= 1u << r;
            lanes.push_back(cand[i]);
            used[i] = 1;
        }
    }
    for (size_t i = 0; i < cand.size(); i++)
        if (!used[i]) rest.push_back(cand[i]);
    // fill to a full warp of lanes, then warp bits, in key order
    std::vector<int> out = lanes;
    for (int s : rest) out.push_back(s);
    return out;
}

void fused_unitary(const std::vector<GateRef> &gates, const std::vector<int> &ids, const int *qs, int k,
                   std::vector<double> &U) {
    // U <- G U for each gate G in order, on the rows of the row-major 2^k x 2^k
    // matrix (the same update on every column): pairs of rows for a one-qubit
    // gate, quads for a two-qubit one
    const int D = 1 << k;
    U.assign((size_t)2 * D * D, 0.0);
    for (int i = 0; i < D; i++) U[2 * (D * i + i)] = 1.0;
    double *u = U.data();
    auto row = [&](int r) { return u + (size_t)2 * D * r; };
    for (int g : ids) {
        const GateRef &gr = gates[g];
        int loc[2] = {0, 0};
        for (int a = 0; a < gr.arity; a++)
            for (int j = 0; j < k; j++)
                if (qs[j] == gr.q[a]) loc[a] = j;
        if (gr.arity == 1) {
            double m[8];
            gate_matrix_1q(gr.kind, gr.theta, m);
            const int s = 1 << loc[0];
            for (int x = 0; x < D; x++) {
                if (x & s) continue;
                double *a = row(x), *b = row(x + s);
                for (int c = 0; c < D; c++) {
                    const double ar = a[2 * c], ai = a[2 * c + 1], br = b[2 * c], bi = b[2 * c + 1];
                    a[2 * c] = m[0] * ar - m[1] * ai + m[2] * br - m[3] * bi;
                    a[2 * c + 1] = m[0] * ai + m[1] * ar + m[2] * bi + m[3] * br;
                    b[2 * c] = m[4] * ar - m[5] * ai + m[6] * br - m[7] * bi;
                    b[2 * c + 1] = m[4] * ai + m[5] * ar + m[6] * bi + m[7] * br;
                }
            }
            continue;
        }
        const int s0 = 1 << loc[0], s1 = 1 << loc[1];   // control, target
        switch (gr.kind) {
        case SV_GATE_CX:    // rows with the control set swap their target halves
            for (int x = 0; x < D; x++)
                if ((x & s0) && !(x & s1)) std::swap_ranges(row(x), row(x) + 2 * D, row(x + s1));
            break;
        case SV_GATE_SWAP:
            for (int x = 0; x < D; x++)
                if ((x & s0) && !(x & s1)) std::swap_ranges(row(x), row(x) + 2 * D, row(x - s0 + s1));
            break;
        case SV_GATE_CZ: case SV_GATE_CP: {
            const double dr = gr.kind == SV_GATE_CZ ? -1.0 : std::cos(gr.theta);
            const double di = gr.kind == SV_GATE_CZ ? 0.0 : std::sin(gr.theta);
            for (int x = 0; x < D; x++)
                if ((x & s0) && (x & s1)) {
                    double *a = row(x);
                    for (int c = 0; c < D; c++) {
                        const double ar = a[2 * c], ai = a[2 * c + 1];
                        a[2 * c] = ar * dr - ai * di;
                        a[2 * c + 1] = ar * di + ai * dr;
                    }
                }
        } break;
        default: {   // any other two-qubit gate: its 4x4 matrix on quads of rows
            double m[32];
            gate_matrix_2q(gr.kind, gr.theta, m);
            std::vector<double> t(8);
            for (int x = 0; x < D; x++) {
                if ((x & s0) || (x & s1)) continue;
                double *rw[4] = {row(x), row(x + s0), row(x + s1), row(x + s0 + s1)};
                for (int c = 0; c < D; c++) {
                    for (int r = 0; r < 4; r++) {
                        double re = 0, im = 0;
                        for (int cc = 0; cc < 4; cc++) {
                            const double mr = m[2 * (4 * r + cc)], mi = m[2 * (4 * r + cc) + 1];
                            re += mr * rw[cc][2 * c] - mi * rw[cc][2 * c + 1];
                            im += mr * rw[cc][2 * c + 1] + mi * rw[cc][2 * c];
                        }
                        t[2 * r] = re;
                        t[2 * r + 1] = im;
                    }
                    for (int r = 0; r < 4; r++) {
                        rw[r][2 * c] = t[2 * r];
                        rw[r][2 * c + 1] = t[2 * r + 1];
                    }
                }
            }
        }
        }
    }
}

// Bank bits of the pair kernel's shared buffer: slot p < 4 keeps its bit;
// slot p >= 4 also flips the 4-bit bank-pair value v_p. A half-warp's 16
// lanes run over the slots of the lowest 4 column qubits of layout 1 (when
// writing) or layout 2 (when reading); the v_p are picked (fixed-seed search)
// so that both sets of 4 slots map to independent bank vectors, i.e. 16
// distinct bank pairs. Falls back to v_p = bit (p mod 4) if none is found.
static void pair_swizzle(DensePairLaunch &D) {
    const int NS = DENSE_K + DENSE_COLS;
    auto indep = [](const uint32_t *w) {
        uint32_t span = 1u;   // bit mask over the 16 bank values reachable
        for (int i = 0; i < 4; i++) {
            if ((span >> w[i]) & 1u) return false;
            uint32_t ns = span;
            for (uint32_t x = 0; x < 16; x++)
                if ((span >> x) & 1u) ns |= 1u << (x ^ w[i]);
            span = ns;
        }
        return true;
    };
    uint32_t v[DENSE_K + DENSE_COLS];
    uint64_t st = 0x9E3779B97F4A7C15ull;
    bool found = false;
    for (int trial = 0; trial < 4096 && !found; trial++) {
        for (int p = 0; p < NS; p++) {
            if (p < 4) v[p] = 1u << p;
            else if (trial == 0) v[p] = 1u << (p & 3);
            else {
                st = st * 6364136223846793005ull + 1442695040888963407ull;
                v[p] = 1u + (uint32_t)((st >> 33) % 15u);
            }
        }
        uint32_t w1[4], w2[4];
        for (int i = 0; i < 4; i++) {
            w1[i] = v[D.s_c1[i]];
            w2[i] = v[D.s_c2[i]];
        }
        found = indep(w1) && indep(w2);
    }
    if (!found)
        for (int p = 4; p < NS; p++) v[p] = 1u << (p & 3);
    for (int p = 0; p < NS; p++) D.xsw[p] = (uint16_t)(p < 4 ? (1u << p) : ((1u << p) | v[p]));
}

bool compile_program(const std::vector<GateRef> &gates, int n, const std::vector<uint32_t> &pog,
                     uint32_t n_parts, bool fp64, int t_cfg, int R, int dense_mode, Program &prog,
                     std::string &err, const std::vector<uint32_t> *inner) {
    prog = Program();
    prog.fp64 = fp64;
    prog.R = R;
    const int t = std::min(n, t_cfg);
    prog.t = t;
    if (t - R > MAX_TB || R > MAX_R || t < R + 5) {
        err = "tile configuration out of range";
        return false;
    }
    std::vector<std::vector<int>> members(n_parts);
    for (size_t g = 0; g < gates.size(); g++) {
        if (pog[g] >= n_parts) {
            err = "part id out of range";
            return false;
        }
        members[pog[g]].push_back((int)g);
    }
    std::vector<uint64_t> gmask(gates.size());
    for (size_t g = 0; g < gates.size(); g++) {
        uint64_t m = 0;
        for (int j = 0; j < gates[g].arity; j++) m |= 1ull << gates[g].q[j];
        gmask[g] = m;
    }
    const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    for (uint32_t pi = 0; pi < n_parts; pi++) {
        const std::vector<int> &gl = members[pi];
        if (gl.empty()) continue;
        uint64_t S = 0;
        for (int g : gl) S |= gmask[g];
        if ((dense_mode & 2) && !fp64 && popc(S) <= DENSE_K && n >= DENSE_K + DENSE_COLS && pi + 1 < n_parts &&
            !members[pi + 1].empty()) {
            // two consecutive dense parts in one pass (multi-level
            // partitioning, Sec. IV-B: a 13-qubit tile as the first level,
            // two 6-qubit products as the second); each part is padded to 6
            // with the other's qubits first, and the tile adds the lowest
            // remaining qubits; paired only if the tile holds qubits 0 and 1
            // (runs of 4 consecutive amplitudes: whole 32-byte sectors)
            uint64_t S2 = 0;
            for (int g : members[pi + 1]) S2 |= gmask[g];
            if (popc(S2) <= DENSE_K) {
                auto pad = [&](uint64_t P, uint64_t pref) {
                    for (int q = n - 1; q >= 0 && popc(P) < DENSE_K; q--)
                        if ((pref >> q) & 1) P |= 1ull << q;
                    for (int q = n - 1; q >= 0 && popc(P) < DENSE_K; q--) P |= 1ull << q;
                    return P;
                };
                const uint64_t P1 = pad(S, S2 & ~S), P2 = pad(S2, S & ~S2);
                uint64_t T = P1 | P2;
                for (int q = 0; q < n && popc(T) < DENSE_K + DENSE_COLS; q++) T |= 1ull << q;
                if ((T & 3ull) == 3ull && popc(T) == DENSE_K + DENSE_COLS) {
                    DensePairLaunch D;
                    std::memset(&D, 0, sizeof(D));
                    D.n = n;
                    D.outer_mask = all & ~T;
                    int f = 0;
                    while (f < 4 && ((T >> f) & 1)) f++;
                    D.prefetch = (uint8_t)f;
                    int slot = 0, j1 = 0, c1 = 0, j2 = 0, c2 = 0, qs1[DENSE_K], qs2[DENSE_K];
                    for (int q = 0; q < n; q++) {
                        if (!((T >> q) & 1)) continue;
                        if ((P1 >> q) & 1) { qs1[j1] = q; D.s_q1[j1] = (uint8_t)slot; D.q1[j1++] = (uint8_t)q; }
                        else { D.s_c1[c1] = (uint8_t)slot; D.c1[c1++] = (uint8_t)q; }
                        if ((P2 >> q) & 1) { qs2[j2] = q; D.s_q2[j2] = (uint8_t)slot; D.q2[j2++] = (uint8_t)q; }
                        else { D.s_c2[c2] = (uint8_t)slot; D.c2[c2++] = (uint8_t)q; }
                        slot++;
                    }
                    pair_swizzle(D);
                    std::vector<double> U;
                    std::vector<uint8_t> img;
                    fused_unitary(gates, gl, qs1, DENSE_K, U);
                    dense_a_image(U.data(), img);
                    prog.pair_img.insert(prog.pair_img.end(), img.begin(), img.end());
                    fused_unitary(gates, members[pi + 1], qs2, DENSE_K, U);
                    dense_a_image(U.data(), img);
                    prog.pair_img.insert(prog.pair_img.end(), img.begin(), img.end());
                    prog.kind.push_back(2);
                    prog.index.push_back((uint32_t)prog.pairs.size());
                    prog.pairs.push_back(D);
                    prog.pair_tiles.push_back(1ull << (n - DENSE_K - DENSE_COLS));
                    pi++;   // the second part is done
                    continue;
                }
            }
        }
        if ((dense_mode & 1) && !fp64 && popc(S) <= DENSE_K && n >= DENSE_K + DENSE_COLS) {
            // dense part: the part's qubits padded to 6 with the highest others
            // (the unitary is the identity on them), columns on the lowest 7
            // remaining qubits, so that the 32 lanes of a warp (columns) stay
            // consecutive amplitudes unless the part itself holds low qubits
            uint64_t P = S, C = 0;
            for (int q = n - 1; q >= 0 && popc(P) < DENSE_K; q--) P |= 1ull << q;
            for (int q = 0; q < n && popc(C) < DENSE_COLS; q++)
                if (!((P >> q) & 1)) C |= 1ull << q;
            DenseLaunch D;
            std::memset(&D, 0, sizeof(D));
            D.n = n;
            D.outer_mask = all & ~(P | C);
            int qs[DENSE_K], jp = 0, jc = 0, js = 0;
            for (int q = 0; q < n; q++) {
                if ((P >> q) & 1) {
                    qs[jp] = q;
                    D.part_q[jp++] = (uint8_t)q;
                    D.slot_part |= (uint16_t)(1u << js);
                    D.slot_q[js++] = (uint8_t)q;
                } else if ((C >> q) & 1) {
                    D.col_q[jc++] = (uint8_t)q;
                    D.slot_q[js++] = (uint8_t)q;
                }
            }
            std::vector<double> U;
            fused_unitary(gates, gl, qs, DENSE_K, U);
            std::vector<uint8_t> img;
            dense_a_image(U.data(), img);
            prog.kind.push_back(1);
            prog.index.push_back((uint32_t)prog.dense.size());
            prog.dense.push_back(D);
            prog.dense_tiles.push_back(1ull << (n - DENSE_K - DENSE_COLS));
            prog.a_img.insert(prog.a_img.end(), img.begin(), img.end());
            continue;
        }
        if (popc(S) > t) {
            err = "part " + std::to_string(pi) + " has " + std::to_string(popc(S)) + " qubits > tile " + std::to_string(t);
            return false;
        }
        uint64_t Tm = S;
        for (int q = 0; q < n && popc(Tm) < t; q++) Tm |= 1ull << q;
        int slot_of[64], q_at[64];
        for (int q = 0, p = 0; q < n; q++)
            if ((Tm >> q) & 1) {
                slot_of[q] = p;
                q_at[p] = q;
                p++;
            }
        PartLaunch L;
        std::memset(&L, 0, sizeof(L));
        L.outer_mask = all & ~Tm;
        L.n = n;
        L.t = t;
        L.phase_begin = (uint32_t)prog.phases.size();
        L.op_begin = (uint32_t)prog.ops.size();
        L.coef_begin = (uint32_t)prog.coefs.size();
        for (int p = 0; p < t; p++) L.tile_q[p] = (uint8_t)q_at[p];
        // part factor: 1/sqrt2 per (unnormalised) H and e^{-i theta/2} per RZ
        double fr = 1.0, fi = 0.0;
        auto fmul = [&](double dr, double di) {
            const double x = fr, y = fi;
            fr = x * dr - y * di;
            fi = x * di + y * dr;
        };
        bool last_tphase = false;
        std::vector<int> remaining = gl;
        bool first = true;
        while (!remaining.empty()) {
            // pass 1: choose the register slots and the gates of this phase
            int sim_slot[64];
            std::memcpy(sim_slot, slot_of, sizeof(slot_of));
            uint32_t Rset = 0;
            uint64_t blocked = 0;
            std::vector<int> sched, rest;
            if (inner && !inner->empty()) {
                // multi-level partitioning: the phase is the next second-level
                // part (the smallest inner id left; its gates in order)
                uint32_t next = UINT32_MAX;
                for (int g : remaining) next = std::min(next, (*inner)[g]);
                for (int g : remaining) {
                    if ((*inner)[g] != next) {
                        rest.push_back(g);
                        continue;
                    }
                    const GateRef &gr = gates[g];
                    Rset |= needed_slots(gr, sim_slot);
                    sched.push_back(g);
                    if (gr.kind == SV_GATE_SWAP) std::swap(sim_slot[gr.q[0]], sim_slot[gr.q[1]]);
                }
                if (popc(Rset) > R) {
                    err = "a second-level part needs " + std::to_string(popc(Rset)) + " register qubits > " +
                          std::to_string(R);
                    return false;
                }
            } else
            for (int g : remaining) {
                const GateRef &gr = gates[g];
                if (gmask[g] & blocked) {
                    blocked |= gmask[g];
                    rest.push_back(g);
                    continue;
                }
                uint32_t need = needed_slots(gr, sim_slot);
                if ((need & ~Rset) && popc(Rset | need) > R) {
                    blocked |= gmask[g];
                    rest.push_back(g);
                    continue;
                }
                Rset |= need;
                sched.push_back(g);
                if (gr.kind == SV_GATE_SWAP) std::swap(sim_slot[gr.q[0]], sim_slot[gr.q[1]]);
            }
            for (int p = t - 1; p >= 0 && popc(Rset) < R; p--) Rset |= 1u << p;
            const bool last = rest.empty();
            // slot -> qubit at the start and at the end of this phase
            int q_end[64];
            for (int q = 0; q < n; q++)
                if ((Tm >> q) & 1) q_end[sim_slot[q]] = q;
            Phase ph;
            std::memset(&ph, 0, sizeof(ph));
            int rb[64], tbit[64];
            for (int p = 0, b = 0; p < t; p++)
                if ((Rset >> p) & 1) {
                    ph.reg[b] = (uint8_t)p;
                    rb[p] = b++;
                }
            std::vector<int> cand;
            std::vector<int> key(t, 0);
            for (int p = 0; p < t; p++) {
                if (!((Rset >> p) & 1)) cand.push_back(p);
                key[p] = last ? q_end[p] : p;   // the last phase stores: lanes on the lowest qubits
            }
            std::vector<int> thr = order_thread_slots(cand, key, fp64);
            for (size_t j = 0; j < thr.size(); j++) {
                ph.thr[j] = (uint8_t)thr[j];
                tbit[thr[j]] = (int)j;
            }
            // pass 2: emit ops
            ph.op_begin = (uint32_t)prog.ops.size();
            bool tphase = false;
            auto coef = [&](std::initializer_list<double> v) {
                uint32_t at = (uint32_t)prog.coefs.size();
                prog.coefs.insert(prog.coefs.end(), v.begin(), v.end());
                return at;
            };
            auto emit = [&](uint8_t kind, int a, int b, int tb, uint32_t c) {
                Op op;
                op.kind = kind;
                op.a = (uint8_t)a;
                op.b = (uint8_t)b;
                op.tb = (uint8_t)tb;
                op.coef = c;
                prog.ops.push_back(op);
            };
            // one gate's ops (the gate alone)
            auto emit_one = [&](int g) -> bool {
                const GateRef &gr = gates[g];
                const double th = gr.theta;
                const int s0 = slot_of[gr.q[0]];
                const bool r0 = (Rset >> s0) & 1;
                switch (gr.kind) {
                case SV_GATE_H:
                    emit(OP_H, rb[s0], 0, 0, 0);
                    fmul(std::sqrt(0.5), 0.0);
                    break;
                case SV_GATE_X: emit(OP_X, rb[s0], 0, 0, 0); break;
                case SV_GATE_Y: emit(OP_Y, rb[s0], 0, 0, 0); break;
                case SV_GATE_RX: case SV_GATE_RY: {
                    // the largest entry joins the part factor: RX = c [[1, -it], [-it, 1]]
                    // (t = s/c) or -is [[it, 1], [1, it]] (t = c/s); RY = c [[1, -t], [t, 1]]
                    // or s [[t, -1], [1, t]], whichever keeps |t| <= 1
                    const double c = std::cos(th / 2), sn = std::sin(th / 2);
                    const bool rx = gr.kind == SV_GATE_RX;
                    if (std::fabs(c) >= std::fabs(sn)) {
                        fmul(c, 0.0);
                        emit(rx ? OP_RXS : OP_RYS, rb[s0], 0, 0, coef({sn / c}));
                    } else {
                        if (rx) fmul(0.0, -sn);
                        else fmul(sn, 0.0);
                        emit(rx ? OP_RXS : OP_RYS, rb[s0], 1, 0, coef({c / sn}));
                    }
                } break;
                case SV_GATE_Z: case SV_GATE_S: case SV_GATE_T: case SV_GATE_P: {
                    double ang = gr.kind == SV_GATE_Z ? M_PI : gr.kind == SV_GATE_S ? M_PI / 2 : gr.kind == SV_GATE_T ? M_PI / 4 : th;
                    double dr = gr.kind == SV_GATE_Z ? -1.0 : std::cos(ang), di = gr.kind == SV_GATE_Z ? 0.0 : std::sin(ang);
                    if (gr.kind == SV_GATE_S) { dr = 0.0; di = 1.0; }
                    if (r0) {
                        if (gr.kind == SV_GATE_Z) emit(OP_Z, rb[s0], 0, 0, 0);
                        else emit(OP_P, rb[s0], 0, 0, coef({dr, di}));
                    } else {
                        emit(OP_TD, 0, 0, tbit[s0], coef({1.0, 0.0, dr, di}));
                        tphase = true;
                    }
                } break;
                case SV_GATE_RZ: {
                    // RZ(t) = e^{-it/2} diag(1, e^{it}): the global phase joins the part factor
                    fmul(std::cos(th / 2), -std::sin(th / 2));
                    if (r0) emit(OP_P, rb[s0], 0, 0, coef({std::cos(th), std::sin(th)}));
                    else {
                        emit(OP_TD, 0, 0, tbit[s0], coef({1.0, 0.0, std::cos(th), std::sin(th)}));
                        tphase = true;
                    }
                } break;
                case SV_GATE_CX: {
                    const int s1 = slot_of[gr.q[1]];
                    if (r0) emit(OP_CX, rb[s0], rb[s1], 0, 0);
                    else emit(OP_CXT, 0, rb[s1], tbit[s0], 0);
                } break;
                case SV_GATE_CZ: case SV_GATE_CP: {
                    const int s1 = slot_of[gr.q[1]];
                    const bool r1 = (Rset >> s1) & 1;
                    const bool cz = gr.kind == SV_GATE_CZ;
                    const double dr = cz ? -1.0 : std::cos(th), di = cz ? 0.0 : std::sin(th);
                    if (r0 && r1) {
                        if (cz) emit(OP_CZ, rb[s0], rb[s1], 0, 0);
                        else emit(OP_CP, rb[s0], rb[s1], 0, coef({dr, di}));
                    } else if (r0 || r1) {
                        const int rs = r0 ? s0 : s1, ts = r0 ? s1 : s0;
                        if (cz) emit(OP_CZT, rb[rs], 0, tbit[ts], 0);
                        else emit(OP_CPT, rb[rs], 0, tbit[ts], coef({dr, di}));
                    } else {
                        emit(OP_TP2, 0, tbit[s1], tbit[s0], coef({dr, di}));
                        tphase = true;
                    }
                } break;
                case SV_GATE_SWAP:
                    std::swap(slot_of[gr.q[0]], slot_of[gr.q[1]]);
                    break;
                default:
                    err = "unknown gate kind";
                    return false;
                }
                return true;
            };
            // Runs of one-qubit gates on one qubit with no multi-qubit gate on it
            // in between (gates on other qubits commute with them) become one
            // op: their product, as a phase (diagonal; the entry of |0> joins
            // the part factor) or a general 2x2 matrix.
            auto emit_fused = [&](int q, const std::vector<int> &run) -> bool {
                if (run.size() == 1) return emit_one(run[0]);
                double M[8] = {1, 0, 0, 0, 0, 0, 1, 0};
                for (int g : run) {
                    double U[8], T[8];
                    gate_matrix_1q(gates[g].kind, gates[g].theta, U);
                    for (int r = 0; r < 2; r++)
                        for (int c = 0; c < 2; c++) {
                            double re = 0, im = 0;
                            for (int k = 0; k < 2; k++) {
                                const double ar = U[2 * (2 * r + k)], ai = U[2 * (2 * r + k) + 1];
                                const double br = M[2 * (2 * k + c)], bi = M[2 * (2 * k + c) + 1];
                                re += ar * br - ai * bi;
                                im += ar * bi + ai * br;
                            }
                            T[2 * (2 * r + c)] = re;
                            T[2 * (2 * r + c) + 1] = im;
                        }
                    std::memcpy(M, T, sizeof(M));
                }
                const int sq = slot_of[q];
                const double off = std::hypot(M[2], M[3]) + std::hypot(M[4], M[5]);
                if (off < 1e-14) {
                    // diag(m00, m11) = m00 diag(1, m11 / m00), |m00| = 1
                    const double d0r = M[0], d0i = M[1], d1r = M[6], d1i = M[7];
                    fmul(d0r, d0i);
                    const double pr = d1r * d0r + d1i * d0i, pi = d1i * d0r - d1r * d0i;
                    if (std::fabs(pr - 1.0) < 1e-15 && std::fabs(pi) < 1e-15) return true;   // identity
                    if ((Rset >> sq) & 1) emit(OP_P, rb[sq], 0, 0, coef({pr, pi}));
                    else {
                        emit(OP_TD, 0, 0, tbit[sq], coef({1.0, 0.0, pr, pi}));
                        tphase = true;
                    }
                    return true;
                }
                if (!((Rset >> sq) & 1)) {
                    err = "fused non-diagonal gate on a thread slot";
                    return false;
                }
                // divide by the larger of m00 and m01 (the part factor takes it):
                // [[1, u], [v, w]] or [[u, 1], [v, w]], entries of modulus <= 1
                {
                    const bool f1 = std::hypot(M[2], M[3]) > std::hypot(M[0], M[1]);
                    const double pr = f1 ? M[2] : M[0], pi = f1 ? M[3] : M[1];
                    const double den = pr * pr + pi * pi;
                    auto div = [&](double xr, double xi, double &qr, double &qi) {
                        qr = (xr * pr + xi * pi) / den;
                        qi = (xi * pr - xr * pi) / den;
                    };
                    double ur, ui, vr, vi, wr, wi;
                    div(f1 ? M[0] : M[2], f1 ? M[1] : M[3], ur, ui);
                    div(M[4], M[5], vr, vi);
                    div(M[6], M[7], wr, wi);
                    fmul(pr, pi);
                    emit(OP_U2S, rb[sq], f1 ? 1 : 0, 0, coef({ur, ui, vr, vi, wr, wi}));
                }
                return true;
            };
            std::vector<std::vector<int>> pend(n);
            std::vector<int> pend_order;
            auto flush = [&](int q) -> bool {
                if (pend[q].empty()) return true;
                const bool ok = emit_fused(q, pend[q]);
                pend[q].clear();
                return ok;
            };
            for (int g : sched) {
                const GateRef &gr = gates[g];
                if (gr.arity == 1) {
                    if (pend[gr.q[0]].empty()) pend_order.push_back(gr.q[0]);
                    pend[gr.q[0]].push_back(g);
                    continue;
                }
                for (int j = 0; j < gr.arity; j++)
                    if (!flush(gr.q[j])) return false;
                if (!emit_one(g)) return false;
            }
            for (int q : pend_order)
                if (!flush(q)) return false;
            // the last phase's per-thread phase is applied with the part factor at the store
            // Diagonal gates on register bits commute with each other and with
            // every op on other register bits: a run of them (interleaved with
            // such ops) merges into one OP_DIAG holding the product's phase for
            // each of the 2^R register indices. The run ends where an op acts
            // non-diagonally on a register bit the product depends on.
            {
                const int NR = 1 << R;
                std::vector<Op> in(prog.ops.begin() + ph.op_begin, prog.ops.end());
                prog.ops.resize(ph.op_begin);
                std::vector<double> D(2 * NR);
                uint32_t dep = 0;
                int merged = 0;
                Op single{};
                auto reset = [&]() {
                    for (int i = 0; i < NR; i++) { D[2 * i] = 1.0; D[2 * i + 1] = 0.0; }
                    dep = 0;
                    merged = 0;
                };
                auto mulphase = [&](int i, double pr, double pi) {
                    const double x = D[2 * i], y = D[2 * i + 1];
                    D[2 * i] = x * pr - y * pi;
                    D[2 * i + 1] = x * pi + y * pr;
                };
                auto flush = [&]() {
                    if (merged == 1) prog.ops.push_back(single);
                    else if (merged > 1) {
                        Op op{};
                        op.kind = OP_DIAG;
                        op.coef = (uint32_t)prog.coefs.size();
                        prog.coefs.insert(prog.coefs.end(), D.begin(), D.end());
                        prog.ops.push_back(op);
                    }
                    reset();
                };
                reset();
                for (const Op &op : in) {
                    const double *c = prog.coefs.data() + op.coef;
                    bool diag = true;
                    switch (op.kind) {
                    case OP_P: for (int i = 0; i < NR; i++) if ((i >> op.a) & 1) mulphase(i, c[0], c[1]); break;
                    case OP_Z: for (int i = 0; i < NR; i++) if ((i >> op.a) & 1) mulphase(i, -1.0, 0.0); break;
                    case OP_D:
                        for (int i = 0; i < NR; i++) mulphase(i, (i >> op.a) & 1 ? c[2] : c[0], (i >> op.a) & 1 ? c[3] : c[1]);
                        break;
                    case OP_CZ:
                        for (int i = 0; i < NR; i++) if (((i >> op.a) & 1) && ((i >> op.b) & 1)) mulphase(i, -1.0, 0.0);
                        break;
                    case OP_CP:
                        for (int i = 0; i < NR; i++) if (((i >> op.a) & 1) && ((i >> op.b) & 1)) mulphase(i, c[0], c[1]);
                        break;
                    default: diag = false; break;
                    }
                    if (diag) {
                        dep |= 1u << op.a;
                        if (op.kind == OP_CZ || op.kind == OP_CP) dep |= 1u << op.b;
                        merged++;
                        single = op;
                        continue;
                    }
                    // register bits the op acts on non-diagonally
                    uint32_t touch = 0;
                    switch (op.kind) {
                    case OP_H: case OP_U2: case OP_RX: case OP_RY: case OP_X: case OP_Y: case OP_RXS: case OP_RYS:
                    case OP_U2S: touch = 1u << op.a; break;
                    case OP_CX: touch = (1u << op.a) | (1u << op.b); break;
                    case OP_CXT: touch = 1u << op.b; break;
                    default: touch = 0; break;   // thread-bit phases: diagonal, they commute
                    }
                    if (touch & dep) flush();
                    prog.ops.push_back(op);
                }
                flush();
            }
            if (tphase && !last) emit(OP_TAPPLY, 0, 0, 0, 0);
            if (last) last_tphase = tphase;
            ph.op_count = (uint32_t)prog.ops.size() - ph.op_begin;
            prog.phases.push_back(ph);
            if (last) {
                for (int b = 0; b < R; b++) L.store_reg_q[b] = (uint8_t)q_end[ph.reg[b]];
                for (int j = 0; j < t - R; j++) L.store_thr_q[j] = (uint8_t)q_end[ph.thr[j]];
            }
            remaining.swap(rest);
            first = false;
        }
        L.n_phases = (uint32_t)prog.phases.size() - L.phase_begin;
        L.op_end = (uint32_t)prog.ops.size();
        L.coef_end = (uint32_t)prog.coefs.size();
        // the part factor is one complex scalar: any op that multiplies every
        // amplitude by a per-index phase (a merged diagonal) takes it into its
        // coefficients, which saves the multiply at the store unless the last
        // phase also left a per-thread phase to apply there
        if (!last_tphase && (fr != 1.0 || fi != 0.0)) {
            for (uint32_t o = L.op_begin; o < (uint32_t)prog.ops.size(); o++) {
                if (prog.ops[o].kind != OP_DIAG) continue;
                double *c = prog.coefs.data() + prog.ops[o].coef;
                for (int i = 0; i < (1 << R); i++) {
                    const double x = c[2 * i], y = c[2 * i + 1];
                    c[2 * i] = x * fr - y * fi;
                    c[2 * i + 1] = x * fi + y * fr;
                }
                fr = 1.0;
                fi = 0.0;
                break;
            }
        }
        L.gr = fr;
        L.gi = fi;
        L.flags = (last_tphase || fr != 1.0 || fi != 0.0) ? PL_STORE_FACTOR : 0u;
        prog.kind.push_back(0);
        prog.index.push_back((uint32_t)prog.parts.size());
        prog.parts.push_back(L);
        prog.n_tiles.push_back(1ull << (n - t));
    }
    return true;
}

// Real floating-point operations per amplitude of the whole state that the
// program's kernels execute (an FMA counts two; sign changes, permutations
// and shared-memory moves count none): per op of a gate-list part, the
// arithmetic of its template in ops_core.cuh over the amplitudes it touches,
// plus the store factor; per dense part, the split-BF16 products (3 x 128
// real MACs per real output, 1536 per complex amplitude, tensor cores).
void program_flops(const Program &prog, double &alu_per_amp, double &tensor_per_amp) {
    alu_per_amp = 0.0;
    tensor_per_amp = 0.0;
    const int NR = 1 << prog.R;
    for (size_t i = 0; i < prog.kind.size(); i++) {
        if (prog.kind[i] == 1 || prog.kind[i] == 2) {
            tensor_per_amp += (prog.kind[i] == 2 ? 2.0 : 1.0) * 2.0 * 3.0 * 2.0 * 128.0;
            continue;
        }
        const PartLaunch &L = prog.parts[prog.index[i]];
        for (uint32_t p = 0; p < L.n_phases; p++) {
            const Phase &ph = prog.phases[L.phase_begin + p];
            for (uint32_t k = 0; k < ph.op_count; k++) {
                const Op &op = prog.ops[ph.op_begin + k];
                switch (op.kind) {
                case OP_H: alu_per_amp += 2.0; break;                 // a + b, a - b per component pair
                case OP_RX: case OP_RY: alu_per_amp += 6.0; break;    // c x + s y per component
                case OP_U2: alu_per_amp += 14.0; break;               // 2x2 complex matrix-vector
                case OP_RXS: case OP_RYS: alu_per_amp += 4.0; break;  // one multiply-add per component
                case OP_U2S: alu_per_amp += 11.0; break;              // x + u y (8), v x + w y (14) per pair
                case OP_D: case OP_DIAG: case OP_TAPPLY: alu_per_amp += 6.0; break;   // complex product, all
                case OP_P: case OP_CPT: alu_per_amp += 3.0; break;    // complex product on half
                case OP_CP: alu_per_amp += 1.5; break;                // complex product on a quarter
                default: break;                                       // X, Y, Z, CX, CZ, SWAP, thread phases
                }
            }
        }
        if (L.flags & PL_STORE_FACTOR) alu_per_amp += 6.0;
        (void)NR;
    }
}

}  // namespace hisv
