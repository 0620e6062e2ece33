// Gate DAG and acyclic part builders (host, exact integer code).
//
// Sec. IV-A: gates are vertices, qubit wires are edges, every qubit has an
// entry and an exit vertex; a part's working set L is its number of distinct
// qubits; parts are disjoint, exhaustive, non-empty, L <= k, with an acyclic
// part graph. Sec. IV-B: Nat, DFS and dagP builders. The readings of the
// details the paper leaves open are stated at each builder in partition.cpp.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace hisv {

struct GateRef {
    int kind;
    int arity;
    int q[3];
    double theta;
};

struct Dag {
    int n = 0;
    int G = 0;
    std::vector<uint64_t> qmask;                 // qubits of each gate
    std::vector<std::vector<int>> preds, succs;  // distinct neighbours, operand order
    std::vector<std::vector<int>> qubits;
};

// Builds the DAG; returns false with a message on a bad qubit index.
bool build_dag(const std::vector<GateRef> &gates, int n, Dag &dag, std::string &err);

// All builders return part_of_gate with parts numbered in schedule order
// (Kahn order of the part graph keyed by each part's smallest gate index).
std::vector<uint32_t> part_nat(const Dag &dag, int k);
std::vector<uint32_t> part_dfs(const Dag &dag, int k, uint64_t seed, int trials);
std::vector<uint32_t> part_dagp(const Dag &dag, int k);
// The minimum number of parts (breadth-first search over down-sets); small
// circuits only (<= 256 gates, bounded search), false with a message beyond.
bool part_exact(const Dag &dag, int k, std::vector<uint32_t> &pog, std::string &err);
// Beam search over down-sets with parts grown from each available gate (any
// circuit size); width <= 0: 16.
std::vector<uint32_t> part_beam(const Dag &dag, int k, int width);
std::vector<uint32_t> schedule_parts(const Dag &dag, const std::vector<uint32_t> &pog);
// One builder by its method code (1 Nat, 2 DFS, 3 dagP, 4 exact, 5 beam;
// trials = DFS trials or beam width).
bool run_builder(const Dag &dag, int method, int k, uint64_t seed, int trials, std::vector<uint32_t> &pog,
                 std::string &err);
// Multi-level partitioning (Sec. IV-B): first level with builder m1 under
// k1, then each first-level part re-partitioned with builder m2 under k2.
// outer = first-level part of each gate (schedule order); inner = global
// second-level part (first-level order, then each part's own schedule).
bool part_multilevel(const std::vector<GateRef> &gates, int n, int m1, int k1, int m2, int k2, uint64_t seed,
                     int trials, std::vector<uint32_t> &outer, std::vector<uint32_t> &inner, std::string &err);

}  // namespace hisv
