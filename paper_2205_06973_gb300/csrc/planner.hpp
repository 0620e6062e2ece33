// Part planner: turns a partition into the device program of the part kernel.
#pragma once
#include <string>
#include <vector>

#include "dense.hpp"
#include "partition.hpp"
#include "program.hpp"

namespace hisv {

struct Program {
    bool fp64 = false;
    int t = 0;                           // tile qubits
    int R = 0;                           // register bits per thread
    std::vector<PartLaunch> parts;       // in execution order
    std::vector<uint64_t> n_tiles;       // CTAs (outer assignments) per part
    std::vector<Phase> phases;
    std::vector<Op> ops;
    std::vector<double> coefs;
    // execution order over all parts: kind 0 = gate-list part parts[index],
    // kind 1 = dense tensor-core part dense[index] (A image a_img[index]),
    // kind 2 = two dense parts in one pass pairs[index] (images
    // pair_img[2 index], pair_img[2 index + 1])
    std::vector<uint8_t> kind;
    std::vector<uint32_t> index;
    std::vector<DenseLaunch> dense;
    std::vector<uint64_t> dense_tiles;
    std::vector<uint8_t> a_img;           // DENSE_A_BYTES per dense part
    std::vector<DensePairLaunch> pairs;
    std::vector<uint64_t> pair_tiles;
    std::vector<uint8_t> pair_img;        // 2 x DENSE_A_BYTES per pair
};

// Gate matrices of the library (row-major complex, interleaved re/im):
// 2x2 for 1-qubit kinds, 4x4 with local index l = b_q0 + 2 b_q1 for 2-qubit.
void gate_matrix_1q(int kind, double theta, double m[8]);
void gate_matrix_2q(int kind, double theta, double m[32]);
bool gate_is_two_qubit(int kind);

// Compile the parts (part_of_gate numbered in execution order) for a tile of
// t_cfg qubits (t = min(n, t_cfg)) and R register bits.
// dense_mode: bit 0 = every part of at most 6 qubits runs as a dense
// tensor-core part (complex64, n >= 13); bit 1 = two consecutive such parts
// run in one pass where their qubits and qubits 0, 1 fit a 13-qubit tile.
// inner (optional): the second-level part of every gate (multi-level
// partitioning, Sec. IV-B); each becomes one register phase of its
// first-level part instead of the greedy phase split (error if one needs
// more than R register qubits).
bool compile_program(const std::vector<GateRef> &gates, int n, const std::vector<uint32_t> &pog,
                     uint32_t n_parts, bool fp64, int t_cfg, int R, int dense_mode, Program &prog,
                     std::string &err, const std::vector<uint32_t> *inner = nullptr);

// Floating-point operations per state amplitude that the program's kernels
// execute: CUDA-core arithmetic (alu) and tensor-core products (tensor).
void program_flops(const Program &prog, double &alu_per_amp, double &tensor_per_amp);

// Fused unitary of gates acting on the qubits qs[0..k) (local bit j <-> qs[j]):
// U = G_last ... G_first as a 2^k x 2^k row-major interleaved complex matrix.
void fused_unitary(const std::vector<GateRef> &gates, const std::vector<int> &ids, const int *qs, int k,
                   std::vector<double> &U);

}  // namespace hisv
