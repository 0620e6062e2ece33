// Device program of one plan: the per-part instructions the part kernel runs.
//
// A part (Sec. IV-A) touches at most k qubits. Its tile is the part's qubits
// padded with the lowest remaining qubits up to t (the padding of Sec. IV-B,
// multi-level partitioning, for spatial locality); one CTA owns one tile =
// one binary assignment of the n - t outer qubits (Algorithm 1, outer loop).
// Tile positions 0..t-1 are slots; slot p holds one qubit of the tile.
//
// Inside a CTA the 2^t amplitudes live in registers: 2^R per thread. A phase
// fixes which R slots are register bits (the rest are thread-index bits:
// 5 lane bits, then warp bits). All gates of a phase act on register bits
// only, except diagonal gates and controls, which may sit on thread bits.
// Between phases the tile is transposed through shared memory. This is a
// second level of partitioning inside the part, with limit R (Sec. IV-B,
// multi-level partitioning), chosen greedily along the part's gate order.
#pragma once
#include <cstdint>

namespace hisv {

enum OpKind : uint8_t {
    OP_H = 0,    // a: reg bit; unnormalised (a+b, a-b), the 1/sqrt2 goes into the part factor
    OP_U2,       // a; coef: m00 m01 m10 m11 (re, im each) -> 8 reals
    OP_RX,       // a; coef: c, s
    OP_RY,       // a; coef: c, s
    OP_X,        // a
    OP_Y,        // a
    OP_D,        // a; coef: d0 (re, im), d1 (re, im)  (diagonal)
    OP_P,        // a; coef: d1 (re, im)               (diag(1, d1); RZ = e^{-it/2} P(t))
    OP_Z,        // a                                  (diag(1, -1))
    OP_CX,       // a = control reg bit, b = target reg bit
    OP_CP,       // a, b reg bits; coef: d (re, im) on |11>
    OP_CZ,       // a, b reg bits
    OP_CXT,      // b = target reg bit, tb = control thread bit
    OP_CPT,      // a = reg bit, tb = thread bit; coef: d
    OP_CZT,      // a = reg bit, tb = thread bit
    OP_TD,       // tb; coef: d0, d1: per-thread phase *= (bit ? d1 : d0)
    OP_TP2,      // tb, b = second thread bit; coef: d: per-thread phase *= d if both set
    OP_TAPPLY,   // multiply the thread's amplitudes by its phase, reset the phase to 1
    OP_DIAG,     // coef: 2^R phases (re, im): register amplitude i *= phase i (merged diagonal gates)
    // Rotations with their largest entry factored out into the part factor
    // (one multiply-add per output component instead of two); b = form:
    OP_RXS,      // a; coef t. b = 0: RX = c [[1, -it], [-it, 1]], t = s/c; b = 1: RX = -is [[it, 1], [1, it]], t = c/s
    OP_RYS,      // a; coef t. b = 0: RY = c [[1, -t], [t, 1]], t = s/c;    b = 1: RY = s [[t, -1], [1, t]], t = c/s
    OP_U2S,      // a; coef u, v, w (re, im). b = 0: m00 [[1, u], [v, w]]; b = 1: m01 [[u, 1], [v, w]]
    OP_COUNT
};

struct Op {
    uint8_t kind;
    uint8_t a;
    uint8_t b;
    uint8_t tb;
    uint32_t coef;   // index of the first coefficient (in reals)
};

constexpr int MAX_R = 6;
constexpr int MAX_TB = 16;

struct Phase {
    uint8_t reg[8];          // tile slot of register bit b (b < R)
    uint8_t thr[MAX_TB];     // tile slot of thread bit j (j < t - R)
    uint32_t op_begin;
    uint32_t op_count;
};
static_assert(sizeof(Phase) == 32, "Phase layout");

// Launch record of one part (passed by value to the kernel).
struct PartLaunch {
    uint64_t outer_mask;     // qubits outside the tile (deposit target of the tile index)
    uint32_t phase_begin;
    uint32_t n_phases;
    int32_t n;
    int32_t t;
    uint32_t flags;          // PL_STORE_FACTOR: multiply by (gr, gi) x per-thread phase at the store
    uint32_t pad;
    uint32_t op_begin, op_end;      // this part's ops and coefficients (contiguous ranges); the
    uint32_t coef_begin, coef_end;  // kernel stages them in shared memory when they fit
    double gr, gi;           // part factor: 2^{-h/2} for h unnormalised H gates times RZ global phases
    uint8_t tile_q[32];      // global qubit of tile slot p (p < t); the gather/copy layout
    uint8_t store_reg_q[8];  // global qubit of register bit b in the last phase (after SWAP relabels)
    uint8_t store_thr_q[MAX_TB];
};

constexpr uint32_t PL_STORE_FACTOR = 1u;
constexpr uint32_t PROG_SMEM_BYTES = 8192;   // per-CTA shared-memory copy of one part's program

}  // namespace hisv
