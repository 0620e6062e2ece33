// Dense fused-part path: a part acting on 6 qubits is applied as one 64x64
// complex matrix, i.e. a 128x128 real GEMM on interleaved (re, im) data, on
// the tcgen05 tensor cores in split BF16 (X_hi R_hi + X_lo R_hi + X_hi R_lo,
// FP32 accumulation in tensor memory), 128 state columns per tile.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace hisv {

constexpr int DENSE_K = 6;                    // qubits of a dense part
constexpr int DENSE_COLS = 7;                 // column qubits of one tile (128 columns)
constexpr int DENSE_A_BYTES = 64 * 1024;      // R image: [hi, lo] x [k-block 0, 1] x 128 rows x 128 B

// Launch record of one dense part (by value).
struct DenseLaunch {
    uint64_t outer_mask;       // qubits outside the tile: the tile index is deposited here
    int32_t n;
    uint8_t part_q[DENSE_K];   // qubit of local bit j of the 64-amplitude vector (ascending)
    uint8_t col_q[DENSE_COLS]; // qubit of column bit j (ascending)
    uint8_t slot_q[16];        // the 13 tile qubits in ascending order (gather layout)
    uint16_t slot_part;        // bit s set: slot s is a part qubit
    uint16_t pad;
};

// Launch record of a pass that applies two dense parts (by value): the tile
// is the 13 qubits T = P1 u P2 u (lowest others); layout j has its part's
// qubits as rows and the 7 other tile qubits as columns. s_* are the slots
// (0..12, ascending qubit order of T) of those qubits.
struct DensePairLaunch {
    uint64_t outer_mask;       // qubits outside the tile
    int32_t n;
    uint8_t q1[DENSE_K], c1[DENSE_COLS], q2[DENSE_K], c2[DENSE_COLS];
    uint8_t s_q1[DENSE_K], s_c1[DENSE_COLS], s_q2[DENSE_K], s_c2[DENSE_COLS];
    uint8_t prefetch;          // f: qubits 0..f-1 are tile qubits (2 <= f <= 4): L2 warm-up by runs of 2^f
    uint8_t pad[3];
    // shared-buffer element offset of each tile slot (XOR-linear in the slot
    // bits; bits above 3 keep their place, the low 4 bits pick the bank
    // pair): chosen so that the 16 lanes of a half-warp, which run over the
    // slots of the lowest 4 column qubits of either layout, hit 16 distinct
    // bank pairs
    uint16_t xsw[DENSE_K + DENSE_COLS];
};

// Host: build the A image of a 64x64 complex unitary U (row-major, interleaved
// re/im doubles): real block form R[2i+c][2j+d], split to BF16 hi/lo, laid out
// K-major with the 128-byte swizzle the tensor-core descriptors expect.
void dense_a_image(const double *U, std::vector<uint8_t> &img);

// One dense pass. d_norms: FP64 accumulators of one apply, zeroed before its
// first dense pass: [0] = input sum |a|^2 (summed by dense pass 0), [1 + j] =
// output sum of dense pass j. Pass j > 0 rescales its output by
// sqrt([0] / [j]) (the exact evolution is unitary), which removes the norm
// drift of the split-BF16 tensor-core arithmetic.
cudaError_t launch_dense6(void *sv, const DenseLaunch &L, const void *a_img, uint64_t n_tiles, int *d_err,
                          double *d_norms, uint32_t dense_idx, cudaStream_t st);

// One pass of two dense parts: U1 (image img2, layout 1), then U2 (image
// img2 + DENSE_A_BYTES, layout 2), on every 13-qubit tile; the norm
// accumulators and the rescale as for launch_dense6, dense_idx counting the
// tensor-core passes of the apply.
cudaError_t launch_dense_pair(void *sv, const DensePairLaunch &L, const void *img2, uint64_t n_tiles, int *d_err,
                              double *d_norms, uint32_t dense_idx, cudaStream_t st);

}  // namespace hisv
