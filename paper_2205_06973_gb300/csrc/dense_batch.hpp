// Batched dense kernel: the <= 6-qubit parts of many circuits (>= 13 qubits)
// as tensor-core passes in one persistent launch (see dense_batch.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace hisv {

// One dense pass of one circuit of the batch (48 bytes).
struct DenseBatchPart {
    uint64_t sv_off;       // first amplitude of the circuit's state in the batch buffer
    uint64_t outer_mask;   // the circuit's qubits outside the tile (tile index deposited here)
    uint32_t circuit;      // index of the circuit's tile counter
    uint32_t dn_prev;      // norm slot of the circuit's previous dense pass, or NO_PREV
    uint32_t dn_out;       // norm slot this pass accumulates its output norm into
    uint32_t pad0;
    uint8_t part_q[6];     // the part's qubits, ascending (padded to 6)
    uint8_t col_q[7];      // the tile's column qubits, ascending
    uint8_t n;
    uint8_t pad1[2];
};
static_assert(sizeof(DenseBatchPart) == 48, "DenseBatchPart layout");

constexpr uint32_t DENSE_BATCH_NO_PREV = 0xFFFFFFFFu;

// A range of tiles of one pass (32 bytes); a circuit's pass w is queued
// before its pass w + 1.
struct DenseBatchItem {
    uint32_t part;         // DenseBatchPart index (also its R image index)
    uint32_t circuit;      // the pass's circuit (its tile counter)
    uint32_t tile_begin;
    uint32_t tile_count;
    uint32_t wait;         // the circuit's tile counter must reach this first (4 per finished tile)
    uint32_t pad[3];
};
static_assert(sizeof(DenseBatchItem) == 32, "DenseBatchItem layout");

// Words of the error record: [0] the first failed wait's site code (0 = no
// error; any launch that sees it set stops taking work), [1..6] for a failed
// dependency wait: item, circuit, target count, count seen, CTA, item number
// of the CTA; [7] bit 4 (site / 10 - 1) + site % 10 set for every site that
// failed.
constexpr int DENSE_BATCH_ERR_WORDS = 8;

// items[n_items] over parts[]; r_imgs: one 64 KiB R image per part; done:
// n circuit counters then the queue ticket, zeroed before the launch; dn:
// one FP64 norm slot per pass, zeroed before the launch; err: the error
// record (DENSE_BATCH_ERR_WORDS ints).
cudaError_t launch_dense6_batch(void *svbase, const DenseBatchPart *parts, const DenseBatchItem *items,
                                uint32_t n_items, const void *r_imgs, uint32_t *done, uint32_t *head, int *err,
                                double *dn, cudaStream_t st);

}  // namespace hisv
