// Two dense 6-qubit parts in one HBM pass on the sm_103a tensor cores.
//
// Two consecutive parts of the schedule, on the 6-qubit sets P1 and P2 (each
// padded to 6, preferring the other part's qubits), fit one tile of 13
// qubits T (P1 and P2 plus the lowest remaining qubits). This is the paper's
// multi-level partitioning (Sec. IV-B) with the HBM pass as the first level
// (limit 13 for the tile) and two tensor-core products as the second level
// (limit 6): the tile is read from HBM once, both 64x64 unitaries U1 and U2
// are applied to it on chip, and it is written back once, where two k_dense6
// passes would move the state through HBM twice.
//
// Per tile (8192 amplitudes):
//   layout 1: column n = assignment of the 7 qubits T \ P1, row = P1 bits;
//   layout 2: column n = assignment of T \ P2, row = P2 bits.
// The GEMMs are those of k_dense6 (D = X^T R^T, M = 128 columns, N = K = 128
// reals, split BF16 with FP32 accumulation in tensor memory). Between them the
// tile is re-laid from layout 1 to layout 2 through a 64 KiB shared-memory
// buffer indexed by the tile's 13 slot bits (XOR-swizzled per slot).
//
// Warp roles (13 warps, one CTA per SM, persistent over the tiles):
//  * 8 converter warps (two per TMEM lane quarter, 32 amplitudes of column
//    n per thread): HBM -> registers -> BF16 hi/lo -> tcgen05.st into A1
//    (layout 1), as in k_dense6;
//  * one thread of the MMA warp issues MMA1 (D1 = A1 R1^T) and MMA2
//    (D2 = A2 R2^T), each as soon as its operand and accumulator are ready;
//  * 4 middle warps take a tile from D1 (tcgen05.ld, column n of layout 1,
//    FP32) through the shared buffer (read back as column n of layout 2) to
//    BF16 hi/lo in A2 (tcgen05.st);
//  * 4 epilogue warps: tcgen05.ld of D2, the norm rescale, stores to HBM.
// TMEM: A1 at column 0, D1 at 128, A2 at 256, D2 at 384 (all 512 columns).
// Each stage has one buffer, released by an mbarrier when its consumer is
// done, so no producer runs more than one phase ahead of any waiter. Every
// wait is bounded; on expiry the role records an error and leaves its loop,
// the MMA thread waits (bounded) for its last commit, and the TMEM is freed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "dense.hpp"
#include "dense_common.cuh"

namespace hisv {

using namespace dense_detail;

namespace {

// 17 warps (at most 5 per scheduler: 96 registers a thread); TMEM lane
// quarter = warp & 3
constexpr int PR_EPI_WARPS = 4;                         // warps 0-3
constexpr int PR_CONV_BEGIN = 4;                        // warps 4-11: two per quarter, half = (warp - 4) >> 2
constexpr int PR_CONV_END = 12;
constexpr int PR_MID_BEGIN = 12;                        // warps 12-15
constexpr int PR_MID_END = 16;
constexpr int PR_MMA_WARP = 16;
constexpr int PR_THREADS = (PR_MMA_WARP + 1) * 32;
constexpr int PR_CONV_THREADS = 8 * 32;
constexpr int PR_MID_THREADS = 4 * 32;
constexpr int PR_EPI_THREADS = PR_EPI_WARPS * 32;
constexpr uint32_t PR_TMEM_COLS = 512;
constexpr uint32_t TM_A1 = 0, TM_D1 = 128, TM_A2 = 256, TM_D2 = 384;
constexpr uint32_t PR_X_BYTES = 8192 * 8;               // one tile of complex64
constexpr uint32_t PR_BAR_OFF = 2 * DENSE_A_BYTES + PR_X_BYTES;
constexpr uint32_t PR_ROW_OFF = PR_BAR_OFF + 256;         // row tables (1536 B)
constexpr uint32_t PR_LINE_OFF = PR_BAR_OFF + 4096;
constexpr uint32_t PR_SMEM = PR_LINE_OFF + 64 * PR_CONV_THREADS + 1024;   // 8 run offsets a converter; + slack
constexpr uint32_t PR_WAIT_LIMIT = 1u << 24;
constexpr uint32_t PR_POLL_LIMIT = 1u << 28;            // non-blocking polls without progress (seconds)
static_assert(PR_SMEM <= 227 * 1024, "shared memory layout");

// Non-blocking test of the barrier phase with the given parity (the MMA
// thread polls two pipelines and must not be suspended on one of them).
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}


// split a complex64 amplitude into BF16 (hi, lo) pairs: v = hi + lo + O(2^-16 |v|)
__device__ __forceinline__ void split_bf16(float2 v, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat162 bh = __floats2bfloat162_rn(v.x, v.y);
    const float2 hf = __bfloat1622float2(bh);
    const __nv_bfloat162 bl = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&bh);
    lo = *reinterpret_cast<const uint32_t *>(&bl);
}

// the 24 MMAs of one tile: D = X_hi R_hi + X_lo R_hi + X_hi R_lo. The R
// descriptors are the image's base descriptor plus the offset in its
// 16-byte address field (the image lies below 256 KiB of shared memory, so
// the field does not overflow); the base is opaque to the compiler, so the
// 24 descriptors are formed at each issue rather than held in registers
__device__ __forceinline__ void issue_tile_mmas(uint32_t d, uint32_t a, uint64_t rdesc, uint32_t idesc) {
    asm volatile("" : "+l"(rdesc));
    uint32_t acc = 0;
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const uint32_t xsel = p == 1 ? 64u : 0u, rsel = p == 2 ? 1u : 0u;
#pragma unroll
        for (int ks = 0; ks < 8; ks++) {
            const uint32_t off = (rsel * 2 + (ks >> 2)) * 16384 + (ks & 3) * 32;
            umma_bf16_ts(d, a + xsel + 8 * ks, rdesc + (off >> 4), idesc, acc);
            acc = 1;
        }
    }
}

template <int W1, int W2>
__global__ void __launch_bounds__(PR_THREADS, 1)
k_dense6_pair(float2 *__restrict__ sv, const __grid_constant__ DensePairLaunch L, const uint8_t *__restrict__ img,
              uint64_t n_tiles, int *__restrict__ err, double *__restrict__ dn, uint32_t dense_idx) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *const base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *const sR1 = base;
    uint8_t *const sR2 = base + DENSE_A_BYTES;
    float2 *const sX = reinterpret_cast<float2 *>(base + 2 * DENSE_A_BYTES);
    uint64_t *const bars = reinterpret_cast<uint64_t *>(base + PR_BAR_OFF);
    uint64_t *const afull = bars + 0, *const d1full = bars + 1, *const d1empty = bars + 2, *const xfull = bars + 3;
    uint64_t *const xfree = bars + 4, *const a2full = bars + 5, *const d2full = bars + 6, *const d2empty = bars + 7;
    uint32_t *const tslot = reinterpret_cast<uint32_t *>(bars + 16);
    // per row m of a 64-amplitude column: its shared-buffer offset in layout 1
    // and 2 (XOR of the row bits' slot offsets) and its global offset in
    // layout 1 and 2 (the row bits deposited on the part's qubits); read by
    // all lanes at once (broadcast) instead of being held in registers
    uint32_t *const xrow1 = reinterpret_cast<uint32_t *>(base + PR_ROW_OFF);
    uint32_t *const xrow2 = xrow1 + 64;
    uint64_t *const grow1 = reinterpret_cast<uint64_t *>(xrow1 + 128);
    uint64_t *const grow2 = grow1 + 64;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < 64) {
        uint32_t x1 = 0, x2 = 0;
        uint64_t g1 = 0, g2 = 0;
        for (int b = 0; b < DENSE_K; b++)
            if ((tid >> b) & 1) {
                x1 ^= L.xsw[L.s_q1[b]];
                x2 ^= L.xsw[L.s_q2[b]];
                g1 |= 1ull << L.q1[b];
                g2 |= 1ull << L.q2[b];
            }
        xrow1[tid] = x1;
        xrow2[tid] = x2;
        grow1[tid] = g1;
        grow2[tid] = g2;
    }

    for (int i = tid; i < 2 * DENSE_A_BYTES / 16; i += PR_THREADS)
        reinterpret_cast<uint4 *>(sR1)[i] = reinterpret_cast<const uint4 *>(img)[i];
    if (tid == 0) {
        mbar_init(afull, PR_CONV_THREADS);
        mbar_init(d1full, 1);
        mbar_init(d1empty, PR_MID_THREADS);
        mbar_init(xfull, PR_MID_THREADS);
        mbar_init(xfree, PR_MID_THREADS);
        mbar_init(a2full, PR_MID_THREADS);
        mbar_init(d2full, 1);
        mbar_init(d2empty, PR_EPI_THREADS);
        mbar_init_fence();
    }
    if (warp == PR_MMA_WARP) {
        tmem_alloc(tslot, PR_TMEM_COLS);
        tmem_relinquish();
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // R images visible to the MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    // the previous kernel on the stream has completed and its writes are visible
    asm volatile("griddepcontrol.wait;\n" ::: "memory");

    const int q = warp & 3;
    const uint32_t n_col = 32 * q + lane;
    const uint64_t dgrid = deposit_bits(gridDim.x, L.outer_mask);
    const uint32_t lane_q = (uint32_t)(32 * q) << 16;

    if (warp >= PR_CONV_BEGIN && warp < PR_CONV_END) {
        // ------------------------------------------------ converters (layout 1)
        const int h = (warp - PR_CONV_BEGIN) >> 2;   // amplitudes 32h..32h+31 of the column (row bit 5)
        uint64_t coff = h ? 1ull << L.q1[DENSE_K - 1] : 0ull;
#pragma unroll
        for (int b = 0; b < DENSE_COLS; b++)
            if ((n_col >> b) & 1) coff |= 1ull << L.c1[b];
        const int ctid = tid - PR_CONV_BEGIN * 32;
        // L2 warm-up of the next tile: its runs of 2^f consecutive amplitudes
        // (f = L.prefetch: the tile holds qubits 0..f-1, 2 <= f <= 4), 8192 >>
        // f of them, 2^(5-f) per converter thread; offsets stored run-major
        // (consecutive threads, consecutive words)
        const int f = L.prefetch;
        const int nrun = 1 << (5 - f);
        const uint32_t run_bytes = 8u << f;
        uint64_t *const lineoff = reinterpret_cast<uint64_t *>(base + PR_LINE_OFF) + ctid;
        {
            const uint64_t all = L.n >= 64 ? ~0ull : ((1ull << L.n) - 1);
            const uint64_t tq = all & ~L.outer_mask & ~((1ull << f) - 1);
            for (int u = 0; u < nrun; u++)
                lineoff[u * PR_CONV_THREADS] = deposit_bits((uint64_t)(ctid + PR_CONV_THREADS * u), tq);
        }
        double in_norm = 0.0;
        uint64_t tb = deposit_bits(blockIdx.x, L.outer_mask);
        uint64_t tpf = masked_add(tb, dgrid, L.outer_mask);
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, i++) {
            if (tile + gridDim.x < n_tiles) {
                if (f >= 4) {   // whole 128-byte lines
#pragma unroll
                    for (int u = 0; u < 2; u++)
                        asm volatile("prefetch.global.L2 [%0];\n" ::"l"(sv + (tpf | lineoff[u * PR_CONV_THREADS])));
                } else {        // runs of 32 or 64 bytes: exactly those bytes
                    for (int u = 0; u < nrun; u++)
                        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n"
                                     ::"l"(sv + (tpf | lineoff[u * PR_CONV_THREADS])), "r"(run_bytes) : "memory");
                }
            }
            const float2 *const src = sv + (tb | coff);
            const uint32_t ta = tmem + lane_q + TM_A1 + 32 * h;
            float tile_in = 0.0f;
            bool ok = true;
            // both rounds of 16 loads are in flight before the wait for A1
            float2 x0[16], x1[16];
#pragma unroll
            for (int j = 0; j < 16; j += W1) ld_amps<W1>(src + grow1[j], x0 + j);
#pragma unroll
            for (int j = 0; j < 16; j += W1) ld_amps<W1>(src + grow1[16 + j], x1 + j);
            {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    tile_in = fmaf(x0[j].x, x0[j].x, fmaf(x0[j].y, x0[j].y, tile_in));
                    split_bf16(x0[j], hi[j], lo[j]);
                }
                // MMA1 of the previous tile has read A1 (warp-uniform: the
                // tcgen05 stores below are .sync.aligned)
                ok = __all_sync(0xffffffffu, i < 1 || mbar_wait(d1full, (i - 1) & 1, PR_WAIT_LIMIT));
                if (ok) {
                    tc_fence_after();
                    tmem_st16(ta, hi);
                    tmem_st16(ta + 64, lo);
                }
            }
            if (ok) {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    tile_in = fmaf(x1[j].x, x1[j].x, fmaf(x1[j].y, x1[j].y, tile_in));
                    split_bf16(x1[j], hi[j], lo[j]);
                }
                tmem_st16(ta + 16, hi);
                tmem_st16(ta + 64 + 16, lo);
            }
            if (!ok) {
                atomicExch(err, 1);
                break;
            }
            tmem_st_wait();
            tc_fence_before();
            mbar_arrive(afull);
            if (dense_idx == 0) in_norm += (double)tile_in;
            tb = masked_add(tb, dgrid, L.outer_mask);
            tpf = masked_add(tpf, dgrid, L.outer_mask);
        }
        if (dense_idx == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) in_norm += __shfl_xor_sync(0xffffffffu, in_norm, o);
            if (lane == 0) atomicAdd(dn, in_norm);
        }
    } else if (warp == PR_MMA_WARP) {
        // ------------------------------------------------ MMA issuer
        // MMA1 of tile i1 and MMA2 of tile i2 < i1, each issued as soon as its
        // operand is written and its accumulator is free (single polls of
        // both, so that neither waits behind the other)
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, 128);
            const uint64_t rd1 = sw128_desc(smem_u32(sR1)), rd2 = sw128_desc(smem_u32(sR2));
            const uint32_t ntc = blockIdx.x < n_tiles ? (uint32_t)((n_tiles - 1 - blockIdx.x) / gridDim.x + 1) : 0u;
            uint64_t *last = nullptr;   // barrier and phase of the last commit
            uint32_t last_par = 0, i1 = 0, i2 = 0, idle = 0;
            while (i2 < ntc) {
                bool did = false;
                if (i1 < ntc && mbar_test(afull, i1 & 1) && (i1 == 0 || mbar_test(d1empty, (i1 - 1) & 1))) {
                    tc_fence_after();
                    issue_tile_mmas(tmem + TM_D1, tmem + TM_A1, rd1, idesc);
                    umma_commit(d1full);   // D1 ready, A1 consumed
                    last = d1full;
                    last_par = i1 & 1;
                    i1++;
                    did = true;
                }
                if (i2 < i1 && mbar_test(a2full, i2 & 1) && (i2 == 0 || mbar_test(d2empty, (i2 - 1) & 1))) {
                    tc_fence_after();
                    issue_tile_mmas(tmem + TM_D2, tmem + TM_A2, rd2, idesc);
                    umma_commit(d2full);   // D2 ready, A2 consumed
                    last = d2full;
                    last_par = i2 & 1;
                    i2++;
                    did = true;
                }
                idle = did ? 0u : idle + 1;
                if (idle > PR_POLL_LIMIT) {
                    atomicExch(err, 1);
                    break;
                }
            }
            // every MMA issued has completed before the TMEM is freed (a
            // commit tracks all earlier MMAs of this thread)
            if (last && !mbar_wait(last, last_par, PR_WAIT_LIMIT)) atomicExch(err, 1);
        }
    } else if (warp >= PR_MID_BEGIN && warp < PR_MID_END) {
        // ------------------------------------------------ middle: layout 1 -> 2
        uint32_t xw = 0, xr = 0;   // this column's part of the buffer offsets (layouts 1, 2)
#pragma unroll
        for (int b = 0; b < DENSE_COLS; b++) {
            if ((n_col >> b) & 1) {
                xw ^= L.xsw[L.s_c1[b]];
                xr ^= L.xsw[L.s_c2[b]];
            }
        }
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, i++) {
            // D1 of tile i is complete; every middle thread has read the
            // shared buffer of the previous tile
            if (!__all_sync(0xffffffffu, mbar_wait(d1full, i & 1, PR_WAIT_LIMIT) &&
                                             (i < 1 || mbar_wait(xfree, (i - 1) & 1, PR_WAIT_LIMIT)))) {
                atomicExch(err, 1);
                break;
            }
            tc_fence_after();
            const uint32_t td = tmem + lane_q + TM_D1;
#pragma unroll 1
            for (int g = 0; g < 4; g++) {
                uint32_t r[32];
                tmem_ld32(td + 32 * g, r);
                tmem_ld_wait();
                if (g == 3) {
                    tc_fence_before();
                    mbar_arrive(d1empty);
                }
#pragma unroll
                for (int j = 0; j < 16; j++)
                    sX[xw ^ xrow1[16 * g + j]] = make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
            }
            mbar_arrive(xfull);
            // the whole tile is in the buffer; MMA2 of the previous tile has read A2
            if (!__all_sync(0xffffffffu, mbar_wait(xfull, i & 1, PR_WAIT_LIMIT) &&
                                             (i < 1 || mbar_wait(d2full, (i - 1) & 1, PR_WAIT_LIMIT)))) {
                atomicExch(err, 1);
                break;
            }
            tc_fence_after();
            const uint32_t ta = tmem + lane_q + TM_A2;
#pragma unroll 1
            for (int g = 0; g < 4; g++) {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; j++) split_bf16(sX[xr ^ xrow2[16 * g + j]], hi[j], lo[j]);
                if (g == 3) mbar_arrive(xfree);   // this thread's reads of the buffer are done
                tmem_st16(ta + 16 * g, hi);
                tmem_st16(ta + 64 + 16 * g, lo);
            }
            tmem_st_wait();
            tc_fence_before();
            mbar_arrive(a2full);
        }
    } else {
        // ------------------------------------------------ epilogue (layout 2)
        uint64_t coff = 0;
#pragma unroll
        for (int b = 0; b < DENSE_COLS; b++)
            if ((n_col >> b) & 1) coff |= 1ull << L.c2[b];
        // unitarity: rescale to the input norm of the apply, correcting the
        // drift measured on the previous tensor-core pass
        float scale = 1.0f;
        if (dense_idx > 0) {
            const double n0 = dn[0], prev = dn[dense_idx];
            if (n0 > 0.0 && prev > 0.0) scale = (float)sqrt(n0 / prev);
        }
        double out_norm = 0.0;
        uint64_t tb = deposit_bits(blockIdx.x, L.outer_mask);
        uint32_t i = 0;
        for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, i++) {
            if (!__all_sync(0xffffffffu, mbar_wait(d2full, i & 1, PR_WAIT_LIMIT))) {   // warp-uniform (tcgen05.ld)
                atomicExch(err, 1);
                break;
            }
            tc_fence_after();
            const uint32_t td = tmem + lane_q + TM_D2;
            float2 *const dst = sv + (tb | coff);
            float tile_out = 0.0f;
#pragma unroll 1
            for (int g = 0; g < 4; g++) {
                uint32_t r[32];
                tmem_ld32(td + 32 * g, r);
                tmem_ld_wait();
                if (g == 3) {
                    tc_fence_before();
                    mbar_arrive(d2empty);
                }
#pragma unroll
                for (int j = 0; j < 16; j += W2) {
                    float2 y[W2];
#pragma unroll
                    for (int w = 0; w < W2; w++) {
                        y[w] = make_float2(__uint_as_float(r[2 * (j + w)]) * scale,
                                           __uint_as_float(r[2 * (j + w) + 1]) * scale);
                        tile_out = fmaf(y[w].x, y[w].x, fmaf(y[w].y, y[w].y, tile_out));
                    }
                    st_amps<W2>(dst + grow2[16 * g + j], y);
                }
            }
            out_norm += (double)tile_out;
            tb = masked_add(tb, dgrid, L.outer_mask);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) out_norm += __shfl_xor_sync(0xffffffffu, out_norm, o);
        if (lane == 0) atomicAdd(dn + 1 + dense_idx, out_norm);
    }
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    __syncthreads();
    if (warp == PR_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, PR_TMEM_COLS);
    }
}

template <int W1, int W2>
cudaError_t pair_attr() {
    return cudaFuncSetAttribute(k_dense6_pair<W1, W2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PR_SMEM);
}

template <int W1, int W2>
cudaError_t pair_launch(const cudaLaunchConfig_t &cfg, float2 *sv, const DensePairLaunch &L, const uint8_t *img,
                        uint64_t n_tiles, int *err, double *dn, uint32_t idx) {
    return cudaLaunchKernelEx(&cfg, k_dense6_pair<W1, W2>, sv, L, img, n_tiles, err, dn, idx);
}

// amplitudes per lane access of a layout: its part qubits 0, 1, ... in a row
// make that many low bits of the row index consecutive amplitudes
int lane_width(const uint8_t *qs, bool a32) {
    int z = 0;
    while (z < DENSE_K && qs[z] == z) z++;
    return (z >= 2 && a32) ? 4 : (z >= 1 ? 2 : 1);
}

}  // namespace

cudaError_t launch_dense_pair(void *sv, const DensePairLaunch &L, const void *img2, uint64_t n_tiles, int *d_err,
                              double *d_norms, uint32_t dense_idx, cudaStream_t st) {
    static std::atomic<uint64_t> attr_set{0};
    static std::mutex mu;
    static int sms[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    if (!((attr_set.load(std::memory_order_acquire) >> dev) & 1)) {
        std::lock_guard<std::mutex> lk(mu);
        if (!((attr_set.load(std::memory_order_relaxed) >> dev) & 1)) {
            const cudaError_t es[9] = {pair_attr<1, 1>(), pair_attr<1, 2>(), pair_attr<1, 4>(),
                                       pair_attr<2, 1>(), pair_attr<2, 2>(), pair_attr<2, 4>(),
                                       pair_attr<4, 1>(), pair_attr<4, 2>(), pair_attr<4, 4>()};
            for (cudaError_t x : es)
                if (x != cudaSuccess) return x;
            e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            attr_set.fetch_or(1ull << dev, std::memory_order_release);
        }
    }
    if (reinterpret_cast<uintptr_t>(sv) & 15) return cudaErrorMisalignedAddress;
    uint64_t grid = (uint64_t)sms[dev];
    if (grid > n_tiles) grid = n_tiles;
    if (grid < 1) grid = 1;
    const bool a32 = (reinterpret_cast<uintptr_t>(sv) & 31) == 0;
    const int w1 = lane_width(L.q1, a32), w2 = lane_width(L.q2, a32);
    float2 *const p = reinterpret_cast<float2 *>(sv);
    const uint8_t *const a = reinterpret_cast<const uint8_t *>(img2);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(PR_THREADS);
    cfg.dynamicSmemBytes = PR_SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    switch (w1 * 8 + w2) {
    case 9: e = pair_launch<1, 1>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    case 10: e = pair_launch<1, 2>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    case 12: e = pair_launch<1, 4>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    case 17: e = pair_launch<2, 1>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    case 18: e = pair_launch<2, 2>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    case 20: e = pair_launch<2, 4>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    case 33: e = pair_launch<4, 1>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    case 34: e = pair_launch<4, 2>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    default: e = pair_launch<4, 4>(cfg, p, L, a, n_tiles, d_err, d_norms, dense_idx); break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace hisv
