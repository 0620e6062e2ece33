// Batched dense kernel: the dense parts (<= 6 qubits, fused 64x64 unitaries)
// of many circuits of >= 13 qubits in one persistent launch.
//
// The tile machinery is the one of k_dense6 (dense.cu): a tile is 128 columns
// x 64 amplitudes of one circuit's state; 8 converter warps load it with
// coalesced global loads, split it to BF16 hi/lo and write it into a TMEM A
// buffer; one thread issues the 24 split-BF16 MMAs against the pass's R image
// in shared memory; 4 epilogue warps read the accumulator and store the
// amplitudes. What the batch adds:
//  * a device work queue of items (circuit pass, range of tiles) in wave
//    order; the converter leader takes the next item with an atomic ticket and
//    waits (bounded, acquire) until the circuit's tile counter shows that its
//    earlier passes are complete; an item only waits on items with smaller
//    tickets, which running CTAs already hold, so the queue cannot deadlock;
//  * the R image of each item is copied into one of two shared buffers (full /
//    empty mbarriers: the MMA thread commits "empty" after the item's last
//    tile);
//  * per-tile metadata (state offset, pass, R buffer, norm scale) goes from
//    the converter leader to the MMA thread (ordered by the A buffer's full
//    barrier) and to the epilogue (a four-deep ring with its own full / empty
//    barriers);
//  * each epilogue warp adds its share of the pass's output norm, then
//    increments the circuit's tile counter with release semantics, so a later
//    pass that observes the count (acquire) sees both the stored amplitudes
//    and the norm. A pass rescales its output to unit norm, correcting the
//    drift measured on the circuit's previous dense pass (the batch's states
//    start in |0...0>, so their exact norm is 1).
// Every wait is bounded; on expiry the role records the error, the converters
// publish how many tiles they produced so that the other roles stop there,
// and the TMEM is freed on exit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "dense.hpp"
#include "dense_batch.hpp"
#include "dense_common.cuh"

namespace hisv {

using namespace dense_detail;

namespace {

constexpr int EPI_WARPS = 4;
constexpr int CONV_WARPS = 8;
constexpr int MMA_WARP = EPI_WARPS + CONV_WARPS;
constexpr int THREADS = (MMA_WARP + 1) * 32;
constexpr int CONV_THREADS = CONV_WARPS * 32;
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int NMETA = 4;
constexpr uint32_t TMEM_COLS = 512;                   // D0, D1, A0, A1 at 0, 128, 256, 384
constexpr uint32_t OFF_MISC = 2 * DENSE_A_BYTES;       // two R buffers, then barriers and metadata
constexpr uint32_t SMEM = OFF_MISC + 1024 + 1024;      // > half of the SM: one CTA (and its TMEM) per SM
constexpr uint32_t WAIT_LIMIT = 1u << 24;              // bounded polls (seconds with the back-off below)
constexpr uint32_t SPIN_POLLS = 4096;                  // polls before a wait starts to sleep between polls
constexpr uint32_t DEP_LIMIT = 1u << 22;               // bounded dependency polls (about a second)

struct TileMeta {
    uint64_t tb;       // first amplitude of the tile's circuit + the tile's outer bits
    uint32_t part;     // DenseBatchPart index
    uint32_t rbuf;     // R buffer holding the pass's image
    uint32_t first;    // first tile of its item (the R buffer was just filled)
    uint32_t last;     // last tile of its item (the R buffer is free after its MMAs)
    float scale;       // norm correction of the pass
    uint32_t pad;
};

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}

// W consecutive complex64 amplitudes cached in L2 only: the passes of one
// circuit read what other CTAs of the same launch wrote.
template <int W>
__device__ __forceinline__ void ld_amps_cg(const float2 *p, float2 *x) {
    if constexpr (W == 1) {
        x[0] = __ldcg(p);
    } else if constexpr (W == 2) {
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
        x[0] = make_float2(v.x, v.y);
        x[1] = make_float2(v.z, v.w);
    } else {
        asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=f"(x[0].x), "=f"(x[0].y), "=f"(x[1].x), "=f"(x[1].y), "=f"(x[2].x), "=f"(x[2].y),
                       "=f"(x[3].x), "=f"(x[3].y)
                     : "l"(p)
                     : "memory");
    }
}

// Column bits of the lane and the part-bit offsets of an item's pass.
struct Geo {
    uint64_t coff;
    uint64_t pbit[DENSE_K];
    int w;             // amplitudes per lane access (1, 2, 4)
};
__device__ __forceinline__ void geometry(const DenseBatchPart &P, uint32_t n_col, Geo &g) {
    g.coff = 0;
#pragma unroll
    for (int b = 0; b < DENSE_COLS; b++)
        if ((n_col >> b) & 1) g.coff |= 1ull << P.col_q[b];
#pragma unroll
    for (int b = 0; b < DENSE_K; b++) g.pbit[b] = 1ull << P.part_q[b];
    int z = 0;
    while (z < DENSE_K && P.part_q[z] == z) z++;
    g.w = z >= 2 ? 4 : (z == 1 ? 2 : 1);
}

// Converter part of one tile: 32 amplitudes of the lane's column (half h),
// split to BF16 and written into TMEM (hi at ta, lo at ta + 64).
template <int W>
__device__ __forceinline__ void convert_tile(const float2 *src, const Geo &g, uint32_t ta) {
#pragma unroll
    for (int gg = 0; gg < 2; gg++) {
        float2 x[16];
#pragma unroll
        for (int j = 0; j < 16; j += W) {
            const int m = 16 * gg + j;
            uint64_t o = 0;
#pragma unroll
            for (int bb = 0; bb < 5; bb++)
                if ((m >> bb) & 1) o |= g.pbit[bb];
            ld_amps_cg<W>(src + o, x + j);
        }
        uint32_t hi[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; j++) {
            const float2 v = x[j];
            const __nv_bfloat162 bh = __floats2bfloat162_rn(v.x, v.y);
            const float2 hf = __bfloat1622float2(bh);
            const __nv_bfloat162 bl = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
            hi[j] = *reinterpret_cast<const uint32_t *>(&bh);
            lo[j] = *reinterpret_cast<const uint32_t *>(&bl);
        }
        tmem_st16(ta + 16 * gg, hi);
        tmem_st16(ta + 64 + 16 * gg, lo);
    }
}

// Epilogue part of one tile: the 64 output amplitudes of the lane's column
// from the accumulator at td, scaled, stored; returns the sum of |y|^2.
template <int W>
__device__ __forceinline__ float store_tile(float2 *dst, const Geo &g, uint32_t td, float scale, uint64_t *dempty) {
    float tile_out = 0.0f;
#pragma unroll
    for (int gg = 0; gg < 4; gg++) {
        uint32_t r[32];
        tmem_ld32(td + 32 * gg, r);
        tmem_ld_wait();
        if (gg == 3) {
            tc_fence_before();
            mbar_arrive(dempty);
        }
#pragma unroll
        for (int j = 0; j < 16; j += W) {
            const int m = 16 * gg + j;
            uint64_t o = 0;
#pragma unroll
            for (int bb = 0; bb < 6; bb++)
                if ((m >> bb) & 1) o |= g.pbit[bb];
            float2 y[W];
#pragma unroll
            for (int w = 0; w < W; w++) {
                y[w] = make_float2(__uint_as_float(r[2 * (j + w)]) * scale, __uint_as_float(r[2 * (j + w) + 1]) * scale);
                tile_out = fmaf(y[w].x, y[w].x, fmaf(y[w].y, y[w].y, tile_out));
            }
            st_amps<W>(dst + o, y);
        }
    }
    return tile_out;
}

// Wait for a barrier phase, or for the converters to have published a tile
// count <= tile (no more tiles); returns 1 on the phase, 0 on the end, -1 on
// timeout.
__device__ __forceinline__ int wait_or_end(uint64_t *bar, uint32_t parity, const volatile uint32_t *ntiles,
                                           uint32_t tile) {
    for (uint32_t k = 0; k < WAIT_LIMIT; k++) {
        if (mbar_try(bar, parity)) return 1;
        if (*ntiles <= tile) return 0;
        if (k >= SPIN_POLLS) __nanosleep(128);
    }
    return -1;
}

// Converter wait: the phase, or false once any converter has given up.
__device__ __forceinline__ bool conv_wait(uint64_t *bar, uint32_t parity, const volatile int *abort) {
    for (uint32_t k = 0; k < WAIT_LIMIT; k++) {
        if (mbar_try(bar, parity)) return true;
        if (*abort) return false;
        if (k >= SPIN_POLLS) __nanosleep(128);
    }
    return false;
}

}  // namespace

__global__ void __launch_bounds__(THREADS, 1)
k_dense6_batch(float2 *__restrict__ svbase, const DenseBatchPart *__restrict__ parts,
               const DenseBatchItem *__restrict__ items, uint32_t n_items, const uint8_t *__restrict__ r_imgs,
               uint32_t *__restrict__ done, uint32_t *__restrict__ head, int *__restrict__ err,
               double *__restrict__ dn) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *const base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *const sR0 = base;                                    // R buffers at 0 and DENSE_A_BYTES
    uint64_t *const bars = reinterpret_cast<uint64_t *>(base + OFF_MISC);
    uint64_t *const rfull = bars, *const rempty = bars + 2, *const afull = bars + 4, *const dfull = bars + 6,
                    *const dempty = bars + 8, *const mfull = bars + 10, *const mempty = bars + 10 + NMETA;
    uint32_t *const misc = reinterpret_cast<uint32_t *>(base + OFF_MISC + 256);
    uint32_t *const tslot = misc;                                  // TMEM base address
    volatile uint32_t *const ntiles = misc + 1;                    // tiles produced (set at the end)
    uint32_t *const nmin = misc + 2;                               // min over converters of their tile count
    volatile int *const abort_flag = reinterpret_cast<volatile int *>(misc + 3);
    volatile uint32_t *const s_item = misc + 4;                    // [2] claimed item (by parity of seq)
    volatile int *const s_ok = reinterpret_cast<volatile int *>(misc + 6);          // [2]
    volatile float *const s_scale = reinterpret_cast<volatile float *>(misc + 8);   // [2]
    TileMeta *const meta = reinterpret_cast<TileMeta *>(base + OFF_MISC + 512);     // [NMETA]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            mbar_init(&rfull[b], CONV_THREADS);
            mbar_init(&rempty[b], 1);
            mbar_init(&afull[b], CONV_THREADS);
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], EPI_THREADS);
        }
        for (int m = 0; m < NMETA; m++) {
            mbar_init(&mfull[m], 1);
            mbar_init(&mempty[m], EPI_THREADS);
        }
        *ntiles = 0xFFFFFFFFu;
        *nmin = 0xFFFFFFFFu;
        *abort_flag = 0;
        mbar_init_fence();
    }
    if (warp == MMA_WARP) {
        tmem_alloc(tslot, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    const int q = warp & 3, h = warp >= EPI_WARPS ? ((warp - EPI_WARPS) >> 2) & 1 : 0;
    const uint32_t n_col = 32 * q + lane;

    if (warp >= EPI_WARPS && warp < MMA_WARP) {
        // ------------------------------------------------------ converters
        // Every converter thread passes the same named barriers: a thread that
        // gives up sets the abort flag and skips to the next claim, where the
        // leader turns the flag into a uniform stop.
        const int ctid = tid - EPI_THREADS;
        uint32_t i = 0, seq = 0;
        while (true) {
            const uint32_t slot = seq & 1;
            if (ctid == 0) {   // the leader takes the next item and waits for its dependency
                uint32_t it = n_items;
                int ok = *abort_flag ? 0 : 1;
                float scale = 1.0f;
                if (ok) {
                    it = atomicAdd(head, 1u);
                    if (it < n_items) {
                        const DenseBatchItem I = items[it];
                        const DenseBatchPart &P = parts[I.part];
                        if (I.wait) {
                            uint32_t k = 0;
                            while (ld_acquire_u32(done + P.circuit) < I.wait) {
                                if (++k > DEP_LIMIT) {
                                    ok = 0;
                                    break;
                                }
                                __nanosleep(64);
                            }
                        }
                        if (ok && P.dn_prev != DENSE_BATCH_NO_PREV) {
                            const double prev = *reinterpret_cast<volatile double *>(dn + P.dn_prev);
                            if (prev > 0.0) scale = (float)sqrt(1.0 / prev);
                        }
                    }
                }
                s_item[slot] = it;
                s_ok[slot] = ok;
                s_scale[slot] = scale;
            }
            asm volatile("bar.sync 1, %0;\n" ::"n"(CONV_THREADS) : "memory");
            const uint32_t it = s_item[slot];
            const int ok = s_ok[slot];
            const float scale = s_scale[slot];
            if (!ok) {
                if (ctid == 0) atomicExch(err, 1);
                break;
            }
            if (it >= n_items) break;
            seq++;
            const DenseBatchItem I = items[it];
            const DenseBatchPart P = parts[I.part];
            // the pass's R image into buffer rb, once the MMAs of the item two
            // claims back (same buffer) are done
            const uint32_t rb = slot, use = (seq - 1) >> 1;
            if (use >= 1 && !conv_wait(&rempty[rb], (use - 1) & 1, abort_flag)) {
                atomicExch(err, 1);
                *abort_flag = 1;
                continue;
            }
            {
                const uint4 *src = reinterpret_cast<const uint4 *>(r_imgs + (size_t)I.part * DENSE_A_BYTES);
                uint4 *dst = reinterpret_cast<uint4 *>(sR0 + rb * DENSE_A_BYTES);
                for (int k = ctid; k < DENSE_A_BYTES / 16; k += CONV_THREADS) dst[k] = __ldg(src + k);
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(&rfull[rb]);
            }
            Geo g;
            geometry(P, n_col, g);
            const uint64_t hoff = h ? g.pbit[DENSE_K - 1] : 0ull;
            const uint64_t low = P.outer_mask & (~P.outer_mask + 1);   // tile index 1 deposited
            uint64_t tb = deposit_bits(I.tile_begin, P.outer_mask);
            for (uint32_t t = 0; t < I.tile_count; t++) {
                const uint32_t b = i & 1, m = i & (NMETA - 1);
                if ((i >= 2 && !conv_wait(&dfull[b], ((i >> 1) - 1) & 1, abort_flag)) ||
                    (i >= NMETA && !conv_wait(&mempty[m], ((i / NMETA) - 1) & 1, abort_flag))) {
                    atomicExch(err, 1);
                    *abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t tabs = P.sv_off + tb;
                const float2 *const src = svbase + (tabs + (g.coff | hoff));
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + 256 + 128 * b + 32 * h;
                if (g.w == 4) convert_tile<4>(src, g, ta);
                else if (g.w == 2) convert_tile<2>(src, g, ta);
                else convert_tile<1>(src, g, ta);
                if (ctid == 0) {
                    TileMeta &M = meta[m];
                    M.tb = tabs;
                    M.part = I.part;
                    M.rbuf = rb;
                    M.first = t == 0;
                    M.last = t + 1 == I.tile_count;
                    M.scale = scale;
                }
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(&afull[b]);
                if (ctid == 0) mbar_arrive(&mfull[m]);
                i++;
                tb = masked_add(tb, low, P.outer_mask);
            }
        }
        // the other roles stop after the tiles every converter has produced
        atomicMin(nmin, i);
        asm volatile("bar.sync 1, %0;\n" ::"n"(CONV_THREADS) : "memory");
        if (ctid == 0) *ntiles = *reinterpret_cast<volatile uint32_t *>(nmin);
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(128, 128);
            uint32_t i = 0, ruse[2] = {0, 0};
            while (true) {
                const uint32_t b = i & 1, u = i >> 1;
                const int r = wait_or_end(&afull[b], u & 1, ntiles, i);
                if (r == 0) break;
                if (r < 0 || (i >= 2 && wait_or_end(&dempty[b], (u - 1) & 1, ntiles, i) != 1)) {
                    atomicExch(err, 1);
                    break;
                }
                const TileMeta M = meta[i & (NMETA - 1)];
                if (M.first) {
                    if (wait_or_end(&rfull[M.rbuf], ruse[M.rbuf] & 1, ntiles, i) != 1) {
                        atomicExch(err, 1);
                        break;
                    }
                    ruse[M.rbuf]++;
                }
                tc_fence_after();
                const uint32_t sb = smem_u32(sR0 + M.rbuf * DENSE_A_BYTES);
                const uint32_t d = tmem + 128 * b, a = tmem + 256 + 128 * b;
                uint32_t acc = 0;
#pragma unroll
                for (int p = 0; p < 3; p++) {
                    // p = 0: X_hi R_hi, 1: X_lo R_hi, 2: X_hi R_lo
                    const uint32_t xsel = p == 1 ? 64u : 0u, rsel = p == 2 ? 1u : 0u;
#pragma unroll
                    for (int ks = 0; ks < 8; ks++) {
                        const uint32_t ra = sb + (rsel * 2 + (ks >> 2)) * 16384 + (ks & 3) * 32;
                        umma_bf16_ts(d, a + xsel + 8 * ks, sw128_desc(ra), idesc, acc);
                        acc = 1;
                    }
                }
                umma_commit(&dfull[b]);                  // accumulator ready, A buffer consumed
                if (M.last) umma_commit(&rempty[M.rbuf]);   // the item's R buffer is free
                i++;
            }
            // the MMAs issued complete before the TMEM is freed
            if (i > 0 && !mbar_wait(&dfull[(i - 1) & 1], ((i - 1) >> 1) & 1, WAIT_LIMIT)) atomicExch(err, 1);
        }
    } else {
        // ------------------------------------------------------ epilogue
        uint32_t i = 0;
        while (true) {
            const uint32_t b = i & 1, m = i & (NMETA - 1);
            const int r = wait_or_end(&mfull[m], (i / NMETA) & 1, ntiles, i);
            if (r == 0) break;
            if (r < 0) {
                atomicExch(err, 1);
                break;
            }
            const TileMeta M = meta[m];
            mbar_arrive(&mempty[m]);
            const DenseBatchPart P = parts[M.part];
            Geo g;
            geometry(P, n_col, g);
            const int rd = wait_or_end(&dfull[b], (i >> 1) & 1, ntiles, i);
            if (rd != 1) {
                if (rd < 0) atomicExch(err, 1);
                break;
            }
            tc_fence_after();
            const uint32_t td = tmem + ((uint32_t)(32 * q) << 16) + 128 * b;
            float2 *const dst = svbase + (M.tb + g.coff);
            float part_norm;
            if (g.w == 4) part_norm = store_tile<4>(dst, g, td, M.scale, &dempty[b]);
            else if (g.w == 2) part_norm = store_tile<2>(dst, g, td, M.scale, &dempty[b]);
            else part_norm = store_tile<1>(dst, g, td, M.scale, &dempty[b]);
            double s = (double)part_norm;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            __syncwarp();   // the warp's stores are ordered before lane 0's release below
            if (lane == 0) {
                atomicAdd(dn + P.dn_out, s);
                __threadfence();
                red_release_add_u32(done + P.circuit, 1u);   // one of four per tile
            }
            __syncwarp();
            i++;
        }
    }
    __syncthreads();
    if (warp == MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

cudaError_t launch_dense6_batch(void *svbase, const DenseBatchPart *parts, const DenseBatchItem *items,
                                uint32_t n_items, const void *r_imgs, uint32_t *done, uint32_t *head, int *err,
                                double *dn, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_dense6_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM)) !=
        cudaSuccess)
        return e;
    if (reinterpret_cast<uintptr_t>(svbase) & 31) return cudaErrorMisalignedAddress;
    unsigned grid = (unsigned)sms;
    if (n_items < grid) grid = n_items < 1 ? 1 : n_items;
    k_dense6_batch<<<grid, THREADS, SMEM, st>>>(reinterpret_cast<float2 *>(svbase), parts, items, n_items,
                                                reinterpret_cast<const uint8_t *>(r_imgs), done, head, err, dn);
    return cudaGetLastError();
}

}  // namespace hisv
