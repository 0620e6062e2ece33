// Batched dense kernel: the dense parts (<= 6 qubits, fused 64x64 unitaries)
// of many circuits of >= 13 qubits in one persistent launch.
//
// The tile machinery is the one of k_dense6 (dense.cu): a tile is 128 columns
// x 64 amplitudes of one circuit's state; 8 converter warps load it with
// coalesced global loads, split it to BF16 hi/lo and write it into a TMEM A
// buffer; one thread issues the 24 split-BF16 MMAs against the pass's R image
// in shared memory; 4 epilogue warps read the accumulator and store the
// amplitudes. What the batch adds:
//  * a scheduler warp that runs one item ahead of the converters: it takes
//    the next item (a circuit pass and a range of its tiles) from a device
//    queue in wave order with an atomic ticket, waits (bounded, acquire) until
//    the circuit's tile counter shows that its earlier passes are complete,
//    starts a bulk copy of the pass's R image into one of two shared buffers
//    and hands the item to the converters through a two-slot ring. An item
//    only waits on items with smaller tickets, which running CTAs already
//    hold, so the queue cannot deadlock;
//  * per-tile metadata (state offset, pass record, R buffer, norm scale) goes
//    from the converter leader to the MMA thread (ordered by the A buffer's full
//    barrier) and to the epilogue (a four-deep ring with its own full / empty
//    barriers); the MMA thread frees an R buffer after the last tile of its
//    item;
//  * each epilogue warp adds its share of the pass's output norm, then
//    increments the circuit's tile counter with release semantics, so a later
//    pass that observes the count (acquire) sees both the stored amplitudes
//    and the norm. A pass's output is rescaled to unit norm, correcting the
//    drift measured on the circuit's previous dense pass (the batch's states
//    start in |0...0>, so their exact norm is 1);
//  * stores keep the default cache policy: the host orders the work in groups
//    of circuits whose states fit in L2 together, so a circuit's next pass
//    mostly reads from L2.
// Every wait is bounded; on expiry the role records the error (the first
// failing wait's site code: 11-14 scheduler, 21-22 converters, 31-33 MMA
// thread, 41-42 epilogue) and stops, the
// converters publish how many tiles they all produced so that the MMA thread
// and the epilogue stop there, the scheduler waits for its bulk copies, and
// the TMEM is freed on exit.
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
constexpr int SCHED_WARP = MMA_WARP + 1;
constexpr int THREADS = (SCHED_WARP + 1) * 32;
constexpr int CONV_THREADS = CONV_WARPS * 32;
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int NMETA = 4;
constexpr uint32_t TMEM_COLS = 512;                   // D0, D1, A0, A1 at 0, 128, 256, 384
constexpr uint32_t OFF_MISC = 2 * DENSE_A_BYTES;       // two R buffers, then barriers, rings, flags
constexpr uint32_t OFF_FLAGS = OFF_MISC + 256;
constexpr uint32_t OFF_DESC = OFF_MISC + 512;
constexpr uint32_t OFF_META = OFF_MISC + 768;
constexpr uint32_t SMEM = OFF_MISC + 2048 + 1024;      // + alignment slack; > half of the SM: one CTA per SM
constexpr uint32_t WAIT_LIMIT = 1u << 23;              // bounded mbarrier polls (about 10 s: a poll can take ~1 us)
constexpr uint32_t SPIN_POLLS = 4096;                  // polls before a wait starts to sleep between polls
constexpr uint32_t DEP_LIMIT = 1u << 22;               // bounded dependency polls (about a second)

// An item handed from the scheduler to the converters.
struct ItemDesc {
    DenseBatchPart P;
    uint32_t tile_begin, tile_count;
    uint32_t stop;     // no more items (queue empty or an error)
    float scale;       // unit-norm rescale of the pass (from the previous pass's output norm)
};
static_assert(sizeof(ItemDesc) == 64, "ItemDesc layout");

// Per-tile record from the converter leader to the MMA thread and epilogue.
struct TileMeta {
    DenseBatchPart P;
    uint64_t tb;       // first amplitude of the tile's circuit + the tile's outer bits
    uint32_t rbuf;     // R buffer holding the pass's image
    uint32_t first;    // first tile of its item (wait for the R image)
    uint32_t last;     // last tile of its item (the R buffer is free after its MMAs)
    float scale;
};
static_assert(sizeof(TileMeta) == 72, "TileMeta layout");
static_assert(OFF_META + NMETA * sizeof(TileMeta) <= OFF_MISC + 2048, "shared memory layout");

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
// Bulk copy of bytes (multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
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

// W consecutive complex64 amplitudes stored with the default cache policy:
// the circuit's next pass reads them again, from L2 when its group of
// circuits fits there.
template <int W>
__device__ __forceinline__ void st_amps_wb(float2 *p, const float2 *y) {
    if constexpr (W == 1) {
        *p = y[0];
    } else if constexpr (W == 2) {
        *reinterpret_cast<float4 *>(p) = make_float4(y[0].x, y[0].y, y[1].x, y[1].y);
    } else {
        asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
                     ::"l"(p), "f"(y[0].x), "f"(y[0].y), "f"(y[1].x), "f"(y[1].y), "f"(y[2].x), "f"(y[2].y),
                       "f"(y[3].x), "f"(y[3].y)
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
// all loaded before any is converted (the loads mostly hit L2; their latency
// bounds the kernel, so as many as possible are in flight), split to BF16 and
// written into TMEM (hi at ta, lo at ta + 64).
template <int W>
__device__ __forceinline__ void convert_tile(const float2 *src, const Geo &g, uint32_t ta) {
    float2 xa[32];
#pragma unroll
    for (int j = 0; j < 32; j += W) {
        uint64_t o = 0;
#pragma unroll
        for (int bb = 0; bb < 5; bb++)
            if ((j >> bb) & 1) o |= g.pbit[bb];
        ld_amps_cg<W>(src + o, xa + j);
    }
#pragma unroll
    for (int gg = 0; gg < 2; gg++) {
        const float2 *x = xa + 16 * gg;
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
            st_amps_wb<W>(dst + o, y);
        }
    }
    return tile_out;
}

// Wait for a barrier phase, or for the converters to have published a tile
// count <= tile (no more tiles); 1 on the phase, 0 on the end, -1 on timeout.
__device__ __forceinline__ int wait_or_end(uint64_t *bar, uint32_t parity, const volatile uint32_t *ntiles,
                                           uint32_t tile) {
    for (uint32_t k = 0; k < WAIT_LIMIT; k++) {
        if (mbar_try(bar, parity)) return 1;
        if (*ntiles <= tile) return 0;
        if (k >= SPIN_POLLS) __nanosleep(128);
    }
    return -1;
}

// Wait for a barrier phase, or false once the CTA's abort flag is set (or
// after the limit). Warp-uniform: the warp proceeds only if every lane saw
// the phase.
__device__ __forceinline__ bool wait_warp(uint64_t *bar, uint32_t parity, const volatile int *abort_flag) {
    bool ok = false;
    for (uint32_t k = 0; k < WAIT_LIMIT; k++) {
        if (mbar_try(bar, parity)) {
            ok = true;
            break;
        }
        if (*abort_flag) break;
        if (k >= SPIN_POLLS) __nanosleep(128);
    }
    return __all_sync(0xffffffffu, ok);
}

// Record a failed wait: the first site's code in err[0], every site's bit
// 4 (code / 10 - 1) + code % 10 in err[7].
__device__ __forceinline__ int fail_site(int *err, int code) {
    atomicOr(err + 7, 1 << (4 * (code / 10 - 1) + code % 10));
    return atomicCAS(err, 0, code);
}

// Single-thread bounded wait (scheduler).
__device__ __forceinline__ bool wait_one(uint64_t *bar, uint32_t parity) {
    for (uint32_t k = 0; k < WAIT_LIMIT; k++) {
        if (mbar_try(bar, parity)) return true;
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
                    *const dempty = bars + 8, *const ifull = bars + 10, *const iempty = bars + 12,
                    *const mfull = bars + 14, *const mempty = bars + 14 + NMETA;
    uint32_t *const flags = reinterpret_cast<uint32_t *>(base + OFF_FLAGS);
    uint32_t *const tslot = flags;                                 // TMEM base address
    volatile uint32_t *const ntiles = flags + 1;                   // tiles produced (set at the end)
    uint32_t *const nmin = flags + 2;                              // min over converters of their tile count
    volatile int *const abort_flag = reinterpret_cast<volatile int *>(flags + 3);
    ItemDesc *const desc = reinterpret_cast<ItemDesc *>(base + OFF_DESC);   // [2]
    TileMeta *const meta = reinterpret_cast<TileMeta *>(base + OFF_META);   // [NMETA]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int b = 0; b < 2; b++) {
            mbar_init(&rfull[b], 1);
            mbar_init(&rempty[b], 1);
            mbar_init(&afull[b], CONV_THREADS);
            mbar_init(&dfull[b], 1);
            mbar_init(&dempty[b], EPI_THREADS);
            mbar_init(&ifull[b], 1);
            mbar_init(&iempty[b], CONV_THREADS);
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

    if (warp == SCHED_WARP) {
        // ------------------------------------------------------ scheduler
        if (lane == 0) {
            uint32_t seq = 0;
            while (true) {
                const uint32_t s = seq & 1, use = seq >> 1;
                // the slot is free once the converters have read item seq - 2
                if (seq >= 2 && !wait_one(&iempty[s], (use - 1) & 1)) {
                    fail_site(err, 11);
                    *abort_flag = 1;
                    break;   // the converters' waits give up on the abort flag
                }
                ItemDesc &D = desc[s];
                // no more work once this CTA or any other has recorded an error
                const bool stop = *abort_flag || *reinterpret_cast<volatile int *>(err) != 0;
                const uint32_t it = stop ? n_items : atomicAdd(head, 1u);
                bool ok = it < n_items;
                DenseBatchItem I{};
                DenseBatchPart P{};
                float scale = 1.0f;
                if (ok) {
                    I = items[it];
                    P = parts[I.part];   // in flight during the dependency poll
                    if (I.wait) {
                        uint32_t k = 0, seen;
                        while ((seen = ld_acquire_u32(done + I.circuit)) < I.wait) {
                            if (++k > DEP_LIMIT) {
                                ok = false;
                                if (fail_site(err, 12) == 0) {
                                    err[1] = (int)it;
                                    err[2] = (int)I.circuit;
                                    err[3] = (int)I.wait;
                                    err[4] = (int)seen;
                                    err[5] = (int)blockIdx.x;
                                    err[6] = (int)seq;
                                }
                                break;
                            }
                            if ((k & 255) == 0 && *reinterpret_cast<volatile int *>(err) != 0) {
                                ok = false;   // another CTA failed: stop here too
                                break;
                            }
                            __nanosleep(64);
                        }
                    }
                    // unit-norm rescale from the previous pass's output norm (final
                    // now; read from L2: its line may hold later passes' running sums)
                    if (ok && P.dn_prev != DENSE_BATCH_NO_PREV) {
                        const double prev = __ldcg(dn + P.dn_prev);
                        if (prev > 0.0) scale = (float)sqrt(1.0 / prev);
                    }
                    // the R buffer is free once the MMAs of item seq - 2 are done
                    if (ok && seq >= 2 && !wait_one(&rempty[s], (use - 1) & 1)) {
                        ok = false;
                        fail_site(err, 13);
                    }
                }
                if (!ok) {
                    D.stop = 1;
                    mbar_arrive(&ifull[s]);
                    break;
                }
                bulk_g2s(sR0 + s * DENSE_A_BYTES, r_imgs + (size_t)I.part * DENSE_A_BYTES, DENSE_A_BYTES, &rfull[s]);
                D.P = P;
                D.tile_begin = I.tile_begin;
                D.tile_count = I.tile_count;
                D.stop = 0;
                D.scale = scale;
                mbar_arrive(&ifull[s]);
                seq++;
            }
            // the bulk copies issued (items seq - 2, seq - 1) have landed before the CTA ends
            for (uint32_t j = seq >= 2 ? seq - 2 : 0; j < seq; j++)
                if (!wait_one(&rfull[j & 1], (j >> 1) & 1)) fail_site(err, 14);
        }
    } else if (warp >= EPI_WARPS && warp < MMA_WARP) {
        // ------------------------------------------------------ converters
        const int ctid = tid - EPI_THREADS;
        uint32_t i = 0, seq = 0;
        while (true) {
            const uint32_t s = seq & 1;
            if (!wait_warp(&ifull[s], (seq >> 1) & 1, abort_flag)) {
                if (lane == 0) fail_site(err, 21);
                *abort_flag = 1;
                break;
            }
            const ItemDesc &D = desc[s];
            if (D.stop) break;
            const DenseBatchPart P = D.P;
            const uint32_t tile_begin = D.tile_begin, tile_count = D.tile_count;
            const float scale = D.scale;
            mbar_arrive(&iempty[s]);   // the descriptor is in registers: the slot is free
            const uint32_t rb = s;
            Geo g;
            geometry(P, n_col, g);
            const uint64_t hoff = h ? g.pbit[DENSE_K - 1] : 0ull;
            const uint64_t low = P.outer_mask & (~P.outer_mask + 1);   // tile index 1 deposited
            uint64_t tb = deposit_bits(tile_begin, P.outer_mask);
            bool bad = false;
            for (uint32_t t = 0; t < tile_count; t++) {
                const uint32_t b = i & 1, m = i & (NMETA - 1);
                if ((i >= 2 && !wait_warp(&dfull[b], ((i >> 1) - 1) & 1, abort_flag)) ||
                    (i >= NMETA && !wait_warp(&mempty[m], ((i / NMETA) - 1) & 1, abort_flag))) {
                    bad = true;
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
                    M.P = P;
                    M.tb = tabs;
                    M.rbuf = rb;
                    M.first = t == 0;
                    M.last = t + 1 == tile_count;
                    M.scale = scale;
                }
                tmem_st_wait();
                tc_fence_before();
                mbar_arrive(&afull[b]);
                if (ctid == 0) mbar_arrive(&mfull[m]);
                i++;
                tb = masked_add(tb, low, P.outer_mask);
            }
            if (bad) {
                if (lane == 0) fail_site(err, 22);
                *abort_flag = 1;
                break;
            }
            seq++;
        }
        // the MMA thread and the epilogue stop after the tiles every converter produced
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
                    fail_site(err, 31);
                    break;
                }
                const TileMeta &M = meta[i & (NMETA - 1)];
                const uint32_t rbuf = M.rbuf, last = M.last;
                if (M.first) {
                    if (wait_or_end(&rfull[rbuf], ruse[rbuf] & 1, ntiles, i) != 1) {
                        fail_site(err, 32);
                        break;
                    }
                    ruse[rbuf]++;
                }
                tc_fence_after();
                const uint32_t sb = smem_u32(sR0 + rbuf * DENSE_A_BYTES);
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
                umma_commit(&dfull[b]);                 // accumulator ready, A buffer consumed
                if (last) umma_commit(&rempty[rbuf]);   // the item's R buffer is free
                i++;
            }
            // the MMAs issued complete before the TMEM is freed
            if (i > 0 && !wait_one(&dfull[(i - 1) & 1], ((i - 1) >> 1) & 1)) fail_site(err, 33);
        }
    } else {
        // ------------------------------------------------------ epilogue
        uint32_t i = 0;
        while (true) {
            const uint32_t b = i & 1, m = i & (NMETA - 1);
            const int r = wait_or_end(&mfull[m], (i / NMETA) & 1, ntiles, i);
            if (__any_sync(0xffffffffu, r != 1)) {
                if (__any_sync(0xffffffffu, r < 0) && lane == 0) fail_site(err, 41);
                break;
            }
            const TileMeta &M = meta[m];
            const DenseBatchPart P = M.P;
            const uint64_t mtb = M.tb;
            const float scale = M.scale;
            mbar_arrive(&mempty[m]);
            Geo g;
            geometry(P, n_col, g);
            const int rd = wait_or_end(&dfull[b], (i >> 1) & 1, ntiles, i);
            if (__any_sync(0xffffffffu, rd != 1)) {
                if (__any_sync(0xffffffffu, rd < 0) && lane == 0) fail_site(err, 42);
                break;
            }
            tc_fence_after();
            const uint32_t td = tmem + ((uint32_t)(32 * q) << 16) + 128 * b;
            float2 *const dst = svbase + (mtb + g.coff);
            float part_norm;
            if (g.w == 4) part_norm = store_tile<4>(dst, g, td, scale, &dempty[b]);
            else if (g.w == 2) part_norm = store_tile<2>(dst, g, td, scale, &dempty[b]);
            else part_norm = store_tile<1>(dst, g, td, scale, &dempty[b]);
            double sum = (double)part_norm;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            __syncwarp();   // the warp's stores are ordered before lane 0's release below
            if (lane == 0) {
                atomicAdd(dn + P.dn_out, sum);
                // the fence stays: without it, runs of 16-tile items stalled
                // one CTA's pipeline until its bounded waits gave up
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
    if ((reinterpret_cast<uintptr_t>(svbase) & 31) || (reinterpret_cast<uintptr_t>(r_imgs) & 15))
        return cudaErrorMisalignedAddress;
    unsigned grid = (unsigned)sms;
    if (n_items < grid) grid = n_items < 1 ? 1 : n_items;
    k_dense6_batch<<<grid, THREADS, SMEM, st>>>(reinterpret_cast<float2 *>(svbase), parts, items, n_items,
                                                reinterpret_cast<const uint8_t *>(r_imgs), done, head, err, dn);
    return cudaGetLastError();
}

}  // namespace hisv
