// C ABI of the batched persistent launch (sv_batch_*; declared in include/hisvsim.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "abi_internal.hpp"
#include "batch.hpp"
#include "dense_batch.hpp"
#include "planner.hpp"

using namespace hisv;

namespace {
sv_status bfail(sv_status st, const std::string &msg) {
    set_last_error(msg);
    return st;
}
#define BCUDA(call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail(SV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
}  // namespace

struct sv_batch {
    uint32_t n = 0;                      // circuits
    std::vector<int> nq;                 // qubits per circuit
    std::vector<uint64_t> off;           // first amplitude per circuit
    uint64_t total = 0;                  // amplitudes in all states
    std::vector<sv_plan *> plans;
    cudaStream_t stream = nullptr;       // the caller's stream: graph launches, probabilities, frees
    bool own_stream = false;
    cudaStream_t prep = nullptr;         // private: allocations, uploads and the graph capture, so that
                                         // building a batch never enqueues on (or captures) a stream that
                                         // another thread uses for earlier batches
    int warps = 8;                       // warps per CTA
    int chunk = 16;                      // tiles per queue item
    bool hold_last = false;              // testing: the last item waits for tiles that never complete
    int dense_min = 0;                   // circuits of >= this many qubits (and >= 13) with parts of <= 6
                                         // qubits run on the batched tensor-core kernel; 0 = off
    int dense_chunk = 2;                 // tiles (2^13 amplitudes) per dense work item
    int dense_group = 1024;              // tiles of state per group of circuits in the dense work order
    // device
    float2 *sv = nullptr;
    uint64_t *d_off = nullptr;
    uint32_t *d_nq = nullptr;
    uint32_t *d_done = nullptr;          // n counters + the two queue tickets (gate lists, dense)
    int *d_err = nullptr;                // error word, then the dense kernel's record of a failed wait
    double *d_norms = nullptr;
    std::vector<double> h_norms;
    // compiled program (rebuilt when plans or the configuration change)
    bool built = false;
    BatchLaunch launch{};
    void *d_prog = nullptr;              // one allocation: items, parts, phases, ops, coefs
    uint32_t n_items = 0, n_parts = 0;
    void *d_dprog = nullptr;             // one allocation: dense items, parts, R images, norm slots
    uint32_t n_dense_items = 0, n_dense_parts = 0, n_dense_circ = 0;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
};

static void drop_program(sv_batch *b) {
    if (b->prep) cudaStreamSynchronize(b->prep);   // no upload into the program is still in flight
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    dev_free(b->d_prog, b->stream);   // after the launches already queued on the stream
    dev_free(b->d_dprog, b->stream);
    b->d_prog = nullptr;
    b->d_dprog = nullptr;
    b->n_items = b->n_parts = b->n_dense_items = b->n_dense_parts = b->n_dense_circ = 0;
    b->built = false;
}

extern "C" {

sv_status sv_batch_create(uint32_t n_circuits, const int *n_qubits, void *stream, sv_batch **out) {
    if (!out) return bfail(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_circuits == 0 || !n_qubits) return bfail(SV_ERR_ARG, "need at least one circuit");
    std::unique_ptr<sv_batch> b(new sv_batch());
    b->n = n_circuits;
    b->nq.assign(n_qubits, n_qubits + n_circuits);
    b->off.resize(n_circuits);
    for (uint32_t i = 0; i < n_circuits; i++) {
        if (b->nq[i] < BATCH_MIN_QUBITS || b->nq[i] > 30)
            return bfail(SV_ERR_ARG, "batched circuits need 10..30 qubits (circuit " + std::to_string(i) + ")");
        b->off[i] = b->total;
        b->total += 1ull << b->nq[i];
    }
    b->plans.assign(n_circuits, nullptr);
    b->h_norms.assign(n_circuits, 0.0);
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    if (!b->stream) {   // graph launches need a non-legacy stream
        BCUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        b->own_stream = true;
    }
    {
        cudaError_t pe = cudaStreamCreateWithFlags(&b->prep, cudaStreamNonBlocking);
        if (pe != cudaSuccess) {
            if (b->own_stream) cudaStreamDestroy(b->stream);
            return bfail(SV_ERR_CUDA, std::string("batch stream: ") + cudaGetErrorString(pe));
        }
    }
    // allocated and initialised on the private stream, which is synchronised
    // before the batch is returned: the buffers are ready for any stream
    cudaStream_t st = b->prep;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&b->sv), sizeof(float2) * b->total, st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&b->d_off), sizeof(uint64_t) * n_circuits, st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&b->d_nq), sizeof(uint32_t) * n_circuits, st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&b->d_done), sizeof(uint32_t) * (n_circuits + 2), st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&b->d_err), sizeof(int) * DENSE_BATCH_ERR_WORDS, st);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&b->d_norms), sizeof(double) * n_circuits, st);
    std::vector<uint32_t> nq32(b->nq.begin(), b->nq.end());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_off, b->off.data(), sizeof(uint64_t) * n_circuits, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_nq, nq32.data(), sizeof(uint32_t) * n_circuits, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int) * DENSE_BATCH_ERR_WORDS, st);
    if (e == cudaSuccess) e = launch_batch_reset(b->sv, b->d_off, n_circuits, b->total, st);
    cudaError_t se = cudaStreamSynchronize(st);   // also: the host vectors above go out of scope
    if (e == cudaSuccess) e = se;
    if (e != cudaSuccess) {
        cudaGetLastError();
        dev_free(b->sv, st); dev_free(b->d_off, st); dev_free(b->d_nq, st); dev_free(b->d_done, st);
        dev_free(b->d_err, st); dev_free(b->d_norms, st);
        cudaStreamSynchronize(st);
        cudaStreamDestroy(b->prep);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        return bfail(e == cudaErrorMemoryAllocation ? SV_ERR_OOM : SV_ERR_CUDA,
                     std::string("batch allocation: ") + cudaGetErrorString(e));
    }
    *out = b.release();
    return SV_OK;
}

sv_status sv_batch_set_plan(sv_batch *b, uint32_t i, sv_plan *p) {
    if (!b || !p) return bfail(SV_ERR_ARG, "NULL argument");
    if (i >= b->n) return bfail(SV_ERR_ARG, "circuit index out of range");
    if (p->n != b->nq[i]) return bfail(SV_ERR_ARG, "plan qubit count differs from circuit " + std::to_string(i));
    if (p->method == SV_PART_NONE) return bfail(SV_ERR_ARG, "batched circuits need a partitioned plan");
    if (p->max_part > BATCH_TILE_QUBITS) return bfail(SV_ERR_PARTITION, "batched parts are limited to 9 qubits (k <= 9)");
    b->plans[i] = p;
    drop_program(b);
    return SV_OK;
}

sv_status sv_batch_config(sv_batch *b, int warps_per_cta, int tiles_per_item) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    if (warps_per_cta < 0 || warps_per_cta > 8 || tiles_per_item < 0 || tiles_per_item > 4096)
        return bfail(SV_ERR_ARG, "warps_per_cta in [1, 8], tiles_per_item in [1, 4096] (0 = default)");
    b->warps = warps_per_cta ? warps_per_cta : 8;
    b->chunk = tiles_per_item ? tiles_per_item : 16;
    drop_program(b);
    return SV_OK;
}

// The dense circuits: the dense kernel is on, the circuit has enough qubits
// and its plan's parts have at most 6 qubits, so the planner makes every
// part a dense tensor-core pass. One DenseBatchPart and one R image per pass,
// work items of dense_chunk tiles in wave order, one norm slot per pass.
// Worker threads compile the circuits on all host cores; a dense circuit's R
// images go straight to their place on the device (a batch of thousands of
// circuits has hundreds of thousands of passes, 64 KiB of image each).
struct DenseLayout {
    std::vector<char> dense;             // per circuit
    std::vector<uint32_t> base, npass;   // first pass, passes per circuit
    uint32_t n_parts = 0, n_circ = 0;
    std::vector<DenseBatchItem> items;
    size_t s_items = 0, s_parts = 0, s_img = 0, s_dn = 0;
};

static void dense_layout(sv_batch *b, DenseLayout &D) {
    D.dense.assign(b->n, 0);
    D.base.assign(b->n, 0);
    D.npass.assign(b->n, 0);
    const int dmin = std::max(b->dense_min, DENSE_K + DENSE_COLS);
    for (uint32_t c = 0; c < b->n; c++) {
        const sv_plan *p = b->plans[c];
        if (b->dense_min <= 0 || p->n < dmin || p->max_part > DENSE_K) continue;
        D.dense[c] = 1;
        D.base[c] = D.n_parts;
        D.npass[c] = p->n_parts;
        D.n_parts += p->n_parts;
        D.n_circ++;
    }
    // Groups of circuits whose states together hold about dense_group tiles
    // (64 KiB each), circuits sorted by pass count so that a group's waves
    // stay full; each group's items in wave order, one group after another.
    // A group's states stay in L2 from one pass to the next.
    std::vector<uint32_t> order;
    for (uint32_t c = 0; c < b->n; c++)
        if (D.dense[c]) order.push_back(c);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        return D.npass[x] != D.npass[y] ? D.npass[x] > D.npass[y] : b->nq[x] > b->nq[y];
    });
    size_t g0 = 0;
    while (g0 < order.size()) {
        size_t g1 = g0;
        uint64_t tiles = 0;
        uint32_t gP = 0;
        while (g1 < order.size() && (g1 == g0 || tiles < (uint64_t)b->dense_group)) {
            const uint32_t c = order[g1++];
            tiles += 1ull << (b->nq[c] - DENSE_K - DENSE_COLS);
            gP = std::max(gP, D.npass[c]);
        }
        for (uint32_t w = 0; w < gP; w++)
            for (size_t k = g0; k < g1; k++) {
                const uint32_t c = order[k];
                if (w >= D.npass[c]) continue;
                const uint32_t nt = 1u << (b->nq[c] - DENSE_K - DENSE_COLS);
                for (uint32_t t0 = 0; t0 < nt; t0 += (uint32_t)b->dense_chunk) {
                    DenseBatchItem it{};
                    it.part = D.base[c] + w;
                    it.circuit = c;
                    it.tile_begin = t0;
                    it.tile_count = std::min<uint32_t>((uint32_t)b->dense_chunk, nt - t0);
                    it.wait = 4 * nt * w;   // every tile of the circuit's earlier passes, four warps each
                    D.items.push_back(it);
                }
            }
        g0 = g1;
    }
    if (b->hold_last && !D.items.empty()) D.items.back().wait = 0xFFFFFFFFu;
    auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
    D.s_items = al(D.items.size() * sizeof(DenseBatchItem));
    D.s_parts = al((size_t)D.n_parts * sizeof(DenseBatchPart));
    D.s_img = (size_t)D.n_parts * DENSE_A_BYTES;
    D.s_dn = al((size_t)D.n_parts * sizeof(double));
}

static sv_status build_program(sv_batch *b) {
    for (uint32_t c = 0; c < b->n; c++)
        if (!b->plans[c]) return bfail(SV_ERR_ARG, "circuit " + std::to_string(c) + " has no plan");
    DenseLayout D;
    dense_layout(b, D);
    char *dd = nullptr;
    if (D.n_circ) {
        cudaError_t e = dev_alloc(reinterpret_cast<void **>(&dd), D.s_items + D.s_parts + D.s_img + D.s_dn, b->prep);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(SV_ERR_OOM, std::string("dense batch program: ") + cudaGetErrorString(e));
        }
        b->d_dprog = dd;
    }
    int dev = 0;
    BCUDA(cudaGetDevice(&dev));
    std::vector<Program> gl(b->n);                 // gate-list programs (circuits not on the dense kernel)
    std::vector<DenseBatchPart> dparts(D.n_parts);
    std::vector<std::string> errs(b->n);
    std::atomic<uint32_t> next(0);
    auto work = [&]() {
        cudaSetDevice(dev);
        for (uint32_t c = next++; c < b->n; c = next++) {
            sv_plan *p = b->plans[c];
            if (!D.dense[c]) {
                if (!compile_program(p->gates, p->n, p->pog, p->n_parts, false, BATCH_TILE_QUBITS, BATCH_REG_BITS, 0,
                                     gl[c], errs[c]) && errs[c].empty())
                    errs[c] = "compile failed";
                continue;
            }
            Program pr;
            if (!compile_program(p->gates, p->n, p->pog, p->n_parts, false, BATCH_TILE_QUBITS, BATCH_REG_BITS, 1, pr,
                                 errs[c])) {
                if (errs[c].empty()) errs[c] = "compile failed";
                continue;
            }
            bool all = pr.kind.size() == D.npass[c];
            for (size_t w = 0; all && w < pr.kind.size(); w++) all = pr.kind[w] == 1 && pr.index[w] == w;
            if (!all) {
                errs[c] = "circuit " + std::to_string(c) + ": a part did not compile to a dense pass";
                continue;
            }
            for (uint32_t w = 0; w < D.npass[c]; w++) {
                const DenseLaunch &L = pr.dense[w];
                DenseBatchPart &P = dparts[D.base[c] + w];
                std::memset(&P, 0, sizeof(P));
                P.sv_off = b->off[c];
                P.outer_mask = L.outer_mask;
                P.circuit = c;
                P.dn_prev = w == 0 ? DENSE_BATCH_NO_PREV : D.base[c] + w - 1;
                P.dn_out = D.base[c] + w;
                std::memcpy(P.part_q, L.part_q, DENSE_K);
                std::memcpy(P.col_q, L.col_q, DENSE_COLS);
                P.n = (uint8_t)b->nq[c];
            }
            // a pageable source is staged before the call returns: pr may go
            cudaError_t e = cudaMemcpyAsync(dd + D.s_items + D.s_parts + (size_t)D.base[c] * DENSE_A_BYTES,
                                            pr.a_img.data(), (size_t)D.npass[c] * DENSE_A_BYTES,
                                            cudaMemcpyHostToDevice, b->prep);
            if (e != cudaSuccess) errs[c] = std::string("R image upload: ") + cudaGetErrorString(e);
        }
    };
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min({nt, 32u, b->n}));
    std::vector<std::thread> th;
    for (unsigned k = 1; k < nt; k++) th.emplace_back(work);
    work();
    for (auto &t : th) t.join();
    for (uint32_t c = 0; c < b->n; c++)
        if (!errs[c].empty()) {
            cudaStreamSynchronize(b->prep);   // no upload into the program is left in flight when it is freed
            return bfail(SV_ERR_PARTITION, errs[c]);
        }
    if (D.n_circ) {
        BCUDA(cudaMemcpyAsync(dd, D.items.data(), D.items.size() * sizeof(DenseBatchItem), cudaMemcpyHostToDevice,
                              b->prep));
        BCUDA(cudaMemcpyAsync(dd + D.s_items, dparts.data(), dparts.size() * sizeof(DenseBatchPart),
                              cudaMemcpyHostToDevice, b->prep));
        b->n_dense_items = (uint32_t)D.items.size();
        b->n_dense_parts = D.n_parts;
        b->n_dense_circ = D.n_circ;
    }
    std::vector<PartLaunch> parts;
    std::vector<Phase> phases;
    std::vector<Op> ops;
    std::vector<float> coefs;
    std::vector<uint32_t> part_base(b->n), n_parts(b->n);
    uint32_t maxP = 0;
    for (uint32_t c = 0; c < b->n; c++) {
        if (D.dense[c]) {
            n_parts[c] = 0;
            continue;
        }
        const Program &prog = gl[c];
        const uint32_t ph0 = (uint32_t)phases.size(), op0 = (uint32_t)ops.size(), cf0 = (uint32_t)coefs.size();
        part_base[c] = (uint32_t)parts.size();
        n_parts[c] = (uint32_t)prog.parts.size();
        maxP = std::max(maxP, n_parts[c]);
        for (PartLaunch L : prog.parts) {
            L.phase_begin += ph0;
            L.op_begin += op0;
            L.op_end += op0;
            L.coef_begin += cf0;
            L.coef_end += cf0;
            parts.push_back(L);
        }
        for (Phase ph : prog.phases) {
            ph.op_begin += op0;
            phases.push_back(ph);
        }
        for (Op op : prog.ops) {
            op.coef += cf0;
            ops.push_back(op);
        }
        for (double v : prog.coefs) coefs.push_back((float)v);
    }
    std::vector<BatchItem> items;
    for (uint32_t w = 0; w < maxP; w++)
        for (uint32_t c = 0; c < b->n; c++) {
            if (w >= n_parts[c]) continue;
            const uint32_t nt = 1u << (b->nq[c] - BATCH_TILE_QUBITS);
            for (uint32_t t0 = 0; t0 < nt; t0 += (uint32_t)b->chunk) {
                BatchItem it;
                it.circuit = c;
                it.part = part_base[c] + w;
                it.tile_begin = t0;
                it.tile_count = std::min<uint32_t>((uint32_t)b->chunk, nt - t0);
                it.wait = w * nt;
                items.push_back(it);
            }
        }
    if (b->hold_last && !items.empty()) items.back().wait = 0xFFFFFFFFu;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t s_items = al(items.size() * sizeof(BatchItem)), s_parts = al(parts.size() * sizeof(PartLaunch));
    const size_t s_ph = al(phases.size() * sizeof(Phase)), s_op = al(ops.size() * sizeof(Op));
    const size_t s_cf = al(std::max<size_t>(1, coefs.size()) * sizeof(float));
    char *d = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&d), s_items + s_parts + s_ph + s_op + s_cf, b->prep);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(SV_ERR_OOM, std::string("batch program: ") + cudaGetErrorString(e));
    }
    b->d_prog = d;
    std::vector<char> host(s_items + s_parts + s_ph + s_op + s_cf, 0);
    // (an empty vector's data() may be null, which memcpy must not get)
    auto put = [&](size_t at, const void *src, size_t bytes) {
        if (bytes) std::memcpy(host.data() + at, src, bytes);
    };
    put(0, items.data(), items.size() * sizeof(BatchItem));
    put(s_items, parts.data(), parts.size() * sizeof(PartLaunch));
    put(s_items + s_parts, phases.data(), phases.size() * sizeof(Phase));
    put(s_items + s_parts + s_ph, ops.data(), ops.size() * sizeof(Op));
    put(s_items + s_parts + s_ph + s_op, coefs.data(), coefs.size() * sizeof(float));
    BCUDA(cudaMemcpyAsync(d, host.data(), host.size(), cudaMemcpyHostToDevice, b->prep));
    // every upload (gate lists, dense items, parts and R images) is complete
    // before the graph can be launched on any stream
    BCUDA(cudaStreamSynchronize(b->prep));
    BatchLaunch &B = b->launch;
    B.svbase = b->sv;
    B.items = reinterpret_cast<const BatchItem *>(d);
    B.n_items = (uint32_t)items.size();
    B.circ_off = b->d_off;
    B.parts = reinterpret_cast<const PartLaunch *>(d + s_items);
    B.phases = reinterpret_cast<const Phase *>(d + s_items + s_parts);
    B.ops = reinterpret_cast<const Op *>(d + s_items + s_parts + s_ph);
    B.coefs = reinterpret_cast<const float *>(d + s_items + s_parts + s_ph + s_op);
    B.done = b->d_done;
    B.head = b->d_done + b->n;
    B.err = b->d_err;
    b->n_items = B.n_items;
    b->n_parts = (uint32_t)parts.size();
    int n_ctas = 0;
    BCUDA(batch_prepare(b->warps, &n_ctas));
    // one graph: zero the tile counters, the tickets and the dense passes'
    // norm slots, then the persistent launches (dense circuits, gate lists)
    const size_t ds_items = D.s_items, ds_parts = D.s_parts, ds_img = D.s_img;
    // captured on the private stream (nothing else is ever enqueued there),
    // launched on the caller's stream
    BCUDA(cudaStreamBeginCapture(b->prep, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaMemsetAsync(b->d_done, 0, sizeof(uint32_t) * (b->n + 2), b->prep);
    if (ce == cudaSuccess && b->n_dense_items) {
        double *dn = reinterpret_cast<double *>(dd + ds_items + ds_parts + ds_img);
        ce = cudaMemsetAsync(dn, 0, sizeof(double) * b->n_dense_parts, b->prep);
        if (ce == cudaSuccess)
            ce = launch_dense6_batch(b->sv, reinterpret_cast<const DenseBatchPart *>(dd + ds_items),
                                     reinterpret_cast<const DenseBatchItem *>(dd), b->n_dense_items,
                                     dd + ds_items + ds_parts, b->d_done, b->d_done + b->n + 1, b->d_err, dn,
                                     b->prep);
    }
    if (ce == cudaSuccess && B.n_items) ce = launch_batch(B, b->warps, n_ctas, b->prep);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(b->prep, &g);
    if (ce != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(SV_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    b->graph = g;
    BCUDA(cudaGraphInstantiate(&b->gexec, g, 0));
    b->built = true;
    return SV_OK;
}

static sv_status batch_check(sv_batch *b) {
    int h[DENSE_BATCH_ERR_WORDS] = {};
    BCUDA(cudaMemcpyAsync(h, b->d_err, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
    BCUDA(cudaStreamSynchronize(b->stream));
    if (h[0]) {
        BCUDA(cudaMemsetAsync(b->d_err, 0, sizeof(h), b->stream));
        std::string msg = "a bounded wait of the batched kernel gave up (wait site " + std::to_string(h[0]);
        if (h[0] == 12) {   // the dense scheduler's dependency wait: item, circuit, target, counter seen
            msg += "; item " + std::to_string((uint32_t)h[1]) + " circuit " + std::to_string((uint32_t)h[2]) +
                   " waits for " + std::to_string((uint32_t)h[3]) + ", counter " + std::to_string((uint32_t)h[4]) +
                   ", CTA " + std::to_string(h[5]) + " item #" + std::to_string(h[6]);
        }
        if (h[7]) msg += "; failed sites bitmask (bit 4 (site / 10 - 1) + site % 10): " + std::to_string(h[7]);
        return bfail(SV_ERR_TIMEOUT, msg + ")");
    }
    return SV_OK;
}

sv_status sv_batch_run(sv_batch *b, uint32_t flags) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    if (!b->built) {
        sv_status st = build_program(b);
        if (st != SV_OK) {
            drop_program(b);
            return st;
        }
    }
    BCUDA(cudaGraphLaunch(b->gexec, b->stream));
    if (flags & SV_FLAG_SYNC) return batch_check(b);
    return SV_OK;
}

sv_status sv_batch_prepare(sv_batch *b) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    if (!b->built) {
        sv_status st = build_program(b);
        if (st != SV_OK) {
            drop_program(b);
            return st;
        }
    }
    return SV_OK;
}

sv_status sv_batch_hold_last_item(sv_batch *b, int on) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    b->hold_last = on != 0;
    drop_program(b);
    return SV_OK;
}

sv_status sv_batch_sync(sv_batch *b) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    return batch_check(b);
}

sv_status sv_batch_reset(sv_batch *b) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    BCUDA(launch_batch_reset(b->sv, b->d_off, b->n, b->total, b->stream));
    return SV_OK;
}

sv_status sv_batch_probs(sv_batch *b, void *dev_out, double *norms_host) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    BCUDA(launch_batch_probs(b->sv, b->d_off, b->d_nq, b->n, reinterpret_cast<float *>(dev_out), b->d_norms,
                             b->stream));
    if (norms_host) {
        BCUDA(cudaMemcpyAsync(b->h_norms.data(), b->d_norms, sizeof(double) * b->n, cudaMemcpyDeviceToHost,
                              b->stream));
        BCUDA(cudaStreamSynchronize(b->stream));
        if (b->n) std::memcpy(norms_host, b->h_norms.data(), sizeof(double) * b->n);
    }
    return SV_OK;
}

sv_status sv_batch_state(sv_batch *b, uint32_t i, void **dev_ptr, size_t *bytes) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    if (i >= b->n) return bfail(SV_ERR_ARG, "circuit index out of range");
    if (dev_ptr) *dev_ptr = b->sv + b->off[i];
    if (bytes) *bytes = sizeof(float2) << b->nq[i];
    return SV_OK;
}

sv_status sv_batch_copy_state(sv_batch *b, uint32_t i, void *host_dst, size_t bytes) {
    if (!b || !host_dst) return bfail(SV_ERR_ARG, "NULL argument");
    if (i >= b->n) return bfail(SV_ERR_ARG, "circuit index out of range");
    if (bytes != (sizeof(float2) << b->nq[i])) return bfail(SV_ERR_ARG, "bytes must equal the state size");
    BCUDA(cudaMemcpyAsync(host_dst, b->sv + b->off[i], bytes, cudaMemcpyDeviceToHost, b->stream));
    return batch_check(b);
}

sv_status sv_batch_info(sv_batch *b, uint64_t *total_amplitudes, uint32_t *n_items, uint32_t *n_parts) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    if (total_amplitudes) *total_amplitudes = b->total;
    if (n_items) *n_items = b->n_items;
    if (n_parts) *n_parts = b->n_parts;
    return SV_OK;
}

sv_status sv_batch_set_dense(sv_batch *b, int min_qubits, int tiles_per_item, int group_tiles) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    if (min_qubits < 0 || min_qubits > 30 || tiles_per_item < 0 || tiles_per_item > 4096 || group_tiles < 0)
        return bfail(SV_ERR_ARG, "min_qubits in [0, 30] (0 = off), tiles_per_item in [1, 4096] (0 = default), "
                                 "group_tiles >= 0 (0 = default)");
    b->dense_min = min_qubits;
    b->dense_chunk = tiles_per_item ? tiles_per_item : 2;
    b->dense_group = group_tiles ? group_tiles : 1024;
    drop_program(b);
    return SV_OK;
}

sv_status sv_batch_dense_info(sv_batch *b, uint32_t *n_circuits, uint32_t *n_items, uint32_t *n_passes) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    if (n_circuits) *n_circuits = b->n_dense_circ;
    if (n_items) *n_items = b->n_dense_items;
    if (n_passes) *n_passes = b->n_dense_parts;
    return SV_OK;
}

sv_status sv_batch_destroy(sv_batch *b) {
    if (!b) return bfail(SV_ERR_ARG, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    drop_program(b);
    dev_free(b->sv, b->stream);
    dev_free(b->d_off, b->stream);
    dev_free(b->d_nq, b->stream);
    dev_free(b->d_done, b->stream);
    dev_free(b->d_err, b->stream);
    dev_free(b->d_norms, b->stream);
    if (b->own_stream) {
        cudaStreamSynchronize(b->stream);   // the frees complete before the stream goes
        cudaStreamDestroy(b->stream);
    }
    cudaStreamDestroy(b->prep);             // idle: drop_program synchronised it
    delete b;
    if (e != cudaSuccess) return bfail(SV_ERR_CUDA, std::string("pending batch work failed: ") + cudaGetErrorString(e));
    return SV_OK;
}

}  // extern "C"
