// C ABI of the library (declared in include/hisvsim.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hisvsim.h"
#include "abi_internal.hpp"
#include "dense.hpp"
#include "kernels.hpp"
#include "partition.hpp"
#include "planner.hpp"

using namespace hisv;

namespace {
thread_local std::string g_err = "no error";

sv_status fail(sv_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

#define CUDA_TRY(call)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(SV_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));    \
    } while (0)

constexpr int kProbBlocks = 152 * 8;
// per-state reduction scratch: kProbBlocks partial sums and the norm
// (sv_measure_probs), then 3 * kProbBlocks block results and 4 outputs
// (sv_measure_summary)
constexpr int kSummaryAt = kProbBlocks + 1;
constexpr int kPartialsLen = kSummaryAt + 3 * kProbBlocks + 4;
}  // namespace

namespace hisv {
void set_last_error(const std::string &msg) { g_err = msg; }
}

static size_t amp_bytes(sv_precision p) { return p == SV_C64 ? 8 : 16; }
// complex128 and its double-float form share the FP64 program (tile, register bits)
static bool is_fp64(const sv_state *s) { return s->prec != SV_C64; }
static bool is_df(const sv_state *s) { return s->prec == SV_C128DF; }
constexpr uint64_t kStageAmps = 1ull << 21;   // 32 MiB of double2 per staged download chunk

// Default tile: 2^12 complex64 / 2^11 complex128 amplitudes per CTA (two
// 64 KiB shared buffers, three CTAs per SM), grown so that the tile holds
// the plan's largest part and, where the limit allows, enough of the lowest
// free qubits that every contiguous run of a gathered tile fills a 32-byte
// sector: two qubits (4 amplitudes) for complex64, one for the 16-byte
// complex128 forms. A part without the state's low qubits otherwise reads
// runs of one amplitude, and the shared-memory fill of the tile, not the
// HBM traffic, sets the pace (measured at k = 12: 1.4-1.8x slower per pass
// with the 2^12 tile than with 2^13).
static int default_tile(bool fp64, int max_part) {
    int t = fp64 ? 11 : 12;
    const int fill = fp64 ? 1 : 2;
    if (max_part + fill > t) t = max_part + fill;
    return t > part_tmax(fp64) ? part_tmax(fp64) : t;
}

extern "C" {

const char *sv_last_error(void) { return g_err.c_str(); }
const char *sv_version(void) { return "hisvsim-gb300 0.1 (sm_103a)"; }

}  // extern "C"

static sv_status create_state(int n, sv_precision prec, void *dev_buf, size_t dev_buf_bytes, void *stream, bool init,
                              sv_state **out) {
    if (!out) return fail(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 36) return fail(SV_ERR_ARG, "n_qubits must be in [1, 36]");
    if (prec != SV_C64 && prec != SV_C128 && prec != SV_C128DF) return fail(SV_ERR_ARG, "bad precision");
    const size_t bytes = amp_bytes(prec) << n;
    if (dev_buf && dev_buf_bytes < bytes) return fail(SV_ERR_ARG, "dev_buf smaller than 2^n amplitudes");
    if (dev_buf && (reinterpret_cast<uintptr_t>(dev_buf) & 15)) return fail(SV_ERR_ARG, "dev_buf must be 16-byte aligned");
    std::unique_ptr<sv_state> s(new sv_state());
    s->n = n;
    s->prec = prec;
    s->bytes = bytes;
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaGetDevice(&s->dev));
    if (dev_buf) {
        s->buf = dev_buf;
    } else {
        cudaError_t e = dev_alloc(&s->buf, bytes, s->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(SV_ERR_OOM, std::string("state allocation: ") + cudaGetErrorString(e));
        }
        s->owns = true;
    }
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&s->d_partials), sizeof(double) * kPartialsLen, s->stream);
    if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&s->d_err), sizeof(int), s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (s->owns) dev_free(s->buf, s->stream);
        dev_free(s->d_partials, s->stream);
        dev_free(s->d_err, s->stream);
        return fail(SV_ERR_OOM, std::string("scratch allocation: ") + cudaGetErrorString(e));
    }
    if (init) e = launch_set_basis(is_fp64(s.get()), s->buf, n, 0, s->stream, is_df(s.get()));
    if (e != cudaSuccess) {
        if (s->owns) dev_free(s->buf, s->stream);
        dev_free(s->d_partials, s->stream);
        dev_free(s->d_err, s->stream);
        return fail(SV_ERR_CUDA, std::string("init: ") + cudaGetErrorString(e));
    }
    *out = s.release();
    return SV_OK;
}

extern "C" {

sv_status sv_create(int n, sv_precision prec, void *dev_buf, size_t dev_buf_bytes, void *stream, sv_state **out) {
    return create_state(n, prec, dev_buf, dev_buf_bytes, stream, true, out);
}

sv_status sv_attach(int n, sv_precision prec, void *dev_buf, size_t dev_buf_bytes, void *stream, sv_state **out) {
    if (!dev_buf) return fail(SV_ERR_ARG, "sv_attach needs dev_buf");
    return create_state(n, prec, dev_buf, dev_buf_bytes, stream, false, out);
}

sv_status sv_destroy(sv_state *s) {
    if (!s) return fail(SV_ERR_ARG, "state is NULL");
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (s->owns) dev_free(s->buf, s->stream);
    dev_free(s->d_partials, s->stream);
    dev_free(s->d_err, s->stream);
    dev_free(s->d_dnorm, s->stream);
    dev_free(s->d_stage, s->stream);
    delete s;
    if (e != cudaSuccess) return fail(SV_ERR_CUDA, std::string("pending work failed: ") + cudaGetErrorString(e));
    return SV_OK;
}

sv_status sv_set_basis(sv_state *s, uint64_t index) {
    if (!s) return fail(SV_ERR_ARG, "state is NULL");
    if (index >> s->n) return fail(SV_ERR_ARG, "basis index >= 2^n");
    CUDA_TRY(launch_set_basis(is_fp64(s), s->buf, s->n, index, s->stream, is_df(s)));
    return SV_OK;
}

sv_status sv_upload(sv_state *s, const void *src, size_t bytes) {
    if (!s || !src) return fail(SV_ERR_ARG, "NULL argument");
    if (bytes != s->bytes) return fail(SV_ERR_ARG, "bytes must equal the state size");
    CUDA_TRY(cudaMemcpyAsync(s->buf, src, bytes, cudaMemcpyHostToDevice, s->stream));
    if (is_df(s)) CUDA_TRY(launch_to_df(s->buf, 1ull << s->n, s->stream));   // double2 -> hi + lo, in place
    return SV_OK;
}

// Device -> host copy of the state (stream-ordered). A double-float state
// goes through a staging buffer in chunks, each converted to double2 first.
static sv_status copy_out(sv_state *s, void *dst) {
    if (!is_df(s)) {
        CUDA_TRY(cudaMemcpyAsync(dst, s->buf, s->bytes, cudaMemcpyDeviceToHost, s->stream));
        return SV_OK;
    }
    const uint64_t N = 1ull << s->n, chunk = std::min<uint64_t>(N, kStageAmps);
    if (!s->d_stage) {
        cudaError_t e = dev_alloc(&s->d_stage, 16 * chunk, s->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s->d_stage = nullptr;
            return fail(SV_ERR_OOM, std::string("download staging: ") + cudaGetErrorString(e));
        }
    }
    for (uint64_t i = 0; i < N; i += chunk) {
        const uint64_t m = std::min(chunk, N - i);
        CUDA_TRY(launch_from_df(static_cast<char *>(s->buf) + 16 * i, s->d_stage, m, s->stream));
        CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(dst) + 16 * i, s->d_stage, 16 * m, cudaMemcpyDeviceToHost,
                                 s->stream));
    }
    return SV_OK;
}

sv_status sv_copy_state(sv_state *s, void *dst, size_t bytes) {
    if (!s || !dst) return fail(SV_ERR_ARG, "NULL argument");
    if (bytes != s->bytes) return fail(SV_ERR_ARG, "bytes must equal the state size");
    sv_status st = copy_out(s, dst);
    if (st != SV_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return SV_OK;
}

sv_status sv_download(sv_state *s, void *dst, size_t bytes) {
    if (!s || !dst) return fail(SV_ERR_ARG, "NULL argument");
    if (bytes != s->bytes) return fail(SV_ERR_ARG, "bytes must equal the state size");
    return copy_out(s, dst);
}

sv_status sv_export_c128(sv_state *s, void *dev_dst, size_t bytes) {
    if (!s || !dev_dst) return fail(SV_ERR_ARG, "NULL argument");
    if (s->prec == SV_C64) return fail(SV_ERR_ARG, "sv_export_c128 needs a complex128 state");
    if (bytes != s->bytes) return fail(SV_ERR_ARG, "bytes must equal the state size");
    if (is_df(s)) CUDA_TRY(launch_from_df(s->buf, dev_dst, 1ull << s->n, s->stream));
    else CUDA_TRY(cudaMemcpyAsync(dev_dst, s->buf, bytes, cudaMemcpyDeviceToDevice, s->stream));
    return SV_OK;
}

sv_status sv_device_ptr(sv_state *s, void **ptr, size_t *bytes) {
    if (!s) return fail(SV_ERR_ARG, "state is NULL");
    if (ptr) *ptr = s->buf;
    if (bytes) *bytes = s->bytes;
    return SV_OK;
}

static sv_status check_device_error(sv_state *s) {
    int h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, s->d_err, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (h) {
        CUDA_TRY(cudaMemsetAsync(s->d_err, 0, sizeof(int), s->stream));
        return fail(SV_ERR_TIMEOUT, "a bounded device wait of the tensor-core kernel gave up");
    }
    return SV_OK;
}

sv_status sv_sync(sv_state *s) {
    if (!s) return fail(SV_ERR_ARG, "state is NULL");
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

sv_status sv_set_tile(sv_state *s, int t) {
    if (!s) return fail(SV_ERR_ARG, "state is NULL");
    if (t != 0 && (t < part_tmin() || t > part_tmax(is_fp64(s))))
        return fail(SV_ERR_ARG, "tile_qubits out of range");
    s->tile = t;
    return SV_OK;
}

sv_status sv_plan_build(const sv_gate *gates, size_t n_gates, int n, sv_method m, int k, uint64_t seed,
                        int dfs_trials, sv_plan **out) {
    if (!out) return fail(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 36) return fail(SV_ERR_ARG, "n_qubits must be in [1, 36]");
    if (n_gates && !gates) return fail(SV_ERR_ARG, "gates is NULL");
    if (m < SV_PART_NONE || m > SV_PART_BEAM) return fail(SV_ERR_ARG, "bad method");
    std::unique_ptr<sv_plan> p(new sv_plan());
    p->n = n;
    p->method = m;
    p->k = k;
    p->gates.resize(n_gates);
    int max_arity = 0;
    for (size_t i = 0; i < n_gates; i++) {
        const sv_gate &g = gates[i];
        if (g.kind >= SV_GATE_COUNT) return fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": bad kind");
        const int want = gate_is_two_qubit(g.kind) ? 2 : 1;
        if (g.arity != want) return fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": arity does not match kind");
        GateRef &r = p->gates[i];
        r.kind = g.kind;
        r.arity = g.arity;
        r.theta = g.theta;
        for (int j = 0; j < 3; j++) r.q[j] = j < g.arity ? (int)g.q[j] : 0;
        for (int j = 0; j < g.arity; j++)
            if (g.q[j] >= (uint32_t)n) return fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": qubit out of range");
        if (g.arity == 2 && g.q[0] == g.q[1]) return fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": repeated qubit");
        max_arity = std::max(max_arity, (int)g.arity);
    }
    if (m != SV_PART_NONE) {
        if (k < 1) return fail(SV_ERR_ARG, "k must be >= 1");
        if (max_arity > k) return fail(SV_ERR_PARTITION, "a gate has more qubits than k");
        Dag dag;
        std::string err;
        if (!build_dag(p->gates, n, dag, err)) return fail(SV_ERR_ARG, err);
        if (m == SV_PART_NAT) p->pog = part_nat(dag, k);
        else if (m == SV_PART_DFS) p->pog = part_dfs(dag, k, seed, dfs_trials);
        else if (m == SV_PART_DAGP) p->pog = part_dagp(dag, k);
        else if (m == SV_PART_BEAM) p->pog = part_beam(dag, k, dfs_trials);
        else if (!part_exact(dag, k, p->pog, err)) return fail(SV_ERR_ARG, err);
        for (uint32_t x : p->pog) p->n_parts = std::max(p->n_parts, x + 1);
        std::vector<uint64_t> pm(p->n_parts, 0);
        for (size_t i = 0; i < n_gates; i++) pm[p->pog[i]] |= dag.qmask[i];
        for (uint64_t m : pm) p->max_part = std::max(p->max_part, __builtin_popcountll(m));
    } else {
        p->pog.resize(n_gates);
        for (size_t i = 0; i < n_gates; i++) p->pog[i] = (uint32_t)i;
        p->n_parts = (uint32_t)n_gates;
    }
    *out = p.release();
    return SV_OK;
}

sv_status sv_plan_build_ml(const sv_gate *gates, size_t n_gates, int n, sv_method m1, int k1, sv_method m2, int k2,
                           uint64_t seed, int dfs_trials, sv_plan **out) {
    if (!out) return fail(SV_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (m1 == SV_PART_NONE || m2 < SV_PART_NAT || m2 > SV_PART_BEAM)
        return fail(SV_ERR_ARG, "both levels need a part builder");
    if (k2 < 1 || k2 > k1) return fail(SV_ERR_ARG, "k2 must be in [1, k1]");
    sv_plan *p = nullptr;
    sv_status st = sv_plan_build(gates, n_gates, n, m1, k1, seed, dfs_trials, &p);
    if (st != SV_OK) return st;
    std::unique_ptr<sv_plan> hold(p);
    for (const GateRef &g : p->gates)
        if (g.arity > k2) return fail(SV_ERR_PARTITION, "a gate has more qubits than k2");
    std::vector<uint32_t> outer, inner;
    std::string err;
    if (!part_multilevel(p->gates, n, (int)m1, k1, (int)m2, k2, seed, dfs_trials, outer, inner, err))
        return fail(SV_ERR_ARG, err);
    if (outer != p->pog) return fail(SV_ERR_INTERNAL, "first-level partition differs from the plan's");
    p->inner = std::move(inner);
    for (uint32_t x : p->inner) p->n_inner = std::max(p->n_inner, x + 1);
    p->k2 = k2;
    *out = hold.release();
    return SV_OK;
}

sv_status sv_plan_export_inner(const sv_plan *p, uint32_t *inner, size_t n_gates, uint32_t *n_inner) {
    if (!p) return fail(SV_ERR_ARG, "plan is NULL");
    if (n_gates != p->gates.size()) return fail(SV_ERR_ARG, "n_gates does not match the plan");
    if (p->inner.empty() && n_gates) return fail(SV_ERR_ARG, "the plan has one level");
    if (inner && n_gates) std::memcpy(inner, p->inner.data(), sizeof(uint32_t) * n_gates);
    if (n_inner) *n_inner = p->n_inner;
    return SV_OK;
}

sv_status sv_plan_export(const sv_plan *p, uint32_t *pog, size_t n_gates, uint32_t *n_parts) {
    if (!p) return fail(SV_ERR_ARG, "plan is NULL");
    if (n_gates != p->gates.size()) return fail(SV_ERR_ARG, "n_gates does not match the plan");
    if (pog && n_gates) std::memcpy(pog, p->pog.data(), sizeof(uint32_t) * n_gates);
    if (n_parts) *n_parts = p->n_parts;
    return SV_OK;
}

static sv_status get_host_program(sv_plan *p, bool fp64, int t, int dense, const Program **out) {
    std::lock_guard<std::recursive_mutex> lk(p->mu);
    auto key = std::make_tuple(fp64, t, dense);
    auto it = p->host_progs.find(key);
    if (it == p->host_progs.end()) {
        std::unique_ptr<Program> prog(new Program());
        std::string err;
        const int R = (dense >> 4) ? (dense >> 4) : part_R(fp64);
        if (!compile_program(p->gates, p->n, p->pog, p->n_parts, fp64, t, R, dense & 3, *prog, err,
                             p->inner.empty() ? nullptr : &p->inner))
            return fail(SV_ERR_PARTITION, err);
        it = p->host_progs.emplace(key, std::move(prog)).first;
    }
    *out = it->second.get();
    return SV_OK;
}

// Program variant of the flags: bit 0 = tensor-core dense parts (complex64
// only), bit 1 = two of them per pass where they fit one tile, bits 4-7 =
// register bits per thread when not the precision's default.
static int dense_mode(uint32_t flags, bool fp64) {
    const bool tc = (flags & SV_FLAG_TC_DENSE) && !fp64;
    return (tc ? 1 : 0) | ((tc && (flags & SV_FLAG_TC_PAIRS)) ? 2 : 0) | (int)(((flags >> 8) & 0xFu) << 4);
}

sv_status sv_plan_stats(sv_plan *p, sv_precision prec, int t, uint32_t flags, uint32_t *passes, uint32_t *phases,
                        uint32_t *ops, uint32_t *dense) {
    if (!p) return fail(SV_ERR_ARG, "plan is NULL");
    const bool fp64 = prec != SV_C64;
    if (t == 0) t = default_tile(fp64, p->max_part);
    if (t < part_tmin() || t > part_tmax(fp64)) return fail(SV_ERR_ARG, "tile_qubits out of range");
    if (p->method == SV_PART_NONE || p->n < part_tmin() || (flags & SV_FLAG_GATEWISE)) {
        if (passes) *passes = (uint32_t)p->gates.size();
        if (phases) *phases = 0;
        if (ops) *ops = 0;
        if (dense) *dense = 0;
        return SV_OK;
    }
    const Program *prog = nullptr;
    sv_status st = get_host_program(p, fp64, t, dense_mode(flags, fp64), &prog);
    if (st != SV_OK) return st;
    if (passes) *passes = (uint32_t)prog->kind.size();
    if (phases) *phases = (uint32_t)prog->phases.size();
    if (ops) *ops = (uint32_t)prog->ops.size();
    if (dense) *dense = (uint32_t)(prog->dense.size() + prog->pairs.size());
    return SV_OK;
}

// The plan's specialised part kernels for (precision, tile, dense mode),
// compiled and loaded on first use.
static sv_status get_jit_program(sv_plan *p, sv_precision prec, int t, int dense, const Program *hp,
                                 JitProgram **out) {
    std::lock_guard<std::recursive_mutex> lk(p->mu);
    auto key = std::make_tuple((int)prec, t, dense);
    auto it = p->jit_progs.find(key);
    if (it == p->jit_progs.end()) {
        std::unique_ptr<JitProgram> jp(new JitProgram());
        std::string err;
        if (!jit_compile(*hp, *jp, err, true, prec == SV_C128DF))
            return fail(SV_ERR_CUDA, "specialised part kernels: " + err);
        it = p->jit_progs.emplace(key, std::move(jp)).first;
    }
    *out = it->second.get();
    return SV_OK;
}

sv_status sv_plan_specialise(sv_plan *p, sv_precision prec, int t, uint32_t flags, int load, double *compile_s) {
    if (!p) return fail(SV_ERR_ARG, "plan is NULL");
    const bool fp64 = prec != SV_C64;
    if (t == 0) t = default_tile(fp64, p->max_part);
    if (t < part_tmin() || t > part_tmax(fp64)) return fail(SV_ERR_ARG, "tile_qubits out of range");
    const Program *hp = nullptr;
    sv_status st = get_host_program(p, fp64, t, dense_mode(flags, fp64), &hp);
    if (st != SV_OK) return st;
    if (load) {
        JitProgram *jp = nullptr;
        st = get_jit_program(p, prec, t, dense_mode(flags, fp64), hp, &jp);
        if (st != SV_OK) return st;
        if (compile_s) *compile_s = jp->compile_s;
        return SV_OK;
    }
    JitProgram jp;
    std::string err;
    if (!jit_compile(*hp, jp, err, false, prec == SV_C128DF))
        return fail(SV_ERR_CUDA, "specialised part kernels: " + err);
    if (compile_s) *compile_s = jp.compile_s;
    return SV_OK;
}

sv_status sv_plan_source(sv_plan *p, sv_precision prec, int t, uint32_t flags, uint32_t part, char *buf, size_t cap,
                         size_t *len) {
    if (!p) return fail(SV_ERR_ARG, "plan is NULL");
    const bool fp64 = prec != SV_C64;
    if (t == 0) t = default_tile(fp64, p->max_part);
    if (t < part_tmin() || t > part_tmax(fp64)) return fail(SV_ERR_ARG, "tile_qubits out of range");
    const Program *hp = nullptr;
    sv_status st = get_host_program(p, fp64, t, dense_mode(flags, fp64), &hp);
    if (st != SV_OK) return st;
    if (part >= hp->parts.size()) return fail(SV_ERR_ARG, "part index out of range");
    const std::string src = jit_part_source(*hp, part, prec == SV_C128DF);
    if (len) *len = src.size();
    if (buf && cap) {
        const size_t m = std::min(cap - 1, src.size());
        std::memcpy(buf, src.data(), m);
        buf[m] = '\0';
    }
    return SV_OK;
}

sv_status sv_plan_flops(sv_plan *p, sv_precision prec, int t, uint32_t flags, double *alu_flops,
                        double *tensor_flops) {
    if (!p) return fail(SV_ERR_ARG, "plan is NULL");
    const bool fp64 = prec != SV_C64;
    if (t == 0) t = default_tile(fp64, p->max_part);
    if (t < part_tmin() || t > part_tmax(fp64)) return fail(SV_ERR_ARG, "tile_qubits out of range");
    double a = 0.0, b = 0.0;
    if (p->method == SV_PART_NONE || p->n < part_tmin() || (flags & SV_FLAG_GATEWISE)) {
        // one general matrix per gate: 14 flops per amplitude for a 2x2, 30 for a 4x4
        for (const GateRef &g : p->gates) a += g.arity == 1 ? 14.0 : 30.0;
    } else {
        const Program *hp = nullptr;
        sv_status st = get_host_program(p, fp64, t, dense_mode(flags, fp64), &hp);
        if (st != SV_OK) return st;
        program_flops(*hp, a, b);
    }
    const double N = std::ldexp(1.0, p->n);
    if (alu_flops) *alu_flops = a * N;
    if (tensor_flops) *tensor_flops = b * N;
    return SV_OK;
}

sv_status sv_plan_destroy(sv_plan *p) {
    if (!p) return fail(SV_ERR_ARG, "plan is NULL");
    for (auto &kv : p->jit_progs) jit_release(*kv.second);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : p->dev_progs) {   // no apply of the plan may be in flight
        cudaSetDevice(kv.second.dev);
        dev_free(kv.second.d_phases, 0);
        dev_free(kv.second.d_ops, 0);
        dev_free(kv.second.d_coefs, 0);
        dev_free(kv.second.d_aimg, 0);
        dev_free(kv.second.d_pimg, 0);
    }
    cudaSetDevice(cur);
    delete p;
    return SV_OK;
}

static void free_dev(DevProgram &d, cudaStream_t st) {
    dev_free(d.d_phases, st);
    dev_free(d.d_ops, st);
    dev_free(d.d_coefs, st);
    dev_free(d.d_aimg, st);
    dev_free(d.d_pimg, st);
}

static sv_status get_dev_program(sv_state *s, sv_plan *p, int t, int dense, const Program **hp,
                                 const DevProgram **dp) {
    std::lock_guard<std::recursive_mutex> lk(p->mu);
    const bool fp64 = is_fp64(s);
    sv_status st = get_host_program(p, fp64, t, dense, hp);
    if (st != SV_OK) return st;
    auto key = std::make_tuple(s->dev, fp64, t, dense);
    auto it = p->dev_progs.find(key);
    if (it == p->dev_progs.end()) {
        const Program &prog = **hp;
        DevProgram d;
        d.dev = s->dev;
        const size_t nph = std::max<size_t>(1, prog.phases.size()), nop = std::max<size_t>(1, prog.ops.size());
        const size_t ncf = std::max<size_t>(1, prog.coefs.size()), nim = std::max<size_t>(16, prog.a_img.size());
        const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
        cudaStream_t st = s->stream;
        cudaError_t e = dev_alloc(reinterpret_cast<void **>(&d.d_phases), sizeof(Phase) * nph, st);
        if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&d.d_ops), sizeof(Op) * nop, st);
        if (e == cudaSuccess) e = dev_alloc(&d.d_coefs, rsz * ncf, st);
        if (e == cudaSuccess) e = dev_alloc(reinterpret_cast<void **>(&d.d_aimg), nim, st);
        if (e == cudaSuccess && !prog.pair_img.empty())
            e = dev_alloc(reinterpret_cast<void **>(&d.d_pimg), prog.pair_img.size(), st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_dev(d, st);
            return fail(SV_ERR_OOM, std::string("program upload: ") + cudaGetErrorString(e));
        }
        std::vector<float> cf32;
        const void *cf = prog.coefs.data();
        if (!fp64) {
            cf32.assign(prog.coefs.begin(), prog.coefs.end());
            cf = cf32.data();
        }
        if (!prog.phases.empty())
            e = cudaMemcpyAsync(d.d_phases, prog.phases.data(), sizeof(Phase) * prog.phases.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !prog.ops.empty())
            e = cudaMemcpyAsync(d.d_ops, prog.ops.data(), sizeof(Op) * prog.ops.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !prog.coefs.empty())
            e = cudaMemcpyAsync(d.d_coefs, cf, rsz * prog.coefs.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !prog.a_img.empty())
            e = cudaMemcpyAsync(d.d_aimg, prog.a_img.data(), prog.a_img.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && !prog.pair_img.empty())
            e = cudaMemcpyAsync(d.d_pimg, prog.pair_img.data(), prog.pair_img.size(), cudaMemcpyHostToDevice, st);
        // the program is shared by every state that applies the plan, on any
        // stream: it is complete before it is published (cf32 also dies here)
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            free_dev(d, st);
            return fail(SV_ERR_CUDA, std::string("program upload: ") + cudaGetErrorString(e));
        }
        it = p->dev_progs.emplace(key, d).first;
    }
    *dp = &it->second;
    return SV_OK;
}

static sv_status apply_gatewise(sv_state *s, sv_plan *p) {
    const bool fp64 = is_fp64(s);
    std::unique_lock<std::recursive_mutex> lk(p->mu);
    if (p->mats.size() != p->gates.size()) {
        p->mats.assign(p->gates.size(), {});
        for (size_t i = 0; i < p->gates.size(); i++) {
            const GateRef &g = p->gates[i];
            if (g.arity == 1) {
                p->mats[i].resize(8);
                gate_matrix_1q(g.kind, g.theta, p->mats[i].data());
            } else {
                p->mats[i].resize(32);
                gate_matrix_2q(g.kind, g.theta, p->mats[i].data());
            }
        }
    }
    lk.unlock();   // the matrices are complete and only read from here
    for (size_t i = 0; i < p->gates.size(); i++) {
        const GateRef &g = p->gates[i];
        cudaError_t e;
        if (g.arity == 1) e = launch_gate1(fp64, s->buf, s->n, g.q[0], p->mats[i].data(), s->stream);
        else e = launch_gate2(fp64, s->buf, s->n, g.q[0], g.q[1], p->mats[i].data(), s->stream);
        if (e != cudaSuccess) return fail(SV_ERR_CUDA, std::string("gate launch: ") + cudaGetErrorString(e));
    }
    return SV_OK;
}

sv_status sv_apply_parts(sv_state *s, sv_plan *p, uint32_t flags) {
    if (!s || !p) return fail(SV_ERR_ARG, "NULL argument");
    if (p->n != s->n) return fail(SV_ERR_ARG, "plan and state qubit counts differ");
    sv_status st = SV_OK;
    if (is_df(s)) {
        if ((flags & SV_FLAG_GATEWISE) || p->method == SV_PART_NONE || s->n < part_tmin())
            return fail(SV_ERR_ARG, "a double-float state runs parts of a partitioned plan (n >= 10) only");
        flags = (flags | SV_FLAG_SPECIALISE) & ~SV_FLAG_TC_DENSE;
    }
    if ((flags & SV_FLAG_GATEWISE) || p->method == SV_PART_NONE || s->n < part_tmin()) {
        st = apply_gatewise(s, p);
    } else {
        const bool fp64 = is_fp64(s);
        const int t = s->tile ? s->tile : default_tile(fp64, p->max_part);
        const Program *hp = nullptr;
        const DevProgram *dp = nullptr;
        st = get_dev_program(s, p, t, dense_mode(flags, fp64), &hp, &dp);
        if (st != SV_OK) return st;
        JitProgram *jp = nullptr;
        if (((flags >> 8) & 0xFu) && !(flags & SV_FLAG_SPECIALISE))
            return fail(SV_ERR_ARG, "register bits other than the default need SV_FLAG_SPECIALISE");
        if ((flags & SV_FLAG_SPECIALISE) && !hp->parts.empty()) {
            st = get_jit_program(p, s->prec, t, dense_mode(flags, fp64), hp, &jp);
            if (st != SV_OK) return st;
        }
        if (!hp->dense.empty() || !hp->pairs.empty()) {
            const size_t need = hp->dense.size() + hp->pairs.size() + 1;
            if (s->dnorm_cap < need) {
                dev_free(s->d_dnorm, s->stream);
                s->d_dnorm = nullptr;
                s->dnorm_cap = 0;
                cudaError_t e = dev_alloc(reinterpret_cast<void **>(&s->d_dnorm), sizeof(double) * need, s->stream);
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    return fail(SV_ERR_OOM, std::string("norm accumulators: ") + cudaGetErrorString(e));
                }
                s->dnorm_cap = need;
            }
            CUDA_TRY(cudaMemsetAsync(s->d_dnorm, 0, sizeof(double) * need, s->stream));
        }
        uint32_t didx = 0;   // tensor-core passes of this apply, in order (norm accumulators)
        for (size_t i = 0; i < hp->kind.size(); i++) {
            const uint32_t j = hp->index[i];
            cudaError_t e;
            if (hp->kind[i] == 0 && jp)
                e = jit_launch(*jp, j, s->buf, hp->n_tiles[j], s->stream);
            else if (hp->kind[i] == 0)
                e = launch_part(fp64, hp->t, s->buf, hp->parts[j], dp->d_phases, dp->d_ops, dp->d_coefs,
                                hp->n_tiles[j], s->stream);
            else if (hp->kind[i] == 1)
                e = launch_dense6(s->buf, hp->dense[j], dp->d_aimg + (size_t)j * DENSE_A_BYTES, hp->dense_tiles[j],
                                  s->d_err, s->d_dnorm, didx++, s->stream);
            else
                e = launch_dense_pair(s->buf, hp->pairs[j], dp->d_pimg + (size_t)j * 2 * DENSE_A_BYTES,
                                      hp->pair_tiles[j], s->d_err, s->d_dnorm, didx++, s->stream);
            if (e != cudaSuccess) return fail(SV_ERR_CUDA, std::string("part launch: ") + cudaGetErrorString(e));
        }
    }
    if (st != SV_OK) return st;
    if (flags & SV_FLAG_SYNC) {
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        return check_device_error(s);
    }
    return SV_OK;
}

sv_status sv_measure_probs(sv_state *s, void *dev_out, int out_fp64, double *norm_out) {
    if (!s) return fail(SV_ERR_ARG, "state is NULL");
    double *d_norm = s->d_partials + kProbBlocks;
    CUDA_TRY(launch_probs(is_fp64(s), s->buf, s->n, dev_out, out_fp64, s->d_partials, kProbBlocks, d_norm, s->stream,
                          is_df(s)));
    if (norm_out) {
        CUDA_TRY(cudaMemcpyAsync(&s->h_norm, d_norm, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
        CUDA_TRY(cudaStreamSynchronize(s->stream));
        *norm_out = s->h_norm;
    }
    return SV_OK;
}

sv_status sv_alu_probe(int fp64, double *flops_per_s) {
    if (!flops_per_s) return fail(SV_ERR_ARG, "flops_per_s is NULL");
    CUDA_TRY(alu_probe(fp64 != 0, flops_per_s, nullptr));
    return SV_OK;
}

sv_status sv_measure_summary(sv_state *s, double *norm_out, double *p0_out, uint64_t *argmax_out,
                             double *pmax_out) {
    if (!s) return fail(SV_ERR_ARG, "state is NULL");
    double *scratch = s->d_partials + kSummaryAt, *d_out = scratch + 3 * kProbBlocks;
    CUDA_TRY(launch_summary(is_fp64(s), s->buf, s->n, scratch, kProbBlocks, d_out, s->stream, is_df(s)));
    double h[4];
    CUDA_TRY(cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (norm_out) *norm_out = h[0];
    if (p0_out) *p0_out = h[1];
    if (pmax_out) *pmax_out = h[2];
    if (argmax_out) std::memcpy(argmax_out, &h[3], sizeof(uint64_t));
    return SV_OK;
}

}  // extern "C"
