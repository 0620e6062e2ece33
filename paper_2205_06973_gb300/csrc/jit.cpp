// Part kernels specialised for one plan (host side): source generation,
// run-time compilation with NVRTC for sm_103a, loading and launch.
//
// The interpreter kernel k_part decodes every op of a part at run time
// (dispatch on the op kind and on its register bits); that decoding is most
// of its instructions. Here each gate-list part of a compiled program
// becomes its own kernel, in which the tile layout, the register phases and
// every op (with its coefficients) are compile-time constants. NVRTC is
// loaded with dlopen when first needed, so the library itself does not
// depend on it.
#include "jit.hpp"

#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <mutex>
#include <sstream>
#include <thread>

#include "jit_sources.inc"   // kJitOpsCore, kJitPrelude (generated by build.py)

namespace hisv {
namespace {

struct Nvrtc {
    bool ok = false;
    std::string why;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    decltype(&nvrtcGetErrorString) errstr = nullptr;
};

Nvrtc load_nvrtc() {
    Nvrtc n;
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    void *h = nullptr;
    for (const char *nm : names)
        if ((h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) {
        n.why = "libnvrtc.so.13 not found (dlopen)";
        return n;
    }
    n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
    n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
    n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
    n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    n.errstr = reinterpret_cast<decltype(n.errstr)>(dlsym(h, "nvrtcGetErrorString"));
    n.ok = n.create && n.compile && n.cubin_size && n.cubin && n.log_size && n.log && n.destroy && n.errstr;
    if (!n.ok) n.why = "libnvrtc lacks an expected symbol";
    return n;
}

Nvrtc &nvrtc() {
    static Nvrtc n = load_nvrtc();
    return n;
}

// Exact literal of a coefficient in the kernel's precision (hexadecimal
// floating point: the value the interpreter would read, rounded to nearest).
// Literal in one of the kernel's number formats: 0 float (v rounded to
// nearest), 1 double, 2 double-float (hi = v rounded to float, lo = the rest
// rounded to float).
std::string lit(double v, int mode) {
    char b[96];
    if (mode == 1) std::snprintf(b, sizeof(b), "(%a)", v);
    else if (mode == 2) {
        const float hi = (float)v, lo = (float)(v - (double)hi);
        std::snprintf(b, sizeof(b), "(df(%af, %af))", (double)hi, (double)lo);
    } else std::snprintf(b, sizeof(b), "(%af)", (double)(float)v);
    return b;
}

unsigned swz_host(int p, bool fp64) {
    if (!fp64) return p < 4 ? (1u << p) : ((1u << p) | (1u << (p & 3)));
    return p < 3 ? (1u << p) : ((1u << p) | (1u << (p % 3)));
}

template <typename T>
std::string table(const char *type, const char *name, const std::vector<T> &v) {
    std::ostringstream o;
    const char *suffix = sizeof(T) == 8 ? "ull" : "u";
    o << "    const " << type << " " << name << "[" << v.size() << "] = {";
    for (size_t i = 0; i < v.size(); i++)
        o << (i ? ", " : "") << "0x" << std::hex << (unsigned long long)v[i] << std::dec << suffix;
    o << "};\n";
    return o.str();
}

int min_blocks(int threads, size_t smem) {
    int by_smem = (int)((227u * 1024u) / smem);
    int by_thr = 2048 / threads;
    int m = std::min(by_smem, by_thr);
    return m < 1 ? 1 : m;
}

}  // namespace

bool jit_available(std::string *why) {
    Nvrtc &n = nvrtc();
    if (!n.ok && why) *why = n.why;
    return n.ok;
}

std::string jit_part_source(const Program &prog, size_t pi, bool df) {
    const PartLaunch &L = prog.parts[pi];
    const bool fp64 = prog.fp64;
    const int mode = df ? 2 : fp64 ? 1 : 0;
    const int t = prog.t, R = prog.R, TB = t - R, NT = 1 << TB, NRr = 1 << R;
    const size_t smem = 2 * ((size_t)(fp64 ? 16 : 8) << t);
    std::ostringstream o;
    o << "extern \"C\" __global__ void __launch_bounds__(" << NT << ", " << min_blocks(NT, smem) << ")\n"
      << "hisv_part_" << pi << "(hisv::C *__restrict__ sv, unsigned long long n_tiles) {\n"
      << "    using namespace hisv;\n"
      << "    extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      << "    C *const buf0 = reinterpret_cast<C *>(smem_raw);\n"
      << "    C *const buf1 = buf0 + " << (1 << t) << ";\n"
      << "    const int tid = threadIdx.x;\n"
      << "    const u64 OUTER = 0x" << std::hex << L.outer_mask << std::dec << "ull;\n";
    const uint32_t nph = L.n_phases;
    // per-thread parts of the addresses: the gather layout (thread bit j on
    // tile slot j), each phase's shared-memory layout and the store layout
    o << "    u64 c_thr = 0, st_thr = 0;\n    u32 s_cthr = 0";
    for (uint32_t p = 0; p < nph; p++) o << ", sp" << p << " = 0";
    o << ";\n";
    for (int j = 0; j < TB; j++) {
        o << "    if ((tid >> " << j << ") & 1) { c_thr |= 0x" << std::hex << (1ull << L.tile_q[j]) << "ull; st_thr |= 0x"
          << (1ull << L.store_thr_q[j]) << "ull; s_cthr ^= 0x" << swz_host(j, fp64) << "u;";
        for (uint32_t p = 0; p < nph; p++)
            o << " sp" << std::dec << p << " ^= 0x" << std::hex << swz_host(prog.phases[L.phase_begin + p].thr[j], fp64) << "u;";
        o << std::dec << " }\n";
    }
    std::vector<uint64_t> GO(NRr), SG(NRr);
    std::vector<uint32_t> SO(NRr);
    for (int i = 0; i < NRr; i++) {
        uint64_t g = 0, s = 0;
        uint32_t so = 0;
        for (int b = 0; b < R; b++)
            if ((i >> b) & 1) {
                g |= 1ull << L.tile_q[TB + b];
                so ^= swz_host(TB + b, fp64);
                s |= 1ull << L.store_reg_q[b];
            }
        GO[i] = g;
        SO[i] = so;
        SG[i] = s;
    }
    o << table("u64", "GO", GO) << table("u32", "SO", SO) << table("u64", "SG", SG);
    for (uint32_t p = 0; p < nph; p++) {
        const Phase &ph = prog.phases[L.phase_begin + p];
        std::vector<uint32_t> SR(NRr);
        for (int i = 0; i < NRr; i++) {
            uint32_t v = 0;
            for (int b = 0; b < R; b++)
                if ((i >> b) & 1) v ^= swz_host(ph.reg[b], fp64);
            SR[i] = v;
        }
        o << table("u32", ("SR" + std::to_string(p)).c_str(), SR);
    }
    o << "    C a[NR];\n"
      << "    u64 tile = blockIdx.x;\n"
      << "    u64 base = tile < n_tiles ? deposit64(tile, OUTER) : 0ull;\n"
      << "    if (tile < n_tiles) {\n"
      << "        const C *src = sv + (base | c_thr);\n"
      << "#pragma unroll\n"
      << "        for (int i = 0; i < NR; i++) cp_async(buf0 + (s_cthr ^ SO[i]), src + GO[i]);\n"
      << "    }\n"
      << "    cp_commit();\n"
      << "    for (u32 it = 0; tile < n_tiles; tile += gridDim.x, it++) {\n"
      << "        C *const cur = (it & 1) ? buf1 : buf0;\n"
      << "        C *const nxt = (it & 1) ? buf0 : buf1;\n"
      << "        __syncthreads();\n"
      << "        const u64 ntile = tile + gridDim.x;\n"
      << "        const u64 nbase = ntile < n_tiles ? deposit64(ntile, OUTER) : 0ull;\n"
      << "        if (ntile < n_tiles) {\n"
      << "            const C *src = sv + (nbase | c_thr);\n"
      << "#pragma unroll\n"
      << "            for (int i = 0; i < NR; i++) cp_async(nxt + (s_cthr ^ SO[i]), src + GO[i]);\n"
      << "        }\n"
      << "        cp_commit();\n"
      << "        cp_wait1();\n"
      << "        __syncthreads();\n"
      << "        Real tpr = 1, tpi = 0;\n"
      << "        (void)tpr; (void)tpi;\n";
    const std::vector<double> &cf = prog.coefs;
    auto L_ = [&](uint32_t at) { return lit(cf[at], mode); };
    auto L_lit = [&](double v) { return lit(v, mode); };
    // Per-thread phases (OP_TD / OP_TP2) multiply every amplitude a thread
    // holds by one scalar, which commutes with every op of the phase. Where a
    // phase has a merged diagonal (OP_DIAG), that scalar (and, in the last
    // phase, the part factor) is multiplied into the diagonal's coefficients
    // at run time, once per distinct coefficient, in place of a separate
    // complex multiply of every amplitude (OP_TAPPLY or the store factor).
    bool store_folded = false;
    for (uint32_t p = 0; p < nph; p++) {
        const Phase &ph = prog.phases[L.phase_begin + p];
        if (p > 0)
            o << "        __syncthreads();\n#pragma unroll\n        for (int i = 0; i < NR; i++) cur[sp" << p - 1
              << " ^ SR" << p - 1 << "[i]] = a[i];\n        __syncthreads();\n";
        o << "#pragma unroll\n        for (int i = 0; i < NR; i++) a[i] = cur[sp" << p << " ^ SR" << p << "[i]];\n";
        const bool last = p + 1 == nph;
        int first_diag = -1;
        bool tapply = false;
        for (uint32_t k = 0; k < ph.op_count; k++) {
            const uint8_t kd = prog.ops[ph.op_begin + k].kind;
            if (kd == OP_DIAG && first_diag < 0) first_diag = (int)k;
            if (kd == OP_TAPPLY) tapply = true;
        }
        const bool fold_store = last && (L.flags & PL_STORE_FACTOR) && first_diag >= 0;
        const bool fold = first_diag >= 0 && (tapply || fold_store);
        if (fold) store_folded = fold_store;
        // with folding, the per-thread phase is complete before the ops run
        std::vector<uint32_t> order;
        if (fold)
            for (uint32_t k = 0; k < ph.op_count; k++) {
                const uint8_t kd = prog.ops[ph.op_begin + k].kind;
                if (kd == OP_TD || kd == OP_TP2) order.push_back(k);
            }
        for (uint32_t k = 0; k < ph.op_count; k++) {
            const uint8_t kd = prog.ops[ph.op_begin + k].kind;
            if (fold && (kd == OP_TD || kd == OP_TP2 || kd == OP_TAPPLY)) continue;
            order.push_back(k);
        }
        for (uint32_t k : order) {
            const Op &op = prog.ops[ph.op_begin + k];
            const uint32_t c = op.coef;
            const std::string tb = "((tid >> " + std::to_string(op.tb) + ") & 1)";
            const int A = op.a, B = op.b;
            o << "        ";
            if (fold && (int)k == first_diag) {
                // coefficient q = d_q x g x (per-thread phase), g the part
                // factor in the last phase (else 1); one complex product per
                // distinct d_q x g
                double gr = 1.0, gi = 0.0;
                if (fold_store) { gr = L.gr; gi = L.gi; }
                std::vector<std::pair<double, double>> vals;
                std::vector<int> which(NRr);
                for (int q = 0; q < NRr; q++) {
                    const double dr = cf[c + 2 * q], di = cf[c + 2 * q + 1];
                    const double er = dr * gr - di * gi, ei = dr * gi + di * gr;
                    int w = -1;
                    for (size_t v = 0; v < vals.size(); v++)
                        if (vals[v].first == er && vals[v].second == ei) w = (int)v;
                    if (w < 0) { w = (int)vals.size(); vals.push_back({er, ei}); }
                    which[q] = w;
                }
                o << "{ ";
                for (size_t v = 0; v < vals.size(); v++) {
                    const double er = vals[v].first, ei = vals[v].second;
                    const std::string nm = "e" + std::to_string(v);
                    if (er == 1.0 && ei == 0.0) o << "const Real " << nm << "r = tpr, " << nm << "i = tpi; ";
                    else if (er == -1.0 && ei == 0.0) o << "const Real " << nm << "r = -tpr, " << nm << "i = -tpi; ";
                    else if (er == 0.0 && ei == 1.0) o << "const Real " << nm << "r = -tpi, " << nm << "i = tpr; ";
                    else if (er == 0.0 && ei == -1.0) o << "const Real " << nm << "r = tpi, " << nm << "i = -tpr; ";
                    else
                        o << "const Real " << nm << "r = " << L_lit(er) << " * tpr - " << L_lit(ei) << " * tpi, " << nm
                          << "i = " << L_lit(er) << " * tpi + " << L_lit(ei) << " * tpr; ";
                }
                for (int q = 0; q < NRr; q++)
                    o << "cmul_in(a[" << q << "], e" << which[q] << "r, e" << which[q] << "i); ";
                o << "tpr = 1; tpi = 0; }\n";
                continue;
            }
            switch (op.kind) {
            case OP_H:
                if (mode == 0) o << "op_h2<" << A << ">(a);";   // packed f32x2
                else o << "op_h<NR, " << A << ">(a);";
                break;
            case OP_U2:
                o << "{ const Real m[8] = {";
                for (int q = 0; q < 8; q++) o << (q ? ", " : "") << L_(c + q);
                o << "}; op_u2<NR, " << A << ">(a, m); }";
                break;
            case OP_RXS: o << "op_rxs<NR, " << A << ", " << B << ">(a, " << L_(c) << ");"; break;
            case OP_RYS:
                if (mode == 0) o << "op_rys2<" << A << ", " << B << ">(a, " << L_(c) << ");";
                else o << "op_rys<NR, " << A << ", " << B << ">(a, " << L_(c) << ");";
                break;
            case OP_U2S:
                o << "op_u2s<NR, " << A << ", " << B << ">(a";
                for (int q = 0; q < 6; q++) o << ", " << L_(c + q);
                o << ");";
                break;
            case OP_RX: o << "op_rx<NR, " << A << ">(a, " << L_(c) << ", " << L_(c + 1) << ");"; break;
            case OP_RY: o << "op_ry<NR, " << A << ">(a, " << L_(c) << ", " << L_(c + 1) << ");"; break;
            case OP_X: o << "op_x<" << A << ">(a);"; break;
            case OP_Y: o << "op_y<" << A << ">(a);"; break;
            case OP_D:
                o << "op_d<NR, " << A << ">(a, " << L_(c) << ", " << L_(c + 1) << ", " << L_(c + 2) << ", " << L_(c + 3) << ");";
                break;
            case OP_P: o << "op_p<NR, " << A << ">(a, " << L_(c) << ", " << L_(c + 1) << ");"; break;
            case OP_Z: o << "op_z<NR, " << A << ">(a);"; break;
            case OP_CX: o << "op_cx<" << A << ", " << B << ">(a);"; break;
            case OP_CP:
                if (A != B) o << "op_cp<NR, " << A << ", " << B << ">(a, " << L_(c) << ", " << L_(c + 1) << ");";
                break;
            case OP_CZ:
                if (A != B) o << "op_cz<NR, " << A << ", " << B << ">(a);";
                break;
            case OP_CXT: o << "op_cxt<" << B << ">(a, " << tb << " != 0);"; break;
            case OP_CPT:
                o << "{ const bool c_ = " << tb << " != 0; op_p<NR, " << A << ">(a, c_ ? " << L_(c) << " : (Real)1, c_ ? "
                  << L_(c + 1) << " : (Real)0); }";
                break;
            case OP_CZT:
                // a sign, not a complex product
                o << "op_sgn<" << A << ">(a, " << tb << " != 0);";
                break;
            case OP_TD:
                o << "{ const bool c_ = " << tb << " != 0; tmul(tpr, tpi, c_ ? " << L_(c + 2) << " : " << L_(c) << ", c_ ? "
                  << L_(c + 3) << " : " << L_(c + 1) << "); }";
                break;
            case OP_TP2:
                o << "{ const bool c_ = " << tb << " && ((tid >> " << B << ") & 1); tmul(tpr, tpi, c_ ? " << L_(c)
                  << " : (Real)1, c_ ? " << L_(c + 1) << " : (Real)0); }";
                break;
            case OP_DIAG:
                // entries of exactly 1, -1, i or -i are a copy, negation or
                // swap: the same values the complex product gives, cheaper
                for (int q = 0; q < NRr; q++) {
                    const double dr = cf[c + 2 * q], di = cf[c + 2 * q + 1];
                    const std::string aq = "a[" + std::to_string(q) + "]";
                    if (dr == 1.0 && di == 0.0) continue;
                    if (dr == -1.0 && di == 0.0) o << aq << ".x = -" << aq << ".x; " << aq << ".y = -" << aq << ".y; ";
                    else if (dr == 0.0 && di == 1.0) o << "{ const Real x_ = " << aq << ".x; " << aq << ".x = -" << aq << ".y; " << aq << ".y = x_; } ";
                    else if (dr == 0.0 && di == -1.0) o << "{ const Real x_ = " << aq << ".x; " << aq << ".x = " << aq << ".y; " << aq << ".y = -x_; } ";
                    else o << "cmul_in(" << aq << ", " << L_(c + 2 * q) << ", " << L_(c + 2 * q + 1) << "); ";
                }
                break;
            case OP_TAPPLY:
                o << "{\n#pragma unroll\n        for (int i = 0; i < NR; i++) cmul_in(a[i], tpr, tpi);\n        tpr = 1; tpi = 0; }";
                break;
            default: break;
            }
            o << "\n";
        }
    }
    if ((L.flags & PL_STORE_FACTOR) && !store_folded) {
        o << "        { const Real gr = " << lit(L.gr, mode) << ", gi = " << lit(L.gi, mode) << ";\n"
          << "          const Real fr = gr * tpr - gi * tpi, fi = gr * tpi + gi * tpr;\n"
          << "#pragma unroll\n          for (int i = 0; i < NR; i++) cmul_in(a[i], fr, fi); }\n";
    }
    o << "#pragma unroll\n        for (int i = 0; i < NR; i++) st_amp(sv + (base | st_thr | SG[i]), a[i]);\n"
      << "        base = nbase;\n"
      << "    }\n"
      << "    cp_wait0();\n"
      << "}\n";
    return o.str();
}

bool jit_compile(const Program &prog, JitProgram &out, std::string &err, bool load, bool df) {
    Nvrtc &n = nvrtc();
    if (!n.ok) {
        err = "run-time compiler unavailable: " + n.why;
        return false;
    }
    const auto t0 = std::chrono::steady_clock::now();
    out = JitProgram();
    out.fp64 = prog.fp64;
    out.t = prog.t;
    out.R = prog.R;
    out.threads = 1 << (prog.t - prog.R);
    out.smem = 2 * ((size_t)(prog.fp64 ? 16 : 8) << prog.t);
    const size_t P = prog.parts.size();
    out.kern.assign(P, nullptr);
    if (P == 0) return true;
    unsigned hw = std::thread::hardware_concurrency();
    const size_t nchunks = std::min<size_t>(P, std::max(1u, std::min(hw ? hw : 4u, 32u)));
    std::vector<std::vector<char>> cubins(nchunks);
    std::vector<std::string> errs(nchunks);
    const std::string defs_fp = std::string("-DHISV_FP64=") + (prog.fp64 ? "1" : "0");
    const std::string defs_df = std::string("-DHISV_DF=") + (df ? "1" : "0");
    const std::string defs_r = "-DHISV_R=" + std::to_string(prog.R);
    auto work = [&](size_t ci) {
        std::string src = "#include \"jit_prelude.cuh\"\n";
        for (size_t i = ci; i < P; i += nchunks) src += jit_part_source(prog, i, df);
        const char *hdrs[2] = {kJitOpsCore, kJitPrelude};
        const char *hnames[2] = {"ops_core.cuh", "jit_prelude.cuh"};
        nvrtcProgram pr = nullptr;
        nvrtcResult r = n.create(&pr, src.c_str(), "hisv_parts.cu", 2, hdrs, hnames);
        if (r != NVRTC_SUCCESS) {
            errs[ci] = std::string("nvrtcCreateProgram: ") + n.errstr(r);
            return;
        }
        const char *opts[] = {"--gpu-architecture=sm_103a", "--std=c++17", defs_fp.c_str(), defs_r.c_str(),
                              defs_df.c_str()};
        r = n.compile(pr, 5, opts);
        if (r != NVRTC_SUCCESS) {
            size_t ls = 0;
            n.log_size(pr, &ls);
            std::string log(ls, '\0');
            if (ls) n.log(pr, &log[0]);
            errs[ci] = std::string("nvrtcCompileProgram: ") + n.errstr(r) + "\n" + log.substr(0, 4000);
            n.destroy(&pr);
            return;
        }
        size_t cs = 0;
        n.cubin_size(pr, &cs);
        cubins[ci].resize(cs);
        n.cubin(pr, cubins[ci].data());
        n.destroy(&pr);
    };
    std::vector<std::thread> th;
    for (size_t ci = 0; ci < nchunks; ci++) th.emplace_back(work, ci);
    for (auto &x : th) x.join();
    for (size_t ci = 0; ci < nchunks; ci++)
        if (!errs[ci].empty()) {
            err = errs[ci];
            return false;
        }
    if (!load) {
        out.compile_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return true;
    }
    for (size_t ci = 0; ci < nchunks; ci++) {
        cudaLibrary_t lib = nullptr;
        cudaError_t e = cudaLibraryLoadData(&lib, cubins[ci].data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
        if (e != cudaSuccess) {
            err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e);
            jit_release(out);
            return false;
        }
        out.libs.push_back(lib);
        for (size_t i = ci; i < P; i += nchunks) {
            const std::string name = "hisv_part_" + std::to_string(i);
            e = cudaLibraryGetKernel(&out.kern[i], lib, name.c_str());
            if (e != cudaSuccess) {
                err = "cudaLibraryGetKernel(" + name + "): " + cudaGetErrorString(e);
                jit_release(out);
                return false;
            }
        }
    }
    out.compile_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return true;
}

cudaError_t jit_launch(JitProgram &jp, size_t i, void *sv, uint64_t n_tiles, cudaStream_t st) {
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!((jp.attr_devices >> dev) & 1)) {
            int nb_min = 1 << 30;
            for (cudaKernel_t k : jp.kern) {
                e = cudaKernelSetAttributeForDevice(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jp.smem, dev);
                if (e != cudaSuccess) return e;
                int nb = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, reinterpret_cast<const void *>(k), jp.threads,
                                                                  jp.smem);
                if (e != cudaSuccess) return e;
                nb_min = std::min(nb_min, nb);
            }
            e = cudaDeviceGetAttribute(&jp.sms[dev], cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            jp.resident[dev] = nb_min < 1 ? 1 : nb_min;
            jp.attr_devices |= 1ull << dev;
        }
    }
    uint64_t grid = (uint64_t)jp.sms[dev] * jp.resident[dev];
    if (grid > n_tiles) grid = n_tiles;
    if (grid < 1) grid = 1;
    unsigned long long nt = n_tiles;
    void *args[2] = {&sv, &nt};
    e = cudaLaunchKernel(reinterpret_cast<const void *>(jp.kern[i]), dim3((unsigned)grid), dim3(jp.threads), args,
                         jp.smem, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

void jit_release(JitProgram &jp) {
    for (cudaLibrary_t l : jp.libs) cudaLibraryUnload(l);
    jp.libs.clear();
    jp.kern.clear();
}

}  // namespace hisv
