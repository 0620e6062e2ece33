// OpenQASM 2.0 front-end: a program text becomes the library's gate list.
//
// Supported: the OPENQASM header, include (the standard gates are built in),
// qreg (several registers are laid out one after another), creg, gate
// definitions with parameters (expanded at each use), barrier and measure
// (ignored: the simulator returns the state before measurement), register
// broadcast (h q; cx a, b; with whole registers of equal size), and
// parameter expressions with + - * / ^, unary minus, parentheses, pi and
// sin cos tan exp ln sqrt. reset, if, opaque gates and measurement in the
// middle of a circuit are rejected.
//
// Gates map onto the library's set exactly (matrices as in qelib1 /
// common simulator practice: u1(l) = p(l) = diag(1, e^{il}),
// u3(t,f,l) = [[c, -e^{il} s], [e^{if} s, e^{i(f+l)} c]]; rz is the standard
// diag(e^{-il/2}, e^{il/2}), which differs from u1 by a global phase):
//   u3(t,f,l) = p(f) ry(t) p(l) (p(l) first); u2(f,l) = u3(pi/2,f,l);
//   sdg = p(-pi/2); tdg = p(-pi/4); cu1 = cp; crz(l) = p(l/2) t, cx, p(-l/2) t, cx;
//   cu3(t,f,l) c,x = p((l+f)/2) c, p((l-f)/2) x, cx, u3(-t/2,0,-(f+l)/2) x, cx,
//   u3(t/2,f,0) x; cry(t) = cu3(t,0,0); crx(t) = cu3(t,-pi/2,pi/2);
//   ch = cu3(pi/2,0,pi); cy = sdg x, cx, s x; ccx: the 6-CX / 7-T network;
//   cswap = cx x,y, ccx c,y,x, cx x,y; rzz(t) = cx, p(t) on the second, cx.
#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "abi_internal.hpp"

namespace {

struct Tok {
    enum Kind { ID, NUM, STR, SYM, END } kind;
    std::string text;
    double num = 0;
    int line = 0;
};

struct QasmError : std::runtime_error {
    using std::runtime_error::runtime_error;
};

std::vector<Tok> tokenize(const char *s) {
    std::vector<Tok> out;
    int line = 1;
    size_t i = 0, n = std::strlen(s);
    while (i < n) {
        const char c = s[i];
        if (c == '\n') { line++; i++; continue; }
        if (std::isspace((unsigned char)c)) { i++; continue; }
        if (c == '/' && i + 1 < n && s[i + 1] == '/') {
            while (i < n && s[i] != '\n') i++;
            continue;
        }
        Tok t;
        t.line = line;
        if (std::isalpha((unsigned char)c) || c == '_') {
            size_t j = i;
            while (j < n && (std::isalnum((unsigned char)s[j]) || s[j] == '_')) j++;
            t.kind = Tok::ID;
            t.text.assign(s + i, j - i);
            i = j;
        } else if (std::isdigit((unsigned char)c) || (c == '.' && i + 1 < n && std::isdigit((unsigned char)s[i + 1]))) {
            char *end = nullptr;
            t.kind = Tok::NUM;
            t.num = std::strtod(s + i, &end);
            t.text.assign(s + i, end - (s + i));
            i = end - s;
        } else if (c == '"') {
            size_t j = i + 1;
            while (j < n && s[j] != '"') j++;
            if (j >= n) throw QasmError("line " + std::to_string(line) + ": unterminated string");
            t.kind = Tok::STR;
            t.text.assign(s + i + 1, j - i - 1);
            i = j + 1;
        } else if (c == '-' && i + 1 < n && s[i + 1] == '>') {
            t.kind = Tok::SYM;
            t.text = "->";
            i += 2;
        } else if (c == '=' && i + 1 < n && s[i + 1] == '=') {
            t.kind = Tok::SYM;
            t.text = "==";
            i += 2;
        } else if (std::strchr(";,()[]{}+-*/^", c)) {
            t.kind = Tok::SYM;
            t.text.assign(1, c);
            i++;
        } else {
            throw QasmError("line " + std::to_string(line) + ": unexpected character '" + std::string(1, c) + "'");
        }
        out.push_back(t);
    }
    Tok e;
    e.kind = Tok::END;
    e.line = line;
    out.push_back(e);
    return out;
}

struct GateDef {
    std::vector<std::string> params, args;
    size_t body_begin = 0, body_end = 0;   // token range of the body (inside the braces)
};

// A gate application inside a definition or at top level: name, parameter
// expressions (token ranges) and operands.
struct Operand {
    std::string reg;   // top level: register name; in a body: argument name
    long index = -1;   // -1: the whole register (top level only)
};

class Parser {
  public:
    explicit Parser(const char *text) : t_(tokenize(text)) {}

    void run() {
        header();
        while (peek().kind != Tok::END) statement();
    }

    int n_qubits() const { return nq_; }
    std::vector<sv_gate> gates;

  private:
    std::vector<Tok> t_;
    size_t p_ = 0;
    std::map<std::string, std::pair<int, int>> qregs_;   // name -> (offset, size)
    std::map<std::string, int> cregs_;
    std::map<std::string, GateDef> defs_;
    int nq_ = 0;
    bool measured_ = false;
    int depth_ = 0;

    const Tok &peek(size_t k = 0) const { return t_[std::min(p_ + k, t_.size() - 1)]; }
    [[noreturn]] void fail(const std::string &m) const {
        throw QasmError("line " + std::to_string(peek().line) + ": " + m);
    }
    bool is(const char *sym) const { return peek().kind == Tok::SYM && peek().text == sym; }
    void expect(const char *sym) {
        if (!is(sym)) fail(std::string("expected '") + sym + "'");
        p_++;
    }
    std::string ident() {
        if (peek().kind != Tok::ID) fail("expected an identifier");
        return t_[p_++].text;
    }
    long integer() {
        if (peek().kind != Tok::NUM) fail("expected an integer");
        const double v = t_[p_++].num;
        if (v < 0 || v != std::floor(v) || v > 1e9) fail("expected a non-negative integer");
        return (long)v;
    }

    void header() {
        if (peek().kind == Tok::ID && peek().text == "OPENQASM") {
            p_++;
            if (peek().kind != Tok::NUM) fail("expected a version number");
            const double v = t_[p_++].num;
            if (v < 2.0 || v >= 3.0) fail("only OpenQASM 2.x is supported");
            expect(";");
        }
    }

    // ---------------------------------------------------------------- exprs
    double expr(const std::map<std::string, double> &env) {
        double v = term(env);
        while (is("+") || is("-")) {
            const bool plus = is("+");
            p_++;
            const double r = term(env);
            v = plus ? v + r : v - r;
        }
        return v;
    }
    double term(const std::map<std::string, double> &env) {
        double v = unary(env);
        while (is("*") || is("/")) {
            const bool mul = is("*");
            p_++;
            const double r = unary(env);
            v = mul ? v * r : v / r;
        }
        return v;
    }
    // unary minus binds looser than ^ (-a^b = -(a^b)); ^ is right-associative
    double unary(const std::map<std::string, double> &env) {
        if (is("-")) {
            p_++;
            return -unary(env);
        }
        if (is("+")) {
            p_++;
            return unary(env);
        }
        return power(env);
    }
    double power(const std::map<std::string, double> &env) {
        const double b = atom(env);
        if (is("^")) {
            p_++;
            return std::pow(b, unary(env));
        }
        return b;
    }
    double atom(const std::map<std::string, double> &env) {
        if (peek().kind == Tok::NUM) return t_[p_++].num;
        if (is("(")) {
            p_++;
            const double v = expr(env);
            expect(")");
            return v;
        }
        const std::string id = ident();
        if (id == "pi") return M_PI;
        static const std::map<std::string, double (*)(double)> fn = {
            {"sin", [](double x) { return std::sin(x); }}, {"cos", [](double x) { return std::cos(x); }},
            {"tan", [](double x) { return std::tan(x); }}, {"exp", [](double x) { return std::exp(x); }},
            {"ln", [](double x) { return std::log(x); }},  {"sqrt", [](double x) { return std::sqrt(x); }}};
        auto f = fn.find(id);
        if (f != fn.end()) {
            expect("(");
            const double v = expr(env);
            expect(")");
            return f->second(v);
        }
        auto e = env.find(id);
        if (e == env.end()) fail("unknown parameter '" + id + "'");
        return e->second;
    }

    // ----------------------------------------------------------- statements
    void statement() {
        const Tok &t = peek();
        if (t.kind != Tok::ID) fail("expected a statement");
        const std::string kw = t.text;
        if (kw == "include") {
            p_++;
            if (peek().kind != Tok::STR) fail("expected a file name");
            p_++;
            expect(";");   // the standard gates are built in
        } else if (kw == "qreg" || kw == "creg") {
            p_++;
            const std::string name = ident();
            expect("[");
            const long sz = integer();
            expect("]");
            expect(";");
            if (sz < 1) fail("empty register");
            if (qregs_.count(name) || cregs_.count(name)) fail("register '" + name + "' declared twice");
            if (kw == "qreg") {
                qregs_[name] = {nq_, (int)sz};
                nq_ += (int)sz;
                if (nq_ > 36) fail("more than 36 qubits");
            } else {
                cregs_[name] = (int)sz;
            }
        } else if (kw == "gate") {
            p_++;
            define();
        } else if (kw == "opaque") {
            fail("opaque gates have no definition to simulate");
        } else if (kw == "barrier") {
            while (!is(";")) {
                if (peek().kind == Tok::END) fail("expected ';'");
                p_++;
            }
            p_++;
        } else if (kw == "measure") {
            while (!is(";")) {
                if (peek().kind == Tok::END) fail("expected ';'");
                p_++;
            }
            p_++;
            measured_ = true;
        } else if (kw == "reset") {
            fail("reset is not unitary");
        } else if (kw == "if") {
            fail("classically controlled gates are not supported");
        } else {
            top_level_gate();
        }
    }

    void define() {
        GateDef d;
        const std::string name = ident();
        if (is("(")) {
            p_++;
            while (!is(")")) {
                d.params.push_back(ident());
                if (is(",")) p_++;
                else if (!is(")")) fail("expected ',' or ')'");
            }
            p_++;
        }
        while (!is("{")) {
            d.args.push_back(ident());
            if (is(",")) p_++;
            else if (!is("{")) fail("expected ',' or '{'");
        }
        p_++;
        d.body_begin = p_;
        int level = 1;
        while (level > 0) {
            if (peek().kind == Tok::END) fail("unterminated gate body");
            if (is("{")) level++;
            if (is("}")) level--;
            p_++;
        }
        d.body_end = p_ - 1;
        if (d.args.empty()) fail("gate '" + name + "' has no qubit arguments");
        defs_[name] = d;
    }

    // name(params) operands ;  at top level: operands are reg or reg[i]
    void top_level_gate() {
        const std::string name = ident();
        std::vector<double> params;
        const std::map<std::string, double> none;
        if (is("(")) {
            p_++;
            while (!is(")")) {
                params.push_back(expr(none));
                if (is(",")) p_++;
                else if (!is(")")) fail("expected ',' or ')'");
            }
            p_++;
        }
        std::vector<Operand> ops;
        while (!is(";")) {
            Operand o;
            o.reg = ident();
            if (!qregs_.count(o.reg)) fail("unknown quantum register '" + o.reg + "'");
            if (is("[")) {
                p_++;
                o.index = integer();
                expect("]");
                if (o.index >= qregs_[o.reg].second) fail("index out of range for '" + o.reg + "'");
            }
            ops.push_back(o);
            if (is(",")) p_++;
            else if (!is(";")) fail("expected ',' or ';'");
        }
        p_++;
        if (measured_) fail("gates after a measurement are not supported");
        // broadcast over whole registers
        int width = 1;
        for (const Operand &o : ops)
            if (o.index < 0) {
                const int sz = qregs_[o.reg].second;
                if (width != 1 && sz != width) fail("registers of different sizes in one gate");
                width = sz;
            }
        for (int k = 0; k < width; k++) {
            std::vector<int> qs;
            for (const Operand &o : ops) qs.push_back(qregs_[o.reg].first + (int)(o.index < 0 ? k : o.index));
            apply(name, params, qs);
        }
    }

    void emit(int kind, std::initializer_list<int> qs, double theta = 0.0) {
        sv_gate g;
        std::memset(&g, 0, sizeof(g));
        g.kind = (uint16_t)kind;
        g.arity = (uint16_t)qs.size();
        int j = 0;
        for (int q : qs) g.q[j++] = (uint32_t)q;
        g.theta = theta;
        gates.push_back(g);
    }
    void u3(double t, double f, double l, int q) {
        emit(SV_GATE_P, {q}, l);
        emit(SV_GATE_RY, {q}, t);
        emit(SV_GATE_P, {q}, f);
    }
    void cu3(double t, double f, double l, int c, int x) {
        emit(SV_GATE_P, {c}, (l + f) / 2);
        emit(SV_GATE_P, {x}, (l - f) / 2);
        emit(SV_GATE_CX, {c, x});
        u3(-t / 2, 0, -(f + l) / 2, x);
        emit(SV_GATE_CX, {c, x});
        u3(t / 2, f, 0, x);
    }
    void ccx(int a, int b, int c) {
        emit(SV_GATE_H, {c});
        emit(SV_GATE_CX, {b, c});
        emit(SV_GATE_P, {c}, -M_PI / 4);
        emit(SV_GATE_CX, {a, c});
        emit(SV_GATE_T, {c});
        emit(SV_GATE_CX, {b, c});
        emit(SV_GATE_P, {c}, -M_PI / 4);
        emit(SV_GATE_CX, {a, c});
        emit(SV_GATE_T, {b});
        emit(SV_GATE_T, {c});
        emit(SV_GATE_H, {c});
        emit(SV_GATE_CX, {a, b});
        emit(SV_GATE_T, {a});
        emit(SV_GATE_P, {b}, -M_PI / 4);
        emit(SV_GATE_CX, {a, b});
    }

    void apply(const std::string &name, const std::vector<double> &ps, const std::vector<int> &qs) {
        auto need = [&](size_t np, size_t nq) {
            if (ps.size() != np) fail("gate '" + name + "' takes " + std::to_string(np) + " parameters");
            if (qs.size() != nq) fail("gate '" + name + "' takes " + std::to_string(nq) + " qubits");
            for (size_t i = 0; i < qs.size(); i++)
                for (size_t j = i + 1; j < qs.size(); j++)
                    if (qs[i] == qs[j]) fail("gate '" + name + "' repeats a qubit");
        };
        static const std::map<std::string, int> simple1 = {
            {"x", SV_GATE_X}, {"y", SV_GATE_Y}, {"z", SV_GATE_Z}, {"h", SV_GATE_H}, {"s", SV_GATE_S}, {"t", SV_GATE_T}};
        static const std::map<std::string, int> rot1 = {
            {"rx", SV_GATE_RX}, {"ry", SV_GATE_RY}, {"rz", SV_GATE_RZ}, {"p", SV_GATE_P}, {"u1", SV_GATE_P},
            {"phase", SV_GATE_P}};
        auto user = defs_.find(name);
        if (user != defs_.end()) {
            expand(user->second, name, ps, qs);
            return;
        }
        if (simple1.count(name)) { need(0, 1); emit(simple1.at(name), {qs[0]}); }
        else if (rot1.count(name)) { need(1, 1); emit(rot1.at(name), {qs[0]}, ps[0]); }
        else if (name == "id" || name == "u0") { need(name == "u0" ? 1 : 0, 1); }
        else if (name == "sdg") { need(0, 1); emit(SV_GATE_P, {qs[0]}, -M_PI / 2); }
        else if (name == "tdg") { need(0, 1); emit(SV_GATE_P, {qs[0]}, -M_PI / 4); }
        else if (name == "u2") { need(2, 1); u3(M_PI / 2, ps[0], ps[1], qs[0]); }
        else if (name == "u3" || name == "u" || name == "U") { need(3, 1); u3(ps[0], ps[1], ps[2], qs[0]); }
        else if (name == "cx" || name == "CX" || name == "cnot") { need(0, 2); emit(SV_GATE_CX, {qs[0], qs[1]}); }
        else if (name == "cz") { need(0, 2); emit(SV_GATE_CZ, {qs[0], qs[1]}); }
        else if (name == "cp" || name == "cu1" || name == "cphase") { need(1, 2); emit(SV_GATE_CP, {qs[0], qs[1]}, ps[0]); }
        else if (name == "swap") { need(0, 2); emit(SV_GATE_SWAP, {qs[0], qs[1]}); }
        else if (name == "cy") {
            need(0, 2);
            emit(SV_GATE_P, {qs[1]}, -M_PI / 2);
            emit(SV_GATE_CX, {qs[0], qs[1]});
            emit(SV_GATE_S, {qs[1]});
        } else if (name == "crz") {
            need(1, 2);
            emit(SV_GATE_P, {qs[1]}, ps[0] / 2);
            emit(SV_GATE_CX, {qs[0], qs[1]});
            emit(SV_GATE_P, {qs[1]}, -ps[0] / 2);
            emit(SV_GATE_CX, {qs[0], qs[1]});
        } else if (name == "cu3" || name == "cu") {
            if (name == "cu" && ps.size() == 4) {   // cu(t,f,l,g): cu3 with a phase g on the control
                need(4, 2);
                emit(SV_GATE_P, {qs[0]}, ps[3]);
                cu3(ps[0], ps[1], ps[2], qs[0], qs[1]);
            } else {
                need(3, 2);
                cu3(ps[0], ps[1], ps[2], qs[0], qs[1]);
            }
        } else if (name == "cry") { need(1, 2); cu3(ps[0], 0, 0, qs[0], qs[1]); }
        else if (name == "crx") { need(1, 2); cu3(ps[0], -M_PI / 2, M_PI / 2, qs[0], qs[1]); }
        else if (name == "ch") { need(0, 2); cu3(M_PI / 2, 0, M_PI, qs[0], qs[1]); }
        else if (name == "rzz") {
            need(1, 2);
            emit(SV_GATE_CX, {qs[0], qs[1]});
            emit(SV_GATE_P, {qs[1]}, ps[0]);
            emit(SV_GATE_CX, {qs[0], qs[1]});
        } else if (name == "ccx" || name == "toffoli") { need(0, 3); ccx(qs[0], qs[1], qs[2]); }
        else if (name == "cswap" || name == "fredkin") {
            need(0, 3);
            emit(SV_GATE_CX, {qs[2], qs[1]});
            ccx(qs[0], qs[1], qs[2]);
            emit(SV_GATE_CX, {qs[2], qs[1]});
        } else {
            fail("unknown gate '" + name + "'");
        }
    }

    void expand(const GateDef &d, const std::string &name, const std::vector<double> &ps, const std::vector<int> &qs) {
        if (ps.size() != d.params.size()) fail("gate '" + name + "' takes " + std::to_string(d.params.size()) + " parameters");
        if (qs.size() != d.args.size()) fail("gate '" + name + "' takes " + std::to_string(d.args.size()) + " qubits");
        if (++depth_ > 64) fail("gate definitions nest too deeply");
        std::map<std::string, double> env;
        for (size_t i = 0; i < ps.size(); i++) env[d.params[i]] = ps[i];
        std::map<std::string, int> arg;
        for (size_t i = 0; i < qs.size(); i++) arg[d.args[i]] = qs[i];
        const size_t save = p_;
        p_ = d.body_begin;
        while (p_ < d.body_end) {
            const std::string g = ident();
            if (g == "barrier") {
                while (!is(";")) p_++;
                p_++;
                continue;
            }
            std::vector<double> sub;
            if (is("(")) {
                p_++;
                while (!is(")")) {
                    sub.push_back(expr(env));
                    if (is(",")) p_++;
                    else if (!is(")")) fail("expected ',' or ')'");
                }
                p_++;
            }
            std::vector<int> sq;
            while (!is(";")) {
                const std::string a = ident();
                auto it = arg.find(a);
                if (it == arg.end()) fail("unknown argument '" + a + "' in gate '" + name + "'");
                sq.push_back(it->second);
                if (is(",")) p_++;
                else if (!is(";")) fail("expected ',' or ';'");
            }
            p_++;
            apply(g, sub, sq);
        }
        p_ = save;
        depth_--;
    }
};

sv_status qfail(sv_status st, const std::string &msg) {
    hisv::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" {

sv_status sv_qasm_parse(const char *text, sv_gate **out_gates, size_t *out_n_gates, int *out_n_qubits) {
    if (!text || !out_gates || !out_n_gates || !out_n_qubits) return qfail(SV_ERR_ARG, "NULL argument");
    *out_gates = nullptr;
    *out_n_gates = 0;
    *out_n_qubits = 0;
    try {
        Parser p(text);
        p.run();
        if (p.n_qubits() < 1) return qfail(SV_ERR_ARG, "no quantum register");
        sv_gate *g = static_cast<sv_gate *>(std::malloc(sizeof(sv_gate) * std::max<size_t>(1, p.gates.size())));
        if (!g) return qfail(SV_ERR_OOM, "gate array");
        if (!p.gates.empty()) std::memcpy(g, p.gates.data(), sizeof(sv_gate) * p.gates.size());
        *out_gates = g;
        *out_n_gates = p.gates.size();
        *out_n_qubits = p.n_qubits();
        return SV_OK;
    } catch (const QasmError &e) {
        return qfail(SV_ERR_ARG, std::string("qasm: ") + e.what());
    } catch (const std::exception &e) {
        return qfail(SV_ERR_INTERNAL, std::string("qasm: ") + e.what());
    }
}

void sv_free_gates(sv_gate *gates) { std::free(gates); }

}  // extern "C"
