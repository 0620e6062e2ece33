/*
 * CPU oracle for the hierarchical state-vector simulation (test
 * infrastructure only: the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it; the product library never links or calls it).
 *
 * Plain complex128 state-vector simulation, written from the paper:
 *   - state layout: 2^n amplitudes, little-endian index x = sum_q b_q 2^q
 *     (Sec. II-B, Fig. 1 caption);
 *   - a gate is a small unitary applied to the amplitudes picked out at the
 *     positions of its qubits (Sec. III-A): for a 1-qubit gate on q every
 *     pair (x, x + 2^q) with b_q = 0 is multiplied by the 2x2 matrix;
 *     a 2-qubit gate on operands (q0, q1) uses local index l = b_q0 + 2 b_q1
 *     and a 4x4 matrix;
 *   - orc_run_alg1 follows Algorithm 1 (Gather-Execute-Scatter, Sec. III-C):
 *     for each part in schedule order and each binary assignment of the
 *     qubits outside the part, gather the 2^w inner amplitudes, run the
 *     part's gates on the inner vector with remapped qubits, scatter back.
 *
 * Gate conventions (the paper defines X, Y, Z, H in Sec. II-A; the rest is
 * the standard textbook convention):
 *   RX(t) = [[c, -i s], [-i s, c]], RY(t) = [[c, -s], [s, c]],
 *   c = cos(t/2), s = sin(t/2); RZ(t) = diag(e^{-i t/2}, e^{i t/2});
 *   P(t) = diag(1, e^{i t}); S = P(pi/2); T = P(pi/4);
 *   CX(c, t) flips b_t when b_c = 1; CZ = diag(1,1,1,-1);
 *   CP(t) = diag(1,1,1,e^{i t}); SWAP exchanges the two bits.
 *
 * Every function is deliberately the plain loop; OpenMP only splits the
 * independent outer loop over amplitude groups.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double re, im; } cplx;

/* gate codes of this file (independent from any other numbering) */
enum {
    OG_H = 0, OG_X, OG_Y, OG_Z, OG_S, OG_T, OG_RX, OG_RY, OG_RZ, OG_P,
    OG_CX, OG_CZ, OG_CP, OG_SWAP, OG_COUNT
};

typedef struct {
    int32_t kind;
    int32_t nq;
    int32_t q[2];
    double theta;
} ogate;

static cplx cmk(double re, double im) { cplx z; z.re = re; z.im = im; return z; }
static cplx cmul(cplx a, cplx b) { return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static cplx cadd(cplx a, cplx b) { return cmk(a.re + b.re, a.im + b.im); }

/* 2x2 matrix of a 1-qubit gate, row-major: m[r][c] */
static int mat1(int kind, double th, cplx m[2][2]) {
    const double r2 = 1.0 / sqrt(2.0);
    double c = cos(th / 2), s = sin(th / 2);
    memset(m, 0, sizeof(cplx) * 4);
    switch (kind) {
    case OG_H: m[0][0] = cmk(r2, 0); m[0][1] = cmk(r2, 0); m[1][0] = cmk(r2, 0); m[1][1] = cmk(-r2, 0); break;
    case OG_X: m[0][1] = cmk(1, 0); m[1][0] = cmk(1, 0); break;
    case OG_Y: m[0][1] = cmk(0, -1); m[1][0] = cmk(0, 1); break;
    case OG_Z: m[0][0] = cmk(1, 0); m[1][1] = cmk(-1, 0); break;
    case OG_S: m[0][0] = cmk(1, 0); m[1][1] = cmk(0, 1); break;
    case OG_T: m[0][0] = cmk(1, 0); m[1][1] = cmk(cos(M_PI / 4), sin(M_PI / 4)); break;
    case OG_RX: m[0][0] = cmk(c, 0); m[0][1] = cmk(0, -s); m[1][0] = cmk(0, -s); m[1][1] = cmk(c, 0); break;
    case OG_RY: m[0][0] = cmk(c, 0); m[0][1] = cmk(-s, 0); m[1][0] = cmk(s, 0); m[1][1] = cmk(c, 0); break;
    case OG_RZ: m[0][0] = cmk(cos(-th / 2), sin(-th / 2)); m[1][1] = cmk(cos(th / 2), sin(th / 2)); break;
    case OG_P: m[0][0] = cmk(1, 0); m[1][1] = cmk(cos(th), sin(th)); break;
    default: return -1;
    }
    return 0;
}

/* 4x4 matrix of a 2-qubit gate on operands (q0, q1), local index l = b_q0 + 2 b_q1 */
static int mat2(int kind, double th, cplx m[4][4]) {
    memset(m, 0, sizeof(cplx) * 16);
    switch (kind) {
    case OG_CX: /* control q0, target q1: |b_q1 b_q0> = |t c>; l=1 (c=1,t=0) <-> l=3 (c=1,t=1) */
        m[0][0] = cmk(1, 0); m[2][2] = cmk(1, 0); m[1][3] = cmk(1, 0); m[3][1] = cmk(1, 0); break;
    case OG_CZ:
        m[0][0] = cmk(1, 0); m[1][1] = cmk(1, 0); m[2][2] = cmk(1, 0); m[3][3] = cmk(-1, 0); break;
    case OG_CP:
        m[0][0] = cmk(1, 0); m[1][1] = cmk(1, 0); m[2][2] = cmk(1, 0); m[3][3] = cmk(cos(th), sin(th)); break;
    case OG_SWAP: /* l=1 (b_q0=1,b_q1=0) <-> l=2 (b_q0=0,b_q1=1) */
        m[0][0] = cmk(1, 0); m[1][2] = cmk(1, 0); m[2][1] = cmk(1, 0); m[3][3] = cmk(1, 0); break;
    default: return -1;
    }
    return 0;
}

static int is_two_qubit(int kind) { return kind >= OG_CX && kind < OG_COUNT; }

/* Apply one gate to an n-qubit vector with the given (already remapped) operands. */
static int apply_gate(cplx *sv, int n, int kind, int nq, const int32_t *q, double th) {
    const int64_t N = (int64_t)1 << n;
    if (nq == 1 && !is_two_qubit(kind)) {
        cplx m[2][2];
        if (mat1(kind, th, m)) return -1;
        if (q[0] < 0 || q[0] >= n) return -2;
        const int64_t s = (int64_t)1 << q[0];
        #pragma omp parallel for schedule(static) if (N >= (1 << 16))
        for (int64_t x = 0; x < N; x++) {
            if (x & s) continue;
            cplx a0 = sv[x], a1 = sv[x + s];
            sv[x] = cadd(cmul(m[0][0], a0), cmul(m[0][1], a1));
            sv[x + s] = cadd(cmul(m[1][0], a0), cmul(m[1][1], a1));
        }
        return 0;
    }
    if (nq == 2 && is_two_qubit(kind)) {
        cplx m[4][4];
        if (mat2(kind, th, m)) return -1;
        if (q[0] < 0 || q[0] >= n || q[1] < 0 || q[1] >= n || q[0] == q[1]) return -2;
        const int64_t s0 = (int64_t)1 << q[0], s1 = (int64_t)1 << q[1];
        #pragma omp parallel for schedule(static) if (N >= (1 << 16))
        for (int64_t x = 0; x < N; x++) {
            if ((x & s0) || (x & s1)) continue;
            int64_t idx[4] = {x, x + s0, x + s1, x + s0 + s1};
            cplx a[4], b[4];
            for (int l = 0; l < 4; l++) a[l] = sv[idx[l]];
            for (int r = 0; r < 4; r++) {
                b[r] = cmk(0, 0);
                for (int c = 0; c < 4; c++) b[r] = cadd(b[r], cmul(m[r][c], a[c]));
            }
            for (int l = 0; l < 4; l++) sv[idx[l]] = b[l];
        }
        return 0;
    }
    return -1;
}

/* ---- exported API (double* = interleaved re,im, 2^n entries) ---- */

int orc_apply_gate(double *sv, int n, const ogate *g) {
    return apply_gate((cplx *)sv, n, g->kind, g->nq, g->q, g->theta);
}

/* Gate-by-gate simulation: psi <- U_G ... U_1 psi (Sec. II-B). */
int orc_run(double *sv, int n, const ogate *gates, int64_t ngates) {
    for (int64_t i = 0; i < ngates; i++) {
        int rc = apply_gate((cplx *)sv, n, gates[i].kind, gates[i].nq, gates[i].q, gates[i].theta);
        if (rc) return rc;
    }
    return 0;
}

/* Place the bits of v, lowest first, at the positions listed in pos[0..cnt). */
static int64_t deposit(int64_t v, const int *pos, int cnt) {
    int64_t x = 0;
    for (int j = 0; j < cnt; j++)
        if ((v >> j) & 1) x |= (int64_t)1 << pos[j];
    return x;
}

/*
 * Partitioned mode (Sec. III-C; Algorithm 1). A part whose gates act on the
 * qubit set S is a unitary on the 2^|S|-dimensional factor of the state.
 * Written as a matrix whose row index is the assignment of the qubits outside
 * S and whose column index is the assignment of S, the state is a stack of
 * independent 2^|S|-vectors, one per row, and the part acts on every row
 * alone. So for each part, in increasing id (the schedule): the state is
 * re-laid into that matrix, the part's gates (increasing gate index, qubits
 * renamed to column bits) are applied to each row, and the matrix is laid
 * back out. Column bit j holds the j-th smallest qubit of S (order_mode 0)
 * or the j-th largest (order_mode 1); any bijection gives the same state.
 */
int orc_run_alg1(double *svd, int n, const ogate *gates, int64_t ngates,
                 const uint32_t *part_of_gate, uint32_t n_parts, int order_mode) {
    cplx *state = (cplx *)svd;
    const int64_t N = (int64_t)1 << n;
    cplx *matrix = (cplx *)malloc(sizeof(cplx) * N);
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (ngates > 0 ? ngates : 1));
    if (!matrix || !members) { free(matrix); free(members); return -3; }
    int rc = 0;
    for (uint32_t part = 0; part < n_parts && !rc; part++) {
        int64_t count = 0;
        uint64_t used = 0;
        for (int64_t g = 0; g < ngates; g++)
            if (part_of_gate[g] == part) {
                members[count++] = g;
                for (int j = 0; j < gates[g].nq; j++) used |= (uint64_t)1 << gates[g].q[j];
            }
        if (count == 0) continue;
        int cols[64], rest[64], width = 0, others = 0, column_of[64];
        for (int q = 0; q < n; q++) {
            if ((used >> q) & 1) cols[width++] = q; else rest[others++] = q;
        }
        if (order_mode == 1)
            for (int j = 0; j < width / 2; j++) { int t = cols[j]; cols[j] = cols[width - 1 - j]; cols[width - 1 - j] = t; }
        for (int j = 0; j < width; j++) column_of[cols[j]] = j;
        const int64_t C = (int64_t)1 << width, R = (int64_t)1 << others;
        #pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < R; r++) {
            const int64_t row = deposit(r, rest, others);
            for (int64_t c = 0; c < C; c++) matrix[r * C + c] = state[row | deposit(c, cols, width)];
        }
        int err = 0;
        #pragma omp parallel for schedule(static) reduction(|:err)
        for (int64_t r = 0; r < R; r++)
            for (int64_t i = 0; i < count; i++) {
                const ogate *g = &gates[members[i]];
                int32_t q[2] = {0, 0};
                for (int j = 0; j < g->nq; j++) q[j] = column_of[g->q[j]];
                if (apply_gate(matrix + r * C, width, g->kind, g->nq, q, g->theta)) err |= 1;
            }
        if (err) { rc = -4; break; }
        #pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < R; r++) {
            const int64_t row = deposit(r, rest, others);
            for (int64_t c = 0; c < C; c++) state[row | deposit(c, cols, width)] = matrix[r * C + c];
        }
    }
    free(matrix);
    free(members);
    return rc;
}

/* |a_x|^2 and the norm sum, in double. */
double orc_probs(const double *sv, int n, double *probs) {
    const int64_t N = (int64_t)1 << n;
    double s = 0;
    for (int64_t x = 0; x < N; x++) {
        double p = sv[2 * x] * sv[2 * x] + sv[2 * x + 1] * sv[2 * x + 1];
        if (probs) probs[x] = p;
        s += p;
    }
    return s;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
