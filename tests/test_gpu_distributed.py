"""The distributed state vector's local steps on the GPU (Sec. III-D): the
2^p ranks' slices held as separate CUDA tensors in one process, every part
and every local SWAP pass applied to each slice by the library's kernels
through the C ABI (sv_attach + sv_apply_parts, ``library_local_apply``), and
each exchange done by the chunk rule that the all-to-all implements (device
copies between the slices; one GPU, so no collective runs). The gathered
state, mapped back through the final layout, must equal the oracle's
gate-by-gate result within the stated tolerance of the precision."""
import numpy as np
import pytest
import torch

import synth
from oracle import partition as opart
from oracle import sim
from paper_2205_06973_gb300 import distributed as D
from tests.gpu_util import TOL, native

pytestmark = pytest.mark.gpu


def _circuit(n, seed):
    return synth.layered(n, 6, seed=seed, two_q=("CX", "CZ")) + synth.qft(n)[: 3 * n]


def _rand_state(n, seed):
    a = np.asarray(synth.random_amplitudes(n, seed))
    v = a[:, 0] + 1j * a[:, 1]
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n,p,k,precision,tc", [(15, 2, 13, "c64", True), (14, 3, 9, "c64", False),
                                                (13, 2, 10, "c128", False), (12, 1, 8, "c64", False)])
def test_sharded_local_steps_match_oracle(n, p, k, precision, tc):
    native()
    g = _circuit(n, 5 * n + p)
    pog = opart.partition(g, n, "dagp", k)
    parts = [[x for x in range(len(g)) if pog[x] == i] for i in range(max(pog) + 1)]
    psi = _rand_state(n, 3 * n + p)
    world, l = 1 << p, n - p
    dt = torch.complex64 if precision == "c64" else torch.complex128
    rows = [torch.from_numpy(psi[r << l:(r + 1) << l].copy()).to(dt).cuda() for r in range(world)]
    local = D.library_local_apply(precision, "dagp", 10, tc=tc)
    qsets = [sorted({q for x in ids for q in g[x][1]}) for ids in parts]
    steps, pos = D.plan_steps(qsets, n, p)
    n_exchanges = 0
    for st in steps:
        if st[0] == "swap":
            sw = [("SWAP", (a, b), 0.0) for a, b in st[1]]
            rows = [local(r, sw, l) for r in rows]
        elif st[0] == "exchange":
            n_exchanges += 1
            P = st[1]
            s = len(P)
            bits = [x - l for x in P]
            mask = sum(1 << b for b in bits)
            chunk = 1 << (l - s)
            new = [torch.empty_like(r) for r in rows]
            for r in range(world):
                v = sum(((r >> b) & 1) << j for j, b in enumerate(bits))
                for w in range(1 << s):
                    src = (r & ~mask) | D._deposit(w, bits)
                    new[r][w * chunk:(w + 1) * chunk] = rows[src][v * chunk:(v + 1) * chunk]
            rows = new
        else:
            _, i, m = st
            gl = [(g[x][0], tuple(m[q] for q in g[x][1]), g[x][2]) for x in parts[i]]
            rows = [local(r, gl, l) for r in rows]
    torch.cuda.synchronize()
    assert n_exchanges >= 1
    full = torch.cat(rows).cpu().numpy().astype(np.complex128)
    X = np.arange(1 << n)
    x = np.zeros_like(X)
    for q, pp in enumerate(pos):
        x |= ((X >> pp) & 1) << q
    out = np.empty_like(full)
    out[x] = full
    err = float(np.abs(out - sim.run(n, g, psi)).max())
    assert err <= TOL[precision], err
