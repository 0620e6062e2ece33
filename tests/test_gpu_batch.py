"""GPU parity of the batched persistent launch (sv_batch_*): many small,
uneven circuits in one graph-captured kernel, each compared with the CPU
oracle (complex64 tolerance: max-abs 1e-5), and the same result alone and in
the batch."""
import numpy as np
import pytest
import torch

import synth
from oracle import sim
from tests.gpu_util import native

pytestmark = pytest.mark.gpu


def _circuits(count, start=0):
    return [synth.batch_circuit(i) for i in range(start, start + count)]


def test_batch_matches_oracle_per_circuit():
    native()
    from paper_2205_06973_gb300.batch import Batch
    circs = [c for c in _circuits(40) if c[0] <= 15][:16]
    circs.append((10, synth.qft(10)))
    circs.append((12, synth.layered(12, 6, seed=3, two_q=("CX", "CZ"))))
    b = Batch(circs, method="dagp", k=9)
    b.run(sync=True)
    probs, norms = b.probs()
    probs = probs.cpu().numpy()
    for i, (n, g) in enumerate(circs):
        ref = sim.run(n, g)
        out = b.state_host(i).numpy().astype(np.complex128)
        assert np.abs(out - ref).max() <= 1e-5, i
        p = probs[b.offsets[i]:b.offsets[i + 1]]
        assert np.abs(p - np.abs(ref) ** 2).max() <= 1e-6, i
        assert abs(norms[i] - 1.0) <= 1e-5, i
    # a second run applies every circuit again to its current state
    b.run(sync=True)
    for i, (n, g) in enumerate(circs[:3]):
        ref = sim.run(n, g, sim.run(n, g))
        out = b.state_host(i).numpy().astype(np.complex128)
        assert np.abs(out - ref).max() <= 1e-5, i
    b.close()


def test_batch_alone_equals_in_batch():
    native()
    from paper_2205_06973_gb300.batch import Batch
    circs = _circuits(24, start=100)
    big = Batch(circs, method="dagp", k=9, warps_per_cta=4, tiles_per_item=8)
    big.run(sync=True)
    for i in (0, 7, 23):
        alone = Batch([circs[i]], method="dagp", k=9)
        alone.run(sync=True)
        a = alone.state_host(0).numpy()
        m = big.state_host(i).numpy()
        assert np.abs(a - m).max() <= 1e-6, i
        alone.close()
    big.close()


@pytest.mark.parametrize("warps,chunk", [(1, 1), (2, 64), (8, 4)])
def test_batch_configurations(warps, chunk):
    native()
    from paper_2205_06973_gb300.batch import Batch
    circs = [c for c in _circuits(12, start=300)]
    b = Batch(circs, method="nat", k=8, warps_per_cta=warps, tiles_per_item=chunk)
    b.run(sync=True)
    _, norms = b.probs()
    assert np.abs(norms - 1.0).max() <= 1e-5
    for i in (0, 5):
        n, g = circs[i]
        ref = sim.run(n, g)
        assert np.abs(b.state_host(i).numpy() - ref).max() <= 1e-5
    b.reset()
    _, norms = b.probs()
    assert np.abs(norms - 1.0).max() == 0.0
    b.close()


def test_batch_bounded_wait_reports_timeout_and_recovers():
    """The failure path of the batched kernel without a GPU fault: an item
    whose dependency never completes (planted with sv_batch_hold_last_item)
    gives up its bounded wait, the run reports SV_ERR_TIMEOUT, and the same
    batch then runs correctly once the hold is lifted."""
    import time
    N, _ = native()
    from paper_2205_06973_gb300.batch import Batch
    circs = _circuits(4, start=200)
    b = Batch(circs, method="dfs", k=9)
    N.check(N.lib.sv_batch_hold_last_item(b.h, 1))
    t0 = time.perf_counter()
    with pytest.raises(N.SvError) as e:
        b.run(sync=True)
    assert e.value.status == N.SV_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    N.check(N.lib.sv_batch_hold_last_item(b.h, 0))
    b.reset()
    b.run(sync=True)
    for i, (n, g) in enumerate(circs):
        out = b.state_host(i).numpy().astype(np.complex128)
        assert np.abs(out - sim.run(n, g)).max() <= 1e-5, i
    b.close()


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dense_mix():
    """Circuits of 13..17 qubits for the tensor-core kernel and 10..12 for
    the gate-list kernel, from the batch family plus a QFT and a layered
    circuit (every gate kind of the layered generator)."""
    circs = [c for c in _circuits(80) if 13 <= c[0] <= 17][:10]
    circs += [c for c in _circuits(30, start=500) if c[0] <= 12][:4]
    circs.append((14, synth.qft(14)))
    circs.append((16, synth.layered(16, 8, seed=11)))
    return circs


def test_batch_dense_matches_oracle_per_circuit():
    """Circuits of >= 13 qubits on the batched tensor-core kernel (parts of at
    most 6 qubits as fused 64x64 unitaries, split BF16) and the rest on the
    gate-list kernel, in one graph: every final state against the oracle
    (max-abs 1e-5, relative L2 1e-4, fidelity 0.99999), unit norms, a
    second run on the current states, and reset + run again."""
    native()
    from paper_2205_06973_gb300.batch import Batch
    circs = _dense_mix()
    b = Batch(circs, method="dagp", k=9, dense_min_qubits=13)
    b.run(sync=True)
    info = b.info()
    n_dense = sum(1 for n, _ in circs if n >= 13)
    assert info["dense_circuits"] == n_dense
    assert info["dense_passes"] >= n_dense and info["dense_items"] >= info["dense_passes"]
    refs = [sim.run(n, g) for n, g in circs]
    _, norms = b.probs()
    for i, (n, g) in enumerate(circs):
        out = b.state_host(i).numpy().astype(np.complex128)
        ref = refs[i]
        assert np.abs(out - ref).max() <= 1e-5, i
        assert _rel_l2(out, ref) <= 1e-4, i
        assert abs(np.vdot(ref, out)) ** 2 >= 0.99999, i
        assert abs(norms[i] - 1.0) <= 1e-5, i
    b.run(sync=True)   # every circuit again, on its current state
    for i in (0, 5, len(circs) - 1):
        n, g = circs[i]
        ref = sim.run(n, g, refs[i])
        out = b.state_host(i).numpy().astype(np.complex128)
        assert np.abs(out - ref).max() <= 1e-5, i
    b.reset()
    b.run(sync=True)
    for i in (1, len(circs) - 2):
        out = b.state_host(i).numpy().astype(np.complex128)
        assert np.abs(out - refs[i]).max() <= 1e-5, i
    b.close()


@pytest.mark.parametrize("chunk,group", [(1, 1 << 30), (3, 5), (64, 1 << 30), (2, 1), (0, 0)])
def test_batch_dense_items_and_single_state_path(chunk, group):
    """Work items of 1, 3 (ragged) and 64 tiles, in plain wave order or in
    circuit groups of 5 or 1 tiles of state (and the defaults), give the same
    states, and those equal the single-state tensor-core path (sv_apply_parts
    with SV_FLAG_TC_DENSE) on the same plan to rounding."""
    native()
    from paper_2205_06973_gb300 import api
    from paper_2205_06973_gb300.batch import Batch
    circs = [c for c in _circuits(60, start=40) if c[0] >= 15][:4]
    circs.append((13, synth.layered(13, 10, seed=4)))
    b = Batch(circs, method="dfs", k=9, dense_min_qubits=13, dense_tiles_per_item=chunk,
              dense_group_tiles=group)
    b.run(sync=True)
    assert b.info()["dense_circuits"] == len(circs)
    for i, (n, g) in enumerate(circs):
        out = b.state_host(i).numpy()
        st = api.State(n, "c64")
        st.apply(b.plans[i], tc=True)
        one = st.copy_to_host().numpy()
        st.close()
        assert np.abs(out - one).max() <= 1e-6, i
        assert np.abs(out.astype(np.complex128) - sim.run(n, g)).max() <= 1e-5, i
    b.close()


def test_batch_dense_bounded_wait_reports_timeout_and_recovers():
    """The tensor-core batch kernel's failure path without a GPU fault: its
    last work item waits for a tile count that is never reached, the bounded
    dependency wait gives up, the converters stop together, the other roles
    drain and free the tensor memory, the run reports SV_ERR_TIMEOUT, and the
    batch runs correctly once the hold is lifted."""
    import time
    N, _ = native()
    from paper_2205_06973_gb300.batch import Batch
    circs = [c for c in _circuits(40, start=220) if c[0] >= 13][:3]
    b = Batch(circs, method="dfs", k=9, dense_min_qubits=13)
    N.check(N.lib.sv_batch_hold_last_item(b.h, 1))
    t0 = time.perf_counter()
    with pytest.raises(N.SvError) as e:
        b.run(sync=True)
    assert e.value.status == N.SV_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    N.check(N.lib.sv_batch_hold_last_item(b.h, 0))
    b.reset()
    b.run(sync=True)
    for i, (n, g) in enumerate(circs):
        out = b.state_host(i).numpy().astype(np.complex128)
        assert np.abs(out - sim.run(n, g)).max() <= 1e-5, i
    b.close()
