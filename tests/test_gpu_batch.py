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
