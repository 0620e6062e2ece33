"""The 33-qubit QFT workload at full size (2^33 complex64 = 64 GiB): H plus
controlled-phase ladders and final swaps (577 gates) on a seeded basis state,
checked against the closed form on sampled amplitudes (every amplitude has
modulus 2^-16.5, so the samples also pin the phases) and on the norm, for
every plan bench.py times on this workload: the tensor-core plans (one and
two dense parts per pass), the specialised gate-list plans at k = 10 and 12,
and the two-level plans (Sec. IV-B) of its multi-level section."""
import numpy as np
import pytest
import torch

import synth
from oracle import closed_form as cf
from tests.gpu_util import native

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qft33():
    _, api = native()
    free, _ = torch.cuda.mem_get_info()
    if free < (70 << 30):
        pytest.skip("needs about 70 GiB of free device memory")
    n, g, x = synth.qft_basis(33)
    st = api.State(n, "c64")
    ys = torch.from_numpy(synth.splitmix_block(33, 0, 4096).astype(np.int64) & ((1 << 33) - 1))
    ys = torch.cat([ys, torch.tensor([0, 1, (1 << 33) - 1, 1 << 32], dtype=torch.int64)])
    ref = cf.qft_basis_amplitude(n, x, ys.numpy().astype(np.uint64))
    yield api, n, g, x, st, ys.cuda(), ref
    st.close()


@pytest.mark.parametrize("method,k,tc,jit,inner", [
    ("dagp", 12, False, False, None), ("dagp", 6, True, False, None),
    ("beam", 6, True, False, None), ("beam", 6, 2, False, None),
    ("beam", 10, False, True, None), ("beam", 12, False, True, None),
    ("dagp", 10, False, True, ("dagp", 5)), ("beam", 10, False, True, ("beam", 5)),
    ("beam", 12, False, True, ("dagp", 5)), ("beam", 12, False, True, ("beam", 5)),
])
def test_qft33_sampled_closed_form(qft33, method, k, tc, jit, inner):
    api, n, g, x, st, ys, ref = qft33
    plan = api.Plan(g, n, method, k, dfs_trials=64 if (method == "beam" and k <= 6) else 16, inner=inner)
    st.set_basis(x)
    st.apply(plan, sync=True, tc=tc, jit=jit)
    got = st.amplitudes()[ys].cpu().numpy().astype(np.complex128)
    assert np.abs(got - ref).max() <= 1e-5            # the stated complex64 bound
    rel = np.abs(got - ref).max() / 2 ** -16.5          # every |a| is 2^-16.5, so pin the phases too
    assert rel <= (1e-3 if tc else 1e-4), rel
    norm = st.probs()
    assert abs(norm - 1.0) <= 1e-5
    plan.close()
