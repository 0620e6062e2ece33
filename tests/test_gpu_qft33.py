"""The 33-qubit QFT workload at full size (2^33 complex64 = 64 GiB): H plus
controlled-phase ladders and final swaps (577 gates) on a seeded basis state,
checked against the closed form on sampled amplitudes (every amplitude has
modulus 2^-16.5, so the samples also pin the phases) and on the norm."""
import numpy as np
import pytest
import torch

import synth
from oracle import closed_form as cf
from tests.gpu_util import native

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method,k,tc", [("dagp", 12, False), ("dagp", 6, True)])
def test_qft33_sampled_closed_form(method, k, tc):
    _, api = native()
    free, _ = torch.cuda.mem_get_info()
    if free < (70 << 30):
        pytest.skip("needs about 70 GiB of free device memory")
    n, g, x = synth.qft_basis(33)
    plan = api.Plan(g, n, method, k)
    st = api.State(n, "c64")
    st.set_basis(x)
    st.apply(plan, sync=True, tc=tc)
    amps = st.amplitudes()
    ys = torch.from_numpy(synth.splitmix_block(33, 0, 4096).astype(np.int64) & ((1 << 33) - 1))
    ys = torch.cat([ys, torch.tensor([0, 1, (1 << 33) - 1, 1 << 32], dtype=torch.int64)])
    got = amps[ys.cuda()].cpu().numpy().astype(np.complex128)
    ref = cf.qft_basis_amplitude(n, x, ys.numpy().astype(np.uint64))
    assert np.abs(got - ref).max() <= 1e-5            # the stated complex64 bound
    rel = np.abs(got - ref).max() / 2 ** -16.5          # every |a| is 2^-16.5, so pin the phases too
    assert rel <= (1e-3 if tc else 1e-4), rel
    norm = st.probs()
    assert abs(norm - 1.0) <= 1e-5
    st.close()
    plan.close()
