"""Helpers shared by the GPU tests: run a circuit through the C ABI and
compare with the oracle."""
import numpy as np
import torch

import synth


def native():
    from paper_2205_06973_gb300 import build
    build.build()
    from paper_2205_06973_gb300 import _native, api
    return _native, api


def random_state(n, seed):
    a = synth.random_amplitudes(n, seed)
    v = a[:, 0] + 1j * a[:, 1]
    return v / np.linalg.norm(v)


def run_gpu(n, gates, method="dagp", k=8, precision="c64", tile=0, psi=None, basis=0, gatewise=False,
            seed=0, tc=False, jit=False):
    _, api = native()
    plan = api.Plan(gates, n, method if not gatewise else "none", k, seed=seed)
    st = api.State(n, precision, tile=tile)
    if psi is not None:
        dt = torch.complex64 if precision == "c64" else torch.complex128
        st.upload(torch.from_numpy(np.ascontiguousarray(psi)).to(dt).pin_memory())
    else:
        st.set_basis(basis)
    st.apply(plan, gatewise=gatewise, sync=True, tc=tc, jit=jit)
    out = st.copy_to_host().numpy().astype(np.complex128)
    st.close()
    plan.close()
    return out


def max_abs(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max())


TOL = {"c64": 1e-5, "c128": 1e-12, "c128df": 1e-12}
