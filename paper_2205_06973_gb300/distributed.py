"""State vector distributed over ranks (Sec. III-D, multi-node design).

An n-qubit state is split over 2^p ranks: p *process* qubits address the
rank and l = n - p *local* qubits address the amplitude inside the rank's
slice of 2^l amplitudes. A part may only run where all of its qubits are
local; before a part that needs a process qubit, the ranks exchange data so
that the needed qubits become local and as many unneeded local qubits
become process qubits (one all-to-all; the paper's "gather the states
residing in the remote ranks to form new local states"). The multi-level
partition of Sec. IV-B supplies the parts: the first level under L_m = l
decides where the exchanges happen, and each first-level part's
second-level parts run on every rank's slice as ordinary part passes.

Layout. ``pos[q]`` is the physical bit position of logical qubit q:
positions 0..l-1 index the local slice, positions l..n-1 the rank (position
l + j is bit j of the rank). An exchange swaps s process positions P with
the top s local positions (l - s .. l - 1): with those local bits on top,
the slice is 2^s contiguous chunks, chunk u goes to the rank whose bits at P
equal u, and the chunks received come back in rank order, so the exchange
is one all_to_all_single with no packing. Unneeded qubits are first moved
to the top local positions by a local pass of SWAP gates. Which local
qubits leave is decided by their next use (the one used farthest ahead
leaves first).

The data plane is torch.distributed (NCCL on GPUs: all_to_all_single of
device tensors; gloo on CPU tensors); every local step (part passes, the
local SWAP pass) goes through ``local_apply(state_slice, gates, n_local)``,
which by default runs the library's kernels (sv_apply_parts) on the slice.
Not measured on hardware: every run in this build has one GPU.
"""
from __future__ import annotations

import math

INF = float("inf")


def _deposit(v, positions):
    out = 0
    for j, p in enumerate(positions):
        if (v >> j) & 1:
            out |= 1 << p
    return out


def plan_steps(part_qubits, n, p):
    """Exchange plan for parts (in execution order) with the given qubit
    sets on 2^p ranks. Returns (steps, pos): steps are ("swap", [(a, b)...])
    local SWAPs of physical positions, ("exchange", P) the all-to-all that
    swaps process positions P (ascending) with the top len(P) local
    positions, and ("part", i, {logical: physical}) a part run on the slices;
    pos is the final layout."""
    l = n - p
    pos = list(range(n))
    who = list(range(n))
    steps = []
    for i, S in enumerate(part_qubits):
        S = set(S)
        if len(S) > l:
            raise ValueError(f"part {i} has {len(S)} qubits > {l} local qubits")
        need = sorted((q for q in S if pos[q] >= l), key=lambda q: pos[q])
        if need:
            s = len(need)

            def next_use(q):
                for j in range(i + 1, len(part_qubits)):
                    if q in part_qubits[j]:
                        return j
                return INF
            cand = [q for q in range(n) if pos[q] < l and q not in S]
            # farthest next use leaves first; ties: the higher position (fewer local moves)
            cand.sort(key=lambda q: (-next_use(q), -pos[q]))
            evict = cand[:s]
            top = list(range(l - s, l))
            swaps = []
            movers = [q for q in evict if pos[q] < l - s]
            for t in top:
                if who[t] in evict:
                    continue
                e = movers.pop()
                a, b = pos[e], t
                swaps.append((a, b))
                qa, qb = who[a], who[b]
                who[a], who[b] = qb, qa
                pos[qa], pos[qb] = b, a
            if swaps:
                steps.append(("swap", swaps))
            P = [pos[q] for q in need]
            steps.append(("exchange", P))
            for j, pp in enumerate(P):
                t = l - s + j
                qa, qb = who[t], who[pp]
                who[t], who[pp] = qb, qa
                pos[qa], pos[qb] = pp, t
        steps.append(("part", i, {q: pos[q] for q in S}))
    return steps, pos


def count_exchanges(part_qubits, n, p):
    steps, _ = plan_steps(part_qubits, n, p)
    return sum(1 for s in steps if s[0] == "exchange"), sum(len(s[1]) for s in steps if s[0] == "exchange")


def exchange(local, P, l, rank, world, group=None):
    """The all-to-all of one exchange step: this rank's slice ``local`` (a 1-D
    tensor of 2^l amplitudes whose top len(P) local bits are the qubits that
    leave) -> the new slice. P: the process positions (>= l) swapped with
    the top local positions, in the same order."""
    import torch
    import torch.distributed as dist
    s = len(P)
    mask_bits = [pp - l for pp in P]
    mask = sum(1 << b for b in mask_bits)
    chunk = local.numel() >> s
    in_splits = [0] * world
    out_splits = [0] * world
    for u in range(1 << s):
        dst = (rank & ~mask) | _deposit(u, mask_bits)
        in_splits[dst] = chunk
        out_splits[dst] = chunk
    out = torch.empty_like(local)
    dist.all_to_all_single(out, local, output_split_sizes=out_splits, input_split_sizes=in_splits, group=group)
    return out


def library_local_apply(precision="c64", method="dagp", k=10, tc=True):
    """The default local step: the library's part kernels on the slice (a
    CUDA tensor of complex amplitudes), through the C ABI."""
    from . import api

    def apply(local, gates, n_local):
        import torch
        if not local.is_cuda:
            raise RuntimeError("the library's local step needs the slice on a CUDA device")
        plan = api.Plan(gates, n_local, method, min(k, n_local))
        st = api.State.over(local, n_local, precision)
        st.apply(plan, tc=tc and precision == "c64")
        st.sync()
        st.close()
        plan.close()
        return local
    return apply


class ShardedState:
    """One rank's slice of a state distributed over 2^p ranks."""

    def __init__(self, n, local, rank, world, group=None, local_apply=None):
        p = int(round(math.log2(world)))
        if 1 << p != world:
            raise ValueError("the number of ranks must be a power of two (Sec. III-D)")
        self.n, self.p, self.l = n, p, n - p
        if local.numel() != 1 << self.l:
            raise ValueError("the slice must hold 2^(n - p) amplitudes")
        self.local = local
        self.rank, self.world, self.group = rank, world, group
        self.pos = list(range(n))
        self.apply_local = local_apply if local_apply is not None else library_local_apply()
        self.stats = {"exchanges": 0, "exchanged_qubits": 0, "local_swap_passes": 0, "parts": 0,
                      "bytes_sent": 0}

    def run(self, gates, parts):
        """Apply the circuit: parts = the gate ids of each part in execution
        order (a first-level partition under L_m = l, or any finer one)."""
        qsets = [sorted({q for g in ids for q in gates[g][1]}) for ids in parts]
        steps, final = plan_steps(qsets, self.n, self.p)
        for st in steps:
            if st[0] == "swap":
                sw = [("SWAP", (a, b), 0.0) for a, b in st[1]]
                self.local = self.apply_local(self.local, sw, self.l)
                self.stats["local_swap_passes"] += 1
            elif st[0] == "exchange":
                self.local = exchange(self.local, st[1], self.l, self.rank, self.world, self.group)
                self.stats["exchanges"] += 1
                self.stats["exchanged_qubits"] += len(st[1])
                s = len(st[1])
                self.stats["bytes_sent"] += (self.local.numel() - (self.local.numel() >> s)) * \
                    self.local.element_size()
            else:
                _, i, m = st
                g = [(gates[x][0], tuple(m[q] for q in gates[x][1]), gates[x][2]) for x in parts[i]]
                self.local = self.apply_local(self.local, g, self.l)
                self.stats["parts"] += 1
        self.pos = final
        return self

    def logical_index_map(self):
        """For every (rank, local index) in rank-major order, the logical
        basis index x it holds under the current layout (numpy int64)."""
        import numpy as np
        X = np.arange(1 << self.n, dtype=np.int64)
        x = np.zeros_like(X)
        for q, pp in enumerate(self.pos):
            x |= ((X >> pp) & 1) << q
        return x
