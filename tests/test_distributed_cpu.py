"""The distributed state vector (Sec. III-D) on CPU ranks: the exchange plan's
invariants, the exchange index algebra emulated in one process, and gloo
worlds of 2, 4 and 8 ranks against the single-state oracle. The local step of
each rank (a part's gates on its slice) is the oracle here, standing in for
the library's kernels, which need a GPU; the exchanges are the real
torch.distributed all-to-alls."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import synth
from oracle import partition as opart
from oracle import sim
from paper_2205_06973_gb300 import distributed as D


def _circuit(n, seed):
    return synth.layered(n, 6, seed=seed, two_q=("CX", "CZ")) + synth.qft(n)[: 3 * n]


def _parts(gates, n, k, method="dagp"):
    pog = opart.partition(gates, n, method, k)
    P = max(pog) + 1
    return [[g for g in range(len(gates)) if pog[g] == p] for p in range(P)]


def _rand_state(n, seed):
    a = np.asarray(synth.random_amplitudes(n, seed))
    v = a[:, 0] + 1j * a[:, 1]
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("n,p,k", [(10, 1, 6), (10, 2, 7), (12, 3, 9), (9, 2, 4)])
def test_plan_invariants(n, p, k):
    """Every part runs with all its qubits local; every exchange swaps
    process positions with the top local positions; the layout stays a
    permutation of the positions."""
    g = _circuit(n, n + p)
    parts = _parts(g, n, k)
    qsets = [sorted({q for x in ids for q in g[x][1]}) for ids in parts]
    steps, pos = D.plan_steps(qsets, n, p)
    l = n - p
    cur = list(range(n))
    for st in steps:
        if st[0] == "swap":
            for a, b in st[1]:
                assert a < l and b < l
                qa, qb = cur.index(a), cur.index(b)
                cur[qa], cur[qb] = b, a
        elif st[0] == "exchange":
            P = st[1]
            assert P == sorted(P) and all(x >= l for x in P) and len(P) <= min(p, l)
            top = list(range(l - len(P), l))
            for j, pp in enumerate(P):
                qa, qb = cur.index(top[j]), cur.index(pp)
                cur[qa], cur[qb] = pp, top[j]
        else:
            _, i, m = st
            assert all(cur[q] < l for q in qsets[i])
            assert m == {q: cur[q] for q in qsets[i]}
    assert cur == pos and sorted(pos) == list(range(n))


def _emulate(n, p, gates, parts, psi):
    """The run of ShardedState on all ranks at once in one process: slices as
    rows of a matrix, the exchange done by the chunk rule the all-to-all
    implements, the local steps by the oracle."""
    world, l = 1 << p, n - p
    rows = [psi[r << l:(r + 1) << l].copy() for r in range(world)]
    qsets = [sorted({q for x in ids for q in gates[x][1]}) for ids in parts]
    steps, pos = D.plan_steps(qsets, n, p)
    for st in steps:
        if st[0] == "swap":
            sw = [("SWAP", (a, b), 0.0) for a, b in st[1]]
            rows = [sim.run(l, sw, r) for r in rows]
        elif st[0] == "exchange":
            P = st[1]
            s = len(P)
            bits = [x - l for x in P]
            mask = sum(1 << b for b in bits)
            chunk = 1 << (l - s)
            new = [np.empty_like(r) for r in rows]
            for r in range(world):
                v = sum(((r >> b) & 1) << j for j, b in enumerate(bits))
                for w in range(1 << s):
                    src = (r & ~mask) | D._deposit(w, bits)
                    new[r][w * chunk:(w + 1) * chunk] = rows[src][v * chunk:(v + 1) * chunk]
            rows = new
        else:
            _, i, m = st
            g = [(gates[x][0], tuple(m[q] for q in gates[x][1]), gates[x][2]) for x in parts[i]]
            rows = [sim.run(l, g, r) for r in rows]
    full = np.concatenate(rows)
    X = np.arange(1 << n)
    x = np.zeros_like(X)
    for q, pp in enumerate(pos):
        x |= ((X >> pp) & 1) << q
    out = np.empty_like(full)
    out[x] = full
    return out


@pytest.mark.parametrize("n,p,k,method", [(10, 1, 6, "dagp"), (10, 2, 8, "nat"), (11, 3, 8, "dfs"),
                                          (9, 2, 7, "dagp")])
def test_exchange_algebra_emulated(n, p, k, method):
    g = _circuit(n, 2 * n + p)
    parts = _parts(g, n, k, method)
    psi = _rand_state(n, n + 7 * p)
    assert np.abs(_emulate(n, p, g, parts, psi) - sim.run(n, g, psi)).max() <= 1e-12


def test_planned_exchanges_follow_the_partition():
    """Fewer, larger parts need fewer exchanges: dagP's and the beam
    builder's first-level partitions of the 28-qubit layered circuit on 8
    ranks (L_m = 25) against Nat's (the paper's argument for dagP in the
    multi-node runs)."""
    n, g = synth.layered_28q()
    p = 3
    counts = {}
    for m in ("nat", "dagp"):
        pog = opart.partition(g, n, m, n - p)
        P = max(pog) + 1
        qsets = [sorted({q for x in range(len(g)) if pog[x] == i for q in g[x][1]}) for i in range(P)]
        counts[m] = D.count_exchanges(qsets, n, p)
    assert counts["dagp"][0] <= counts["nat"][0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, n, k, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        g = _circuit(n, 3 * n + ws)
        parts = _parts(g, n, k)
        psi = _rand_state(n, 11 + ws)
        l = n - (ws.bit_length() - 1)
        local = torch.from_numpy(psi[rank << l:(rank + 1) << l].copy())

        def oracle_step(sl, gates, nl):
            return torch.from_numpy(sim.run(nl, gates, sl.numpy()))
        st = D.ShardedState(n, local, rank, ws, local_apply=oracle_step).run(g, parts)
        allv = [torch.empty_like(st.local) for _ in range(ws)]
        dist.all_gather(allv, st.local)
        if rank == 0:
            full = torch.cat(allv).numpy()
            out = np.empty_like(full)
            out[st.logical_index_map()] = full
            err = float(np.abs(out - sim.run(n, g, psi)).max())
            q.put((err, st.stats))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,n,k", [(2, 10, 7), (4, 10, 6), (8, 11, 7)])
def test_gloo_ranks_match_oracle(ws, n, k):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, n, k, q)) for r in range(ws)]
    for pr in procs:
        pr.start()
    err, stats = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert err <= 1e-12, err
    assert stats["exchanges"] >= 1 and stats["parts"] >= 1


def _dying_worker(rank, ws, port, q):
    """Rank 1 fails in its first local step (before any exchange); rank 0
    must get an error from its next all-to-all instead of waiting forever."""
    import datetime
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws, timeout=datetime.timedelta(seconds=10))
    n, k = 10, 6
    g = _circuit(n, 3 * n + ws)
    parts = _parts(g, n, k)
    psi = _rand_state(n, 11 + ws)
    l = n - 1
    local = torch.from_numpy(psi[rank << l:(rank + 1) << l].copy())

    def step(sl, gates, nl):
        if rank == 1:
            raise RuntimeError("injected failure of rank 1")
        return torch.from_numpy(sim.run(nl, gates, sl.numpy()))
    try:
        D.ShardedState(n, local, rank, ws, local_apply=step).run(g, parts)
        q.put((rank, "finished"))
    except Exception as e:   # rank 1: the injected failure; rank 0: the failed collective
        q.put((rank, type(e).__name__ + ": " + str(e)[:200]))
    # no destroy_process_group: the peer is gone


def test_rank_failure_is_reported_not_hung():
    """A rank that dies between steps (a host-side failure, no GPU involved)
    is seen by the other rank as an error of its next exchange, within the
    process group's timeout."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        if pr.is_alive():
            pr.kill()
    assert got[1].startswith("RuntimeError: injected failure"), got
    assert got[0] != "finished", got
