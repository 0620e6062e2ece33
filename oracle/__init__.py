"""CPU oracle of the hierarchical state-vector simulation.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package. The product library never calls it, and it shares
no code with the CUDA path: its only common input is the seeded generator
module ``synth``.

Contents
--------
* ``sv_oracle.c`` / ``sim``   - complex128 gate-by-gate simulator and a literal
  Algorithm 1 (Gather-Execute-Scatter) mode, plain C with OpenMP.
* ``partition``              - the gate DAG (Sec. IV-A), the working set L,
  the Nat / DFS / dagP part builders (Sec. IV-B), the part schedule, the
  validity checks of the acyclic partitioning problem and a brute-force
  minimum part count for tiny DAGs.
* ``closed_form``            - exact results used as pins: the QFT of a state
  (discrete Fourier transform) and the GHZ state.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
except the *quality* of dagP relative to the paper's own dagP code, which is
"parity unpinned" (the paper's code and circuits are not available); the
partitioner's validity and its agreement with brute force on tiny DAGs are
pinned.
"""
