"""CPU oracle for locally entanglement-optimal MPS trajectories (arXiv 2508.05745).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the method in numpy/scipy (and, for the MPS trajectory, in C++17), written to
be checked against the paper by eye.
Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The GPU library never
calls it and shares no code with it; the only common input is the seeded
problem description produced by ``paper_2508_05745_gb300.inputs``.

Modules:
  philox        Philox4x64-10 counter-based generator (Salmon et al., SC'11).
  unravel       Hill-Wootters entanglement of formation and the optimal
                unraveling of a single-qubit channel (Sec. IV.B, App. F).
  trajectories  dense state-vector trajectories, exact density-matrix evolution
                and MPS trajectories with truncation (Sec. IV.A, Alg. 1,
                Thm. 1 / App. B error estimator).
  adjoint       expected-entropy cost of a remixed Kraus set and its FP64
                finite-difference gradient (the differentiation workload).
  cpp           ctypes binding of mps_oracle.cpp: the MPS trajectory restated in
                plain C++17 FP64 (own Jacobi eigensolver and SVD, Householder
                QR), OpenMP over trajectories; the timed CPU baseline.

Every function is pinned by tests in ``tests/test_oracle_*.py`` against closed
forms, invariants, brute force or independent library routines.  Functions
marked "parity unpinned" in their docstring have no such pin.
"""
