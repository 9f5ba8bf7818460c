"""CPU oracle for the entanglement-aware MPS/MPO two-site update (TEST INFRASTRUCTURE).

This package is test infrastructure, not part of the product.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  It shares no code with the CUDA path: it takes only its
seeded inputs from ``workloads`` and computes everything else itself, in
FP64 / complex128, with NumPy library primitives (matrix products, QR, SVD)
and no blocking, fusion or reordering beyond what the paper states.

Modules
-------
statevector    dense state vector (Eq. qstate) and pure-state fidelity (Eq. pureF)
densitymatrix  dense density matrix, Kraus channels, Wang fidelity (Eq. Wang)
superop        superoperators of channels in the vectorised-MPO convention
textbook_mps   textbook MPS / MPO with the paper's entanglement-aware
               truncation: canonical centre moved by QR (Section
               "Canonicalization"), SVD of the two-site tensor (Section
               "Truncation fidelity"), truncation fidelities (Eq. fT-pure,
               Eq. fT-mixed), running product (Eq. prod) and target schedule
               (Eq. uniform and the adaptive strategies of Fig. 1).

Parity status
-------------
Every function is pinned by the ``-m "not gpu"`` tests against closed forms,
invariants, brute force or special cases, except one statement that the
paper itself gives only as an approximation: the multi-cut relation
F(n) ~ prod f_i (Eq. prod).  That relation is parity unpinned; the tests
report the gap and check the exact single-cut identity instead.
"""
