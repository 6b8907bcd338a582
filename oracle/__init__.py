"""CPU oracle for the actuated PD + IPC quasi-static solve (test infrastructure).

Plain, slow, FP64 NumPy/SciPy restatement of the paper's method, used only to
check the CUDA path: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path never calls into this package.  It shares no code with the
CUDA library; both sides only consume the arrays made by the seeded input
generator.

Modules
-------
fem       elastic energy of Eq. 1 with the polar local step, PD matrix of Eq. 2
distance  point-triangle / edge-edge distances with exact gradient and Hessian
          (closed forms per closest-feature case, differentiated by a small
          second-order forward-mode AD type)
contact   constraint set, barrier of Eq. 3, PSD projection, additive CCD
solver    global step of Eq. 4 (direct solve; Schur form of Eq. 8-9; Woodbury
          form of Eq. 11) and the outer loop of Algorithm 1

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, finite differences, brute force,
library routines and algebraic identities); none is "parity unpinned".
"""
