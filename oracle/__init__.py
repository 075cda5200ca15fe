"""CPU oracle for the KKT hot path of Pacaud & Shin (arXiv 2403.15913).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
benchmark's CPU-baseline leg may import or run anything here; the library's
product path never does, and the CUDA path shares no code with it.

Plain, slow, obviously-correct FP64 implementations, each function citing the
passage of the paper it follows:

* ``tray``      the distillation-column model and its derivatives (Sec. VI-A)
* ``symbolic``  the pinned fill-reducing ordering, elimination tree,
                postorder, column counts and supernode partition (Sec. V-B:
                symbolic analysis done once for the fixed pattern)
* ``cholesky``  left-looking column Cholesky and triangular solves (Sec. V-B)
* ``ldlt``      dense Bunch-Kaufman LDL^T: solutions and inertia of the
                indefinite KKT matrix (Eq. inertia)
* ``kkt``       the condensed KKT system (Eq. kkt:condensed), its dense
                solution and inertia (Eq. inertia), Lifted-KKT with Richardson
                refinement (Sec. IV-A, Sec. V-B) and HyKKT with CG on the
                Schur complement (Eq. hykkt, Eq. schurcomp)
* ``ipm``       a minimal filter line-search interior-point loop (Sec. III)

Parity status of every function is listed in the module headers.
"""
