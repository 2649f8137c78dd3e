"""Plain complex128 CPU oracle of the moving-PML sweeping preconditioner.

TEST INFRASTRUCTURE ONLY. This package is a slow, deliberately simple
restatement of Poulson, Engquist, Li and Ying, "A parallel sweeping
preconditioner for heterogeneous 3D Helmholtz equations" (arXiv:1204.0111).
Only the test-suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The GPU library in
``paper_1204_0111_gb300`` shares no code with it and never calls it.

Every routine is written in the order of the paper's definitions, using
numpy / scipy primitives (sparse assembly, dense matmul, triangular solve)
as single steps, with no blocking, fusion or reordering of its own:

* ``discretize``   Eq. (1.1), Eq. (1.5), the block tridiagonal form (1.2) and the
                   PML of §1.1 (stretch profile read as documented there).
* ``panels``       panels of §1.1 / Alg. 1.4 and the PML-padded auxiliary problems H_i.
* ``symbolic``     the supernodal nested-dissection tree of §2.1 (separator-tree figure).
* ``multifrontal`` the front partition and partial LDL^T and the multifrontal
                   solve of §2.2.
* ``sweep``        Alg. 1.3 (T_i), Alg. 1.4 (setup), Alg. 1.5 (apply).
* ``gmres``        right-preconditioned restarted GMRES(k) of §2.4.
* ``naive``        Algs. 1.1 and 1.2 on dense plane blocks (tiny grids only).

Readings of points the paper leaves open are stated in each module.
Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines, dense solves, brute-force symbolic
elimination or the paper's separator-tree figure; none is "parity unpinned".
"""
