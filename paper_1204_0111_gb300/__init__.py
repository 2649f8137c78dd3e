"""GB300 (sm_103a) moving-PML sweeping preconditioner for 3D Helmholtz.

``paper_1204_0111_gb300.psp`` binds the C-ABI library ``libpsp.so`` built from
``csrc/``; ``paper_1204_0111_gb300.workloads`` generates seeded inputs.
Importing the package itself loads nothing.

Typical use (device arrays from torch; host numpy arrays work too)::

    import torch
    from paper_1204_0111_gb300 import psp, workloads
    w = workloads.cube_lens(100)
    P = psp.SweepingPreconditioner(torch.from_numpy(w.c).cuda(), w.h, w.omega, w.gamma,
                                   w.panel_depth, pad=w.pad, pml_C=w.pml_C, alpha=w.alpha,
                                   precision="c64")        # or "c128"
    P.tune_sweep()                                         # optional: pick the sweep schedule
    f = torch.from_numpy(w.rhs()).cuda()
    u = torch.zeros_like(f)
    info = P.solve(f, u, tol=1e-5, k=20)                   # GMRES(k), x0 = 0

``psp.SweepingPreconditionerBatch`` holds several independent problems in one handle.
"""
