"""GB300 (sm_103a) moving-PML sweeping preconditioner for 3D Helmholtz.

``paper_1204_0111_gb300.psp`` binds the C-ABI library ``libpsp.so`` built from
``csrc/``; ``paper_1204_0111_gb300.workloads`` generates seeded inputs.
Importing the package itself loads nothing.
"""
