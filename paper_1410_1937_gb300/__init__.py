"""GB300-native variable-coefficient Poisson solver for the cartesian-grid VOF pressure projection.

``paper_1410_1937_gb300.inputs`` builds seeded synthetic workloads (numpy only).
``paper_1410_1937_gb300.vofp`` binds the C-ABI library ``libvofp.so`` (hand-written sm_103a
kernels); importing it fails loudly when the library has not been built.
"""
