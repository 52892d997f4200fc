"""FP64 CPU oracle of the qHP TD-CFIE marching-on-in-time hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct restatement of
the paper's method (Sec. II-IV) used to check the CUDA path.  Only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline / reference leg may import it; the
product package never imports it and shares no code, header, table or helper with it
(the only shared inputs are the seeded generators in synth/).

Modules: topology (edges, Lambda, Sigma), bc (barycentric refinement, BC functions),
quad.c/cquad (FP64 quadrature), assemble (retarded and static matrices), formulation
(projectors, T_k, r_n, post-processing), mot (marching and brute-force block solve),
rhs (incident-field tests), mlp (learned-guess network), farfield (far field of marched
currents and the Rayleigh limit of the PEC sphere), comparators (the standard TD-EFIE and
mixed TD-MFIE of the paper's comparisons).  The Mie series of the transient physics
check lives with the tests (tests/mie_series.py).
Parity-unpinned parts are listed in the module headers that contain them.
"""
