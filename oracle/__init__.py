"""FP64 CPU oracle of the two-grid Helmholtz method (arXiv 2509.17494).

TEST INFRASTRUCTURE ONLY.  A plain, slow, independent restatement of the
paper's method used to check the GPU library.  The library never imports it;
only tests, `__graft_entry__.smoke()` and the benchmark's CPU-baseline arm do.

Modules: fem (Q_p assembly, Section 3.1), qsfem (coarse operator, Sections
3.2-3.3), dd (Algorithm 2), twogrid (Algorithm 1), krylov (outer FGMRES),
lfa (Sections 5-6 local Fourier analysis).
"""
