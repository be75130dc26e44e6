"""Oracle: a plain, slow, single-threaded FP64 CPU restatement of the MadFlow
leading-order integrand (arXiv:2106.10279, Sec. 2 and Fig. 1).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library (no kernels, headers, tables or helpers); the
only common input is the seeded data of the top-level ``workloads`` module.

Contents, each following the passage it cites:

* ``philox``     counter-based uniforms (Philox4x64-10, Salmon et al. SC'11),
                 the random numbers the Vegas iteration draws (Sec. 2.2).
* ``pdf``        log-bicubic interpolation of x f(x, Q^2) tables (PDFFlow,
                 Sec. 1 and Fig. 1).
* ``phasespace`` the x1, x2 map, flat massless n-body phase space with
                 3n-4 numbers ("RAMBO on diet") and the massive rescaling of
                 RAMBO (Sec. 2.4), plus classic 4n-number RAMBO as a check.
* ``feynman``    tree-level Feynman diagrams with explicit Dirac matrices and
                 explicit SU(3) colour tensors; |M|^2 summed over colours and
                 helicities by brute force (Sec. 2.3).
* ``integrand``  cuts, parton luminosity, flux and unit conversion: the
                 per-event weight L(x1,x2) x sigma-hat (Fig. 1).
* ``vegas``      the adaptive grid map, accumulators, refinement and the
                 combination of iterations (VegasFlow, Sec. 2.2).

Every function is pinned by a test in ``tests/test_oracle_*.py`` against a
closed form, a library routine, an invariant or brute force.
"""
