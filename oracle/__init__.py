"""FP64 CPU oracle for the SwiG nested sampler's hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product imports, calls or links this
package; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline (and its ``--impl reference`` arm) may use it.  It shares no code with
the CUDA library: the only module both sides read is ``swig_inputs`` (seeded
random draws, grid, noise model, detector site table), which holds none of the
method's arithmetic.

Modules
-------
physics     prior transform (Table I), TaylorF2 phase/amplitude, antenna
            patterns and geocentric time delays (Sec. 3.1, Eq. 2 templates)
likelihood  noise-weighted inner product and matched-filter log-likelihood
            (Eq. 2), phase, distance and time marginalisation and the post-hoc
            draws of d_L and t_c (Sec. 3.1, App. A), heterodyned likelihood
            (Sec. 3.4)
nested      nested sampling with batch deletion (Sec. 2.2, Eq. 1) driven by a
            Slice-within-Gibbs kernel (Sec. 2.3, Eq. 3; Sec. 3.2)
pp          credible levels, KS and Fisher combination (Sec. 5.1, App. B)
mlp         forward/backward of the learned slice-proposal network
philox      Philox-4x32-10 counter-based generator (Salmon et al. 2011)

Parity pins live in ``tests/test_oracle_*.py``; every function here is pinned
against something other than itself (closed forms, textbook series, brute
force, library quadrature), except where a docstring says "parity unpinned".
"""
