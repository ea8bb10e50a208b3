"""Plain, slow FP64 CPU oracle of the multi-patch FC-SDNN spatial operator.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline
and reference legs do. It shares no code with the CUDA library; the only
common inputs are the seeded generators in paper_2506_16076_gb300/workloads.py
(geometry and initial states, no method arithmetic) and the method data files
(FC-Gram tables, SDNN stand-in weights), which the paper itself treats as
precomputed data loaded from disc (Sec. 2.2, Sec. 5.1).

Every function follows a passage of Bruno & Leibovici, "General-domain
FC-based shock-dynamics solver I: Basic elements" (arXiv 2506.16076), cited
by section and equation label. Spectral derivatives and filters are evaluated in
extended precision (long double) and rounded once to FP64; the DFT is numpy's FFT on
long-double data, pinned against the explicit sum of its definition.

Modules:
  fc         FC-Gram continuation, derivative, filter (Sec. 2.2, Sec. 4.3)
  euler      Euler fluxes, EOS, sound speed, MWSB, proxy (Sec. 2.1, Sec. 5.1); the product
             rules of the adiabatic-wall form (Remark adiabatic)
  geometry   patches, metrics, fringes, donors, Neville interpolation (Sec. 3)
  viscosity  SDNN stand-in classification, preliminary viscosity, SB operator (Sec. 5)
  solver     semi-discrete operator L (flux form; product-rule form on adiabatic wall
             patches when Params.wall_form = 1), SSPRK(5,4) step, BCs, exchange, dt
             (Sec. 4, Alg. 1)
  riemann    exact Riemann solver for the shock-tube pin (textbook; not in the paper)
  adjoint    discrete adjoint of the stage/step with mu and dt frozen (either wall form;
             the product-rule form's pointwise Jacobian by the complex step)

Parity unpinned: the SDNN stand-in classifier (the paper's network and weights
are not published) is pinned only against its own training labels and the
physics tests, not against the paper's detector.
"""
