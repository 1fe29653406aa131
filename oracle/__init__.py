"""Plain, slow FP64 CPU oracle for the transformer density-operator method.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg (and its reference arm) may import or run anything in this package. The product path
(paper_2502_20723_gb300) never imports it, and this package imports nothing from the
product except the seeded input generators in paper_2502_20723_gb300.synth.

Modules:
  lindblad     dense and row-wise vectorised Lindbladian (Eq. VecLin), exact steady state
  transformer  the ansatz log rho (appendix "Transformer Density Operator Architecture")
  estimators   cost (Eq. lossnetk), local estimator, gradient, log-derivatives, SR
  philox       Philox4x32-10 counter RNG (Salmon et al., SC'11)
  sampler      Metropolis-Hastings on |rho|^2 ("Efficient Sampling Strategy")
  observables  mixed-state observables, purity

Every function states the passage of the paper it follows. Parity pins for each function
are in tests/test_oracle_*.py. Functions without an independent pin say "parity unpinned".
"""
