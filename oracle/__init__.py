"""FP64 CPU oracle for the D2Q9 lattice Boltzmann outflow method of
"Reduction of Outflow Boundary Influence on Aerodynamic Performance using
Neural Networks" (arXiv 2506.05293).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of the method that the CUDA library is checked against.  Only the
test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may import it.  The product path (the C-ABI library and its
Python binding) never imports, links or calls anything in here, and nothing in
here imports the product.  The two sides share only the seeded input
generators in ``synth/``, which hold none of the method's arithmetic.

Modules
-------
lbm   -- lattice (Sec. 2.1, Eqs. 1-4), BGK and MRT collision, pull streaming,
         full-way bounce-back (Eq. 11), momentum exchange (Eqs. 13-14),
         Zou & He boundaries (Sec. 2.2, Eqs. 5-10), the NN direct outflow
         (Sec. 3.1, Eq. 15) and the characteristic outflow (Sec. 4, Eqs. 17-28),
         plus a whole-domain solver that applies them in the paper's order.
mlp   -- the small MLPs of Secs. 3.1 and 4.2: forward, hand-derived backward,
         MSE loss (Eq. 16) and Adam.
cbc_segment -- training of the CBC tuner through short simulation segments
         (Sec. 4.2): the truncated lattice's forward pass in torch float64 and
         its reverse-mode gradient with respect to the tuner's parameters.
post  -- force coefficients (Eq. 12) and the Strouhal number (Sec. 2.3).
rng   -- the SplitMix64 counter-based generator used for the inlet
         perturbation (an independent copy lives on the CUDA side).

Every floating-point quantity is float64.
"""
