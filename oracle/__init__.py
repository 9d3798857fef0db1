"""FP64 CPU oracle of the quasi-static PIC slice loop (arXiv:2109.10277, Sec. 2-3).

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, links or runs
anything here; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

The oracle is a plain, slow restatement of the paper's method in PyTorch CPU
float64 ops (``torch.matmul`` is the only library primitive used as a step, for
the dense DST-I).  It shares no code with the CUDA path.  Because every step is
written with differentiable torch ops, running it under ``torch.autograd`` is the
oracle's taped FP64 adjoint.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):
  dst / poisson_solve  pinned: eigenmodes, S.S = (N/2) I, brute-force sums, 5-point residual
  ddx / ddy            pinned: exact on quadratics, orientation
  shape / deposit      pinned: partition of unity, charge conservation, brute-force B-spline
  gather               pinned: affine reproduction, transpose identity with deposit
  derivs               pinned: Lorentz-force chain rule, invariant Psi - psi(x_p)
  ab5 step             pinned: exact on quartic derivatives, order-5 convergence
  sweep                pinned: zero-beam invariant, symmetry, Ez ~ -d(psi)/d(zeta),
                       conservation of sum(rho - Jz), discrete linear wake
  beam binning         pinned: brute-force bin membership
  beam deposit         pinned: rho_b = q n_b at the nodes of an affine-density lattice beam (all
                       orders), J_b = rho_b u / gamma, slice charge of a random beam, and the
                       linear wake built from the driver's closed-form density
  explicit B_perp      pinned: Laplacian/shifted DST eigenmodes, PCG against a dense solve and exact for
                       constant chi, source terms against central differences of the deposited current
                       along the particle equations, linear wake, agreement with a converged
                       predictor-corrector as dzeta shrinks
  beam moments         pinned: numpy weighted covariance, shear and offset invariance of the emittance
  predictor-corrector  pinned at the workloads' setting (5 iterations, mixing 0.05): linear wake
                       within 5 % converging under dzeta and dx refinement; lag behind a converged
                       iteration second order in dzeta
  beam push            pinned: uniform-B gyration, uniform-E energy gain, time reversibility
  plasma species       pinned: a split into two half-density species is exact, heavy mobile ions
                       reproduce the immobile background, a positron plasma's wake differs at second
                       order in n_b, mobile light ions raise the plasma frequency by sqrt(1 + m_e/M)
  slice loop / sweep   SliceLoop.slice is the per-slice body the sweep and the temporal pipeline
                       drive; the pipeline over CPU ranks reproduces the serial loop bit for bit
  blowout regime        inside the electron-free channel behind a dense driver the transverse
                       force ExmBy is x/2 and Ez is flat across it (ion-channel focusing);
                       beyond that the blowout-regime physics (512^2 n_b=5) is parity unpinned
  working_precision    a test knob: the same steps in another float type (rounding floors)
"""
from .qsa import *  # noqa: F401,F403
