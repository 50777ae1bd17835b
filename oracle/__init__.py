"""Plain FP64 CPU oracle for the TDGL + Poisson time step of FerroX (arXiv 2210.15668).

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU
baseline legs of `bench.py` may import this package.  The product path (the
CUDA library and its Python binding) never imports, links or calls it, and it
shares no code with the CUDA path: the only common module is the seeded input
generator `paper_2210_15668_gb300.inputs`, which holds data, not arithmetic.

What it computes (SI units, float64 everywhere):
  stack.py        per-plane material table from the layer list (Fig. 1a, Table 1)
  poisson.py      finite-volume form of  div(eps grad Phi) = div P - rho  (Eq. Poisson),
                  periodic x/y, Dirichlet electrodes (Methods, electrical BCs), and an
                  exact separable direct solver (2-D FFT in x/y + tridiagonal in z)
  tdgl.py         the TDGL force of Eq. TDGL2, the polarization boundary conditions
                  (Methods, Eqs. Pbc/PbcFree/PbcDir), and the first/second-order
                  predictor-corrector time step (Methods, Steps 0, 1a/1b, 2a/2b)
  carriers.py     Maxwell-Boltzmann carrier charge (Eq. MaxBolt_ne_np, Eq. rho) and the
                  nonlinear Poisson solve by damped Newton (the paper's lagged fixed point
                  is kept too, Methods "Numerical Approach")
  diagnostics.py  interface charge Q and V_fe (Results, MFIM section), electrode charges
  nn.py           FP64 reference of the small 3-D convolutional network's layers

Readings of points the paper leaves open are stated in each function's docstring;
they are the same readings the CUDA path implements.
"""
from .stack import EPS0, Q_E, K_B, planes  # noqa: F401
from . import poisson, tdgl, carriers, diagnostics  # noqa: F401
