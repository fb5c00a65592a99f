"""Plain, slow FP64 CPU oracle for the rank-adaptive sweep-based SI-DSA of the steady
first-order S_N radiative transfer equation in 2D x-y (Guo & Peng, "Highly efficient
rank-adaptive sweep-based SI-DSA for the radiative transfer equation via mild space
augmentation").

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code with the
CUDA library: operators are assembled here by Gauss quadrature from their integral
definitions (App. B), transport solves are direct sparse LU solves of each
per-ordinate system (the quantity the sweep of Sec. 2.2 computes), and the low-rank
algorithm follows Sec. 3 / Alg. 1-2 step by step with numpy / scipy primitives.

Modules:
  quadrature  -- CL(N_theta, N_Omega_z) angular quadrature (App. A)
  dg          -- upwind DG-Q1 matrices D_x^+-, D_y^+-, Sigma_t, Sigma_s, G, g^bc (Sec. 2.1, App. B)
  transport   -- per-ordinate solves (Eq. mat-vec, Eq. SI), upwind block Gauss-Seidel (Sec. 2.2)
  dsa         -- modified-interior-penalty diffusion correction (Eq. DSA; reading in the module)
  si_dsa      -- full-rank SI-DSA (Sec. 2.2 and Alg. 1 with the full-rank SI step)
  philox      -- Philox4x32-10 counter-based generator (Salmon et al., SC'11)
  lowrank     -- rank-adaptive low-rank SI and SI-DSA (Sec. 3.1-3.4, Alg. 1, Alg. 2)
  adjoint     -- discrete adjoint SI-DSA and detector-response gradients
  timedep     -- backward-Euler steps (Sec. 3.7): coupled solve, full-rank and low-rank SI-DSA
"""
from .quadrature import cl_quadrature  # noqa: F401
from .dg import Discretisation  # noqa: F401
