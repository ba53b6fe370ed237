"""Plain FP64 CPU oracle of the D2V16 MRT flux-limiter FDLBM time step.

TEST INFRASTRUCTURE ONLY: the checker of the GPU library.  Only the tests, the
smoke check and the benchmark's CPU-baseline leg may import this package.  It
shares no code with the CUDA path.

    fdlbm_oracle.c  the step, written literally from the paper (dense transforms,
                    literal theta/psi limiter), compiled with gcc (+OpenMP)
    oracle.py       ctypes wrapper and build step
    riemann.py      exact Riemann solver for the ideal gas (pins the shock-tube runs)
    analytic.py     closed forms: Couette profile, transport coefficients, RH states
"""
from .oracle import (Oracle, build, load, matrices, central_matrix, feq, feq_hat, psi,  # noqa: F401
                     collision, update_patch)
