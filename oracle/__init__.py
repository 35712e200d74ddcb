"""Plain, slow FP64 CPU oracle of the reconstruction path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  Nothing in the library imports this
package, and it imports nothing from the library; the two share only the
seeded input generators of `synth`.

  fdtd.c / fdtd.py  K (staggered pressure/velocity leapfrog + point sensors)
                    and K* (reverse sweep of the same program), paper Sec. 2
  wavelet.py        periodic orthonormal Daubechies DWT, E_s and E_s*,
                    paper Sec. 4 (Prop. 4.2, the diagonal level scaling)
  solve.py          CG on (E_s* K* K E_s + alpha I) u = E_s* K* y, paper
                    Eq. (linear_minimization) in coefficient form
"""
from .fdtd import Wave, set_threads, max_threads, sponge_sigma, sponge_sigma_max  # noqa: F401
from .wavelet import Wavelet, daubechies, highpass  # noqa: F401
from .fourier import FourierPrior  # noqa: F401
from .solve import cg, cg_converged, normal_op, rhs, Breakdown  # noqa: F401
