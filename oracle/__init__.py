"""FP64 CPU oracle for the pseudo-spectral sPTT channel time step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library in ``paper_2606_09468_gb300/``; the two meet only through the
seeded input generators in ``ptt_inputs`` (which hold none of the method's
arithmetic) and through the C ABI the tests call.

The oracle is plain and slow on purpose: direct (matrix) Fourier and Chebyshev
sums, the Chebyshev derivative matrix written from its textbook definition,
dense LU on each Fourier mode's tau system (the velocity solved as one coupled
v-phi system, not by an influence matrix), and brute-force diagnostics.

Modules
  spectral  Fourier-Chebyshev building blocks (Sec. 2, numerical details).
  ptt2d     The 2D (z-independent) channel: Eqs. 1-3, the SBDF4 step, the
            per-mode tau solves and the diagnostics of Sec. 3 (Eqs. 4-5).
  ptt3d     The 3D channel (Sec. 2 geometry): the same step with the spanwise
            direction, the v-eta velocity solve and six c components.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except
the chaotic regime beyond ~100 steps, which no closed form reaches (parity
unpinned there beyond the round-off comparison with the GPU path).
"""
from .spectral import *  # noqa: F401,F403
from . import ptt2d  # noqa: F401
from . import ptt3d  # noqa: F401
