"""Plain FP64 CPU oracle for extended convolution and correlation.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run it.

Every function evaluates the paper's definitions directly, per output point,
with the filter transformed per pixel from its closed-form band-limited
expansion (the transformed coordinate is formed with cos/sin, then |.| and
atan2) -- never through the steering identity the CUDA path relies on.
Boundaries are periodic (indices mod (h, w)); integrals become unit-weight
lattice sums.

Modules:
  filters_so2 -- SO(2) filter models (analytic, radial table) and the
                 decomposition of a sampled filter into angular harmonics
                 (Sec. 4.1, "Filter Decomposition").
  so2         -- extended convolution / correlation (Eqs. Def-EConv,
                 Def-ECorr) and the quantised-rotation sweep (Sec. 5.2).
  scale       -- scale-adaptive smoothing with Mellin harmonics (Sec. 8,
                 Eq. normalization).
"""
