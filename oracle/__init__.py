"""FP64 CPU oracles for the FFT-PIM apply (arXiv 2312.02376).

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import, call or link
anything in this package: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library; the two meet only in the seeded input generators.

Modules
-------
lagrange  clamped Lagrange stencils and weights (Sec. 3.2, Eq. PGF_interp)
greens    free-space G0 (Eq. 2), brute-force image sums (Eq. 2), the Floquet
          spectral PGF (Eq. pgf) and the neutral static PGF (Eq. lgf)
ewald     Ewald-split ground truth (the plain definition Eq. 1-2 evaluated
          by Ewald splitting); not one of the paper's algorithms
pim       the FFT-PIM operator itself (Sec. 3) with a DIRECT grid convolution
          in place of the FFT, forward, adjoint and position gradient
"""
