"""FP64 CPU oracle (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import this package.  The CUDA library never does, and this
package imports nothing from the library: the two share no code.

Parity status of each function (see the pins in ``tests/test_oracle_pins.py``):

* asm_transfer, fresnel_transfer, nudft_type1, nudft_type2, uniform_dft,
  uniform_idft_crop, diffraction_type1/2/3 and their NU-ASM / NU-FRE wrappers:
  pinned (brute-force pairwise sums, numpy.fft ASM on lattice points, the
  z = 0 Dirichlet closed form, Parseval in band, the adjoint identity, the
  Fresnel Gaussian-beam closed form, the exact complex-source-point solution
  of the Helmholtz equation for ASM, linearity and shift).
* rs_direct (Eq. 10): pinned against the exact complex-source-point solution
  (Rayleigh-Sommerfeld of the first kind is exact for Helmholtz fields) and
  against the ASM on the same samples.
* band_limits: pinned against the classic band-limited ASM limit (o = 0) and
  against direct sampling of the local impulse-response position.
"""
from .diffraction import (  # noqa: F401
    modes, lattice, band_limits, band_mask_1d, asm_transfer, fresnel_transfer,
    nudft_type1, nudft_type2, uniform_dft, uniform_idft_crop,
    diffraction_type1, diffraction_type2, diffraction_type3, nuasm1, nuasm2, nuasm3, nufresnel,
    nufresnel3, rs_direct, rel_l2,
)
