"""CPU float64 oracle for the Yin-Yang multipole gravity solver.

TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` may import this package.  The CUDA library
(``paper_1806_04593_gb300``) never imports it, and it imports nothing from the
library: the two share no code.

See :mod:`oracle.yinyang` for the method and the readings taken where the
paper is silent or garbled.
"""

from .yinyang import (  # noqa: F401
    OracleGrid,
    OraclePolarGrid,
    angular_edges,
    assoc_legendre,
    azimuthal_integrals,
    dlegendre_dtheta,
    legendre_m_over_sin,
    normalisation,
    other_patch_angles,
    other_patch_cartesian,
    overlap_weights,
    polar_integrals,
    polar_integrals_appendix,
    radial_integrals,
)
