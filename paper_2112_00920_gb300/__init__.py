"""GB300-native two-step Brillouin-zone sampling for real-time TDDFT.

The propagation (Eqs. 1-6 with the two-step average of Eq. 9) runs in the
CUDA library ``libtsbz.so`` behind the C ABI of ``include/tsbz.h``; this
package is its thin Python binding.
"""
from ._lib import (HXC_FROZEN, HXC_SCF, PRECISIONS, Propagator, TsbzError, halton, load,  # noqa: F401
                   pulse_samples, shifted_kpoints)
from .build import build as build_library  # noqa: F401
