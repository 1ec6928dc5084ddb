"""GB300-native replica-exchange grand-canonical Monte Carlo (arXiv:1908.11118).

The sampler, the replica exchange and the MBAR reweighting run in the CUDA
library built from ``csrc/`` (C ABI in ``include/regc.h``); ``Regc`` and the
``mbar_*`` functions are its Python binding.
"""
from .regc import (MOVE_DTYPE, SURROGATE_PARAMS, Batch, Regc, mbar_last_info, mbar_query, mbar_solve,  # noqa: F401
                   mu_of_pressure, pressure_of_mu, surrogate_gradient)
from ._lib import RegcError  # noqa: F401
