"""GB300-native finite-temperature TD-DMRG for carrier mobility (hot path).

The computation lives in ``libtdmrg.so`` (CUDA kernels for sm_103a behind the C ABI of
``include/tdmrg.h``); this package only builds it (``build``) and marshals arguments to it
(``binding``)."""
from .binding import Batch, Model, mobility, PREC_C128, PREC_C64_3XTF32, TdmrgError, load  # noqa: F401
