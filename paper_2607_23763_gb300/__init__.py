"""GB300-native cascaded biquad (second-order-section) IIR filtering.

The compute path is the CUDA library ``libsosfilt.so`` (C ABI in
``include/sosfilt.h``); this package only binds it.  See ``SosFilter``.
"""
from ._binding import (SOS_EINVAL, SOS_ENOMEM, SOS_ECUDA, SOS_ETIMEOUT, SOS_EUNSTABLE, SOS_EBUDGET, SOS_OK,
                       SosError, SosFilter, SosServer, BatchPlan, load_library, run_batch, batch_sync_status, autotune,
                       autotune_choice, autotune_batch, autotune_batch_choice, LIB_PATH, EXPORTED)

__all__ = ["SosFilter", "SosServer", "BatchPlan", "SosError", "load_library", "run_batch", "batch_sync_status", "autotune",
           "autotune_choice", "autotune_batch", "autotune_batch_choice", "LIB_PATH", "EXPORTED", "SOS_OK", "SOS_EINVAL",
           "SOS_ENOMEM", "SOS_ECUDA", "SOS_ETIMEOUT", "SOS_EUNSTABLE", "SOS_EBUDGET"]
