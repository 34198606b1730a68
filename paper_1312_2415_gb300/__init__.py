"""GB300-native spin-adapted two-site DMRG (hot path: H_eff matvec inside Davidson and
the SVD truncation of the two-site tensor) behind the C ABI of include/dmrg_gb300.h."""
from .binding import (Batch, Context, DMRGError, EXPORTED, device_memory_in_use, extrapolate,  # noqa: F401
                      load, set_device_memory_cap, test_tc_timeout)
