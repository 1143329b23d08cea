"""GB300-native distance threshold search over historical continuous trajectories.

A CUDA library for sm_103a (``csrc/``, C ABI in ``include/ts.h``) and its Python binding
(``api``). The library is loaded lazily on the first call; there is no CPU fallback.
"""
from .api import (Index, Result, TsError, ts_build_index, ts_free, ts_index_export,  # noqa: F401
                  ts_index_get_info, ts_kernel_launches, ts_last_error, ts_result_arrays, ts_result_copy_to_host,
                  ts_result_count, ts_result_stats, ts_schedule, ts_search, ts_version)
