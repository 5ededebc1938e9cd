"""GB300-native fast-convolution filtered CP-OFDM (TX synthesis / RX analysis).

The compute path is the CUDA library built from ``csrc/`` (see ``build.py``);
``fc`` is its thin ctypes binding.
"""
from .fc import (FC_CONTINUOUS, FC_FLAG_GENERIC_KERNELS, FC_FLAG_REDUCED_RX, FC_OLA, FC_OLS, FC_SYMBOL_SYNC, FcError, Plan, State,  # noqa: F401
                 fc_geometry_check, fc_state_create, fc_state_destroy, fc_state_reset, fc_tx_synthesize_stream,
                 fc_rx_analyze_stream,
                 fc_plan_create, fc_plan_destroy, fc_query, fc_rx_analyze, fc_status_string, fc_tx_synthesize,
                 load_library)
