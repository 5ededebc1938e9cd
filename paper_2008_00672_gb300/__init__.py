"""GB300-native fast-convolution filtered CP-OFDM (TX synthesis / RX analysis).

The compute path is the CUDA library built from ``csrc/`` (see ``build.py``);
``fc`` is its thin ctypes binding.
"""
from .fc import (FC_CONTINUOUS, FC_FLAG_GENERIC_KERNELS, FC_FLAG_IO_BF16, FC_FLAG_IO_TIME, FC_FLAG_REDUCED_RX, FC_FLAG_TENSOR_DFT, FC_OLA, FC_OLS, FC_RX, FC_SYMBOL_SYNC, FC_TX,  # noqa: F401
                 Batch, FcError, Pipeline, Plan, Server, State, fc_batch_create, fc_batch_destroy, fc_batch_launch, fc_plan_autotune,
                 fc_plan_choice,
                 fc_geometry_check, fc_state_bytes, fc_state_create, fc_state_destroy, fc_state_export, fc_state_import,
                 fc_state_reset, fc_tx_synthesize_stream,
                 fc_rx_analyze_stream,
                 fc_plan_create, fc_plan_destroy, fc_query, fc_rx_analyze, fc_status_string, fc_tx_synthesize,
                 load_library)
