"""GB300-native streaming estimator of second-order cyclic statistics (arXiv 2405.16911).

The compute path is libcyc.so (CUDA for sm_103a, C ABI in include/cyc.h); this package is
its thin binding.  There is no fallback: without the built library or a GPU, calls raise.
"""
from ._cyc import *  # noqa: F401,F403
from ._cyc import (CycError, Stream, load, declared_functions, LIB_PATH, HEADER,  # noqa: F401
                   cyc_create, cyc_create_ex, cyc_create_xy, cyc_create_window, cyc_create_full, cyc_create_full_window, cyc_push, cyc_push_xy, cyc_read,
                   cyc_read_windows, cyc_read_spectrum, cyc_detect, cyc_set_wait_budget, cyc_sums, cyc_set_n_eff, cyc_sync, cyc_reset, cyc_destroy,
                   cyc_save, cyc_load, cyc_info, cyc_phase_increment, cyc_estimate_static, cyc_profile, cyc_profile_read, cyc_strerror,
                   cyc_last_error)
from ._cyc import (Server, cyc_server_create, cyc_server_destroy, cyc_server_open,  # noqa: F401
                   cyc_server_submit, cyc_server_poll, cyc_server_drain, cyc_server_read, cyc_server_close,
                   cyc_server_stats)
from ._cyc import (cyc_net_create, cyc_net_destroy, cyc_net_nparams, cyc_net_get_params,  # noqa: F401
                   cyc_net_set_params, cyc_features, cyc_net_forward, cyc_net_gradients, cyc_net_train_step,
                   cyc_propose)
from .build import build  # noqa: F401
