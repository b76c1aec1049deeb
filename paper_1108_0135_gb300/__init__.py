"""libmertens: exact isolated values of the Mertens function on one GB300.

The computation (arXiv:1108.0135, Sec. 2-3) runs entirely in the CUDA library
``_build/libmertens.so`` (sources under ``csrc/``, interface in
``include/libmertens.h``).  This package is its thin ctypes binding: the
functions below have the C names and only marshal arguments.
"""
from ._lib import (  # noqa: F401
    EXPORTS, MERTENS_EINVAL, MERTENS_ENOMEM, MERTENS_ENOTREADY, MERTENS_ENOTSUP, MERTENS_EOVERFLOW,
    MERTENS_ETIMEOUT, MERTENS_OK, MertensError, load, mertens, mertens_describe, mertens_destroy,
    mertens_last_error, mertens_plan, mertens_plan_info, mertens_plan_set_profiling,
    mertens_plan_window, mertens_window_result, mertens_table_create, mertens_table_info,
    mertens_plan_on_table, mertens_table_destroy, mertens_server_use_table, mertens_scan_extremes,
    mertens_probe_int_peaks, mertens_resolve, mertens_window_mu_sum, mertens_window_accumulate,
    mertens_resolve_exchange, mertens_division_constants,
    mertens_autotune, mertens_get_tuning, mertens_set_tuning,
    mertens_result, mertens_result_into, mertens_run, mertens_run_stats_get,
    mertens_server_create, mertens_server_destroy, mertens_server_poll, mertens_server_stats_get,
    mertens_server_submit, mertens_server_times, mertens_server_wait,
    mertens_set_allocator, mertens_sieve_M, mertens_sieve_M_noalloc, mertens_sieve_mu,
    mertens_strerror, use_torch_allocator,
)
