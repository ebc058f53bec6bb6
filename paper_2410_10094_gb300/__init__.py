"""GB300 (sm_103a) sparse COO tensor contraction after Swift (arXiv 2410.10094).

The work happens in ``libstc.so`` (C ABI in include/stc.h, CUDA kernels in ``csrc/``);
this package is its Python binding. Build the library with
``python -m paper_2410_10094_gb300.build``."""
from .binding import (ACC_AUTO, ACC_DENSE, ACC_HASH, ACC_HASH_SCAN, ACC_ROWS, IDS_AUTO, IDS_DENSE, IDS_DIRECT, OPERANDS_AS_GIVEN, OPERANDS_AUTO, OPERANDS_SWAPPED, STRATEGY_AUTO, STRATEGY_GLOBAL, STRATEGY_GROUPED, BatchPlan, BatchProblems, Context, Result, Server, StcError, check,
                      contract, contract_batch, contract_keyed, count, default_context, dense_ids, group_keys, linearize, load, measure_peaks, stc_contract, stc_count,
                      stc_contract_batch, stc_create, stc_ctx_stats, stc_dense_ids, stc_destroy, stc_group_keys, stc_group_keys_static,
                      stc_linearize, stc_opts, stc_result_data,
                      stc_result_free, stc_result_info, stc_result_stats, stc_stats, stc_status_string)

__all__ = [
    "ACC_AUTO", "ACC_DENSE", "ACC_HASH", "ACC_HASH_SCAN", "ACC_ROWS", "IDS_AUTO", "IDS_DENSE", "IDS_DIRECT", "OPERANDS_AS_GIVEN", "OPERANDS_AUTO", "OPERANDS_SWAPPED", "STRATEGY_AUTO", "STRATEGY_GLOBAL", "STRATEGY_GROUPED", "BatchProblems", "Context", "Result", "Server", "StcError", "check", "contract", "contract_batch",
    "count", "default_context", "dense_ids", "group_keys", "linearize", "load", "stc_contract", "stc_count", "stc_create",
    "stc_contract_batch", "stc_ctx_stats", "stc_dense_ids",
    "stc_destroy", "stc_group_keys", "stc_group_keys_static", "stc_linearize", "stc_opts", "stc_result_data", "stc_result_free",
    "stc_result_info", "stc_result_stats", "stc_stats", "stc_status_string",
]
