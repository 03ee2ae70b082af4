"""GB300-native (sm_103a) hot path of LSH-MF (arXiv 2111.11682).

The compute lives in liblshmf.so (C ABI: include/lshmf.h, CUDA sources in
csrc/); `lshmf` is its thin Python binding over torch CUDA tensors.
"""
from .lshmf import (GEN_MINHASH, GEN_RAND, GEN_RPCOS, OPT_MEMORY_LIMIT, OPT_SGD_GROUPS, OPT_SGD_SLOTS,
                    OPT_TEST_WITHHOLD, OPT_WAIT_POLLS, Batch, Config, LshMF, LshmfError, Params, SYMBOLS,
                    autotune_P, autotune_tile, batch_plan, config_from_workload, launch_count, library_path, load, pick_P, plan_batch_P,
                    plain_mf_config)

__all__ = ["Config", "LshMF", "LshmfError", "Params", "SYMBOLS", "config_from_workload", "launch_count", "load",
           "library_path", "plain_mf_config", "Batch", "autotune_P", "autotune_tile", "batch_plan", "pick_P", "plan_batch_P", "GEN_RAND", "GEN_RPCOS", "GEN_MINHASH",
           "OPT_MEMORY_LIMIT", "OPT_WAIT_POLLS", "OPT_SGD_SLOTS", "OPT_SGD_GROUPS", "OPT_TEST_WITHHOLD"]
