"""GB300 (sm_103a) implementation of the tCW template-bank track statistic.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/tcw.h``); ``tcw`` is its Python binding.
"""
from .tcw import (DEVICE, F16, F32, HOST, KERNEL_AUTO, KERNEL_GROUP, KERNEL_LOOKUP,  # noqa: F401
                  OPT_AMPLITUDE_POWER, OPT_AUTOTUNE, OPT_BANK_CHUNK, OPT_BATCH_MEMORY, OPT_KEEP_STATS, OPT_KERNEL,
                  OPT_SKY_LANES, OPT_TILE_SEGMENTS, OPT_TRIAGE_SPREAD, MLP_PARAMS, MLP_WEIGHTS,
                  STAT_NUMBER_COUNT, STAT_POWER, Info, Mlp, Search, TcwError, library_path, load_library,
                  probe_read_bandwidth)
