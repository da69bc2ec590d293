"""GB300 (sm_103a) implementation of the tCW template-bank track statistic.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/tcw.h``); ``tcw`` is its Python binding.
"""
from .tcw import (BANK_LATTICE, BANK_RANDOM, DEVICE, F16, F32, HOST, KERNEL_AUTO,  # noqa: F401
                  KERNEL_GROUP, KERNEL_LOOKUP, MLP_PARAMS, MLP_WEIGHTS, OPT_AMPLITUDE_POWER,
                  OPT_AUTOTUNE, OPT_BANK_CHUNK, OPT_BATCH_MEMORY, OPT_GEN_CHUNK, OPT_KEEP_STATS,
                  OPT_KERNEL, OPT_SKY_LANES, OPT_TILE_SEGMENTS, OPT_TRACK_BINS, OPT_TRIAGE_SPREAD,
                  OPT_TRIAGE_STRIDE, OPT_TRIAGE_TEMPLATES,
                  STAT_NUMBER_COUNT, STAT_POWER, Info, Mlp, Search, TcwError, bank_spec, library_path,
                  load_library, probe_fma_rate, probe_read_bandwidth)
