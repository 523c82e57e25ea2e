"""GB300-native MPSM: massively parallel sort-merge equi-join (Albutiu, Kemper, Neumann).

The join runs in libmpsm.so (hand-written CUDA for sm_103a behind a C ABI,
include/mpsm.h); this package is its thin Python binding.
"""
from .mpsm import (Plan, MPSMError, Options, make_options, strerror, lib,  # noqa: F401
                   SPLIT_HIST, SPLIT_LEARNED, SEARCH_BINARY, SEARCH_LEARNED)
