"""GB300 (sm_103a) warm-start all-pairs shortest paths after minor graph updates.

The compute path is the CUDA library built from csrc/ (C ABI in include/apsp.h);
``apsp`` is its ctypes binding.
"""
from .apsp import (APSP_DEVICE_INPUT, APSP_D_GIVEN, APSP_F32, APSP_I32, APSP_INF_I32,  # noqa: F401
                   APSP_MINIMAX, APSP_UNDIRECTED, ApspError, Batch, Graph, Server)

__version__ = "0.1.0"
