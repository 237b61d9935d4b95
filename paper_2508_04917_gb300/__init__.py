"""GB300-native subdomain-wise ILU0 preconditioning and BiCGSTAB (arXiv 2508.04917 hot path).

The compute path is the CUDA library ``libilu0dd.so`` (C ABI in
``include/ilu0dd.h``); :mod:`.binding` marshals arguments to it.
"""
from .binding import (BF16, DF64, F32, F64, PRECISIONS, Batch, Ilu0DD, Ilu0DDError,  # noqa: F401
                      declared_functions, default_opts, levels_device, library_path, load, partition_bfs, strerror,
                      workspace_size)
