"""GB300-native truncated Lennard-Jones molecular dynamics (arXiv:1210.3450 hot path).

The compute path is the CUDA library built from ``csrc/`` (see ``build.py``);
``ljmd`` is its Python binding.
"""
from .ljmd import (LJBatch, LJSystem, MDError, MD_FP32_FORCE, MD_FP64, MD_MAX_N,  # noqa: F401
                   footprint, load_library, version)
