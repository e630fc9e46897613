"""GB300-native (sm_103a) implementation of the Icarus 3.0 heliosphere hot path (arXiv 2501.15923).

The compute path is libicarus.so (hand-written CUDA behind a C ABI, include/icarus.h); the Python
binding in `icarus.py` only marshals arguments. `inputs.py` generates seeded synthetic drivers.
Importing this package does not load the CUDA library; `paper_2501_15923_gb300.icarus` does.
"""
__all__ = ["inputs", "icarus"]
