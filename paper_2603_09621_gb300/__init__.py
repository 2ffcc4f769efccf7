"""GB300-native Gaussian volume rasteriser for zero-shot MRI super-resolution.

The compute path is the C-ABI CUDA library ``libgsmri.so`` (declared in ``include/gs_api.h``);
``paper_2603_09621_gb300.gs`` is its thin Python binding. Importing this package does not
load the library; ``paper_2603_09621_gb300.gs`` does, and fails loudly if it is missing.
"""
__all__ = ["inputs"]
