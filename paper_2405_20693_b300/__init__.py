"""B300-native (sm_103a) X-ray rasterizer and voxelizer of R^2-Gaussian (arXiv 2405.20693).

The compute path is the C-ABI library ``libr2g.so`` (hand-written CUDA kernels);
``paper_2405_20693_b300.r2g`` is its thin ctypes binding.  ``inputs`` holds the
seeded synthetic input generators.  Submodules are imported lazily so that the
input generators stay usable on machines without the CUDA library.
"""
__all__ = ["inputs", "r2g"]
