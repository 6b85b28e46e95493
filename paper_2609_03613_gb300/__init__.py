"""GB300-native TileGS: 3D Gaussian splatting forward rasterizer with
tile-local depth binning and selective repair (sm_103a CUDA behind a C-ABI).

The compute lives in ``libtilegs.so`` (hand-written CUDA, see ``csrc/``);
``tilegs`` is the thin ctypes binding.  ``scenes`` draws seeded inputs.
"""
