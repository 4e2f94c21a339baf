"""GB300-native batched Smith-Waterman (affine gaps) for many-against-many
protein similarity search.

The compute path is the CUDA library ``libswgb.so`` (C-ABI in
``include/swgb.h``); ``swgb`` is its thin ctypes binding.  ``workload`` draws
seeded synthetic inputs.
"""
