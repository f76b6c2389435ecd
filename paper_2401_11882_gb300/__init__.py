"""GB300-native smoothed, differentiable 2D image-method ray tracing.

The compiled CUDA library is loaded lazily, on the first call that needs it,
so that the seeded scene generators (``scenes``) import without a GPU.
"""
