"""GB300-native grid-indexed Euclidean epsilon self-join.

The join runs in the CUDA library built from ``csrc/`` (C ABI in
``include/sj.h``); ``sj`` is its Python binding and ``datagen`` draws the
seeded synthetic workloads.
"""
__all__ = ["sj", "datagen"]
