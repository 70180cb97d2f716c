"""GB300-native batched R-MATEX: rational Krylov matrix-exponential transient
simulation of RC power grids, every source group a column of one batched
CUDA launch.  ``matex`` is the binding of the C ABI in ``include/matex.h``."""

__all__ = ["matex", "build"]
