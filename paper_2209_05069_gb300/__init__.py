"""GB300-native geometric docking hot path (LiGen-style multi-restart rigid alignment and
greedy torsion optimisation with clash check, arXiv 2209.05069 Section 4).

The compute path is the CUDA library ``libdock.so`` built from ``csrc/`` and reached through
the C-ABI declared in ``include/dock.h``; :mod:`.dock` is its ctypes binding.  Importing this
package loads nothing: ``synth`` (input generation) stays usable on machines without a GPU.
"""
