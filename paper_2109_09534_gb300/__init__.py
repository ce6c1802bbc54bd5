"""GB300-native AO accelerated stochastic nonnegative tensor completion.

The compute path is the C-ABI CUDA library built from ``csrc/`` (declared in
``include/ntc.h``); :mod:`.ntc` is its thin ctypes binding.  Importing this
package does not load the library; :func:`ntc.load` does, and fails loudly
when the library is missing.
"""
__all__ = ["ntc", "synth"]
