"""GB300-native (sm_103a) particle hot path of OpenFPM (arXiv 1804.07598).

The compute lives in ``libfpm.so`` (hand-written CUDA behind a C ABI, declared
in ``include/fpm.h``); ``fpm`` is its thin ctypes binding.  Importing this
package does not load the library: ``fpm.lib()`` does, and fails loudly when
it is missing.
"""
__all__ = ["fpm", "inputs"]
