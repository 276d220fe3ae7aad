"""GB300-native coarse-grid incremental pressure-projection (CGP) library.

The compute path is ``csrc/*.cu`` compiled into ``_lib/libcgp.so`` (C ABI in
``include/cgp.h``); :mod:`.binding` is its thin ctypes binding.  Importing this
package does not load the library; ``binding.load()`` does, and fails loudly if it
cannot be built.
"""
