"""GB300-native two-site DMRG sweep engine (sm_103a).

The compute path lives in libgbdmrg.so (csrc/, C ABI in include/gbdmrg.h);
`gbdmrg` is its ctypes binding and `build` compiles it.  Importing this
package does not load the library; gbdmrg.lib() does, and raises if it has
not been built.
"""
__all__ = ["build", "gbdmrg"]
