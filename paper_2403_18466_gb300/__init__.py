"""GB300-native D2Q9 lattice Boltzmann with a learned, conservative collision.

The compute path is the C-ABI library ``liblbm`` (hand-written sm_103a CUDA);
``lbm`` is its thin ctypes binding.  Submodules are imported lazily so that
``inputs`` (seeded synthetic fields, no method arithmetic) can be used without
loading the CUDA library.
"""
__all__ = ["lbm", "inputs", "autograd", "train", "data"]
