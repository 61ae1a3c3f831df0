"""GB300-native (sm_103a) ground-state AFQMC auxiliary-field update sweep.

The compute path is the C-ABI library ``libafqmc.so`` built from ``csrc/``;
``afqmc`` is its thin ctypes binding (argument marshalling only).  ``inputs``
holds the seeded synthetic input generators.  Importing the package does not
load the CUDA library; ``afqmc.load()`` does, and raises if it is missing.
"""
__all__ = ["afqmc", "inputs"]
