"""GB300-native refinement of candidate mesh pairs for the 3-D intersection
join of closed triangle meshes (edge/face piercing plus +z parity).

Submodules:
  ``pierce``  -- ctypes binding of the C-ABI library ``libpierce.so``
                 (argument marshalling only; every step runs in CUDA kernels).
  ``synth``   -- seeded synthetic mesh datasets (inputs only).
  ``_build``  -- compiles the CUDA library for sm_103a.

Importing the package loads nothing; ``pierce`` loads the library on first use
and raises if it is missing.
"""
