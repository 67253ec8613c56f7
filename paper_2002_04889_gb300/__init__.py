"""GB300-native (sm_103a) finite-volume solver for the 2D nonlinear shallow
water equations on unstructured triangular meshes, after the scheme of
Giles et al., "Performance analysis of Volna-OP2" (Sec. 2).

* ``volna``   -- binding of the C ABI (include/volna_gb.h); ``Solver`` wrapper
* ``inputs``  -- seeded synthetic meshes, bathymetry, initial states, gauges
* ``build``   -- in-tree build of the CUDA library
"""
__version__ = "1.0.0"
