"""GB300-native spectral-element Poisson operator and CG solve.

``sem``    -- the ctypes binding of libsem (names of the C-ABI in include/sem.h)
``Mesh``   -- one problem held by libsem (each method is one sem.run call)
``inputs`` -- seeded synthetic inputs (box vertices, random fields, mixes)
``build``  -- compiles libsem.so in-tree for sm_103a
"""
from . import inputs, sem  # noqa: F401  (sem loads libsem.so lazily, on first call)
from .mesh import Batch, Mesh, Server  # noqa: F401
