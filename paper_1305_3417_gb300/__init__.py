"""GB300-native geometric VoF advection (unsplit PLIC, flux-polyhedron correction).

The compute path is the C-ABI library ``libvof`` (hand-written CUDA for sm_103a)
declared in ``include/vof.h``; :mod:`paper_1305_3417_gb300.vof` is its thin
ctypes binding.  :mod:`paper_1305_3417_gb300.inputs` builds seeded synthetic
meshes and fields.
"""
__version__ = "0.1.0"
