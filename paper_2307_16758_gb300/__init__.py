"""GB300 (sm_103a) finite-volume shallow-water solver on unstructured triangles.

``swe`` is the Python binding of the C ABI (``include/swe.h``); ``workloads``
builds the seeded synthetic meshes and states; ``build`` compiles the CUDA
library in-tree.  Submodules load lazily so that importing the package needs
neither a GPU nor a built library.
"""
__all__ = ["swe", "workloads", "build"]
