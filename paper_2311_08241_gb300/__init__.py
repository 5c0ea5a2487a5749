"""GB300-native split-explicit barotropic subcycle (arXiv 2311.08241, Eq. 4.10-4.12).

    inputs   seeded synthetic meshes, forcing and initial states
    build    nvcc build of the in-tree CUDA library (libsesw.so, sm_103a)
    sesw     ctypes binding of the C-ABI declared in include/sesw.h
"""
