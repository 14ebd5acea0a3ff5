"""GB300 (sm_103a) pyramidal FAST detection with fused 3x3 NMS and per-cell
maximum selection -- the detection hot path of "Faster than FAST:
GPU-Accelerated Frontend for High-Speed VIO" (Nagy, Foehn, Scaramuzza, 2020).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/vio.h``); ``vio`` is its ctypes binding and ``synth`` the seeded
frame generator.  Importing the package does not load the library.
"""
