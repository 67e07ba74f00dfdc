"""GB300-native binocular 2D Gaussian splatting by reprojection and selective
patching: CUDA kernels for sm_103a behind a C ABI (include/gs.h), with a thin
ctypes binding (gs.py) and seeded synthetic inputs (synth.py)."""
