"""FoVolNet hot path on GB300: foveated mask, sparse ray march, neural reconstruction.

Modules:
  fvn       -- ctypes binding of the C ABI in include/fvn.h (argument marshalling only)
  build     -- nvcc build of libfvn.so (csrc/) for sm_103a, in-tree
  workloads -- seeded synthetic inputs: volumes, transfer functions, cameras,
               foveation profiles, blue-noise tiles, network weights
  autotune  -- launch-shape autotuner (march thresholds and CTAs, convolution kernels)
  train     -- training of the reconstruction network on self-rendered pairs
  quality   -- PSNR / SSIM / temporal PSNR measurements for the benchmark
"""
