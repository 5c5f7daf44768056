"""CPU oracle for the foveated renderer: slow, plain, float64.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import, call or link
anything under this directory.  The product path (the CUDA library and its
Python binding) never does, and shares no code with it.

Modules:
  mask     -- Eq. 1-3: threshold table, hashed or tiled noise, sample mask, C_max, ids
  march    -- FP64 emission-absorption ray marcher (C, OpenMP), dense / masked,
              headlight Phong or global shadows
  net      -- FP64 U-Net forward / backward (plain or with the previous output as
              input), kernel prediction + blend, spatial and temporal losses, Adam
  wnet     -- FP64 two-stage network: direct prediction D, kernel prediction K
              applied to D's output at several scales in sequence; forward / backward
  metrics  -- PSNR, SSIM, temporal PSNR
  fallback -- probe set and the denser-mask rule
"""
