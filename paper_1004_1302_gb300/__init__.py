"""GB300 (sm_103a) Splotch per-frame rendering path: CUDA kernels behind a C
ABI (``include/splotch.h``) and a ctypes binding (:mod:`.splotch`)."""
