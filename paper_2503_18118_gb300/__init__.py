"""GB300-native Monte-Carlo evaluation of near-field XL-MIMO multiuser
beamforming: spherical-wave channels generated on the fly, K x K Gram
matrices, ZF/MMSE/MRC receivers, sum rate, capacity and the capacity
saturation point, all computed by hand-written sm_103a CUDA kernels behind a
C ABI (``include/xlmimo.h``).

Importing this package does not load the CUDA library; the first call into
``paper_2503_18118_gb300.xlmimo`` does, and fails loudly if it is missing.
"""
__all__ = ["inputs", "xlmimo"]
