"""GB300 (sm_103a) neural radiance cache hot path: encoding, fused MLP inference,
online training (relative L2 loss, backward pass, Adam) behind a C ABI.

The compute runs in the CUDA library ``libnrc.so`` built from ``csrc/``; the
Python module ``nrc`` only marshals arguments to it.
"""
