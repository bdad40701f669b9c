"""CPU FP64 oracle of the tiled Householder BLR-QR.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only the tests, the smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA library; the only
common module is the seeded input generator, which holds none of the
method's arithmetic.
"""
