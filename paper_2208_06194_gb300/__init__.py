"""Tiled Householder BLR-QR on one GB300 (sm_103a).

Importing the package loads nothing: the CUDA library is loaded by
``paper_2208_06194_gb300.blr`` on first use and fails loudly if it is
missing.  ``workloads`` holds the seeded input generators.
"""
