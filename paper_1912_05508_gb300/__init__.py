"""GB300-native mixed-precision recursive Gram-Schmidt QR and Krylov least squares.

Importing the package loads nothing; the CUDA library is loaded on first use by
``paper_1912_05508_gb300.lls`` (which raises if it has not been built).
"""
