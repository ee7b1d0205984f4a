"""GB300-native Fourier pseudo-spectral BDF2 steppers for the functionalized
Cahn-Hilliard gradient flow (arXiv 2006.04784).

Importing the package loads nothing native; ``paper_2006_04784_gb300.fch``
loads the CUDA library (and fails loudly if it has not been built).
"""
