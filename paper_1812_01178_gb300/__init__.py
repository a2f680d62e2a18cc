"""GB300-native fractional-step Navier-Stokes hot path (ADI sweeps with PDD/PPT
partitioned line solves, FFT/tridiagonal Poisson solve, projection).

The compute path is the C-ABI shared library built from csrc/ (see
paper_1812_01178_gb300.binding); importing this package loads nothing.
"""
