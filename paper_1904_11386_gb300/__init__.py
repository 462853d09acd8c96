"""GB300-native two-component Shan-Chen D3Q19 lattice Boltzmann with soft capsule membranes.

Importing the package loads nothing; `paper_1904_11386_gb300.scbb` loads the CUDA library on first use.
"""
