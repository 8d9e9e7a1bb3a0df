"""GB300-native (sm_103a) Monte Carlo internal dosimetry for 18F PET/CT.

Importing the package loads nothing; ``paper_2111_11687_gb300.nmdose`` binds the
CUDA library (``libnmdose.so``) on first use and raises if it is missing.
"""
