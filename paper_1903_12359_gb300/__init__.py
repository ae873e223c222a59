"""GB300-native PGCP: parallelizable global conformal parameterization via partial welding.

Importing the package loads nothing native; ``paper_1903_12359_gb300.api``
loads the CUDA library and raises if it is missing.
"""
