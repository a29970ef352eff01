"""GB300-native minimum-spanning-forest solver (Borůvka and Filter-Borůvka rounds).

Importing the package loads nothing; the CUDA library is loaded by
``paper_2302_12199_gb300.mst`` on first use and fails loudly when missing.
"""
