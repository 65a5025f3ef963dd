"""GB300-native RI-MP2 energy and gradient-intermediate engine (sm_103a CUDA behind a C ABI).

Submodules are imported explicitly (``from paper_2410_21888_gb300 import rimp2``); this
file imports nothing so that the input generators load without the CUDA library.
"""
