"""CPU oracle of the RI-MP2 hot path: plain, slow, FP64 (or exact) reference code.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's CPU
baseline import anything from here; the GPU library shares no code with it.
"""
