"""FP64 CPU oracle of the Gaussian splatting rasterizer hot path.

Test infrastructure only: the tests, the smoke check and the benchmark's CPU
baseline use it; the product path never does.
"""
