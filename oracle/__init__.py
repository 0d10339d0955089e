"""FP64 CPU oracle for Rand-QLP -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct numpy (float64) implementations that check the
CUDA path: the factorisation chain (``rqlp_oracle``), a one-sided Jacobi SVD
for brute-force pins (``jacobi_svd``), the bounds of Theorems 1-3
(``bounds``) and the reference MLP used by the learned (q, p) predictor
(``mlp_oracle``). Only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; it shares no code with the CUDA
library and never imports it.
"""
