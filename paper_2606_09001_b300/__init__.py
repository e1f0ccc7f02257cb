"""B300-native smoothed-aggregation AMG-preconditioned Krylov solver with a
reverse-mode adjoint (the method of the JAX-AMG paper, rebuilt on hand-written
sm_103a CUDA kernels behind a C ABI)."""
