"""FP64 CPU oracle for the barrier-augmented Lagrangian (BAL) time step.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously-correct
restatement of what the method computes (Sec. 3 and Sec. 4 of arXiv 2407.00046,
"Barrier-Augmented Lagrangian for GPU-based Elastodynamic Contact"), written in
NumPy/SciPy (and PyTorch CPU autograd for derivatives of the distance
functions), FP64 throughout. It shares no code with the CUDA path. Only the
tests, the smoke check and the benchmark's CPU-baseline / reference arm may
import it; the product path never does.

Modules
  elastic   Neo-Hookean energy, P, dP/dF, per-tet gradient / PSD-projected Hessian
  barrier   IPC clamped log barrier b(d, dhat) and its derivatives (Sec. 3.3)
  distance  point-triangle / edge-edge unsigned distance with region
            classification, and autodiff gradients / Hessians of d
  contact   candidate pairs, active set, per-pair AL + barrier terms (Sec. 3.3)
  system    global energy, gradient, assembled projected Hessian, Lambda
  bal       Algorithm 1 (primal-dual loop) with exact linear solves, line search,
            time step (Sec. 3.1)
  adjoint   FP64 adjoint of the time step (not in the paper)

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, finite differences, brute force or textbook special cases, except
the stiffness grouping's convergence benefit (parity unpinned: a performance
property only).
"""
