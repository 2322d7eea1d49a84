"""Plain FP64 CPU oracle for the D-SKI hot path of "Scaling Gaussian Process
Regression with Derivatives" (Eriksson et al., NeurIPS 2018).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs call it.  It shares no code with
the CUDA library (no headers, helpers, tables or constant generators) and it
imports nothing from the product package.

Every routine is written for a reader checking it against the paper by eye:
NumPy / SciPy FP64, the definitions written out, no blocking, fusion or
reordering beyond what the definition states.  Each function cites the part of
the paper it follows.

Modules
-------
keys    Keys cubic-convolution kernel, its derivative, 1-D stencils (Sec. 3.1)
quintic six-point quintic kernel (Meijering et al.), its derivative, 1-D stencils (Sec. 3.1)
dse     exact derivative SE kernel matrix K^grad (Sec. 2, App. A, App. B)
dski    D-SKI: grid, Kronecker factors, explicit sparse [W; dW], K~ (Sec. 3.1)
solve   dense Cholesky, pivoted Cholesky, QR-form preconditioner, PCG (Sec. 2, 3.3)
slq     Lanczos-from-CG tridiagonals and stochastic Lanczos quadrature (Sec. 2)
mll     log marginal likelihood and its hyperparameter gradient (Eq. 1)
probes  counter-based SplitMix64 Rademacher probes (the random draws of SLQ)
predict D-SKI predictive mean / gradient and the preconditioner variance
        estimate, exact GP mean and D-SKI variance for the pins (Sec. 5)

Pins: every routine is pinned in ``tests/test_oracle_*.py`` against closed
forms, finite differences, invariants or brute force; none is "parity
unpinned".
"""
