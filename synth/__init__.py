"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
runs.  Holds no arithmetic of the method: point clouds, target fields with
their analytic gradients, and the problem parameters."""
