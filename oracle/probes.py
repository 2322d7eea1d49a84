"""Counter-based SplitMix64 Rademacher probes for SLQ (Sec. 2).

The probes are the random draws of the stochastic trace estimator.  Both the
oracle and the CUDA library implement the same counter-based generator from
its published definition (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): the k-th output (k = 1, 2,
...) of the SplitMix64 stream seeded with s is mix64(s + k * GAMMA), with
GAMMA = 0x9E3779B97F4A7C15 and mix64 the "variant 13" finaliser
  z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
  z *= 0x94D049BB133111EB; z ^= z >> 31          (all mod 2^64).
Probe j, row e (row index in the user's block order [values; d/dx_1; ...])
takes counter k = j * N + e + 1 and value +1 if the top bit of the output is
0, else -1.  Preconditioned probes (``preconditioned_probes``) draw w of
length N + r this way and map it through C = [D^{1/2}, L], so that
E[z z^T] = C C^T = M.

Test infrastructure only (see ``oracle/__init__``).
"""
import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def mix64(z):
    """SplitMix64 finaliser on Python ints (mod 2^64)."""
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def splitmix64_stream(seed, count):
    """The sequential generator: state += GAMMA, output mix64(state)."""
    state = seed & MASK
    out = []
    for _ in range(count):
        state = (state + GAMMA) & MASK
        out.append(mix64(state))
    return out


def splitmix64_at(seed, k):
    """k-th output (k >= 1) of the stream, computed directly from the counter."""
    return mix64((seed + k * GAMMA) & MASK)


def _mix64_vec(z):
    z = z.astype(np.uint64)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def rademacher(seed, N, P):
    """N x P probe matrix (column j = probe j, rows in block order)."""
    k = (np.arange(N * P, dtype=np.uint64).reshape(P, N) + np.uint64(1))
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK) + k * np.uint64(GAMMA)
        bits = _mix64_vec(z) >> np.uint64(63)
    return np.where(bits == 0, 1.0, -1.0).T.copy()


def preconditioned_probes(seed, precond, P):
    """N x P probes z_j = D^{1/2} w1 + L w2, w = rademacher(seed, N + r, P)
    (``precond`` an oracle.solve.QRPreconditioner)."""
    N, r = precond.L.shape
    return precond.factor_apply(rademacher(seed, N + r, P))
