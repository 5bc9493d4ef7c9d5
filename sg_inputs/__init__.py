"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  This module holds no arithmetic of the method: only problem
descriptions (mesh size, KL parameters, PCE orders, subdomain layout) and
seeded random arrays.  Every workload is synthetic; the paper's own
workloads are synthetic lognormal fields on the unit square as well.
"""
import numpy as np

# The five problem families.  sigma2 is the variance of the Gaussian field
# g; b is the correlation length (b_x = b_y).
CONFIGS = {
    # 32x32 mesh, L=2, p=2 (P=6), q=4 (K=15), 2x2 RAS boxes, overlap 1
    "poisson32_L2_p2": dict(N=32, L=2, p=2, q=4, sigma2=0.3, b=0.5, sx=2, sy=2, overlap=1),
    # 256x256 mesh, L=4, p=3 (P=35), q=6 (K=210), 8x8 RAS boxes, overlap 2
    "poisson256_L4_p3": dict(N=256, L=4, p=3, q=6, sigma2=0.3, b=0.5, sx=8, sy=8, overlap=2),
    # 512x512 mesh, L=6, p=3 (P=84), q=6 (K=924), var 0.5, corr. length 0.2
    "poisson512_L6_p3": dict(N=512, L=6, p=3, q=6, sigma2=0.5, b=0.2, sx=16, sy=16, overlap=2),
    # 384x384 mesh, L=4, p=4 (P=70), q=8 (K=495)
    "poisson384_L4_p4": dict(N=384, L=4, p=4, q=8, sigma2=0.3, b=0.5, sx=16, sy=16, overlap=2),
}


def splitmix64(seed):
    """Generator of successive splitmix64 outputs (published constants of
    Steele, Lea and Flood's SplittableRandom)."""
    mask = (1 << 64) - 1
    state = seed & mask
    while True:
        state = (state + 0x9E3779B97F4A7C15) & mask
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        yield z ^ (z >> 31)


def batch_system(seed):
    """One of the uneven batch systems (seeds 0..11): mesh 64..384, L in
    2..5, p in 2..4, q = 2p, correlation length uniform in [0.1, 1]."""
    g = splitmix64(seed)
    u = [next(g) for _ in range(4)]
    N = 64 + 32 * (u[0] % 11)
    L = 2 + (u[1] % 4)
    p = 2 + (u[2] % 3)
    b = 0.1 + 0.9 * ((u[3] >> 11) * 2.0 ** -53)
    S = int(min(max(round(N / 24), 4), 16))
    return dict(N=N, L=L, p=p, q=2 * p, sigma2=0.3, b=b, sx=S, sy=S, overlap=2)


def random_block(n, P, seed, dtype=np.float64):
    """Seeded standard-normal block [n, P] (operator inputs, manufactured
    solutions)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, P)).astype(dtype)
