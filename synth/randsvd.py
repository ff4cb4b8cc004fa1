"""randsvd-style dense test systems (Sec. 3.1.2, geometrically spaced singular values).

The paper draws its random dense matrices with MATLAB's
gallery('randsvd', n, kappa, 3): A = U diag(sigma) V^T with random orthogonal
U, V and sigma_i = kappa^(-(i-1)/(n-1)), so ||A||_2 = 1 and kappa_2(A) =
kappa.  MATLAB's random streams cannot be reproduced here; this module draws
the same distribution from numpy's PCG64:

  rng = numpy.random.default_rng(seed), then in this order
    G1 = rng.standard_normal((n, n))        -> U = Haar(G1)
    G2 = rng.standard_normal((n, n))        -> V = Haar(G2)
    X  = rng.standard_normal((n, nrhs))     (x_true)
    g  = rng.uniform(-4, 4, n)              (graded variant only: D = diag(10^g))
  A = U diag(sigma) V^T  (then A <- D A for the graded variant), B = A X,
  all in fp64.  Haar(G) is the Q factor of G = QR with the signs of R's
  diagonal moved into Q (Mezzadri's recipe for Haar-distributed orthogonal
  matrices).

The QR and products may run on a CUDA device through torch (for n in the
thousands); the draws always come from numpy, so the distribution and the
draw order do not depend on where the algebra runs.
"""

import math

import numpy as np


def _haar_np(G):
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def _algebra_torch(G1, G2, sigma, device):
    import torch
    t1 = torch.from_numpy(G1).to(device)
    t2 = torch.from_numpy(G2).to(device)
    Q1, R1 = torch.linalg.qr(t1)
    Q1 = Q1 * torch.sign(torch.diagonal(R1))[None, :]
    del t1, R1
    Q2, R2 = torch.linalg.qr(t2)
    Q2 = Q2 * torch.sign(torch.diagonal(R2))[None, :]
    del t2, R2
    s = torch.from_numpy(sigma).to(device)
    A = (Q1 * s[None, :]) @ Q2.T
    return A


def singular_values(n, kappa, mode=3):
    """randsvd's singular values: mode 3 geometric, sigma_i = kappa^(-(i-1)/(n-1));
    mode 2 one small value, sigma = (1, ..., 1, 1/kappa)."""
    if n == 1:
        return np.ones(1)
    if mode == 3:
        return float(kappa) ** (-np.arange(n, dtype=np.float64) / (n - 1))
    if mode == 2:
        s = np.ones(n)
        s[-1] = 1.0 / float(kappa)
        return s
    raise ValueError(f"randsvd mode {mode} not provided")


def randsvd_system(n, kappa, seed, nrhs=1, graded=False, device=None, mode=3):
    """Return (A, B, X) as float64 numpy arrays (A row-major n x n, B and X n x nrhs).

    ``device``: a torch device string to run the QR/products there (the
    result is copied back to host memory).  ``mode``: the singular value
    distribution (3 geometric, 2 one small value); the draws are the same."""
    rng = np.random.default_rng(seed)
    G1 = rng.standard_normal((n, n))
    G2 = rng.standard_normal((n, n))
    X = rng.standard_normal((n, nrhs))
    g = rng.uniform(-4.0, 4.0, n) if graded else None
    sigma = singular_values(n, kappa, mode)
    A_t = None
    if device is not None:
        import torch
        try:
            A_t = _algebra_torch(G1, G2, sigma, device)
        except RuntimeError:
            # torch's linear-algebra library cannot be loaded (e.g. under a
            # profiler): the same algebra with numpy on the host
            A_t = None
    if A_t is not None:
        if graded:
            A_t = torch.from_numpy(10.0 ** g).to(device)[:, None] * A_t
        B_t = A_t @ torch.from_numpy(X).to(device)
        A = A_t.cpu().numpy()
        B = B_t.cpu().numpy()
    else:
        U = _haar_np(G1)
        V = _haar_np(G2)
        A = (U * sigma[None, :]) @ V.T
        if graded:
            A = (10.0 ** g)[:, None] * A
        B = A @ X
    return np.ascontiguousarray(A), np.ascontiguousarray(B), X


def batched_systems(count, seed=0, n_lo=32, n_hi=512, logk_lo=1.0, logk_hi=6.0):
    """Sizes and condition numbers of the batched workload.

    A master generator default_rng(seed) draws n_j = integers(n_lo, n_hi + 1)
    for all j, then kappa_j = 10^uniform(logk_lo, logk_hi); system j is then
    randsvd_system(n_j, kappa_j, seed=1000 + j)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    ks = 10.0 ** rng.uniform(logk_lo, logk_hi, size=count)
    return [(int(n), float(k), 1000 + j) for j, (n, k) in enumerate(zip(ns, ks))]


HSD = "fp16,fp32,fp64"
BSD = "bf16,fp32,fp64"
SDQ = "fp32,fp64,dd"


def serving_pool(count, seed=0, n_lo=256, n_hi=8192, logk_lo=2.0, logk_hi=10.0):
    """Sizes, condition numbers and triples of the serving workload's pool.

    A generator default_rng(seed) draws, for j = 0..count-1 in turn,
    n_j = round(exp(uniform(ln n_lo, ln n_hi))), kappa_j =
    10^uniform(logk_lo, logk_hi) and a triple uniformly from (half, single,
    double), (bfloat16, single, double) and (single, double, double-double);
    system j is randsvd_system(n_j, kappa_j, seed=5000 + j)."""
    rng = np.random.default_rng(seed)
    triples = (HSD, BSD, SDQ)
    out = []
    for j in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        kappa = float(10.0 ** rng.uniform(logk_lo, logk_hi))
        out.append((n, kappa, triples[int(rng.integers(3))], 5000 + j))
    return out


def poisson_arrivals(rate, duration, pool_size, seed=0):
    """Arrival times (seconds from the start) of a Poisson process of the
    given rate over [0, duration), and for each arrival the pool index it
    requests (uniform).  Exponential gaps and indices come from
    default_rng(seed + 1), alternately."""
    rng = np.random.default_rng(seed + 1)
    times, picks = [], []
    t = 0.0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        times.append(t)
        picks.append(int(rng.integers(pool_size)))
    return times, picks


# Named workloads: (n, kappa, triple name, graded) lists.


def workloads(name):
    """The dense workloads the tests and the bench use, by name.

    small_n100      n = 100, kappa = 1e2, (half, single, double)
    sweep_n2000     n = 2000, kappa in {1e2,1e4,1e6,1e8} at (half, single,
                    double) and {1e8,1e10,1e12} at (single, double,
                    double-double), each also graded (row scalings 10^U(-4,4))
    large           n in {8192, 16384}, kappa in {1e3,1e6,1e10}
    """
    if name == "small_n100":
        return [(100, 1e2, HSD, False)]
    if name == "sweep_n2000":
        out = []
        for graded in (False, True):
            for k in (1e2, 1e4, 1e6, 1e8):
                out.append((2000, k, HSD, graded))
            for k in (1e8, 1e10, 1e12):
                out.append((2000, k, SDQ, graded))
        return out
    if name == "large":
        out = []
        for n in (8192, 16384):
            for k in (1e3, 1e6, 1e10):
                for t in (BSD, HSD, SDQ):
                    out.append((n, k, t, False))
        return out
    raise KeyError(name)


def kappa_inf(A):
    """Infinity-norm condition number (fp64 LAPACK inverse; diagnostic only)."""
    Ainv = np.linalg.inv(A)
    return float(np.max(np.sum(np.abs(A), 1)) * np.max(np.sum(np.abs(Ainv), 1)))
