"""Seeded synthetic workloads for the QMC-slicing kernel sum.

This module only *draws inputs*: point clouds, weights, slicing directions and
the harness-level parameter choices (median rule, radius).  It contains none of
the summation method's arithmetic, so both the FP64 oracle and the CUDA path
can consume exactly the same FP32 arrays.

Every generator is a pure function of its seed (``numpy.random.default_rng``,
FP64 draws cast to FP32 at the end).  The shapes and distributions follow the
paper's workloads (Sec. 4.3 and App. H: Letters / MNIST / FashionMNIST /
CIFAR10 sized problems), which are not available here; synthetic stand-ins are
used instead:

* ``small_gauss``   d=3, N=M=1000, uniform in the unit ball, Gauss sigma=0.5,
                    P=64 spherical-Fibonacci directions, N_ft=256, W=8.
* ``mnist_laplace`` d=784, N=M=60000, each coordinate 0 w.p. 0.8 else U(0,1)
                    (MNIST-shaped, App. H "Higher Dimensions"), w=1/N,
                    Laplace with 1/alpha = median pair distance (median rule,
                    Sec. 4.1), P=2048 orthogonal directions, N_ft=1024.
* ``gauss64_negdist`` d=64, N=M=200000, x,y ~ N(0,I), w ~ N(0,1), negative
                    distance kernel, P=4096 Sobol directions, N_ft=2048.
* ``mmd_flow16``    d=16, N=M=100000 MMD-flow problem (App. H, MMD flows).
* ``batch256_problems`` 256 Gauss problems of uneven N, M, d and N_ft.
* ``gpu_compare30`` d=30, N=M=960000 PCA-shaped data summed against itself
                    (App. H, "GPU Comparison").

Direction designs (Sec. 4.1 "QMC Sequences"): iid uniform, Sobol mapped through
the normal inverse CDF and normalised, orthogonal (first P columns of
ceil(P/d) Haar-orthogonal matrices) and, for d=3, spherical Fibonacci points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20241001

KERNELS = ("gauss", "laplace", "negdist")


# --------------------------------------------------------------------------
# point clouds
# --------------------------------------------------------------------------
def uniform_ball(rng: np.random.Generator, n: int, d: int) -> np.ndarray:
    """n points uniform in the unit ball of R^d (direction * U^(1/d))."""
    g = rng.standard_normal((n, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    r = rng.random(n) ** (1.0 / d)
    return (g * r[:, None]).astype(np.float32)


def sparse_unit_cube(rng: np.random.Generator, n: int, d: int, p_zero: float = 0.8) -> np.ndarray:
    """MNIST-shaped data: each coordinate is 0 w.p. p_zero, else U(0,1)."""
    vals = rng.random((n, d))
    mask = rng.random((n, d)) < p_zero
    vals[mask] = 0.0
    return vals.astype(np.float32)


def gaussian(rng: np.random.Generator, n: int, d: int, scale: float = 1.0) -> np.ndarray:
    return (scale * rng.standard_normal((n, d))).astype(np.float32)


def uniform_box(rng: np.random.Generator, n: int, d: int, lo: float, hi: float) -> np.ndarray:
    return rng.uniform(lo, hi, (n, d)).astype(np.float32)


# --------------------------------------------------------------------------
# slicing directions (Sec. 4.1); each returns a (P, d) FP32 array of unit rows
# --------------------------------------------------------------------------
def _normalise_rows(a: np.ndarray) -> np.ndarray:
    return a / np.linalg.norm(a, axis=1, keepdims=True)


def directions_iid(rng: np.random.Generator, P: int, d: int) -> np.ndarray:
    """iid uniform on S^{d-1}: xi = g/|g| with g ~ N(0, I)."""
    return _normalise_rows(rng.standard_normal((P, d))).astype(np.float32)


def directions_fibonacci(P: int) -> np.ndarray:
    """Spherical Fibonacci points on S^2: z_p = 1-(2p+1)/P, phi_p = 2 pi p / golden.

    The z-coordinates are the midpoints of P equal cells of [-1, 1], so for a
    vector along e_z the slice average is the composite midpoint rule.
    """
    p = np.arange(P, dtype=np.float64)
    z = 1.0 - (2.0 * p + 1.0) / P
    golden = (1.0 + math.sqrt(5.0)) / 2.0
    phi = 2.0 * math.pi * p / golden
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    xi = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return xi.astype(np.float32)


def haar_orthogonal(rng: np.random.Generator, d: int) -> np.ndarray:
    """A Haar-distributed orthogonal d x d matrix (QR of a Gaussian matrix with
    the sign of diag(R) folded into Q)."""
    g = rng.standard_normal((d, d))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return q


def directions_orthogonal(rng: np.random.Generator, P: int, d: int) -> np.ndarray:
    """First P columns of ceil(P/d) independent Haar-orthogonal matrices."""
    blocks = [haar_orthogonal(rng, d) for _ in range((P + d - 1) // d)]
    cols = np.concatenate(blocks, axis=1)[:, :P]
    return np.ascontiguousarray(cols.T).astype(np.float32)


def directions_sobol(rng: np.random.Generator, P: int, d: int) -> np.ndarray:
    """Scrambled Sobol points in (0,1)^d -> inverse normal CDF -> normalised."""
    from scipy.special import ndtri
    from scipy.stats import qmc

    seed = int(rng.integers(0, 2**31 - 1))
    u = qmc.Sobol(d, scramble=True, seed=seed).random(P)
    u = np.clip(u, 1e-12, 1.0 - 1e-12)
    return _normalise_rows(ndtri(u)).astype(np.float32)


def random_rotation(rng: np.random.Generator, xi: np.ndarray) -> np.ndarray:
    """Randomised QMC design A xi with A ~ Haar(O(d)) (App. D)."""
    a = haar_orthogonal(rng, xi.shape[1])
    return (xi.astype(np.float64) @ a.T).astype(np.float32)


def make_directions(kind: str, P: int, d: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if kind == "fibonacci":
        if d != 3:
            raise ValueError("spherical Fibonacci directions exist for d=3 only")
        return directions_fibonacci(P)
    if kind == "orthogonal":
        return directions_orthogonal(rng, P, d)
    if kind == "sobol":
        return directions_sobol(rng, P, d)
    if kind == "iid":
        return directions_iid(rng, P, d)
    raise ValueError(f"unknown direction design {kind!r}")


# --------------------------------------------------------------------------
# harness-level parameter choices
# --------------------------------------------------------------------------
def median_pair_distance(x: np.ndarray, y: np.ndarray, n_pairs: int, seed: int) -> float:
    """Median rule (Sec. 4.1): median of |x_i - y_j| over n_pairs random pairs."""
    rng = np.random.default_rng(seed)
    i = rng.integers(0, x.shape[0], n_pairs)
    j = rng.integers(0, y.shape[0], n_pairs)
    dist = np.linalg.norm(x[i].astype(np.float64) - y[j].astype(np.float64), axis=1)
    return float(np.median(dist))


def radius(x: np.ndarray, y: np.ndarray) -> float:
    """R = max|x_n| + max|y_m| (App. G, eq. radius_xy), in FP64 on the FP32 data."""
    rx = float(np.max(np.linalg.norm(x.astype(np.float64), axis=1))) if x.shape[0] else 0.0
    ry = float(np.max(np.linalg.norm(y.astype(np.float64), axis=1))) if y.shape[0] else 0.0
    return rx + ry


# --------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------
@dataclass
class Problem:
    name: str
    d: int
    kernel: str            # "gauss" | "laplace" | "negdist" | "matern" | "riesz" | "tps"
    kparam: float          # sigma (gauss), alpha (laplace), beta (matern), r (riesz), unused otherwise
    P: int
    n_ft: int
    x: np.ndarray          # (N, d) float32
    w: np.ndarray          # (N,)  float32
    y: np.ndarray          # (M, d) float32
    xi: np.ndarray         # (P, d) float32 unit rows
    R: float               # radius bound used for the rescaling
    window: int = 8
    meta: dict = field(default_factory=dict)
    kparam2: float = 0.0   # nu (matern), unused otherwise

    @property
    def N(self) -> int:
        return int(self.x.shape[0])

    @property
    def M(self) -> int:
        return int(self.y.shape[0])

    @property
    def point_slices(self) -> int:
        return (self.N + self.M) * self.P


def small_gauss(N: int = 1000, M: int = 1000, P: int = 64, n_ft: int = 256,
                seed: int = SEED_BASE + 1) -> Problem:
    """d=3 Gauss sigma=0.5 on the unit ball, spherical Fibonacci directions."""
    rng = np.random.default_rng(seed)
    x = uniform_ball(rng, N, 3)
    y = uniform_ball(rng, M, 3)
    w = rng.standard_normal(N).astype(np.float32)
    xi = directions_fibonacci(P)
    return Problem("small_gauss", 3, "gauss", 0.5, P, n_ft, x, w, y, xi, radius(x, y))


def mnist_laplace(N: int = 60000, M: int = 60000, P: int = 2048, n_ft: int = 1024,
                  d: int = 784, seed: int = SEED_BASE + 2) -> Problem:
    """MNIST-shaped d=784 problem, Laplace kernel by the median rule."""
    rng = np.random.default_rng(seed)
    x = sparse_unit_cube(rng, N, d)
    y = sparse_unit_cube(rng, M, d)
    w = np.full(N, 1.0 / N, dtype=np.float32)
    med = median_pair_distance(x, y, 1000, seed + 1000)
    xi = directions_orthogonal(rng, P, d)
    return Problem("mnist_laplace", d, "laplace", 1.0 / med, P, n_ft, x, w, y, xi,
                   radius(x, y), meta={"median": med})


def gauss64_negdist(N: int = 200000, M: int = 200000, P: int = 4096, n_ft: int = 2048,
                    d: int = 64, seed: int = SEED_BASE + 3) -> Problem:
    """d=64 Gaussian clouds with the negative distance kernel, Sobol directions."""
    rng = np.random.default_rng(seed)
    x = gaussian(rng, N, d)
    y = gaussian(rng, M, d)
    w = rng.standard_normal(N).astype(np.float32)
    xi = directions_sobol(rng, P, d)
    return Problem("gauss64_negdist", d, "negdist", 0.0, P, n_ft, x, w, y, xi, radius(x, y))


def mmd_flow16(N: int = 100000, M: int = 100000, P: int = 1024, n_ft: int = 1024,
               d: int = 16, seed: int = SEED_BASE + 5) -> dict:
    """MMD-flow state: fixed targets x ~ N(0,I), moving particles y ~ U[-2,2]^d."""
    rng = np.random.default_rng(seed)
    x = gaussian(rng, N, d)
    y = uniform_box(rng, M, d, -2.0, 2.0)
    return {"x": x, "y": y, "d": d, "P": P, "n_ft": n_ft, "seed": seed}


def tiny(d: int, N: int, M: int, P: int, kernel: str, kparam: float, n_ft: int,
         seed: int, dirs: str = "iid", scale: float = 1.0, kparam2: float = 0.0) -> Problem:
    """Small random problem for unit and parity tests."""
    rng = np.random.default_rng(seed)
    x = gaussian(rng, N, d, scale)
    y = gaussian(rng, M, d, scale)
    w = rng.standard_normal(N).astype(np.float32)
    xi = make_directions(dirs, P, d, seed + 7)
    return Problem(f"tiny_d{d}", d, kernel, kparam, P, n_ft, x, w, y, xi, radius(x, y), kparam2=kparam2)


def mnist_matern(N: int = 60000, M: int = 60000, P: int = 2048, n_ft: int = 512, d: int = 784,
                 nu: float = 1.5, seed: int = SEED_BASE + 2) -> Problem:
    """The MNIST-shaped d=784 inputs with the Matern kernel (nu = 3/2 or 7/2, beta by the median
    rule, N_ft = 512 as for the paper's Matern runs)."""
    base = mnist_laplace(N, M, P, 1024, d, seed)
    med = base.meta["median"]
    return Problem(f"mnist_matern{int(2 * nu)}", d, "matern", med, P, n_ft, base.x, base.w, base.y, base.xi,
                   base.R, meta={"median": med}, kparam2=nu)


def repeat_directions(xi: np.ndarray, P: int, seed: int) -> np.ndarray:
    """A P x d direction array in which each of the U = len(xi) given rows
    appears exactly P / U times, in a seeded random order.

    The sliced sum averages over slices, so with equal multiplicities
    (1/P) sum_p t(xi_{pi(p)}) = (1/U) sum_j t(xi_j) exactly: a full-size run
    over P slices can be checked against a reference computed on the U
    distinct directions only.  The random order makes a slice-indexing error
    (a grid spread with one direction and read back with another) change the
    result."""
    U = xi.shape[0]
    if P % U:
        raise ValueError(f"P = {P} is not a multiple of the {U} distinct directions")
    order = np.random.default_rng(seed).permutation(np.repeat(np.arange(U), P // U))
    return np.ascontiguousarray(xi[order])


def batch256_problems(n: int = 256, seed: int = SEED_BASE + 3) -> list:
    """The batched workload: n Gauss problems, N, M log-uniform in [1e3, 1e5],
    d in {3, 16, 64}, N_ft in {256, 512, 1024}, P = 256 (spherical Fibonacci
    for d = 3, else orthogonal), sigma by the median rule (Sec. 4.1)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        N = int(np.exp(rng.uniform(np.log(1e3), np.log(1e5))))
        M = int(np.exp(rng.uniform(np.log(1e3), np.log(1e5))))
        d = int(rng.choice([3, 16, 64]))
        n_ft = int(rng.choice([256, 512, 1024]))
        x = gaussian(rng, N, d)
        y = gaussian(rng, M, d)
        w = rng.standard_normal(N).astype(np.float32)
        sigma = median_pair_distance(x, y, 1000, seed + 7 * i)
        xi = directions_fibonacci(256) if d == 3 else directions_orthogonal(rng, 256, d)
        out.append(Problem(f"batch{i}", d, "gauss", sigma, 256, n_ft, x, w, y, xi, radius(x, y)))
    return out


def pca_like(rng: np.random.Generator, n: int, d: int, decay: float = 0.5) -> np.ndarray:
    """Stand-in for PCA-reduced image data: independent coordinates
    N(0, j^(-2 decay)), j = 1..d (principal components of decaying variance)."""
    sd = np.arange(1, d + 1, dtype=np.float64) ** (-decay)
    return (rng.standard_normal((n, d)) * sd).astype(np.float32)


# N_ft per kernel as in the paper's experiments (App. C Step 2: 128 Gauss, 512
# Matern, 1024 Laplace); the negative distance takes the Laplace value
GPU_COMPARE_NFT = {"gauss": 128, "laplace": 1024, "matern": 512, "negdist": 1024}


def gpu_compare30(kernel: str = "laplace", N: int = 960000, P: int = 5120, d: int = 30,
                  seed: int = SEED_BASE + 6) -> Problem:
    """The GPU-comparison shape (App. H, "GPU Comparison"): d = 30, N = M = 960000,
    the data set summed against itself (y = x) with unit weights, kernel
    parameters by the median rule (Sec. 4.1), P = 5120 (the largest of the
    paper's P = 10 2^k), N_ft per kernel as above (Matern nu = 3/2).  The
    directions returned are the seeded orthogonal start; the paper's distance
    QMC design is formed from it by the library (QS_DIR_DISTANCE)."""
    rng = np.random.default_rng(seed)
    x = pca_like(rng, N, d)
    w = np.ones(N, dtype=np.float32)
    med = median_pair_distance(x, x, 1000, seed + 1000)
    kparam = {"gauss": med, "laplace": 1.0 / med, "matern": med, "negdist": 0.0}[kernel]
    xi = directions_orthogonal(rng, P, d)
    return Problem(f"gpu_compare30_{kernel}", d, kernel, kparam, P, GPU_COMPARE_NFT[kernel], x, w, x, xi,
                   radius(x, x), meta={"median": med}, kparam2=1.5 if kernel == "matern" else 0.0)
