"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the butterfly method.  It only draws the
random numbers that both sides consume (input vectors g, sampled output sets S,
request streams) and names the workloads by their sizes, so that the CPU oracle
and the GPU path are fed bit-identical inputs without sharing any code.

Workload recipes (sizes, kernels, seeds) follow the problem statement of
Li, Yang and Ying, "Multidimensional Butterfly Factorization", §1.1 (eq. for
u(x)=sum K(x,xi) g(xi), point sets X and Omega) and the numerical sections
§3.3 / §4.3 (error estimated on a random sample of output points).
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict

import numpy as np

__all__ = [
    "complex_normal",
    "sample_outputs",
    "Workload",
    "WORKLOADS",
    "request_stream",
]


def complex_normal(n_points: int, nrhs: int = 1, seed: int = 0) -> np.ndarray:
    """g = (a + i b)/sqrt(2), a, b iid N(0,1); shape [nrhs, n_points], complex128.

    E|g|^2 = 1.  Drawn with numpy's PCG64 (`default_rng(seed)`), real parts for all
    entries first, then imaginary parts.
    """
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((nrhs, n_points))
    b = rng.standard_normal((nrhs, n_points))
    return (a + 1j * b) / np.sqrt(2.0)


def sample_outputs(n_points: int, m: int, seed: int = 1) -> np.ndarray:
    """m distinct output indices (natural X order), drawn without replacement, sorted."""
    rng = np.random.default_rng(seed)
    m = min(m, n_points)
    return np.sort(rng.choice(n_points, size=m, replace=False)).astype(np.int64)


@dataclass(frozen=True)
class Workload:
    """A named problem: kernel family, grid size n per axis, dimension, tree depth L,
    maximum rank r, right-hand-side count and the Omega-tree transform."""

    name: str
    kernel: str          # "dft" | "fio_iso" | "fio_ellip"
    dim: int
    n: int
    L: int
    r: int
    nrhs: int
    transform: str = "none"   # "none" | "polar" | "multiscale"
    n_sample: int = 0        # 0: full direct check, else |S|
    seed_g: int = 0
    seed_s: int = 1
    seed_build: int = 7

    @property
    def N(self) -> int:
        return self.n ** self.dim

    def as_dict(self):
        d = asdict(self)
        d["N"] = self.N
        return d


WORKLOADS = {
    # 2-D DFT, n=64, quadtree depth 4 (4x4-point leaves), rank 16, one RHS.
    "dft2_n64_L4_r16": Workload("dft2_n64_L4_r16", "dft", 2, 64, 4, 16, 1),
    # 2-D FIO with isotropic phase x.xi + c(x)|xi|, polar tree on Omega,
    # n=256, depth 6, rank 24; one and 64 RHS; 256 sampled outputs.
    "fio2_polar_n256_L6_r24": Workload("fio2_polar_n256_L6_r24", "fio_iso", 2, 256, 6, 24, 1,
                                        "polar", 256),
    "fio2_polar_n256_L6_r24_x64": Workload("fio2_polar_n256_L6_r24_x64", "fio_iso", 2, 256, 6, 24,
                                            64, "polar", 256),
    # Large 2-D FIO, polar, n=1024, depth 10, rank 24, 16 RHS; 512 sampled outputs.
    "fio2_polar_n1024_L10_r24_x16": Workload("fio2_polar_n1024_L10_r24_x16", "fio_iso", 2, 1024,
                                              10, 24, 16, "polar", 512),
    # 3-D DFT, n=64, octree depth 6 (1-point leaves), rank 32, 32 RHS.
    "dft3_n64_L6_r32_x32": Workload("dft3_n64_L6_r32_x32", "dft", 3, 64, 6, 32, 32, "none", 256),
    # Small cases used by the parity tests (several tiles, ragged polar leaves).
    "dft2_n16_L2_r8": Workload("dft2_n16_L2_r8", "dft", 2, 16, 2, 8, 1),
    "fio2_polar_n32_L4_r12": Workload("fio2_polar_n32_L4_r12", "fio_iso", 2, 32, 4, 12, 1, "polar"),
    "fio2_polar_n64_L4_r24": Workload("fio2_polar_n64_L4_r24", "fio_iso", 2, 64, 4, 24, 1, "polar"),
    "dft3_n8_L2_r16": Workload("dft3_n8_L2_r16", "dft", 3, 8, 2, 16, 1),
    # Further operators of the served mix (2x2- and 4x4-point leaves).
    "dft2_n128_L6_r16": Workload("dft2_n128_L6_r16", "dft", 2, 128, 6, 16, 1),
    "fio2_polar_n128_L6_r24": Workload("fio2_polar_n128_L6_r24", "fio_iso", 2, 128, 6, 24, 1, "polar"),
    "dft2_n256_L6_r16": Workload("dft2_n256_L6_r16", "dft", 2, 256, 6, 16, 1),
}

# The served mix: six resident operators, requests drawn uniformly over them.
SERVE_MIX = ["dft2_n64_L4_r16", "fio2_polar_n64_L4_r24", "dft2_n128_L6_r16", "fio2_polar_n128_L6_r24",
             "dft2_n256_L6_r16", "fio2_polar_n256_L6_r24"]


def request_stream(n_requests: int, operators: list[str], rate_hz: float, max_rhs: int = 32,
                   seed: int = 2):
    """A seeded serving workload: for each request, (arrival time s, operator name, nrhs).

    Operators are drawn uniformly, RHS counts uniformly in 1..max_rhs, inter-arrival
    times exponential with mean 1/rate_hz (Poisson arrivals)."""
    rng = np.random.default_rng(seed)
    ops = rng.integers(0, len(operators), size=n_requests)
    rhs = rng.integers(1, max_rhs + 1, size=n_requests)
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    return [(float(t[k]), operators[int(ops[k])], int(rhs[k])) for k in range(n_requests)]
