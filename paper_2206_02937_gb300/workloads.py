"""Seeded synthetic particle sets shaped like the paper's workloads.

Nothing here computes any part of the Compton step: these are the inputs that
both the CUDA path and the FP64 oracle receive.  Every generator draws from
``numpy.random.Generator(PCG64(seed + 1000))``.  Momenta are float32 in units
of m_e c, cells int32, identifiers uint32 (0..n-1 in generation order).

Workloads (sizes of the benchmark and the parity tests):
  * ``c1``  1D, 64 cells x (64 e + 64 photons); electrons gamma = 10,
            photons eps = 1e-3 m_e c^2, both isotropic; n = 1 (w/V = 1/64),
            dt = 0.05, seed 1.
  * ``c2``  2D nx x ny cells (512 x 512 at full size), cell counts
            floor(ppc n_c + U) with log-normal n_c = exp(0.5 z - 0.125) shared
            by both species; electrons Maxwell-Juttner theta = 1, photons
            Planck kT = 1e-2 m_e c^2, isotropic; dt = 0.05, seed 2.
  * ``c3``  surrogate samples: gamma log-uniform on [1, 1e3], eps
            log-uniform on [1e-4, 1], isotropic and independent.
  * ``c5``  3D cells x 16 per species; electrons dN/dgamma ~ gamma^-2 on
            [1, 1e4], photons a beam at 1e-2 m_e c^2 along +x.
The paper's own training and benchmark data are OSIRIS runs that are not
available; these generators stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed) + 1000))


def isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    """(3, n) unit vectors, uniform on the sphere."""
    mu = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return np.stack([s * np.cos(phi), s * np.sin(phi), mu])


def maxwell_juttner_u(rng: np.random.Generator, n: int, theta: float) -> np.ndarray:
    """|u| samples of the Maxwell-Juttner distribution by Sobol's rejection
    method (as described by Zenitani, Phys. Plasmas 22, 042116, 2015):
    u = -theta ln(X1 X2 X3), eta = -theta ln(X1 X2 X3 X4), accept if
    eta^2 - u^2 > 1."""
    out = np.empty(0)
    while out.size < n:
        m = int((n - out.size) * 1.6) + 64
        X = rng.uniform(0.0, 1.0, (4, m))
        X = np.where(X == 0.0, 1e-300, X)
        u = -theta * np.log(X[0] * X[1] * X[2])
        eta = -theta * np.log(X[0] * X[1] * X[2] * X[3])
        out = np.concatenate([out, u[eta * eta - u * u > 1.0]])
    return out[:n]


def planck_eps(rng: np.random.Generator, n: int, kT: float) -> np.ndarray:
    """Photon energies with density ~ eps^2 / (exp(eps/kT) - 1), by inverse
    interpolation of the cumulative on a fine FP64 table of y = eps/kT."""
    y = np.concatenate([np.linspace(1e-8, 1.0, 20001), np.linspace(1.0, 60.0, 200001)[1:]])
    f = y * y / np.expm1(y)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(y))])
    cdf /= cdf[-1]
    return kT * np.interp(rng.uniform(0.0, 1.0, n), cdf, y)


@dataclass
class Workload:
    name: str
    n_cells: int
    w_over_v: float
    dt: float
    seed: int
    steps: int
    e: dict = field(default_factory=dict)
    g: dict = field(default_factory=dict)

    @property
    def n_e(self) -> int:
        return int(self.e["ux"].shape[0])

    @property
    def n_g(self) -> int:
        return int(self.g["ux"].shape[0])


def _species(mom: np.ndarray, cell: np.ndarray) -> dict:
    mom = mom.astype(np.float32)
    return dict(ux=np.ascontiguousarray(mom[0]), uy=np.ascontiguousarray(mom[1]),
                uz=np.ascontiguousarray(mom[2]), cell=np.ascontiguousarray(cell.astype(np.int32)),
                id=np.arange(cell.shape[0], dtype=np.uint32))


def c1(seed: int = 1) -> Workload:
    rng = rng_for(seed)
    C, ppc = 64, 64
    cell = np.repeat(np.arange(C), ppc)
    ue = np.sqrt(10.0 ** 2 - 1.0) * isotropic(rng, C * ppc)
    kg = 1e-3 * isotropic(rng, C * ppc)
    return Workload("c1: 1D 64 cells x 64+64, gamma=10 e, 1e-3 photons", C, 1.0 / ppc, 0.05, seed, 1,
                    _species(ue, cell), _species(kg, cell))


def lognormal_counts(rng: np.random.Generator, n_cells: int, ppc: int, sigma: float = 0.5) -> np.ndarray:
    z = rng.standard_normal(n_cells)
    n_c = np.exp(sigma * z - 0.5 * sigma * sigma)
    return np.floor(ppc * n_c + rng.uniform(0.0, 1.0, n_cells)).astype(np.int64)


def c2(nx: int = 512, ny: int = 512, ppc: int = 64, seed: int = 2, shuffle: bool = True) -> Workload:
    rng = rng_for(seed)
    C = nx * ny
    counts = lognormal_counts(rng, C, ppc)
    cell = np.repeat(np.arange(C), counts)
    n = cell.shape[0]
    ue = maxwell_juttner_u(rng, n, 1.0) * isotropic(rng, n)
    kg = planck_eps(rng, n, 1e-2) * isotropic(rng, n)
    ce, cg = cell.copy(), cell.copy()
    if shuffle:
        pe, pg = rng.permutation(n), rng.permutation(n)
        ue, ce = ue[:, pe], ce[pe]
        kg, cg = kg[:, pg], cg[pg]
    return Workload(f"c2: 2D {nx}x{ny} cells, log-normal ppc {ppc}, MJ theta=1 e, Planck kT=1e-2", C,
                    1.0 / ppc, 0.05, seed, 100, _species(ue, ce), _species(kg, cg))


def c3(n: int, seed: int = 3) -> tuple[np.ndarray, np.ndarray]:
    """(u, k), each (3, n) float32."""
    rng = rng_for(seed)
    gamma = 10.0 ** rng.uniform(0.0, 3.0, n)
    eps = 10.0 ** rng.uniform(-4.0, 0.0, n)
    u = np.sqrt(np.maximum(gamma * gamma - 1.0, 0.0)) * isotropic(rng, n)
    k = eps * isotropic(rng, n)
    return u.astype(np.float32), k.astype(np.float32)


def c5(n_side: int = 256, ppc: int = 16, seed: int = 5) -> Workload:
    rng = rng_for(seed)
    C = n_side ** 3
    n = C * ppc
    cell = np.repeat(np.arange(C), ppc)
    gamma = 1.0 / (1.0 - rng.uniform(0.0, 1.0, n) * (1.0 - 1e-4))
    ue = np.sqrt(np.maximum(gamma * gamma - 1.0, 0.0)) * isotropic(rng, n)
    kg = np.zeros((3, n))
    kg[0] = 1e-2
    return Workload(f"c5: 3D {n_side}^3 cells x {ppc}, power-law e, +x photon beam", C, 1.0 / ppc, 0.05,
                    seed, 20, _species(ue, cell), _species(kg, cell))


def waterbag(rng, n: int, p0: float) -> np.ndarray:
    """(3, n) momenta of an isotropic waterbag: uniform in the ball |p| <= p0
    (Sec. 3.2 writes f(p) = n0 H(p + p0); read as H(p0 - |p|), the form that
    confines the momenta)."""
    r = p0 * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    return r * isotropic(rng, n)


def waterbag_pairs(n: int, p0: float, seed: int = 25) -> tuple[np.ndarray, np.ndarray]:
    """Training pairs of one transfer-learning stage: electrons and photons
    both from the waterbag of radius p0 (the plasmas of Sec. 3.2's
    training simulations), float32 (3, n) each."""
    rng = rng_for(seed)
    return waterbag(rng, n, p0).astype(np.float32), waterbag(rng, n, p0).astype(np.float32)


def inverse_compton(p_e: float, eps: float = 2.5, n_cells: int = 512, ppc: int = 128, seed: int = 60,
                    dt: float = 0.05) -> Workload:
    """The inverse-Compton benchmark of Sec. 3.3: a monoenergetic electron
    beam (momentum p_e along +x) crossing a monoenergetic isotropic photon gas
    (energy eps), ppc of each species in every one of n_cells 1D cells,
    density 1 (w/V = 1/ppc)."""
    rng = rng_for(seed)
    n = n_cells * ppc
    cell = np.repeat(np.arange(n_cells), ppc)
    ue = np.zeros((3, n))
    ue[0] = p_e
    kg = eps * isotropic(rng, n)
    return Workload(f"inverse Compton: p_e {p_e} beam on an isotropic eps {eps} photon gas", n_cells, 1.0 / ppc,
                    dt, seed, 1, _species(ue, cell), _species(kg, cell))


def pair_arrays(w: Workload) -> tuple[np.ndarray, np.ndarray]:
    """The (3, n) momentum arrays of a workload's species (no pairing)."""
    u = np.stack([w.e["ux"], w.e["uy"], w.e["uz"]])
    k = np.stack([w.g["ux"], w.g["uy"], w.g["uz"]])
    return u, k
