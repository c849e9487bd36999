"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the FP64 oracle.

This module holds the *models* only (random matrices, the Bose-Hubbard dimer in its
Fock basis, Haar targets, drive parameters).  It contains none of the propagation
method's arithmetic: no Magnus coefficients, no commutators, no spectral bounds, no
Chebyshev/Bessel work.  Both sides receive the same host arrays from here and do
everything else on their own.

Random numbers come from a project-written splitmix64 counter generator (Steele,
Lea & Flood 2014, "Fast splittable pseudorandom number generators") followed by the
Box-Muller transform, so the streams are identical on every host and numpy version.

Models (paper §4 and §6):
  * random-matrix model: H0, H1 independent GOE(N) members, Eq. 13 with f = cos-type drive;
    normalisation (G + G^T)/sqrt(2N), G_ij ~ N(0, 1) (semicircle radius 2);
  * Bose-Hubbard dimer, Eq. 18 family: H = -J(a1^+ a2 + h.c.) + (U/2) sum n_i(n_i - 1)
    + f(t) (n1 - n2)/2 in the Fock basis |n, nb - n>, n = 0..nb (tridiagonal H0, diagonal H1);
    and the paper's own form, H = -v(a1^+ a2 + h.c.) + (U/2)(n1 - n2)^2 + f(t)(n2 - n1) with
    f = 2.7 + 2.5 cos 3t.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of the splitmix64 stream started at `seed`."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles strictly inside (0, 1): 53 random bits, centred in their cell."""
    z = splitmix64(seed, n, offset)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


def goe(n: int, seed: int) -> np.ndarray:
    """Real-symmetric GOE(n) member (G + G^T)/sqrt(2n), G_ij ~ N(0,1); float64, C order."""
    g = normal(seed, n * n).reshape(n, n)
    return np.ascontiguousarray((g + g.T) / math.sqrt(2.0 * n))


def ginibre(n: int, seed: int) -> np.ndarray:
    """Complex Ginibre matrix with i.i.d. N(0, 1/2) real and imaginary parts."""
    z = normal(seed, 2 * n * n).reshape(n, n, 2) / math.sqrt(2.0)
    return z[..., 0] + 1j * z[..., 1]


def haar_unitary(n: int, seed: int) -> np.ndarray:
    """Haar-distributed unitary: QR of a Ginibre matrix with the phases of R's diagonal
    moved into Q (Mezzadri 2007, "How to generate random matrices from the classical
    compact groups")."""
    q, r = np.linalg.qr(ginibre(n, seed))
    d = np.diagonal(r)
    return np.ascontiguousarray(q * (d / np.abs(d))[None, :])


@dataclasses.dataclass(frozen=True)
class Drive:
    """f(t) = f_dc + f_ac * cos(omega * t + phi0); one period is T = 2 pi / omega."""
    f_dc: float
    f_ac: float
    omega: float
    phi0: float = 0.0

    @property
    def period(self) -> float:
        return 2.0 * math.pi / self.omega


@dataclasses.dataclass
class DenseModel:
    """H(t) = H0 + f(t) H1 with dense real-symmetric H0, H1 (Eq. 13)."""
    h0: np.ndarray
    h1: np.ndarray
    drive: Drive
    steps: int

    @property
    def n(self) -> int:
        return self.h0.shape[0]


@dataclasses.dataclass
class TridiagModel:
    """H(t) = H0 + f(t) H1 with tridiagonal H0 (diag, sub/super-diagonal) and diagonal H1."""
    h0_diag: np.ndarray
    h0_off: np.ndarray   # H0[i+1, i] = H0[i, i+1], length n-1
    h1_diag: np.ndarray
    drive: Drive
    steps: int

    @property
    def n(self) -> int:
        return self.h0_diag.shape[0]

    def dense(self) -> tuple[np.ndarray, np.ndarray]:
        n = self.n
        h0 = np.diag(self.h0_diag) + np.diag(self.h0_off, -1) + np.diag(self.h0_off, 1)
        return h0, np.diag(self.h1_diag).astype(np.float64) + np.zeros((n, n))


def dimer_matrices(nb: int, J: float = 1.0, U: float | None = None):
    """Bose-Hubbard dimer with nb bosons in the Fock basis |n, nb-n>, n = 0..nb.

    H0 = -J (a1^+ a2 + a2^+ a1) + (U/2)[n1(n1-1) + n2(n2-1)], H1 = (n1 - n2)/2.
    U defaults to 2J/nb (U*nb/J = 2).  Returns (h0_diag, h0_off, h1_diag), float64.
    """
    if U is None:
        U = 2.0 * J / nb
    n = np.arange(nb + 1, dtype=np.float64)
    m = nb - n
    h0_diag = 0.5 * U * (n * (n - 1.0) + m * (m - 1.0))
    k = np.arange(nb, dtype=np.float64)
    h0_off = -J * np.sqrt((k + 1.0) * (nb - k))      # <n+1| a1^+ a2 |n>
    h1_diag = n - 0.5 * nb
    return h0_diag, h0_off, h1_diag


def dimer_matrices_paper(nb: int, v: float = 1.0, U: float | None = None):
    """The paper's dimer form (§4, its Eq. for H0 and H_mod) in the Fock basis |n, nb-n>:

    H0 = -v (a1^+ a2 + a1 a2^+) + (U/2)(n1 - n2)^2, H1 = H_mod = n2 - n1.
    U defaults to 2/nb (the interaction scaled with the boson number, U nb = 2).
    Returns (h0_diag, h0_off, h1_diag), float64.
    """
    if U is None:
        U = 2.0 / nb
    n = np.arange(nb + 1, dtype=np.float64)
    m = nb - n
    h0_diag = 0.5 * U * (n - m) ** 2
    k = np.arange(nb, dtype=np.float64)
    h0_off = -v * np.sqrt((k + 1.0) * (nb - k))
    h1_diag = m - n
    return h0_diag, h0_off, h1_diag


# ---------------------------------------------------------------- the five workloads
def config_goe64() -> DenseModel:
    """GOE N=64, seeds 1 (H0) and 2 (H1); f = cos t, T = 2 pi, M = 200 (plain FP64)."""
    return DenseModel(goe(64, 1), goe(64, 2), Drive(0.0, 1.0, 1.0), 200)


def config_dimer(nb: int = 10000, steps: int = 2000, U: float | None = None) -> TridiagModel:
    """Dimer with nb bosons (dim nb+1): J = 1, U nb/J = 2, eps0 = 0, eps1 = 1.5, omega = 3."""
    d, o, h1 = dimer_matrices(nb, 1.0, U)
    return TridiagModel(d, o, h1, Drive(0.0, 1.5, 3.0), steps)


def config_dimer_paper(nb: int = 10000, steps: int = 8000) -> TridiagModel:
    """The paper's dimer parameters (§7): v = 1, U nb = 2, f(t) = 2.7 + 2.5 cos(3 t)."""
    d, o, h1 = dimer_matrices_paper(nb)
    return TridiagModel(d, o, h1, Drive(2.7, 2.5, 3.0), steps)


def config_goe4096(n: int = 4096, steps: int = 512) -> DenseModel:
    """Dense GOE N=4096, seeds 3, 4; A = 2, omega = 2, M = 512."""
    return DenseModel(goe(n, 3), goe(n, 4), Drive(0.0, 2.0, 2.0), steps)


def config_goe_paper(n: int = 4096, steps: int = 100) -> DenseModel:
    """The paper's timing workload (§6, Table 1): GOE matrices with unit-variance entries
    (G + G^T)/sqrt(2), G_ij ~ N(0, 1), seeds 3 (H0) and 4 (H1); f(t) = cos(pi t), T = 2; M = 100
    steps per period (the runs also fix L = 50 Chebyshev products per step and use the 6th-order
    scheme; those are plan options)."""
    s = math.sqrt(n)  # goe() is normalised by sqrt(2 n); this undoes the sqrt(n) part
    return DenseModel(goe(n, 3) * s, goe(n, 4) * s, Drive(0.0, 1.0, math.pi), steps)


@dataclasses.dataclass(frozen=True)
class ScanInstance:
    n: int
    omega: float
    amplitude: float
    seed_h0: int
    seed_h1: int


def batch_scan(count: int = 48, seed: int = 5, n_lo: int = 256, n_hi: int = 2048):
    """Parameter scan: count instances, N ~ U{n_lo..n_hi}, omega ~ U[0.5, 4], A ~ U[0.5, 3].
    Instance i uses GOE seeds 1000 + 2i (H0) and 1001 + 2i (H1)."""
    u = uniform(seed, 3 * count).reshape(count, 3)
    out = []
    for i in range(count):
        n = n_lo + int(u[i, 0] * (n_hi - n_lo + 1))
        out.append(ScanInstance(min(n, n_hi), 0.5 + 3.5 * float(u[i, 1]),
                                0.5 + 2.5 * float(u[i, 2]), 1000 + 2 * i, 1001 + 2 * i))
    return out


def scan_model(inst: ScanInstance, steps: int = 256) -> DenseModel:
    return DenseModel(goe(inst.n, inst.seed_h0), goe(inst.n, inst.seed_h1),
                      Drive(0.0, inst.amplitude, inst.omega), steps)


@dataclasses.dataclass
class AdjointProblem:
    """Gate-fidelity problem: GOE H0, H1 (seeds 6, 7), Haar target W (seed 8),
    piecewise-constant amplitudes f_m ~ N(1, 0.1^2) (seed 9), T = 2 pi."""
    h0: np.ndarray
    h1: np.ndarray
    target: np.ndarray
    f: np.ndarray
    period: float


def config_adjoint(n: int = 1024, steps: int = 256) -> AdjointProblem:
    return AdjointProblem(goe(n, 6), goe(n, 7), haar_unitary(n, 8),
                          1.0 + 0.1 * normal(9, steps), 2.0 * math.pi)
