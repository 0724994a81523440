"""Seeded synthetic inputs for the cell-list force evaluation.

This module only *constructs inputs*: flows (A, L0, M, T), strain times and
particle positions.  It holds none of the method's arithmetic (no lattice
evolution kernel, no wrapping, no cell assignment, no forces); both the CUDA
path and the CPU oracle read what it produces, and neither is imported here.

Inputs follow the paper's problem statement: a lattice L = [v1 v2 v3] whose
columns are the lattice vectors (Sec. 2), a linear flow u(x) = A x with
L_t = exp(tA) L0 (Sec. 2.1, Eq. for dL/dt), and the Kraynik-Reinelt
condition exp(A t*) L0 = L0 M with M in SL(3,Z) (Sec. 2.2, Eq. kr).

Construction of the KR flows.  For a symmetric M in SL(3,Z) with distinct
positive eigenvalues lambda_k and orthonormal eigenvectors V, the flow
A = V diag(ln lambda_k) V^T / T with a cubic L0 = s I satisfies the KR
condition exactly: exp(T A) L0 = s V diag(lambda) V^T = L0 M.  Particles are
placed affinely with the flow: q(t) = F(tau) L0 s_fcc + delta, where
F(tau) = V diag(lambda^(tau/T)) V^T is the deformation this construction
prescribes, s_fcc are ideal face-centred-cubic fractional sites and delta is a
fixed i.i.d. Gaussian displacement per particle.  The density is preserved
because det F = 1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# The two remapping matrices of the planar and general 3D flows.
M_PLANAR = np.array([[2, 1, 0], [1, 1, 0], [0, 0, 1]], dtype=np.int64)
M_GENERAL = np.array([[3, 2, 1], [2, 2, 1], [1, 1, 1]], dtype=np.int64)
M_IDENTITY = np.eye(3, dtype=np.int64)
M_SHEAR = np.array([[1, 1, 0], [0, 1, 0], [0, 0, 1]], dtype=np.int64)

RHO_DEFAULT = 0.8442
DISPLACEMENT_STD = 0.05
WCA_RC = 2.0 ** (1.0 / 6.0)
LJ_RC = 2.5

POT_LJ = 0
POT_WCA = 1


@dataclasses.dataclass
class Workload:
    """One force-evaluation input: flow, time, positions and potential."""

    name: str
    A: np.ndarray          # (3,3) float64 flow matrix
    L0: np.ndarray         # (3,3) float64, columns are lattice vectors
    M: np.ndarray          # (3,3) int64 remapping matrix, det 1
    T: float               # period of the KR remap
    t: float               # evaluation time
    q: np.ndarray          # (N,3) float64 Cartesian positions, any image
    kind: int = POT_LJ     # POT_LJ or POT_WCA
    rc: float = LJ_RC
    eps: float = 1.0
    sigma: float = 1.0
    shift: int = 1         # energy shifted to zero at rc
    remap: int = 0         # 0: tau = t mod T in [0, T); 1: centred, tau in [-T/2, T/2)

    @property
    def n(self) -> int:
        return int(self.q.shape[0])


def fcc_fractional(k: int) -> np.ndarray:
    """Ideal FCC sites of k^3 conventional cells in the unit cube, shape (4k^3, 3)."""
    basis = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.arange(k, dtype=np.float64)
    cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
    corners = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    sites = (corners[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    return sites / float(k)


def kr_flow(M: np.ndarray, T: float = 1.0):
    """Flow construction for a symmetric M: returns (A, V, lam).

    A = V diag(ln lam) V^T / T.  V has orthonormal columns sorted by eigenvalue.
    """
    Mf = np.asarray(M, dtype=np.float64)
    if not np.allclose(Mf, Mf.T):
        raise ValueError("kr_flow builds flows for symmetric M only")
    lam, V = np.linalg.eigh(Mf)
    if np.any(lam <= 0):
        raise ValueError("M must be positive definite")
    A = (V * (np.log(lam) / T)) @ V.T
    A = 0.5 * (A + A.T)
    return A, V, lam


def _deformation(V, lam, tau, T):
    return (V * (lam ** (tau / T))) @ V.T


def perturbed_fcc(k: int, rho: float, rng: np.random.Generator, *, vacancies: int = 0,
                  std: float = DISPLACEMENT_STD):
    """Fractional FCC sites (with optional random vacancies), box side and displacements."""
    s = fcc_fractional(k)
    if vacancies:
        keep = np.sort(rng.permutation(s.shape[0])[: s.shape[0] - vacancies])
        s = s[keep]
    n = s.shape[0]
    side = (n / rho) ** (1.0 / 3.0)
    delta = rng.normal(0.0, std, size=(n, 3))
    return s, side, delta


def _finish(name, A, L0, M, T, t, s, delta, F, rng, kind, rc, shuffle=True):
    q = (F @ (L0 @ s.T)).T + delta
    if shuffle:
        q = q[rng.permutation(q.shape[0])]
    return Workload(name=name, A=A, L0=L0, M=M, T=T, t=t, q=np.ascontiguousarray(q),
                    kind=kind, rc=rc)


def config_equilibrium_wca(k: int = 10, seed: int = 0) -> Workload:
    """Plain WCA system at rest: N = 4k^3, cubic box at density 0.8442, A = 0, t = 0."""
    rng = np.random.default_rng(seed)
    s, side, delta = perturbed_fcc(k, RHO_DEFAULT, rng)
    L0 = side * np.eye(3)
    return _finish(f"wca_eq_N{s.shape[0]}", np.zeros((3, 3)), L0, M_IDENTITY.copy(), 1.0, 0.0,
                   s, delta, np.eye(3), rng, POT_WCA, WCA_RC)


class StrainSeries:
    """One perturbed FCC system under the KR flow of a symmetric M, at any time t.

    The sites, displacements and particle order are drawn once from the seed;
    positions(t) places them affinely for the flow at time t.  rate scales the
    strain rate: A = rate * V diag(ln lam) V^T / T, period T / rate.
    """

    def __init__(self, M, k, seed, *, T=1.0, rho=RHO_DEFAULT, kind=POT_LJ, rc=None, rate=1.0,
                 vacancies=0, name=None):
        rng = np.random.default_rng(seed)
        self.s, side, self.delta = perturbed_fcc(k, rho, rng, vacancies=vacancies)
        self.period = T / rate
        self.A, self.V, self.lam = kr_flow(M, self.period)
        self.L0 = side * np.eye(3)
        self.M = np.asarray(M, dtype=np.int64).copy()
        self.order = rng.permutation(self.s.shape[0])
        self.kind = kind
        self.rc = (WCA_RC if kind == POT_WCA else LJ_RC) if rc is None else rc
        self.name = name or f"kr_N{self.s.shape[0]}"
        self._sL = self.s @ self.L0.T

    @property
    def n(self):
        return int(self.s.shape[0])

    def positions(self, t):
        tau = t - self.period * math.floor(t / self.period)
        F = _deformation(self.V, self.lam, tau, self.period)
        q = self._sL @ F.T + self.delta
        return np.ascontiguousarray(q[self.order])

    def workload(self, t, name=None):
        return Workload(name=name or f"{self.name}_t{t:.6g}", A=self.A, L0=self.L0, M=self.M,
                        T=self.period, t=t, q=self.positions(t), kind=self.kind, rc=self.rc)


def config_flow(M: np.ndarray, k: int, t: float, seed: int, *, T: float = 1.0,
                rho: float = RHO_DEFAULT, kind: int = POT_LJ, rc: float | None = None,
                rate: float = 1.0, vacancies: int = 0, name: str | None = None) -> Workload:
    """Perturbed FCC under the KR flow of a symmetric M, evaluated at time t."""
    ser = StrainSeries(M, k, seed, T=T, rho=rho, kind=kind, rc=rc, rate=rate, vacancies=vacancies)
    return ser.workload(t, name=name or f"kr_N{ser.n}_t{t:.6g}")


def general_series(k: int = 64, seed: int = 4) -> StrainSeries:
    """General 3D flow (M = [[3,2,1],[2,2,1],[1,1,1]]) on N = 4k^3 LJ particles, rc = 2.5.

    k = 64 gives the N = 1,048,576 system, k = 40 the N = 256,000 one.
    """
    return StrainSeries(M_GENERAL, k, seed, name=f"general_N{4 * k ** 3}")


def general_series_2m(seed: int = 5) -> StrainSeries:
    """General 3D flow on N = 2,097,152 = 2^21 LJ particles, rc = 2.5: an FCC block
    of 81^3 cells (2,125,764 sites) with 28,612 random vacancies."""
    n = 1 << 21
    return StrainSeries(M_GENERAL, 81, seed, vacancies=4 * 81 ** 3 - n, name=f"general_N{n}")


def planar_series(k: int = 20, seed: int = 1) -> StrainSeries:
    return StrainSeries(M_PLANAR, k, seed, name=f"planar_N{4 * k ** 3}")


def config_planar(i: int = 0, nstrain: int = 64, k: int = 20, seed: int = 1) -> Workload:
    """Planar elongational flow, N = 4k^3 (32000 at k = 20), LJ rc = 2.5, t = i / nstrain."""
    return config_flow(M_PLANAR, k, i / nstrain, seed, name=f"planar_N{4 * k ** 3}_i{i}")


def config_general(i: int = 0, nstrain: int = 128, k: int = 40, seed: int = 2,
                   t: float | None = None) -> Workload:
    """General 3D flow, N = 4k^3 (256000 at k = 40), LJ rc = 2.5, t = i / nstrain."""
    tt = i / nstrain if t is None else t
    return config_flow(M_GENERAL, k, tt, seed, name=f"general_N{4 * k ** 3}_t{tt:.6g}")


NEAR_REMAP_T = 1.0 - 2.0 ** -20


class ShearSeries:
    """Lees-Edwards shear (Sec. 2.2) of a cubic perturbed-FCC box of side a: the
    flow u = rate y e_x, A = rate e_x e_y^T, one period T = 1 / rate tilts the box
    by one lattice spacing (exp(T A) L0 = L0 M with M = [[1,1,0],[0,1,0],[0,0,1]]),
    and the remap is taken half way (tau in [-T/2, T/2)), so the tilt never
    exceeds half a spacing.  Positions at time t are the affine image
    (I + tau A) L0 s + delta of the seeded sites.
    """

    def __init__(self, k, seed, *, rate=1.0, rho=RHO_DEFAULT, kind=POT_LJ, rc=None, name=None):
        rng = np.random.default_rng(seed)
        self.s, side, self.delta = perturbed_fcc(k, rho, rng)
        self.A = np.zeros((3, 3))
        self.A[0, 1] = rate
        self.period = 1.0 / rate
        self.L0 = side * np.eye(3)
        self.M = M_SHEAR.copy()
        self.order = rng.permutation(self.s.shape[0])
        self.kind = kind
        self.rc = (WCA_RC if kind == POT_WCA else LJ_RC) if rc is None else rc
        self.name = name or f"shear_N{self.s.shape[0]}"
        self._sL = self.s @ self.L0.T

    @property
    def n(self):
        return int(self.s.shape[0])

    def positions(self, t):
        tau = t - self.period * math.floor(t / self.period + 0.5)
        F = np.eye(3)
        F[0, 1] = tau * self.A[0, 1]
        q = self._sL @ F.T + self.delta
        return np.ascontiguousarray(q[self.order])

    def workload(self, t, name=None):
        return Workload(name=name or f"{self.name}_t{t:.6g}", A=self.A, L0=self.L0, M=self.M, T=self.period,
                        t=t, q=self.positions(t), kind=self.kind, rc=self.rc, remap=1)


def equilibrium_set(k: int = 64, nconf: int = 16, seed: int = 7) -> list:
    """nconf independently perturbed FCC cubes of N = 4k^3 LJ particles at rest (A = 0)."""
    out = []
    for c in range(nconf):
        rng = np.random.default_rng(seed + 1000 * c)
        s, side, delta = perturbed_fcc(k, RHO_DEFAULT, rng)
        L0 = side * np.eye(3)
        q = (s @ L0.T + delta)[rng.permutation(s.shape[0])]
        out.append(Workload(name=f"eq_N{s.shape[0]}_c{c}", A=np.zeros((3, 3)), L0=L0, M=M_IDENTITY.copy(), T=1.0,
                            t=0.0, q=np.ascontiguousarray(q), kind=POT_LJ, rc=LJ_RC))
    return out


def shear_series(k: int = 20, seed: int = 6, rate: float = 1.0) -> ShearSeries:
    """Lees-Edwards shear on N = 4k^3 LJ particles (32000 at k = 20, 1,048,576 at k = 64)."""
    return ShearSeries(k, seed, rate=rate)


def batched_systems(nsys: int = 256, seed: int = 3, nmin: int = 1000, nmax: int = 20000):
    """Independent replicas of uneven N and different flows.

    N ~ U[nmin, nmax]; FCC with kc = ceil((N/4)^(1/3)) cells and 4 kc^3 - N random
    vacancies; density ~ U(0.8, 0.9); flow planar or general (coin flip) at a
    strain rate ~ U(0.5, 2) and phase t ~ U[0, period); WCA or LJ rc = 2.5.
    """
    rng = np.random.default_rng(seed)
    out = []
    for s_idx in range(nsys):
        n = int(rng.integers(nmin, nmax + 1))
        kc = int(math.ceil((n / 4.0) ** (1.0 / 3.0) - 1e-12))
        vac = 4 * kc ** 3 - n
        rho = float(rng.uniform(0.8, 0.9))
        M = M_PLANAR if rng.random() < 0.5 else M_GENERAL
        rate = float(rng.uniform(0.5, 2.0))
        period = 1.0 / rate
        t = float(rng.uniform(0.0, period))
        kind = POT_WCA if rng.random() < 0.5 else POT_LJ
        sub_seed = int(rng.integers(0, 2 ** 31 - 1))
        out.append(config_flow(M, kc, t, sub_seed, rho=rho, kind=kind, rate=rate,
                               vacancies=vac, name=f"batch{s_idx}_N{n}"))
    return out


def maxwell_momenta(n: int, kT: float, seed: int) -> np.ndarray:
    """(n, 3) float64 momenta of unit-mass particles drawn from N(0, kT) per
    component (seeded), with the mean removed (zero total momentum)."""
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, math.sqrt(kT), size=(n, 3))
    return np.ascontiguousarray(p - p.mean(axis=0))


def uniform_random(n: int, L: np.ndarray, seed: int, rc: float = LJ_RC,
                   kind: int = POT_LJ) -> Workload:
    """Uniform random points in a static box L (A = 0), for statistical checks."""
    rng = np.random.default_rng(seed)
    s = rng.random((n, 3))
    q = (np.asarray(L, dtype=np.float64) @ s.T).T
    return Workload(name=f"uniform_N{n}", A=np.zeros((3, 3)), L0=np.asarray(L, dtype=np.float64),
                    M=M_IDENTITY.copy(), T=1.0, t=0.0, q=np.ascontiguousarray(q), kind=kind, rc=rc)


def random_sl3z(rng: np.random.Generator, steps: int = 6) -> np.ndarray:
    """A random unimodular integer matrix built from elementary row operations."""
    M = np.eye(3, dtype=np.int64)
    for _ in range(steps):
        a, b = rng.choice(3, size=2, replace=False)
        c = int(rng.choice([-1, 1]))
        E = np.eye(3, dtype=np.int64)
        E[a, b] = c
        M = M @ E
    return M


def small_random_box(rng: np.random.Generator, n: int, rc: float, hmin: float = 1.0,
                     hmax: float = 3.5):
    """A random skewed triclinic box whose heights lie in [hmin*rc, hmax*rc], plus points.

    Used for brute-force pair-set checks on tiny inputs, including boxes with
    one or two cells per direction.
    """
    for _ in range(1000):
        L = rng.normal(size=(3, 3))
        if np.linalg.det(L) < 0:
            L[:, 0] = -L[:, 0]
        Linv = np.linalg.inv(L)
        h = 1.0 / np.linalg.norm(Linv, axis=1)
        target = rng.uniform(hmin, hmax, size=3) * rc
        L = L @ np.diag(target / h)
        Linv = np.linalg.inv(L)
        h = 1.0 / np.linalg.norm(Linv, axis=1)
        if np.all(h >= hmin * rc * 1.0001):
            s = rng.random((n, 3))
            q = (L @ s.T).T + rng.normal(0, 0.5, size=(n, 3))
            return L, np.ascontiguousarray(q)
    raise RuntimeError("could not build a random box")
