"""FP64 CPU oracle of a Verlet neighbour list with a skin, reused across steps.

TEST INFRASTRUCTURE ONLY: tests use it; the product path never does.

The paper rebuilds the cell list at every step (Sec. 4.1).  The standard next
stage, which the paper does not treat, keeps a list of the pairs within
rc + skin, built from one evaluation of the exact pair definition, and at the
following steps evaluates only the listed pairs, until a pair outside the
list could have come within rc.  Under the flow this needs two things the
equilibrium list does not:

* images: particles are wrapped into the unit cell of L(t) at every step, so a
  listed pair (i, j, n) of the build is the pair (i, j, n + m_j - m_i) at time
  t, m_i the lattice vector the wrap has moved particle i by since the build
  (the fractional coordinates of a particle change only by its peculiar
  displacement, so m_i is the integer nearest to s_i(build) - s_i(t));
* deformation: between remaps L(t) = exp(A (t - t_b)) L(t_b), which stretches
  or compresses every displacement d_b of the build to F d_b with
  d|F d_b|^2/dt = 2 (F d_b)^T A (F d_b) >= 2 mu |F d_b|^2, mu the smallest
  eigenvalue of the symmetric part (A + A^T)/2, so |F d_b| >=
  exp(mu (t - t_b)) |d_b| (mu <= 0 for an incompressible flow).  A pair not in
  the list had |d_b| >= rc + skin, so at time t it is at least
  exp(mu (t - t_b)) (rc + skin) - 2 delta away, delta the largest peculiar
  displacement |L(t) u_i| since the build.  The list is rebuilt when that
  bound falls below rc, and at every remap (L jumps to L M^-1, and the images
  of the list no longer mean the same lattice vectors).

Pairs are decided by the canonical expression of the force oracle (Sec. 2:
d = (q'_j - q'_i) + L n with q' = L frac(L^-1 q), r^2 < rc^2), evaluated in
the same order, so the list's pair set at a step is the brute-force set
whenever the rebuild rule is right.
"""
from __future__ import annotations

import math

import numpy as np

from . import brute, wrap


def _canon_r2(qp, L, i, j, n):
    """r^2 of pairs (i, j, n) in the force oracle's operation order (no fused
    multiply-add: numpy rounds every operation)."""
    f = n.astype(np.float64)
    img = (f[:, 0:1] * L[:, 0][None, :] + f[:, 1:2] * L[:, 1][None, :]) + f[:, 2:3] * L[:, 2][None, :]
    d = (qp[j] - qp[i]) + img
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


class SkinList:
    """Pairs within rc + skin at a build; pairs within rc at later times."""

    def __init__(self, rc, skin, A):
        self.rc = float(rc)
        self.skin = float(skin)
        A = np.asarray(A, dtype=np.float64)
        # slowest contraction rate of the flow: the smallest eigenvalue of (A + A^T)/2
        self.mu = min(float(np.linalg.eigvalsh(0.5 * (A + A.T)).min()), 0.0)
        self.pairs = None
        self.builds = 0

    def build(self, L, Linv, q, t):
        s, qp = wrap(L, Linv, q)
        r = brute(L, s, qp, self.rc + self.skin, want_pairs=True)
        self.pairs = np.asarray(r.pairs, dtype=np.int64).reshape(-1, 5)
        self.sb = s
        self.tb = float(t)
        self.builds += 1

    def _images(self, L, Linv, q):
        s, qp = wrap(L, Linv, q)
        m = np.rint(self.sb - s).astype(np.int64)
        return s, qp, m

    def displacement(self, L, Linv, q):
        """Largest peculiar displacement |L(t) u_i| since the build."""
        s, _, m = self._images(L, Linv, q)
        u = s + m - self.sb
        return float(np.sqrt(((u @ L.T) ** 2).sum(axis=1)).max()) if len(s) else 0.0

    def must_rebuild(self, L, Linv, q, t, remapped):
        if self.pairs is None or remapped:
            return True
        sigma = math.exp(self.mu * (float(t) - self.tb))
        return sigma * (self.rc + self.skin) - 2.0 * self.displacement(L, Linv, q) < self.rc * (1.0 + 1e-12)

    def pairs_at(self, L, Linv, q):
        """Listed pairs within rc at positions q (any image), as (i, j, n) rows in
        the oracle's canonical orientation."""
        _, qp, m = self._images(L, Linv, q)
        p = self.pairs
        i, j = p[:, 0], p[:, 1]
        n = p[:, 2:5] + m[j] - m[i]
        keep = _canon_r2(qp, L, i, j, n) < self.rc * self.rc
        return np.concatenate([p[keep, 0:2], n[keep]], axis=1)


def period_index(t, T, centered=False):
    """Which period the time t falls in (the remap happens between periods)."""
    return math.floor(t / T + (0.5 if centered else 0.0))
