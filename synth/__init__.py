"""Seeded synthetic workloads shared by the oracle and the CUDA library.

This module holds no arithmetic of the SU(2) method itself.  It only fixes
*inputs*: the configurations, the number of kept multiplets per bond sector
(an input recipe, not part of the paper's algorithm) and the Gaussian trial
wavefunctions.  Both the oracle and the library consume what it returns.

Configurations follow the workloads of the hot path (two-site H.psi inside
Davidson, Eq. 2 of the paper):

* ``heis12``   open spin-1/2 Heisenberg chain, L=12, J=1, S=0, D=32.
* ``qc16``     synthetic ab initio skeleton, L=N=16, S=0, D=512.
* ``qc32``     L=N=32, S=0, D=2048.
* ``qc48``     L=N=48, S=0, D=4096 (the batching workload).
* ``qc64``     L=N=64, S=0, D=6144.

Bond-sector recipe (input, not method): at a bond with ``k`` sites on one
side, sectors q=(N_q, 2S_q) get a weight
``w_q = exp(-(N_q - Nbar)^2/(2*0.8^2)) * exp(-S_q(S_q+1)/(2*1.5^2))``
with ``Nbar = k*N/L`` (the particle weight is dropped for spin chains).
``D`` multiplets are apportioned by weight, each sector capped by the number
of multiplets the previous bond can feed into it (which equals the
Weyl-Paldus count when nothing was truncated), with largest-remainder
rounding so that the kept dimensions sum to ``min(D, total cap)``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

SPIN_HALF = 0        # one state per site: N=1, 2S=1
SPATIAL_ORBITAL = 1  # three states per site: |0>, |sigma>, |2>


@dataclass(frozen=True)
class Config:
    name: str
    site_kind: int
    L: int
    N: int
    twoS: int
    D: int
    seed: int

    @property
    def n_left(self) -> int:
        """Sites in the left block at the middle two-site bond."""
        return self.L // 2 - 1

    @property
    def n_right(self) -> int:
        return self.L - self.n_left - 2


CONFIGS = {
    "heis12": Config("heis12", SPIN_HALF, 12, 12, 0, 32, 1001),
    "qc16": Config("qc16", SPATIAL_ORBITAL, 16, 16, 0, 512, 1002),
    "qc32": Config("qc32", SPATIAL_ORBITAL, 32, 32, 0, 2048, 1003),
    "qc48": Config("qc48", SPATIAL_ORBITAL, 48, 48, 0, 4096, 1004),
    "qc64": Config("qc64", SPATIAL_ORBITAL, 64, 64, 0, 6144, 1005),
    # profiling case: the sector-dimension mix of qc32 at a few GB of device memory
    "qc20p": Config("qc20p", SPATIAL_ORBITAL, 20, 20, 0, 1536, 1007),
}


def site_states(site_kind: int):
    """(N, 2S) of the site multiplets in canonical order."""
    if site_kind == SPIN_HALF:
        return [(1, 1)]
    return [(0, 0), (1, 1), (2, 0)]


def weyl_paldus(k: int, n: int, twoS: int) -> int:
    """Number of spin-S multiplets of n electrons in k orbitals."""
    if n < 0 or n > 2 * k or (n - twoS) % 2 or twoS < 0:
        return 0
    a = (n - twoS) // 2
    b = k - (n + twoS) // 2
    if a < 0 or b < 0:
        return 0
    num = (twoS + 1) * math.comb(k + 1, a) * math.comb(k + 1, b)
    assert num % (k + 1) == 0
    return num // (k + 1)


def spin_chain_mult(k: int, twoS: int) -> int:
    """Number of spin-S multiplets of k spin-1/2 sites."""
    if (k - twoS) % 2 or twoS > k or twoS < 0:
        return 0
    a = (k - twoS) // 2
    return math.comb(k, a) - (math.comb(k, a - 1) if a >= 1 else 0)


def _apportion(caps, weights, D):
    """Water-fill D over sectors by weight, capped, with largest remainder."""
    n = len(caps)
    total_cap = sum(caps)
    if total_cap <= D:
        return list(caps)
    # continuous solution a_q = min(cap_q, lam * w_q), sum a_q = D
    lo, hi = 0.0, 1.0
    while sum(min(c, hi * w) for c, w in zip(caps, weights)) < D:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if sum(min(c, mid * w) for c, w in zip(caps, weights)) < D:
            lo = mid
        else:
            hi = mid
    a = [min(c, hi * w) for c, w in zip(caps, weights)]
    d = [min(c, int(math.floor(x))) for c, x in zip(caps, a)]
    rest = D - sum(d)
    order = sorted(range(n), key=lambda i: (-(a[i] - math.floor(a[i])), i))
    i = 0
    while rest > 0:
        q = order[i % n]
        if d[q] < caps[q]:
            d[q] += 1
            rest -= 1
        i += 1
    return d


def _couple(twoA: int, twoB: int):
    return range(abs(twoA - twoB), twoA + twoB + 1, 2)


def bond_sector_chain(cfg: Config, k_max: int):
    """Kept sectors [(N, 2S, d), ...] at bonds with k = 0..k_max sites.

    Bond k is reached from bond k-1 by adding one site; the cap of a sector
    is the number of (sector, site state) products at bond k-1 that couple
    into it.  Sectors with d=0 are dropped.  Order: ascending (N, 2S).
    """
    sites = site_states(cfg.site_kind)
    chain = [[(0, 0, 1)]]
    for k in range(1, k_max + 1):
        caps = {}
        for (n0, s0, d0) in chain[-1]:
            for (ns, ss) in sites:
                for s in _couple(s0, ss):
                    key = (n0 + ns, s)
                    caps[key] = caps.get(key, 0) + d0
        keys = sorted(caps)
        nbar = k * cfg.N / cfg.L
        w = []
        for (n, s) in keys:
            S = s / 2.0
            ws = math.exp(-S * (S + 1) / (2 * 1.5 ** 2))
            if cfg.site_kind == SPATIAL_ORBITAL:
                ws *= math.exp(-((n - nbar) ** 2) / (2 * 0.8 ** 2))
            w.append(ws)
        d = _apportion([caps[q] for q in keys], w, cfg.D)
        chain.append([(n, s, dq) for (n, s), dq in zip(keys, d) if dq > 0])
    return chain


def middle_bond_sectors(cfg: Config):
    """(left sectors, right sectors) of the middle two-site bond."""
    left = bond_sector_chain(cfg, cfg.n_left)[cfg.n_left]
    right = bond_sector_chain(cfg, cfg.n_right)[cfg.n_right]
    return left, right


def gaussian_psi(n: int, seed: int) -> np.ndarray:
    """Seeded N(0,1) vector of length n normalised to unit 2-norm."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n)
    nrm = np.linalg.norm(x)
    return x / nrm if nrm > 0 else x


def psi_seed(cfg: Config) -> int:
    return cfg.seed + 100


N_CHOLESKY = 32


def integrals(L: int, seed: int):
    """Seeded synthetic ab initio integrals (h, (ij|kl)) of L orbitals.

    Draws, in this order, from ``numpy.random.default_rng(seed)``: g (L x L
    standard normal, row-major), u (L values uniform in [-2, 0)), then for
    r = 0..31 the upper triangle i <= j of z^r (standard normal, row-major).
    h_ij = (g_ij + g_ji)/2 * exp(-|i-j|/4) off the diagonal, h_ii = u_i;
    B^r_ij = B^r_ji = 0.1 z^r_ij exp(-|i-j|/4) (standard deviation 0.1 times
    the decay); (ij|kl) = sum_r B^r_ij B^r_kl (chemists' notation: 8-fold
    symmetric and positive semidefinite as an (ij) x (kl) matrix).  No core
    energy.  Returns (h, eri) with eri[i, j, k, l] = (ij|kl).
    """
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((L, L))
    u = rng.uniform(-2.0, 0.0, L)
    iu = np.triu_indices(L)
    z = [rng.standard_normal(len(iu[0])) for _ in range(N_CHOLESKY)]
    i, j = np.indices((L, L))
    decay = np.exp(-np.abs(i - j) / 4.0)
    h = 0.5 * (g + g.T) * decay
    h[np.diag_indices(L)] = u
    B = np.zeros((N_CHOLESKY, L, L))
    for r in range(N_CHOLESKY):
        B[r][iu] = z[r]
        B[r] = np.triu(B[r]) + np.triu(B[r], 1).T
        B[r] *= 0.1 * decay
    eri = np.einsum("rij,rkl->ijkl", B, B)
    return h, eri
