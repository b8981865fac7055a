"""Seeded synthetic lysosomes shaped like the paper's workloads.

The paper (Sec. II.1, III.1) models a lysosome as a sphere holding
monodisperse NPs of diameter d at volume concentration c, placed at random
without overlap, with random easy axes. This module builds such inputs:

* radius R = (d/2) (n/c)^(1/3), so that n d^3 / (8 R^3) = c;
* centres by random sequential addition (RSA): uniform candidates inside the
  sphere of radius R - d/2, each kept iff it lies at least d from every centre
  kept before it;
* easy axes uniform on the unit sphere;
* or, the paper's own choice (Sec. II.4), the nodes of a simple-cubic lattice
  of cell a = d (pi / 6c)^(1/3) nearest the centre, as mean positions for
  the disorder drawn loop by loop (at most (a - d)/2, so no two overlap);
* centres snapped to the float32 grid in units of d about the lysosome centre
  (the origin), so that the float32 copy held by the GPU path is the same
  geometry as the float64 copy held by the oracle (a shift of at most 3e-8 d
  for R = 50 d); snap=False keeps them as drawn.

It holds no step of the kinetic Monte-Carlo method; both the oracle and the
CUDA path take its output as input. Random numbers come from numpy's PCG64
seeded by the caller.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

@dataclasses.dataclass
class Lysosome:
    pos: np.ndarray      # (n, 3) centres, m
    axis: np.ndarray     # (n, 3) unit easy axes
    vol: np.ndarray      # (n,) magnetic volumes, m^3
    Ms: float            # A/m
    Keff: float          # J/m^3
    T: float             # K
    tau0: float          # s
    rho: float = 5200.0  # kg/m^3, magnetite (Sec. III.2.a)
    d: float = 0.0       # diameter, m
    radius: float = 0.0  # lysosome radius, m
    c: float = 0.0       # volume concentration

    @property
    def n(self) -> int:
        return int(self.vol.shape[0])


def sphere_volume(d):
    return math.pi * d ** 3 / 6.0


def lysosome_radius(n, d, c):
    """Radius of the sphere holding n spheres of diameter d at concentration c."""
    return 0.5 * d * (n / c) ** (1.0 / 3.0)


def random_axes(n, rng):
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def _uniform_in_ball(k, radius, rng):
    out = np.empty((0, 3))
    while out.shape[0] < k:
        p = rng.uniform(-radius, radius, size=(2 * k + 16, 3))
        p = p[np.einsum("ij,ij->i", p, p) <= radius * radius]
        out = np.concatenate([out, p])
    return out[:k]


def rsa_positions(n, d, radius, rng, max_batches=100000):
    """Random sequential addition of n non-overlapping spheres of diameter d
    whose centres lie within radius - d/2 of the origin. Candidates are drawn
    in batches and accepted in draw order, which is the sequential rule."""
    from scipy.spatial import cKDTree

    rin = radius - 0.5 * d
    if rin <= 0 and n > 1:
        raise ValueError("lysosome too small for its NPs")
    dd = d * (1.0 + 2e-6)  # keep the snapped centres at least d apart
    acc = np.empty((0, 3))
    tree = None
    for _ in range(max_batches):
        need = n - acc.shape[0]
        if need <= 0:
            break
        cand = _uniform_in_ball(min(max(need * 2, 64), 50000), rin, rng)
        if tree is not None:
            dist, _ = tree.query(cand, k=1, distance_upper_bound=dd)
            cand = cand[~np.isfinite(dist) | (dist >= dd)]
        if cand.shape[0] == 0:
            continue
        ok = np.ones(cand.shape[0], dtype=bool)
        pairs = cKDTree(cand).query_pairs(dd, output_type="ndarray")
        if pairs.size:
            partners = {}
            for a, b in pairs:
                a, b = (a, b) if a < b else (b, a)
                partners.setdefault(b, []).append(a)
            for b in sorted(partners):
                if any(ok[a] for a in partners[b]):
                    ok[b] = False
        cand = cand[ok][:need]
        acc = np.concatenate([acc, cand])
        tree = cKDTree(acc)
    if acc.shape[0] < n:
        raise RuntimeError("RSA did not place %d spheres" % n)
    return acc


def snap_to_float32(pos, d):
    """Round centres to the float32 grid in units of d about the origin."""
    v = (np.asarray(pos, dtype=np.float64) / d).astype(np.float32)
    return v.astype(np.float64) * d


def make_lysosome(n, d, c, Ms=1e6, Keff=1.3e4, T=300.0, tau0=1e-10, seed=0,
                  rho=5200.0, snap=True):
    """One synthetic lysosome: n NPs of diameter d (m) at concentration c.
    snap=False keeps the centres as drawn (float64), so that the float32 frame
    of the GPU path rounds them as it would a caller's positions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    R = lysosome_radius(n, d, c)
    pos = rsa_positions(n, d, R, rng) if n > 0 else np.zeros((0, 3))
    if snap:
        pos = snap_to_float32(pos, d)
    axis = random_axes(n, rng)
    vol = np.full(n, sphere_volume(d))
    return Lysosome(pos=pos, axis=axis, vol=vol, Ms=float(Ms), Keff=float(Keff),
                    T=float(T), tau0=float(tau0), rho=float(rho), d=float(d),
                    radius=float(R), c=float(c))


def lattice_spacing(d, c):
    """Edge of the simple-cubic cell holding one sphere of diameter d at volume
    concentration c: a^3 c = pi d^3 / 6."""
    return d * (math.pi / (6.0 * c)) ** (1.0 / 3.0)


def max_disorder(d, c):
    """Largest displacement that keeps two neighbouring NPs of a simple-cubic
    lattice from overlapping: each may move (a - d) / 2 towards the other
    (Sec. II.4: the disorder is as large as possible without overlap)."""
    return 0.5 * (lattice_spacing(d, c) - d)


def lattice_nodes_lysosome(n, d, c, Ms=1e6, Keff=1.3e4, T=300.0, tau0=1e-10, seed=0,
                           rho=5200.0):
    """The paper's own placement (Sec. II.4): the n nodes of the simple-cubic
    lattice of spacing lattice_spacing(d, c) nearest the centre (a node sits
    at the origin; ties by grid order), random easy axes. The nodes are the
    mean positions around which the disorder is drawn, loop by loop."""
    if not 0.0 < c < math.pi / 6.0:
        raise ValueError("a simple-cubic lattice holds at most pi/6 of the volume")
    a = lattice_spacing(d, c)
    h = int(math.ceil((0.75 * n / math.pi) ** (1.0 / 3.0))) + 2
    g = np.arange(-h, h + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    r2 = np.einsum("ij,ij->i", p, p)
    pos = p[np.argsort(r2, kind="stable")[:n]] * a
    rng = np.random.Generator(np.random.PCG64(seed))
    return Lysosome(pos=pos, axis=random_axes(n, rng), vol=np.full(n, sphere_volume(d)),
                    Ms=float(Ms), Keff=float(Keff), T=float(T), tau0=float(tau0), rho=float(rho),
                    d=float(d), radius=float(lysosome_radius(n, d, c)), c=float(c))


def lattice_lysosome(n_side, spacing, d, Ms=1e6, Keff=1.3e4, T=300.0, tau0=1e-10):
    """Cubic-lattice sphere (no disorder) centred on a lattice site: every site
    within (n_side/2) spacings of the centre. Used for symmetry checks."""
    h = n_side // 2
    g = np.arange(-h, h + 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    p = p[np.einsum("ij,ij->i", p, p) <= h * h]
    pos = p * spacing
    n = pos.shape[0]
    axis = np.tile([0.0, 0.0, 1.0], (n, 1))
    vol = np.full(n, sphere_volume(d))
    return Lysosome(pos=pos, axis=axis, vol=vol, Ms=Ms, Keff=Keff, T=T, tau0=tau0, d=d,
                    radius=float(h * spacing), c=0.0)


def replicate(lys, k):
    """k copies of one lysosome (independent random streams by lysosome index)."""
    return [dataclasses.replace(lys) for _ in range(k)]


# ---------------------------------------------------------------------------
# The paper-shaped workloads. Each returns (lysosomes, run parameters).

def config_small(seed=0):
    """One lysosome of 100 NPs, d = 12 nm, M_S = 1e6 A/m, K_eff = 1.3e4 J/m^3,
    T = 300 K, tau0 = 1e-10 s, 5 % volume concentration; field along z,
    mu0 H_max = 20 mT, f = 100 kHz, 200 steps per period, 20 periods of which
    the first 5 are discarded."""
    lys = make_lysosome(100, 12e-9, 0.05, Ms=1e6, Keff=1.3e4, T=300.0, tau0=1e-10,
                        seed=seed)
    run = dict(mu0Hmax=0.020, f=1e5, S=200, periods=20, discard=5, seed=seed)
    return [lys], run


def config_single2000(replicas=8, seed=0, snap=True):
    """A lysosome of 2000 NPs, d = 14 nm, K_eff = 2e4 J/m^3, 10 % volume
    concentration, otherwise as the 100-NP case; `replicas` copies run as
    independent random streams (the seeds of the kMC draws)."""
    lys = make_lysosome(2000, 14e-9, 0.10, Ms=1e6, Keff=2e4, T=300.0, tau0=1e-10,
                        seed=seed, snap=snap)
    run = dict(mu0Hmax=0.020, f=1e5, S=200, periods=20, discard=5, seed=seed)
    return replicate(lys, replicas), run


def config_sweep8000(c=0.05, mu0Hmax=0.040, seed=0):
    """A lysosome of 8000 NPs, d = 12 nm, K_eff = 1.3e4 J/m^3 at concentration c
    in {1, 2, 5, 10, 20} %, mu0 H_max in {10, 20, 40, 60} mT, f = 100 kHz,
    500 steps per period, 20 periods (5 discarded)."""
    lys = make_lysosome(8000, 12e-9, c, Ms=1e6, Keff=1.3e4, T=300.0, tau0=1e-10,
                        seed=seed)
    run = dict(mu0Hmax=mu0Hmax, f=1e5, S=500, periods=20, discard=5, seed=seed)
    return [lys], run


def config_batched(n_lys=512, seed=0, sigma_ln=0.5):
    """A batch of lysosomes with lognormal NP counts (median 1500, sigma of the
    log 0.5) clipped to [200, 10000], d ~ U[8, 20] nm, K_eff ~ U[1e4, 5e4]
    J/m^3, c ~ U[1, 20] %, mu0 H_max ~ U{10, ..., 80} mT, f = 100 kHz,
    200 steps per period, 20 periods (5 discarded), T = 300 K."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.clip(np.round(1500.0 * np.exp(sigma_ln * rng.standard_normal(n_lys))), 200,
                 10000).astype(int)
    ds = rng.uniform(8e-9, 20e-9, n_lys)
    Ks = rng.uniform(1e4, 5e4, n_lys)
    cs = rng.uniform(0.01, 0.20, n_lys)
    Hs = rng.integers(10, 81, n_lys) * 1e-3
    lys = [make_lysosome(int(ns[q]), float(ds[q]), float(cs[q]), Ms=1e6, Keff=float(Ks[q]),
                         T=300.0, tau0=1e-10, seed=seed * 100003 + q + 1)
           for q in range(n_lys)]
    run = dict(mu0Hmax=Hs, f=1e5, S=200, periods=20, discard=5, seed=seed)
    return lys, run


def config_large50000(seed=0, snap=True):
    """A lysosome of 50000 NPs, d = 16 nm, K_eff = 3e4 J/m^3, 10 % volume
    concentration, mu0 H_max = 40 mT, f = 100 kHz, 500 steps per period,
    50 periods (5 discarded)."""
    lys = make_lysosome(50000, 16e-9, 0.10, Ms=1e6, Keff=3e4, T=300.0, tau0=1e-10,
                        seed=seed, snap=snap)
    run = dict(mu0Hmax=0.040, f=1e5, S=500, periods=50, discard=5, seed=seed)
    return [lys], run
