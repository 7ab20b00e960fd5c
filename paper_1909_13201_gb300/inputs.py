"""Seeded synthetic problem generator for the linearised FSI system.

This module is the one piece shared by the CUDA path and the FP64 oracle.  It
draws the *problem data* only -- geometry (material of every fine element),
coefficients, the frozen Oseen advection field at the fine Q2 nodes and the
right-hand side in a mesh-natural layout -- and holds none of the solver's
arithmetic (no numbering, no assembly, no transfer, no smoother).

The paper's geometries (2D/3D aneurysms and a venous valve, Sec. 4.1-4.2) are
hybrid meshes that are not available; the generators below stand in for them
with the same structure: a solid wall band of 10-40% of the width, an
aneurysm-like fluid pocket cut into the wall, and thin valve-like leaflets.

Natural layouts (a convention shared by the generators, the oracle and the library tests):
  * element e of an n^dim grid on [0,1]^dim: e = i + n*j (+ n*n*k), x fastest;
  * Q2 node of index (p, q, r), 0 <= p,q,r <= 2n, at (p, q, r) * h/2, flat
    index p + (2n+1)*q (+ (2n+1)^2*r);
  * Q1 node (p, q, r), 0 <= p,q,r <= n, at (p, q, r) * h;
  * a vector in natural layout is a dict with arrays
      d: (dim, NQ2), v: (dim, NQ2), p: (2, NQ1)   (p[0] solid copy, p[1] fluid copy).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 13201

BC_CHANNEL_2D = 0   # solid clamped on x=0, x=1, y=0; fluid v=0 on x=0, y=0, y=1; do-nothing x=1
BC_BOX_3D = 1       # d = v = 0 on every face except x=1 (do-nothing)


@dataclass
class Problem:
    """One linearised FSI system (Sec. 2.2 weak form, linearised at d = 0)."""
    dim: int
    n_fine: int                 # fine elements per direction
    n_levels: int               # GMG levels, coarse n = n_fine / 2**(n_levels-1)
    patch: int                  # Vanka group edge b: b^dim pressure vertices per block
    material: np.ndarray        # uint8, n_fine**dim, 1 = solid, 0 = fluid
    advection: np.ndarray       # float64, (dim, NQ2_fine), frozen Oseen velocity w
    mu_s: float
    lambda_s: float
    rho_s: float
    rho_f: float
    mu_f: float
    dt: float
    bc_preset: int
    seed: int
    name: str = ""
    meta: dict = field(default_factory=dict)
    omega: float = 1.0          # Richardson damping recommended for this workload

    @property
    def n_q2(self) -> int:
        return (2 * self.n_fine + 1) ** self.dim

    @property
    def n_q1(self) -> int:
        return (self.n_fine + 1) ** self.dim


def _lex_coords(dim: int, m: int) -> list[np.ndarray]:
    """Integer coordinates (i, j[, k]) of an m^dim lattice in flat lex order, x fastest."""
    idx = np.arange(m ** dim)
    return [(idx // m ** a) % m for a in range(dim)]


def _element_centroids(dim: int, n: int) -> list[np.ndarray]:
    return [(c + 0.5) / n for c in _lex_coords(dim, n)]


def _q2_coords(dim: int, n: int) -> list[np.ndarray]:
    return [c / (2.0 * n) for c in _lex_coords(dim, 2 * n + 1)]


def _advection_2d(rng: np.random.Generator, n: int) -> np.ndarray:
    # stream function psi = sum_{k,l=1..4} a_kl sin(k pi x) sin(l pi y),
    # a_kl ~ N(0,1)/(k^2+l^2); w = (d psi/dy, -d psi/dx), max |w| = 1 at nodes.
    x, y = _q2_coords(2, n)
    a = rng.standard_normal((4, 4))
    wx = np.zeros_like(x)
    wy = np.zeros_like(x)
    for k in range(1, 5):
        for l in range(1, 5):
            c = a[k - 1, l - 1] / (k * k + l * l)
            wx += c * l * math.pi * np.sin(k * math.pi * x) * np.cos(l * math.pi * y)
            wy -= c * k * math.pi * np.cos(k * math.pi * x) * np.sin(l * math.pi * y)
    w = np.stack([wx, wy])
    return w / np.sqrt((w * w).sum(0)).max()


def _advection_3d(rng: np.random.Generator, n: int) -> np.ndarray:
    # w = curl A, A_i = sum_{k,l,m=1..3} a^i_klm sin(k pi x) sin(l pi y) sin(m pi z)/(k^2+l^2+m^2)
    x, y, z = _q2_coords(3, n)
    a = rng.standard_normal((3, 3, 3, 3))
    pi = math.pi
    # grad of each potential component
    dA = np.zeros((3, 3, x.size))  # dA[i, j] = d A_i / d x_j
    for i in range(3):
        for k in range(1, 4):
            sx, cx = np.sin(k * pi * x), np.cos(k * pi * x)
            for l in range(1, 4):
                sy, cy = np.sin(l * pi * y), np.cos(l * pi * y)
                for m in range(1, 4):
                    sz, cz = np.sin(m * pi * z), np.cos(m * pi * z)
                    c = a[i, k - 1, l - 1, m - 1] / (k * k + l * l + m * m)
                    dA[i, 0] += c * k * pi * cx * sy * sz
                    dA[i, 1] += c * l * pi * sx * cy * sz
                    dA[i, 2] += c * m * pi * sx * sy * cz
    w = np.stack([dA[2, 1] - dA[1, 2], dA[0, 2] - dA[2, 0], dA[1, 0] - dA[0, 1]])
    return w / np.sqrt((w * w).sum(0)).max()


def _band(dim: int, n: int, width: float) -> np.ndarray:
    c = _element_centroids(dim, n)
    return (c[1] < width).astype(np.uint8)


def make_channel_2d(n_fine: int, n_levels: int, patch: int, seed: int, *,
                    band_width: float = 0.25, bulge: bool = False,
                    mu_s: float | None = None, mu_s_range=(1e1, 1e3),
                    mu_f: float | None = None, mu_f_range=(1e-3, 1e-1),
                    dt: float = 1e-2, name: str = "") -> Problem:
    """2D channel on [0,1]^2 with a solid wall band y < band_width.

    Draw order: geometry, coefficients, advection.
    bulge=True cuts an aneurysm-like elliptic fluid pocket into the wall:
    centre (xc ~ U[0.3,0.7], band_width), semi-axes (0.2, 0.2 s), s ~ U[0.5,1].
    """
    rng = np.random.default_rng(seed)
    mat = _band(2, n_fine, band_width)
    meta = {"band_width": band_width}
    if bulge:
        xc = rng.uniform(0.3, 0.7)
        s = rng.uniform(0.5, 1.0)
        cx, cy = _element_centroids(2, n_fine)
        inside = ((cx - xc) / 0.2) ** 2 + ((cy - band_width) / (0.2 * s)) ** 2 < 1.0
        mat[inside] = 0
        meta.update(bulge_xc=xc, bulge_s=s)
    if mu_s is None:
        mu_s = float(math.exp(rng.uniform(math.log(mu_s_range[0]), math.log(mu_s_range[1]))))
    if mu_f is None:
        mu_f = float(math.exp(rng.uniform(math.log(mu_f_range[0]), math.log(mu_f_range[1]))))
    w = _advection_2d(rng, n_fine)
    return Problem(dim=2, n_fine=n_fine, n_levels=n_levels, patch=patch, material=mat,
                   advection=w, mu_s=mu_s, lambda_s=4.0 * mu_s, rho_s=1.0, rho_f=1.0,
                   mu_f=mu_f, dt=dt, bc_preset=BC_CHANNEL_2D, seed=seed, name=name, meta=meta)


def make_valve_3d(n_fine: int, n_levels: int, patch: int, seed: int, *,
                  mu_s: float = 1e2, mu_f: float = 3.5e-3, dt: float = 1e-2,
                  name: str = "") -> Problem:
    """3D box [0,1]^3 with two thin valve-like leaflet slabs rooted at y = 0.

    Slab i: |x - x_i| < 1/n_fine (two elements thick), y < h_i, all z;
    x_i ~ U[0.3, 0.7], h_i ~ U[0.4, 0.6].  Draw order: geometry, advection.
    """
    rng = np.random.default_rng(seed)
    cx, cy, _ = _element_centroids(3, n_fine)
    mat = np.zeros(n_fine ** 3, np.uint8)
    slabs = []
    for _ in range(2):
        x0 = rng.uniform(0.3, 0.7)
        h = rng.uniform(0.4, 0.6)
        mat[(np.abs(cx - x0) < 1.0 / n_fine) & (cy < h)] = 1
        slabs.append((x0, h))
    w = _advection_3d(rng, n_fine)
    # omega = 0.7: in 3D a velocity dof lies in up to 8 vertex-centred Vanka
    # blocks (weight 1/8) while its block's pressure has weight 1; undamped
    # additive smoothing over-corrects the interface pressures and diverges
    return Problem(dim=3, n_fine=n_fine, n_levels=n_levels, patch=patch, material=mat,
                   advection=w, mu_s=mu_s, lambda_s=4.0 * mu_s, rho_s=1.0, rho_f=1.0,
                   mu_f=mu_f, dt=dt, bc_preset=BC_BOX_3D, seed=seed, name=name,
                   meta={"slabs": slabs}, omega=0.7)


def make_config(k: int) -> Problem | list[Problem]:
    """The five workloads: 0 small 2D parity case, 1 2D 256^2 channel with
    bulge, 2 3D 32^3 valve box, 3 a batch of 64 uneven 2D systems, 4 2D 128^2
    differentiation case."""
    seed = BASE_SEED + k
    if k == 0:
        return make_channel_2d(16, 3, 1, seed, band_width=0.25, mu_s=1e2, mu_f=1e-2,
                               name="channel2d-16x16-L3")
    if k == 1:
        return make_channel_2d(256, 7, 3, seed, bulge=True, mu_f=1e-2,
                               name="channel2d-bulge-256x256-L7")
    if k == 2:
        return make_valve_3d(32, 4, 1, seed, name="valve3d-32x32x32-L4")
    if k == 3:
        return make_batch(64)
    if k == 4:
        return make_channel_2d(128, 6, 3, seed, bulge=True, mu_f=1e-2,
                               name="channel2d-bulge-128x128-L6")
    raise ValueError(k)


# coarse sizes for the batched workload: fine n -> (coarse n, levels)
BATCH_LEVELS = {32: 4, 48: 4, 64: 5, 96: 5, 128: 6}


def make_batch(count: int = 64, sizes=(32, 48, 64, 96, 128)) -> list[Problem]:
    """Independent 2D channels of uneven size and wall thickness.

    mu_s ~ log-U[1e2, 1e3]: the wall stays elasticity-dominated, as in the
    paper's vessel walls (rho_s L^2 / (mu_s dt^2) <= 1e2 here, ~1e-6 there);
    much softer synthetic walls make the additive field split diverge on
    coarse levels (the inertial d-u coupling it drops dominates).
    mu_f ~ log-U[1e-3, 1e-1]."""
    probs = []
    for i in range(count):
        seed = BASE_SEED * 100 + i
        rng = np.random.default_rng(seed)
        n = int(rng.choice(sizes))
        width = float(rng.uniform(0.1, 0.4))
        sub = int(rng.integers(0, 2**31 - 1))
        probs.append(make_channel_2d(n, BATCH_LEVELS[n], 3, sub, band_width=width, mu_s_range=(1e2, 1e3),
                                     name=f"batch{i}-{n}x{n}"))
    return probs


def natural_vector(prob: Problem, seed: int) -> dict:
    """Seeded N(0,1) vector in the natural layout (d, v at Q2 nodes, two
    pressure copies at Q1 nodes).  Used for right-hand sides b and adjoint
    weights w_J; entries of pressure copies that do not exist are ignored."""
    rng = np.random.default_rng(seed)
    return {
        "d": rng.standard_normal((prob.dim, prob.n_q2)),
        "v": rng.standard_normal((prob.dim, prob.n_q2)),
        "p": rng.standard_normal((2, prob.n_q1)),
    }


def gather_natural(nat: dict, field_: np.ndarray, comp: np.ndarray, node: np.ndarray) -> np.ndarray:
    """Pick the entries of a natural-layout vector named by a dof map
    (field 0 = d, 1 = v, 2 = p; comp = component or pressure copy; node = Q2
    or Q1 node).  Pure indexing, shared by both sides' callers."""
    out = np.empty(field_.size)
    for f, key in enumerate(("d", "v", "p")):
        m = field_ == f
        out[m] = nat[key][comp[m], node[m]]
    return out
