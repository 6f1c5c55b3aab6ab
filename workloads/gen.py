"""Seeded synthetic workloads standing in for the paper's Geant4/SHiP inputs.

The paper builds its (material, momentum-bin) histograms from Geant4 runs of
N = 5e6 muons per bin through a slab of thickness d (Sec. "Building
histograms"), uses 95 log10 momentum bins on 0.18-400 GeV (Sec. "Validation
and benchmarking") and a Snoopy finite-element field map of the SHiP muon
shield.  None of that data exists here, so this module makes seeded
stand-ins with the same shapes and structure:

* histograms: per sample, a Moyal ionisation loss with PDG thin-absorber
  width/most-probable value, a 1/v^2 radiative tail whose mean matches
  b*rho*x, and a Highland-width Rayleigh space angle with a 1 % single-scatter
  1/theta^3 tail; binned on linear axes f = dp/p in [0, f_max) and
  theta in [0, 5*theta0(p_i)) with theta0 taken at the bin's lower edge;
* geometries: an iron block in air, and a shield-like layout of six iron
  magnet blocks with alternating fields plus a concrete wall;
* a smooth node-based field map (tanh-edged blocks with small fringe
  components, all three components non-zero somewhere);
* muon spectra: log-uniform or p^-2.7 momenta with Gaussian/exponential p_T.

Material constants are approximate; they shape the histograms but play no
part in any parity check (the same arrays feed both sides).
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import hashlib
import inspect
import json
import os
from typing import Dict, List, Optional

import numpy as np

# --------------------------------------------------------------------------
# physical constants (PDG), MeV / cm units inside the histogram fixture
# --------------------------------------------------------------------------
_K = 0.307075           # MeV cm^2 / g
_ME = 0.51099895        # MeV
_MMU = 105.6583755      # MeV

# rho [g/cm^3], Z/A, I [MeV], X0 [cm], b [g^-1 cm^2] (radiative loss coefficient)
MATERIALS: Dict[str, Dict[str, float]] = {
    "iron":     dict(rho=7.874, ZA=0.46557, I=286.0e-6, X0=1.757, b=3.5e-6),
    "air":      dict(rho=1.205e-3, ZA=0.49919, I=85.7e-6, X0=30390.0, b=3.0e-6),
    "concrete": dict(rho=2.300, ZA=0.50274, I=135.2e-6, X0=11.55, b=3.0e-6),
    "lead":     dict(rho=11.35, ZA=0.39575, I=823.0e-6, X0=0.5612, b=6.0e-6),
}

# generated histogram sets are cached in the repository's _build/ folder (a build
# product, not source), or where MT_WORKLOAD_CACHE points
_CACHE_DIR = os.environ.get(
    "MT_WORKLOAD_CACHE", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_build",
                                      "workload_cache"))


def _cache_path(tag: str, params: dict) -> str:
    key = hashlib.sha1(json.dumps(params, sort_keys=True).encode()).hexdigest()[:16]
    return os.path.join(_CACHE_DIR, f"{tag}_{key}.npz")


def pbin_edges(p_lo: float, p_hi: float, n_pbin: int) -> np.ndarray:
    """Log-spaced momentum-bin edges p_k = p_lo (p_hi/p_lo)^(k/N), k = 0..N."""
    k = np.arange(n_pbin + 1, dtype=np.float64)
    return p_lo * (p_hi / p_lo) ** (k / n_pbin)


def _highland(p_gev: np.ndarray, x_cm: float, X0: float) -> np.ndarray:
    """Highland multiple-scattering width theta0 [rad] for a unit-charge muon."""
    p = p_gev * 1e3
    E = np.sqrt(p * p + _MMU * _MMU)
    beta = p / E
    t = x_cm / X0
    return 13.6 / (beta * p) * np.sqrt(t) * (1.0 + 0.038 * np.log(t))


LOG_F_RANGE = (1e-10, 1.0)      # -dPz/P axis of the log-axes histograms
LOG_T_RANGE = (1e-9, 1.0)       # dPt/P axis


def _hist_one(rng: np.random.Generator, mat: Dict[str, float], p_a: float, p_b: float,
              x_cm: float, f_max: float, nf: int, ntheta: int, n_samples: int, axes: str = "linear"):
    """One (material, momentum-bin) histogram of counts [nf][ntheta] plus its theta axis.

    axes = "linear": f = dp/p on [0, f_max), theta on [0, 5 theta0(p_lo)).
    axes = "log": the paper's variables -dPz/P = 1 - (1-f) cos(theta) and
    dPt/P = (1-f) sin(theta), log-spaced on LOG_F_RANGE and LOG_T_RANGE."""
    p = rng.uniform(p_a, p_b, n_samples)                     # GeV, Pz ~ U(p_i, p_i+1)
    pm = p * 1e3
    E = np.sqrt(pm * pm + _MMU * _MMU)
    beta2 = (pm / E) ** 2
    bg = pm / _MMU
    rho, ZA, I = mat["rho"], mat["ZA"], mat["I"]
    xi = 0.5 * _K * ZA * rho * x_cm / beta2                   # MeV
    hw = 28.816e-6 * np.sqrt(rho * ZA)                          # plasma energy, MeV
    delta = np.maximum(0.0, 2.0 * np.log(bg) + 2.0 * np.log(hw / I) - 1.0)
    dmp = xi * (np.log(2.0 * _ME * bg * bg / I) + np.log(xi / I) + 0.2 - beta2 - delta)
    z = rng.standard_normal(n_samples)
    lam = -np.log(np.maximum(z * z, 1e-300))                 # Moyal variate, mode 0
    dE = np.maximum(dmp + xi * lam, 0.0)                      # MeV
    f = dE / pm
    # radiative tail: v ~ v^-2 on [v0, 1), probability matched to mean b*rho*x
    v0 = 1e-3
    mean_v = np.log(1.0 / v0) / (1.0 / v0 - 1.0)
    p_rad = min(1.0, mat["b"] * rho * x_cm / mean_v)
    rad = rng.random(n_samples) < p_rad
    u = rng.random(n_samples)
    v = 1.0 / (1.0 / v0 - u * (1.0 / v0 - 1.0))
    f = f + np.where(rad, v, 0.0)
    # scattering: Rayleigh space angle of Highland width, 1 % single-scatter tail
    th0 = _highland(p, x_cm, mat["X0"])
    u1 = 1.0 - rng.random(n_samples)
    u2 = 1.0 - rng.random(n_samples)
    single = rng.random(n_samples) < 0.01
    theta = np.where(single, 2.0 * th0 / np.sqrt(u2), th0 * np.sqrt(-2.0 * np.log(u1)))
    theta_max = 5.0 * float(_highland(np.array([p_a]), x_cm, mat["X0"])[0])
    if axes == "log":
        fc = np.clip(f, 0.0, 1.0)
        fz = fc + (1.0 - fc) * 2.0 * np.sin(0.5 * theta) ** 2       # 1 - (1-f) cos(theta), without cancellation
        t = (1.0 - fc) * np.sin(np.minimum(theta, 0.5 * np.pi))
        (f0, f1), (t0, t1) = LOG_F_RANGE, LOG_T_RANGE
        with np.errstate(divide="ignore"):
            a = np.floor(np.log(np.maximum(fz, 1e-300) / f0) / np.log(f1 / f0) * nf)
            b = np.floor(np.log(np.maximum(t, 1e-300) / t0) / np.log(t1 / t0) * ntheta)
        a = np.clip(a, 0, nf - 1).astype(np.int64)
        b = np.clip(b, 0, ntheta - 1).astype(np.int64)
        counts = np.bincount(a * ntheta + b, minlength=nf * ntheta).astype(np.float64)
        return counts.reshape(nf, ntheta), t1
    a = np.clip(np.floor(f / f_max * nf), 0, nf - 1).astype(np.int64)
    b = np.clip(np.floor(theta / theta_max * ntheta), 0, ntheta - 1).astype(np.int64)
    counts = np.bincount(a * ntheta + b, minlength=nf * ntheta).astype(np.float64)
    return counts.reshape(nf, ntheta), theta_max


def histogram_set(materials: List[str], n_pbin: int = 64, p_lo: float = 1.0, p_hi: float = 400.0,
                  nf: int = 128, ntheta: int = 64, f_max: float = 0.2, n_samples: int = 10**6,
                  step_len: float = 0.02, seed: int = 42, cache: bool = True, axes: str = "linear") -> dict:
    """Histogram set H[M][i] for materials 1..len(materials) (material 0 is vacuum).

    Returns a dict with ``weights`` [n_mat][n_pbin][nf][ntheta] (float64 counts),
    ``f_max`` and ``theta_max`` [n_mat][n_pbin] (float64) and the binning scalars.
    """
    # the key covers the model too: each material's constants and the source of the
    # sampler, so editing either never reuses histograms of the old model
    src = hashlib.sha1((inspect.getsource(_hist_one) + inspect.getsource(_highland)).encode()).hexdigest()[:16]
    params = dict(materials=list(materials), n_pbin=n_pbin, p_lo=p_lo, p_hi=p_hi, nf=nf,
                  ntheta=ntheta, f_max=f_max, n_samples=n_samples, step_len=step_len, seed=seed, v=1,
                  model=[MATERIALS[m] for m in materials], src=src)
    if axes != "linear":
        params["axes"] = axes
    path = _cache_path("hist", params)
    if cache and os.path.exists(path):
        z = np.load(path)
        W, FM, TM = z["weights"], z["f_max"], z["theta_max"]
    else:
        edges = pbin_edges(p_lo, p_hi, n_pbin)
        x_cm = step_len * 100.0
        M = len(materials)
        W = np.zeros((M, n_pbin, nf, ntheta), dtype=np.float64)
        FM = np.full((M, n_pbin), f_max, dtype=np.float64)
        TM = np.zeros((M, n_pbin), dtype=np.float64)

        def one(mi):
            m, i = mi
            rng = np.random.default_rng([seed, m, i])
            W[m, i], TM[m, i] = _hist_one(rng, MATERIALS[materials[m]], edges[i], edges[i + 1],
                                          x_cm, f_max, nf, ntheta, n_samples, axes)

        # each (material, bin) has its own seeded stream, so threading keeps results fixed
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(one, [(m, i) for m in range(M) for i in range(n_pbin)]))
        if cache:
            os.makedirs(_CACHE_DIR, exist_ok=True)
            tmp = path + f".tmp{os.getpid()}.npz"
            np.savez(tmp, weights=W, f_max=FM, theta_max=TM)
            os.replace(tmp, path)
    out = dict(n_mat=W.shape[0], n_pbin=n_pbin, p_lo=float(p_lo), p_hi=float(p_hi),
               nf=nf, ntheta=ntheta, weights=np.ascontiguousarray(W),
               f_max=np.ascontiguousarray(FM), theta_max=np.ascontiguousarray(TM),
               materials=list(materials))
    if axes == "log":
        shape = W.shape[:2]
        out.update(axes="log", f_min=np.full(shape, LOG_F_RANGE[0]), f_max=np.full(shape, LOG_F_RANGE[1]),
                   theta_min=np.full(shape, LOG_T_RANGE[0]), theta_max=np.full(shape, LOG_T_RANGE[1]))
    return out


# --------------------------------------------------------------------------
# geometries (SI units: m, GeV, T)
# --------------------------------------------------------------------------
def _box(lo, hi, mat, block=-1, B=(0.0, 0.0, 0.0)):
    return dict(lo=[float(v) for v in lo], hi=[float(v) for v in hi], material=int(mat),
                block_id=int(block), B=[float(v) for v in B])


def geometry_block1e4() -> dict:
    """Iron block 1x1x2 m (x,y in [-0.5,0.5], z in [0,2]) in air; B = (0,1.7,0) T in iron.

    Materials: 1 = iron, 2 = air.  World bounds |x|,|y| < 2 m, z < 3 m, p_min 0.5 GeV.
    """
    return dict(kind="boxes", boxes=[_box((-0.5, -0.5, 0.0), (0.5, 0.5, 2.0), 1, 0, (0.0, 1.7, 0.0))],
                world_material=2, x_max=2.0, y_max=2.0, z_max=3.0, p_min=0.5)


MAGNET_Z0 = [4.5 * k for k in range(6)]
MAGNET_LEN = 4.0
MAGNET_HALF = 0.6


def geometry_shield1e6() -> dict:
    """Shield-like layout: six iron blocks 1.2x1.2x4 m with 0.5 m air gaps, alternating
    B_y = +-1.7 T (+ for even k), then a 2 m concrete wall z in [27,29], |x|,|y| <= 3 m.

    Materials: 1 = iron, 2 = air (world), 3 = concrete.  World |x|,|y| < 3 m, z < 30 m.
    Block ids 0..5 index the per-magnet field-scale parameters.
    """
    boxes = []
    for k, z0 in enumerate(MAGNET_Z0):
        s = 1.0 if k % 2 == 0 else -1.0
        boxes.append(_box((-MAGNET_HALF, -MAGNET_HALF, z0), (MAGNET_HALF, MAGNET_HALF, z0 + MAGNET_LEN),
                          1, k, (0.0, 1.7 * s, 0.0)))
    boxes.append(_box((-3.0, -3.0, 27.0), (3.0, 3.0, 29.0), 3, -1))
    return dict(kind="boxes", boxes=boxes, world_material=2, x_max=3.0, y_max=3.0, z_max=30.0, p_min=0.5)


def solid(z0: float, z1: float, bottom, top, material: int, block_id: int = -1, B=(0.0, 0.0, 0.0)) -> dict:
    """A solid of the polyhedra geometry: cross-section at height z interpolates the
    counter-clockwise quadrilateral ``bottom`` (at z0) to ``top`` (at z1), vertex by vertex."""
    return dict(z0=float(z0), z1=float(z1), bottom=[list(map(float, v)) for v in bottom],
                top=[list(map(float, v)) for v in top], material=int(material), block_id=int(block_id),
                B=list(map(float, B)))


def _trapezoid(hx_lo: float, hx_hi: float, hy: float, dx: float = 0.0):
    """Counter-clockwise quadrilateral: half-width hx_lo at y = -hy, hx_hi at y = +hy, shifted by dx."""
    return [(-hx_lo + dx, -hy), (hx_lo + dx, -hy), (hx_hi + dx, hy), (-hx_hi + dx, hy)]


def geometry_tapered() -> dict:
    """Shield1e6's layout with tapered magnets (the paper's convex-polyhedron geometry,
    Sec. Simulation item 1): six iron solids in z in [4.5k, 4.5k + 4], whose
    cross-sections are trapezoids (wider at -y than at +y) that narrow along z
    and shift sideways by 2 cm per block, B_y = +-1.7 T alternating; the concrete
    wall z in [27, 29], |x|, |y| <= 3 as a solid with a rectangular section.
    Materials: 1 iron, 2 air (world), 3 concrete.  World |x|, |y| < 3 m, z < 30 m."""
    solids = []
    for k, z0 in enumerate(MAGNET_Z0):
        s = 1.0 if k % 2 == 0 else -1.0
        h0 = 0.75 - 0.04 * k
        h1 = h0 - 0.12
        bot = _trapezoid(h0, h0 - 0.10, 0.60, 0.02 * k)
        top = _trapezoid(h1, h1 - 0.08, 0.55, 0.02 * k + 0.02)
        solids.append(solid(z0, z0 + MAGNET_LEN, bot, top, 1, k, (0.0, 1.7 * s, 0.0)))
    wall = _trapezoid(3.0, 3.0, 3.0)
    solids.append(solid(27.0, 29.0, wall, wall, 3, -1))
    return dict(kind="polyhedra", solids=solids, world_material=2, x_max=3.0, y_max=3.0, z_max=30.0, p_min=0.5)


def _smooth_box(u: np.ndarray, a: float, b: float, w: float) -> np.ndarray:
    return 0.5 * (np.tanh((u - a) / w) - np.tanh((u - b) / w))


def _smooth_box_edge(u: np.ndarray, a: float, b: float, w: float) -> np.ndarray:
    # w * d/du of _smooth_box: peaked at the block ends, used for a fringe B_z
    return 0.5 * (np.tanh((u - b) / w) ** 2 - np.tanh((u - a) / w) ** 2)


def magnet_field_map(nx: int, ny: int, nz: int, half_xy: float, z_lo: float, z_hi: float, magnet_z0,
                     magnet_B, magnet_len: float = MAGNET_LEN, edge_w: float = 0.03) -> dict:
    """Node-based synthetic magnet field, float32 [nz][ny][nx][3].

    Nodes sit at origin + (i,j,k)*spacing over x,y in [-half_xy, half_xy] and z in
    [z_lo, z_hi].  Inside each block B_y ~ magnet_B[k] with tanh edges of width 3 cm,
    plus a small quadrupole-like B_x and a fringe B_z at the block ends.  Every
    component is a sum over blocks of (z profile) x (x-y profile), built as outer
    products.
    """
    x = np.linspace(-half_xy, half_xy, nx)
    y = np.linspace(-half_xy, half_xy, ny)
    z = np.linspace(z_lo, z_hi, nz)
    Sx = _smooth_box(x, -MAGNET_HALF, MAGNET_HALF, edge_w)
    Sy = _smooth_box(y, -MAGNET_HALF, MAGNET_HALF, edge_w)
    SxSy = Sy[:, None] * Sx[None, :]
    quad = (y[:, None] * x[None, :]) / (MAGNET_HALF * MAGNET_HALF) * SxSy
    ylin = (y[:, None] / MAGNET_HALF) * SxSy
    zy = np.zeros(nz)
    ze = np.zeros(nz)
    for z0, b in zip(magnet_z0, magnet_B):
        zy += b * _smooth_box(z, z0, z0 + magnet_len, edge_w)
        ze += b * _smooth_box_edge(z, z0, z0 + magnet_len, edge_w)
    B = np.empty((nz, ny, nx, 3), dtype=np.float32)
    B[..., 0] = (0.1 * zy)[:, None, None] * quad[None]
    B[..., 1] = zy[:, None, None] * SxSy[None]
    B[..., 2] = (0.3 * ze)[:, None, None] * ylin[None]
    spacing = [(2 * half_xy) / (nx - 1), (2 * half_xy) / (ny - 1), (z_hi - z_lo) / (nz - 1)]
    return dict(kind="map", dims=[nx, ny, nz], origin=[-half_xy, -half_xy, z_lo], spacing=spacing, B=B)


def field_map_shield1e6(nx: int = 200, ny: int = 200, nz: int = 600, z_lo: float = -0.5,
                      z_hi: float = 27.5, half_xy: float = 3.0, magnet_z0=None,
                      magnet_B=None, edge_w: float = 0.03) -> dict:
    """Field map of the six-magnet shield: 200x200x600 nodes over x,y in [-3,3] m and
    z in [-0.5, 27.5] m (0.5 m past the magnets at both ends, so the field is ~0 at
    the map boundary), B_y = +-1.7 T alternating."""
    magnet_z0 = MAGNET_Z0 if magnet_z0 is None else magnet_z0
    if magnet_B is None:
        magnet_B = [1.7 if k % 2 == 0 else -1.7 for k in range(len(magnet_z0))]
    return magnet_field_map(nx, ny, nz, half_xy, z_lo, z_hi, magnet_z0, magnet_B, edge_w=edge_w)


# --------------------------------------------------------------------------
# muon spectra -> float32 SoA
# --------------------------------------------------------------------------
def _soa(x, y, z, px, py, pz, q) -> dict:
    n = len(x)
    return dict(x=x.astype(np.float32), y=y.astype(np.float32), z=z.astype(np.float32),
                px=px.astype(np.float32), py=py.astype(np.float32), pz=pz.astype(np.float32),
                q=q.astype(np.int8), steps=np.zeros(n, np.int32), status=np.zeros(n, np.uint8))


def muons_block(n: int, seed: int = 1234) -> dict:
    """p log-uniform 5-300 GeV, q = +-1, x,y ~ U(-0.4,0.4) m, z = 0, px,py ~ N(0,0.5) GeV."""
    rng = np.random.default_rng(seed)
    p = np.exp(rng.uniform(np.log(5.0), np.log(300.0), n))
    px = rng.normal(0.0, 0.5, n)
    py = rng.normal(0.0, 0.5, n)
    bad = px * px + py * py >= p * p
    while bad.any():
        px[bad] = rng.normal(0.0, 0.5, bad.sum())
        py[bad] = rng.normal(0.0, 0.5, bad.sum())
        bad = px * px + py * py >= p * p
    pz = np.sqrt(p * p - px * px - py * py)
    q = np.where(rng.random(n) < 0.5, -1, 1)
    x = rng.uniform(-0.4, 0.4, n)
    y = rng.uniform(-0.4, 0.4, n)
    return _soa(x, y, np.zeros(n), px, py, pz, q)


def muons_shield(n: int, seed: int = 1234, p_lo: float = 10.0, p_hi: float = 350.0) -> dict:
    """dN/dp ~ p^-2.7 on [10,350] GeV (inverse CDF), p_T ~ Exp(1 GeV), uniform azimuth,
    random charge, x,y ~ U(-0.4,0.4) m at z = 0."""
    rng = np.random.default_rng(seed)
    g = -1.7
    u = rng.random(n)
    p = (p_lo ** g + u * (p_hi ** g - p_lo ** g)) ** (1.0 / g)
    pt = rng.exponential(1.0, n)
    bad = pt >= p
    while bad.any():
        pt[bad] = rng.exponential(1.0, bad.sum())
        bad = pt >= p
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    px, py = pt * np.cos(phi), pt * np.sin(phi)
    pz = np.sqrt(p * p - pt * pt)
    q = np.where(rng.random(n) < 0.5, -1, 1)
    x = rng.uniform(-0.4, 0.4, n)
    y = rng.uniform(-0.4, 0.4, n)
    return _soa(x, y, np.zeros(n), px, py, pz, q)


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    geometry: dict
    field: dict
    hist: dict
    muons: dict
    step_len: float
    max_steps: int
    seed: int
    id_offset: int = 0
    instance: int = 0

    @property
    def n(self) -> int:
        return len(self.muons["x"])


def _nearest(field: Optional[str], fmap: dict) -> dict:
    """The map read at the nearest node when field == "nearest"."""
    return dict(fmap, kind="map_nearest") if field == "nearest" else fmap


def workload(name: str, n: Optional[int] = None, hist_samples: Optional[int] = None,
             field: Optional[str] = None, axes: str = "linear") -> Workload:
    """Named workloads.

    * ``block1e4``: 1e4 muons, one iron block in air, analytic per-box field, 200 steps,
      iron+air histograms (64 log bins on 1-400 GeV, 128x64 cells, 1e6 samples each).
    * ``shield1e6``: 1e6 muons through the six-magnet shield and concrete wall, trilinear
      200x200x600 field map, iron/air/concrete histograms, 1500 steps.
    * ``tapered1e6``: shield1e6 with tapered magnets (``geometry_tapered``, polyhedra).
    * ``shield1e8``: shield1e6's spectrum and geometry with a 400x400x1200 map and
      4 materials x 128 bins x 256x128 cells (a 4th material, lead, is present in the
      table set but not placed in the geometry).

    ``n`` and ``hist_samples`` shrink a workload for tests; ``field`` = "box" swaps the map
    for the analytic per-box field and "nearest" reads the map at the nearest node;
    ``axes`` = "log" builds the histograms on the paper's log-scaled axes.
    """
    if name == "block1e4":
        h = histogram_set(["iron", "air"], n_samples=hist_samples or 10**6, axes=axes)
        mu = muons_block(n or 10_000)
        geo = geometry_block1e4()
        fld = dict(kind="box")
        return Workload(name, geo, fld, h, mu, 0.02, 200, 7)
    if name in ("shield1e6", "diff1e6"):
        h = histogram_set(["iron", "air", "concrete"], n_samples=hist_samples or 10**6, axes=axes)
        mu = muons_shield(n or 1_000_000)
        geo = geometry_shield1e6()
        fld = dict(kind="box") if field == "box" else _nearest(field, field_map_shield1e6())
        return Workload(name, geo, fld, h, mu, 0.02, 1500, 7)
    if name == "tapered1e6":
        h = histogram_set(["iron", "air", "concrete"], n_samples=hist_samples or 10**6, axes=axes)
        mu = muons_shield(n or 1_000_000)
        geo = geometry_tapered()
        fld = dict(kind="box") if field == "box" else _nearest(field, field_map_shield1e6())
        return Workload(name, geo, fld, h, mu, 0.02, 1500, 7)
    if name == "shield1e8":
        h = histogram_set(["iron", "air", "concrete", "lead"], n_pbin=128, nf=256, ntheta=128, axes=axes,
                          n_samples=hist_samples or 10**6)
        mu = muons_shield(n or 100_000_000)
        geo = geometry_shield1e6()
        fld = dict(kind="box") if field == "box" else _nearest(field, field_map_shield1e6(400, 400, 1200))
        return Workload(name, geo, fld, h, mu, 0.02, 1500, 7)
    raise KeyError(name)


def batched_instance(i: int, seed: int = 2024, vox_dims=(64, 64, 512), map_dims=(100, 100, 300),
                     half_xy: float = 1.6, n_range=(1000, 1_000_000), n: Optional[int] = None) -> dict:
    """Instance i of the batched workload: six iron blocks 1.2x1.2x4 m with field
    magnitudes U(1.0, 1.9) T (alternating sign) and five gaps U(0.1, 1.0) m, 0.5 m of
    air and a 2 m concrete wall, voxelised to uint8 [nz][ny][nx] over x,y in
    [-1.6, 1.6] m and z in [0, L]; its own node field map over the same x,y and
    z in [-0.5, L]; n muons (log-uniform in n_range) of the p^-2.7 spectrum.
    Materials: 1 iron, 2 air (world), 3 concrete.  World |x|,|y| < 1.6 m, z < L."""
    rng = np.random.default_rng([seed, i])
    Bmag = rng.uniform(1.0, 1.9, 6) * np.array([1.0 if k % 2 == 0 else -1.0 for k in range(6)])
    gaps = rng.uniform(0.1, 1.0, 5)
    z0 = [0.0]
    for g in gaps:
        z0.append(z0[-1] + MAGNET_LEN + g)
    end = z0[-1] + MAGNET_LEN
    wall = (end + 0.5, end + 2.5)
    L = wall[1]
    nxv, nyv, nzv = vox_dims
    sx, sy, sz = 2 * half_xy / nxv, 2 * half_xy / nyv, L / nzv
    xc = -half_xy + (np.arange(nxv) + 0.5) * sx
    yc = -half_xy + (np.arange(nyv) + 0.5) * sy
    zc = (np.arange(nzv) + 0.5) * sz
    in_xy = (np.abs(yc)[:, None] < MAGNET_HALF) & (np.abs(xc)[None, :] < MAGNET_HALF)
    in_block = np.zeros(nzv, bool)
    for a in z0:
        in_block |= (zc >= a) & (zc < a + MAGNET_LEN)
    vox = np.full((nzv, nyv, nxv), 2, np.uint8)
    vox[in_block[:, None, None] & in_xy[None]] = 1
    vox[(zc >= wall[0]) & (zc < wall[1])] = 3
    geo = dict(kind="voxels", voxels=vox, origin=[-half_xy, -half_xy, 0.0], spacing=[sx, sy, sz],
               world_material=2, x_max=half_xy, y_max=half_xy, z_max=L, p_min=0.5)
    fld = magnet_field_map(map_dims[0], map_dims[1], map_dims[2], half_xy, -0.5, L, z0, list(Bmag))
    if n is None:
        n = int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
    mu = muons_shield(n, seed=seed * 7919 + i)
    return dict(geometry=geo, field=fld, muons=mu, n=n, length=L, B=Bmag, gaps=gaps)


def batched_counts(n_inst: int = 256, seed: int = 2024, n_range=(1000, 1_000_000)):
    """Muon counts of the batched workload's instances (same draws as batched_instance)."""
    out = []
    for i in range(n_inst):
        rng = np.random.default_rng([seed, i])
        rng.uniform(1.0, 1.9, 6)
        rng.uniform(0.1, 1.0, 5)
        out.append(int(round(np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]))))))
    return out


def batched_instances(n_inst: int = 256, seed: int = 2024, **kw):
    """Generator over the instances of the batched workload (one in host memory at a time)."""
    for i in range(n_inst):
        yield batched_instance(i, seed=seed, **kw)


BATCH_STEP_LEN = 0.02
BATCH_MAX_STEPS = 2000
BATCH_SEED = 11


def batched_hist(hist_samples: Optional[int] = None) -> dict:
    """Histogram set of the batched workload (iron, air, concrete, as shield1e6)."""
    return histogram_set(["iron", "air", "concrete"], n_samples=hist_samples or 10**6)


SHIELD1E8_MUONS = 100_000_000
SHIELD1E8_CHUNK = 16_000_000


def muons_shield1e8_chunk(c: int, n: int) -> dict:
    """Chunk c (n muons, ids c * SHIELD1E8_CHUNK + m) of the 1e8-muon shield1e8 stream: shield1e6's
    spectrum, each chunk from its own seed so chunks can be made one at a time."""
    return muons_shield(n, seed=1234 * 1000 + c)
