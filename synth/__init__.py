"""Seeded synthetic inputs for the prism-gravity operator: meshes, surveys,
density models and noise.

This module is shared by the CPU oracle (``oracle/``), the CUDA library's
tests and ``bench.py``.  It holds NO arithmetic of the method itself (no
corner function, no forward or adjoint product, no solver): it only draws
geometry and densities with numpy's PCG64 generator from a fixed seed, so
that both sides of every parity test see bit-identical inputs.

Conventions (the paper's Section 2.1 places the observation point at the
origin of the prism's frame and leaves the axis orientation implicit; the
reading used throughout is):

* x, y horizontal in metres; z is DEPTH, positive down; the mesh top is z = 0.
* A station at height h above the mesh top has z = -h (h > 0).
* Cell k = (i, j, l) has linear index k = i + nx*(j + ny*l) (x fastest).
* Densities are density contrasts in kg/m^3; data are in mGal.

Workloads follow the shapes of the paper's experiments (Section 4: the
two-body, dyke and paper-scale regional cases; Table 1 and Table 3 sizes)
at the sizes named in each function.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List

import numpy as np

__all__ = [
    "Mesh", "Survey", "Workload", "uniform_mesh", "grid_survey",
    "random_survey", "WORKLOADS", "make_workload", "add_noise",
    "serving_jobs", "random_vector",
]


@dataclasses.dataclass
class Mesh:
    """Rectilinear mesh given by its three edge arrays (metres, z down)."""
    xe: np.ndarray
    ye: np.ndarray
    ze: np.ndarray

    @property
    def nx(self) -> int:
        return len(self.xe) - 1

    @property
    def ny(self) -> int:
        return len(self.ye) - 1

    @property
    def nz(self) -> int:
        return len(self.ze) - 1

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nnodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)


@dataclasses.dataclass
class Survey:
    """Station coordinates (structure of arrays, metres, z = -height)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray

    @property
    def n(self) -> int:
        return len(self.x)

    def subset(self, idx: np.ndarray) -> "Survey":
        idx = np.asarray(idx)
        return Survey(self.x[idx].copy(), self.y[idx].copy(), self.z[idx].copy())


@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    survey: Survey
    m: np.ndarray              # true density contrast, float64 [M]
    z0: float = 50.0           # depth-weighting offset, w(z) = (z + z0)^-1
    tol: float = 1e-6          # CG relative residual target
    noise_abs: float = 0.0     # mGal
    noise_rel: float = 0.0     # fraction of |d|
    precision: str = "fp64"
    near_cells: float = 3.0
    description: str = ""


def uniform_mesh(nx: int, ny: int, nz: int, dx: float, dy: float, dz: float,
                 x0: float = 0.0, y0: float = 0.0) -> Mesh:
    return Mesh(x0 + dx * np.arange(nx + 1, dtype=np.float64),
                y0 + dy * np.arange(ny + 1, dtype=np.float64),
                dz * np.arange(nz + 1, dtype=np.float64))


def grid_survey(x0: float, x1: float, nxs: int, y0: float, y1: float, nys: int,
                height: float) -> Survey:
    xs = np.linspace(x0, x1, nxs)
    ys = np.linspace(y0, y1, nys)
    X, Y = np.meshgrid(xs, ys, indexing="xy")   # x fastest in the flattened order
    X = X.ravel().copy()
    Y = Y.ravel().copy()
    return Survey(X, Y, np.full(X.shape, -float(height)))


def random_survey(n: int, x0: float, x1: float, y0: float, y1: float,
                  hmin: float, hmax: float, seed: int) -> Survey:
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.uniform(x0, x1, n)
    y = rng.uniform(y0, y1, n)
    h = rng.uniform(hmin, hmax, n)
    return Survey(x, y, -h)


def jittered_grid_survey(n_target: int, x0: float, x1: float, y0: float, y1: float,
                         height: float, jitter: float, rng: np.random.Generator) -> Survey:
    aspect = (x1 - x0) / (y1 - y0)
    nys = max(2, int(round(math.sqrt(n_target / aspect))))
    nxs = max(2, int(round(n_target / nys)))
    s = grid_survey(x0, x1, nxs, y0, y1, nys, height)
    sx = (x1 - x0) / max(nxs - 1, 1)
    sy = (y1 - y0) / max(nys - 1, 1)
    s.x = np.clip(s.x + rng.uniform(-jitter, jitter, s.n) * sx, x0, x1)
    s.y = np.clip(s.y + rng.uniform(-jitter, jitter, s.n) * sy, y0, y1)
    return s


def _cell_centres(mesh: Mesh):
    xc = 0.5 * (mesh.xe[:-1] + mesh.xe[1:])
    yc = 0.5 * (mesh.ye[:-1] + mesh.ye[1:])
    zc = 0.5 * (mesh.ze[:-1] + mesh.ze[1:])
    # broadcast to [nz, ny, nx] so that ravel() gives k = i + nx*(j + ny*l)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    return X, Y, Z


def _block(mesh: Mesh, i0, i1, j0, j1, l0, l1, value) -> np.ndarray:
    m = np.zeros((mesh.nz, mesh.ny, mesh.nx))
    m[l0:l1, j0:j1, i0:i1] = value
    return m.ravel()


def lognormal_background(shape_cells: int, std: float, rng: np.random.Generator) -> np.ndarray:
    b = np.exp(rng.normal(0.0, 0.5, shape_cells))
    return (b - b.mean()) / b.std() * std


# ---------------------------------------------------------------------------
# The five workload shapes.
# ---------------------------------------------------------------------------

def block_20x20x10(seed: int = 0) -> Workload:
    """4,000 cubic 100 m cells under a 21 x 21 station grid at 25 m height,
    100 m spacing; 4 x 4 x 3 block at +300 kg/m^3 in zero background."""
    mesh = uniform_mesh(20, 20, 10, 100.0, 100.0, 100.0)
    survey = grid_survey(0.0, 2000.0, 21, 0.0, 2000.0, 21, 25.0)
    m = _block(mesh, 8, 12, 8, 12, 2, 5, 300.0)
    return Workload("block_20x20x10", mesh, survey, m, z0=50.0, tol=1e-8,
                    noise_abs=0.01, precision="fp64",
                    description="20x20x10 mesh of 100 m cubes, 21x21 stations at 25 m, block +300")


def vslab_80x80x40(seed: int = 0) -> Workload:
    """256,000 cubic 50 m cells under 81 x 81 stations at 10 m height;
    vertical 2 x 40 x 30-cell slab at +400 kg/m^3 in zero background."""
    mesh = uniform_mesh(80, 80, 40, 50.0, 50.0, 50.0)
    survey = grid_survey(0.0, 4000.0, 81, 0.0, 4000.0, 81, 10.0)
    m = _block(mesh, 39, 41, 20, 60, 2, 32, 400.0)
    return Workload("vslab_80x80x40", mesh, survey, m, z0=50.0, tol=1e-6,
                    noise_abs=0.01, noise_rel=0.01, precision="fp64",
                    description="80x80x40 mesh of 50 m cubes, 81x81 stations at 10 m, vertical slab +400")


def dipdyke_150x150x60(seed: int = 0) -> Workload:
    """1.35M cubic 40 m cells under 151 x 151 stations at 10 m height; a
    45-degree dipping dyke (+350 kg/m^3, 3 cells thick) in a seeded
    log-normal background standardised to std 20 kg/m^3."""
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    mesh = uniform_mesh(150, 150, 60, 40.0, 40.0, 40.0)
    survey = grid_survey(0.0, 6000.0, 151, 0.0, 6000.0, 151, 10.0)
    m = lognormal_background(mesh.ncells, 20.0, rng).reshape(mesh.nz, mesh.ny, mesh.nx)
    # Strike along y (j in [30,120)); one cell of lateral shift per layer of
    # cubic cells gives a 45 degree dip toward +x.
    for l in range(1, 50):
        i0 = 40 + l
        m[l, 30:120, i0:i0 + 3] += 350.0
    return Workload("dipdyke_150x150x60", mesh, survey, m.ravel(), z0=50.0, tol=1e-6,
                    precision="mixed", near_cells=3.0,
                    description="150x150x60 mesh of 40 m cubes, 151x151 stations at 10 m, 45 deg dyke +350 in log-normal background")


def paper_210x210x75(seed: int = 0, n_stations: int = 178_797) -> Workload:
    """3,307,500 cubic 100 m cells; 178,797 stations uniform over the
    21 x 21 km footprint at heights U[1, 50] m; random layered model plus
    three dipping dykes, float32-representable values in [-500, 500]."""
    rng = np.random.Generator(np.random.PCG64(5000 + seed))
    mesh = uniform_mesh(210, 210, 75, 100.0, 100.0, 100.0)
    survey = random_survey(n_stations, 0.0, 21000.0, 0.0, 21000.0, 1.0, 50.0, seed=7000 + seed)
    X, Y, Z = _cell_centres(mesh)
    layers = np.cumsum(rng.normal(0.0, 25.0, mesh.nz))
    layers = np.clip(layers - layers.mean(), -150.0, 150.0)
    m = np.broadcast_to(layers[:, None, None], X.shape).copy()
    for _ in range(3):
        strike = rng.uniform(0.0, math.pi)
        dip = math.radians(rng.uniform(30.0, 80.0))
        thick = rng.uniform(200.0, 500.0)
        cx, cy = rng.uniform(4000.0, 17000.0, 2)
        rho = rng.choice([-1.0, 1.0]) * rng.uniform(200.0, 350.0)
        # unit normal of the dyke plane: horizontal direction perpendicular to
        # strike, tilted by the dip
        nxh, nyh = -math.sin(strike), math.cos(strike)
        n = np.array([nxh * math.sin(dip), nyh * math.sin(dip), math.cos(dip)])
        dist = (X - cx) * n[0] + (Y - cy) * n[1] + (Z - 0.0) * n[2]
        along = (X - cx) * math.cos(strike) + (Y - cy) * math.sin(strike)
        inside = (np.abs(dist) < 0.5 * thick) & (np.abs(along) < 6000.0) & (Z < 6000.0)
        m[inside] += rho
    m = np.clip(m, -500.0, 500.0).astype(np.float32).astype(np.float64)
    return Workload("paper_210x210x75", mesh, survey, m.ravel(), z0=50.0, tol=1e-6,
                    precision="mixed", near_cells=3.0,
                    description="210x210x75 mesh of 100 m cubes (3,307,500 cells), 178,797 random stations at 1-50 m, layered + 3 dipping dykes")


def two_body_160x160x80(seed: int = 0) -> Workload:
    """The paper's two-body synthetic (Section 4.1) in shape: 2.05M cubic 125 m
    cells (20 x 20 x 10 km) under 66 x 66 = 4,356 stations at 10 m height; two
    prisms at +1000 kg/m^3: 13-17 km laterally and 1.5-3 km deep, 6-10 km
    laterally and 0.5-3 km deep; 1 % RMS Gaussian noise."""
    a = 125.0
    mesh = uniform_mesh(160, 160, 80, a, a, a)
    survey = grid_survey(0.0, 20000.0, 66, 0.0, 20000.0, 66, 10.0)
    m = np.zeros((80, 160, 160))
    idx = lambda v: int(round(v / a))
    m[idx(1500):idx(3000), idx(13000):idx(17000), idx(13000):idx(17000)] = 1000.0
    m[idx(500):idx(3000), idx(6000):idx(10000), idx(6000):idx(10000)] = 1000.0
    return Workload("two_body_160x160x80", mesh, survey, m.ravel(), z0=50.0, tol=1e-6, noise_rel=0.01,
                    precision="mixed", description="two prisms +1000 kg/m^3, 160x160x80 of 125 m, 66x66 stations")


def tube_slab_100x100x50(seed: int = 0) -> Workload:
    """The paper's curvilinear-tube + dipping-slab synthetic (Section 4.2) in
    shape: 100 x 100 x 50 prisms of 200 x 200 x 100 m (square-based, not cubic),
    196 x 196 = 38,416 stations at 10 m height; a sinuous tube of varying width
    at -1000 kg/m^3 from 1 to 4 km depth and a slab dipping 40 degrees toward
    +y at +1000 kg/m^3.  The paper describes the bodies only qualitatively; this
    is one seeded realisation."""
    rng = np.random.Generator(np.random.PCG64(8000 + seed))
    mesh = uniform_mesh(100, 100, 50, 200.0, 200.0, 100.0)
    survey = grid_survey(0.0, 20000.0, 196, 0.0, 20000.0, 196, 10.0)
    X, Y, Z = _cell_centres(mesh)
    m = np.zeros(X.shape)
    # tube: centreline y = 6 km + 1.5 km sin(2 pi x / 8 km + phase) for x in [2, 18] km
    phase = rng.uniform(0, 2 * math.pi)
    yc = 6000.0 + 1500.0 * np.sin(2 * math.pi * X / 8000.0 + phase)
    width = 600.0 + 300.0 * np.sin(2 * math.pi * X / 5000.0)
    tube = (np.abs(Y - yc) < 0.5 * width) & (X > 2000) & (X < 18000) & (Z > 1000) & (Z < 4000)
    m[tube] = -1000.0
    # slab: top trace at y = 12 km, dipping 40 degrees toward +y, 600 m thick, x in [4, 16] km
    dip = math.radians(40.0)
    dist = (Y - 12000.0) * math.sin(dip) - Z * math.cos(dip)
    slab = (np.abs(dist) < 300.0) & (X > 4000) & (X < 16000) & (Y >= 12000.0) & (Z < 4500)
    m[slab] = 1000.0
    return Workload("tube_slab_100x100x50", mesh, survey, m.ravel(), z0=50.0, tol=1e-6, precision="mixed",
                    description="100x100x50 prisms of 200x200x100 m, 196x196 stations, tube -1000 + 40 deg slab +1000")


WORKLOADS: Dict[str, Callable[..., Workload]] = {
    "block_20x20x10": block_20x20x10,
    "vslab_80x80x40": vslab_80x80x40,
    "dipdyke_150x150x60": dipdyke_150x150x60,
    "paper_210x210x75": paper_210x210x75,
    "two_body_160x160x80": two_body_160x160x80,
    "tube_slab_100x100x50": tube_slab_100x100x50,
}


def make_workload(name: str, seed: int = 0, **kw) -> Workload:
    return WORKLOADS[name](seed=seed, **kw)


def add_noise(d_clean: np.ndarray, noise_abs: float, noise_rel: float, seed: int) -> np.ndarray:
    """Additive white Gaussian noise with per-datum std noise_rel*|d| + noise_abs
    (the paper's Section 4.1 noise experiment uses additive white Gaussian noise)."""
    rng = np.random.Generator(np.random.PCG64(9000 + seed))
    sigma = noise_rel * np.abs(d_clean) + noise_abs
    return d_clean + sigma * rng.standard_normal(d_clean.shape)


def random_vector(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(12000 + seed))
    return scale * rng.standard_normal(n)


def small_random_problem(nx: int, ny: int, nz: int, ns: int, seed: int,
                         cell: float = 10.0, height=(0.5, 8.0), irregular: bool = False):
    """Tiny mesh + scattered stations for brute-force parity. With
    irregular=True the edge spacings are random (rectilinear mesh)."""
    rng = np.random.Generator(np.random.PCG64(20000 + seed))
    if irregular:
        xe = np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, nx) * cell)])
        ye = np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, ny) * cell)])
        ze = np.concatenate([[0.0], np.cumsum(rng.uniform(0.5, 1.5, nz) * cell)])
        mesh = Mesh(xe, ye, ze)
    else:
        mesh = uniform_mesh(nx, ny, nz, cell, cell, cell)
    pad = 2.0 * cell
    sx = rng.uniform(mesh.xe[0] - pad, mesh.xe[-1] + pad, ns)
    sy = rng.uniform(mesh.ye[0] - pad, mesh.ye[-1] + pad, ns)
    sz = -rng.uniform(height[0], height[1], ns)
    m = rng.normal(0.0, 100.0, mesh.ncells)
    return mesh, Survey(sx, sy, sz), m


# ---------------------------------------------------------------------------
# Serving stream: 256 jobs, Poisson arrivals at 20 req/s.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Job:
    arrival_s: float
    kind: str                  # "forward" | "invert"
    mesh: Mesh
    survey: Survey
    m: np.ndarray


def serving_jobs(n_jobs: int = 256, rate_hz: float = 20.0, seed: int = 0,
                 cells=(50_000, 500_000), stations=(1_000, 20_000),
                 cell_size=(25.0, 100.0)) -> List[Job]:
    """Seeded job mix: forward or inversion (50/50), each with its own mesh of
    50k-500k cubic prisms (cell size 25-100 m), a block or dyke model in zero
    background, and 1k-20k stations on a jittered grid at 5-30 m height."""
    rng = np.random.Generator(np.random.PCG64(30000 + seed))
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n_jobs))
    jobs = []
    for q in range(n_jobs):
        M = int(rng.uniform(*cells))
        a = float(rng.uniform(*cell_size))
        nz = int(rng.integers(10, 41))
        nxy = max(4, int(round(math.sqrt(M / nz))))
        nx = nxy
        ny = max(4, M // (nz * nx))
        mesh = uniform_mesh(nx, ny, nz, a, a, a)
        N = int(rng.uniform(*stations))
        survey = jittered_grid_survey(N, 0.0, nx * a, 0.0, ny * a,
                                      float(rng.uniform(5.0, 30.0)), 0.3, rng)
        m = np.zeros((nz, ny, nx))
        if rng.random() < 0.5:
            i0 = int(rng.integers(0, nx - 2)); j0 = int(rng.integers(0, ny - 2))
            l0 = int(rng.integers(0, max(1, nz - 3)))
            m[l0:l0 + int(rng.integers(2, 8)), j0:j0 + int(rng.integers(2, 12)),
              i0:i0 + int(rng.integers(2, 12))] = rng.uniform(100.0, 500.0)
        else:
            j0 = int(rng.integers(0, ny // 2)); j1 = j0 + ny // 3
            i0 = int(rng.integers(0, nx // 2))
            for l in range(0, nz // 2):
                m[l, j0:j1, min(nx - 1, i0 + l):min(nx, i0 + l + 2)] = rng.uniform(100.0, 500.0)
        kind = "forward" if rng.random() < 0.5 else "invert"
        jobs.append(Job(float(t[q]), kind, mesh, survey, m.ravel()))
    return jobs
