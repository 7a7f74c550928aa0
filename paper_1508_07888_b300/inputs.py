"""Seeded synthetic inputs for the M1 radiative-transfer step.

This module only draws inputs: density fields, source positions and
luminosities, initial states and the workload descriptions.  It holds none of
the method's arithmetic (no closure, flux, rate, cross-section, time step or
unit conversion of the solver) and imports neither the GPU library nor the
CPU oracle, so both can be fed from it.

Workloads stand in for the paper's reionisation runs (Sec. 6.6: 128^3 coarse
cells, 3 photon groups [13.6, 24.6, 54.4, 1000] eV, 5e4 K black-body sources,
c/10) and for its HII-region test (Sec. 6.4: corner source of 5e48 photons/s,
n = 1e-3 cm^-3, 1e5 K black body, reflective faces at the source and
transmissive elsewhere).  No dataset is read.

Recipes:
  * density: white noise (numpy PCG64, seed) -> real FFT -> amplitude
    k^(-slope/2) (P(k) ~ k^-slope, k = 0 removed) -> inverse FFT -> unit
    variance g -> n0 = 1e-3 cm^-3 * exp(sigma g), rounded to float32.
  * sources: the nsrc densest cells (ties: lower linear index first).
  * luminosities: log-uniform in [1e48, 1e50] photons/s, or proportional to
    n0^1.5 and normalised to a mean of 1e49 photons/s (float64; every path
    reads them in float64).
  * initial state: N = F = 0, xHI = 1 - 1.2e-3, T = 100 K (1e4 K fixed for
    the Stromgren workload).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 2.99792458e10          # cm/s
KPC = 3.0856775814913673e21      # cm
DX_REF = 6.6 * KPC / 32          # cm, cell size of every workload (6.6 kpc / 32)
GROUPS_3 = (13.6, 24.6, 54.4, 1000.0)
GROUPS_2 = (13.6, 24.6, 1000.0)
GROUPS_1 = (13.6, 1000.0)
ALPHA_B_1E4 = 2.59e-13           # cm^3/s, case-B recombination at 1e4 K (textbook)

BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_INFLOW = 0, 1, 2, 3


def f32(a):
    """Round to float32-representable values, returned as float64."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def lognormal_field(n, sigma: float, slope: float, seed: int, nbar: float = 1e-3):
    """n0 [nz, ny, nx] in cm^-3: exp of a unit-variance Gaussian random field."""
    if np.isscalar(n):
        shape = (int(n),) * 3
    else:
        shape = tuple(int(v) for v in n)
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal(shape)
    wk = np.fft.rfftn(w)
    kz = np.fft.fftfreq(shape[0]) * shape[0]
    ky = np.fft.fftfreq(shape[1]) * shape[1]
    kx = np.fft.rfftfreq(shape[2]) * shape[2]
    k2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (-slope / 4.0)
    g = np.fft.irfftn(wk * amp, s=shape, axes=tuple(range(len(shape))))
    g = (g - g.mean()) / g.std()
    return f32(nbar * np.exp(sigma * g))


def densest_cells(n0: np.ndarray, nsrc: int) -> np.ndarray:
    flat = n0.reshape(-1)
    order = np.lexsort((np.arange(flat.size), -flat))
    return np.ascontiguousarray(order[:nsrc].astype(np.int64))


def loguniform_lum(nsrc: int, seed: int, lo: float = 1e48, hi: float = 1e50):
    rng = np.random.Generator(np.random.PCG64(seed))
    return 10.0 ** rng.uniform(np.log10(lo), np.log10(hi), nsrc)


def density_lum(n0_at_src: np.ndarray, power: float = 1.5, mean: float = 1e49):
    w = np.asarray(n0_at_src, dtype=np.float64) ** power
    return w * (mean / w.mean())


@dataclass
class Box:
    """One uniform box: density, sources and the initial state."""
    n0: np.ndarray                 # [nz, ny, nx] cm^-3 (float32-representable)
    src_cells: np.ndarray          # int64 linear cell indices
    src_Q: np.ndarray              # photons/s per source (whole spectrum)
    xHI0: float = 1.0 - 1.2e-3
    T0: float = 100.0
    dx: float = DX_REF
    T_field: np.ndarray | None = None   # initial temperature per cell (overrides T0)

    @property
    def shape(self):
        return self.n0.shape

    @property
    def ncell(self) -> int:
        return int(self.n0.size)

    def initial_state(self, ngroups: int):
        nz, ny, nx = self.shape
        U = np.zeros((ngroups, nz, ny, nx, 4))
        xHI = np.full(self.shape, self.xHI0)
        T = np.full(self.shape, self.T0) if self.T_field is None else np.array(self.T_field, dtype=np.float64)
        return U, xHI, T


@dataclass
class Workload:
    """A named workload: boxes plus the run settings shared by all of them."""
    name: str
    boxes: list
    edges_eV: tuple
    T_bb: float
    c_frac: float                  # reduced speed of light / c
    steps: int
    ots: bool = False
    isothermal: bool = False
    nsub: int = 0
    rates_const: bool = False
    alphaA: float = 0.0
    alphaB: float = 0.0
    beta: float = 0.0
    bc: list = field(default_factory=lambda: [BC_PERIODIC] * 6)
    cfl: float = 0.9
    inflow: list = field(default_factory=lambda: [0.0] * 6)   # photons/cm^2/s per face (BC_INFLOW)

    @property
    def ngroups(self) -> int:
        return len(self.edges_eV) - 1

    @property
    def c_red(self) -> float:
        return self.c_frac * C_LIGHT

    @property
    def cells(self) -> int:
        return sum(b.ncell for b in self.boxes)

    def nunit(self, box: Box) -> float:
        """Photon-density unit of the stored state: 1e49 photons/s spread over
        one cell face for one cell light-crossing (keeps N = O(1) near
        sources; any positive constant gives the same physics)."""
        return 1e49 / (self.c_red * box.dx * box.dx)


def stromgren(n: int = 32, steps: int = 100, c_frac: float = 0.1) -> Workload:
    """Corner source in a uniform, isothermal (1e4 K) hydrogen box, 1 group.
    The box is one octant of the full-sphere problem: the source cell holds
    Q/8 and the three faces through the source are reflective."""
    dx = 6.6 * KPC / n
    n0 = np.full((n, n, n), 1e-3)
    box = Box(n0=n0, src_cells=np.array([0], dtype=np.int64),
              src_Q=np.array([5e48 / 8.0]), T0=1e4, dx=dx)
    return Workload(name=f"stromgren_{n}^3", boxes=[box], edges_eV=GROUPS_1, T_bb=1e5,
                    c_frac=c_frac, steps=steps, ots=True, isothermal=True,
                    rates_const=True, alphaA=ALPHA_B_1E4, alphaB=ALPHA_B_1E4, beta=0.0,
                    bc=[BC_REFLECTIVE, BC_TRANSMISSIVE] * 3)


def shadow(n: int = 64, steps: int = 3000, c_frac: float = 1.0) -> Workload:
    """The clump test of Sec. 6.5 with static gas (radiative transfer and
    thermochemistry only): a 6.6 kpc box, background 200 atoms/m^3 at
    8000 K, a clump of radius 0.8 kpc centred on (5.4, 3.3, 3.3) kpc with
    40 000 atoms/m^3 at 100 K, a 1e5 K black-body photon flux of
    1e10 photons/m^2/s entering through x = 0, transmissive at x = 6.6 kpc,
    periodic in y and z; 3 groups.  The I-front runs at ~0.17 c in the
    background gas, so the full c is kept (a reduced c below that speed would
    hold the front back)."""
    dx = 6.6 * KPC / n
    c = (np.arange(n) + 0.5) * dx
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r2 = (x - 5.4 * KPC) ** 2 + (y - 3.3 * KPC) ** 2 + (z - 3.3 * KPC) ** 2
    clump = r2 <= (0.8 * KPC) ** 2
    n0 = f32(np.where(clump, 4e4 * 1e-6, 200.0 * 1e-6))
    T = np.where(clump, 100.0, 8000.0)
    box = Box(n0=n0, src_cells=np.zeros(0, dtype=np.int64), src_Q=np.zeros(0), dx=dx, T_field=T)
    return Workload(name=f"shadow_{n}^3", boxes=[box], edges_eV=GROUPS_3, T_bb=1e5, c_frac=c_frac,
                    steps=steps, bc=[BC_INFLOW, BC_TRANSMISSIVE] + [BC_PERIODIC] * 4,
                    inflow=[1e10 * 1e-4, 0.0, 0.0, 0.0, 0.0, 0.0])


def reion(n: int = 128, steps: int = 500, nsrc: int = 64, sigma: float = 1.0,
          slope: float = 2.0, seed: int = 2, lum_seed: int = 102) -> Workload:
    """Lognormal 128^3 box, 64 sources log-uniform in [1e48, 1e50], 3 groups,
    T evolving, c/10, adaptive chemistry steps."""
    n0 = lognormal_field(n, sigma, slope, seed)
    cells = densest_cells(n0, nsrc)
    Q = loguniform_lum(nsrc, lum_seed)
    return Workload(name=f"reion_{n}^3_g3", boxes=[Box(n0=n0, src_cells=cells, src_Q=Q)],
                    edges_eV=GROUPS_3, T_bb=5e4, c_frac=0.1, steps=steps)


def reion_large(n: int = 256, steps: int = 200, nsrc: int = 1024) -> Workload:
    """256^3, sigma = 1.5, P ~ k^-2.5, 1024 sources with Q ~ n0^1.5 (mean 1e49),
    3 groups, c/20, 8 fixed chemistry intervals per step."""
    n0 = lognormal_field(n, 1.5, 2.5, 3)
    cells = densest_cells(n0, nsrc)
    Q = density_lum(n0.reshape(-1)[cells])
    return Workload(name=f"reion_{n}^3_g3_nsub8", boxes=[Box(n0=n0, src_cells=cells, src_Q=Q)],
                    edges_eV=GROUPS_3, T_bb=5e4, c_frac=0.05, steps=steps, nsub=8)


def ensemble(nboxes: int = 64, steps: int = 100, sides=(32, 48, 64, 96), seed: int = 4) -> Workload:
    """Independent periodic boxes of uneven size, 1-16 sources each, 2 groups."""
    rng = np.random.Generator(np.random.PCG64(seed))
    side = rng.choice(np.asarray(sides), size=nboxes)
    nsrc = rng.integers(1, 17, size=nboxes)
    boxes = []
    for b in range(nboxes):
        n0 = lognormal_field(int(side[b]), 1.0, 2.0, 1000 + b)
        cells = densest_cells(n0, int(nsrc[b]))
        Q = loguniform_lum(int(nsrc[b]), 2000 + b)
        boxes.append(Box(n0=n0, src_cells=cells, src_Q=Q))
    return Workload(name=f"ensemble_{nboxes}", boxes=boxes, edges_eV=GROUPS_2, T_bb=5e4,
                    c_frac=0.1, steps=steps)


def adjoint_box(n: int = 64, steps: int = 200, nsrc: int = 16) -> Workload:
    """64^3, sigma = 1, 16 sources, 1 group, 4 fixed chemistry intervals."""
    n0 = lognormal_field(n, 1.0, 2.0, 5)
    cells = densest_cells(n0, nsrc)
    Q = loguniform_lum(nsrc, 105)
    return Workload(name=f"adjoint_{n}^3", boxes=[Box(n0=n0, src_cells=cells, src_Q=Q)],
                    edges_eV=GROUPS_1, T_bb=5e4, c_frac=0.1, steps=steps, nsub=4)


def target_perturbation(nsrc: int, seed: int = 5, scale: float = 0.1) -> np.ndarray:
    """Multiplicative luminosity perturbation exp(scale * z), z ~ N(0, 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(scale * rng.standard_normal(nsrc))


@dataclass
class FineLevel:
    """Refined cells of a CRTA fine level: parent coarse cell (linear index),
    density and initial state of each refined cell."""
    parent: np.ndarray     # int64 [nfine]
    n0: np.ndarray         # [nfine], cm^-3, float32-representable
    xHI: np.ndarray        # [nfine]
    T: np.ndarray          # [nfine]


def refine_densest(box: "Box", frac: float = 0.125, sigma: float = 0.5, seed: int = 7,
                   children: int = 8) -> FineLevel:
    """Split the densest `frac` of the coarse cells into `children` refined
    cells each (ties to the lower index); a child's density is its parent's
    times a lognormal factor (width sigma) normalised so the children's mean
    is the parent's density.  Children start in the parent's initial state."""
    n0 = box.n0.reshape(-1)
    k = max(1, int(round(frac * n0.size)))
    order = np.lexsort((np.arange(n0.size), -n0))
    parents = np.sort(order[:k]).astype(np.int64)
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.exp(sigma * rng.standard_normal((k, children)))
    w /= w.mean(axis=1, keepdims=True)
    nf = f32((n0[parents][:, None] * w).reshape(-1))
    parent = np.repeat(parents, children)
    return FineLevel(parent=parent, n0=nf, xHI=np.full(nf.size, box.xHI0), T=np.full(nf.size, box.T0))


def random_realizable_state(shape, ngroups: int, seed: int, nmax: float = 1.0):
    """Random radiation state with |F| < N in every cell (for transport tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape
    N = rng.uniform(0.0, nmax, (ngroups, nz, ny, nx))
    d = rng.standard_normal((ngroups, nz, ny, nx, 3))
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    f = rng.uniform(0.0, 1.0, (ngroups, nz, ny, nx))
    U = np.empty((ngroups, nz, ny, nx, 4))
    U[..., 0] = N
    U[..., 1:] = d * (f * N)[..., None]
    return U
