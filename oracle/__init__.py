"""FP64 CPU oracle of the M1 radiative-transfer step (test infrastructure).

Thin ctypes/numpy wrapper around ``m1_oracle.c``.  Only the test-suite, the
smoke check and the CPU-baseline leg of the benchmark import this package;
the GPU library never does, and this package imports nothing from it.

The physics (Aubert, Deparis & Ocvirk, arXiv:1508.07888, Secs. 2.2.3-2.2.4)
lives entirely in the C file; this module only marshals arrays.

State layout (all float64, C order):
    U    [G, nz, ny, nx, 4]  = (N/nunit, Fx/(c nunit), Fy/(c nunit), Fz/(c nunit))
    xHI  [nz, ny, nx]        neutral fraction 1 - x
    T    [nz, ny, nx]        K
    n0   [nz, ny, nx]        total hydrogen density, cm^-3
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

from . import build as _build

MAXG = 4
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_INFLOW = 0, 1, 2, 3
ERR_NONFINITE, ERR_SUBCYCLE = 1, 4
NDIAG = 5


class _Params(C.Structure):
    _fields_ = [
        ("G", C.c_int),
        ("sigN", C.c_double * MAXG),
        ("sigE", C.c_double * MAXG),
        ("Eavg", C.c_double * MAXG),
        ("frac", C.c_double * MAXG),
        ("c", C.c_double),
        ("cfl", C.c_double),
        ("ots", C.c_int),
        ("isothermal", C.c_int),
        ("nsub", C.c_int),
        ("rates_const", C.c_int),
        ("alphaA", C.c_double),
        ("alphaB", C.c_double),
        ("beta", C.c_double),
        ("bc", C.c_int * 6),
        ("max_halvings", C.c_int),
        ("flux", C.c_int),
        ("hll", C.POINTER(C.c_double)),
        ("hll_nf", C.c_int),
        ("hll_nm", C.c_int),
        ("inflow", (C.c_double * MAXG) * 6),
    ]

FLUX_GLF, FLUX_HLL = 0, 1


@dataclass
class Params:
    """Oracle run parameters (mirrors ``orc_params``)."""
    sigN: Sequence[float]
    sigE: Sequence[float]
    Eavg: Sequence[float]          # erg
    frac: Sequence[float]
    c: float                       # cm/s, the (reduced) speed of light
    cfl: float = 0.9
    ots: bool = False
    isothermal: bool = False
    nsub: int = 0
    rates_const: bool = False
    alphaA: float = 0.0
    alphaB: float = 0.0
    beta: float = 0.0
    bc: Sequence[int] = field(default_factory=lambda: [BC_PERIODIC] * 6)
    max_halvings: int = 30
    flux: int = FLUX_GLF
    hll_nf: int = 64                # HLL speed table nodes in f (0..1) and mu (-1..1)
    hll_nm: int = 64
    inflow: Sequence = ()           # bc 3: [face] -> stored N^ per group of the incoming beam

    @property
    def G(self) -> int:
        return len(self.sigN)

    def to_c(self) -> _Params:
        p = _Params()
        p.G = self.G
        for i in range(self.G):
            p.sigN[i] = self.sigN[i]
            p.sigE[i] = self.sigE[i]
            p.Eavg[i] = self.Eavg[i]
            p.frac[i] = self.frac[i]
        p.c = self.c
        p.cfl = self.cfl
        p.ots = int(self.ots)
        p.isothermal = int(self.isothermal)
        p.nsub = int(self.nsub)
        p.rates_const = int(self.rates_const)
        p.alphaA, p.alphaB, p.beta = self.alphaA, self.alphaB, self.beta
        for k in range(6):
            p.bc[k] = int(self.bc[k])
        p.max_halvings = int(self.max_halvings)
        p.flux = int(self.flux)
        for f, row in enumerate(self.inflow):
            for g, v in enumerate(row):
                p.inflow[f][g] = float(v)
        if self.flux == FLUX_HLL:
            tab = hll_speed_table(self.hll_nf, self.hll_nm)
            p.hll = tab.ctypes.data_as(C.POINTER(C.c_double))
            p.hll_nf, p.hll_nm = self.hll_nf, self.hll_nm
        return p


_lib = None
_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        PP = C.POINTER(_Params)
        sig = {
            "orc_timestep": (C.c_double, [PP, C.c_double]),
            "orc_courant_number": (C.c_double, [PP, C.c_double]),
            "orc_closure": (C.c_double, [_dp, _dp, _dp, _dp]),
            "orc_glf_flux": (None, [C.c_int, _dp, _dp, _dp]),
            "orc_transport": (None, [PP, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp]),
            "orc_alphaA": (C.c_double, [C.c_double]),
            "orc_alphaB": (C.c_double, [C.c_double]),
            "orc_beta": (C.c_double, [C.c_double]),
            "orc_cool_recA": (C.c_double, [C.c_double]),
            "orc_cool_recB": (C.c_double, [C.c_double]),
            "orc_cool_colion": (C.c_double, [C.c_double]),
            "orc_cool_colexc": (C.c_double, [C.c_double]),
            "orc_cool_brems": (C.c_double, [C.c_double]),
            "orc_cooling": (C.c_double, [PP, C.c_double, C.c_double, C.c_double]),
            "orc_chem_cell": (C.c_int, [PP, C.c_double, C.c_double, C.c_double, _dp, _dp,
                                        _dp, _dp, C.POINTER(C.c_int)]),
            "orc_source_field": (None, [PP, C.c_int64, C.c_int, _i64p, _dp, C.c_double,
                                        C.c_double, _dp]),
            "orc_run": (C.c_int, [PP, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                  _dp, _dp, _dp, _dp, _dp, C.c_int, _dp, _i64p]),
            "orc_run_crta": (C.c_int, [PP, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                       _dp, _dp, _dp, _dp, _dp, C.c_int, _dp, _i64p,
                                       C.c_int64, _i64p, _dp, _dp, _dp]),
            "orc_sigma_HI": (C.c_double, [C.c_double]),
            "orc_transport_cells": (None, [PP, C.c_int, C.c_int, C.c_int, C.c_double, _dp, C.c_int,
                                           C.c_int, _i64p, _dp]),
            "orc_step_cells": (C.c_int, [PP, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                         _dp, _dp, _dp, _dp, _dp, C.c_int, _i64p, _dp, _dp, _dp]),
            "orc_set_threads": (None, [C.c_int]),
            "orc_chem_cell_adj": (C.c_int, [PP, C.c_double, C.c_double, C.c_double, _dp, _dp,
                                            C.c_double, C.c_double, _dp, _dp, _dp, _dp, _dp]),
            "orc_flux_jacobian": (None, [C.c_int, _dp, _dp]),
            "orc_flux_jacobian_fmu": (None, [C.c_double, C.c_double, _dp]),
            "orc_hll_speeds": (None, [PP, C.c_int, _dp, _dp, _dp]),
            "orc_face_flux": (None, [PP, C.c_int, _dp, _dp, _dp]),
            "orc_advance_a": (C.c_double, [C.c_double, C.c_double, C.c_double, C.c_double,
                                           C.c_double]),
            "orc_run_cosmo": (C.c_int, [PP, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                        _dp, _dp, _dp, _dp, _dp, C.c_int, _dp, C.c_double,
                                        C.c_double, C.c_double, _dp]),
            "orc_transport_adj": (C.c_int, [PP, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp,
                                            _dp]),
            "orc_adjoint": (C.c_int, [PP, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                      _dp, _dp, _dp, _dp, _dp, C.c_int, _dp, _dp, _dp]),
            "orc_get_threads": (C.c_int, []),
            "orc_group_table": (None, [C.c_int, _dp, C.c_double, _dp, _dp, _dp, _dp]),
            "orc_group_table_w": (None, [C.c_int, _dp, C.c_double, C.c_int, _dp, _dp, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    if a.dtype == np.int64:
        return a.ctypes.data_as(_i64p)
    raise TypeError(a.dtype)


def set_threads(n: int) -> None:
    """Threads for the oracle's cell loops (results are bit-identical for any n)."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return lib().orc_get_threads()


# ---------------------------------------------------------------- pieces
def timestep(p: Params, dx: float) -> float:
    return lib().orc_timestep(C.byref(p.to_c()), dx)


def courant_number(p: Params, dx: float) -> float:
    return lib().orc_courant_number(C.byref(p.to_c()), dx)


def closure(U4) -> tuple[np.ndarray, float, float, float]:
    """Returns (P6 = Nhat*D as xx,xy,xz,yy,yz,zz ; chi ; a ; g)."""
    U = np.ascontiguousarray(U4, dtype=np.float64)
    P = np.zeros(6)
    a, g = C.c_double(), C.c_double()
    chi = lib().orc_closure(_ptr(U), _ptr(P), C.byref(a), C.byref(g))
    return P, chi, a.value, g.value


def glf_flux(d: int, L, R) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_glf_flux(d, _ptr(L), _ptr(R), _ptr(out))
    return out


def transport(p: Params, U: np.ndarray, lam: float) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    G, nz, ny, nx, four = U.shape
    assert four == 4 and G == p.G
    out = np.empty_like(U)
    lib().orc_transport(C.byref(p.to_c()), nx, ny, nz, lam, _ptr(U), _ptr(out))
    return out


RATE_NAMES = ("alphaA", "alphaB", "beta", "cool_recA", "cool_recB",
              "cool_colion", "cool_colexc", "cool_brems")


def rate(name: str, T: float) -> float:
    assert name in RATE_NAMES
    return getattr(lib(), "orc_" + name)(float(T))


def cooling(p: Params, n0: float, xHI: float, T: float) -> float:
    return lib().orc_cooling(C.byref(p.to_c()), n0, xHI, T)


def chem_cell(p: Params, dt: float, nunit: float, n0: float, S, U, xHI: float, T: float):
    """Thermochemistry of one cell over dt.  Returns (U, xHI, T, ncycles, err)."""
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.float64).reshape(p.G * 4)).copy()
    Sc = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(p.G))
    x, t = C.c_double(xHI), C.c_double(T)
    ncyc = C.c_int()
    err = lib().orc_chem_cell(C.byref(p.to_c()), dt, nunit, n0, _ptr(Sc), _ptr(Uc),
                              C.byref(x), C.byref(t), C.byref(ncyc))
    return Uc.reshape(p.G, 4), x.value, t.value, ncyc.value, err


def source_field(p: Params, shape, cells, Q, dx: float, nunit: float) -> np.ndarray:
    nz, ny, nx = shape
    ncell = nx * ny * nz
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    S = np.zeros((p.G, ncell))
    lib().orc_source_field(C.byref(p.to_c()), ncell, len(cells), _ptr(cells), _ptr(Q),
                           dx, nunit, _ptr(S))
    return S


@dataclass
class RunResult:
    U: np.ndarray
    xHI: np.ndarray
    T: np.ndarray
    hist: np.ndarray
    err: int
    nclamp: int


def run(p: Params, U, xHI, T, n0, dx: float, nunit: float, nsteps: int,
        S: np.ndarray | None = None) -> RunResult:
    """nsteps full steps (transport, chemistry, diagnostics); inputs are copied."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    xHI = np.array(xHI, dtype=np.float64, order="C", copy=True)
    T = np.array(T, dtype=np.float64, order="C", copy=True)
    n0 = np.ascontiguousarray(n0, dtype=np.float64)
    G, nz, ny, nx, _ = U.shape
    assert G == p.G and xHI.shape == (nz, ny, nx) == T.shape == n0.shape
    hist = np.zeros((nsteps, NDIAG))
    ncl = C.c_int64()
    Sp = _ptr(np.ascontiguousarray(S, dtype=np.float64)) if S is not None else None
    if S is not None:
        S = np.ascontiguousarray(S, dtype=np.float64)
        assert S.shape == (G, nx * ny * nz)
        Sp = _ptr(S)
    err = lib().orc_run(C.byref(p.to_c()), nx, ny, nz, dx, nunit, _ptr(U), _ptr(xHI),
                        _ptr(T), _ptr(n0), Sp, nsteps, _ptr(hist), C.byref(ncl))
    return RunResult(U, xHI, T, hist, err, ncl.value)


@dataclass
class CosmoResult:
    run: RunResult
    a: float          # expansion factor after the run


def advance_a(a: float, dt: float, H0: float, Om: float, OL: float) -> float:
    """a after dt (s) from a: one Runge-Kutta step of da/dt = a H0 sqrt(Om/a^3 + OL)."""
    return lib().orc_advance_a(a, dt, H0, Om, OL)


def run_cosmo(p: Params, U, xHI, T_sc, n0, dx: float, nunit: float, nsteps: int, S,
              H0: float, Om: float, OL: float, a0: float) -> CosmoResult:
    """run() in supercomoving units (Sec. 3): U = comoving N^, F^ (units of
    nunit), T_sc = a^2 T, n0 comoving density, dx comoving cell size; a(t)
    from a0 by the Friedmann equation.  The history holds no |F|/N maximum
    (0)."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    xHI = np.array(xHI, dtype=np.float64, order="C", copy=True)
    T = np.array(T_sc, dtype=np.float64, order="C", copy=True)
    n0 = np.ascontiguousarray(n0, dtype=np.float64)
    G, nz, ny, nx, _ = U.shape
    hist = np.zeros((nsteps, NDIAG))
    Sp = None
    if S is not None:
        S = np.ascontiguousarray(S, dtype=np.float64)
        Sp = _ptr(S)
    a = C.c_double(a0)
    err = lib().orc_run_cosmo(C.byref(p.to_c()), nx, ny, nz, dx, nunit, _ptr(U), _ptr(xHI),
                              _ptr(T), _ptr(n0), Sp, nsteps, _ptr(hist), H0, Om, OL, C.byref(a))
    return CosmoResult(RunResult(U, xHI, T, hist, err, 0), a.value)


@dataclass
class CrtaResult:
    coarse: RunResult
    xHI_fine: np.ndarray
    T_fine: np.ndarray


def run_crta(p: Params, U, xHI, T, n0, dx: float, nunit: float, nsteps: int, S,
             parent, n0_fine, xHI_fine, T_fine) -> CrtaResult:
    """run() with a CRTA fine level (Sec. 5): refined cells f run the chemistry
    with the post-transport radiation and the source of their coarse parent
    parent[f] (linear cell index); their radiation result is not kept."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    xHI = np.array(xHI, dtype=np.float64, order="C", copy=True)
    T = np.array(T, dtype=np.float64, order="C", copy=True)
    n0 = np.ascontiguousarray(n0, dtype=np.float64)
    G, nz, ny, nx, _ = U.shape
    parent = np.ascontiguousarray(parent, dtype=np.int64)
    nf = len(parent)
    n0f = np.ascontiguousarray(n0_fine, dtype=np.float64)
    xf = np.array(xHI_fine, dtype=np.float64, copy=True)
    Tf = np.array(T_fine, dtype=np.float64, copy=True)
    assert n0f.shape == xf.shape == Tf.shape == (nf,)
    assert nf == 0 or (parent.min() >= 0 and parent.max() < nx * ny * nz)
    hist = np.zeros((nsteps, NDIAG))
    ncl = C.c_int64()
    Sp = None
    if S is not None:
        S = np.ascontiguousarray(S, dtype=np.float64)
        assert S.shape == (G, nx * ny * nz)
        Sp = _ptr(S)
    err = lib().orc_run_crta(C.byref(p.to_c()), nx, ny, nz, dx, nunit, _ptr(U), _ptr(xHI),
                             _ptr(T), _ptr(n0), Sp, nsteps, _ptr(hist), C.byref(ncl), nf,
                             _ptr(parent), _ptr(n0f), _ptr(xf), _ptr(Tf))
    return CrtaResult(RunResult(U, xHI, T, hist, err, ncl.value), xf, Tf)


def step_cells(p: Params, U, xHI, T, n0, dx: float, nunit: float, cells, S=None):
    """One full step (transport + chemistry) of the listed cells only, from
    the full state.  Returns (U[ncells, G, 4], xHI[ncells], T[ncells], err)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    xHI = np.ascontiguousarray(xHI, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    n0 = np.ascontiguousarray(n0, dtype=np.float64)
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    G, nz, ny, nx, _ = U.shape
    k = len(cells)
    Uo = np.zeros((k, G, 4))
    xo, To = np.zeros(k), np.zeros(k)
    Sp = None
    if S is not None:
        S = np.ascontiguousarray(S, dtype=np.float64)
        Sp = _ptr(S)
    err = lib().orc_step_cells(C.byref(p.to_c()), nx, ny, nz, dx, nunit, _ptr(U), _ptr(xHI),
                               _ptr(T), _ptr(n0), Sp, k, _ptr(cells), _ptr(Uo), _ptr(xo), _ptr(To))
    return Uo, xo, To, err


def chem_cell_adj(p: Params, dt, nunit, n0, S, U, xHI, T, bU, bxHI, bT):
    """Reverse of chem_cell at (U, xHI, T): adjoints of the outputs in, of the
    inputs out.  Returns (bU[G,4], bxHI, bT, dn0, dS[G], n_trials)."""
    Uc = np.ascontiguousarray(np.asarray(U, dtype=np.float64).reshape(p.G * 4))
    Sc = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(p.G))
    b = np.ascontiguousarray(np.asarray(bU, dtype=np.float64).reshape(p.G * 4)).copy()
    bx, bt, dn = C.c_double(bxHI), C.c_double(bT), C.c_double(0.0)
    dS = np.zeros(p.G)
    n = lib().orc_chem_cell_adj(C.byref(p.to_c()), dt, nunit, n0, _ptr(Sc), _ptr(Uc), xHI, T,
                                _ptr(b), C.byref(bx), C.byref(bt), C.byref(dn), _ptr(dS))
    return b.reshape(p.G, 4), bx.value, bt.value, dn.value, dS, n


def flux_jacobian(d: int, U4) -> np.ndarray:
    U = np.ascontiguousarray(U4, dtype=np.float64)
    J = np.zeros((4, 4))
    lib().orc_flux_jacobian(d, _ptr(U), _ptr(J))
    return J


def inflow_density(photon_flux: float, frac, c: float, nunit: float) -> np.ndarray:
    """Stored density N^ per group of an incoming beam (F = c N) carrying
    photon_flux photons/cm^2/s split over the groups by frac."""
    return np.asarray(frac, dtype=np.float64) * photon_flux / (c * nunit)


def flux_jacobian_fmu(f: float, mu: float) -> np.ndarray:
    """Jacobian of the x flux at N = 1, F = f (mu, sqrt(1 - mu^2), 0) on the
    closure's smooth branch (valid up to and at f = 1)."""
    J = np.zeros((4, 4))
    lib().orc_flux_jacobian_fmu(float(f), float(mu), _ptr(J))
    return J


_HLL_TABLES: dict = {}


def hll_speed_table(nf: int = 64, nm: int = 64) -> np.ndarray:
    """Largest eigenvalue of the x-flux Jacobian (units of c) at the nodes
    f_i = 1 - (i/nf)^2, mu_j = -1 + 2j/nm: [nf + 1, nm + 1].  For f < 1 the
    eigenvalues come from numpy's general eigenvalue routine (they are real
    for the M1 system); at f = 1 all four equal mu (free streaming along the
    flux direction), where that routine loses digits on the repeated root."""
    key = (nf, nm)
    if key not in _HLL_TABLES:
        t = np.zeros((nf + 1, nm + 1))
        for i in range(nf + 1):
            f = 1.0 - (i / nf) ** 2
            for j in range(nm + 1):
                mu = -1.0 + 2.0 * j / nm
                if i == 0:
                    t[i, j] = mu
                    continue
                ev = np.linalg.eigvals(flux_jacobian_fmu(f, mu))
                assert np.max(np.abs(ev.imag)) < 1e-6, (i, j, ev)
                t[i, j] = np.max(ev.real)
        _HLL_TABLES[key] = np.ascontiguousarray(t)
    return _HLL_TABLES[key]


def face_flux(p: Params, d: int, L, R) -> np.ndarray:
    """Intercell flux (p.flux: GLF or HLL) between states L and R along d."""
    Lc = np.ascontiguousarray(L, dtype=np.float64)
    Rc = np.ascontiguousarray(R, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_face_flux(C.byref(p.to_c()), d, _ptr(Lc), _ptr(Rc), _ptr(out))
    return out


def hll_speeds(p: Params, d: int, U4) -> tuple[float, float]:
    """(lmin, lmax) of a state along axis d from the interpolated table."""
    U = np.ascontiguousarray(U4, dtype=np.float64)
    a, b = C.c_double(), C.c_double()
    pc = p.to_c()
    lib().orc_hll_speeds(C.byref(pc), d, _ptr(U), C.byref(a), C.byref(b))
    return a.value, b.value


def transport_adj(p: Params, U, lamS, lam: float) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    lamS = np.ascontiguousarray(lamS, dtype=np.float64)
    G, nz, ny, nx, _ = U.shape
    out = np.empty_like(U)
    rc = lib().orc_transport_adj(C.byref(p.to_c()), nx, ny, nz, lam, _ptr(U), _ptr(lamS), _ptr(out))
    assert rc == 0, "adjoint needs periodic boundaries"
    return out


def adjoint(p: Params, U0, xHI0, T0, n0, dx, nunit, nsteps, dLdX, S=None):
    """dL/dS [G, ncell] and dL/dn0 [ncell] of L(X(1..nsteps))."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    G, nz, ny, nx, _ = U0.shape
    ncell = nx * ny * nz
    dS = np.zeros((G, ncell))
    dn0 = np.zeros(ncell)
    dLdX = np.ascontiguousarray(dLdX, dtype=np.float64)
    Sp = None
    if S is not None:
        S = np.ascontiguousarray(S, dtype=np.float64)
        Sp = _ptr(S)
    rc = lib().orc_adjoint(C.byref(p.to_c()), nx, ny, nz, dx, nunit, _ptr(U0),
                           _ptr(np.ascontiguousarray(xHI0, dtype=np.float64)),
                           _ptr(np.ascontiguousarray(T0, dtype=np.float64)),
                           _ptr(np.ascontiguousarray(n0, dtype=np.float64)), Sp, nsteps,
                           _ptr(dLdX), _ptr(dS), _ptr(dn0))
    assert rc == 0, "adjoint needs periodic boundaries"
    return dS, dn0


def sigma_HI(E_eV: float) -> float:
    return lib().orc_sigma_HI(float(E_eV))


def group_table(edges_eV: Sequence[float], T_bb: float, use_sigma: bool = True):
    """Group averages over a black-body photon spectrum.
    Returns dict(sigN, sigE, Eavg [erg], frac), each an array of G floats."""
    e = np.ascontiguousarray(edges_eV, dtype=np.float64)
    G = len(e) - 1
    out = [np.zeros(G) for _ in range(4)]
    lib().orc_group_table_w(G, _ptr(e), float(T_bb), int(use_sigma),
                            *[_ptr(o) for o in out])
    return dict(zip(("sigN", "sigE", "Eavg", "frac"), out))
