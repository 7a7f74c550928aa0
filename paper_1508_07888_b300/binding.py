"""ctypes binding of librt_m1.so (include/rt_m1.h), same names as the C ABI.

Argument marshalling only: every step of the radiative-transfer path runs in
the library's CUDA kernels.  Device memory and streams come from PyTorch.
``lib()`` raises if the library cannot be loaded (there is no CPU fallback).

``Solver`` wraps one handle: it owns the torch device tensors of the state of
each box and forwards to rt_step / rt_set_sources / rt_upload / rt_download.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "librt_m1.so")

RT_MAX_GROUPS = 4
RT_NDIAG = 5
RT_OK, RT_ERR_ARG, RT_ERR_CUDA, RT_ERR_NONFINITE = 0, -1, -2, -3
RT_ERR_REALIZABILITY, RT_ERR_SUBCYCLE, RT_ERR_TIMEOUT, RT_ERR_STATE = -4, -5, -6, -7
RT_ERR_TOO_LARGE = -8
RT_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024
RT_PREC_SPLIT, RT_PREC_FP64, RT_PREC_FP64_STRICT = 0, 1, 2
RT_BC_PERIODIC, RT_BC_TRANSMISSIVE, RT_BC_REFLECTIVE = 0, 1, 2
DIAG_NAMES = ("ionised_fraction", "photons", "max_flux_ratio", "n_ionised", "mean_subcycles")


class rt_params(C.Structure):
    _fields_ = [
        ("ngroups", C.c_int),
        ("sigN", C.c_double * RT_MAX_GROUPS),
        ("sigE", C.c_double * RT_MAX_GROUPS),
        ("Eavg", C.c_double * RT_MAX_GROUPS),
        ("frac", C.c_double * RT_MAX_GROUPS),
        ("c_red", C.c_double),
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
        ("precision", C.c_int),
        ("tune", C.c_int),
        ("flux", C.c_int),
        ("inflow", C.c_double * 6),
        ("cosmo", C.c_int),
        ("H0", C.c_double), ("omega_m", C.c_double), ("omega_l", C.c_double),
        ("a0", C.c_double),
        ("chem_tune", C.c_int),
    ]


class rt_box(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double),
        ("nunit", C.c_double),
        ("U", C.c_void_p),
        ("xHI", C.c_void_p),
        ("T", C.c_void_p),
        ("n0", C.c_void_p),
    ]


class rt_stats(C.Structure):
    _fields_ = [
        ("steps", C.c_int64),
        ("realizability_clamps", C.c_int64),
        ("error_bits", C.c_int),
        ("nboxes", C.c_int),
        ("cells", C.c_int64),
        ("last_diag", C.c_double * RT_NDIAG),
        ("kernel_ms", C.c_double * 3),
        ("kernel_launches", C.c_int64 * 3),
        ("tile_x", C.c_int), ("tile_y", C.c_int),
        ("transport_grid", C.c_int), ("chem_grid", C.c_int),
        ("a", C.c_double),
        ("transport_zchunk", C.c_int),
        ("transport_tma", C.c_int),
        ("transport_lockstep", C.c_int),
        ("chem_grab", C.c_int),
        ("transport_gpb", C.c_int),
    ]


EXPORTS = ("rt_create", "rt_set_sources", "rt_step", "rt_upload", "rt_download", "rt_query",
           "rt_set_profiling", "rt_last_error", "rt_destroy", "rt_timestep", "rt_group_table",
           "rt_transport_static", "rt_adjoint", "rt_set_fine", "rt_hll_speeds")
KERNELS = ("transport", "chemistry", "fine_chemistry")   # chemistry includes the diagnostics

_lib = None


def lib(build_if_missing: bool = True):
    """Load librt_m1.so (building it in-tree with nvcc when it is missing or
    older than its sources).  Raises RuntimeError if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        try:
            from . import build as _build
            _build.build()
        except Exception as e:  # nvcc missing: only an existing library can be used
            if not os.path.exists(LIBPATH):
                raise RuntimeError(f"librt_m1.so is missing and cannot be built: {e}") from e
    if not os.path.exists(LIBPATH):
        raise RuntimeError(f"librt_m1.so not found at {LIBPATH}")
    L = C.CDLL(LIBPATH)
    vp, dp, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
    sig = {
        "rt_create": (C.c_int, [C.POINTER(vp), C.POINTER(rt_params), C.POINTER(rt_box), C.c_int, vp]),
        "rt_set_sources": (C.c_int, [vp, C.c_int, C.c_int, i64p, dp]),
        "rt_set_fine": (C.c_int, [vp, C.c_int, C.c_int64, vp, vp, vp, vp]),
        "rt_hll_speeds": (C.c_int, [C.c_int, C.c_int, dp]),
        "rt_step": (C.c_int, [vp, C.c_int, vp]),
        "rt_upload": (C.c_int, [vp, C.c_int, vp, vp, vp, vp]),
        "rt_download": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "rt_query": (C.c_int, [vp, C.POINTER(rt_stats)]),
        "rt_set_profiling": (C.c_int, [vp, C.c_int]),
        "rt_last_error": (C.c_char_p, [vp]),
        "rt_destroy": (None, [vp]),
        "rt_timestep": (C.c_double, [C.POINTER(rt_params), C.c_double]),
        "rt_group_table": (C.c_int, [C.c_int, dp, C.c_double, dp, dp, dp, dp]),
        "rt_transport_static": (C.c_int, [C.POINTER(rt_params), C.POINTER(rt_box), C.c_int, vp]),
        "rt_adjoint": (C.c_int, [vp, vp, vp, vp, C.c_int, C.c_int, vp, dp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


class RTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rt error {code}: {msg}")
        self.code = code


def _check(code: int, handle=None):
    if code != RT_OK:
        raise RTError(code, lib().rt_last_error(handle).decode())


# ------------------------------------------------------------------ same names
def rt_group_table(edges_eV, T_bb: float):
    e = np.ascontiguousarray(edges_eV, dtype=np.float64)
    G = len(e) - 1
    out = [np.zeros(G) for _ in range(4)]
    dp = C.POINTER(C.c_double)
    _check(lib().rt_group_table(G, e.ctypes.data_as(dp), float(T_bb),
                                *[o.ctypes.data_as(dp) for o in out]))
    return dict(zip(("sigN", "sigE", "Eavg", "frac"), out))


def rt_timestep(p: rt_params, dx: float) -> float:
    return lib().rt_timestep(C.byref(p), float(dx))


def rt_create(p: rt_params, boxes, stream_ptr: int = 0):
    arr = (rt_box * len(boxes))(*boxes)
    h = C.c_void_p()
    _check(lib().rt_create(C.byref(h), C.byref(p), arr, len(boxes), C.c_void_p(stream_ptr)))
    return h


def rt_set_sources(h, box: int, cells, Q):
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    assert cells.shape == Q.shape
    _check(lib().rt_set_sources(h, box, len(cells), cells.ctypes.data_as(C.POINTER(C.c_int64)),
                                Q.ctypes.data_as(C.POINTER(C.c_double))), h)


RT_FLUX_GLF, RT_FLUX_HLL = 0, 1


def rt_hll_speeds(nf: int = 64, nm: int = 64) -> np.ndarray:
    """The library's HLL wave-speed table, [nf + 1, nm + 1] (host helper)."""
    out = np.zeros((nf + 1, nm + 1))
    _check(lib().rt_hll_speeds(nf, nm, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def rt_set_fine(h, box: int, nfine: int, parent_ptr: int, n0_ptr: int, xHI_ptr: int, T_ptr: int):
    """CRTA fine level of a box (device pointers; nfine = 0 removes it)."""
    _check(lib().rt_set_fine(h, box, int(nfine), C.c_void_p(parent_ptr or None),
                             C.c_void_p(n0_ptr or None), C.c_void_p(xHI_ptr or None),
                             C.c_void_p(T_ptr or None)), h)


def rt_step(h, nsteps: int, hist_ptr: int = 0) -> int:
    """Returns the status (raises only on argument/CUDA errors); device-side
    errors (sub-cycle cap, non-finite) are returned for the caller to judge."""
    code = lib().rt_step(h, int(nsteps), C.c_void_p(hist_ptr or None))
    if code in (RT_ERR_ARG, RT_ERR_CUDA, RT_ERR_STATE):
        _check(code, h)
    return code


def rt_upload(h, box: int, U=None, xHI=None, T=None, n0=None):
    ptr = [None if a is None else C.c_void_p(a.ctypes.data) for a in (U, xHI, T, n0)]
    _check(lib().rt_upload(h, box, *ptr), h)


def rt_download(h, box: int, U=None, xHI=None, T=None):
    ptr = [None if a is None else C.c_void_p(a.ctypes.data) for a in (U, xHI, T)]
    _check(lib().rt_download(h, box, *ptr), h)


def rt_query(h) -> rt_stats:
    st = rt_stats()
    _check(lib().rt_query(h, C.byref(st)), h)
    return st


def rt_set_profiling(h, on: bool) -> None:
    _check(lib().rt_set_profiling(h, int(bool(on))), h)


def rt_last_error(h=None) -> str:
    return lib().rt_last_error(h).decode()


def rt_destroy(h) -> None:
    lib().rt_destroy(h)


def rt_adjoint(h, U0_ptr: int, xHI0_ptr: int, T0_ptr: int, nsteps: int, ckpt_every: int,
               dLdX_ptr: int, nsrc: int, dLdn0_ptr: int):
    """Gradient of a loss of the ionised-fraction history (see include/rt_m1.h).
    Returns (status, dL/dQ as a numpy array of nsrc doubles)."""
    dQ = np.zeros(max(nsrc, 1))
    code = lib().rt_adjoint(h, C.c_void_p(U0_ptr), C.c_void_p(xHI0_ptr), C.c_void_p(T0_ptr),
                            int(nsteps), int(ckpt_every), C.c_void_p(dLdX_ptr),
                            dQ.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(dLdn0_ptr))
    if code in (RT_ERR_ARG, RT_ERR_CUDA, RT_ERR_STATE):
        _check(code, h)
    return code, dQ[:nsrc]


def rt_transport_static(p: rt_params, box: rt_box, nsteps: int, stream_ptr: int = 0) -> int:
    """Transport steps that allocate no device memory (see include/rt_m1.h);
    returns the status code."""
    return lib().rt_transport_static(C.byref(p), C.byref(box), int(nsteps), C.c_void_p(stream_ptr or None))


# ------------------------------------------------------------------ helpers
def make_params(ngroups: int, table: dict, c_red: float, *, cfl=0.9, ots=False, isothermal=False,
                nsub=0, rates_const=False, alphaA=0.0, alphaB=0.0, beta=0.0, bc=(0,) * 6,
                max_halvings=30, precision=RT_PREC_SPLIT, tune=0, flux=0, chem_tune=0,
                inflow=(0.0,) * 6, cosmo=None) -> rt_params:
    """cosmo: None, or (H0 [1/s], omega_m, omega_l, a0) for supercomoving units."""
    p = rt_params()
    p.ngroups = ngroups
    for i in range(ngroups):
        p.sigN[i], p.sigE[i] = table["sigN"][i], table["sigE"][i]
        p.Eavg[i], p.frac[i] = table["Eavg"][i], table["frac"][i]
    p.c_red, p.cfl = c_red, cfl
    p.ots, p.isothermal, p.nsub, p.rates_const = int(ots), int(isothermal), int(nsub), int(rates_const)
    p.alphaA, p.alphaB, p.beta = alphaA, alphaB, beta
    for k in range(6):
        p.bc[k] = int(bc[k])
    p.max_halvings = max_halvings
    p.precision = precision
    p.tune = int(tune)
    p.chem_tune = int(chem_tune)
    p.flux = int(flux)
    for k in range(6):
        p.inflow[k] = float(inflow[k])
    if cosmo is not None:
        p.cosmo = 1
        p.H0, p.omega_m, p.omega_l, p.a0 = (float(v) for v in cosmo)
    return p


@dataclass
class BoxState:
    """Torch device tensors of one box (owned by the caller of the library)."""
    U: "object"       # [G, nz, ny, nx, 4] float32 or float64
    xHI: "object"     # [nz, ny, nx] float64
    T: "object"       # [nz, ny, nx] float64
    n0: "object"      # [nz, ny, nx] float32 or float64
    dx: float
    nunit: float


class Solver:
    """One rt_handle over boxes whose state lives in torch CUDA tensors."""

    def __init__(self, params: rt_params, states: list[BoxState], stream=None):
        import torch
        self.torch = torch
        self.params = params
        self.states = states
        self.fp64 = params.precision != RT_PREC_SPLIT
        boxes = []
        for s in states:
            G, nz, ny, nx, _ = s.U.shape
            assert G == params.ngroups
            want = torch.float64 if self.fp64 else torch.float32
            assert s.U.dtype == want and s.n0.dtype == want and s.U.is_contiguous()
            assert s.xHI.dtype == torch.float64 and s.T.dtype == torch.float64
            b = rt_box()
            b.nx, b.ny, b.nz = nx, ny, nz
            b.dx, b.nunit = s.dx, s.nunit
            b.U, b.xHI, b.T, b.n0 = s.U.data_ptr(), s.xHI.data_ptr(), s.T.data_ptr(), s.n0.data_ptr()
            boxes.append(b)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.h = rt_create(params, boxes, self.stream.cuda_stream)

    @classmethod
    def from_numpy(cls, params: rt_params, boxes_np, device="cuda"):
        """boxes_np: iterable of (U, xHI, T, n0, dx, nunit) numpy arrays/values."""
        import torch
        fp = torch.float64 if params.precision != RT_PREC_SPLIT else torch.float32
        states = []
        for U, xHI, T, n0, dx, nunit in boxes_np:
            states.append(BoxState(
                U=torch.as_tensor(np.ascontiguousarray(U), dtype=fp, device=device).contiguous(),
                xHI=torch.as_tensor(np.ascontiguousarray(xHI), dtype=torch.float64, device=device),
                T=torch.as_tensor(np.ascontiguousarray(T), dtype=torch.float64, device=device),
                n0=torch.as_tensor(np.ascontiguousarray(n0), dtype=fp, device=device),
                dx=float(dx), nunit=float(nunit)))
        return cls(params, states)

    def set_sources(self, box: int, cells, Q):
        rt_set_sources(self.h, box, cells, Q)

    def set_fine(self, box: int, parent, n0, xHI, T):
        """CRTA fine level of a box from torch device tensors (kept referenced:
        the library keeps pointers to n0, xHI and T)."""
        t = self.torch
        fp = t.float64 if self.fp64 else t.float32
        parent = t.as_tensor(parent, dtype=t.int64, device="cuda").contiguous()
        n0 = t.as_tensor(n0, dtype=fp, device="cuda").contiguous()
        xHI = t.as_tensor(xHI, dtype=t.float64, device="cuda").contiguous()
        T = t.as_tensor(T, dtype=t.float64, device="cuda").contiguous()
        assert parent.shape == n0.shape == xHI.shape == T.shape and parent.dim() == 1
        self.fine = getattr(self, "fine", {})
        self.fine[box] = (parent, n0, xHI, T)
        rt_set_fine(self.h, box, parent.numel(), parent.data_ptr(), n0.data_ptr(),
                    xHI.data_ptr(), T.data_ptr())
        return xHI, T

    def step(self, nsteps: int, hist=None) -> int:
        return rt_step(self.h, nsteps, hist.data_ptr() if hist is not None else 0)

    def run(self, nsteps: int):
        """nsteps steps; returns (status, history [nsteps, nboxes, RT_NDIAG] numpy)."""
        hist = self.torch.zeros((max(nsteps, 1), len(self.states), RT_NDIAG),
                                dtype=self.torch.float64, device=self.states[0].U.device)
        code = self.step(nsteps, hist)
        return code, hist[:nsteps].cpu().numpy()

    def stats(self) -> rt_stats:
        return rt_query(self.h)

    def numpy_state(self, box: int = 0):
        s = self.states[box]
        self.torch.cuda.synchronize()
        return (s.U.double().cpu().numpy(), s.xHI.cpu().numpy(), s.T.cpu().numpy())

    def close(self):
        if getattr(self, "h", None):
            rt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
