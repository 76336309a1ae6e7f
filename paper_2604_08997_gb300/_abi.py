"""ctypes binding of libsipo (include/sipo.h): argument marshalling only.

Every function here carries the name of the C entry point it calls and does
nothing but convert Python / numpy / torch arguments into plain pointers and
sizes.  All computation happens in the CUDA library; when the library is
missing, `load()` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_double, c_int, c_longlong, c_void_p

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
# SIPO_LIBRARY=checked selects the checked build (libsipo_checked.so)
LIB_PATH = os.path.join(PKG, "libsipo_checked.so" if os.environ.get("SIPO_LIBRARY") == "checked"
                        else "libsipo.so")

SIPO_OK = 0
SIPO_ERR_INVALID_ARG, SIPO_ERR_CUDA, SIPO_ERR_TIMEOUT, SIPO_ERR_NUMERIC = -1, -2, -4, -5
SIPO_F32, SIPO_F64, SIPO_BF16 = 0, 1, 2
SIPO_HOST, SIPO_DEVICE = 0, 1
SIPO_GENERAL, SIPO_CASE1, SIPO_CASE2 = 0, 1, 2
SIPO_OPTIMAL, SIPO_PRIMAL_INFEASIBLE, SIPO_DUAL_INFEASIBLE, SIPO_ITER_LIMIT = 0, 1, 2, 3
SIPO_EXT, SIPO_BAND, SIPO_GEL = 0, 1, 2
ARRAY_LABELS, ARRAY_ACTIVE, ARRAY_Y, ARRAY_LAM_UP, ARRAY_LAM_LO, ARRAY_DOSE = range(6)
STATUS_NAMES = {0: "optimal", 1: "primal_infeasible", 2: "dual_infeasible", 3: "iteration_limit"}


class sipo_geometry(Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("n_angles", c_int),
                ("angles", POINTER(c_double)), ("n_det", c_int), ("vial_radius", c_double),
                ("mu", c_double), ("psf_sigma", c_double * 3), ("psf_trunc", c_double)]


class sipo_case_params(Structure):
    _fields_ = [("kase", c_int), ("w1", c_double), ("w2", c_double), ("tol_lo", c_double),
                ("tol_hi", c_double), ("inhibit_ratio", c_double), ("band_width", c_int)]


class sipo_tolerances(Structure):
    _fields_ = [("kkt_tol", c_double), ("max_iter", c_longlong), ("check_every", c_int),
                ("storage", c_int), ("tile_cfg", c_int), ("primal_weight", c_double)]


class sipo_result(Structure):
    _fields_ = [("status", c_int), ("restarts", c_int), ("iters", c_longlong),
                ("kkt", c_double), ("rel_primal", c_double), ("rel_dual", c_double),
                ("rel_gap", c_double), ("r_primal", c_double), ("r_dual", c_double),
                ("gap", c_double), ("pobj", c_double), ("dobj", c_double), ("u", c_double),
                ("v", c_double), ("omega", c_double), ("f_crit", c_double), ("alpha", c_double),
                ("dtvr_f", c_double), ("dsr", c_double), ("psr_f", c_double), ("s", c_double),
                ("solve_ms", c_double), ("kernel_launches", c_longlong), ("tile_cfg", c_int),
                ("cert_slice", c_int)]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class sipo_response(Structure):
    """Richards' response curve (Eq. 4): alpha, k asymptotes, beta rate, gamma shape, f0 location."""
    _fields_ = [("alpha", c_double), ("k", c_double), ("beta", c_double), ("gamma", c_double),
                ("f0", c_double)]


class sipo_response_result(Structure):
    _fields_ = [("alpha", c_double), ("phi", c_double), ("psr_m", c_double), ("dtvr_m", c_double),
                ("ratio_min", c_double), ("ratio_max", c_double), ("m_band_max", c_double),
                ("m_gel_min", c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class SipoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sipo error {code}: {msg}")
        self.code = code


# exported symbols and their C signatures (restype, argtypes)
SIGNATURES = {
    "sipo_create": (c_int, [POINTER(sipo_geometry), c_void_p, c_int, POINTER(sipo_case_params),
                            POINTER(sipo_tolerances), c_void_p, POINTER(c_void_p)]),
    "sipo_solve": (c_int, [c_void_p, c_void_p, c_int, POINTER(sipo_result)]),
    "sipo_solve_batched": (c_int, [POINTER(c_void_p), c_int, POINTER(c_void_p), c_int,
                                   POINTER(sipo_result)]),
    "sipo_create_bounded": (c_int, [POINTER(sipo_geometry), c_void_p, c_void_p, c_void_p, c_int,
                                    POINTER(sipo_case_params), POINTER(sipo_tolerances), c_void_p,
                                    POINTER(c_void_p)]),
    "sipo_response_map": (c_int, [POINTER(sipo_response), c_void_p, c_void_p, c_longlong, c_double, c_int,
                                  c_void_p]),
    "sipo_response_inhibit_ratio": (c_int, [c_void_p, c_void_p, c_longlong, c_double, POINTER(c_double),
                                            POINTER(c_double), c_void_p]),
    "sipo_response_metrics": (c_int, [c_void_p, POINTER(sipo_response), c_void_p, c_int, c_double,
                                      POINTER(sipo_response_result)]),
    "sipo_warm_start": (c_int, [c_void_p, c_void_p]),
    "sipo_set_primal": (c_int, [c_void_p, c_void_p, c_int, c_double, c_double]),
    "sipo_set_primal_from": (c_int, [c_void_p, c_void_p, c_double, c_double, c_double]),
    "sipo_farkas_from": (c_int, [c_void_p, c_void_p, POINTER(c_int), POINTER(c_int)]),
    "sipo_solve_probe": (c_int, [c_void_p, c_void_p, c_longlong, c_void_p, POINTER(c_int), POINTER(c_int)]),
    "sipo_solve_race": (c_int, [c_void_p, c_void_p, c_void_p, c_longlong, c_void_p, c_void_p, POINTER(c_int),
                                POINTER(c_int)]),
    "sipo_get_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, POINTER(c_double)]),
    "sipo_set_state": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, POINTER(c_double)]),
    "sipo_project": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "sipo_backproject": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "sipo_psf_apply": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "sipo_psf_grad": (c_int, [c_void_p, c_void_p, c_void_p, c_int, POINTER(c_double), c_void_p]),
    "sipo_set_psf_sigma": (c_int, [c_void_p, POINTER(c_double)]),
    "sipo_get_array": (c_int, [c_void_p, c_int, c_void_p, c_int]),
    "sipo_profile": (c_int, [c_void_p, c_int, POINTER(c_double), c_int]),
    "sipo_phase_count": (c_int, []),
    "sipo_phase_name": (c_char_p, [c_int]),
    "sipo_tile_count": (c_int, []),
    "sipo_check_flags": (ctypes.c_uint, []),
    "sipo_wait_selftest": (c_int, [c_longlong, c_int, c_int, POINTER(ctypes.c_uint)]),
    "sipo_kernel_launch_count": (c_longlong, []),
    "sipo_set_tolerances": (c_int, [c_void_p, POINTER(sipo_tolerances)]),
    "sipo_get_trace": (c_int, [c_void_p, POINTER(c_double), c_int]),
    "sipo_dose_metrics_noalloc": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_longlong, c_double,
                                          c_double, POINTER(c_double), c_void_p]),
    "sipo_destroy": (c_int, [c_void_p]),
    "sipo_last_error": (c_char_p, []),
}

_lib = None


def load(path: str | None = None):
    """Loads libsipo.so (built in-tree by paper_2604_08997_gb300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with `python -c 'import __graft_entry__ as g; "
                           "g.build()'` (there is no fallback implementation)")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(rc: int):
    if rc != SIPO_OK:
        raise SipoError(rc, load().sipo_last_error().decode())


# ------------------------------------------------------------ marshalling
def _ptr(a):
    """(pointer, location) of a torch tensor or numpy array (must be contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, SIPO_HOST
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (SIPO_DEVICE if a.is_cuda else SIPO_HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _dtype_code(a) -> int:
    s = str(a.dtype)
    if s.endswith("float32"):
        return SIPO_F32
    if s.endswith("float64"):
        return SIPO_F64
    raise TypeError(f"operators take float32 or float64, got {a.dtype}")


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


def _stream(stream):
    """torch's current stream as a cudaStream_t; torch's default stream (handle 0)
    is passed as cudaStreamLegacy so the library orders its work after torch's."""
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                h = torch.cuda.current_stream().cuda_stream
                return ctypes.c_void_p(h if h else CUDA_STREAM_LEGACY)
        except Exception:
            pass
        return ctypes.c_void_p(CUDA_STREAM_LEGACY)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """Owns one sipo_ctx handle (released by sipo_destroy or on collection)."""

    def __init__(self, handle, shape_vol, shape_sino, storage):
        self.handle = handle
        self.vol_shape = shape_vol
        self.sino_shape = shape_sino
        self.storage = storage

    @property
    def compute_dtype(self):
        return SIPO_F64 if self.storage == SIPO_F64 else SIPO_F32

    def __del__(self):
        try:
            if self.handle:
                sipo_destroy(self)
        except Exception:
            pass


def _marshal(geometry: dict, case: dict, tolerances: dict):
    ang = np.ascontiguousarray(np.asarray(geometry["angles"], dtype=np.float64))
    g = sipo_geometry()
    g.nx, g.ny, g.nz = int(geometry["nx"]), int(geometry["ny"]), int(geometry["nz"])
    g.n_angles = ang.size
    g.angles = ang.ctypes.data_as(POINTER(c_double))
    g.n_det = int(geometry["n_det"])
    g.vial_radius = float(geometry.get("vial_radius", 0.0))
    g.mu = float(geometry.get("mu", 0.0))
    sig = geometry.get("psf_sigma", (0.0, 0.0, 0.0))
    for i in range(3):
        g.psf_sigma[i] = float(sig[i])
    g.psf_trunc = float(geometry.get("psf_trunc", 4.0))
    cp = sipo_case_params(int(case.get("kase", 0)), float(case.get("w1", 1.0)),
                          float(case.get("w2", 1.0)), float(case.get("tol_lo", 0.05)),
                          float(case.get("tol_hi", 0.05)), float(case.get("inhibit_ratio", 0.8)),
                          int(case.get("band_width", 10)))
    tl = sipo_tolerances(float(tolerances.get("kkt_tol", 1e-4)),
                         int(tolerances.get("max_iter", 10000)),
                         int(tolerances.get("check_every", 64)),
                         int(tolerances.get("storage", SIPO_F32)),
                         int(tolerances.get("tile_cfg", -1)),
                         float(tolerances.get("primal_weight", 0.0)))
    return g, ang, cp, tl


def _volume(a, g, name):
    if isinstance(a, np.ndarray) and a.dtype != np.float32:
        raise TypeError(f"{name} must be float32")
    expect = g.nx * g.ny * g.nz
    if int(np.prod(a.shape)) != expect:
        raise ValueError(f"{name} has {int(np.prod(a.shape))} elements, geometry needs {expect}")
    return _ptr(a)


def sipo_create(geometry: dict, f_T, case: dict, tolerances: dict, stream=None) -> Context:
    """sipo_create(geo, f_T, location, case, tol, stream, &ctx).

    geometry: nx, ny, nz, angles (radians), n_det, vial_radius, mu, psf_sigma
    (x, y, z), psf_trunc.  f_T: float32 [ny][nx][nz] numpy array or torch
    tensor (host or CUDA).  case: kase, w1, w2, tol_lo, tol_hi, inhibit_ratio,
    band_width.  tolerances: kkt_tol, max_iter, check_every, storage, tile_cfg,
    primal_weight.
    `stream` None: the context creates its own stream.
    """
    lib = load()
    g, ang, cp, tl = _marshal(geometry, case, tolerances)
    ptr, loc = _volume(f_T, g, "f_T")
    out = c_void_p()
    st = c_void_p(0) if stream is None else _stream(stream)
    _check(lib.sipo_create(ctypes.byref(g), c_void_p(ptr), loc, ctypes.byref(cp),
                           ctypes.byref(tl), st, ctypes.byref(out)))
    del ang
    return Context(out, (g.ny, g.nx, g.nz), (g.n_angles, g.n_det, g.nz), tl.storage)


def sipo_create_bounded(geometry: dict, f_T, f_L, f_U, case: dict, tolerances: dict,
                        stream=None) -> Context:
    """sipo_create_bounded(geo, f_T, f_L, f_U, location, case, tol, stream, &ctx):
    Case 1 with explicit per-voxel dose bounds f_L <= f_U on gel (all three
    float32 [ny][nx][nz], on one side: host or CUDA)."""
    lib = load()
    g, ang, cp, tl = _marshal(geometry, dict(case, kase=SIPO_CASE1), tolerances)
    pt, loc = _volume(f_T, g, "f_T")
    pl, ll = _volume(f_L, g, "f_L")
    pu, lu = _volume(f_U, g, "f_U")
    if not (loc == ll == lu):
        raise ValueError("f_T, f_L and f_U must all be on the host or all on the device")
    out = c_void_p()
    st = c_void_p(0) if stream is None else _stream(stream)
    _check(lib.sipo_create_bounded(ctypes.byref(g), c_void_p(pt), c_void_p(pl), c_void_p(pu), loc,
                                   ctypes.byref(cp), ctypes.byref(tl), st, ctypes.byref(out)))
    del ang
    return Context(out, (g.ny, g.nx, g.nz), (g.n_angles, g.n_det, g.nz), tl.storage)


def _response(M) -> sipo_response:
    if isinstance(M, sipo_response):
        return M
    if isinstance(M, dict):
        return sipo_response(float(M["alpha"]), float(M["k"]), float(M["beta"]), float(M["gamma"]),
                             float(M["f0"]))
    return sipo_response(*[float(x) for x in M])


def sipo_response_map(M, src, dst, inverse: bool, scale: float = 1.0, stream=None):
    """dst = M(scale src) (Eq. 4) or, inverse, M^-1(scale src) (Eq. 5); float32 CUDA tensors."""
    ps, ls = _ptr(src)
    pd, ld = _ptr(dst)
    if ls != SIPO_DEVICE or ld != SIPO_DEVICE:
        raise ValueError("the response map takes device tensors")
    if src.numel() != dst.numel() or str(src.dtype) != "torch.float32" or str(dst.dtype) != "torch.float32":
        raise ValueError("src and dst must be float32 tensors of one size")
    r = _response(M)
    _check(load().sipo_response_map(ctypes.byref(r), c_void_p(ps), c_void_p(pd), int(src.numel()),
                                    float(scale), 1 if inverse else 0, _stream(stream)))
    return dst


def sipo_response_inhibit_ratio(M, m_T, m_crit: float, stream=None) -> tuple[float, float]:
    """Case-2 ratio M^-1(m_crit) / M^-1(min_gel m_T) computed on the device
    (see include/sipo.h); returns (ratio, smallest prescribed response)."""
    if str(m_T.dtype) not in ("torch.float32", "float32"):
        raise ValueError("m_T must be float32")
    p, loc = _ptr(m_T)
    if loc == SIPO_HOST:
        raise ValueError("m_T must be a device tensor")
    r = sipo_response(*M)
    ratio, gmin = c_double(0.0), c_double(0.0)
    _check(load().sipo_response_inhibit_ratio(ctypes.byref(r), c_void_p(p), int(m_T.numel()), float(m_crit),
                                              ctypes.byref(ratio), ctypes.byref(gmin), _stream(stream)))
    return float(ratio.value), float(gmin.value)


def sipo_response_metrics(ctx: Context, M, m_T, alpha: float = 0.0) -> dict:
    """Response-domain post-scaling (Eq. 28; alpha <= 0: minimised) and metrics (Eq. 46)
    of ctx's last solve; m_T float32 [ny][nx][nz], host or CUDA."""
    p, loc = _ptr(m_T)
    if isinstance(m_T, np.ndarray) and m_T.dtype != np.float32:
        raise TypeError("m_T must be float32")
    r = _response(M)
    out = sipo_response_result()
    _check(load().sipo_response_metrics(ctx.handle, ctypes.byref(r), c_void_p(p), loc, float(alpha),
                                        ctypes.byref(out)))
    return out.as_dict()


def sipo_solve(ctx: Context, y_out=None) -> dict:
    """sipo_solve(ctx, y_out, location, &result); returns the result as a dict."""
    res = sipo_result()
    if y_out is None:
        ptr, loc = 0, SIPO_HOST
    else:
        ptr, loc = _ptr(y_out)
    _check(load().sipo_solve(ctx.handle, c_void_p(ptr), loc, ctypes.byref(res)))
    return res.as_dict()


def sipo_warm_start(dst: Context, src: Context) -> None:
    """sipo_warm_start(dst, src): dst's next solve starts from src's last T(z)."""
    _check(load().sipo_warm_start(dst.handle, src.handle))


def sipo_set_primal(ctx: Context, y, u: float = -1.0, v: float = -1.0) -> None:
    """sipo_set_primal(ctx, y, location, u, v): ctx's next solve starts from
    the primal point y (host or device, the compute dtype, [n_angles][n_det][nz])
    with u~ = u, v~ = v (negative: the smallest the point allows) and zero duals."""
    p, loc = _ptr(y)
    _check(load().sipo_set_primal(ctx.handle, c_void_p(p), loc, float(u), float(v)))


def sipo_set_primal_from(dst: Context, src: Context, scale: float = 1.0, u: float = -1.0,
                         v: float = -1.0) -> None:
    """sipo_set_primal_from(dst, src, scale, u, v): dst's next solve starts from
    scale times the point src's last solve returned, without leaving the device."""
    _check(load().sipo_set_primal_from(dst.handle, src.handle, float(scale), float(u), float(v)))


def sipo_farkas_from(ctx: Context, src: Context) -> tuple[bool, int]:
    """sipo_farkas_from(ctx, src): does src's last dual point prove ctx's LP
    infeasible?  Returns (certified, slice or -1)."""
    cert, sl = c_int(0), c_int(-1)
    _check(load().sipo_farkas_from(ctx.handle, src.handle, ctypes.byref(cert), ctypes.byref(sl)))
    return bool(cert.value), int(sl.value)


def sipo_solve_probe(ctx: Context, target: Context, probe_every: int = 1024) -> tuple[dict, bool, int]:
    """sipo_solve of ctx, testing its dual point as a Farkas ray of target's LP
    every probe_every iterations; returns (result, certified, slice or -1)."""
    res = sipo_result()
    cert, sl = c_int(0), c_int(-1)
    _check(load().sipo_solve_probe(ctx.handle, target.handle, int(probe_every), ctypes.byref(res),
                                   ctypes.byref(cert), ctypes.byref(sl)))
    return res.as_dict(), bool(cert.value), int(sl.value)


def sipo_solve_race(ctx: Context, target: Context, rival: Context, probe_every: int = 1024
                    ) -> tuple[dict, dict, bool, int]:
    """sipo_solve_probe of ctx (Farkas probes of target) with rival solved at
    the same time on its own stream; returns (ctx's result, rival's result,
    certified, slice or -1)."""
    res, rres = sipo_result(), sipo_result()
    cert, sl = c_int(0), c_int(-1)
    _check(load().sipo_solve_race(ctx.handle, target.handle, rival.handle, int(probe_every), ctypes.byref(res),
                                  ctypes.byref(rres), ctypes.byref(cert), ctypes.byref(sl)))
    return res.as_dict(), rres.as_dict(), bool(cert.value), int(sl.value)


def sipo_get_state(ctx: Context, y, lam_up, lam_lo) -> dict:
    """Checkpoint: T(z) of ctx's last check into y [n_angles*n_det*nz], lam_up, lam_lo
    [ny*nx*nz] (compute dtype, all host or all CUDA); returns u, v, omega, iters."""
    py, ly = _ptr(y)
    pu, lu = _ptr(lam_up)
    pl, ll = _ptr(lam_lo)
    if not (ly == lu == ll):
        raise ValueError("y, lam_up and lam_lo must all be on the host or all on the device")
    sc = (c_double * 4)()
    _check(load().sipo_get_state(ctx.handle, c_void_p(py), c_void_p(pu), c_void_p(pl), ly, sc))
    return {"u": sc[0], "v": sc[1], "omega": sc[2], "iters": int(sc[3])}


def sipo_set_state(ctx: Context, y, lam_up, lam_lo, u: float = -1.0, v: float = -1.0,
                   omega: float = -1.0) -> None:
    """Resume: ctx's next solve starts from (y, lam_up, lam_lo, u~, v~, omega)."""
    py, ly = _ptr(y)
    pu, lu = _ptr(lam_up)
    pl, ll = _ptr(lam_lo)
    if not (ly == lu == ll):
        raise ValueError("y, lam_up and lam_lo must all be on the host or all on the device")
    sc = (c_double * 4)(float(u), float(v), float(omega), 0.0)
    _check(load().sipo_set_state(ctx.handle, c_void_p(py), c_void_p(pu), c_void_p(pl), ly, sc))


def sipo_solve_batched(ctxs, y_outs=None) -> list[dict]:
    n = len(ctxs)
    arr = (c_void_p * n)(*[c.handle.value if isinstance(c.handle, c_void_p) else c.handle for c in ctxs])
    results = (sipo_result * n)()
    loc = SIPO_HOST
    yo = None
    if y_outs is not None:
        ptrs = []
        for y in y_outs:
            if y is None:
                ptrs.append(0)
            else:
                p, loc = _ptr(y)
                ptrs.append(p)
        yo = (c_void_p * n)(*ptrs)
    _check(load().sipo_solve_batched(arr, n, yo, loc, results))
    return [r.as_dict() for r in results]


def sipo_project(ctx: Context, vol, sino, stream=None):
    """sino = A vol = P_mu K vol (device tensors of the context's compute dtype)."""
    pv, lv = _ptr(vol)
    ps, ls = _ptr(sino)
    if lv != SIPO_DEVICE or ls != SIPO_DEVICE:
        raise ValueError("operators take device tensors")
    _check(load().sipo_project(ctx.handle, c_void_p(pv), c_void_p(ps), _dtype_code(vol),
                               _stream(stream)))
    return sino


def sipo_backproject(ctx: Context, sino, vol, stream=None):
    """vol = A^T sino = K P_mu^T sino."""
    ps, ls = _ptr(sino)
    pv, lv = _ptr(vol)
    if lv != SIPO_DEVICE or ls != SIPO_DEVICE:
        raise ValueError("operators take device tensors")
    _check(load().sipo_backproject(ctx.handle, c_void_p(ps), c_void_p(pv), _dtype_code(sino),
                                   _stream(stream)))
    return vol


def sipo_psf_apply(ctx: Context, vin, vout, deriv_axis: int = -1, stream=None):
    pi, _ = _ptr(vin)
    po, _ = _ptr(vout)
    _check(load().sipo_psf_apply(ctx.handle, c_void_p(pi), c_void_p(po), _dtype_code(vin),
                                 int(deriv_axis), _stream(stream)))
    return vout


def sipo_psf_grad(ctx: Context, sino, vol, stream=None) -> np.ndarray:
    ps, _ = _ptr(sino)
    pv, _ = _ptr(vol)
    g = (c_double * 3)()
    _check(load().sipo_psf_grad(ctx.handle, c_void_p(ps), c_void_p(pv), _dtype_code(sino), g,
                                _stream(stream)))
    return np.array(list(g))


def sipo_set_psf_sigma(ctx: Context, sigma):
    s = (c_double * 3)(*[float(x) for x in sigma])
    _check(load().sipo_set_psf_sigma(ctx.handle, s))


def sipo_get_array(ctx: Context, which: int, out):
    p, loc = _ptr(out)
    _check(load().sipo_get_array(ctx.handle, int(which), c_void_p(p), loc))
    return out


def sipo_profile(ctx: Context, iters: int) -> dict:
    lib = load()
    n = lib.sipo_phase_count()
    ms = (c_double * n)()
    _check(lib.sipo_profile(ctx.handle, int(iters), ms, n))
    return {lib.sipo_phase_name(i).decode(): ms[i] for i in range(n)}


def sipo_kernel_launch_count() -> int:
    return int(load().sipo_kernel_launch_count())


def sipo_tile_count() -> int:
    """Entries of the backprojector tile table (values of tolerances["tile_cfg"])."""
    return int(load().sipo_tile_count())


def sipo_wait_selftest(budget_cycles: int, arrive: bool, threads: int = 128) -> tuple[int, int]:
    """Runs the staged backprojector's bounded mbarrier wait on its own (see
    include/sipo.h); returns (library return code, threads whose wait gave
    up).  SIPO_ERR_TIMEOUT is the expected code when `arrive` is False."""
    out = ctypes.c_uint(0)
    rc = load().sipo_wait_selftest(int(budget_cycles), int(bool(arrive)), int(threads), ctypes.byref(out))
    if rc not in (SIPO_OK, SIPO_ERR_TIMEOUT):
        _check(rc)
    return int(rc), int(out.value)


def sipo_set_tolerances(ctx: Context, kkt_tol: float, max_iter: int, check_every: int = 64,
                        storage: int | None = None):
    tl = sipo_tolerances(float(kkt_tol), int(max_iter), int(check_every),
                         int(ctx.storage if storage is None else storage), -1, 0.0)
    _check(load().sipo_set_tolerances(ctx.handle, ctypes.byref(tl)))


TRACE_FIELDS = ("k", "kkt", "rel_primal", "rel_dual", "rel_gap", "pobj", "omega", "restarts",
                "farkas_epoch", "farkas_residual")


def sipo_get_trace(ctx: Context, max_entries: int = 4096) -> np.ndarray:
    """Per-check convergence trace of the last solve, shape (n, 10) (TRACE_FIELDS)."""
    buf = np.zeros((max_entries, len(TRACE_FIELDS)), np.float64)
    n = load().sipo_get_trace(ctx.handle, buf.ctypes.data_as(POINTER(c_double)), int(max_entries))
    if n < 0:
        _check(n)
    return buf[:n].copy()


def sipo_dose_metrics_noalloc(dose, labels, f_T, f_crit: float, lower_scale: float,
                              stream=None) -> np.ndarray:
    """Metrics of a device dose field without device allocation (see include/sipo.h):
    returns [dtvr_f, dsr, psr_f, alpha, s].

    dose (float32 or float64), labels (uint8) and f_T (float32) must be device
    tensors of the same number of elements on one device; anything else is
    refused here, before the library is called, because the kernel reads
    n = dose.numel() elements of each."""
    if str(labels.dtype) not in ("torch.uint8", "uint8"):
        raise ValueError(f"labels must be uint8, got {labels.dtype}")
    if str(f_T.dtype) not in ("torch.float32", "float32"):
        raise ValueError(f"f_T must be float32, got {f_T.dtype}")
    code = _dtype_code(dose)
    n = int(dose.numel()) if hasattr(dose, "numel") else int(dose.size)
    for name, a in (("labels", labels), ("f_T", f_T)):
        m = int(a.numel()) if hasattr(a, "numel") else int(a.size)
        if m != n:
            raise ValueError(f"{name} has {m} elements, dose has {n}")
    pd, ld = _ptr(dose)
    pl, ll = _ptr(labels)
    pf, lf = _ptr(f_T)
    if SIPO_HOST in (ld, ll, lf):
        raise ValueError("dose, labels and f_T must be device tensors")
    if not (dose.device == labels.device == f_T.device):
        raise ValueError("dose, labels and f_T must be on one device")
    out = (c_double * 5)()
    _check(load().sipo_dose_metrics_noalloc(c_void_p(pd), code, c_void_p(pl),
                                            c_void_p(pf), n, float(f_crit),
                                            float(lower_scale), out, _stream(stream)))
    return np.array(list(out))


def sipo_destroy(ctx: Context):
    if ctx.handle:
        load().sipo_destroy(ctx.handle)
        ctx.handle = None
