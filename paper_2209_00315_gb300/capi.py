"""ctypes binding of the C ABI in include/ot.h (argument marshalling only).

Every function keeps the name of its C entry point.  Arrays are torch float64
tensors: CUDA tensors are passed as device pointers (``memspace = DEVICE``)
and the work runs on the current torch stream; CPU tensors or numpy arrays are
passed as host pointers (``memspace = HOST``), for the calls that accept them.
The shared library ``libotgb.so`` must have been built (``build.build()``);
there is no other implementation behind these functions.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libotgb.so")

OT_OK = 0
STATUS = {0: "OT_OK", 1: "OT_ERR_INVALID_ARG", 2: "OT_ERR_MASS_MISMATCH", 3: "OT_ERR_NEGATIVE_DENSITY",
          4: "OT_ERR_NOT_CONVERGED", 5: "OT_ERR_BREAKDOWN", 6: "OT_ERR_NONFINITE", 7: "OT_ERR_CUDA", 8: "OT_ERR_OOM"}
OT_MEM_DEVICE, OT_MEM_HOST = 0, 1
OT_PREC_FP64, OT_PREC_MIXED = 0, 1
OT_PRECOND_BB, OT_PRECOND_SIMPLE, OT_PRECOND_HYBRID = 0, 1, 2
OT_MAX_STAGES = 40

EXPORTED = ["ot_default_options", "ot_mesh_create", "ot_mesh_destroy", "ot_mesh_info", "ot_ipm_solve",
            "ot_ipm_solve_batched", "ot_newton_solve", "ot_cost_grad", "ot_last_error", "ot_residual", "ot_kkt_apply", "ot_schur_apply",
            "ot_bb_apply", "ot_cost_dual", "ot_kernel_timing_enable", "ot_kernel_timing_count",
            "ot_kernel_timing_read", "ot_kernel_launches", "ot_kkt_apply_noalloc", "ot_tune_newton",
            "ot_simple_apply"]


class OTError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class ot_mesh_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32)]


class ot_options(C.Structure):
    _fields_ = [("memspace", C.c_int32), ("precision", C.c_int32), ("mu_factor", C.c_double),
                ("tau", C.c_double), ("newton_tol", C.c_double), ("final_newton_tol", C.c_double),
                ("eps_out", C.c_double), ("final_eps_out", C.c_double), ("eps_schur", C.c_double),
                ("fgmres_restart", C.c_int32), ("fgmres_max_iter", C.c_int32), ("schur_max_iter", C.c_int32),
                ("lap_cycles", C.c_int32), ("smooth_sweeps", C.c_int32), ("coarse_sweeps", C.c_int32),
                ("max_newton", C.c_int32), ("verbose", C.c_int32), ("gs_shadow", C.c_int32),
                ("graphs", C.c_int32), ("precond", C.c_int32), ("simple_mu", C.c_double),
                ("pdl", C.c_int32)]


class ot_stats(C.Structure):
    _fields_ = [("stages", C.c_int32), ("newton_steps", C.c_int32), ("fgmres_iters", C.c_int64),
                ("inner_iters", C.c_int64), ("final_residual", C.c_double), ("mu", C.c_double),
                ("gap", C.c_double), ("cost", C.c_double), ("dual", C.c_double), ("seconds", C.c_double),
                ("stage_mu", C.c_double * OT_MAX_STAGES), ("stage_newton", C.c_int32 * OT_MAX_STAGES),
                ("stage_outer", C.c_int64 * OT_MAX_STAGES), ("stage_inner", C.c_int64 * OT_MAX_STAGES),
                ("stage_seconds", C.c_double * OT_MAX_STAGES), ("stage_residual", C.c_double * OT_MAX_STAGES)]

    def as_dict(self) -> dict:
        n = self.stages
        return {
            "stages": n, "newton_steps": self.newton_steps, "fgmres_iters": self.fgmres_iters,
            "inner_iters": self.inner_iters, "final_residual": self.final_residual, "mu": self.mu,
            "gap": self.gap, "cost": self.cost, "dual": self.dual, "seconds": self.seconds,
            "stage_mu": list(self.stage_mu[:n]), "stage_newton": list(self.stage_newton[:n]),
            "stage_outer": list(self.stage_outer[:n]), "stage_inner": list(self.stage_inner[:n]),
            "stage_seconds": list(self.stage_seconds[:n]), "stage_residual": list(self.stage_residual[:n]),
        }


_LIB = None
_P = C.c_void_p
_D = C.c_double
_I = C.c_int32


def load():
    """Load libotgb.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    sig = {
        "ot_default_options": (None, [C.POINTER(ot_options)]),
        "ot_mesh_create": (_I, [C.POINTER(ot_mesh_desc), C.POINTER(_P)]),
        "ot_mesh_destroy": (None, [_P]),
        "ot_mesh_info": (_I, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64), _P]),
        "ot_ipm_solve": (_I, [_P, _P, _P, _I, _D, _D, C.POINTER(ot_options), _I, _P, _P, _P, C.POINTER(_D),
                              C.POINTER(ot_stats), _P]),
        "ot_ipm_solve_batched": (_I, [_I, _P, _P, _P, _P, _D, _D, C.POINTER(ot_options), _P, _P, _P, _P,
                                      C.POINTER(ot_stats), _P, _I]),
        "ot_newton_solve": (_I, [_P, _I, _D, _P, _P, _P, _P, _P, C.POINTER(ot_options), _P, _P, _P,
                                 C.POINTER(ot_stats), _P]),
        "ot_cost_grad": (_I, [_P, _I, _D, _P, _P, _P, _P, _P, C.POINTER(ot_options), _P, _P, _P]),
        "ot_tune_newton": (_I, [_P, _I, _D, _P, _P, _P, _P, _P, C.POINTER(ot_options), _I, _P, _P, _P]),
        "ot_last_error": (C.c_char_p, []),
        "ot_residual": (_I, [_P, _I, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
        "ot_kkt_apply": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
        "ot_schur_apply": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
        "ot_kkt_apply_noalloc": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
        "ot_bb_apply": (_I, [_P, _I, C.POINTER(ot_options), _P, _P, _P, _P, _P, _P, _P, _P]),
        "ot_simple_apply": (_I, [_P, _I, C.POINTER(ot_options), _P, _P, _P, _P, _P, _P, _P, _P]),
        "ot_cost_dual": (_I, [_P, _I, _P, _P, _P, _P, C.POINTER(_D), C.POINTER(_D), _P]),
        "ot_kernel_timing_enable": (None, [_I, _I]),
        "ot_kernel_timing_count": (_I, []),
        "ot_kernel_launches": (C.c_int64, []),
        "ot_kernel_timing_read": (_I, [_I, C.POINTER(C.c_char_p), C.POINTER(_D), C.POINTER(C.c_int64),
                                       C.POINTER(_D)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(code: int):
    if code != OT_OK:
        raise OTError(code, load().ot_last_error().decode())


def default_options(**overrides) -> ot_options:
    """ot_options filled by ot_default_options, then the given fields overridden."""
    o = ot_options()
    load().ot_default_options(C.byref(o))
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": OT_PREC_FP64, "mixed": OT_PREC_MIXED}[v]
        if k == "precond" and isinstance(v, str):
            v = {"bb": OT_PRECOND_BB, "simple": OT_PRECOND_SIMPLE, "hybrid": OT_PRECOND_HYBRID}[v]
        setattr(o, k, v)
    return o


def _dev_ptr(t: torch.Tensor) -> int:
    """Device pointer of a contiguous CUDA float64 tensor (the operator-level calls need device memory)."""
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise ValueError("expected a CUDA tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 tensor")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is not None:
        return int(stream)
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return 0


OT_MESH_STRUCTURED_SQUARE, OT_MESH_CARTESIAN_CUBE = 0, 1


class Mesh:
    """Owner of an ot_mesh: the structured unit-square mesh with n x n squares
    (kind "square"), or the 3D grid of n^3 cubes of test 4 (kind "cube", operator-level
    calls only)."""

    def __init__(self, n: int, kind: str = "square"):
        self._lib = load()
        self._h = _P()
        self.kind = kind
        desc = ot_mesh_desc({"square": OT_MESH_STRUCTURED_SQUARE, "cube": OT_MESH_CARTESIAN_CUBE}[kind], int(n))
        _check(self._lib.ot_mesh_create(C.byref(desc), C.byref(self._h)))
        self.n = int(n)
        nc, nf, ne = C.c_int64(), C.c_int64(), C.c_int64()
        _check(self._lib.ot_mesh_info(self._h, C.byref(nc), C.byref(nf), C.byref(ne), None))
        self.n_coarse, self.n_fine, self.n_edges_fine = nc.value, nf.value, ne.value
        areas = torch.empty(self.n_coarse, dtype=torch.float64)
        _check(self._lib.ot_mesh_info(self._h, None, None, None, C.c_void_p(areas.data_ptr())))
        self.coarse_areas = areas  # |c'| (host)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.ot_mesh_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ot_mesh_create(n: int) -> Mesh:
    return Mesh(n)


def _as_f64(x, device):
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64))
    x = x.to(dtype=torch.float64)
    if device is not None:
        x = x.to(device)
    return x.contiguous()


def ot_ipm_solve(mesh: Mesh, rho_in, rho_f, K: int, mu0: float = 1.0, tol: float = 1e-6, options=None,
                 warm_start=None, stream=None) -> dict:
    """Interior-point solve.  CUDA inputs -> device pointers, outputs CUDA tensors;
    CPU tensors / numpy -> host pointers (copies inside the library), outputs CPU tensors.
    warm_start: optional (rho, phi, s)."""
    o = options if options is not None else default_options()
    on_dev = isinstance(rho_in, torch.Tensor) and rho_in.is_cuda
    o.memspace = OT_MEM_DEVICE if on_dev else OT_MEM_HOST
    dev = rho_in.device if on_dev else None
    r0 = _as_f64(rho_in, dev)
    r1 = _as_f64(rho_f, dev)
    Np, Nr = (K + 1) * mesh.n_fine, K * mesh.n_coarse
    alloc = (lambda n: torch.empty(n, dtype=torch.float64, device=dev)) if on_dev else \
        (lambda n: torch.empty(n, dtype=torch.float64).pin_memory() if torch.cuda.is_available()
         else torch.empty(n, dtype=torch.float64))
    if warm_start is not None:
        rho, phi, s = (_as_f64(t, dev).clone() for t in warm_start)
    else:
        rho, phi, s = alloc(Nr), alloc(Np), alloc(Nr)
    cost = C.c_double()
    st = ot_stats()
    _check(load().ot_ipm_solve(mesh.handle, r0.data_ptr(), r1.data_ptr(), int(K), float(mu0), float(tol),
                               C.byref(o), int(warm_start is not None), rho.data_ptr(), phi.data_ptr(),
                               s.data_ptr(), C.byref(cost), C.byref(st), _stream(stream) if on_dev else 0))
    return {"rho": rho, "phi": phi, "s": s, "cost": cost.value, "stats": st.as_dict()}


def ot_ipm_solve_batched(problems, mu0: float = 1.0, tol: float = 1e-6, options=None, n_streams: int = 16,
                         raise_on_error: bool = True):
    """Independent solves run concurrently on n_streams CUDA streams.

    problems: list of (mesh, rho_in, rho_f, K) with CUDA float64 densities.
    Returns one dict per problem, like ot_ipm_solve, plus its status code
    ("status", 0 = OT_OK); with raise_on_error, raises for the first failed
    problem once all have run."""
    o = options if options is not None else default_options()
    o.memspace = OT_MEM_DEVICE
    n = len(problems)
    keep = []
    meshes = (_P * n)(*[p[0].handle for p in problems])
    Ks = (_I * n)(*[int(p[3]) for p in problems])
    out = []
    for mesh, r0, r1, K in problems:
        if not (isinstance(r0, torch.Tensor) and r0.is_cuda and isinstance(r1, torch.Tensor) and r1.is_cuda):
            raise ValueError("ot_ipm_solve_batched takes CUDA densities")
        r0 = r0.to(torch.float64).contiguous()
        r1 = r1.to(torch.float64).contiguous()
        dev = r0.device
        Np, Nr = (K + 1) * mesh.n_fine, K * mesh.n_coarse
        res = {"rho": torch.empty(Nr, dtype=torch.float64, device=dev),
               "phi": torch.empty(Np, dtype=torch.float64, device=dev),
               "s": torch.empty(Nr, dtype=torch.float64, device=dev)}
        keep.append((r0, r1))
        out.append(res)
    ptrs = lambda xs: (_P * n)(*[x.data_ptr() for x in xs])  # noqa: E731
    r0p, r1p = ptrs([k[0] for k in keep]), ptrs([k[1] for k in keep])
    rhop, phip, sp = ptrs([r["rho"] for r in out]), ptrs([r["phi"] for r in out]), ptrs([r["s"] for r in out])
    cost = (_D * n)()
    stats = (ot_stats * n)()
    status = (_I * n)()
    torch.cuda.synchronize()
    code = load().ot_ipm_solve_batched(n, meshes, Ks, r0p, r1p, float(mu0), float(tol), C.byref(o), rhop, phip, sp,
                                       cost, stats, status, int(n_streams))
    for p, res in enumerate(out):
        res["cost"] = cost[p]
        res["stats"] = stats[p].as_dict()
        res["status"] = status[p]
    if raise_on_error:
        _check(code)
    return out


def ot_newton_solve(mesh: Mesh, K: int, mu: float, phi, rho, s, rho_in, rho_f, options=None, stream=None):
    o = options if options is not None else default_options()
    o.memspace = OT_MEM_DEVICE
    Np, Nr = (K + 1) * mesh.n_fine, K * mesh.n_coarse
    dphi = torch.empty(Np, dtype=torch.float64, device=phi.device)
    drho = torch.empty(Nr, dtype=torch.float64, device=phi.device)
    ds = torch.empty(Nr, dtype=torch.float64, device=phi.device)
    st = ot_stats()
    _check(load().ot_newton_solve(mesh.handle, int(K), float(mu), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s),
                                  _dev_ptr(rho_in), _dev_ptr(rho_f), C.byref(o), _dev_ptr(dphi), _dev_ptr(drho),
                                  _dev_ptr(ds), C.byref(st), _stream(stream)))
    return dphi, drho, ds, st.as_dict()


def ot_cost_grad(mesh: Mesh, K: int, mu: float, phi, rho, s, rho_in, rho_f, options=None, stream=None):
    o = options if options is not None else default_options()
    o.memspace = OT_MEM_DEVICE
    gin = torch.empty(mesh.n_coarse, dtype=torch.float64, device=phi.device)
    gf = torch.empty(mesh.n_coarse, dtype=torch.float64, device=phi.device)
    _check(load().ot_cost_grad(mesh.handle, int(K), float(mu), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s),
                               _dev_ptr(rho_in), _dev_ptr(rho_f), C.byref(o), _dev_ptr(gin), _dev_ptr(gf),
                               _stream(stream)))
    return gin, gf



TUNE_GRID = [(sw, cs, lc) for sw in (1, 2, 3) for cs in (6, 10) for lc in (1, 2)]   # the library's built-in grid


def ot_tune_newton(mesh: Mesh, K: int, mu: float, phi, rho, s, rho_in, rho_f, options=None, candidates=None,
                   stream=None):
    """Timed trials of (smooth_sweeps, coarse_sweeps, lap_cycles) on one Newton solve at the given
    device state; returns (options with the fastest setting, seconds per candidate, -1 = failed)."""
    o = options if options is not None else default_options()
    o.memspace = OT_MEM_DEVICE
    cand = list(candidates) if candidates is not None else TUNE_GRID
    arr = (C.c_int32 * (3 * len(cand)))(*[int(v) for c in cand for v in c])
    sec = (C.c_double * len(cand))()
    _check(load().ot_tune_newton(mesh.handle, int(K), float(mu), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s),
                                 _dev_ptr(rho_in), _dev_ptr(rho_f), C.byref(o), len(cand),
                                 C.cast(arr, C.c_void_p), C.cast(sec, C.c_void_p), _stream(stream)))
    return o, list(sec)

def ot_residual(mesh: Mesh, K: int, mu: float, phi, rho, s, rho_in, rho_f, stream=None):
    Fphi = torch.empty_like(phi)
    Frho = torch.empty_like(rho)
    Fs = torch.empty_like(s)
    norms = (C.c_double * 4)()
    _check(load().ot_residual(mesh.handle, int(K), float(mu), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s),
                              _dev_ptr(rho_in), _dev_ptr(rho_f), _dev_ptr(Fphi), _dev_ptr(Frho), _dev_ptr(Fs),
                              C.cast(norms, _P), _stream(stream)))
    return Fphi, Frho, Fs, list(norms)


def ot_kkt_apply(mesh: Mesh, K: int, phi, rho, s, rho_in, rho_f, x, stream=None):
    y = torch.empty_like(x)
    _check(load().ot_kkt_apply(mesh.handle, int(K), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s), _dev_ptr(rho_in),
                               _dev_ptr(rho_f), _dev_ptr(x), _dev_ptr(y), _stream(stream)))
    return y


def ot_kkt_apply_noalloc(n: int, K: int, phi, rho, s, rho_in, rho_f, x, out, stream=None):
    """Projected KKT operator without any device allocation by the library: the
    caller provides ``out`` (same shape as ``x``); the only scratch is the
    library's file-scope device array (K <= 4096).  For callers whose device
    memory is reserved by another allocator or whose loop cannot absorb the
    synchronisation of cudaMalloc/cudaFree."""
    _check(load().ot_kkt_apply_noalloc(int(n), int(K), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s),
                                       _dev_ptr(rho_in), _dev_ptr(rho_f), _dev_ptr(x), _dev_ptr(out),
                                       _stream(stream)))
    return out


def ot_schur_apply(mesh: Mesh, K: int, phi, rho, s, z, stream=None):
    out = torch.empty_like(z)
    _check(load().ot_schur_apply(mesh.handle, int(K), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s), _dev_ptr(z),
                                 _dev_ptr(out), _stream(stream)))
    return out


def ot_simple_apply(mesh: Mesh, K: int, phi, rho, s, rho_in, rho_f, v, options=None, stream=None):
    """One SIMPLE preconditioner application (Sec. 4.2) at (phi, rho, s): returns (x; y)."""
    o = options if options is not None else default_options()
    out = torch.empty_like(v)
    _check(load().ot_simple_apply(mesh.handle, int(K), C.byref(o), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s),
                                  _dev_ptr(rho_in), _dev_ptr(rho_f), _dev_ptr(v), _dev_ptr(out), _stream(stream)))
    return out


def ot_bb_apply(mesh: Mesh, K: int, phi, rho, s, rho_in, rho_f, v, options=None, stream=None):
    o = options if options is not None else default_options()
    out = torch.empty_like(v)
    _check(load().ot_bb_apply(mesh.handle, int(K), C.byref(o), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(s),
                              _dev_ptr(rho_in), _dev_ptr(rho_f), _dev_ptr(v), _dev_ptr(out), _stream(stream)))
    return out


def ot_kernel_launches() -> int:
    """Kernel launches made by the library since it was loaded."""
    return int(load().ot_kernel_launches())


def ot_kernel_timing_groups() -> list:
    lib = load()
    names = []
    for i in range(lib.ot_kernel_timing_count()):
        nm = C.c_char_p()
        _check(lib.ot_kernel_timing_read(i, C.byref(nm), None, None, None))
        names.append(nm.value.decode())
    return names


def ot_kernel_timing_enable(groups=True, sample_every: int = 1) -> None:
    """groups: True (all), False (off), or an iterable of group names; one launch in
    ``sample_every`` of each group is timed."""
    if groups is True:
        mask = -1
    elif groups is False or groups is None:
        mask = 0
    else:
        names = ot_kernel_timing_groups()
        mask = 0
        for g in groups:
            mask |= 1 << names.index(g)
    load().ot_kernel_timing_enable(int(mask), int(sample_every))


def ot_kernel_timing_read() -> dict:
    """{group: (milliseconds, launches, algorithmic bytes)} accumulated since the last enable."""
    lib = load()
    out = {}
    for i in range(lib.ot_kernel_timing_count()):
        nm, ms, n, b = C.c_char_p(), C.c_double(), C.c_int64(), C.c_double()
        _check(lib.ot_kernel_timing_read(i, C.byref(nm), C.byref(ms), C.byref(n), C.byref(b)))
        out[nm.value.decode()] = (ms.value, n.value, b.value)
    return out


def ot_cost_dual(mesh: Mesh, K: int, phi, rho, rho_in, rho_f, stream=None):
    c, d = C.c_double(), C.c_double()
    _check(load().ot_cost_dual(mesh.handle, int(K), _dev_ptr(phi), _dev_ptr(rho), _dev_ptr(rho_in),
                               _dev_ptr(rho_f), C.byref(c), C.byref(d), _stream(stream)))
    return c.value, d.value
