"""GB300 agglomeration h-multigrid for Compact DG discretisations of Poisson's
equation (Pan & Persson, arXiv 2012.08024) -- Python binding of libcdgmg.so.

The binding only marshals arguments: the host set-up (Sections 2-4.1) runs in
the library's C++ code and every step of the solve phase (Section 4) runs in its
CUDA kernels.  PyTorch provides the device buffer and the stream.  There is no
fallback: if the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcdgmg.so")

CDG_MAX_LEVELS = 16
ERRORS = {1: "EINVAL", 2: "EMESH", 3: "ENOCONV", 4: "EBREAKDOWN", 5: "ECUDA", 6: "ETIMEOUT",
          7: "ENOMEM", 8: "ESTATE"}


class CdgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class cdg_mesh(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n_vertices", C.c_int64), ("xyz", C.c_void_p),
                ("n_elements", C.c_int64), ("elem", C.c_void_p), ("n_bfaces", C.c_int64),
                ("bface", C.c_void_p), ("btag", C.c_void_p)]


class cdg_options(C.Structure):
    _fields_ = [("p", C.c_int32), ("gamma", C.c_double), ("nu_pre", C.c_int32), ("nu_post", C.c_int32),
                ("omega", C.c_double), ("max_levels", C.c_int32), ("seed", C.c_uint64),
                ("precision", C.c_int32), ("switch_kind", C.c_int32), ("face_switch", C.c_void_p),
                ("enumeration", C.c_void_p), ("kappa", C.c_void_p), ("coarsen", C.c_int32),
                ("tol", C.c_double), ("maxit", C.c_int32), ("nrhs", C.c_int32),
                ("krylov", C.c_int32), ("restart", C.c_int32), ("pmg", C.c_int32), ("autotune", C.c_int32),
                ("beta", C.c_double), ("velocity", C.c_double * 3), ("solve_graph", C.c_int32),
                ("tensor_cores", C.c_int32), ("fuse_transfers", C.c_int32), ("tc_fp64_apply", C.c_int32),
                ("persistent_vcycle", C.c_int32)]


class cdg_info(C.Structure):
    _fields_ = [("dim", C.c_int32), ("p", C.c_int32), ("n_p", C.c_int32), ("n_levels", C.c_int32),
                ("nq", C.c_int32), ("nfq", C.c_int32), ("n_elements", C.c_int64),
                ("n_interior_faces", C.c_int64), ("n_bfaces", C.c_int64), ("n_dofs", C.c_int64),
                ("n_l", C.c_int64 * CDG_MAX_LEVELS), ("nnzb_l", C.c_int64 * CDG_MAX_LEVELS),
                ("h_avg", C.c_double), ("C_D", C.c_double), ("device_bytes", C.c_int64),
                ("setup_seconds", C.c_double * 4), ("n_meshes", C.c_int32),
                ("np_l", C.c_int32 * CDG_MAX_LEVELS), ("n_plevels", C.c_int32), ("solve_graph", C.c_int32)]


_lib = None

# every exported symbol with its argument types (checked against include/cdg.h by the tests)
_P, _I32, _I64, _D, _U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint64
SIGNATURES = {
    "cdg_default_options": (None, [_P]),
    "cdg_create": (_I32, [_P, _P, _P]),
    "cdg_create_batched": (_I32, [_P, _I32, _P, _P]),
    "cdg_batch_offsets": (_I32, [_P, _P, _P, _P]),
    "cdg_destroy": (None, [_P]),
    "cdg_last_error": (C.c_char_p, [_P]),
    "cdg_query": (_I32, [_P, _P]),
    "cdg_tuning": (_I32, [_P, _I32, _P]),
    "cdg_apply_f32": (_I32, [_P, _I32, _P, _P, _P]),
    "cdg_quadrature_points": (_I32, [_P, _P, _P, _P]),
    "cdg_export_level": (_I32, [_P, _I32, _P, _P, _P, _P, _P, _P]),
    "cdg_export_agglomeration": (_I32, [_P, _I32, _P]),
    "cdg_bind_device": (_I32, [_P, _P, _I64, _P]),
    "cdg_set_precision": (_I32, [_P, _I32]),
    "cdg_set_wait_limit": (_I32, [_P, _I32]),
    "cdg_apply_multi": (_I32, [_P, _P, _P, _P]),
    "cdg_fp64_fma_probe": (_I32, [_I32, _I64, _P, _P]),
    "cdg_convert": (_I32, [_P, _P, _I64, _I32, _P]),
    "cdg_rhs": (_I32, [_P, _P, _P, _P, _P, _P]),
    "cdg_solve": (_I32, [_P, _P, _P, _P, _P, _I32, _P, _P, _I32, _P]),
    "cdg_solve_b": (_I32, [_P, _P, _P, _I32, _P, _P, _P]),
    "cdg_apply": (_I32, [_P, _I32, _P, _P, _P]),
    "cdg_residual": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "cdg_smooth": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "cdg_restrict": (_I32, [_P, _I32, _P, _P, _P]),
    "cdg_prolong": (_I32, [_P, _I32, _P, _P, _P]),
    "cdg_coarse_solve": (_I32, [_P, _P, _P, _P]),
    "cdg_vcycle": (_I32, [_P, _P, _P, _P]),
    "cdg_to_tree": (_I32, [_P, _P, _P, _P]),
    "cdg_to_user": (_I32, [_P, _P, _P, _P]),
    "cdg_kernel_launches": (_I64, []),
    "cdg_smooth_static": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "cdg_solve_adjoint": (_I32, [_P, _P, _P, _P, _P, _P]),
    "cdg_solve_multi": (_I32, [_P, _P, _P, _P, _P, _P]),
    "cdg_rhs_adjoint": (_I32, [_P, _P, _P, _P]),
    "cdg_kappa_gradient": (_I32, [_P, _P, _P, _P, _P, _P]),
}


def lib():
    """Loads libcdgmg.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2012_08024_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(lib().cdg_kernel_launches())


def convert(x, stream=None):
    """binary64 <-> binary32 conversion of a CUDA tensor by the library's
    kernel (cdg_convert): float64 in -> float32 out (round to nearest even),
    float32 in -> float64 out (exact)."""
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype not in (torch.float64, torch.float32):
        raise ValueError("convert: a float64 or float32 CUDA tensor is required")
    x = x.contiguous()
    to32 = x.dtype == torch.float64
    out = torch.empty(x.shape, dtype=torch.float32 if to32 else torch.float64, device=x.device)
    rc = lib().cdg_convert(_ptr(x), _ptr(out), x.numel(), int(to32), _stream_ptr(stream))
    if rc:
        raise CdgError(rc, "cdg_convert failed")
    return out


def _dvec(t, n: int, name: str, dtype: str = "float64") -> int | None:
    """Device pointer of a CUDA tensor of `dtype` holding at least n contiguous
    elements (None passes through for nullable arguments).  A host tensor, a
    wrong dtype or a short buffer raises here instead of reaching a kernel."""
    if t is None:
        return None
    import torch
    want = getattr(torch, dtype)
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name}: a CUDA tensor is required")
    if t.dtype != want:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {want}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: the tensor must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{name}: {t.numel()} elements, at least {n} required")
    return t.data_ptr()


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()        # torch tensor


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


PRECISION = {"fp64": 0, "fp32": 1, "bf16": 2}
COARSEN = {"flux": 0, "primal": 1}
KRYLOV = {"cg": 0, "gmres": 1}


class Solver:
    """Host set-up of one mesh (cdg_create) plus its device solve phase."""

    def __init__(self, mesh, p: int = 2, gamma: float = 1e4, nu_pre: int = 1, nu_post: int = 1,
                 omega: float = 2.0 / 3.0, max_levels: int = 4, seed: int = 0, precision: str = "fp64",
                 switch_kind: int = 0, face_switch=None, enumeration=None, kappa=None,
                 coarsen: str = "flux", tol: float = 1e-10, maxit: int = 500, nrhs: int = 0,
                 krylov: str = "cg", restart: int = 50, autotune: bool = True, pmg: bool = False,
                 beta: float = 0.0, velocity=(0.0, 0.0, 0.0), tensor_cores: bool = True,
                 single_graph: bool = True, fuse_transfers: int = 0, tc_fp64_apply: bool = False,
                 persistent_vcycle: bool = False):
        L = lib()
        self._keep = []
        self.nrhs = nrhs
        xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
        elem = np.ascontiguousarray(mesh.elem, dtype=np.int64)
        bface = np.ascontiguousarray(mesh.bface, dtype=np.int64).reshape(-1, mesh.dim)
        btag = np.ascontiguousarray(mesh.btag, dtype=np.int32)
        m = cdg_mesh(mesh.dim, xyz.shape[0], xyz.ctypes.data, elem.shape[0], elem.ctypes.data,
                     bface.shape[0], bface.ctypes.data if len(bface) else None,
                     btag.ctypes.data if len(btag) else None)
        o = cdg_options()
        L.cdg_default_options(C.byref(o))
        o.p, o.gamma, o.nu_pre, o.nu_post, o.omega = p, gamma, nu_pre, nu_post, omega
        o.max_levels, o.seed = max_levels, seed
        o.precision, o.switch_kind = PRECISION[precision], switch_kind
        o.coarsen, o.tol, o.maxit = COARSEN[coarsen], tol, maxit
        o.nrhs = nrhs
        o.krylov, o.restart, o.autotune = KRYLOV[krylov], restart, int(autotune)
        o.pmg = int(pmg)
        o.beta = beta
        o.tensor_cores = int(tensor_cores)
        o.solve_graph = int(single_graph)
        o.fuse_transfers = int(fuse_transfers) if not isinstance(fuse_transfers, bool) else 3 * int(fuse_transfers)
        o.tc_fp64_apply = int(tc_fp64_apply)
        o.persistent_vcycle = int(persistent_vcycle)
        vel = list(velocity) + [0.0] * (3 - len(velocity))
        for c in range(3):
            o.velocity[c] = float(vel[c])
        arrs = {}
        if face_switch is not None:
            arrs["fs"] = np.ascontiguousarray(face_switch, dtype=np.int8)
            o.face_switch = arrs["fs"].ctypes.data
        if enumeration is not None:
            arrs["en"] = np.ascontiguousarray(enumeration, dtype=np.int64)
            o.enumeration = arrs["en"].ctypes.data
        if kappa is not None:
            arrs["ka"] = np.ascontiguousarray(kappa, dtype=np.float64)
            o.kappa = arrs["ka"].ctypes.data
        h = C.c_void_p()
        rc = L.cdg_create(C.byref(m), C.byref(o), C.byref(h))
        if rc:
            raise CdgError(rc, L.cdg_last_error(None).decode())
        self._h = h
        self.precision = precision
        self.buffer = None
        inf = cdg_info()
        L.cdg_query(h, C.byref(inf))
        self.info = {k: (list(getattr(inf, k))[:inf.n_levels] if k in ("n_l", "nnzb_l", "np_l") else
                         list(getattr(inf, k)) if k == "setup_seconds" else getattr(inf, k))
                     for k, _ in cdg_info._fields_}
        self.np_ = inf.n_p
        self.n_levels = inf.n_levels
        self.ne = inf.n_elements
        self.maxit = maxit

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.cdg_destroy(h)
            self._h = None

    def _check(self, rc):
        if rc:
            raise CdgError(rc, lib().cdg_last_error(self._h).decode())

    # ---------------------------------------------------------------- host side
    def quadrature_points(self):
        d, ne, nbf = self.info["dim"], self.ne, self.info["n_bfaces"]
        xq = np.empty((ne, self.info["nq"], d))
        xbq = np.empty((nbf, self.info["nfq"], d))
        btag = np.empty(nbf, dtype=np.int32)
        self._check(lib().cdg_quadrature_points(self._h, xq.ctypes.data, xbq.ctypes.data, btag.ctypes.data))
        return xq, xbq, btag

    def export_level(self, level: int):
        n = self.info["n_l"][level]
        nnzb = self.info["nnzb_l"][level]
        npb = self.info["np_l"][level]
        npc = self.info["np_l"][level + 1] if level + 1 < self.n_levels else npb
        out = dict(perm=np.empty(n, dtype=np.int64), parent=np.empty(n, dtype=np.int32),
                   rowptr=np.empty(n + 1, dtype=np.int64), col=np.empty(nnzb, dtype=np.int32),
                   val=np.empty((nnzb, npb, npb)), L=np.zeros((n, npb, npc)))
        self._check(lib().cdg_export_level(self._h, level, *(out[k].ctypes.data for k in
                                                             ("perm", "parent", "rowptr", "col", "val", "L"))))
        return out

    def export_agglomeration(self, level: int):
        par = np.empty(self.info["n_l"][level], dtype=np.int64)
        self._check(lib().cdg_export_agglomeration(self._h, level, par.ctypes.data))
        return par

    # ---------------------------------------------------------------- device side
    def bind(self, device="cuda"):
        import torch
        nbytes = int(self.info["device_bytes"])
        self.buffer = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.buffer.data_ptr()
        aligned = (base + 255) & ~255
        self._check(lib().cdg_bind_device(self._h, aligned, nbytes, _stream_ptr(None)))
        return self

    def set_precision(self, precision: str):
        """Switch the V-cycle precision without repeating the host set-up
        (cdg_set_precision); releases the device binding, so bind() again."""
        self._check(lib().cdg_set_precision(self._h, PRECISION[precision]))
        self.precision = precision
        self.buffer = None
        inf = cdg_info()
        lib().cdg_query(self._h, C.byref(inf))
        self.info["device_bytes"] = inf.device_bytes
        return self

    def set_wait_limit(self, limit: int):
        """Failure injection (cdg_set_wait_limit): iteration limit of the bounded
        device waits inside kernel loops; 0 = give up at once, < 0 = defaults."""
        self._check(lib().cdg_set_wait_limit(self._h, int(limit)))
        return self

    def solve_graph(self) -> bool:
        """True once a CG solve (or a GMRES restart cycle) of this handle ran as one CUDA graph launch."""
        inf = cdg_info()
        lib().cdg_query(self._h, C.byref(inf))
        return bool(inf.solve_graph)

    def tuning(self):
        """Autotuned launch configuration per level (cdg_tuning)."""
        keys = ("apply64_unroll", "residual64_unroll", "vcycle_residual_unroll", "vcycle_smoother_unroll",
                "multi_smoother_tile", "multi_smoother_rows", "multi_residual_tile", "multi_residual_rows",
                "multi_apply64_tile", "multi_apply64_rows", "multi_smoother_cols", "multi_residual_cols",
                "multi_apply64_cols")
        out = []
        for l in range(self.n_levels):
            a = (C.c_int32 * 13)()
            self._check(lib().cdg_tuning(self._h, l, a))
            out.append({k: int(v) for k, v in zip(keys, a) if v})
        return out

    def _dev(self, x):
        return _ptr(x)

    def _lvl(self, level: int) -> int:
        """Length of a tree-order vector of `level` (0 outside the hierarchy: the
        library then rejects the level itself)."""
        if not 0 <= level < self.n_levels:
            return 0
        return self.info["n_l"][level] * self.info["np_l"][level]

    def _sizes(self):
        ne, nbf = self.ne, self.info["n_bfaces"]
        return ne * self.info["nq"], nbf * self.info["nfq"], ne * self.np_

    def solve(self, f_q, gD=None, gN=None, u0=None, stream=None):
        """Device tensors in user order; returns (u, residual history, iterations)."""
        import torch
        nf, nb, nu = self._sizes()
        pf, pd, pn = _dvec(f_q, nf, "f_q"), _dvec(gD, nb, "gD"), _dvec(gN, nb, "gN")
        u = torch.empty((self.ne, self.np_), dtype=torch.float64, device=f_q.device) if u0 is None else u0
        hist = np.zeros(self.maxit + 1)
        it = C.c_int32(0)
        rc = lib().cdg_solve(self._h, pf, pd, pn, _dvec(u, nu, "u0"), 0 if u0 is None else 1,
                             hist.ctypes.data, C.byref(it), 0, _stream_ptr(stream))
        if rc not in (0, 3):
            self._check(rc)
        return u, hist[:it.value + 1], it.value, rc

    def solve_host(self, f_q: np.ndarray, gD=None, gN=None, stream=None):
        """Host numpy arrays in and out (copies inside the call)."""
        f_q = np.ascontiguousarray(f_q, dtype=np.float64)
        gD = None if gD is None else np.ascontiguousarray(gD, dtype=np.float64)
        gN = None if gN is None else np.ascontiguousarray(gN, dtype=np.float64)
        u = np.empty((self.ne, self.np_))
        hist = np.zeros(self.maxit + 1)
        it = C.c_int32(0)
        rc = lib().cdg_solve(self._h, _ptr(f_q), _ptr(gD), _ptr(gN), _ptr(u), 0, hist.ctypes.data,
                             C.byref(it), 1, _stream_ptr(stream))
        if rc not in (0, 3):
            self._check(rc)
        return u, hist[:it.value + 1], it.value, rc

    def solve_b(self, b, stream=None):
        import torch
        u = torch.empty((self.ne, self.np_), dtype=torch.float64, device=b.device)
        hist = np.zeros(self.maxit + 1)
        it = C.c_int32(0)
        rc = lib().cdg_solve_b(self._h, _dvec(b, self._sizes()[2], "b"), _ptr(u), 0, hist.ctypes.data, C.byref(it),
                               _stream_ptr(stream))
        if rc not in (0, 3):
            self._check(rc)
        return u, hist[:it.value + 1], it.value, rc

    def apply_multi(self, x, y, stream=None):
        """y = A_0 x for the R columns (tree order, [n][n_p][R] FP64 device tensors),
        by the method solve_multi uses (cdg_apply_multi)."""
        n = self._sizes()[2] * self.nrhs
        self._check(lib().cdg_apply_multi(self._h, _dvec(x, n, "x"), _dvec(y, n, "y"), _stream_ptr(stream)))

    def solve_multi(self, f_q, stream=None):
        """f_q [R][n_elements][nq] device -> u [R][n_elements][n_p], per-column
        residual histories, iteration counts, status."""
        import torch
        R = self.nrhs
        u = torch.empty((R, self.ne, self.np_), dtype=torch.float64, device=f_q.device)
        hist = np.zeros((R, self.maxit + 1))
        its = np.zeros(R, dtype=np.int32)
        f_q = f_q.contiguous()
        rc = lib().cdg_solve_multi(self._h, _dvec(f_q, R * self._sizes()[0], "f_q"), _ptr(u), hist.ctypes.data,
                                   its.ctypes.data, _stream_ptr(stream))
        if rc not in (0, 3):
            self._check(rc)
        return u, [hist[r, :its[r] + 1] for r in range(R)], its, rc

    def solve_adjoint(self, dLdu, stream=None):
        import torch
        lam = torch.empty((self.ne, self.np_), dtype=torch.float64, device=dLdu.device)
        hist = np.zeros(self.maxit + 1)
        it = C.c_int32(0)
        rc = lib().cdg_solve_adjoint(self._h, _dvec(dLdu, self._sizes()[2], "dLdu"), _ptr(lam), hist.ctypes.data,
                                     C.byref(it), _stream_ptr(stream))
        if rc not in (0, 3):
            self._check(rc)
        return lam, hist[:it.value + 1], it.value, rc

    def rhs_adjoint(self, lam, stream=None):
        import torch
        out = torch.empty((self.ne, self.info["nq"]), dtype=torch.float64, device=lam.device)
        self._check(lib().cdg_rhs_adjoint(self._h, _dvec(lam, self._sizes()[2], "lambda"), _ptr(out),
                                          _stream_ptr(stream)))
        return out

    def kappa_gradient(self, lam, u, gD=None, stream=None):
        import torch
        out = torch.empty(self.ne, dtype=torch.float64, device=lam.device)
        _, nb, nu = self._sizes()
        self._check(lib().cdg_kappa_gradient(self._h, _dvec(lam, nu, "lambda"), _dvec(u, nu, "u"),
                                             _dvec(gD, nb, "gD"), _ptr(out), _stream_ptr(stream)))
        return out

    def rhs(self, f_q, gD=None, gN=None, stream=None):
        import torch
        b = torch.empty((self.ne, self.np_), dtype=torch.float64, device=f_q.device)
        nf, nb, _ = self._sizes()
        self._check(lib().cdg_rhs(self._h, _dvec(f_q, nf, "f_q"), _dvec(gD, nb, "gD"), _dvec(gN, nb, "gN"), _ptr(b),
                                  _stream_ptr(stream)))
        return b

    def apply(self, level, x, y, stream=None):
        n = self._lvl(level)
        self._check(lib().cdg_apply(self._h, level, _dvec(x, n, "x"), _dvec(y, n, "y"), _stream_ptr(stream)))

    def residual(self, level, x, b, y, stream=None):
        n = self._lvl(level)
        self._check(lib().cdg_residual(self._h, level, _dvec(x, n, "x"), _dvec(b, n, "b"), _dvec(y, n, "y"),
                                       _stream_ptr(stream)))

    def apply_f32(self, level, x, y, stream=None):
        """y = A_l x with the FP32 operator copy of the FP32 V-cycle (float32 tensors)."""
        n = self._lvl(level)
        self._check(lib().cdg_apply_f32(self._h, level, _dvec(x, n, "x", "float32"), _dvec(y, n, "y", "float32"),
                                        _stream_ptr(stream)))

    def smooth(self, level, x, b, y, stream=None):
        n = self._lvl(level)
        self._check(lib().cdg_smooth(self._h, level, _dvec(x, n, "x"), _dvec(b, n, "b"), _dvec(y, n, "y"),
                                     _stream_ptr(stream)))

    def smooth_static(self, level, x, b, y, stream=None):
        """cdg_smooth without using the handle's buffer for its intermediate
        (fixed library scratch; see include/cdg.h).  Raises CdgError like the
        other device methods (a level beyond the fixed scratch: CDG_EINVAL)."""
        n = self._lvl(level)
        self._check(lib().cdg_smooth_static(self._h, level, _dvec(x, n, "x"), _dvec(b, n, "b"), _dvec(y, n, "y"),
                                            _stream_ptr(stream)))

    def restrict(self, level, r, bc, stream=None):
        self._check(lib().cdg_restrict(self._h, level, _dvec(r, self._lvl(level), "r"),
                                       _dvec(bc, self._lvl(level + 1), "bc"), _stream_ptr(stream)))

    def prolong(self, level, xc, x, stream=None):
        self._check(lib().cdg_prolong(self._h, level, _dvec(xc, self._lvl(level + 1), "xc"),
                                      _dvec(x, self._lvl(level), "x"), _stream_ptr(stream)))

    def coarse_solve(self, b, x, stream=None):
        n = self._lvl(self.n_levels - 1)
        self._check(lib().cdg_coarse_solve(self._h, _dvec(b, n, "b"), _dvec(x, n, "x"), _stream_ptr(stream)))

    def vcycle(self, r, z, stream=None):
        n = self._sizes()[2]
        self._check(lib().cdg_vcycle(self._h, _dvec(r, n, "r"), _dvec(z, n, "z"), _stream_ptr(stream)))

    def to_tree(self, user, tree, stream=None):
        n = self._sizes()[2]
        self._check(lib().cdg_to_tree(self._h, _dvec(user, n, "user"), _dvec(tree, n, "tree"), _stream_ptr(stream)))

    def to_user(self, tree, user, stream=None):
        n = self._sizes()[2]
        self._check(lib().cdg_to_user(self._h, _dvec(tree, n, "tree"), _dvec(user, n, "user"), _stream_ptr(stream)))


class BatchSolver(Solver):
    """Many independent meshes in one handle (cdg_create_batched): every kernel
    of the solve phase processes all meshes per launch; per-mesh CG scalars."""

    def __init__(self, meshes, p: int = 2, gamma: float = 1e4, nu_pre: int = 1, nu_post: int = 1,
                 omega: float = 2.0 / 3.0, max_levels: int = 4, seed: int = 0, precision: str = "fp64",
                 switch_kind: int = 0, coarsen: str = "flux", tol: float = 1e-10, maxit: int = 500,
                 single_graph: bool = True, fuse_transfers: int = 0, persistent_vcycle: bool = False):
        L = lib()
        keep, ms = [], (cdg_mesh * len(meshes))()
        for i, mesh in enumerate(meshes):
            xyz = np.ascontiguousarray(mesh.xyz, dtype=np.float64)
            elem = np.ascontiguousarray(mesh.elem, dtype=np.int64)
            bface = np.ascontiguousarray(mesh.bface, dtype=np.int64).reshape(-1, mesh.dim)
            btag = np.ascontiguousarray(mesh.btag, dtype=np.int32)
            keep += [xyz, elem, bface, btag]
            ms[i] = cdg_mesh(mesh.dim, xyz.shape[0], xyz.ctypes.data, elem.shape[0], elem.ctypes.data,
                             bface.shape[0], bface.ctypes.data if len(bface) else None,
                             btag.ctypes.data if len(btag) else None)
        o = cdg_options()
        L.cdg_default_options(C.byref(o))
        o.p, o.gamma, o.nu_pre, o.nu_post, o.omega = p, gamma, nu_pre, nu_post, omega
        o.max_levels, o.seed = max_levels, seed
        o.precision, o.switch_kind = PRECISION[precision], switch_kind
        o.coarsen, o.tol, o.maxit = COARSEN[coarsen], tol, maxit
        o.solve_graph = int(single_graph)
        o.fuse_transfers = int(fuse_transfers) if not isinstance(fuse_transfers, bool) else 3 * int(fuse_transfers)
        o.persistent_vcycle = int(persistent_vcycle)
        h = C.c_void_p()
        rc = L.cdg_create_batched(ms, len(meshes), C.byref(o), C.byref(h))
        if rc:
            raise CdgError(rc, L.cdg_last_error(None).decode())
        self._h = h
        self.precision = precision
        self.buffer = None
        inf = cdg_info()
        L.cdg_query(h, C.byref(inf))
        self.info = {k: (list(getattr(inf, k))[:inf.n_levels] if k in ("n_l", "nnzb_l", "np_l") else
                         list(getattr(inf, k)) if k == "setup_seconds" else getattr(inf, k))
                     for k, _ in cdg_info._fields_}
        self.np_ = inf.n_p
        self.n_levels = inf.n_levels
        self.ne = inf.n_elements
        self.maxit = maxit
        self.n_meshes = inf.n_meshes
        self.elem_offsets = np.zeros(self.n_meshes + 1, dtype=np.int64)
        self.bface_offsets = np.zeros(self.n_meshes + 1, dtype=np.int64)
        L.cdg_batch_offsets(h, None, self.elem_offsets.ctypes.data, self.bface_offsets.ctypes.data)

    def solve(self, f_q, gD=None, gN=None, u0=None, stream=None):
        """Device tensors (all meshes concatenated); returns u, per-mesh residual
        histories (list), per-mesh iteration counts (array), status."""
        import torch
        u = torch.empty((self.ne, self.np_), dtype=torch.float64, device=f_q.device) if u0 is None else u0
        hist = np.zeros((self.n_meshes, self.maxit + 1))
        its = np.zeros(self.n_meshes, dtype=np.int32)
        rc = lib().cdg_solve(self._h, _ptr(f_q), _ptr(gD), _ptr(gN), _ptr(u), 0 if u0 is None else 1,
                             hist.ctypes.data, its.ctypes.data, 0, _stream_ptr(stream))
        if rc not in (0, 3):
            self._check(rc)
        return u, [hist[m, :its[m] + 1] for m in range(self.n_meshes)], its, rc

    solve_host = None
    solve_b = None
    solve_adjoint = None
