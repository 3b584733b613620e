"""Python binding of libgm (include/gm.h): argument marshalling only.

Every operator application, fault update, solve and time step runs in the CUDA
library; this module converts torch tensors / numpy arrays to pointers and
status codes to exceptions.  There is no CPU fallback: if the shared library is
missing or fails to load, importing the binding raises.

Device vectors are torch CUDA tensors (float64 or float32) laid out as the C
ABI states: displacements (3, N) field-major, pressures (N,), coupled (4, N).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import LIB

__all__ = ["lib", "GMError", "Solver", "TetSolver", "OP", "OPEN", "STICK", "SLIP", "load_library"]

OP = {"KB": 0, "KT": 1, "A22": 2, "APU": 3, "AUP": 4, "J": 5}
OPEN, STICK, SLIP = 0, 1, 2
F64, F32 = 0, 1


class GMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gm error {code}: {msg}")
        self.code = code


class FaultParams(C.Structure):
    _fields_ = [("kn", C.c_double), ("ks", C.c_double), ("f", C.c_double), ("w0", C.c_double),
                ("wk_par", C.c_double), ("k_perp", C.c_double), ("MF", C.c_double),
                ("tn0", C.c_double), ("tau0", C.c_double * 2)]


class SolveReport(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double), ("status", C.c_int)]


class StepOpts(C.Structure):
    _fields_ = [("newton_rtol", C.c_double), ("newton_maxit", C.c_int),
                ("outer_rtol", C.c_double), ("outer_maxit", C.c_int),
                ("inner_rtol", C.c_double), ("inner_maxit", C.c_int),
                ("precision", C.c_int), ("schur_precond", C.c_int)]


class StepReport(C.Structure):
    _fields_ = [("newton", C.c_int), ("outer", C.c_int), ("inner_k", C.c_longlong),
                ("inner_a", C.c_longlong), ("applies", C.c_longlong), ("rhat", C.c_double),
                ("rhat0", C.c_double), ("n_open", C.c_int), ("n_stick", C.c_int),
                ("n_slip", C.c_int), ("min_yield_margin", C.c_double),
                ("min_normal_margin", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIG = {
    "gm_version": (C.c_char_p, []),
    "gm_create": (C.c_int, [C.POINTER(_P), C.c_int]),
    "gm_destroy": (C.c_int, [_P]),
    "gm_last_error": (C.c_char_p, [_P]),
    "gm_mesh_structured": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _D, _D, _D]),
    "gm_fault_plane": (C.c_int, [_P, C.c_int, C.POINTER(FaultParams)]),
    "gm_set_materials": (C.c_int, [_P, _D, _D, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double]),
    "gm_set_dirichlet": (C.c_int, [_P, C.POINTER(C.c_uint8), C.c_int64]),
    "gm_set_loads": (C.c_int, [_P, _D, _D]),
    "gm_assemble_or_bind": (C.c_int, [_P]),
    "gm_set_timestep": (C.c_int, [_P, C.c_double]),
    "gm_apply_operator": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "gm_fault_update": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "gm_pcg_solve": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_int, C.POINTER(SolveReport), _P]),
    "gm_prevost_solve": (C.c_int, [_P, _P, _P, C.c_double, C.c_int, C.c_double, C.c_int,
                                   C.POINTER(SolveReport), _P]),
    "gm_residual": (C.c_int, [_P, _P, _P, _P, _D, _P]),
    "gm_residual_noalloc": (C.c_int, [_P, _P, _P, _P, _D, _P]),
    "gm_partitioned_step": (C.c_int, [_P, C.c_double, C.POINTER(StepOpts), C.POINTER(StepReport), _P]),
    "gm_get_state": (C.c_int, [_P, _D, _D, _D, _D, C.POINTER(C.c_int8)]),
    "gm_set_state": (C.c_int, [_P, _D, _D, _D, C.POINTER(C.c_int8)]),
    "gm_state_device": (C.c_int, [_P, C.POINTER(_P), C.POINTER(_P)]),
    "gm_sizes": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "gm_counters": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "gm_set_permeability": (C.c_int, [_P, _D, C.c_int64]),
    "gm_set_friction": (C.c_int, [_P, _D, C.c_int64]),
    "gm_adjoint_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _D, C.c_double, C.c_int,
                                  C.POINTER(SolveReport), _P]),
    "gm_set_adjoint_options": (C.c_int, [_P, C.c_int, C.c_double, C.c_int]),
    "gm_set_insitu": (C.c_int, [_P, _P, _P, C.c_int64]),
    "gm_tet_create": (C.c_int, [C.POINTER(_P), C.c_int]),
    "gm_tet_destroy": (C.c_int, [_P]),
    "gm_tet_last_error": (C.c_char_p, [_P]),
    "gm_tet_mesh": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64]),
    "gm_tet_materials": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_double]),
    "gm_tet_apply": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_int, _P]),
    "gm_tet_dirichlet": (C.c_int, [_P, C.POINTER(C.c_uint8), C.c_int64]),
    "gm_tet_surface_load": (C.c_int, [_P, _P, C.c_int64, C.c_double]),
    "gm_tet_step": (C.c_int, [_P, C.c_double, _P, _P, C.c_double, C.c_int, C.POINTER(SolveReport), _P]),
    "gm_tet_fault": (C.c_int, [_P, _P, C.c_int64, _P, C.c_int64, _D, C.POINTER(FaultParams)]),
    "gm_tet_loads": (C.c_int, [_P, _D, _D]),
    "gm_tet_fault_apply": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, _P]),
    "gm_tet_fault_step": (C.c_int, [_P, C.c_double, _P, _P, C.POINTER(StepOpts), C.POINTER(StepReport), _P]),
    "gm_tet_fault_state": (C.c_int, [_P, C.POINTER(C.c_int8), _D, _D]),
    "gm_set_preconditioner": (C.c_int, [_P, C.c_int]),
    "gm_adjoint_sweep_step": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _D,
                                        C.c_double, C.c_int, C.POINTER(SolveReport), _P]),
}

_lib = None


def load_library(path: str = LIB):
    """Load libgm.so (built by __graft_entry__.build()).  Raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libgm.so not found at {path}: build it with __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIG.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def lib():
    return load_library()


def _dptr(a):
    """Host float64 numpy array -> POINTER(c_double) (array must stay alive)."""
    return a.ctypes.data_as(_D)


def _tptr(t):
    return C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Solver:
    """One context: a structured grid, an optional fault plane, materials,
    constraints and loads, bound on one GPU."""

    def __init__(self, device: int = 0):
        self._L = load_library()
        h = _P()
        rc = self._L.gm_create(C.byref(h), int(device))
        if rc != 0:
            raise GMError(rc, "gm_create failed")
        self.h = h
        self.device = device
        self.N = self.n_el = self.P = 0

    def close(self):
        if getattr(self, "h", None):
            self._L.gm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != 0:
            msg = self._L.gm_last_error(self.h)
            raise GMError(rc, msg.decode() if msg else "")
        return rc

    # -- set-up --------------------------------------------------------------
    def mesh(self, nx, ny, nz, origin, h, shear=(0.0, 0.0)):
        o = np.ascontiguousarray(origin, np.float64)
        hh = np.ascontiguousarray(h, np.float64)
        s = np.ascontiguousarray(shear, np.float64)
        self._chk(self._L.gm_mesh_structured(self.h, nx, ny, nz, _dptr(o), _dptr(hh), _dptr(s)))

    def fault(self, kf, kn, ks, f, w0, wk_par, k_perp, MF, tn0, tau0):
        fp = FaultParams(kn, ks, f, w0, wk_par, k_perp, MF, tn0, (C.c_double * 2)(*tau0))
        self._chk(self._L.gm_fault_plane(self.h, int(kf), C.byref(fp)))

    def set_preconditioner(self, kind):
        """gm_set_preconditioner: 0 block Jacobi (nodal and lip-pair blocks),
        1 multigrid V-cycle for the FP32 K_T inner solves."""
        self._chk(self._L.gm_set_preconditioner(self.h, int(kind)))

    def set_insitu(self, tn0=None, tau0=None):
        """gm_set_insitu: per-pair in-situ tractions, tn0 (P,) and tau0 (P, 2) in
        the fault frame (t1, t2); None for both restores the uniform values."""
        if tn0 is None and tau0 is None:
            self._chk(self._L.gm_set_insitu(self.h, None, None, self.P))
            return
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(tn0, np.float64), (self.P,)))
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(tau0, np.float64), (self.P, 2)).T)
        self._chk(self._L.gm_set_insitu(self.h, _dptr(a), _dptr(b), self.P))

    def materials(self, E, k, nu, alpha, M, mu_f):
        E = np.ascontiguousarray(np.atleast_1d(E), np.float64)
        k = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(k), E.shape), np.float64)
        self._chk(self._L.gm_set_materials(self.h, _dptr(E), _dptr(k), E.size, nu, alpha, M, mu_f))

    def dirichlet(self, fixed):
        f = np.ascontiguousarray(fixed, np.uint8).reshape(-1)
        self._chk(self._L.gm_set_dirichlet(self.h, f.ctypes.data_as(C.POINTER(C.c_uint8)), f.size))

    def loads(self, fu=None, fp=None):
        a = None if fu is None else np.ascontiguousarray(fu, np.float64).reshape(-1)
        b = None if fp is None else np.ascontiguousarray(fp, np.float64).reshape(-1)
        self._chk(self._L.gm_set_loads(self.h, None if a is None else _dptr(a),
                                       None if b is None else _dptr(b)))

    def bind(self):
        self._chk(self._L.gm_assemble_or_bind(self.h))
        n, e, p = C.c_int64(), C.c_int64(), C.c_int64()
        self._chk(self._L.gm_sizes(self.h, C.byref(n), C.byref(e), C.byref(p)))
        self.N, self.n_el, self.P = n.value, e.value, p.value

    def timestep(self, dt):
        self._chk(self._L.gm_set_timestep(self.h, float(dt)))

    @classmethod
    def from_problem(cls, prob, device: int = 0):
        """Set up from any object with the attributes of a problem description
        (nx, ny, nz, origin, h, shear, kf, fault, E, k, nu, alpha, M, mu_f,
        fixed, fu, fp)."""
        s = cls(device)
        s.mesh(prob.nx, prob.ny, prob.nz, prob.origin, prob.h, prob.shear)
        if prob.kf is not None:
            fp = prob.fault
            per_pair = np.ndim(fp.tn0) > 0 or np.ndim(fp.tau0) > 1
            s.fault(prob.kf, fp.kn, fp.ks, fp.f, fp.w0, fp.wk_par, fp.k_perp, fp.MF,
                    float(np.mean(fp.tn0)), np.mean(np.reshape(fp.tau0, (-1, 2)), axis=0))
        E = np.asarray(prob.E, np.float64)
        s.materials(E, np.broadcast_to(np.asarray(prob.k, np.float64), E.shape), prob.nu, prob.alpha,
                    prob.M, prob.mu_f)
        s.dirichlet(prob.fixed)
        s.loads(prob.fu, prob.fp)
        s.bind()
        if prob.kf is not None and per_pair:
            s.set_insitu(fp.tn0, fp.tau0)
        return s

    # -- operators -------------------------------------------------------------
    def apply(self, which, x, y=None, stream=None):
        """y = A x for which in OP ('KB','KT','A22','APU','AUP','J'); x, y CUDA tensors."""
        import torch
        w = OP[which] if isinstance(which, str) else int(which)
        N = self.N
        shape_out = {0: (3, N), 1: (3, N), 2: (N,), 3: (3, N), 4: (N,), 5: (4, N)}[w]
        if y is None:
            y = torch.empty(shape_out, dtype=x.dtype, device=x.device)
        dt = F64 if x.dtype == torch.float64 else F32
        assert x.is_contiguous() and y.is_contiguous() and y.dtype == x.dtype
        self._chk(self._L.gm_apply_operator(self.h, w, _tptr(x), _tptr(y), dt, _stream_ptr(stream)))
        return y

    def fault_update(self, u, stream=None):
        """Return map at total displacement u (3, N) float64 CUDA tensor."""
        import torch
        P = self.P
        dev = u.device
        out = dict(flags=torch.empty(P, dtype=torch.int8, device=dev),
                   tn=torch.empty(P, dtype=torch.float64, device=dev),
                   ts=torch.empty((2, P), dtype=torch.float64, device=dev),
                   dlie=torch.empty((2, P), dtype=torch.float64, device=dev),
                   T=torch.empty((3, P), dtype=torch.float64, device=dev))
        self._chk(self._L.gm_fault_update(self.h, _tptr(u), _tptr(out["flags"]), _tptr(out["tn"]),
                                          _tptr(out["ts"]), _tptr(out["dlie"]), _tptr(out["T"]),
                                          _stream_ptr(stream)))
        return out

    def pcg(self, which, b, x=None, rtol=1e-10, maxit=10000, stream=None):
        import torch
        w = OP[which] if isinstance(which, str) else int(which)
        if x is None:
            x = torch.zeros_like(b)
        rep = SolveReport()
        self._chk(self._L.gm_pcg_solve(self.h, w, _tptr(b), _tptr(x), rtol, maxit, C.byref(rep),
                                       _stream_ptr(stream)))
        return x, dict(iterations=rep.iterations, rel_residual=rep.rel_residual)

    def prevost(self, b, outer_rtol=1e-10, outer_maxit=500, inner_rtol=1e-12, inner_maxit=20000,
                stream=None):
        import torch
        x = torch.zeros_like(b)
        rep = SolveReport()
        self._chk(self._L.gm_prevost_solve(self.h, _tptr(b), _tptr(x), outer_rtol, outer_maxit,
                                           inner_rtol, inner_maxit, C.byref(rep), _stream_ptr(stream)))
        return x, dict(iterations=rep.iterations, rel_residual=rep.rel_residual)

    def residual(self, du, dp, stream=None):
        import torch
        b = torch.empty((4, self.N), dtype=torch.float64, device=du.device)
        rh = C.c_double()
        self._chk(self._L.gm_residual(self.h, _tptr(du), _tptr(dp), _tptr(b), C.byref(rh),
                                      _stream_ptr(stream)))
        return b, rh.value

    def residual_noalloc(self, du, dp, b=None, stream=None):
        """gm_residual_noalloc: the same residual with no device allocation in
        the call (the output b must be passed or is created here by torch)."""
        import torch
        if b is None:
            b = torch.empty((4, self.N), dtype=torch.float64, device=du.device)
        rh = C.c_double()
        self._chk(self._L.gm_residual_noalloc(self.h, _tptr(du), _tptr(dp), _tptr(b), C.byref(rh),
                                              _stream_ptr(stream)))
        return b, rh.value

    def step(self, dt, newton_rtol=None, precision=F64, newton_maxit=50, outer_rtol=None,
             outer_maxit=500, inner_rtol=None, inner_maxit=20000, schur_precond=0, stream=None):
        """One implicit step.  schur_precond 0: A22^-1 preconditioner of the
        partitioned CG (the paper's); 1: fixed-stress augmented A22."""
        if (newton_rtol is None and outer_rtol is None and inner_rtol is None and precision == F64
                and schur_precond == 0):
            opts = None
        else:
            d_outer = 1e-8 if precision == F64 else 1e-1
            d_inner = 1e-10 if precision == F64 else 1e-2
            opts = StepOpts(1e-10 if newton_rtol is None else newton_rtol, newton_maxit,
                            d_outer if outer_rtol is None else outer_rtol, outer_maxit,
                            d_inner if inner_rtol is None else inner_rtol, inner_maxit, precision,
                            schur_precond)
        rep = StepReport()
        self._chk(self._L.gm_partitioned_step(self.h, float(dt), None if opts is None else C.byref(opts),
                                              C.byref(rep), _stream_ptr(stream)))
        return rep.as_dict()

    # -- state -----------------------------------------------------------------
    def get_state(self):
        N, P = self.N, self.P
        u = np.empty(3 * N)
        p = np.empty(N)
        slip = np.empty(max(2 * P, 1))
        dlie = np.empty(max(2 * P, 1))
        flags = np.empty(max(P, 1), np.int8)
        self._chk(self._L.gm_get_state(self.h, _dptr(u), _dptr(p), _dptr(slip), _dptr(dlie),
                                       flags.ctypes.data_as(C.POINTER(C.c_int8))))
        return dict(u=u.reshape(3, N), p=p, slip=slip[:2 * P].reshape(2, P),
                    dlie=dlie[:2 * P].reshape(2, P), flags=flags[:P])

    def set_state(self, u=None, p=None, dlie=None, flags=None):
        a = None if u is None else np.ascontiguousarray(u, np.float64).reshape(-1)
        b = None if p is None else np.ascontiguousarray(p, np.float64).reshape(-1)
        d = None if dlie is None else np.ascontiguousarray(dlie, np.float64).reshape(-1)
        f = None if flags is None else np.ascontiguousarray(flags, np.int8).reshape(-1)
        self._chk(self._L.gm_set_state(self.h, None if a is None else _dptr(a),
                                       None if b is None else _dptr(b),
                                       None if d is None else _dptr(d),
                                       None if f is None else f.ctypes.data_as(C.POINTER(C.c_int8))))

    def set_permeability(self, k):
        """Element permeabilities (n_el values or one), state kept."""
        a = np.ascontiguousarray(np.atleast_1d(k), np.float64)
        self._chk(self._L.gm_set_permeability(self.h, _dptr(a), a.size))

    def set_friction(self, f):
        """Friction coefficient: one value or one per fault pair."""
        a = np.ascontiguousarray(np.atleast_1d(f), np.float64)
        self._chk(self._L.gm_set_friction(self.h, _dptr(a), a.size))

    def adjoint(self, dJ_du=None, dJ_dp=None, dJ_dslip=None, rtol=1e-10, maxit=300, stream=None):
        """gm_adjoint_step for the last converged step.  Inputs are CUDA
        float64 tensors shaped (3, N), (N,), (2, P) or None.  Returns
        (g_logk (n_el,), g_f (P,), g_logQ float, report)."""
        import torch
        dev = torch.device("cuda", self.device)
        gk = torch.empty(self.n_el, dtype=torch.float64, device=dev)
        gf = torch.zeros(max(self.P, 1), dtype=torch.float64, device=dev)
        gq = C.c_double()
        rep = SolveReport()
        keep = [t.contiguous() if t is not None else None for t in (dJ_du, dJ_dp, dJ_dslip)]
        ptr = [None if t is None else _tptr(t) for t in keep]
        self._chk(self._L.gm_adjoint_step(self.h, ptr[0], ptr[1], ptr[2], _tptr(gk), _tptr(gf),
                                          C.byref(gq), rtol, maxit, C.byref(rep), _stream_ptr(stream)))
        return gk, gf[:self.P], gq.value, dict(iterations=rep.iterations, rel_residual=rep.rel_residual)

    def set_adjoint_options(self, precision=F64, prec_rtol=1e-8, schur_precond=0):
        """gm_set_adjoint_options: precision (F64/F32) and tolerance of the
        adjoint solves' preconditioner, and its Schur preconditioner."""
        self._chk(self._L.gm_set_adjoint_options(self.h, precision, prec_rtol, schur_precond))

    def adjoint_sweep_step(self, dJ_du=None, dJ_dp=None, dJ_dslip=None, lam_next=None,
                           mu_next=None, frozen_next=None, rtol=1e-10, maxit=300, stream=None):
        """gm_adjoint_sweep_step: one step of a multi-step reverse sweep (the
        context must hold the step's state and return map).  Returns
        (lam (4, N), mu (2, P), frozen (6, P), g_logk, g_f, g_logQ)."""
        import torch
        dev = torch.device("cuda", self.device)
        f64 = dict(dtype=torch.float64, device=dev)
        lam = torch.empty((4, self.N), **f64)
        mu = torch.empty((2, self.P), **f64)
        fz = torch.empty((6, self.P), **f64)
        gk = torch.empty(self.n_el, **f64)
        gf = torch.empty(self.P, **f64)
        gq = C.c_double()
        rep = SolveReport()
        ins = [None if t is None else t.contiguous() for t in (dJ_du, dJ_dp, dJ_dslip, lam_next, mu_next, frozen_next)]
        ptr = [None if t is None else _tptr(t) for t in ins]
        self._chk(self._L.gm_adjoint_sweep_step(self.h, *ptr, _tptr(lam), _tptr(mu), _tptr(fz), _tptr(gk),
                                                _tptr(gf), C.byref(gq), rtol, maxit, C.byref(rep),
                                                _stream_ptr(stream)))
        return lam, mu, fz, gk, gf, gq.value

    def counters(self):
        """(kernel launches, bulk operator applies) since bind."""
        a, b = C.c_int64(), C.c_int64()
        self._chk(self._L.gm_counters(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def state_device(self):
        """(u_ptr, p_ptr) raw device pointers of the accepted state."""
        u, p = _P(), _P()
        self._chk(self._L.gm_state_device(self.h, C.byref(u), C.byref(p)))
        return u.value, p.value


def implicit_step_fn():
    """torch.autograd.Function for one implicit step as a function of the
    element log-permeabilities, the friction coefficient and the log scaling
    of the fluid sources.  forward(logk, f, logQ, solver, dt, (fu, fp_base), kw)
    runs gm_partitioned_step from the solver's current state and returns
    (slip (2, P), p (N,)); backward calls gm_adjoint_step.  The solver's state
    advances in forward; restore it with set_state to re-evaluate."""
    import torch

    class ImplicitStep(torch.autograd.Function):
        @staticmethod
        def forward(ctx, logk, f, logQ, solver, dt, loads, kw):
            fu, fp_base = loads
            solver.set_permeability(torch.exp(logk.detach()).cpu().numpy())
            solver.set_friction(np.array([float(f)]))
            solver.loads(fu, np.asarray(fp_base) * float(torch.exp(logQ.detach())))
            solver.step(dt, **(kw or {}))
            st = solver.get_state()
            dev = torch.device("cuda", solver.device)
            ctx.solver = solver
            return (torch.as_tensor(st["slip"], device=dev), torch.as_tensor(st["p"], device=dev))

        @staticmethod
        def backward(ctx, g_slip, g_p):
            s = ctx.solver
            gk, gf, gq, _ = s.adjoint(dJ_dp=g_p.to(torch.float64).contiguous(),
                                      dJ_dslip=g_slip.to(torch.float64).contiguous())
            return (gk, gf.sum(), torch.tensor(gq, dtype=torch.float64, device=gk.device),
                    None, None, None, None)

    return ImplicitStep


class TetSolver:
    """Operators of P1 tetrahedra on an unstructured mesh (include/gm_tet.h):
    argument marshalling only."""

    def __init__(self, device: int = 0):
        self._L = load_library()
        h = _P()
        rc = self._L.gm_tet_create(C.byref(h), int(device))
        if rc != 0:
            raise GMError(rc, "gm_tet_create failed")
        self.h = h
        self.device = device
        self.N = self.M = 0

    def close(self):
        if getattr(self, "h", None):
            self._L.gm_tet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != 0:
            msg = self._L.gm_tet_last_error(self.h)
            raise GMError(rc, msg.decode() if msg else "")

    def mesh(self, nodes, tets):
        x = np.ascontiguousarray(nodes, np.float64).reshape(-1)
        t = np.ascontiguousarray(tets, np.int64).reshape(-1)
        self._chk(self._L.gm_tet_mesh(self.h, _dptr(x), x.size // 3,
                                      t.ctypes.data_as(C.c_void_p), t.size // 4))
        self.N, self.M = x.size // 3, t.size // 4

    def materials(self, E, nu, alpha, M, k, mu_f):
        self._chk(self._L.gm_tet_materials(self.h, float(E), float(nu), float(alpha), float(M), float(k),
                                           float(mu_f)))

    def dirichlet(self, fixed):
        f = np.ascontiguousarray(fixed, np.uint8).reshape(-1)
        self._chk(self._L.gm_tet_dirichlet(self.h, f.ctypes.data_as(C.POINTER(C.c_uint8)), f.size))

    def surface_load(self, tris, sigma0):
        t = np.ascontiguousarray(tris, np.int64).reshape(-1)
        self._chk(self._L.gm_tet_surface_load(self.h, t.ctypes.data_as(C.c_void_p), t.size // 3, float(sigma0)))

    def step(self, dt, u, p, rtol=1e-12, maxit=5000, stream=None):
        """gm_tet_step: u (3, N), p (N,) float64 CUDA tensors updated in place."""
        rep = SolveReport()
        self._chk(self._L.gm_tet_step(self.h, float(dt), _tptr(u), _tptr(p), rtol, maxit, C.byref(rep),
                                      _stream_ptr(stream)))
        return dict(iterations=rep.iterations, rel_residual=rep.rel_residual)

    @classmethod
    def from_problem(cls, prob, device: int = 0):
        """Mesh and materials; for a problem with loads (workloads.TetProblem)
        also its Dirichlet constraints and surface traction."""
        s = cls(device)
        s.mesh(prob.nodes, prob.tets)
        s.materials(prob.E, prob.nu, prob.alpha, prob.M, prob.k, prob.mu_f)
        if getattr(prob, "fixed", None) is not None:
            s.dirichlet(prob.fixed)
        if getattr(prob, "load_tris", None) is not None:
            s.surface_load(prob.load_tris, prob.sigma0)
        return s

    def apply(self, which, x, dt=0.0, y=None, stream=None):
        """y = A x for which in ('KB', 'APU', 'AUP', 'A22', 'J'); x, y CUDA tensors."""
        import torch
        w = OP[which] if isinstance(which, str) else int(which)
        shape_out = {0: (3, self.N), 1: (3, self.N), 2: (self.N,), 3: (3, self.N), 4: (self.N,),
                     5: (4, self.N)}[w]
        if y is None:
            y = torch.empty(shape_out, dtype=x.dtype, device=x.device)
        dt_code = F64 if x.dtype == torch.float64 else F32
        assert x.is_contiguous() and y.is_contiguous() and y.dtype == x.dtype
        self._chk(self._L.gm_tet_apply(self.h, w, _tptr(x), _tptr(y), float(dt), dt_code, _stream_ptr(stream)))
        return y


class TetFaultSolver(TetSolver):
    """P1 tetrahedra with one fault of duplicated nodes and interface elements
    on its triangles (include/gm_tet.h, gm_tet_fault*): argument marshalling
    only.  The state (u (3, N), p (N,)) lives in CUDA float64 tensors owned
    here; the fault history lives in the library."""

    def fault(self, pairs, tris, t1_ref, params):
        pr = np.ascontiguousarray(np.asarray(pairs, np.int64).T).reshape(-1)
        tr = np.ascontiguousarray(tris, np.int64).reshape(-1)
        r = np.ascontiguousarray(t1_ref, np.float64)
        if isinstance(params, FaultParams):
            fp = params
        else:
            if np.ndim(params.tn0) > 0 or np.ndim(params.tau0) > 1:
                raise ValueError("the tetrahedral fault takes uniform in-situ tractions")
            fp = FaultParams(params.kn, params.ks, params.f, params.w0, params.wk_par, params.k_perp,
                             params.MF, float(params.tn0), (C.c_double * 2)(*params.tau0))
        self._chk(self._L.gm_tet_fault(self.h, pr.ctypes.data_as(C.c_void_p), pr.size // 2,
                                       tr.ctypes.data_as(C.c_void_p), tr.size // 3, _dptr(r), C.byref(fp)))
        self.P = pr.size // 2

    def loads(self, fu=None, fp=None):
        a = None if fu is None else np.ascontiguousarray(fu, np.float64).reshape(-1)
        b = None if fp is None else np.ascontiguousarray(fp, np.float64).reshape(-1)
        self._chk(self._L.gm_tet_loads(self.h, None if a is None else _dptr(a), None if b is None else _dptr(b)))

    def fault_apply(self, which, x, dt=0.0, stream=None):
        """gm_tet_fault_apply for which in ('KT', 'APU', 'AUP', 'A22'); float64 CUDA tensors."""
        import torch
        w = OP[which] if isinstance(which, str) else int(which)
        y = torch.empty({1: (3, self.N), 2: (self.N,), 3: (3, self.N), 4: (self.N,)}[w], dtype=torch.float64,
                        device=x.device)
        assert x.dtype == torch.float64 and x.is_contiguous()
        self._chk(self._L.gm_tet_fault_apply(self.h, w, _tptr(x), _tptr(y), float(dt), _stream_ptr(stream)))
        return y

    def fault_step(self, dt, u, p, newton_rtol=1e-12, newton_maxit=50, outer_rtol=None, outer_maxit=5000,
                   inner_rtol=None, inner_maxit=20000, precision=F64, stream=None):
        """gm_tet_fault_step: u (3, N), p (N,) float64 CUDA tensors updated in place.
        precision F32 runs the inner K_T solves in FP32 inside the FP64 Newton
        loop; the tolerances default to 1e-11 / 1e-13 (outer / inner) in FP64
        and to 1e-1 / 1e-2 in FP32, where Newton refines the inexact solves."""
        if outer_rtol is None:
            outer_rtol = 1e-11 if precision == F64 else 1e-1
        if inner_rtol is None:
            inner_rtol = 1e-13 if precision == F64 else 1e-2
        o = StepOpts(newton_rtol, newton_maxit, outer_rtol, outer_maxit, inner_rtol, inner_maxit, precision, 0)
        rep = StepReport()
        self._chk(self._L.gm_tet_fault_step(self.h, float(dt), _tptr(u), _tptr(p), C.byref(o), C.byref(rep),
                                            _stream_ptr(stream)))
        return rep.as_dict()

    def fault_state(self):
        flags = np.zeros(self.P, np.int8)
        slip = np.zeros(2 * self.P)
        dlie = np.zeros(2 * self.P)
        self._chk(self._L.gm_tet_fault_state(self.h, flags.ctypes.data_as(C.POINTER(C.c_int8)), _dptr(slip),
                                             _dptr(dlie)))
        return dict(flags=flags, slip=slip.reshape(2, self.P).T.copy(), dlie=dlie.reshape(2, self.P).T.copy())

    @classmethod
    def from_problem(cls, prob, device: int = 0):
        """A workloads.FaultedTetProblem: mesh, uniform materials, constraints,
        loads and the fault."""
        E = np.asarray(prob.E, float)
        k = np.asarray(prob.k, float)
        if np.any(E != E.flat[0]) or np.any(k != k.flat[0]):
            raise ValueError("the tetrahedral path takes uniform E and k")
        s = cls(device)
        s.mesh(prob.nodes, prob.tets)
        s.materials(E.flat[0], prob.nu, prob.alpha, prob.M, k.flat[0], prob.mu_f)
        s.dirichlet(prob.fixed)
        s.loads(prob.fu, prob.fp)
        s.fault(prob.pairs, prob.fault_tris, prob.t1_ref, prob.fault)
        return s


def run_until_slip(solver, dts, Q, step_kw=None):
    """Step through dts until the first pair is in the slipping state (the
    onset of inelastic slip, Sec. 5) and return (steps taken, elapsed time,
    injected volume Q * time, final state); (len(dts), t, Q t, state) with
    state["flags"] free of slip if no pair slipped.  Sequences library calls
    only: solver.step(dt, **step_kw) and solver.get_state()."""
    kw = dict(step_kw or {})
    t = 0.0
    st = None
    for n, dt in enumerate(dts):
        solver.step(dt, **kw)
        t += dt
        st = solver.get_state()
        if np.any(np.asarray(st["flags"]) == SLIP):
            return n + 1, t, Q * t, st
    return len(dts), t, Q * t, st


def run_with_adjoint(solver, dts, objective_grad, checkpoint_every=5, step_kw=None, rtol=1e-10, maxit=300):
    """Run len(dts) implicit steps from the solver's current state, then the
    reverse sweep of the multi-step adjoint (inelastic slip as history).

    objective_grad(final_state) returns (dJ_du, dJ_dp, dJ_dslip) for an
    objective of the final state (CUDA float64 tensors shaped (3, N), (N,),
    (2, P), or None).  Forward states are checkpointed on the host every
    `checkpoint_every` steps; each segment is recomputed from its checkpoint
    during the sweep.  Every computation runs in the library; this function
    only sequences calls.  Returns (final_state, g_logk, g_f, g_logQ) with
    g_f per pair; the solver ends holding the final state."""
    import torch
    kw = dict(step_kw or {})
    K = len(dts)
    dev = torch.device("cuda", solver.device)
    ckpt = {0: solver.get_state()}
    for n in range(K):
        solver.step(dts[n], **kw)
        if (n + 1) % checkpoint_every == 0 and n + 1 < K:
            ckpt[n + 1] = solver.get_state()
    final = solver.get_state()
    dJ_du, dJ_dp, dJ_dslip = objective_grad(final)
    g_logk = torch.zeros(solver.n_el, dtype=torch.float64, device=dev)
    g_f = torch.zeros(solver.P, dtype=torch.float64, device=dev)
    g_logQ = 0.0
    lam = mu = fz = None
    starts = sorted(ckpt)
    for si, s0 in enumerate(reversed(starts)):
        s1 = K if si == 0 else starts[len(starts) - si]
        solver.set_state(u=ckpt[s0]["u"], p=ckpt[s0]["p"], dlie=ckpt[s0]["dlie"], flags=ckpt[s0]["flags"])
        states = {s0: ckpt[s0]}
        for n in range(s0, s1):
            solver.step(dts[n], **kw)
            states[n + 1] = solver.get_state()
        for n in range(s1, s0, -1):
            st, prev = states[n], states[n - 1]
            solver.set_state(u=st["u"], p=st["p"], dlie=prev["dlie"], flags=st["flags"])
            solver.timestep(dts[n - 1])
            solver.fault_update(torch.as_tensor(st["u"], device=dev))
            last = n == K
            lam, mu, fz, gk, gf, gq = solver.adjoint_sweep_step(
                dJ_du if last else None, dJ_dp if last else None, dJ_dslip if last else None,
                lam, mu, fz, rtol=rtol, maxit=maxit)
            g_logk += gk
            g_f += gf
            g_logQ += gq
    solver.set_state(u=final["u"], p=final["p"], dlie=final["dlie"], flags=final["flags"])
    return final, g_logk, g_f, g_logQ
