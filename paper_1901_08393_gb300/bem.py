"""Thin ctypes binding of libbem_gb300.so (C ABI in include/bem.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  Arrays may be numpy arrays (host) or torch tensors (host or CUDA);
PyTorch is used only to supply the CUDA stream and device buffers.  If the
compiled library is missing the binding raises instead of falling back to any
other implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbem_gb300.so")

BEM_OK = 0
BEM_ERR_INVALID = -1
BEM_ERR_OOM = -2
BEM_ERR_NOT_CONVERGED = -3
BEM_ERR_MESH = -4
BEM_ERR_CUDA = -5
PREC_F64 = 0
PREC_F32 = 1
PREC_DF64 = 2
PRECOND_NONE = 0
PRECOND_JACOBI = 1
PRECOND_BLOCK = 2
PRECOND_CALDERON = 3
FAR_TILE_VARIANTS = 14
REFINE_BISEC3 = 1
BASIS_P0 = 0
BASIS_DUAL = 1

EXPORTS = [
    "bem_context_create", "bem_context_destroy", "bem_last_error", "bem_context_memory",
    "bem_mesh_upload", "bem_mesh_destroy", "bem_mesh_info", "bem_mesh_download", "bem_mesh_geometry",
    "bem_assemble_V", "bem_assemble_V_update", "bem_operator_destroy", "bem_operator_info",
    "bem_operator_read", "bem_operator_entries", "bem_operator_matvec", "bem_solve_capacity",
    "bem_zz_estimate", "bem_dorfler", "bem_refine", "bem_mark_refine", "bem_adaptive_run",
    "bem_profile_enable", "bem_profile_read", "bem_launch_count", "bem_operator_matvec_noalloc", "bem_context_set_persistent",
    "bem_server_create", "bem_server_submit", "bem_server_wait", "bem_server_stats", "bem_server_destroy",
    "bem_server_profile_enable", "bem_server_profile_read",
    "bem_batch_create", "bem_batch_run", "bem_batch_info", "bem_batch_destroy",
    "bem_mesh_barycentric", "bem_operator_dual", "bem_zz_estimate_dual", "bem_operator_preconditioner",
    "bem_far_tiles", "bem_debug_barrier_fault", "bem_batch_waves",
]
PRODUCTS_DEFAULT, PRODUCTS_FP32, PRODUCTS_FP16 = 0, 1, 2
KERNEL_FAR = 0
KERNEL_NEAR = 1
KERNEL_MATVEC = 2


class AssemblyOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("ss_order", C.c_int32), ("tile", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_it", C.c_int32), ("precond", C.c_int32),
                ("max_outer", C.c_int32), ("inner_tol", C.c_double), ("reliable_delta", C.c_double),
                ("inexact_lambda", C.c_double), ("h_mode", C.c_int32), ("products", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("outer", C.c_int32), ("relres", C.c_double),
                ("converged", C.c_int32), ("lambda_min", C.c_double), ("lambda_max", C.c_double)]


class LevelRecord(C.Structure):
    _fields_ = [("N", C.c_int64), ("M", C.c_int64), ("cap", C.c_double), ("eta2_total", C.c_double),
                ("iterations", C.c_int32), ("n_marked", C.c_int32), ("relres", C.c_double),
                ("ms_assemble", C.c_double), ("ms_solve", C.c_double), ("ms_adapt", C.c_double),
                ("outer", C.c_int32)]


class AdaptiveOpts(C.Structure):
    _fields_ = [("theta", C.c_double), ("max_N", C.c_int64), ("max_levels", C.c_int32),
                ("h_mode", C.c_int32), ("assembly", AssemblyOpts), ("solve", SolveOpts),
                ("incremental", C.c_int32), ("basis", C.c_int32)]


SERVER_HISTORY = 16


class RequestResult(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("done", C.c_int32), ("levels", C.c_int32),
                ("N_final", C.c_int64), ("cap", C.c_double), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("estimate_bytes", C.c_int64),
                ("cap_history", C.c_double * SERVER_HISTORY), ("N_history", C.c_int64 * SERVER_HISTORY),
                ("message", C.c_char * 256)]


class BatchResult(C.Structure):
    _fields_ = [("cap", C.c_double), ("iterations", C.c_int32), ("outer", C.c_int32), ("relres", C.c_double),
                ("converged", C.c_int32), ("status", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int64), ("in_flight", C.c_int64), ("peak_in_flight", C.c_int64),
                ("in_flight_bytes", C.c_int64), ("peak_bytes", C.c_int64), ("budget", C.c_int64),
                ("clock", C.c_double)]


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bem error {code}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing: run __graft_entry__.build() first")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    P = C.POINTER
    sig = {
        "bem_context_create": [vp, i64, P(vp)],
        "bem_context_destroy": [vp],
        "bem_context_memory": [vp, P(i64)],
        "bem_mesh_upload": [vp, vp, i64, vp, i64, vp, P(vp)],
        "bem_mesh_destroy": [vp],
        "bem_mesh_info": [vp, P(i64), P(i64), P(i64)],
        "bem_mesh_download": [vp, vp, vp, vp, vp],
        "bem_mesh_geometry": [vp, vp, vp],
        "bem_assemble_V": [vp, P(AssemblyOpts), P(vp)],
        "bem_assemble_V_update": [vp, vp, P(AssemblyOpts), P(vp)],
        "bem_operator_destroy": [vp],
        "bem_operator_info": [vp, P(i64), P(i32)],
        "bem_operator_read": [vp, i64, i64, i64, i64, vp],
        "bem_operator_entries": [vp, vp, vp, i64, vp],
        "bem_operator_matvec": [vp, vp, vp],
        "bem_solve_capacity": [vp, P(SolveOpts), vp, P(d), vp, P(SolveInfo)],
        "bem_zz_estimate": [vp, vp, i32, vp, vp],
        "bem_dorfler": [vp, vp, i64, d, vp, P(i64)],
        "bem_refine": [vp, vp, i32, P(vp)],
        "bem_mark_refine": [vp, vp, d, i32, vp, P(i64), P(vp)],
        "bem_adaptive_run": [vp, P(AdaptiveOpts), P(LevelRecord), P(i32), P(vp)],
        "bem_profile_enable": [vp, i32],
        "bem_profile_read": [vp, i32, P(i64), P(d), P(d)],
        "bem_launch_count": [vp, P(i64)],
        "bem_operator_matvec_noalloc": [vp, vp, vp],
        "bem_context_set_persistent": [vp, i32],
        "bem_server_create": [i32, i64, P(AdaptiveOpts), P(vp)],
        "bem_server_submit": [vp, vp, i64, vp, i64, i32, i64, P(i64)],
        "bem_server_wait": [vp, i64, P(RequestResult)],
        "bem_server_stats": [vp, P(ServerStats)],
        "bem_server_destroy": [vp],
        "bem_server_profile_enable": [vp, i32],
        "bem_server_profile_read": [vp, i32, P(i64), P(C.c_double), P(C.c_double)],
        "bem_batch_create": [vp, i32, vp, P(AssemblyOpts), P(SolveOpts), i32, P(vp)],
        "bem_batch_run": [vp, vp],
        "bem_batch_info": [vp, P(i32), P(i32), P(i32)],
        "bem_batch_destroy": [vp],
        "bem_mesh_barycentric": [vp, P(vp)],
        "bem_operator_dual": [vp, vp, P(vp)],
        "bem_zz_estimate_dual": [vp, vp, i32, vp, vp],
        "bem_operator_preconditioner": [vp, i32, vp],
        "bem_far_tiles": [vp, vp],
        "bem_debug_barrier_fault": [vp, i64, i32],
        "bem_batch_waves": [vp, P(i32), P(i64), vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int32
    L.bem_last_error.argtypes = [vp]
    L.bem_last_error.restype = C.c_char_p
    _lib = L
    return L


def _arr(a, dtype):
    """(keep-alive object, pointer) for a numpy array or a torch tensor."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch

        tdt = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8,
               np.int64: torch.int64, np.float32: torch.float32}[dtype]
        t = a.contiguous()
        if t.dtype != tdt:
            t = t.to(tdt)
        return t, t.data_ptr()
    x = np.ascontiguousarray(a, dtype=dtype)
    return x, x.ctypes.data


def _current_stream():
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


class Context:
    """Library context bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None, hbm_budget_bytes: int = 0):
        L = lib()
        h = C.c_void_p()
        s = _current_stream() if stream is None else int(stream)
        st = L.bem_context_create(C.c_void_p(s), int(hbm_budget_bytes), C.byref(h))
        if st != BEM_OK:
            raise BemError(st, "context creation failed (no CUDA device?)")
        self.h = h
        self.L = L

    def check(self, st):
        if st != BEM_OK:
            raise BemError(st, self.L.bem_last_error(self.h).decode())

    def memory_in_use(self) -> int:
        v = C.c_int64()
        self.check(self.L.bem_context_memory(self.h, C.byref(v)))
        return int(v.value)

    def profile(self, on: bool = True):
        self.check(self.L.bem_profile_enable(self.h, int(on)))

    def profile_read(self, kernel: int):
        n, ms, u = C.c_int64(), C.c_double(), C.c_double()
        self.check(self.L.bem_profile_read(self.h, kernel, C.byref(n), C.byref(ms), C.byref(u)))
        return int(n.value), float(ms.value), float(u.value)

    def set_persistent(self, on: bool):
        self.check(self.L.bem_context_set_persistent(self.h, int(on)))

    def far_tiles(self):
        """Autotuned far-field tile variant per (precision, size class); 0 = not yet timed."""
        out = (C.c_int32 * 12)()
        self.check(self.L.bem_far_tiles(self.h, out))
        return [list(out[4 * p:4 * p + 4]) for p in range(3)]

    def barrier_fault(self, wait_limit_ns: int = 0, absent_cta: int = -1):
        """Failure-detection hook of the persistent solvers: grid-barrier wait limit
        (0: default 2 s) and a CTA that leaves at its first barrier (-1: none)."""
        self.check(self.L.bem_debug_barrier_fault(self.h, int(wait_limit_ns), int(absent_cta)))

    def launch_count(self) -> int:
        n = C.c_int64()
        self.check(self.L.bem_launch_count(self.h, C.byref(n)))
        return int(n.value)

    def last_error(self) -> str:
        return self.L.bem_last_error(self.h).decode()

    def close(self):
        if self.h:
            self.L.bem_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx: Context, handle):
        self.ctx, self.h = ctx, handle

    @classmethod
    def upload(cls, ctx: Context, verts, tris, ref_edge=None):
        v, pv = _arr(verts, np.float64)
        t, pt = _arr(tris, np.int32)
        r, pr = _arr(ref_edge, np.uint8)
        M = int(v.shape[0]) if len(v.shape) == 2 else int(v.shape[0]) // 3
        N = int(t.shape[0]) if len(t.shape) == 2 else int(t.shape[0]) // 3
        h = C.c_void_p()
        ctx.check(ctx.L.bem_mesh_upload(ctx.h, pv, M, pt, N, pr, C.byref(h)))
        return cls(ctx, h)

    def info(self):
        M, N, nn = C.c_int64(), C.c_int64(), C.c_int64()
        self.ctx.check(self.ctx.L.bem_mesh_info(self.h, C.byref(M), C.byref(N), C.byref(nn)))
        return int(M.value), int(N.value), int(nn.value)

    @property
    def N(self):
        return self.info()[1]

    @property
    def M(self):
        return self.info()[0]

    def download(self):
        M, N, _ = self.info()
        v = np.zeros((M, 3))
        t = np.zeros((N, 3), dtype=np.int32)
        p = np.zeros(N, dtype=np.int32)
        k = np.zeros(N, dtype=np.uint8)
        self.ctx.check(self.ctx.L.bem_mesh_download(self.h, v.ctypes.data, t.ctypes.data, p.ctypes.data,
                                                    k.ctypes.data))
        return v, t, p, k

    def barycentric(self) -> "Mesh":
        """Barycentric refinement (Sec. 2.1): children of triangle T at 6T .. 6T+5."""
        h = C.c_void_p()
        self.ctx.check(self.ctx.L.bem_mesh_barycentric(self.h, C.byref(h)))
        return Mesh(self.ctx, h)

    def geometry(self):
        N = self.N
        a, d = np.zeros(N), np.zeros(N)
        self.ctx.check(self.ctx.L.bem_mesh_geometry(self.h, a.ctypes.data, d.ctypes.data))
        return a, d

    def close(self):
        # a handle outlived by its context was released with the context's memory pool
        if self.h and self.ctx.h:
            self.ctx.L.bem_mesh_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    def __init__(self, mesh: Mesh, handle):
        self.mesh, self.ctx, self.h = mesh, mesh.ctx, handle

    @classmethod
    def assemble(cls, mesh: Mesh, precision=PREC_F64, ss_order=4, tile=0):
        o = AssemblyOpts(precision, ss_order, tile)
        h = C.c_void_p()
        mesh.ctx.check(mesh.ctx.L.bem_assemble_V(mesh.h, C.byref(o), C.byref(h)))
        return cls(mesh, h)

    @classmethod
    def update(cls, fine: Mesh, coarse: "Operator"):
        h = C.c_void_p()
        fine.ctx.check(fine.ctx.L.bem_assemble_V_update(fine.h, coarse.h, None, C.byref(h)))
        return cls(fine, h)

    @classmethod
    def dual(cls, bary_op: "Operator", mesh: Mesh):
        """V^dual = P^T V^bary P (Sec. 2.6) of mesh, from the operator of its barycentric
        refinement; an M x M operator, one unknown per vertex."""
        h = C.c_void_p()
        mesh.ctx.check(mesh.ctx.L.bem_operator_dual(bary_op.h, mesh.h, C.byref(h)))
        return cls(mesh, h)

    def info(self):
        N, p = C.c_int64(), C.c_int32()
        self.ctx.check(self.ctx.L.bem_operator_info(self.h, C.byref(N), C.byref(p)))
        return int(N.value), int(p.value)

    def read(self, i0=0, ni=None, j0=0, nj=None):
        N, p = self.info()
        ni = N - i0 if ni is None else ni
        nj = N - j0 if nj is None else nj
        out = np.zeros((ni, nj), dtype=np.float32 if p == PREC_F32 else np.float64)
        self.ctx.check(self.ctx.L.bem_operator_read(self.h, i0, ni, j0, nj, out.ctypes.data))
        return out

    def entries(self, I, J):
        Ia, pI = _arr(I, np.int64)
        Ja, pJ = _arr(J, np.int64)
        out = np.zeros(int(Ia.shape[0]))
        self.ctx.check(self.ctx.L.bem_operator_entries(self.h, pI, pJ, int(Ia.shape[0]), out.ctypes.data))
        return out

    def preconditioner(self, which=0):
        """D^reg (which=0) or C = S D^reg S (which=1) of a dual operator (Sec. 2.6), FP32, M x M."""
        N = self.info()[0]
        out = np.zeros((N, N), dtype=np.float32)
        self.ctx.check(self.ctx.L.bem_operator_preconditioner(self.h, which, out.ctypes.data))
        return out

    def matvec(self, x):
        xa, px = _arr(x, np.float64)
        y = np.zeros(int(xa.shape[0]))
        self.ctx.check(self.ctx.L.bem_operator_matvec(self.h, px, y.ctypes.data))
        return y

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.L.bem_operator_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_capacity(op: Operator, tol=1e-10, max_it=10000, precond=PRECOND_JACOBI, x0=None,
                   max_outer=20, inner_tol=1e-5, phi_out=None, raise_not_converged=True, reliable_delta=0.0,
                   inexact_lambda=0.0, h_mode=0, products=0):
    """Cap and x with V x = |T| (Eq. 2.5, 2.8).  phi_out may be a CUDA tensor."""
    o = SolveOpts(tol, max_it, precond, max_outer, inner_tol, reliable_delta, inexact_lambda, h_mode, products)
    info = SolveInfo()
    cap = C.c_double()
    N = op.info()[0]
    x0a, px0 = _arr(x0, np.float64)
    if phi_out is None:
        phi = np.zeros(N)
        pphi = phi.ctypes.data
    else:
        phi, pphi = phi_out, phi_out.data_ptr()
    st = op.ctx.L.bem_solve_capacity(op.h, C.byref(o), px0, C.byref(cap), pphi, C.byref(info))
    if st != BEM_OK and (st != BEM_ERR_NOT_CONVERGED or raise_not_converged):
        op.ctx.check(st)
    return float(cap.value), phi, {"iterations": info.iterations, "outer": info.outer,
                                   "relres": info.relres, "converged": bool(info.converged),
                                   "lambda_min": info.lambda_min, "lambda_max": info.lambda_max}


def zz_estimate(mesh: Mesh, phi, h_mode=0):
    pa, pp = _arr(phi, np.float64)
    N = mesh.N
    eta2 = np.zeros(N)
    tot = np.zeros(2)
    mesh.ctx.check(mesh.ctx.L.bem_zz_estimate(mesh.h, pp, h_mode, eta2.ctypes.data, tot.ctypes.data))
    return eta2, float(tot[0]), float(tot[1])


def zz_estimate_dual(mesh: Mesh, x, h_mode=0):
    """eta(T)^2 of Eq. 1.6 for the dual solution x (one value per vertex of mesh)."""
    xa, px = _arr(x, np.float64)
    eta2 = np.zeros(mesh.N)
    tot = np.zeros(2)
    mesh.ctx.check(mesh.ctx.L.bem_zz_estimate_dual(mesh.h, px, h_mode, eta2.ctypes.data, tot.ctypes.data))
    return eta2, float(tot[0]), float(tot[1])


def dorfler(ctx: Context, eta2, theta=0.5):
    ea, pe = _arr(eta2, np.float64)
    N = int(ea.shape[0])
    m = np.zeros(N, dtype=np.uint8)
    nm = C.c_int64()
    ctx.check(ctx.L.bem_dorfler(ctx.h, pe, N, theta, m.ctypes.data if N else None, C.byref(nm)))
    return m, int(nm.value)


def refine(mesh: Mesh, marked, bisec3=False) -> Mesh:
    ma, pm = _arr(marked, np.uint8)
    h = C.c_void_p()
    mesh.ctx.check(mesh.ctx.L.bem_refine(mesh.h, pm, REFINE_BISEC3 if bisec3 else 0, C.byref(h)))
    return Mesh(mesh.ctx, h)


def mark_refine(mesh: Mesh, eta2, theta=0.5, bisec3=False):
    ea, pe = _arr(eta2, np.float64)
    N = mesh.N
    m = np.zeros(N, dtype=np.uint8)
    nm = C.c_int64()
    h = C.c_void_p()
    mesh.ctx.check(mesh.ctx.L.bem_mark_refine(mesh.h, pe, theta, REFINE_BISEC3 if bisec3 else 0,
                                              m.ctypes.data, C.byref(nm), C.byref(h)))
    return m, int(nm.value), Mesh(mesh.ctx, h)


def adaptive_run(mesh: Mesh, theta=0.5, max_N=20000, max_levels=64, h_mode=0, precision=PREC_F64,
                 ss_order=4, tol=1e-12, max_it=20000, precond=PRECOND_JACOBI, incremental=True,
                 max_outer=20, inner_tol=1e-5, want_final=False, reliable_delta=0.0, inexact_lambda=0.0,
                 basis=BASIS_P0, tile=0, products=0):
    """Alg. 1 in the library's native loop; returns (records, final Mesh or None)."""
    o = AdaptiveOpts(theta, max_N, max_levels, h_mode, AssemblyOpts(precision, ss_order, tile),
                     SolveOpts(tol, max_it, precond, max_outer, inner_tol, reliable_delta, inexact_lambda, h_mode,
                               products),
                     int(incremental), int(basis))
    recs = (LevelRecord * max_levels)()
    n = C.c_int32()
    fin = C.c_void_p()
    mesh.ctx.check(mesh.ctx.L.bem_adaptive_run(mesh.h, C.byref(o), recs, C.byref(n),
                                               C.byref(fin) if want_final else None))
    out = [{f: getattr(recs[k], f) for f, _ in LevelRecord._fields_} for k in range(n.value)]
    return out, (Mesh(mesh.ctx, fin) if want_final and fin.value else None)


class Batch:
    """Independent problems assembled and solved together (bem_batch_*), in waves
    that fit the device memory: per wave one launch per assembly phase and one
    cooperative launch of the solver; with use_graph each wave is recorded as a CUDA
    graph once and replayed."""

    def __init__(self, ctx: Context, meshes, precision=PREC_DF64, ss_order=4, tol=1e-10, max_it=10000,
                 precond=PRECOND_JACOBI, reliable_delta=0.0, use_graph=True, tile=0, products=0):
        self.ctx, self.meshes, self.h = ctx, list(meshes), None
        arr = (C.c_void_p * len(self.meshes))(*[m.h.value if hasattr(m.h, "value") else m.h for m in self.meshes])
        h = C.c_void_p()
        ctx.check(ctx.L.bem_batch_create(ctx.h, len(self.meshes), arr, C.byref(AssemblyOpts(precision, ss_order, tile)),
                                         C.byref(SolveOpts(tol, max_it, precond, 20, 1e-5, reliable_delta, 0.0, 0,
                                                           products)),
                                         int(bool(use_graph)), C.byref(h)))
        self.h = h

    def run(self, raise_not_converged=True):
        """Assemble and solve every problem; a list of result dicts."""
        res = (BatchResult * len(self.meshes))()
        st = self.ctx.L.bem_batch_run(self.h, res)
        if st != BEM_OK and (st != BEM_ERR_NOT_CONVERGED or raise_not_converged):
            self.ctx.check(st)
        return [{f: getattr(r, f) for f, _ in BatchResult._fields_} for r in res]

    def info(self):
        n, g, used = C.c_int32(), C.c_int32(), C.c_int32()
        self.ctx.check(self.ctx.L.bem_batch_info(self.h, C.byref(n), C.byref(g), C.byref(used)))
        return {"count": n.value, "ctas": g.value, "graph_used": used.value}

    def waves(self):
        """(number of waves, arena bytes, wave of each problem)."""
        w, b = C.c_int32(), C.c_int64()
        of = np.zeros(len(self.meshes), dtype=np.int32)
        self.ctx.check(self.ctx.L.bem_batch_waves(self.h, C.byref(w), C.byref(b), of.ctypes.data))
        return int(w.value), int(b.value), of

    def close(self):
        if self.h is not None and self.ctx.h:
            self.ctx.L.bem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (bem_server_*): submit meshes, wait for results."""

    def __init__(self, slots=4, hbm_budget_bytes=64 << 30, theta=0.5, precision=PREC_F32, tol=1e-10,
                 max_it=20000, h_mode=0, ss_order=4, incremental=True, max_outer=20, inner_tol=1e-5,
                 reliable_delta=0.0, precond=PRECOND_JACOBI, basis=BASIS_P0, products=0):
        self.L = lib()
        o = AdaptiveOpts(theta, 0, 1, h_mode, AssemblyOpts(precision, ss_order),
                         SolveOpts(tol, max_it, precond, max_outer, inner_tol, reliable_delta, 0.0, h_mode, products),
                         int(incremental), int(basis))
        h = C.c_void_p()
        st = self.L.bem_server_create(slots, int(hbm_budget_bytes), C.byref(o), C.byref(h))
        if st != BEM_OK:
            raise BemError(st, "server creation failed")
        self.h = h

    def submit(self, verts, tris, max_levels, max_N):
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        rid = C.c_int64()
        st = self.L.bem_server_submit(self.h, v.ctypes.data, v.shape[0], t.ctypes.data, t.shape[0],
                                      int(max_levels), int(max_N), C.byref(rid))
        if st != BEM_OK:
            raise BemError(st, "submit failed")
        return int(rid.value)

    def wait(self, rid):
        r = RequestResult()
        st = self.L.bem_server_wait(self.h, rid, C.byref(r))
        if st != BEM_OK:
            raise BemError(st, "unknown request")
        n = min(r.levels, SERVER_HISTORY)
        return {"id": r.id, "status": r.status, "levels": r.levels, "N_final": r.N_final, "cap": r.cap,
                "t_submit": r.t_submit, "t_start": r.t_start, "t_done": r.t_done,
                "estimate_bytes": r.estimate_bytes, "caps": list(r.cap_history[:n]),
                "Ns": list(r.N_history[:n]), "message": r.message.decode(errors="replace")}

    def profile(self, on: bool = True):
        """Profile the slots' hot kernels from each slot's next request on."""
        st = self.L.bem_server_profile_enable(self.h, int(on))
        if st != BEM_OK:
            raise BemError(st, "server profile enable failed")

    def profile_read(self, kernel: int):
        """(launches, ms, units) summed over the slots; the server must be idle."""
        n, ms, u = C.c_int64(), C.c_double(), C.c_double()
        st = self.L.bem_server_profile_read(self.h, int(kernel), C.byref(n), C.byref(ms), C.byref(u))
        if st != BEM_OK:
            raise BemError(st, "server profile read needs an idle server")
        return int(n.value), float(ms.value), float(u.value)

    def stats(self):
        s = ServerStats()
        self.L.bem_server_stats(self.h, C.byref(s))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.h:
            self.L.bem_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
