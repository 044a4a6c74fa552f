"""ctypes binding of the C ABI in include/sg.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

SG_FP64, SG_MIXED, SG_FP32, SG_BF16 = 0, 1, 2, 3
SG_WARM_PREV, SG_WARM_LEARNED = 0, 1
SG_PC_NN2, SG_PC_NN1, SG_PC_LUMPED = 0, 1, 2
SG_ENOTCONV = -4


class SGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sg error {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("N", C.c_int), ("nsub_x", C.c_int), ("nsub_y", C.c_int)]


class KL(C.Structure):
    _fields_ = [("M", C.c_int), ("sigma", C.c_double), ("bx", C.c_double), ("by", C.c_double), ("g0", C.c_double),
                ("modes", C.c_void_p), ("lambdas", C.c_void_p)]


class PCE(C.Structure):
    _fields_ = [("p", C.c_int), ("p_in", C.c_int)]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("tol", C.c_double), ("alpha0", C.c_double), ("alpha1", C.c_double),
                ("max_iter", C.c_int), ("precision", C.c_int), ("warm", C.c_int),
                ("inner_tol", C.c_double), ("inner_max_iter", C.c_int), ("autotune", C.c_int),
                ("warm_train_steps", C.c_int), ("warm_lr", C.c_double), ("precond", C.c_int)]


class Mesh(C.Structure):
    _fields_ = [("nv", C.c_int), ("xy", C.c_void_p), ("dirichlet", C.c_void_p), ("ne", C.c_int),
                ("tri", C.c_void_p), ("part", C.c_void_p)]


class MeshPlan(C.Structure):
    _fields_ = [("nsub", C.c_int), ("n_free", C.c_int), ("n_gamma", C.c_int), ("n_corner", C.c_int), ("P", C.c_int),
                ("P_in", C.c_int), ("nnz_G", C.c_int), ("n_sub_nodes", C.c_int), ("max_owners", C.c_int),
                ("max_corners", C.c_int), ("max_gamma", C.c_int), ("row_entries", C.c_longlong),
                ("coarse_dim", C.c_longlong), ("bytes_rows", C.c_longlong), ("bytes_inverses", C.c_longlong),
                ("bytes_coarse_basis", C.c_longlong), ("bytes_coarse_matrix", C.c_longlong),
                ("bytes_vectors", C.c_longlong), ("mma", C.c_int), ("fits", C.c_int)]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int), ("x0", C.c_double), ("y0", C.c_double), ("width", C.c_double),
                ("freq", C.c_double), ("amp", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int), ("step_index", C.c_int), ("iters_last", C.c_int),
                ("iters_total", C.c_longlong), ("inner_total", C.c_longlong), ("relres_last", C.c_double),
                ("ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Sizes(C.Structure):
    _fields_ = [("N", C.c_int), ("nsub", C.c_int), ("P", C.c_int), ("P_in", C.c_int), ("n_free", C.c_int),
                ("n_gamma", C.c_int), ("n_corner", C.c_int), ("n_sub_nodes", C.c_int),
                ("device_bytes", C.c_longlong), ("fp32_precond", C.c_int), ("compiled_apply", C.c_int)]


class Plan(C.Structure):
    _fields_ = [("L", C.c_int), ("P", C.c_int), ("P_in", C.c_int), ("nsub", C.c_int), ("nnz_G", C.c_int),
                ("apply_variant", C.c_int * 2), ("apply_lines", C.c_int * 2), ("apply_tiles", C.c_int * 2),
                ("apply_smem", C.c_longlong * 2), ("line_kind", C.c_int * 2), ("line_modes", C.c_int * 2),
                ("line_groups", C.c_int * 2), ("line_block", (C.c_int * 3) * 2), ("line_smem", C.c_longlong * 2),
                ("mma", C.c_int), ("mma_kp", C.c_int), ("mma_nc", C.c_int), ("mma_mt", C.c_int),
                ("mma_nb", C.c_int), ("mma_smem", C.c_longlong), ("fits", C.c_int)]


def _plain(v):
    if isinstance(v, C.Array):
        return [_plain(x) for x in v]
    return v


_LIB = None


def library_path() -> str:
    return _build.OUT


def load_library(path: Optional[str] = None):
    """Load libsg; raises if it is missing (there is no fallback implementation)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run paper_2512_23027_gb300.build.build())")
    lib = C.CDLL(path)
    P = C.POINTER
    D = P(C.c_double)
    lib.sg_setup.argtypes = [P(Grid), P(KL), P(PCE), P(Params), P(Source), C.c_void_p, P(C.c_void_p)]
    lib.sg_setup_mesh.argtypes = [P(Mesh), P(KL), P(PCE), P(Params), P(Source), C.c_void_p, P(C.c_void_p)]
    lib.sg_step.argtypes = [C.c_void_p, C.c_int, P(Stats)]
    lib.sg_solve_batch.argtypes = [P(C.c_void_p), C.c_int, C.c_int, P(Stats)]
    lib.sg_get_field.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int]
    lib.sg_get_moments.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    lib.sg_get_moments_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.sg_get_moments_noalloc.restype = C.c_int
    lib.sg_get_state.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    lib.sg_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    lib.sg_step_host.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, P(Stats)]
    lib.sg_get_sizes.argtypes = [C.c_void_p, P(Sizes)]
    lib.sg_plan_query.argtypes = [P(Grid), P(KL), P(PCE), P(Params), P(Plan)]
    lib.sg_mesh_plan_query.argtypes = [P(Mesh), P(KL), P(PCE), P(Params), P(MeshPlan)]
    lib.sg_partition_rcb.argtypes = [C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]
    lib.sg_partition_rcb.restype = C.c_int
    lib.sg_mesh_plan_query.restype = C.c_int
    lib.sg_plan_query.restype = C.c_int
    lib.sg_get_iters.argtypes = [C.c_void_p, P(C.c_int), D, C.c_int]
    lib.sg_destroy.argtypes = [C.c_void_p]
    lib.sg_set_enqueue_mode.argtypes = [C.c_void_p, C.c_int]
    lib.sg_set_enqueue_mode.restype = C.c_int
    lib.sg_kernel_timing.argtypes = [C.c_void_p, C.c_int, P(C.c_double), P(C.c_longlong)]
    lib.sg_kernel_timing.restype = C.c_int
    lib.sg_warm_weights.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    lib.sg_warm_weights.restype = C.c_int
    lib.sg_warm_status.argtypes = [C.c_void_p, P(C.c_int), P(C.c_int), P(C.c_float)]
    lib.sg_warm_status.restype = C.c_int
    lib.sg_mlp_eval.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, P(C.c_double)]
    lib.sg_mlp_eval.restype = C.c_int
    lib.sg_launch_count.argtypes = [C.c_void_p]
    lib.sg_launch_count.restype = C.c_longlong
    lib.sg_strerror.argtypes = [C.c_int]
    lib.sg_strerror.restype = C.c_char_p
    lib.sg_last_error.argtypes = [C.c_void_p]
    lib.sg_last_error.restype = C.c_char_p
    lib.sg_sample_field.restype = C.c_int
    for f in ("sg_setup", "sg_setup_mesh", "sg_step", "sg_solve_batch", "sg_get_field", "sg_get_moments", "sg_get_state",
              "sg_set_state", "sg_step_host", "sg_get_sizes", "sg_get_iters", "sg_destroy"):
        getattr(lib, f).restype = C.c_int
    _LIB = lib
    return lib


def _ptr(a) -> int:
    """Address of a contiguous numpy array or torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _on_device(a) -> int:
    return int(bool(getattr(a, "is_cuda", False)))


class Solver:
    """One SG-DD wave problem on the GPU (wraps an sg_handle)."""

    def __init__(self, prob, precision: int = SG_FP64, warm: int = SG_WARM_PREV, stream=None,
                 tol: Optional[float] = None, inner_tol: float = 0.0, inner_max_iter: int = 0,
                 max_iter: Optional[int] = None, autotune: bool = False, warm_train_steps: int = 0,
                 warm_lr: float = 0.0, kl_modes=None, kl_lambdas=None, precond: int = SG_PC_NN2,
                 mesh=None):
        """kl_modes / kl_lambdas: the caller's KL (M x 2 N^2 eigenfunction values at the element
        centroids in the library's element order, and M eigenvalues), or None for the analytic one.
        mesh: (xy (nv, 2), dirichlet (nv,), tri (ne, 3), part (ne,)) of a partitioned triangle mesh
        (sg_setup_mesh; prob.N and prob.s are then unused, kl_modes hold the triangle centroids)."""
        self.lib = load_library()
        self.prob = prob
        s = prob.source
        self._grid = Grid(prob.N, prob.s, prob.s)
        self._kl_arrays = None
        mp = lp = None
        if kl_modes is not None:
            m = np.ascontiguousarray(kl_modes, dtype=np.float64)
            lam = np.ascontiguousarray(kl_lambdas, dtype=np.float64) if kl_lambdas is not None else None
            self._kl_arrays = (m, lam)   # kept alive for the duration of sg_setup
            mp = m.ctypes.data
            lp = lam.ctypes.data if lam is not None else None
        self._kl = KL(prob.M, prob.sigma, prob.bx, prob.by, prob.g0, mp, lp)
        self._pce = PCE(prob.p, prob.p_in)
        self._prm = Params(prob.dt, prob.tol if tol is None else tol, prob.alpha0, prob.alpha1,
                           prob.max_iter if max_iter is None else max_iter, precision, warm, inner_tol,
                           inner_max_iter, int(bool(autotune)), warm_train_steps, warm_lr, precond)
        self._src = Source(s.kind, s.x0, s.y0, s.width, s.freq, s.amp)
        st = 0
        if stream is not None:
            st = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.stream = st
        h = C.c_void_p()
        if mesh is not None:
            xy, dirichlet, tri, part = mesh
            xy = np.ascontiguousarray(xy, dtype=np.float64)
            dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
            tri = np.ascontiguousarray(tri, dtype=np.int32)
            part = np.ascontiguousarray(part, dtype=np.int32)
            self._mesh_arrays = (xy, dirichlet, tri, part)   # kept alive for the duration of sg_setup_mesh
            self._mesh = Mesh(xy.shape[0], xy.ctypes.data, dirichlet.ctypes.data, tri.shape[0], tri.ctypes.data,
                              part.ctypes.data)
            rc = self.lib.sg_setup_mesh(C.byref(self._mesh), C.byref(self._kl), C.byref(self._pce),
                                        C.byref(self._prm), C.byref(self._src), C.c_void_p(st), C.byref(h))
        else:
            rc = self.lib.sg_setup(C.byref(self._grid), C.byref(self._kl), C.byref(self._pce), C.byref(self._prm),
                                   C.byref(self._src), C.c_void_p(st), C.byref(h))
        if rc != 0:
            raise SGError(rc, self.lib.sg_last_error(None).decode())
        self.h = h
        sz = Sizes()
        self._check(self.lib.sg_get_sizes(self.h, C.byref(sz)))
        self.sizes = {f: getattr(sz, f) for f, _ in Sizes._fields_}
        self.P = sz.P
        self.n_free = sz.n_free

    def _check(self, rc, allow_notconv=False):
        if rc == 0 or (allow_notconv and rc == SG_ENOTCONV):
            return rc
        raise SGError(rc, (self.lib.sg_strerror(rc) or b"").decode() + ": " +
                      (self.lib.sg_last_error(self.h) or b"").decode())

    def step(self, n: int = 1, allow_notconv: bool = False) -> dict:
        st = Stats()
        rc = self._check(self.lib.sg_step(self.h, n, C.byref(st)), allow_notconv)
        d = st.as_dict()
        d["rc"] = rc
        return d

    def iters(self, cap: int = 1 << 20):
        it = (C.c_int * cap)()
        rr = (C.c_double * cap)()
        n = self.lib.sg_get_iters(self.h, it, rr, cap)
        return list(it[:n]), list(rr[:n])

    def field(self, mode: int = -1, out=None):
        """Displacement PCE coefficients U_n: (n_free, P) for mode = -1, else (n_free,).
        `out` may be a float64 numpy array or a CUDA torch tensor."""
        shape = (self.n_free, self.P) if mode < 0 else (self.n_free,)
        if out is None:
            out = np.zeros(shape)
        self._check(self.lib.sg_get_field(self.h, mode, C.c_void_p(_ptr(out)), _on_device(out)))
        return out

    def moments(self):
        mean = np.zeros(self.n_free)
        var = np.zeros(self.n_free)
        self._check(self.lib.sg_get_moments(self.h, C.c_void_p(_ptr(mean)), C.c_void_p(_ptr(var)), 0))
        return mean, var

    def sample(self, xi, nodes):
        """Surrogate samples u(x_j, xi_s) = sum_k U_k(x_j) Psi_k(xi_s): xi (nsamp, M), nodes (npts,) free-node
        indices; numpy in, numpy out (host path), or CUDA torch tensors in and out (device path)."""
        on_dev = _on_device(xi)
        if on_dev:
            import torch
            out = torch.empty((xi.shape[0], nodes.shape[0]), dtype=torch.float64, device=xi.device)
        else:
            xi = np.ascontiguousarray(xi, dtype=np.float64)
            nodes = np.ascontiguousarray(nodes, dtype=np.int32)
            out = np.zeros((xi.shape[0], nodes.shape[0]))
        self._check(self.lib.sg_sample_field(self.h, int(xi.shape[0]), C.c_void_p(_ptr(xi)), int(nodes.shape[0]),
                                             C.c_void_p(_ptr(nodes)), C.c_void_p(_ptr(out)), on_dev))
        return out

    def get_state(self, out=None):
        if out is None:
            out = np.zeros(3 * self.n_free * self.P + 1)
        self._check(self.lib.sg_get_state(self.h, C.c_void_p(_ptr(out)), _on_device(out)))
        return out

    def set_state(self, state):
        self._check(self.lib.sg_set_state(self.h, C.c_void_p(_ptr(state)), _on_device(state)))

    def step_host(self, n: int, f_host=None, u_host=None) -> dict:
        st = Stats()
        fp = C.c_void_p(_ptr(f_host)) if f_host is not None else None
        up = C.c_void_p(_ptr(u_host)) if u_host is not None else None
        self._check(self.lib.sg_step_host(self.h, n, fp, up, C.byref(st)))
        return st.as_dict()

    def set_eager(self, eager: bool):
        """Host-driven enqueue (True) or one CUDA graph per step (False, default)."""
        self._check(self.lib.sg_set_enqueue_mode(self.h, int(bool(eager))))

    def kernel_timing(self, which: int):
        """Return (ms, launches) accumulated for the previously selected kernel class and
        select `which` (0 none, 1 preconditioner step, 2 fused apply, 3 tensor-core product, 4 applies
        with FP64 inputs and outputs) for the
        following eager steps."""
        ms = C.c_double()
        n = C.c_longlong()
        self._check(self.lib.sg_kernel_timing(self.h, which, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def warm_weights(self, new=None):
        """FP32 master weights of the warm-start network (copy); `new` replaces them."""
        out = np.zeros(1249, dtype=np.float32)
        setp = None
        if new is not None:
            new = np.ascontiguousarray(new, dtype=np.float32)
            setp = C.c_void_p(new.ctypes.data)
        self._check(self.lib.sg_warm_weights(self.h, C.c_void_p(out.ctypes.data), setp, 1249))
        return out

    def warm_status(self):
        a, b, l = C.c_int(), C.c_int(), C.c_float()
        self._check(self.lib.sg_warm_status(self.h, C.byref(a), C.byref(b), C.byref(l)))
        return {"trained": a.value, "train_left": b.value, "loss": l.value}

    def launch_count(self) -> int:
        """Kernels launched by the library so far in this process (device-side count)."""
        return int(self.lib.sg_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.sg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def plan_query(prob, precision: int = SG_FP64) -> dict:
    """Launch plan of the per-step kernels for `prob` (host-only; no GPU needed), as a dict of the
    sg_plan fields; two-element lists are [FP64 kernels, FP32 kernels]."""
    lib = load_library()
    grid, kl, pce = Grid(prob.N, prob.s, prob.s), KL(prob.M, prob.sigma, prob.bx, prob.by, prob.g0), PCE(prob.p, prob.p_in)
    prm = Params(prob.dt, prob.tol, prob.alpha0, prob.alpha1, prob.max_iter, precision, SG_WARM_PREV, 0.0, 0, 0, 0, 0.0)
    out = Plan()
    rc = lib.sg_plan_query(C.byref(grid), C.byref(kl), C.byref(pce), C.byref(prm), C.byref(out))
    if rc != 0:
        raise SGError(rc, lib.sg_last_error(None).decode())
    return {f: _plain(getattr(out, f)) for f, _ in Plan._fields_}


def partition_rcb(xy, tri, nparts: int) -> np.ndarray:
    """Triangle -> subdomain ids by the library's recursive coordinate bisection (host only)."""
    lib = load_library()
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    part = np.zeros(tri.shape[0], dtype=np.int32)
    rc = lib.sg_partition_rcb(xy.shape[0], xy.ctypes.data, tri.shape[0], tri.ctypes.data, int(nparts), part.ctypes.data)
    if rc != 0:
        raise SGError(rc, lib.sg_last_error(None).decode())
    return part


def mesh_plan_query(prob, mesh, precision: int = SG_FP64, precond: int = SG_PC_NN2) -> dict:
    """Sizes and device-memory needs of `prob` on mesh = (xy, dirichlet, tri, part) (host-only; no GPU
    needed), as a dict of the sg_mesh_plan fields."""
    lib = load_library()
    xy, dirichlet, tri, part = mesh
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    part = np.ascontiguousarray(part, dtype=np.int32)
    m = Mesh(xy.shape[0], xy.ctypes.data, dirichlet.ctypes.data, tri.shape[0], tri.ctypes.data, part.ctypes.data)
    kl, pce = KL(prob.M, prob.sigma, prob.bx, prob.by, prob.g0), PCE(prob.p, prob.p_in)
    prm = Params(prob.dt, prob.tol, prob.alpha0, prob.alpha1, prob.max_iter, precision, SG_WARM_PREV, 0.0, 0, 0, 0, 0.0,
                 precond)
    out = MeshPlan()
    rc = lib.sg_mesh_plan_query(C.byref(m), C.byref(kl), C.byref(pce), C.byref(prm), C.byref(out))
    if rc != 0:
        raise SGError(rc, lib.sg_last_error(None).decode())
    return {f: getattr(out, f) for f, _ in MeshPlan._fields_}


def solve_batch(solvers: Sequence[Solver], nsteps: int):
    lib = load_library()
    n = len(solvers)
    hs = (C.c_void_p * n)(*[s.h for s in solvers])
    st = (Stats * n)()
    rc = lib.sg_solve_batch(hs, n, nsteps, st)
    if rc not in (0, SG_ENOTCONV):
        raise SGError(rc, (lib.sg_strerror(rc) or b"").decode())
    return [s.as_dict() for s in st]
