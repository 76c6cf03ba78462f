"""Thin ctypes binding of libviv.so (the C ABI declared in include/viv.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  PyTorch supplies device memory (through the caching allocator)
and the CUDA stream.  There is no fallback: if the library cannot be loaded,
importing the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libviv.so")

VIV_FP64, VIV_MIXED = 0, 1
VIV_RES, VIV_JAC = 1, 2
VIV_PIVOT_THRESHOLD, VIV_PIVOT_WINDOW = 0, 1
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_PIVOT", 5: "ERR_NEWTON",
          6: "ERR_NONFINITE", 7: "ERR_TIMEOUT", 8: "ERR_ADMISSION", 9: "ERR_STATE"}
KINDS = ("residual", "jacobian", "face_border", "front_assemble", "panel_lu", "trsm", "schur_gemm",
         "fwd_solve", "bwd_solve", "spmv", "vector", "tc_schur_gemm", "tc_split")
KINDS_N = len(KINDS)
FIELD = {0: "ux", 1: "uy", 2: "xx", 3: "xy", 4: "p", 5: "lx", 6: "ly", 7: "dx", 8: "dy",
         9: "uz", 10: "xz", 11: "lz"}


class VivError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_elems", C.c_int64), ("n_gamma_faces", C.c_int64),
                ("X", C.c_void_p), ("conn", C.c_void_p), ("tags", C.c_void_p),
                ("gamma_faces", C.c_void_p), ("leaf_elems", C.c_int32), ("dim", C.c_int32),
                ("span", C.c_double), ("wrap", C.c_void_p), ("elem_type", C.c_int32)]


class MeshInfo(C.Structure):
    _fields_ = [("n_dofs", C.c_int64), ("nnz", C.c_int64), ("n_fronts", C.c_int64),
                ("max_front", C.c_int64), ("n_levels", C.c_int64), ("factor_flops", C.c_double),
                ("front_entries", C.c_size_t), ("device_bytes_fp64", C.c_size_t),
                ("device_bytes_mixed", C.c_size_t), ("n_colors", C.c_int32),
                ("gemm_flops", C.c_double), ("panel_flops", C.c_double), ("trsm_flops", C.c_double),
                ("outer_flops", C.c_double), ("tc_split_chunks", C.c_int64), ("tc_tiles", C.c_int64),
                ("tc_image_bytes", C.c_size_t), ("window_tc_flops", C.c_double),
                ("window_lu_flops", C.c_double), ("window_gemm_flops", C.c_double),
                ("block_level_mask", C.c_int64), ("dim", C.c_int32),
                ("elem_type", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double), ("k", C.c_double), ("dt", C.c_double),
                ("lame_scale", C.c_double), ("newton_tol", C.c_double), ("max_newton", C.c_int32),
                ("precision", C.c_int32), ("refine_tol", C.c_double), ("refine_max", C.c_int32),
                ("pivot_threshold", C.c_double), ("source", C.c_int32), ("source_amp", C.c_double),
                ("pivoting", C.c_int32), ("jacobian_fp32", C.c_int32), ("predictor", C.c_int32),
                ("Re", C.c_double), ("Ustar", C.c_double), ("U_inf", C.c_double), ("D", C.c_double),
                ("span_L", C.c_double), ("cfl_target", C.c_double), ("dt_max", C.c_double),
                ("lame_constant", C.c_int32), ("factor_reuse", C.c_int32)]


class StepInfo(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("refine_sweeps", C.c_int32),
                ("perturbed_pivots", C.c_int32), ("threshold_misses", C.c_int32),
                ("res_norm0", C.c_double), ("res_norm", C.c_double), ("t", C.c_double),
                ("delta", C.c_double * 2), ("force", C.c_double * 2), ("dt", C.c_double), ("cfl", C.c_double),
                ("reused_factor_solves", C.c_int32)]

    def as_dict(self):
        return dict(newton_iters=self.newton_iters, refine_sweeps=self.refine_sweeps,
                    perturbed_pivots=self.perturbed_pivots, threshold_misses=self.threshold_misses,
                    res_norm0=self.res_norm0, res_norm=self.res_norm, t=self.t,
                    delta=list(self.delta), force=list(self.force), dt=self.dt, cfl=self.cfl,
                    reused_factor_solves=self.reused_factor_solves)


class ForceStats(C.Structure):
    _fields_ = [("cd_mean", C.c_double), ("cd_amp", C.c_double), ("cl_mean", C.c_double), ("cl_amp", C.c_double),
                ("cl_rms", C.c_double), ("frequency", C.c_double), ("strouhal", C.c_double),
                ("samples", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("params", Params), ("u0", C.c_void_p), ("n_steps", C.c_int32),
                ("arrival_time", C.c_double)]


class Result(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int), ("steps_done", C.c_int32), ("newton_total", C.c_int32),
                ("t", C.c_double), ("delta", C.c_double * 2), ("force", C.c_double * 2),
                ("submit_s", C.c_double), ("admit_s", C.c_double), ("finish_s", C.c_double),
                ("step_ms_mean", C.c_double), ("step_ms_max", C.c_double), ("message", C.c_char * 160)]

    def as_dict(self):
        return dict(id=self.id, status=STATUS.get(self.status, self.status), steps_done=self.steps_done,
                    newton_total=self.newton_total, t=self.t, delta=list(self.delta), force=list(self.force),
                    submit_s=self.submit_s, admit_s=self.admit_s, finish_s=self.finish_s,
                    step_ms_mean=self.step_ms_mean, step_ms_max=self.step_ms_max,
                    message=self.message.decode(errors="replace"))


class ServerStats(C.Structure):
    _fields_ = [("step_ms_p50", C.c_double), ("step_ms_p99", C.c_double), ("steps", C.c_int64),
                ("cases_done", C.c_int64), ("elapsed_s", C.c_double), ("peak_active", C.c_int32),
                ("active", C.c_int32), ("pending", C.c_int32), ("peak_bytes", C.c_size_t),
                ("steady_ms_p50", C.c_double), ("steady_ms_p99", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


# every symbol declared in include/viv.h, with its ctypes signature
_P = C.c_void_p
SIGNATURES = {
    "viv_mesh_create": (C.c_int, [C.POINTER(MeshDesc), C.c_void_p, C.c_void_p, C.POINTER(_P)]),
    "viv_mesh_analyze": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(_P)]),
    "viv_mesh_info": (C.c_int, [_P, C.POINTER(MeshInfo)]),
    "viv_mesh_dof_labels": (C.c_int, [_P, _P, _P]),
    "viv_mesh_pattern": (C.c_int, [_P, _P, _P]),
    "viv_mesh_fronts": (C.c_int, [_P, _P, _P, _P, _P]),
    "viv_mesh_element_slots": (C.c_int, [_P, _P, _P, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "viv_mesh_destroy": (C.c_int, [_P]),
    "viv_case_create": (C.c_int, [_P, C.POINTER(Params), _P, _P, C.POINTER(_P)]),
    "viv_case_destroy": (C.c_int, [_P]),
    "viv_case_params": (C.c_int, [_P, C.POINTER(Params)]),
    "viv_case_save": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    "viv_case_load": (C.c_int, [_P, _P, C.c_size_t]),
    "viv_set_state": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, C.c_double]),
    "viv_set_history": (C.c_int, [_P, C.c_int, _P, _P]),
    "viv_get_state": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, C.POINTER(C.c_double)]),
    "viv_begin_step": (C.c_int, [_P]),
    "viv_assemble": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double)]),
    "viv_get_residual": (C.c_int, [_P, _P]),
    "viv_get_jacobian": (C.c_int, [_P, _P]),
    "viv_factor": (C.c_int, [_P]),
    "viv_border_block": (C.c_int, [_P, _P]),
    "viv_solve": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "viv_solve_rhs": (C.c_int, [_P, C.c_int, _P, _P, C.POINTER(C.c_int)]),
    "viv_update": (C.c_int, [_P]),
    "viv_lu_solve_noalloc": (C.c_int, [_P, _P, _P]),
    "viv_tc_schur_update": (C.c_int, [_P, C.c_int, _P, C.c_int, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P, _P]),
    "viv_step": (C.c_int, [_P, C.POINTER(StepInfo)]),
    "viv_step_host": (C.c_int, [_P, _P, _P, C.POINTER(StepInfo)]),
    "viv_state_size": (C.c_int64, [_P]),
    "viv_case_graphs": (C.c_int, [_P, C.c_int]),
    "viv_autotune": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    "viv_server_create": (C.c_int, [C.c_size_t, C.c_int32, C.POINTER(_P)]),
    "viv_server_submit": (C.c_int, [_P, C.POINTER(Request), C.POINTER(C.c_int64)]),
    "viv_server_poll": (C.c_int, [_P, _P, C.c_int32, C.POINTER(C.c_int32), C.c_int32]),
    "viv_server_state": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P]),
    "viv_server_stats": (C.c_int, [_P, C.POINTER(ServerStats)]),
    "viv_server_destroy": (C.c_int, [_P]),
    "viv_kernel_launches": (C.c_int64, []),
    "viv_force_analysis": (C.c_int, [_P, _P, _P, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double,
                                     C.POINTER(ForceStats)]),
    "viv_profile": (C.c_int, [_P, C.c_int]),
    "viv_profile_read": (C.c_int, [_P, _P, _P]),
    "viv_profile_levels": (C.c_int, [_P, _P, C.c_int32, _P]),
    "viv_set_big_front": (C.c_int, [_P, C.c_int32]),
    "viv_set_block_levels": (C.c_int, [_P, C.c_int64]),
    "viv_last_error": (C.c_char_p, []),
    "viv_version": (C.c_char_p, []),
}

_lib = None


def load(path=LIB_PATH):
    """Load libviv.so and attach signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libviv.so not built ({path}); run paper_2609_31477_b300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise VivError(status, _lib.viv_last_error().decode())


def _ptr(a):
    return C.c_void_p(a.ctypes.data) if a is not None else None


def _dev_ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class _TorchAllocator:
    """Routes library allocations to torch's CUDA caching allocator."""

    def __init__(self, device, stream):
        import torch
        self.torch = torch
        self.device = device
        self.stream = stream
        self._alloc = ALLOC_FN(self.alloc)
        self._free = FREE_FN(self.free)
        self.struct = Allocator(self._alloc, self._free, None)

    def alloc(self, n, ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(n), self.device, self.stream)
        except Exception:
            return None

    def free(self, p, ctx):
        self.torch.cuda.caching_allocator_delete(p)


def _desc(mesh):
    X = np.ascontiguousarray(mesh["X"], dtype=np.float64)
    conn = np.ascontiguousarray(mesh["conn"], dtype=np.int64)
    tags = np.ascontiguousarray(mesh["tags"], dtype=np.int32)
    gf = np.ascontiguousarray(mesh["gamma_faces"], dtype=np.int64).reshape(-1, 2)
    dim = int(X.shape[1])
    wrap = np.ascontiguousarray(mesh.get("wrap", np.zeros(len(conn), np.int64)), dtype=np.int64)
    keep = (X, conn, tags, gf, wrap)
    d = MeshDesc(len(X), len(conn), len(gf), _ptr(X).value, _ptr(conn).value, _ptr(tags).value,
                 _ptr(gf).value if len(gf) else None, int(mesh.get("leaf_elems", 0)), dim,
                 float(mesh.get("span", 0.0)), _ptr(wrap).value if dim == 3 else None,
                 1 if mesh.get("elem") == "tri6" else 0)
    return d, keep


class Mesh:
    """Mesh analysed by the library: numbering, CSR pattern, e2nz, nested
    dissection, symbolic factorisation.  device=False analyses on the host
    only (no GPU needed).

    `mesh` is a dict: X (n, 2) or (n, 3) reference coordinates (the dimension
    follows), conn (E, 9) Q2 quads, (E, 27) Q2 hexahedra or (E, 6) P2-P1
    triangles with elem="tri6", tags (n,) VIV_TAG bit sets, gamma_faces (F, 2)
    (element, local edge or face); 3-D meshes periodic in z add span and wrap
    (per element, the bit mask of local nodes at X + span e_z), and
    leaf_elems optionally sets the dissection's leaf size.  The generators of
    paper_2609_31477_b300.inputs return such dicts."""

    def __init__(self, mesh, device=True, torch_alloc=True, stream=None):
        lib = load()
        self.mesh = mesh
        d, keep = _desc(mesh)
        h = C.c_void_p()
        self._alloc = None
        if device:
            import torch
            dev = torch.cuda.current_device()
            st = stream if stream is not None else torch.cuda.current_stream()
            self.stream = st
            if torch_alloc:
                self._alloc = _TorchAllocator(dev, st.cuda_stream)
            _check(lib.viv_mesh_create(C.byref(d), C.byref(self._alloc.struct) if self._alloc else None,
                                       C.c_void_p(st.cuda_stream), C.byref(h)))
        else:
            self.stream = None
            _check(lib.viv_mesh_analyze(C.byref(d), C.byref(h)))
        self.h = h
        self.refresh_info()
        self.n_dofs = self.info["n_dofs"]
        self.n_nodes = len(mesh["X"])
        self.dim = int(self.info["dim"])

    def dof_labels(self):
        node = np.empty(self.n_dofs, np.int64)
        field = np.empty(self.n_dofs, np.int32)
        _check(_lib.viv_mesh_dof_labels(self.h, _ptr(node), _ptr(field)))
        return node, field

    def pattern(self):
        rp = np.empty(self.n_dofs + 1, np.int64)
        _check(_lib.viv_mesh_pattern(self.h, _ptr(rp), None))
        col = np.empty(rp[-1], np.int32)
        _check(_lib.viv_mesh_pattern(self.h, _ptr(rp), _ptr(col)))
        return rp, col

    def refresh_info(self):
        """Re-read viv_mesh_info (the schedule counters change with the large-front
        threshold and the autotuner's per-level choice)."""
        info = MeshInfo()
        _check(_lib.viv_mesh_info(self.h, C.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in MeshInfo._fields_}
        return self.info

    def fronts(self):
        n = int(self.info["n_fronts"])
        a = [np.empty(n, np.int32) for _ in range(4)]
        _check(_lib.viv_mesh_fronts(self.h, *[_ptr(x) for x in a]))
        return dict(m=a[0], p=a[1], level=a[2], parent=a[3])

    def element_slots(self):
        """CSR value index of every structural pair of every element (E, pairs)
        and Gamma edge/face (F, pairs) - viv_mesh_element_slots."""
        ne, nf = C.c_int32(), C.c_int32()
        _check(_lib.viv_mesh_element_slots(self.h, None, None, C.byref(ne), C.byref(nf)))
        E, F = len(self.mesh["conn"]), len(np.asarray(self.mesh["gamma_faces"]).reshape(-1, 2))
        es = np.empty((E, ne.value), np.int32)
        fs = np.empty((F, nf.value), np.int32)
        _check(_lib.viv_mesh_element_slots(self.h, _ptr(es), _ptr(fs), C.byref(ne), C.byref(nf)))
        return es, fs

    def state_size(self):
        return int(_lib.viv_state_size(self.h))

    def close(self):
        if self.h:
            _lib.viv_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Case:
    """Device state of one cylinder case and its Newton/BDF driver."""

    def __init__(self, mesh: Mesh, u0, rho, mu, k, dt, precision=VIV_FP64, lame_scale=1.0,
                 newton_tol=1e-10, max_newton=25, refine_tol=0.0, refine_max=0, pivot_threshold=0.01,
                 stream=None, source=0, source_amp=0.0, pivoting=0, jacobian_fp32=0, predictor=0,
                 Re=0.0, Ustar=0.0, U_inf=0.0, D=0.0, span_L=0.0, cfl_target=0.0, dt_max=0.0, lame_constant=0,
                 factor_reuse=0):
        lib = load()
        self.mesh = mesh
        self.params = Params(rho, mu, k, dt, lame_scale, newton_tol, max_newton, precision, refine_tol,
                             refine_max, pivot_threshold, source, source_amp, pivoting, jacobian_fp32,
                             predictor, Re, Ustar, U_inf, D, span_L, cfl_target, dt_max, lame_constant,
                             factor_reuse)
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        import torch
        # each case owns a non-default stream (graphs cannot capture the legacy stream)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        torch.cuda.current_stream().synchronize()
        h = C.c_void_p()
        _check(lib.viv_case_create(mesh.h, C.byref(self.params), _ptr(u0),
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h
        self.n = mesh.n_nodes
        self.dim = mesh.dim

    # state ---------------------------------------------------------------------
    def resolved_params(self):
        """The parameters as the library runs them (mu and k after Re / U*)."""
        p = Params()
        _check(_lib.viv_case_params(self.h, C.byref(p)))
        return {f: getattr(p, f) for f, _ in Params._fields_}

    def save(self):
        """Checkpoint of the case between steps (bytes)."""
        n = C.c_size_t()
        _check(_lib.viv_case_save(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(_lib.viv_case_save(self.h, buf, C.byref(n)))
        return buf.raw[:n.value]

    def load(self, data: bytes):
        buf = C.create_string_buffer(data, len(data))
        _check(_lib.viv_case_load(self.h, buf, len(data)))

    def set_state(self, u=None, p=None, x=None, lam=None, delta=None, t=0.0):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (u, p, x, lam, delta)]
        _check(_lib.viv_set_state(self.h, 0, *[_ptr(a) for a in arrs], C.c_double(t)))

    def set_history(self, u_prev, x_prev):
        a = np.ascontiguousarray(u_prev, dtype=np.float64)
        b = np.ascontiguousarray(x_prev, dtype=np.float64)
        _check(_lib.viv_set_history(self.h, 0, _ptr(a), _ptr(b)))

    def get_state(self):
        n, D = self.n, self.dim
        u, p, x, lam, d = (np.empty((n, D)), np.empty(n), np.empty((n, D)), np.empty((n, D)), np.empty(2))
        t = C.c_double()
        _check(_lib.viv_get_state(self.h, 0, _ptr(u), _ptr(p), _ptr(x), _ptr(lam), _ptr(d), C.byref(t)))
        return dict(u=u, p=p, x=x, lam=lam, delta=d, t=t.value)

    # steps of the method -------------------------------------------------------
    def begin_step(self):
        _check(_lib.viv_begin_step(self.h))

    def assemble(self, what=VIV_RES | VIV_JAC):
        nr = C.c_double()
        _check(_lib.viv_assemble(self.h, what, C.byref(nr) if what & VIV_RES else None))
        return nr.value

    def residual(self):
        r = np.empty(self.mesh.n_dofs)
        _check(_lib.viv_get_residual(self.h, _ptr(r)))
        return r

    def jacobian_values(self):
        v = np.empty(self.mesh.info["nnz"])
        _check(_lib.viv_get_jacobian(self.h, _ptr(v)))
        return v

    def factor(self):
        _check(_lib.viv_factor(self.h))

    def border_block(self):
        """FP64 border Schur block S_b = D - C A^{-1} B of the last factorisation (2 x 2)."""
        S = np.empty(4)
        _check(_lib.viv_border_block(self.h, _ptr(S)))
        return S.reshape(2, 2)

    def solve(self):
        sw = C.c_int()
        _check(_lib.viv_solve(self.h, C.byref(sw)))
        return sw.value

    def solve_rhs(self, b):
        b = np.ascontiguousarray(b, dtype=np.float64)
        y = np.empty_like(b)
        sw = C.c_int()
        _check(_lib.viv_solve_rhs(self.h, 0, _ptr(b), _ptr(y), C.byref(sw)))
        return y, sw.value

    def update(self):
        _check(_lib.viv_update(self.h))

    def lu_solve_noalloc(self, b_dev, x_dev):
        """One unrefined forward/backward solve into caller-owned device
        tensors, using the library's fixed workspace (no allocation)."""
        _check(_lib.viv_lu_solve_noalloc(self.h, _dev_ptr(b_dev), _dev_ptr(x_dev)))

    def step(self):
        info = StepInfo()
        _check(_lib.viv_step(self.h, C.byref(info)))
        return info.as_dict()

    def step_host(self, state_in, state_out):
        info = StepInfo()
        _check(_lib.viv_step_host(self.h, _ptr(state_in), _ptr(state_out), C.byref(info)))
        return info.as_dict()

    def graphs(self, on=True):
        _check(_lib.viv_case_graphs(self.h, int(on)))

    def autotune(self):
        bf, ms = C.c_int32(), C.c_double()
        _check(_lib.viv_autotune(self.h, C.byref(bf), C.byref(ms)))
        return bf.value, ms.value

    def set_big_front(self, big_front):
        _check(_lib.viv_set_big_front(self.h, int(big_front)))

    def set_block_levels(self, mask):
        _check(_lib.viv_set_block_levels(self.h, int(mask)))

    def profile(self, on=True):
        _check(_lib.viv_profile(self.h, int(on)))

    def profile_read(self):
        ms = np.zeros(KINDS_N)
        cnt = np.zeros(KINDS_N, np.int64)
        _check(_lib.viv_profile_read(self.h, _ptr(ms), _ptr(cnt)))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KINDS)}

    def profile_levels(self):
        """Factorisation time (ms) per elimination-tree level and kernel kind at the
        last profile_read: a list (one entry per level) of {kind: ms}."""
        n = C.c_int32()
        ms = np.zeros(256 * KINDS_N)
        _check(_lib.viv_profile_levels(self.h, _ptr(ms), 256, C.byref(n)))
        ms = ms[:n.value * KINDS_N].reshape(n.value, KINDS_N)
        return [{k: float(row[i]) for i, k in enumerate(KINDS) if row[i] > 0} for row in ms]

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if self.h:
            _lib.viv_case_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop of the library (viv_server_*): continuous admission of
    cases by predicted device memory, concurrent cases on their own streams."""

    def __init__(self, mem_budget_bytes, max_active=8):
        lib = load()
        h = C.c_void_p()
        _check(lib.viv_server_create(int(mem_budget_bytes), int(max_active), C.byref(h)))
        self.h = h
        self._keep = []

    def submit(self, mesh: Mesh, u0, Re, Ustar, dt, n_steps, arrival_time=0.0, precision=VIV_MIXED,
               U_inf=1.0, D=1.0, rho=1.0, newton_tol=1e-10, max_newton=25, pivoting=VIV_PIVOT_THRESHOLD,
               jacobian_fp32=0, predictor=0):
        # mu and k are derived from Re and U* by the library (vivParams)
        prm = Params(rho, 0.0, 0.0, dt, 1.0, newton_tol, max_newton, precision, 0.0, 0,
                     0.01, 0, 0.0, pivoting, jacobian_fp32, predictor, Re, Ustar, U_inf, D, 0.0, 0.0, 0.0, 0)
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        req = Request(mesh.h.value, prm, u0.ctypes.data, int(n_steps), float(arrival_time))
        rid = C.c_int64()
        _check(_lib.viv_server_submit(self.h, C.byref(req), C.byref(rid)))
        return rid.value

    def poll(self, max_results=64, wait_ms=0):
        buf = (Result * max_results)()
        n = C.c_int32()
        _check(_lib.viv_server_poll(self.h, buf, max_results, C.byref(n), int(wait_ms)))
        return [buf[i].as_dict() for i in range(n.value)]

    def state(self, rid, n_nodes, dim=2):
        u, p, x, lam, d = (np.empty((n_nodes, dim)), np.empty(n_nodes), np.empty((n_nodes, dim)),
                           np.empty((n_nodes, dim)), np.empty(2))
        _check(_lib.viv_server_state(self.h, rid, _ptr(u), _ptr(p), _ptr(x), _ptr(lam), _ptr(d)))
        return dict(u=u, p=p, x=x, lam=lam, delta=d)

    def stats(self):
        st = ServerStats()
        _check(_lib.viv_server_stats(self.h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def wait_all(self, count, timeout_s=600.0):
        import time
        out, t0 = [], time.time()
        while len(out) < count and time.time() - t0 < timeout_s:
            out += self.poll(64, 200)
        return out

    def close(self):
        if self.h:
            _lib.viv_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tc_schur_update(a, b, c, err, stream=None):
    """c -= a @ b with the tcgen05 3xTF32 kernel; a, b, c are column-major
    FP32 CUDA tensors (stride(0) == 1), err a device int32 flag."""
    import torch
    M, K = a.shape
    N = b.shape[1]
    st = stream if stream is not None else torch.cuda.current_stream()
    ld = lambda t: t.stride(1) if t.shape[1] > 1 else max(1, t.shape[0])   # any ld >= rows for one column
    _check(load().viv_tc_schur_update(_dev_ptr(a), ld(a), _dev_ptr(b), ld(b), _dev_ptr(c), ld(c), M, N, K,
                                      _dev_ptr(err), C.c_void_p(st.cuda_stream)))


def force_analysis(t, F, rho=1.0, U=1.0, D=1.0, t_start=0.0):
    """Drag / lift coefficients and Strouhal number of a force history
    (t: n times, F: n x 2 fluid forces) - viv_force_analysis."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    fx, fy = np.ascontiguousarray(F[:, 0]), np.ascontiguousarray(F[:, 1])
    st = ForceStats()
    _check(load().viv_force_analysis(_ptr(t), _ptr(fx), _ptr(fy), len(t), rho, U, D, t_start, C.byref(st)))
    return {f: getattr(st, f) for f, _ in ForceStats._fields_}


def kernel_launches():
    return int(load().viv_kernel_launches())


def viv_case(mesh_obj, Re, Ustar, dt, u0, precision=VIV_FP64, U_inf=1.0, D=1.0, rho=1.0, **kw):
    """A cylinder case given by Reynolds number and reduced velocity; the
    library derives mu and the spring stiffness from them (vivParams)."""
    return Case(mesh_obj, u0, rho, 0.0, 0.0, dt, precision=precision, Re=Re, Ustar=Ustar, U_inf=U_inf, D=D, **kw)
