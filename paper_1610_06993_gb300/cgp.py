"""Thin ctypes binding of ``libcgp.so`` (the C ABI declared in ``include/cgp.h``).

Every function here only marshals arguments: torch tensors become device pointers, numpy arrays
become host pointers, and the CUDA library does all the work. There is no CPU fallback: if the
library has not been built, importing the functions raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcgp.so")

CGP_OK = 0
CGP_ERR_ARG = 1
CGP_ERR_MESH = 2
CGP_ERR_CUDA = 3
CGP_ERR_NOT_CONVERGED = 4
CGP_ERR_NAN = 5
CGP_ERR_TIMEOUT = 6
CGP_ERR_NOMEM = 7
CGP_ERR_STATE = 8
CGP_FP64 = 0
CGP_MIXED = 1
CGP_BC_U = 1
CGP_BC_V = 2


class cgp_params(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double), ("dt", C.c_double), ("levels", C.c_int),
                ("precision", C.c_int), ("rtol", C.c_double), ("inner_rtol", C.c_double),
                ("max_iter", C.c_int), ("max_outer", C.c_int), ("spmv_lanes", C.c_int),
                ("block_threads", C.c_int), ("coarse_solver", C.c_int), ("spmv_format", C.c_int),
                ("precond_degree", C.c_int), ("precond_ratio", C.c_double), ("warm_start", C.c_int),
                ("mass_degree", C.c_int), ("momentum_degree", C.c_int), ("solver_format", C.c_int),
                ("restrict_mode", C.c_int), ("projection", C.c_int), ("fine_order", C.c_int),
                ("momentum_rtol", C.c_double)]


class cgp_mesh_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("n_tris", C.c_int), ("xy_host", C.POINTER(C.c_double)),
                ("tri_host", C.POINTER(C.c_int))]


class cgp_info(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("n_fine", "n_coarse", "tris_fine", "tris_coarse", "nnz_fine",
                                       "nnz_coarse", "levels", "n_colours", "grid_blocks",
                                       "block_threads", "spmv_lanes", "coarse_kernel", "solver_format",
                                       "fine_order")]


class cgp_stats(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("momentum_iters", "momentum_outer", "momentum_status",
                                       "poisson_iters", "poisson_outer", "poisson_status", "mass_iters",
                                       "mass_status", "barrier_status")] + \
               [(k, C.c_double) for k in ("momentum_rel_res", "poisson_rel_res", "mass_rel_res")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_VP = C.c_void_p
_SIGNATURES = {
    "cgp_default_params": (None, [C.POINTER(cgp_params)]),
    "cgp_mesh_create": (C.c_int, [C.POINTER(cgp_mesh_desc), C.POINTER(cgp_params), C.POINTER(_VP)]),
    "cgp_refine": (C.c_int, [C.POINTER(cgp_mesh_desc), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                             _VP, _VP, _VP, _VP]),
    "cgp_refine_order": (C.c_int, [C.POINTER(cgp_mesh_desc), C.c_int, _VP]),
    "cgp_mesh_info": (C.c_int, [_VP, C.POINTER(cgp_info)]),
    "cgp_fine_mesh": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_set_bc": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_set_dirichlet_values": (C.c_int, [_VP, _VP, _VP]),
    "cgp_assemble": (C.c_int, [_VP, _VP, _VP]),
    "cgp_momentum_solve": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_restrict": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_poisson_solve": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_prolong_correct": (C.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "cgp_step": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_assemble_incremental": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_poisson_solve_many": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP]),
    "cgp_pressure_update": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "cgp_step_host": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_get_stats": (C.c_int, [_VP, _VP, C.POINTER(cgp_stats)]),
    "cgp_autotune": (C.c_int, [_VP, _VP]),
    "cgp_cg_solve_noalloc": (C.c_int, [C.c_int, _VP, _VP, _VP, _VP, _VP, C.c_double, C.c_int, _VP, _VP, _VP,
                                       _VP]),
    "cgp_wait_probe": (C.c_int, [_VP, C.c_int, C.c_double, _VP, _VP]),
    "cgp_set_surface": (C.c_int, [_VP, C.c_int, _VP, C.POINTER(C.c_int)]),
    "cgp_body_force": (C.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "cgp_reattachment": (C.c_int, [_VP, _VP, C.c_double, _VP, _VP, _VP, _VP]),
    "cgp_batch_create": (C.c_int, [_VP, C.c_int, _VP, _VP, C.POINTER(_VP)]),
    "cgp_batch_info": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_batch_step": (C.c_int, [_VP, _VP]),
    "cgp_batch_run": (C.c_int, [_VP, C.c_int, _VP]),
    "cgp_batch_get_stats": (C.c_int, [_VP, _VP, _VP]),
    "cgp_batch_poisson_solve": (C.c_int, [_VP, _VP]),
    "cgp_batch_destroy": (C.c_int, [_VP]),
    "cgp_copy_coarse_rhs": (C.c_int, [_VP, _VP, _VP]),
    "cgp_predict_pressure": (C.c_int, [_VP, _VP, _VP]),
    "cgp_spmv": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_fine_order": (C.c_int, [_VP, _VP]),
    "cgp_solver_spmv": (C.c_int, [_VP, _VP, _VP, _VP]),
    "cgp_gemm_bf16": (C.c_int, [C.c_int, C.c_int, C.c_int, _VP, _VP, _VP, _VP]),
    "cgp_ws_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(_VP)]),
    "cgp_ws_set_params": (C.c_int, [_VP] + [_VP] * 6),
    "cgp_ws_get_params": (C.c_int, [_VP] + [_VP] * 6),
    "cgp_ws_get_grads": (C.c_int, [_VP] + [_VP] * 6),
    "cgp_ws_set_mask": (C.c_int, [_VP, _VP]),
    "cgp_ws_forward": (C.c_int, [_VP, _VP, C.c_int, _VP, _VP]),
    "cgp_ws_train_step": (C.c_int, [_VP, _VP, _VP, C.c_int, C.c_float, _VP, _VP]),
    "cgp_ws_status": (C.c_int, [_VP, _VP]),
    "cgp_ws_destroy": (C.c_int, [_VP]),
    "cgp_ws_forward_residual": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int, _VP, _VP]),
    "cgp_ws_train_step_residual": (C.c_int, [_VP, _VP, _VP, _VP, _VP, C.c_int, C.c_float, _VP, _VP]),
    "cgp_extrapolate": (C.c_int, [C.c_longlong, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP]),
    "cgp_mesh_destroy": (C.c_int, [_VP]),
    "cgp_status_str": (C.c_char_p, [C.c_int]),
}

_lib = None


def load() -> C.CDLL:
    """Load ``libcgp.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CGP CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -m paper_1610_06993_gb300.build`)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class CGPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {load().cgp_status_str(code).decode()}")


def _check(code: int, where: str) -> int:
    if code != CGP_OK:
        raise CGPError(code, where)
    return code


def _ptr(t) -> int | None:
    """Device pointer of a torch tensor, host pointer of a numpy array, or None."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return t.ctypes.data
    assert t.is_contiguous()
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def default_params(**kw) -> cgp_params:
    p = cgp_params()
    load().cgp_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ---- the C entry points, same names, argument marshalling only -----------------------------

def cgp_mesh_create(xy: np.ndarray, tri: np.ndarray, params: cgp_params) -> int:
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    d = cgp_mesh_desc(int(xy.shape[0]), int(tri.shape[0]), xy.ctypes.data_as(C.POINTER(C.c_double)),
                      tri.ctypes.data_as(C.POINTER(C.c_int)))
    h = _VP()
    _check(load().cgp_mesh_create(C.byref(d), C.byref(params), C.byref(h)), "cgp_mesh_create")
    return h.value


def cgp_refine(xy: np.ndarray, tri: np.ndarray, levels: int):
    """Host-only refinement query. Returns ``(xy_f, tri_f, sp, colour)``."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    d = cgp_mesh_desc(int(xy.shape[0]), int(tri.shape[0]), xy.ctypes.data_as(C.POINTER(C.c_double)),
                      tri.ctypes.data_as(C.POINTER(C.c_int)))
    nf, tf = C.c_int(), C.c_int()
    _check(load().cgp_refine(C.byref(d), levels, C.byref(nf), C.byref(tf), None, None, None, None), "cgp_refine")
    xf = np.empty((nf.value, 2), dtype=np.float64)
    tr = np.empty((tf.value, 3), dtype=np.int32)
    sp = np.empty((nf.value, 2), dtype=np.int32)
    col = np.empty(tf.value, dtype=np.int32)
    _check(load().cgp_refine(C.byref(d), levels, C.byref(nf), C.byref(tf), xf.ctypes.data, tr.ctypes.data,
                             sp.ctypes.data, col.ctypes.data), "cgp_refine")
    return xf, tr, sp, col


def cgp_refine_order(xy: np.ndarray, tri: np.ndarray, levels: int) -> np.ndarray:
    """Host-only query of the stored fine-node order (fine_order = 0): perm[i] is the refinement-
    order index of stored node i."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    d = cgp_mesh_desc(int(xy.shape[0]), int(tri.shape[0]), xy.ctypes.data_as(C.POINTER(C.c_double)),
                      tri.ctypes.data_as(C.POINTER(C.c_int)))
    nf, tf = C.c_int(), C.c_int()
    _check(load().cgp_refine(C.byref(d), levels, C.byref(nf), C.byref(tf), None, None, None, None), "cgp_refine")
    perm = np.empty(nf.value, dtype=np.int32)
    _check(load().cgp_refine_order(C.byref(d), levels, perm.ctypes.data), "cgp_refine_order")
    return perm


def cgp_mesh_info(ctx: int) -> cgp_info:
    info = cgp_info()
    _check(load().cgp_mesh_info(ctx, C.byref(info)), "cgp_mesh_info")
    return info


def cgp_fine_mesh(ctx: int):
    info = cgp_mesh_info(ctx)
    xy = np.empty((info.n_fine, 2), dtype=np.float64)
    tri = np.empty((info.tris_fine, 3), dtype=np.int32)
    onb = np.empty(info.n_fine, dtype=np.uint8)
    _check(load().cgp_fine_mesh(ctx, xy.ctypes.data, tri.ctypes.data, onb.ctypes.data), "cgp_fine_mesh")
    return xy, tri, onb.astype(bool)


def cgp_set_bc(ctx: int, vel_mask: np.ndarray, p_mask: np.ndarray, g: np.ndarray) -> None:
    vm = np.ascontiguousarray(vel_mask, dtype=np.uint8)
    pm = np.ascontiguousarray(p_mask, dtype=np.uint8)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    _check(load().cgp_set_bc(ctx, vm.ctypes.data, pm.ctypes.data, gg.ctypes.data), "cgp_set_bc")


def cgp_set_dirichlet_values(ctx: int, g_dev, stream=None) -> None:
    _check(load().cgp_set_dirichlet_values(ctx, _ptr(g_dev), _stream(stream)), "cgp_set_dirichlet_values")


def cgp_assemble(ctx: int, u_dev, stream=None) -> None:
    _check(load().cgp_assemble(ctx, _ptr(u_dev), _stream(stream)), "cgp_assemble")


def cgp_momentum_solve(ctx: int, u_dev, ut_dev, stream=None) -> None:
    _check(load().cgp_momentum_solve(ctx, _ptr(u_dev), _ptr(ut_dev), _stream(stream)), "cgp_momentum_solve")


def cgp_restrict(ctx: int, ut_dev, bc_dev, stream=None) -> None:
    _check(load().cgp_restrict(ctx, _ptr(ut_dev), _ptr(bc_dev), _stream(stream)), "cgp_restrict")


def cgp_poisson_solve(ctx: int, bc_dev, pc_dev, stream=None) -> None:
    _check(load().cgp_poisson_solve(ctx, _ptr(bc_dev), _ptr(pc_dev), _stream(stream)), "cgp_poisson_solve")


def cgp_prolong_correct(ctx: int, pc_dev, ut_dev, u_dev, pf_dev=None, gp_dev=None, stream=None) -> None:
    _check(load().cgp_prolong_correct(ctx, _ptr(pc_dev), _ptr(ut_dev), _ptr(u_dev), _ptr(pf_dev), _ptr(gp_dev),
                                      _stream(stream)), "cgp_prolong_correct")


def cgp_step(ctx: int, u_dev, pc_dev, stream=None) -> None:
    _check(load().cgp_step(ctx, _ptr(u_dev), _ptr(pc_dev), _stream(stream)), "cgp_step")


def cgp_poisson_solve_many(ctx: int, b_dev, x_dev, iters_dev=None, rel_dev=None, status_dev=None, stream=None) -> None:
    """Solve the coarse Poisson system for every row of b_dev [nrhs][n_coarse] into x_dev."""
    nrhs = int(b_dev.shape[0])
    _check(load().cgp_poisson_solve_many(ctx, nrhs, _ptr(b_dev), _ptr(x_dev), _ptr(iters_dev), _ptr(rel_dev),
                                         _ptr(status_dev), _stream(stream)), "cgp_poisson_solve_many")


def cgp_assemble_incremental(ctx: int, u_dev, pc_dev, stream=None) -> None:
    _check(load().cgp_assemble_incremental(ctx, _ptr(u_dev), _ptr(pc_dev), _stream(stream)),
           "cgp_assemble_incremental")


def cgp_pressure_update(ctx: int, bc_dev, phi_dev, pc_dev, stream=None) -> None:
    _check(load().cgp_pressure_update(ctx, _ptr(bc_dev), _ptr(phi_dev), _ptr(pc_dev), _stream(stream)),
           "cgp_pressure_update")


def cgp_step_host(ctx: int, u_host, pc_host, stream=None) -> None:
    """``u_host``/``pc_host``: contiguous float64 host buffers (numpy arrays or pinned CPU tensors)."""
    _check(load().cgp_step_host(ctx, _ptr(u_host), _ptr(pc_host), _stream(stream)), "cgp_step_host")


def cgp_get_stats(ctx: int, stream=None, check: bool = False) -> cgp_stats:
    st = cgp_stats()
    code = load().cgp_get_stats(ctx, _stream(stream), C.byref(st))
    if code in (CGP_ERR_ARG, CGP_ERR_CUDA) or (check and code != CGP_OK):
        raise CGPError(code, "cgp_get_stats")
    st.code = code
    return st


def cgp_autotune(ctx: int, stream=None) -> None:
    _check(load().cgp_autotune(ctx, _stream(stream)), "cgp_autotune")


def cgp_cg_solve_noalloc(rp_dev, ci_dev, val_dev, b_dev, x_dev, rtol: float, max_iter: int, status_dev=None,
                         iters_dev=None, rel_res_dev=None, stream=None) -> None:
    """Allocation-free CG solve of a CSR system held in caller device tensors (see cgp.h)."""
    n = int(b_dev.numel())
    _check(load().cgp_cg_solve_noalloc(n, _ptr(rp_dev), _ptr(ci_dev), _ptr(val_dev), _ptr(b_dev), _ptr(x_dev),
                                       float(rtol), int(max_iter), _ptr(status_dev), _ptr(iters_dev),
                                       _ptr(rel_res_dev), _stream(stream)), "cgp_cg_solve_noalloc")


def cgp_wait_probe(ctx: int, missing_blocks: int, limit_ms: float, status_dev, stream=None) -> None:
    """One bounded grid barrier that waits for ``missing_blocks`` more blocks than were launched."""
    _check(load().cgp_wait_probe(ctx, int(missing_blocks), float(limit_ms), _ptr(status_dev), _stream(stream)),
           "cgp_wait_probe")


def cgp_set_surface(ctx: int, which: int, node_mask: np.ndarray) -> int:
    """Body (which = 0) or wall (which = 1) of the diagnostics; returns its edge count."""
    m = np.ascontiguousarray(node_mask, dtype=np.uint8)
    n = C.c_int(0)
    _check(load().cgp_set_surface(ctx, int(which), _ptr(m), C.byref(n)), "cgp_set_surface")
    return n.value


def cgp_body_force(ctx: int, u_dev, pc_dev, force_dev, stream=None) -> None:
    _check(load().cgp_body_force(ctx, _ptr(u_dev), _ptr(pc_dev), _ptr(force_dev), _stream(stream)), "cgp_body_force")


def cgp_reattachment(ctx: int, u_dev, x_start: float, xr_dev, x_dev=None, tau_dev=None, stream=None) -> None:
    _check(load().cgp_reattachment(ctx, _ptr(u_dev), float(x_start), _ptr(xr_dev), _ptr(x_dev), _ptr(tau_dev),
                                   _stream(stream)), "cgp_reattachment")


def cgp_batch_create(ctxs, u_devs, pc_devs) -> int:
    n = len(ctxs)
    arr_c = (C.c_void_p * n)(*ctxs)
    arr_u = (C.c_void_p * n)(*[_ptr(t) for t in u_devs])
    arr_p = (C.c_void_p * n)(*[_ptr(t) for t in pc_devs])
    h = _VP()
    _check(load().cgp_batch_create(arr_c, n, arr_u, arr_p, C.byref(h)), "cgp_batch_create")
    return h.value


def cgp_batch_info(b: int, n: int):
    blocks = C.c_int()
    gf = np.zeros(n, dtype=np.int32)
    gc = np.zeros(n, dtype=np.int32)
    _check(load().cgp_batch_info(b, C.byref(blocks), gf.ctypes.data, gc.ctypes.data), "cgp_batch_info")
    return blocks.value, gf, gc


def cgp_batch_step(b: int, stream=None) -> None:
    _check(load().cgp_batch_step(b, _stream(stream)), "cgp_batch_step")


def cgp_batch_run(b: int, steps: int, stream=None) -> None:
    _check(load().cgp_batch_run(b, int(steps), _stream(stream)), "cgp_batch_run")


def cgp_batch_poisson_solve(b: int, stream=None) -> None:
    _check(load().cgp_batch_poisson_solve(b, _stream(stream)), "cgp_batch_poisson_solve")


def cgp_batch_get_stats(b: int, n: int, stream=None, check: bool = False):
    arr = (cgp_stats * n)()
    code = load().cgp_batch_get_stats(b, _stream(stream), arr)
    if code in (CGP_ERR_ARG, CGP_ERR_CUDA) or (check and code != CGP_OK):
        raise CGPError(code, "cgp_batch_get_stats")
    return list(arr), code


def cgp_batch_destroy(b: int) -> None:
    _check(load().cgp_batch_destroy(b), "cgp_batch_destroy")


def cgp_fine_order(ctx: int, n_fine: int) -> np.ndarray:
    """Refinement-order index of every stored fine node (the library's storage order)."""
    perm = np.empty(n_fine, dtype=np.int32)
    _check(load().cgp_fine_order(ctx, _ptr(perm)), "cgp_fine_order")
    return perm


def cgp_solver_spmv(ctx: int, x_dev, y_dev, stream=None) -> None:
    _check(load().cgp_solver_spmv(ctx, _ptr(x_dev), _ptr(y_dev), _stream(stream)), "cgp_solver_spmv")


def cgp_spmv(ctx: int, x_dev, y_dev, stream=None) -> None:
    _check(load().cgp_spmv(ctx, _ptr(x_dev), _ptr(y_dev), _stream(stream)), "cgp_spmv")


def cgp_predict_pressure(ctx: int, pc_dev, stream=None) -> None:
    _check(load().cgp_predict_pressure(ctx, _ptr(pc_dev), _stream(stream)), "cgp_predict_pressure")


def cgp_copy_coarse_rhs(ctx: int, bc_dev, stream=None) -> None:
    _check(load().cgp_copy_coarse_rhs(ctx, _ptr(bc_dev), _stream(stream)), "cgp_copy_coarse_rhs")


def cgp_gemm_bf16(A_dev, B_dev, C_dev, stream=None) -> None:
    """C[M,N] (float32) = A[M,K] B[N,K]^T for bfloat16 device tensors A, B."""
    M, K = A_dev.shape
    N = B_dev.shape[0]
    _check(load().cgp_gemm_bf16(M, N, K, _ptr(A_dev), _ptr(B_dev), _ptr(C_dev), _stream(stream)), "cgp_gemm_bf16")


def cgp_ws_create(n: int, hidden: int, batch_max: int) -> int:
    h = _VP()
    _check(load().cgp_ws_create(n, hidden, batch_max, C.byref(h)), "cgp_ws_create")
    return h.value


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def cgp_ws_set_params(w: int, params) -> None:
    arrs = [_f32(p) for p in params]
    _check(load().cgp_ws_set_params(w, *[a.ctypes.data for a in arrs]), "cgp_ws_set_params")


def _ws_read(fn, w: int, n: int, hidden: int):
    out = [np.empty((hidden, n), np.float32), np.empty(hidden, np.float32), np.empty((hidden, hidden), np.float32),
           np.empty(hidden, np.float32), np.empty((n, hidden), np.float32), np.empty(n, np.float32)]
    _check(fn(w, *[a.ctypes.data for a in out]), "cgp_ws_read")
    return out


def cgp_ws_get_params(w: int, n: int, hidden: int):
    return _ws_read(load().cgp_ws_get_params, w, n, hidden)


def cgp_ws_get_grads(w: int, n: int, hidden: int):
    return _ws_read(load().cgp_ws_get_grads, w, n, hidden)


def cgp_ws_set_mask(w: int, held: np.ndarray) -> None:
    m = np.ascontiguousarray(held, dtype=np.uint8)
    _check(load().cgp_ws_set_mask(w, m.ctypes.data), "cgp_ws_set_mask")


def cgp_ws_forward(w: int, b_dev, p_dev, stream=None) -> None:
    _check(load().cgp_ws_forward(w, _ptr(b_dev), int(b_dev.shape[0]), _ptr(p_dev), _stream(stream)), "cgp_ws_forward")


def cgp_ws_train_step(w: int, b_dev, p_dev, lr: float, loss_dev=None, stream=None) -> None:
    _check(load().cgp_ws_train_step(w, _ptr(b_dev), _ptr(p_dev), int(b_dev.shape[0]), float(lr), _ptr(loss_dev),
                                    _stream(stream)), "cgp_ws_train_step")


def cgp_ws_status(w: int, stream=None) -> int:
    return load().cgp_ws_status(w, _stream(stream))


def cgp_ws_forward_residual(w: int, ctx: int, b_dev, base_dev, p_dev, stream=None) -> None:
    _check(load().cgp_ws_forward_residual(w, ctx, _ptr(b_dev), _ptr(base_dev), int(b_dev.shape[0]), _ptr(p_dev),
                                          _stream(stream)), "cgp_ws_forward_residual")


def cgp_ws_train_step_residual(w: int, ctx: int, b_dev, p_dev, base_dev, lr: float, loss_dev=None,
                               stream=None) -> None:
    _check(load().cgp_ws_train_step_residual(w, ctx, _ptr(b_dev), _ptr(p_dev), _ptr(base_dev), int(b_dev.shape[0]),
                                             float(lr), _ptr(loss_dev), _stream(stream)), "cgp_ws_train_step_residual")


def cgp_extrapolate(order: int, v, out_dev, stream=None) -> None:
    """out = extrapolation of order ``order`` through the tensors v[0] (newest) .. v[order]."""
    vs = [_ptr(x) for x in v] + [None] * (4 - len(v))
    _check(load().cgp_extrapolate(int(out_dev.numel()), int(order), *vs, _ptr(out_dev), _stream(stream)),
           "cgp_extrapolate")


def cgp_ws_destroy(w: int) -> None:
    _check(load().cgp_ws_destroy(w), "cgp_ws_destroy")


def cgp_mesh_destroy(ctx: int) -> None:
    _check(load().cgp_mesh_destroy(ctx), "cgp_mesh_destroy")


def cgp_status_str(code: int) -> str:
    return load().cgp_status_str(code).decode()
