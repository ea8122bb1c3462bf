"""Thin Python binding of librbws (include/rbws.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: host arrays are passed as numpy float64 arrays,
device arrays as torch CUDA tensors (their data_ptr()).  The shared library
must have been built (paper_2311_13862_gb300.build.build()); if it is missing
or a call fails, an exception is raised -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librbws.so")

RBWS_OK = 0
RBWS_WARN_NOT_CONVERGED = 1
ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NO_BASIS, ERR_NOT_SPD, ERR_DEVICE_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7, -8)
STATUS_NAMES = {0: "OK", 1: "WARN_NOT_CONVERGED", -1: "ERR_INVALID_ARG", -2: "ERR_OOM", -3: "ERR_CUDA",
                -4: "ERR_NO_BASIS", -5: "ERR_NOT_SPD", -6: "ERR_DEVICE_TIMEOUT", -7: "ERR_STATE",
                -8: "ERR_UNSUPPORTED"}
WARM_ZERO, WARM_GALERKIN, WARM_LEARNED, WARM_LEARNED_CORRECTED, WARM_L1ROC = 0, 1, 2, 3, 4
PREC_NONE, PREC_JACOBI, PREC_MSRB, PREC_MG = 0, 1, 2, 3
FP64, FP32_IR = 0, 1


class RbwsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib().rbws_last_error().decode()
        super().__init__("%s: %s (%s)" % (where, STATUS_NAMES.get(status, status), msg))


class rbws_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32)]


class rbws_blocks(C.Structure):
    _fields_ = [("bx", C.c_int32), ("by", C.c_int32), ("bz", C.c_int32)]


class rbws_profile(C.Structure):
    _fields_ = [("launches", C.c_int64), ("samples", C.c_int64), ("stencil_ms", C.c_double),
                ("update_ms", C.c_double), ("active_dofs", C.c_double), ("elem_bytes", C.c_int32),
                ("schedule", C.c_int32), ("precond_ms", C.c_double), ("mg_fine_ms", C.c_double * 4),
                ("mg_prolong_ms", C.c_double)]


class rbws_axes(C.Structure):
    _fields_ = [("kappa_scale", C.c_double * 3), ("neumann_hi", C.c_int32 * 3), ("reserved", C.c_int32)]


class rbws_options(C.Structure):
    _fields_ = [("max_iters", C.c_int32), ("precond", C.c_int32), ("precision", C.c_int32),
                ("max_restarts", C.c_int32), ("inner_tol", C.c_double), ("max_outer", C.c_int32),
                ("check_every", C.c_int32), ("stream", C.c_void_p),
                ("profile", C.POINTER(rbws_profile)), ("relres_hist", C.c_void_p), ("hist_len", C.c_int32),
                ("wait_cycles", C.c_int64), ("ru_mode", C.c_int32), ("persistent", C.c_int32)]


_L = None


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librbws.so is not built: run paper_2311_13862_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        L.rbws_last_error.restype = C.c_char_p
        L.rbws_options_default.argtypes = [C.POINTER(rbws_options)]
        L.rbws_problem_create.argtypes = [C.POINTER(rbws_grid), C.POINTER(rbws_blocks), P, i32, P, C.c_int,
                                          C.POINTER(P)]
        L.rbws_problem_create_ex.argtypes = [C.POINTER(rbws_grid), C.POINTER(rbws_blocks), P, i32, P,
                                             C.POINTER(rbws_axes), C.c_int, C.POINTER(P)]
        L.rbws_gaussian_source_ex.argtypes = [P, P, i32, P]
        L.rbws_problem_create_field.argtypes = [C.POINTER(rbws_grid), i32, P, P, P, P, C.c_int, C.POINTER(P)]
        L.rbws_dirichlet_lift.argtypes = [P, P, P]
        L.rbws_affine_sources.argtypes = [P, P, i32, P, i32, P]
        L.rbws_problem_destroy.argtypes = [P]
        L.rbws_problem_info.argtypes = [P, C.POINTER(i64), C.POINTER(i32), C.POINTER(i32)]
        L.rbws_apply_operator.argtypes = [P, P, i32, P, P, i32, P]
        L.rbws_apply_preconditioner.argtypes = [P, P, i32, i32, P, P, P]
        L.rbws_offline_l1roc.argtypes = [P, P, i32, i32, d, P, P, C.POINTER(i32)]
        L.rbws_l1roc_info.argtypes = [P, C.POINTER(i32), P, P]
        L.rbws_l1roc_coefficients.argtypes = [P, P, i32, P]
        L.rbws_rb_residuals.argtypes = [P, P, i32, i32, P]
        L.rbws_gaussian_source.argtypes = [P, P, i32, P]
        L.rbws_apply_mg32.argtypes = [P, P, i32, P, P, P]
        L.rbws_update_ff.argtypes = [P, P, i32, P, P, P, P]
        L.rbws_apply_operator_interleaved.argtypes = [P, P, i32, P, P, i32, P]
        L.rbws_autotune_layout.argtypes = [P, i32, i32, C.POINTER(d), C.POINTER(d), C.POINTER(i32)]
        L.rbws_solve_batch_rhs.argtypes = [P, P, i32, P, d, i32, C.POINTER(rbws_options), P, P, P, P]
        L.rbws_offline_greedy_rhs.argtypes = [P, P, P, i32, i32, d, d, P, P, C.POINTER(i32)]
        L.rbws_apply_operator_static.argtypes = [P, P, i32, P, P, i32, P]
        L.rbws_offline_greedy.argtypes = [P, P, i32, i32, d, d, i32, P, P, C.POINTER(i32)]
        L.rbws_set_basis.argtypes = [P, i32, P, P, P]
        L.rbws_get_basis.argtypes = [P, P, P, P]
        L.rbws_reduced_solve.argtypes = [P, P, i32, P]
        L.rbws_solve_batch.argtypes = [P, P, i32, d, i32, C.POINTER(rbws_options), P, P, P, P]
        L.rbws_train_surrogate.argtypes = [P, P, i32, P, i32, i32, i32, d, d, d, C.c_uint64, C.POINTER(d)]
        L.rbws_surrogate_set_params.argtypes = [P, i32, P, P, d, d]
        L.rbws_surrogate_get_params.argtypes = [P, C.POINTER(i32), P, P]
        L.rbws_surrogate_forward.argtypes = [P, P, i32, i32, P]
        L.rbws_surrogate_loss_grad.argtypes = [P, P, P, i32, C.POINTER(d), P]
        L.rbws_save.argtypes = [P, C.c_char_p]
        L.rbws_load.argtypes = [C.c_char_p, C.c_int, C.POINTER(P)]
        L.rbws_solve_requests.argtypes = [i32, P, P, P, d, i32, C.POINTER(rbws_options), P, P, P, P]
        L.rbws_autotune.argtypes = [P, i32, C.c_char_p, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                    C.POINTER(i32), C.POINTER(d)]
        for name in ("rbws_problem_create", "rbws_problem_info", "rbws_apply_operator", "rbws_apply_operator_static",
                     "rbws_offline_greedy", "rbws_set_basis", "rbws_get_basis", "rbws_reduced_solve",
                     "rbws_solve_batch", "rbws_train_surrogate", "rbws_surrogate_set_params",
                     "rbws_surrogate_get_params", "rbws_surrogate_forward", "rbws_surrogate_loss_grad",
                     "rbws_solve_requests", "rbws_autotune", "rbws_save", "rbws_load", "rbws_apply_preconditioner",
                     "rbws_offline_l1roc", "rbws_l1roc_info", "rbws_l1roc_coefficients", "rbws_rb_residuals",
                     "rbws_gaussian_source", "rbws_solve_batch_rhs", "rbws_offline_greedy_rhs", "rbws_apply_mg32"):
            getattr(L, name).restype = C.c_int
        _L = L
    return _L


def _check(rc, where):
    if rc < 0:
        raise RbwsError(rc, where)
    return rc


def _host(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _hp(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dp(t):
    """Device pointer of a CUDA tensor (contiguous required)."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def rbws_options_default(**kw) -> rbws_options:
    o = rbws_options()
    _lib().rbws_options_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def rbws_problem_create(grid, blocks, Q=None, f=None, device=0, subdomain_map=None, kappa_scale=None,
                        neumann=None):
    """blocks: (bx, by, bz) for the block rule, or None with subdomain_map = a uint8 [nz][ny][nx]
    array of subdomain ids < Q.  kappa_scale (diffusion tensor diagonal) and neumann (per axis, 1
    for a Neumann face at coordinate 1) select rbws_problem_create_ex."""
    g = rbws_grid(*grid)
    if subdomain_map is not None:
        if blocks is not None or Q is None:
            raise ValueError("give either blocks, or subdomain_map with Q")
        m = np.ascontiguousarray(subdomain_map, dtype=np.uint8).reshape(-1)
        if m.size != grid[0] * grid[1] * grid[2]:
            raise ValueError("subdomain_map must have nx*ny*nz entries")
        bref, mp = None, m.ctypes.data_as(C.c_void_p)
    else:
        bref, mp = C.byref(rbws_blocks(*blocks)), None
        Q = blocks[0] * blocks[1] * blocks[2] if Q is None else Q
    fh = None if f is None else _host(f)
    h = C.c_void_p()
    if kappa_scale is None and neumann is None:
        _check(_lib().rbws_problem_create(C.byref(g), bref, mp, Q, _hp(fh), device, C.byref(h)),
               "rbws_problem_create")
    else:
        ax = rbws_axes((C.c_double * 3)(*(kappa_scale or (1.0, 1.0, 1.0))), (C.c_int32 * 3)(*(neumann or (0, 0, 0))), 0)
        _check(_lib().rbws_problem_create_ex(C.byref(g), bref, mp, Q, _hp(fh), C.byref(ax), device, C.byref(h)),
               "rbws_problem_create_ex")
    return h


def rbws_problem_create_field(grid, kfx, kfy, kfz, f=None, device=0):
    """A problem whose coefficient is given at the cell faces per affine term: kfx [Q][nz][ny][nx+1],
    kfy [Q][nz][ny+1][nx], kfz [Q][nz+1][ny][nx] (host arrays, copied)."""
    nx, ny, nz = grid
    kfx = _host(kfx)
    Q = kfx.shape[0]
    kfx = kfx.reshape(Q, nz, ny, nx + 1)
    kfy = _host(kfy).reshape(Q, nz, ny + 1, nx)
    kfz = _host(kfz).reshape(Q, nz + 1, ny, nx)
    fh = None if f is None else _host(f)
    h = C.c_void_p()
    _check(_lib().rbws_problem_create_field(C.byref(rbws_grid(*grid)), Q, _hp(kfx), _hp(kfy), _hp(kfz), _hp(fh),
                                            device, C.byref(h)), "rbws_problem_create_field")
    return h, Q


def rbws_dirichlet_lift(h, g, lift_out):
    """lift_out (CUDA float64 [Q][n]) = the right-hand side that Dirichlet data g (host, the six
    boundary planes x=0, x=1, y=0, y=1, z=0, z=1) adds through each term of a face-field problem."""
    gh = _host(g)
    _check(_lib().rbws_dirichlet_lift(h, _hp(gh), _dp(lift_out)), "rbws_dirichlet_lift")


def rbws_affine_sources(h, F, theta, f_out):
    """f_out[b] = sum_k theta[b][k] F[k]: F CUDA float64 [K][n], theta host [B][K], f_out CUDA [B][n]."""
    th = _host(np.atleast_2d(theta))
    _check(_lib().rbws_affine_sources(h, _dp(F), th.shape[1], _hp(th), th.shape[0], _dp(f_out)),
           "rbws_affine_sources")


def rbws_problem_destroy(h):
    _lib().rbws_problem_destroy(h)


def rbws_problem_info(h):
    n, Q, N = C.c_int64(), C.c_int32(), C.c_int32()
    _check(_lib().rbws_problem_info(h, C.byref(n), C.byref(Q), C.byref(N)), "rbws_problem_info")
    return n.value, Q.value, N.value


def rbws_apply_preconditioner(h, mu, x, y, precond=PREC_MG, stream=None):
    """y[b] = P(mu_b) x[b] (Jacobi or one multigrid V-cycle); x, y CUDA float64 [B][n]."""
    mu = _host(np.atleast_2d(mu))
    _check(_lib().rbws_apply_preconditioner(h, _hp(mu), mu.shape[0], precond, _dp(x), _dp(y), stream),
           "rbws_apply_preconditioner")


def rbws_apply_operator(h, mu, x, y, precision=FP64, stream=None):
    mu = _host(np.atleast_2d(mu))
    _check(_lib().rbws_apply_operator(h, _hp(mu), mu.shape[0], _dp(x), _dp(y), precision, stream),
           "rbws_apply_operator")


def rbws_apply_operator_interleaved(h, mu, x, y, precision=FP64, stream=None):
    """y = A(mu_b) x in the mu-interleaved layout: x, y CUDA tensors [n][B] (instance fastest)."""
    mu = _host(np.atleast_2d(mu))
    _check(_lib().rbws_apply_operator_interleaved(h, _hp(mu), mu.shape[0], _dp(x), _dp(y), precision, stream),
           "rbws_apply_operator_interleaved")


def rbws_autotune_layout(h, B, precision=FP32_IR):
    """Times the planar and the mu-interleaved operator apply: returns (planar_ms, interleaved_ms,
    layout) with layout 0 planar, 1 interleaved (the faster)."""
    tp, ti, lay = C.c_double(0.0), C.c_double(0.0), C.c_int32(0)
    _check(_lib().rbws_autotune_layout(h, B, precision, C.byref(tp), C.byref(ti), C.byref(lay)),
           "rbws_autotune_layout")
    return tp.value, ti.value, lay.value


def rbws_update_ff(h, mu, u0, d, u_out, r_out):
    """One float-float reliable update from u0 with correction d (test entry point):
    u_out = u0 + d, r_out = f - A(mu)(u0 + d), both FP64 device tensors [B][n]."""
    mu = _host(np.atleast_2d(mu))
    _check(_lib().rbws_update_ff(h, _hp(mu), mu.shape[0], _dp(u0), _dp(d), _dp(u_out), _dp(r_out)),
           "rbws_update_ff")


def rbws_apply_operator_static(h, mu, x, y, precision=FP64, stream=None):
    """rbws_apply_operator without device allocation (scratch in a static device array)."""
    mu = _host(np.atleast_2d(mu))
    _check(_lib().rbws_apply_operator_static(h, _hp(mu), mu.shape[0], _dp(x), _dp(y), precision, stream),
           "rbws_apply_operator_static")


INDICATOR_RESIDUAL, INDICATOR_L1 = 0, 1


def rbws_offline_l1roc(h, mu_train, n_max, snapshot_tol=1e-12):
    """Offline L1ROC (Algorithm 5): returns (N, selected [n_max], eta_hist [n_max])."""
    mu = _host(np.atleast_2d(mu_train))
    sel = np.full(n_max, -1, dtype=np.int32)
    eta = np.full(n_max, np.nan)
    n_out = C.c_int32(0)
    _check(_lib().rbws_offline_l1roc(h, _hp(mu), mu.shape[0], n_max, snapshot_tol, _hp(sel), _hp(eta),
                                     C.byref(n_out)), "rbws_offline_l1roc")
    return n_out.value, sel, eta


def rbws_l1roc_info(h):
    """(collocation node indices [M], T [N][N]) of the L1ROC basis."""
    _, _, N = rbws_problem_info(h)
    M = C.c_int32(0)
    _check(_lib().rbws_l1roc_info(h, C.byref(M), None, None), "rbws_l1roc_info")
    pts = np.zeros(M.value, dtype=np.int64)
    T = np.zeros((N, N))
    _check(_lib().rbws_l1roc_info(h, C.byref(M), _hp(pts), _hp(T)), "rbws_l1roc_info")
    return pts, T


def rbws_l1roc_coefficients(h, mu):
    """Online L1ROC coefficients c [B][N]."""
    mu = _host(np.atleast_2d(mu))
    _, _, N = rbws_problem_info(h)
    c = np.empty((mu.shape[0], N))
    _check(_lib().rbws_l1roc_coefficients(h, _hp(mu), mu.shape[0], _hp(c)), "rbws_l1roc_coefficients")
    return c


def rbws_apply_mg32(h, mu, x, y, stream=None):
    """One FP32 V-cycle y = MG(x) as the mixed-precision iteration applies it (x, y CUDA float32 [B][n])."""
    mu = _host(np.atleast_2d(mu))
    _check(_lib().rbws_apply_mg32(h, _hp(mu), mu.shape[0], _dp(x), _dp(y), stream), "rbws_apply_mg32")


def rbws_gaussian_source(h, params, f_out):
    """f_out (CUDA float64 [B][n]) = exp(-|x - c_b|^2 / (2 s_b^2)); params [B][4] = (c_x, c_y, c_z, s_b)."""
    prm = _host(np.atleast_2d(params))
    _check(_lib().rbws_gaussian_source(h, _hp(prm), prm.shape[0], _dp(f_out)), "rbws_gaussian_source")


def rbws_gaussian_source_ex(h, params, f_out):
    """f_out (CUDA float64 [B][n]) = (offset + amplitude exp(-|x - c_b|^2 / width)) times each node's
    relative control volume; params [B][6] = (c_x, c_y, c_z, width, amplitude, offset)."""
    prm = _host(np.atleast_2d(params))
    _check(_lib().rbws_gaussian_source_ex(h, _hp(prm), prm.shape[0], _dp(f_out)), "rbws_gaussian_source_ex")


def rbws_solve_batch_rhs(h, mu, f, tol, warm, u_out, options: rbws_options | None = None):
    """rbws_solve_batch with right-hand sides f (CUDA float64 [B][n]); returns (status, iters, relres,
    inst_status)."""
    mu = _host(np.atleast_2d(mu))
    B = mu.shape[0]
    it = np.zeros(B, dtype=np.int32)
    rel = np.zeros(B)
    st = np.zeros(B, dtype=np.int32)
    rc = _check(_lib().rbws_solve_batch_rhs(h, _hp(mu), B, _dp(f), tol, warm,
                                            None if options is None else C.byref(options), _dp(u_out), _hp(it),
                                            _hp(rel), _hp(st)), "rbws_solve_batch_rhs")
    return rc, it, rel, st


def rbws_offline_greedy_rhs(h, mu_train, f_train, n_max, greedy_tol=0.0, snapshot_tol=1e-12):
    """Greedy with a right-hand side per training parameter (f_train: CUDA float64 [n_train][n]);
    returns (N, selected, indicator history)."""
    mu = _host(np.atleast_2d(mu_train))
    sel = np.full(n_max, -1, dtype=np.int32)
    eta = np.full(n_max, np.nan)
    n = C.c_int32(0)
    _check(_lib().rbws_offline_greedy_rhs(h, _hp(mu), _dp(f_train), mu.shape[0], n_max, greedy_tol, snapshot_tol,
                                          _hp(sel), _hp(eta), C.byref(n)), "rbws_offline_greedy_rhs")
    return n.value, sel[:n.value], eta[:n.value]


def rbws_rb_residuals(h, mu, n_use):
    """||f - A(mu) W_n c_n|| / ||f|| [B] of the Galerkin RB solutions with the first n_use basis vectors."""
    mu = _host(np.atleast_2d(mu))
    rel = np.empty(mu.shape[0])
    _check(_lib().rbws_rb_residuals(h, _hp(mu), mu.shape[0], int(n_use), _hp(rel)), "rbws_rb_residuals")
    return rel


def rbws_offline_greedy(h, mu_train, n_max, greedy_tol=0.0, snapshot_tol=1e-12, indicator=INDICATOR_RESIDUAL):
    mu = _host(np.atleast_2d(mu_train))
    sel = np.full(n_max, -1, dtype=np.int32)
    eta = np.full(n_max, np.nan)
    n_out = C.c_int32(0)
    _check(_lib().rbws_offline_greedy(h, _hp(mu), mu.shape[0], n_max, greedy_tol, snapshot_tol, indicator,
                                      _hp(sel), _hp(eta), C.byref(n_out)), "rbws_offline_greedy")
    N = n_out.value
    return N, sel[:N], eta[:N]


def rbws_set_basis(h, W, ANq, fN):
    W, ANq, fN = _host(W), _host(ANq), _host(fN)
    _check(_lib().rbws_set_basis(h, W.shape[0], _hp(W), _hp(ANq), _hp(fN)), "rbws_set_basis")


def rbws_get_basis(h):
    n, Q, N = rbws_problem_info(h)
    W = np.empty((N, n))
    ANq = np.empty((Q, N, N))
    fN = np.empty(N)
    _check(_lib().rbws_get_basis(h, _hp(W), _hp(ANq), _hp(fN)), "rbws_get_basis")
    return W, ANq, fN


def rbws_reduced_solve(h, mu):
    mu = _host(np.atleast_2d(mu))
    _, _, N = rbws_problem_info(h)
    c = np.empty((mu.shape[0], N))
    _check(_lib().rbws_reduced_solve(h, _hp(mu), mu.shape[0], _hp(c)), "rbws_reduced_solve")
    return c


def rbws_solve_batch(h, mu, tol, warm, u_out, options: rbws_options | None = None):
    """Returns (status, iters, relres, inst_status); u_out is a CUDA float64 tensor [B][n]."""
    mu = _host(np.atleast_2d(mu))
    B = mu.shape[0]
    it = np.zeros(B, dtype=np.int32)
    rel = np.zeros(B)
    st = np.zeros(B, dtype=np.int32)
    rc = _check(_lib().rbws_solve_batch(h, _hp(mu), B, tol, warm, None if options is None else C.byref(options),
                                        _dp(u_out), _hp(it), _hp(rel), _hp(st)), "rbws_solve_batch")
    return rc, it, rel, st


def rbws_solve_batch_history(h, mu, tol, warm, u_out, hist_len, options: rbws_options | None = None):
    """rbws_solve_batch with the FP64 residual history: returns (status, iters, relres,
    inst_status, hist) with hist [B][hist_len] (NaN past each instance's last iteration)."""
    B = np.atleast_2d(mu).shape[0]
    hist = np.full((B, hist_len), np.nan)
    o = options if options is not None else rbws_options_default()
    o.relres_hist = hist.ctypes.data_as(C.c_void_p)
    o.hist_len = hist_len
    try:
        rc, it, rel, st = rbws_solve_batch(h, mu, tol, warm, u_out, o)
    finally:
        o.relres_hist = None
        o.hist_len = 0
    return rc, it, rel, st, hist


def mlp_param_count(p, H, N):
    return H * p + H + 2 * (H * H + H) + N * H + N


def rbws_train_surrogate(h, mu, hidden=256, epochs=2000, batch=256, lr=1e-3, mu_lo=0.1, mu_hi=10.0,
                         seed=0, targets=None):
    mu = _host(np.atleast_2d(mu))
    t = None if targets is None else _host(targets)
    loss = C.c_double(0)
    _check(_lib().rbws_train_surrogate(h, _hp(mu), mu.shape[0], _hp(t), hidden, epochs, batch, lr, mu_lo,
                                       mu_hi, seed, C.byref(loss)), "rbws_train_surrogate")
    return loss.value


def rbws_surrogate_set_params(h, hidden, params, coef_scale=None, mu_lo=0.1, mu_hi=10.0):
    params = _host(params, np.float32)
    cs = None if coef_scale is None else _host(coef_scale, np.float32)
    _check(_lib().rbws_surrogate_set_params(h, hidden, _hp(params), _hp(cs), mu_lo, mu_hi),
           "rbws_surrogate_set_params")


def rbws_surrogate_get_params(h):
    n, Q, N = rbws_problem_info(h)
    H = C.c_int32(0)
    _check(_lib().rbws_surrogate_get_params(h, C.byref(H), None, None), "rbws_surrogate_get_params")
    params = np.empty(mlp_param_count(Q, H.value, N), dtype=np.float32)
    cs = np.empty(N, dtype=np.float32)
    _check(_lib().rbws_surrogate_get_params(h, None, _hp(params), _hp(cs)), "rbws_surrogate_get_params")
    return H.value, params, cs


def rbws_surrogate_forward(h, mu, corrected=False):
    mu = _host(np.atleast_2d(mu))
    _, _, N = rbws_problem_info(h)
    c = np.empty((mu.shape[0], N))
    _check(_lib().rbws_surrogate_forward(h, _hp(mu), mu.shape[0], int(bool(corrected)), _hp(c)),
           "rbws_surrogate_forward")
    return c


def rbws_surrogate_loss_grad(h, x, t):
    x = _host(np.atleast_2d(x), np.float32)
    t = _host(np.atleast_2d(t), np.float32)
    n, Q, N = rbws_problem_info(h)
    H, params, _ = rbws_surrogate_get_params(h)
    g = np.empty(params.size, dtype=np.float32)
    loss = C.c_double(0)
    _check(_lib().rbws_surrogate_loss_grad(h, _hp(x), _hp(t), x.shape[0], C.byref(loss), _hp(g)),
           "rbws_surrogate_loss_grad")
    return loss.value, g


def rbws_solve_requests(handles, mus, u_outs, tol, warm, options: rbws_options | None = None):
    """One request per (handle, mu, u_out); returns (status, iters, relres, inst_status, latency_ms)."""
    n = len(handles)
    H = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    mus = [_host(np.ravel(m)) for m in mus]
    M = (C.c_void_p * n)(*[m.ctypes.data for m in mus])
    U = (C.c_void_p * n)(*[_dp(u).value for u in u_outs])
    it = np.zeros(n, dtype=np.int32)
    rel = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    lat = np.zeros(n)
    rc = _check(_lib().rbws_solve_requests(n, H, M, U, tol, warm, None if options is None else C.byref(options),
                                           _hp(it), _hp(rel), _hp(st), _hp(lat)), "rbws_solve_requests")
    return rc, it, rel, st, lat


def rbws_autotune(h, B, cache_path=None):
    """Returns (tx, ty, zc, ms, schedule) of the fastest FP32 configuration for batches of B."""
    tx, ty, zc, sc, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
    path = None if cache_path is None else str(cache_path).encode()
    _check(_lib().rbws_autotune(h, B, path, C.byref(tx), C.byref(ty), C.byref(zc), C.byref(sc), C.byref(ms)),
           "rbws_autotune")
    return tx.value, ty.value, zc.value, ms.value, sc.value


def rbws_save(h, path):
    _check(_lib().rbws_save(h, str(path).encode()), "rbws_save")


def rbws_load(path, device=0):
    h = C.c_void_p()
    _check(_lib().rbws_load(str(path).encode(), device, C.byref(h)), "rbws_load")
    return h


class Problem:
    """Owning wrapper around an rbws_problem handle."""

    def __init__(self, grid, blocks=None, f=None, device=0, handle=None, subdomain_map=None, Q=None,
                 kappa_scale=None, neumann=None):
        self.grid = tuple(grid)
        self.n = grid[0] * grid[1] * grid[2]
        if subdomain_map is not None:
            self.blocks, self.Q = None, int(Q)
        else:
            self.blocks = tuple(blocks)
            self.Q = blocks[0] * blocks[1] * blocks[2]
        if handle is not None:
            self.h = handle
        else:
            self.h = rbws_problem_create(grid, self.blocks, self.Q, f, device, subdomain_map, kappa_scale, neumann)

    @classmethod
    def field(cls, grid, kfx, kfy, kfz, f=None, device=0):
        """A face-field problem (rbws_problem_create_field)."""
        h, Q = rbws_problem_create_field(grid, kfx, kfy, kfz, f, device)
        obj = cls.__new__(cls)
        obj.grid, obj.blocks, obj.n, obj.Q, obj.h = tuple(grid), None, grid[0] * grid[1] * grid[2], Q, h
        return obj

    @classmethod
    def load(cls, path, device=0):
        """Wraps a problem restored by rbws_load."""
        h = rbws_load(path, device)
        n, Q, _ = rbws_problem_info(h)
        obj = cls.__new__(cls)
        obj.grid, obj.blocks, obj.n, obj.Q, obj.h = None, None, n, Q, h
        return obj

    def close(self):
        if self.h:
            rbws_problem_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
