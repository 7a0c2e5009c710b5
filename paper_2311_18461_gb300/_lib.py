"""ctypes binding of libstst.so: one Python function per C entry point, same names and argument order.

Vectors are torch tensors on the CUDA device (complex128, contiguous) or raw
device pointers (int); the binding passes their addresses. Negative status
codes raise StstError; non-negative ones are returned.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "libstst.so")

STST_PREC_FP64, STST_PREC_FP32, STST_PREC_BF16 = 0, 1, 2
STST_FORM_LS, STST_FORM_UW = 0, 1
STST_OK, STST_NOT_CONVERGED, STST_BREAKDOWN, STST_NOT_HPD, STST_TIMEOUT = 0, 1, 2, 3, 4
STST_ERR_ARG, STST_ERR_HANDLE, STST_ERR_OOM, STST_ERR_CUDA, STST_ERR_STATE = -1, -2, -3, -4, -5
STATUS = {0: "OK", 1: "NOT_CONVERGED", 2: "BREAKDOWN", 3: "NOT_HPD", 4: "TIMEOUT", -1: "ERR_ARG",
          -2: "ERR_HANDLE", -3: "ERR_OOM", -4: "ERR_CUDA", -5: "ERR_STATE"}


class StstError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = _strerror(status)
        if status == -4:
            detail += "; " + stst_last_cuda_error()
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")


_lib = None


def lib():
    """Load libstst.so (raises if it has not been built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise RuntimeError(f"CUDA library not built: {library_path} missing (run __graft_entry__.build())")
        L = ctypes.CDLL(library_path)
        P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        IP, DP = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
        sig = {
            "stst_create": [ctypes.POINTER(P), I, IP, IP, D, D, I, P],
            "stst_create2": [ctypes.POINTER(P), I, IP, IP, D, D, I, I, P],
            "stst_destroy": [P],
            "stst_sizes": [P, ctypes.POINTER(LL), IP],
            "stst_quadrature_points": [P, I, P],
            "stst_assemble_1d": [I, I, D, I, P, P, P, P, P, P, IP, P],
            "stst_set_potential": [P, I, P],
            "stst_set_geometry": [P, P, P],
            "stst_geometry_info": [P, IP, IP, DP],
            "stst_build_fd": [P],
            "stst_apply_sys": [P, P, P],
            "stst_apply_prec": [P, P, P],
            "stst_rhs": [P, P, P, P, P],
            "stst_rhs_noalloc": [P, P, P, P, P],
            "stst_rhs_lift": [P, P, P, P, P],
            "stst_pcg_solve": [P, P, P, D, I, IP, DP],
            "stst_ir_solve": [P, P, P, D, I, D, I, IP, IP, DP],
            "stst_profile": [P, I],
            "stst_batch_create": [ctypes.POINTER(P), I, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), P],
            "stst_batch_solve": [P, D, I, IP, DP, IP],
            "stst_batch_destroy": [P],
            "stst_plan_info": [P, IP, IP, DP],
            "stst_pcg_graph_info": [P, IP, IP],
            "stst_set_prec_operator": [P, I],
            "stst_profile_read": [P, I, ctypes.c_char_p, I, ctypes.POINTER(LL), DP],
            "stst_set_autotune": [I],
            "stst_set_time_solver": [I],
            "stst_set_fused_transforms": [I],
            "stst_fused_transforms_info": [P, IP],
            "stst_fused_transforms_split": [P, IP, IP],
            "stst_set_pencil": [I],
            "stst_pencil_info": [P, IP],
            "stst_set_tensor_products": [I],
            "stst_set_fused_matvec": [I],
            "stst_persistent_solve": [I, P, P, P, D, I, I, IP, IP, DP, P],
            "stst_tensor_products_info": [P, IP],
            "stst_time_solver_info": [P, I, IP, IP, IP],
            "stst_tile_info": [P, I, IP, IP, DP],
            "stst_ws_create": [ctypes.POINTER(P), I, IP, I, ctypes.c_ulonglong, P],
            "stst_ws_destroy": [P],
            "stst_ws_num_params": [P, ctypes.POINTER(LL)],
            "stst_ws_get_params": [P, P],
            "stst_ws_set_params": [P, P],
            "stst_ws_forward": [P, P, I, P, ctypes.c_float],
            "stst_ws_set_output_scale": [P, P],
            "stst_ws_grad": [P, P, P, P, P, I, P, DP],
            "stst_ws_train_step": [P, P, P, P, P, I, ctypes.c_float, DP],
            "stst_pod_basis": [P, I, LL, P, I, I, P, P],
            "stst_pod_project": [P, I, LL, P, I, P, P],
            "stst_pod_expand": [P, I, LL, P, I, ctypes.c_float, ctypes.c_float, P, P, P],
            "stst_ws_whiten": [P, I, I, P, P, LL, P],
            "stst_ws_target_scale": [P, I, I, P, P, P, P],
            "stst_ws_cascade": [P, P, P, P, I, I, P, P, P, P, P],
            "stst_pcg_solve_guarded": [P, P, P, D, I, IP, DP, IP],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = I
        L.stst_strerror.argtypes = [I]
        L.stst_strerror.restype = ctypes.c_char_p
        L.stst_last_cuda_error.argtypes = []
        L.stst_last_cuda_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _strerror(status):
    try:
        return lib().stst_strerror(status).decode()
    except Exception:
        return ""


def stst_strerror(status):
    return lib().stst_strerror(status).decode()


def stst_last_cuda_error():
    try:
        return lib().stst_last_cuda_error().decode()
    except Exception:
        return ""


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return t.data_ptr()


def _chk(status, where):
    if status < 0:
        raise StstError(status, where)
    return status


def _stream_ptr(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def stst_create(d, n_el, p, T=1.0, nu=1.0, prec_mode=STST_PREC_FP64, stream=None):
    h = ctypes.c_void_p()
    ne = (ctypes.c_int * (d + 1))(*n_el)
    pp = (ctypes.c_int * (d + 1))(*p)
    _chk(lib().stst_create(ctypes.byref(h), d, ne, pp, float(T), float(nu), int(prec_mode), _stream_ptr(stream)),
         "stst_create")
    return h


def stst_create2(d, n_el, p, T=1.0, nu=1.0, prec_mode=STST_PREC_FP64, formulation=STST_FORM_LS, stream=None):
    ne = (ctypes.c_int * (d + 1))(*[int(v) for v in n_el])
    pp = (ctypes.c_int * (d + 1))(*[int(v) for v in p])
    h = ctypes.c_void_p()
    _chk(lib().stst_create2(ctypes.byref(h), int(d), ne, pp, float(T), float(nu), int(prec_mode), int(formulation),
                            _stream_ptr(stream)), "stst_create2")
    return h


def stst_destroy(h):
    return _chk(lib().stst_destroy(h), "stst_destroy")


def stst_sizes(h, d):
    n_dof = ctypes.c_longlong()
    n = (ctypes.c_int * (d + 1))()
    _chk(lib().stst_sizes(h, ctypes.byref(n_dof), n), "stst_sizes")
    return n_dof.value, list(n)


def stst_quadrature_points(h, dir, pts):
    return _chk(lib().stst_quadrature_points(h, int(dir), _ptr(pts)), "stst_quadrature_points")


def stst_assemble_1d(p, n_el, length, bc, weight, M, L, J, K, K2, stream=None):
    n = ctypes.c_int()
    _chk(lib().stst_assemble_1d(int(p), int(n_el), float(length), int(bc), _ptr(weight), _ptr(M), _ptr(L), _ptr(J),
                                _ptr(K), _ptr(K2), ctypes.byref(n), _stream_ptr(stream)), "stst_assemble_1d")
    return n.value


def stst_set_potential(h, rank, v_qp):
    return _chk(lib().stst_set_potential(h, int(rank), _ptr(v_qp)), "stst_set_potential")


def stst_set_geometry(h, jac, hess):
    return _chk(lib().stst_set_geometry(h, _ptr(jac), _ptr(hess)), "stst_set_geometry")


def stst_geometry_info(h, with_scales=False):
    """(mapped, stored entries per row), and with_scales the list of P-hat's eigenvalue scales s_l."""
    m, w = ctypes.c_int(), ctypes.c_int()
    sc = (ctypes.c_double * 3)()
    _chk(lib().stst_geometry_info(h, ctypes.byref(m), ctypes.byref(w), sc), "stst_geometry_info")
    return (m.value, w.value, list(sc)) if with_scales else (m.value, w.value)


def stst_build_fd(h):
    return _chk(lib().stst_build_fd(h), "stst_build_fd")


def stst_apply_sys(h, x, y):
    return _chk(lib().stst_apply_sys(h, _ptr(x), _ptr(y)), "stst_apply_sys")


def stst_apply_prec(h, r, s):
    return _chk(lib().stst_apply_prec(h, _ptr(r), _ptr(s)), "stst_apply_prec")


def stst_rhs(h, f_qp, u0_qp, rhs, c0):
    return _chk(lib().stst_rhs(h, _ptr(f_qp), _ptr(u0_qp), _ptr(rhs), _ptr(c0)), "stst_rhs")


def stst_rhs_noalloc(h, f_qp, u0_qp, rhs, c0):
    return _chk(lib().stst_rhs_noalloc(h, _ptr(f_qp), _ptr(u0_qp), _ptr(rhs), _ptr(c0)), "stst_rhs_noalloc")


def stst_rhs_lift(h, f_qp, u_qp, rhs, xd):
    return _chk(lib().stst_rhs_lift(h, _ptr(f_qp), _ptr(u_qp), _ptr(rhs), _ptr(xd)), "stst_rhs_lift")


def stst_pcg_solve(h, rhs, x, tol, maxit):
    it = ctypes.c_int()
    rr = ctypes.c_double()
    s = _chk(lib().stst_pcg_solve(h, _ptr(rhs), _ptr(x), float(tol), int(maxit), ctypes.byref(it), ctypes.byref(rr)),
             "stst_pcg_solve")
    return s, it.value, rr.value


def stst_ir_solve(h, rhs, x, tol, maxit, inner_tol, inner_maxit):
    it = ctypes.c_int()
    outer = ctypes.c_int()
    rr = ctypes.c_double()
    s = _chk(lib().stst_ir_solve(h, _ptr(rhs), _ptr(x), float(tol), int(maxit), float(inner_tol), int(inner_maxit),
                                 ctypes.byref(it), ctypes.byref(outer), ctypes.byref(rr)), "stst_ir_solve")
    return s, it.value, outer.value, rr.value


def stst_profile(h, enable):
    return _chk(lib().stst_profile(h, int(enable)), "stst_profile")


def stst_batch_create(handles, rhs, x, stream=None):
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    rs = (ctypes.c_void_p * n)(*[_ptr(t) for t in rhs])
    xs = (ctypes.c_void_p * n)(*[_ptr(t) for t in x])
    b = ctypes.c_void_p()
    _chk(lib().stst_batch_create(ctypes.byref(b), n, hs, rs, xs, _stream_ptr(stream)), "stst_batch_create")
    return b


def stst_batch_solve(b, count, tol, maxit):
    it = (ctypes.c_int * count)()
    rr = (ctypes.c_double * count)()
    st = (ctypes.c_int * count)()
    s = _chk(lib().stst_batch_solve(b, float(tol), int(maxit), it, rr, st), "stst_batch_solve")
    return s, list(it), list(rr), list(st)


def stst_batch_destroy(b):
    return _chk(lib().stst_batch_destroy(b), "stst_batch_destroy")


def stst_plan_info(h):
    n = ctypes.c_int()
    a = ctypes.c_int()
    f = ctypes.c_double()
    _chk(lib().stst_plan_info(h, ctypes.byref(n), ctypes.byref(a), ctypes.byref(f)), "stst_plan_info")
    return n.value, a.value, f.value


def stst_set_prec_operator(h, op):
    return _chk(lib().stst_set_prec_operator(h, int(op)), "stst_set_prec_operator")


def stst_pcg_graph_info(h):
    k = ctypes.c_int()
    i = ctypes.c_int()
    _chk(lib().stst_pcg_graph_info(h, ctypes.byref(k), ctypes.byref(i)), "stst_pcg_graph_info")
    return k.value, i.value


def stst_profile_read(h):
    """All records as {kernel name: (launches, total ms)}."""
    out = {}
    idx = 0
    while True:
        name = ctypes.create_string_buffer(64)
        cnt = ctypes.c_longlong()
        ms = ctypes.c_double()
        if lib().stst_profile_read(h, idx, name, 64, ctypes.byref(cnt), ctypes.byref(ms)) != 0:
            break
        out[name.value.decode()] = (cnt.value, ms.value)
        idx += 1
    return out


def stst_set_autotune(mode):
    return _chk(lib().stst_set_autotune(int(mode)), "stst_set_autotune")


def stst_set_fused_transforms(mode):
    return _chk(lib().stst_set_fused_transforms(int(mode)), "stst_set_fused_transforms")


def stst_fused_transforms_info(h):
    f = ctypes.c_int()
    _chk(lib().stst_fused_transforms_info(h, ctypes.byref(f)), "stst_fused_transforms_info")
    return f.value


def stst_fused_transforms_split(h):
    f, b = ctypes.c_int(), ctypes.c_int()
    _chk(lib().stst_fused_transforms_split(h, ctypes.byref(f), ctypes.byref(b)), "stst_fused_transforms_split")
    return f.value, b.value


def stst_set_pencil(mode):
    return _chk(lib().stst_set_pencil(int(mode)), "stst_set_pencil")


def stst_pencil_info(h):
    f = ctypes.c_int()
    _chk(lib().stst_pencil_info(h, ctypes.byref(f)), "stst_pencil_info")
    return f.value


def stst_persistent_solve(handles, rhs, x, tol=1e-8, maxit=200, cluster_ctas=0, stream=None):
    """All problems in one launch, one thread-block cluster each; returns (status, iterations, relres,
    statuses): the largest per-problem status, then per-problem lists (errors raise StstError)."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    rs = (ctypes.c_void_p * n)(*[_ptr(t) for t in rhs])
    xs = (ctypes.c_void_p * n)(*[_ptr(t) for t in x])
    it = (ctypes.c_int * n)()
    stv = (ctypes.c_int * n)()
    rr = (ctypes.c_double * n)()
    s = _chk(lib().stst_persistent_solve(n, hs, rs, xs, float(tol), int(maxit), int(cluster_ctas), it, stv, rr,
                                         _stream_ptr(stream)), "stst_persistent_solve")
    return s, list(it), list(rr), list(stv)


def stst_set_fused_matvec(mode):
    return _chk(lib().stst_set_fused_matvec(int(mode)), "stst_set_fused_matvec")


def stst_set_tensor_products(mode):
    return _chk(lib().stst_set_tensor_products(int(mode)), "stst_set_tensor_products")


def stst_tensor_products_info(h):
    f = ctypes.c_int()
    _chk(lib().stst_tensor_products_info(h, ctypes.byref(f)), "stst_tensor_products_info")
    return f.value


def stst_set_time_solver(mode):
    return _chk(lib().stst_set_time_solver(int(mode)), "stst_set_time_solver")


def stst_time_solver_info(h, precision):
    S = ctypes.c_int()
    L = ctypes.c_int()
    used = ctypes.c_int()
    _chk(lib().stst_time_solver_info(h, int(precision), ctypes.byref(S), ctypes.byref(L), ctypes.byref(used)),
         "stst_time_solver_info")
    return S.value, L.value, used.value


def stst_tile_info(h, dir):
    c = ctypes.c_int()
    r = ctypes.c_int()
    us = ctypes.c_double()
    _chk(lib().stst_tile_info(h, int(dir), ctypes.byref(c), ctypes.byref(r), ctypes.byref(us)), "stst_tile_info")
    return c.value, r.value, us.value


def stst_ws_create(sizes, max_batch, seed=0, stream=None):
    """Network sizes[0] -> ... -> sizes[-1] (tanh between layers); returns the handle."""
    n_layers = len(sizes) - 1
    arr = (ctypes.c_int * len(sizes))(*[int(v) for v in sizes])
    w = ctypes.c_void_p()
    _chk(lib().stst_ws_create(ctypes.byref(w), n_layers, arr, int(max_batch), int(seed), _stream_ptr(stream)),
         "stst_ws_create")
    return w


def stst_ws_destroy(w):
    return _chk(lib().stst_ws_destroy(w), "stst_ws_destroy")


def stst_ws_num_params(w):
    n = ctypes.c_longlong()
    _chk(lib().stst_ws_num_params(w, ctypes.byref(n)), "stst_ws_num_params")
    return n.value


def stst_ws_get_params(w, params):
    return _chk(lib().stst_ws_get_params(w, _ptr(params)), "stst_ws_get_params")


def stst_ws_set_params(w, params):
    return _chk(lib().stst_ws_set_params(w, _ptr(params)), "stst_ws_set_params")


def stst_ws_forward(w, X, batch, Y, beta=0.0):
    return _chk(lib().stst_ws_forward(w, _ptr(X), int(batch), _ptr(Y), float(beta)), "stst_ws_forward")


def stst_ws_set_output_scale(w, scale):
    return _chk(lib().stst_ws_set_output_scale(w, _ptr(scale)), "stst_ws_set_output_scale")


def stst_ws_grad(w, X, T, weight, idx, batch, grad, want_loss=True):
    loss = ctypes.c_double()
    _chk(lib().stst_ws_grad(w, _ptr(X), _ptr(T), _ptr(weight), _ptr(idx), int(batch), _ptr(grad),
                            ctypes.byref(loss) if want_loss else None), "stst_ws_grad")
    return loss.value if want_loss else None


def stst_ws_train_step(w, X, T, weight, idx, batch, lr, want_loss=False):
    loss = ctypes.c_double()
    _chk(lib().stst_ws_train_step(w, _ptr(X), _ptr(T), _ptr(weight), _ptr(idx), int(batch), float(lr),
                                  ctypes.byref(loss) if want_loss else None), "stst_ws_train_step")
    return loss.value if want_loss else None


def stst_pod_basis(Y, n, m, Omega, K, power_its, Q, stream=None):
    return _chk(lib().stst_pod_basis(_ptr(Y), int(n), int(m), _ptr(Omega), int(K), int(power_its), _ptr(Q),
                                     _stream_ptr(stream)), "stst_pod_basis")


def stst_pod_project(Y, n, m, Q, K, C, stream=None):
    return _chk(lib().stst_pod_project(_ptr(Y), int(n), int(m), _ptr(Q), int(K), _ptr(C), _stream_ptr(stream)),
                "stst_pod_project")


def stst_ws_whiten(F, n, K, Fw, Q=None, m=0, stream=None):
    return _chk(lib().stst_ws_whiten(_ptr(F), int(n), int(K), _ptr(Fw), _ptr(Q), int(m), _stream_ptr(stream)),
                "stst_ws_whiten")


def stst_ws_target_scale(T, n, K, Ts, so, w, stream=None):
    return _chk(lib().stst_ws_target_scale(_ptr(T), int(n), int(K), _ptr(Ts), _ptr(so), _ptr(w),
                                           _stream_ptr(stream)), "stst_ws_target_scale")


def stst_ws_cascade(T0, Y, scale_prev, resid, n, K, scale, targets, so, out_scale, stream=None):
    return _chk(lib().stst_ws_cascade(_ptr(T0), _ptr(Y), _ptr(scale_prev), _ptr(resid), int(n), int(K), _ptr(scale),
                                      _ptr(targets), _ptr(so), _ptr(out_scale), _stream_ptr(stream)),
                "stst_ws_cascade")


def stst_pod_expand(Q, K, m, C, n, alpha, beta, phase, X, stream=None):
    return _chk(lib().stst_pod_expand(_ptr(Q), int(K), int(m), _ptr(C), int(n), float(alpha), float(beta),
                                      _ptr(phase), _ptr(X), _stream_ptr(stream)), "stst_pod_expand")


def stst_pcg_solve_guarded(h, rhs, x, tol, maxit):
    it = ctypes.c_int()
    rr = ctypes.c_double()
    used = ctypes.c_int()
    s = _chk(lib().stst_pcg_solve_guarded(h, _ptr(rhs), _ptr(x), float(tol), int(maxit), ctypes.byref(it),
                                          ctypes.byref(rr), ctypes.byref(used)), "stst_pcg_solve_guarded")
    return s, it.value, rr.value, used.value


class Problem:
    """Owns a handle; convenience around the C calls (allocation of device vectors via torch)."""

    def __init__(self, d, n_el, p, T=1.0, nu=1.0, prec_mode=STST_PREC_FP64, stream=None, device="cuda",
                 formulation=STST_FORM_LS):
        import torch
        self.torch = torch
        self.d = d
        if isinstance(p, int):
            p = [p] * (d + 1)
        self.p = list(p)
        self.n_el = list(n_el)
        self.device = device
        self.formulation = formulation
        self.h = stst_create2(d, n_el, p, T, nu, prec_mode, formulation, stream)
        self.n_dof, self.n = stst_sizes(self.h, d)
        self.N_s = self.n_dof // self.n[0]

    def close(self):
        if self.h is not None:
            stst_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self):
        return self.torch.zeros(self.n_dof, dtype=self.torch.complex128, device=self.device)

    def quad_points(self, l):
        Q = self.n_el[l] * (self.p[l] + 2)
        t = self.torch.empty(Q, dtype=self.torch.float64, device=self.device)
        stst_quadrature_points(self.h, l, t)
        return t

    def set_potential(self, v_qp, rank):
        return stst_set_potential(self.h, rank, v_qp)

    def set_geometry(self, jac, hess):
        """Mapped domain: the map's first and second derivatives at the spatial quadrature grid (device
        float64 tensors, shapes (N_q, d, d) and (N_q, d, d, d)); None removes it."""
        return stst_set_geometry(self.h, jac, hess)

    def set_prec_operator(self, op):
        """0: the paper's P-hat; 1: the potential-aware P_V (rebuild with build_fd)."""
        return stst_set_prec_operator(self.h, op)

    def build_fd(self):
        return stst_build_fd(self.h)

    def apply_sys(self, x, y=None):
        y = self.vec() if y is None else y
        stst_apply_sys(self.h, x, y)
        return y

    def apply_prec(self, r, s=None):
        s = self.vec() if s is None else s
        stst_apply_prec(self.h, r, s)
        return s

    def rhs(self, f_qp=None, u0_qp=None, want_c0=False):
        b = self.vec()
        c0 = self.torch.zeros(self.N_s, dtype=self.torch.complex128, device=self.device) if want_c0 else None
        stst_rhs(self.h, f_qp, u0_qp, b, c0)
        return (b, c0) if want_c0 else b

    def rhs_lift(self, f_qp, u_qp, want_xd=False):
        """Right-hand side with the Dirichlet and initial values of u_qp imposed (stst_rhs_lift); with
        want_xd also the lifting's coefficients on the full basis (prod_l (n_el_l + p_l), time fastest)."""
        b = self.vec()
        xd = None
        if want_xd:
            m_tot = 1
            for l in range(self.d + 1):
                m_tot *= self.n_el[l] + self.p[l]
            xd = self.torch.zeros(m_tot, dtype=self.torch.complex128, device=self.device)
        stst_rhs_lift(self.h, f_qp, u_qp, b, xd)
        return (b, xd) if want_xd else b

    def pcg(self, rhs, x=None, tol=1e-8, maxit=200):
        x = self.vec() if x is None else x
        s, it, rr = stst_pcg_solve(self.h, rhs, x, tol, maxit)
        return x, s, it, rr

    def pcg_guarded(self, rhs, x, tol=1e-8, maxit=200):
        """PCG from the guess in x (replaced by 0 on the device when it is worse than 0)."""
        s, it, rr, used = stst_pcg_solve_guarded(self.h, rhs, x, tol, maxit)
        return x, s, it, rr, used

    def ir(self, rhs, x=None, tol=1e-8, maxit=20, inner_tol=1e-4, inner_maxit=50):
        x = self.vec() if x is None else x
        s, it, outer, rr = stst_ir_solve(self.h, rhs, x, tol, maxit, inner_tol, inner_maxit)
        return x, s, it, outer, rr
