"""GB300 FBIM: Python binding of the C ABI in include/fbim.h.

Argument marshalling only: every step of the method runs in the CUDA library
``libfbim.so`` built in-tree by ``paper_1709_01480_gb300.build``.  There is no
CPU fallback; importing this package without the built library raises.

Arrays are torch tensors on the handle's device (float64, contiguous) or raw
device addresses (int).  Host-side inputs of ``FBIM(...)`` are numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfbim.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_1709_01480_gb300.build` "
        "(there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

FBIM_FP64, FBIM_FP32 = 0, 1
STATUS = {0: "FBIM_OK", 1: "FBIM_ERR_INVALID_ARG", 2: "FBIM_ERR_CUDA", 3: "FBIM_ERR_OOM",
          4: "FBIM_ERR_OVERLAP", 5: "FBIM_ERR_NONFINITE", 6: "FBIM_ERR_NOT_CONVERGED",
          7: "FBIM_ERR_TIMEOUT", 8: "FBIM_ERR_SETUP"}

# every symbol declared in include/fbim.h
EXPORTS = [
    "fbim_default_params", "fbim_choose_ewald", "fbim_setup", "fbim_update_config",
    "fbim_apply_stokeslet", "fbim_apply_real", "fbim_apply_wave", "fbim_get_info",
    "fbim_destroy", "fbim_last_error", "fbim_host_expint_e1", "fbim_host_alpert_rule",
    "fbim_set_timing", "fbim_stage_times", "fbim_mobility_solve", "fbim_brownian_slip",
    "fbim_philox_normals", "fbim_apply_real_noalloc", "fbim_rfd_step",
    "fbim_batch_create", "fbim_batch_solve", "fbim_batch_get_info", "fbim_batch_destroy",
    "fbim_batch_last_error", "fbim_batch_slip", "fbim_update_config_displaced", "fbim_host_lanczos_sqrt",
    "fbim_second_kind_solve", "fbim_second_kind_apply", "fbim_second_kind_rhs",
    "fbim_mlp_param_count", "fbim_mlp_create", "fbim_mlp_destroy", "fbim_mlp_last_error",
    "fbim_mlp_set_params", "fbim_mlp_get_params", "fbim_mlp_set_normalization", "fbim_mlp_forward",
    "fbim_mlp_gradient", "fbim_mlp_adam_step", "fbim_mlp_launches", "fbim_coarse_pairs",
    "fbim_coarse_enable", "fbim_coarse_stats", "fbim_apply_stokeslet_fp64",
    "fbim_set_residual_audit", "fbim_residual_audit", "fbim_precondition", "fbim_bd_step",
    "fbim_bd_update",
]
STAGES = ["gather", "spread", "fft_fwd", "scale", "fft_inv", "pairs", "interp", "finish"]


class FbimError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("alpert_order", ctypes.c_int), ("grid", ctypes.c_int),
                ("support", ctypes.c_int), ("eta", ctypes.c_double), ("stream", ctypes.c_void_p),
                ("device", ctypes.c_int), ("restart", ctypes.c_int), ("autotune", ctypes.c_int),
                ("grid_tune", ctypes.c_int), ("split_tune", ctypes.c_int), ("fp32_support", ctypes.c_int),
                ("tensor_cores", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n_b", ctypes.c_int), ("n_p", ctypes.c_int), ("n_nodes", ctypes.c_int),
                ("L", ctypes.c_double), ("xi", ctypes.c_double), ("r_c", ctypes.c_double),
                ("tol", ctypes.c_double), ("n_box", ctypes.c_int), ("grid", ctypes.c_int),
                ("support", ctypes.c_int), ("eta_s", ctypes.c_double), ("h", ctypes.c_double),
                ("alpert_order", ctypes.c_int), ("alpert_nodes", ctypes.c_int),
                ("alpert_window", ctypes.c_int), ("alpert_band", ctypes.c_int), ("precision", ctypes.c_int),
                ("tile", ctypes.c_int), ("pair_entries", ctypes.c_longlong),
                ("wave_variant", ctypes.c_int), ("variant_ms", ctypes.c_double * 2),
                ("launches", ctypes.c_longlong), ("grid_min", ctypes.c_int), ("grid_tune_ms", ctypes.c_double),
                ("split_candidates", ctypes.c_int), ("split_cost_ms", ctypes.c_double),
                ("interp_variant", ctypes.c_int), ("interp_ms", ctypes.c_double * 2),
                ("support32", ctypes.c_int), ("eta_s32", ctypes.c_double), ("fp64_fft", ctypes.c_int),
                ("coarse_fallbacks", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["variant_ms"] = list(self.variant_ms)
        d["interp_ms"] = list(self.interp_ms)
        return d


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_handles", ctypes.c_int), ("n_systems", ctypes.c_int), ("n_unknowns", ctypes.c_longlong),
                ("restart", ctypes.c_int), ("branches", ctypes.c_int), ("graph_kernels", ctypes.c_longlong * 7),
                ("launches", ctypes.c_longlong), ("graph_launches", ctypes.c_longlong)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["graph_kernels"] = list(self.graph_kernels)
        return d




_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)

_lib.fbim_default_params.argtypes = [ctypes.POINTER(Params)]
_lib.fbim_choose_ewald.argtypes = [_D, _D, _D, _D, _IP, _DP, _DP, _IP, _IP, _DP]
_lib.fbim_setup.argtypes = [ctypes.POINTER(_P), _I, _I, _DP, _DP, _D, _D, _D, _D, ctypes.POINTER(Params)]
_lib.fbim_update_config.argtypes = [_P, _P]
_lib.fbim_update_config_displaced.argtypes = [_P, _P, _D, _P]
_lib.fbim_second_kind_solve.argtypes = [_P, _P, _D, _I, _P, _P, _IP, _DP]
_lib.fbim_second_kind_apply.argtypes = [_P, _P, _P]
_lib.fbim_second_kind_rhs.argtypes = [_P, _P, _P]
_lib.fbim_apply_stokeslet.argtypes = [_P, _P, _P]
_lib.fbim_apply_real.argtypes = [_P, _P, _P]
_lib.fbim_apply_wave.argtypes = [_P, _P, _P]
_lib.fbim_apply_real_noalloc.argtypes = [_P, _P, _P]
_lib.fbim_apply_stokeslet_fp64.argtypes = [_P, _P, _P]
_lib.fbim_rfd_step.argtypes = [_P, _P, _D, _D, _D, ctypes.c_uint64, ctypes.c_uint64, _P, _P, _P, _D, _I, _P, _IP]
_lib.fbim_get_info.argtypes = [_P, ctypes.POINTER(Info)]
_lib.fbim_destroy.argtypes = [_P]
_lib.fbim_destroy.restype = None
_lib.fbim_last_error.argtypes = [_P]
_lib.fbim_last_error.restype = ctypes.c_char_p
_lib.fbim_host_expint_e1.argtypes = [_D]
_lib.fbim_host_expint_e1.restype = _D
_lib.fbim_host_alpert_rule.argtypes = [_I, _DP, _DP, _IP]
_lib.fbim_host_lanczos_sqrt.argtypes = [_DP, _DP, _I, _D, _DP]
_lib.fbim_set_timing.argtypes = [_P, _I]
_lib.fbim_mobility_solve.argtypes = [_P, _P, _P, _D, _I, _P, _P, _IP, _DP]
_lib.fbim_brownian_slip.argtypes = [_P, ctypes.c_uint64, ctypes.c_uint64, _D, _D, _P, _P, _D, _I, _P, _IP]
_lib.fbim_philox_normals.argtypes = [_P, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_size_t, _P]
_lib.fbim_stage_times.argtypes = [_P, _DP, ctypes.POINTER(ctypes.c_longlong), _I]
_lib.fbim_batch_create.argtypes = [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), _IP]
_lib.fbim_batch_solve.argtypes = [_P, _P, _P, _D, _I, _P, _IP, _DP]
_lib.fbim_batch_get_info.argtypes = [_P, ctypes.POINTER(BatchInfo)]
_lib.fbim_batch_slip.argtypes = [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint64, _D, _D, _D, _I, _P, _IP]
_lib.fbim_batch_destroy.argtypes = [_P]
_lib.fbim_batch_destroy.restype = None
_lib.fbim_batch_last_error.argtypes = [_P]
_lib.fbim_batch_last_error.restype = ctypes.c_char_p
_FP = ctypes.POINTER(ctypes.c_float)
_lib.fbim_mlp_param_count.restype = _I
_lib.fbim_mlp_create.argtypes = [ctypes.POINTER(_P), _I, _P, _I]
_lib.fbim_mlp_destroy.argtypes = [_P]
_lib.fbim_mlp_destroy.restype = None
_lib.fbim_mlp_last_error.argtypes = [_P]
_lib.fbim_mlp_last_error.restype = ctypes.c_char_p
_lib.fbim_mlp_set_params.argtypes = [_P, _FP]
_lib.fbim_mlp_get_params.argtypes = [_P, _FP]
_lib.fbim_mlp_set_normalization.argtypes = [_P, _FP, _FP, _FP]
_lib.fbim_mlp_forward.argtypes = [_P, _I, _P, _P]
_lib.fbim_mlp_gradient.argtypes = [_P, _I, _P, _P, _P, _DP]
_lib.fbim_mlp_adam_step.argtypes = [_P, _I, _P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, _DP]
_lib.fbim_mlp_launches.argtypes = [_P]
_lib.fbim_mlp_launches.restype = ctypes.c_longlong
_lib.fbim_coarse_pairs.argtypes = [_P, _D, _I, _P, _P, _IP]
_lib.fbim_coarse_enable.argtypes = [_P, _P, _D]
_lib.fbim_coarse_stats.argtypes = [_P, _IP, _IP]
_lib.fbim_set_residual_audit.argtypes = [_P, _I]
_lib.fbim_precondition.argtypes = [_P, _P, _P]
_lib.fbim_bd_step.argtypes = [_P, _I, _P, _D, _D, _D, ctypes.c_uint64, ctypes.c_uint64, _P, _P, _P, _D, _D, _I, _P,
                              _I, _P, _IP]
_lib.fbim_residual_audit.argtypes = [_P, _I, _DP, _DP, _IP]
_lib.fbim_bd_update.argtypes = [_P, ctypes.c_size_t, _D, _D, _P, _P, _P, _P]


def lib():
    return _lib


def bd_update(Q, U, dt, c=0.0, Up=None, Um=None, stream=None):
    """Q += dt U + c (Up - Um) (or Q += dt U without Up, Um) on the device: the position
    update of the Brownian dynamics steps for velocities from a batched solve."""
    import torch
    ts = [t for t in (Q, U, Up, Um) if t is not None]
    n = Q.numel()
    for t in ts:
        if t.dtype != torch.float64 or not t.is_contiguous() or not t.is_cuda or t.numel() != n \
                or t.device != Q.device:
            raise ValueError("bd_update: contiguous float64 CUDA tensors of equal size on one device")
    if (Up is None) != (Um is None):
        raise ValueError("bd_update: give both Up and Um or neither")
    if stream is None:
        stream = torch.cuda.current_stream(Q.device)
    opt = lambda t: None if t is None else _ptr(t)
    with torch.cuda.device(Q.device):
        _check(_lib.fbim_bd_update(ctypes.c_void_p(stream.cuda_stream), n, float(dt), float(c), _ptr(U), opt(Up),
                                   opt(Um), _ptr(Q)))


def _check(status, handle=None):
    if status != 0:
        msg = _lib.fbim_last_error(handle)
        raise FbimError(status, msg.decode() if msg else "")


def _ptr(t):
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def host_expint_e1(z: float) -> float:
    return _lib.fbim_host_expint_e1(float(z))


def host_alpert_rule(order: int = 4):
    v = np.zeros(order - 1)
    w = np.zeros(order - 1)
    a = ctypes.c_int(0)
    _check(_lib.fbim_host_alpert_rule(order, _dptr(v), _dptr(w), ctypes.byref(a)))
    return v, w, a.value


def host_lanczos_sqrt(alpha, beta, wnorm=1.0):
    """wnorm sqrt(T) e_1 for the symmetric tridiagonal T = tridiag(beta, alpha, beta) (host routine)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    if b.size + 1 != a.size or a.size < 1:
        raise ValueError("beta needs len(alpha) - 1 entries")
    out = np.zeros(a.size)
    bb = b if b.size else np.zeros(1)
    _check(_lib.fbim_host_lanczos_sqrt(_dptr(a), _dptr(bb), a.size, float(wnorm), _dptr(out)))
    return out


def choose_ewald(L, r_c, tol, xi=0.0):
    nb, M, P = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rc, x, es = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.fbim_choose_ewald(L, r_c, tol, xi, ctypes.byref(nb), ctypes.byref(rc), ctypes.byref(x),
                                  ctypes.byref(M), ctypes.byref(P), ctypes.byref(es)))
    return dict(n_box=nb.value, r_c=rc.value, xi=x.value, grid=M.value, support=P.value, eta_s=es.value)


class FBIM:
    """One suspension of rigid bodies of a single shape in a periodic box."""

    def __init__(self, ref_nodes, Q, L, *, tol=1e-8, r_c=0.0, xi=0.0, precision="fp64", order=4,
                 grid=0, support=0, eta=1.0, stream=None, device=0, restart=60, wave="auto", grid_tune=True,
                 split_tune=False, fp32_support=0, tensor_cores=True):
        ref = np.ascontiguousarray(ref_nodes, dtype=np.float64)
        Qh = np.ascontiguousarray(Q, dtype=np.float64)
        self.n_p = ref.shape[0]
        self.n_b = Qh.shape[0]
        p = Params()
        _lib.fbim_default_params(ctypes.byref(p))
        p.precision = FBIM_FP32 if precision == "fp32" else FBIM_FP64
        p.alpert_order = order
        p.grid = grid
        p.support = support
        p.eta = eta
        p.device = device
        p.restart = restart
        p.autotune = {"auto": 1, "tile": 0, "warp": 2}[wave]
        p.grid_tune = 1 if grid_tune else 0
        p.split_tune = 1 if split_tune else 0
        p.fp32_support = fp32_support
        p.tensor_cores = 1 if tensor_cores else 0
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        p.stream = stream
        self._stream = stream
        h = ctypes.c_void_p()
        _check(_lib.fbim_setup(ctypes.byref(h), self.n_b, self.n_p, _dptr(ref), _dptr(Qh), float(L),
                               float(r_c), float(xi), float(tol), ctypes.byref(p)))
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    @property
    def info(self):
        i = Info()
        _check(_lib.fbim_get_info(self._h, ctypes.byref(i)), self._h)
        return i.as_dict()

    @property
    def n(self):
        return self.n_b * self.n_p

    def _out(self, like, shape):
        import torch
        return torch.empty(shape, dtype=torch.float64, device=like.device)

    def _vec(self, t, numel, name):
        """The library receives bare pointers: check that t is a contiguous float64 CUDA
        tensor of numel entries on the handle's device (raw integer addresses pass as
        given).  Returns t."""
        if t is None or isinstance(t, int):
            return t
        import torch
        if (not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous()
                or t.device.type != "cuda" or t.device.index not in (None, self.device)
                or (numel is not None and t.numel() != numel)):
            what = f"{t.dtype} {tuple(t.shape)} on {t.device}" if isinstance(t, torch.Tensor) else type(t).__name__
            raise FbimError(1, f"{name}: expected a contiguous float64 tensor of {numel} entries on "
                               f"cuda:{self.device}, got {what}")
        return t

    def apply_stokeslet(self, mu, out=None):
        self._vec(mu, 2 * self.n, "mu")
        self._vec(out, 2 * self.n, "out")
        v = out if out is not None else self._out(mu, (self.n, 2))
        _check(_lib.fbim_apply_stokeslet(self._h, _ptr(mu), _ptr(v)), self._h)
        return v

    def apply_stokeslet_fp64(self, mu, out=None):
        """The FP64 operator of the refinement residuals (FP64 whatever the handle's precision)."""
        self._vec(mu, 2 * self.n, "mu")
        self._vec(out, 2 * self.n, "out")
        v = out if out is not None else self._out(mu, (self.n, 2))
        _check(_lib.fbim_apply_stokeslet_fp64(self._h, _ptr(mu), _ptr(v)), self._h)
        return v

    def apply_real(self, mu, out=None):
        self._vec(mu, 2 * self.n, "mu")
        self._vec(out, 2 * self.n, "out")
        v = out if out is not None else self._out(mu, (self.n, 2))
        _check(_lib.fbim_apply_real(self._h, _ptr(mu), _ptr(v)), self._h)
        return v

    def apply_real_noalloc(self, mu, out):
        """Real-space operator into the caller's ``out``; allocates no device memory.

        ``mu`` and ``out`` must be float64, contiguous, shaped (n, 2) and on the
        handle's device: the library receives bare pointers and cannot check them.
        """
        for name, t in (("mu", mu), ("out", out)):
            if isinstance(t, int):
                continue
            import torch
            if (t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape) != (self.n, 2)
                    or t.device.type != "cuda" or t.device.index not in (None, self.device)):
                raise FbimError(1, f"apply_real_noalloc: {name} must be a contiguous float64 ({self.n}, 2) "
                                   f"tensor on cuda:{self.device}, got {t.dtype} {tuple(t.shape)} on {t.device}")
        _check(_lib.fbim_apply_real_noalloc(self._h, _ptr(mu), _ptr(out)), self._h)
        return out

    def apply_wave(self, mu, out=None):
        self._vec(mu, 2 * self.n, "mu")
        self._vec(out, 2 * self.n, "out")
        v = out if out is not None else self._out(mu, (self.n, 2))
        _check(_lib.fbim_apply_wave(self._h, _ptr(mu), _ptr(v)), self._h)
        return v

    def mobility_solve(self, F, slip=None, tol=1e-6, max_iter=500, want_mu=False, check=True):
        """Solve the saddle system; returns (U [n_b, 3], mu or None, iterations, relative residual)."""
        import torch
        self._vec(F, 3 * self.n_b, "F")
        self._vec(slip, 2 * self.n, "slip")
        U = torch.empty((self.n_b, 3), dtype=torch.float64, device=F.device)
        mu = torch.empty((self.n, 2), dtype=torch.float64, device=F.device) if want_mu else None
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        st = _lib.fbim_mobility_solve(self._h, _ptr(F), None if slip is None else _ptr(slip), float(tol),
                                      int(max_iter), _ptr(U), None if mu is None else _ptr(mu),
                                      ctypes.byref(it), ctypes.byref(res))
        if check or st not in (0, 6):
            _check(st, self._h)
        return U, mu, it.value, res.value

    def brownian_slip(self, kT=1.0, dt=1.0, W_r=None, Z_w=None, seed=0, counter=0, tol=1e-6, max_iter=200):
        """Random slip [N, 2]; returns (slip, Lanczos iterations)."""
        import torch
        self._vec(W_r, 2 * self.n, "W_r")
        self._vec(Z_w, None, "Z_w")
        dev = W_r.device if W_r is not None else torch.device("cuda", self.device)
        out = torch.empty((self.n, 2), dtype=torch.float64, device=dev)
        it = ctypes.c_int(0)
        _check(_lib.fbim_brownian_slip(self._h, int(seed), int(counter), float(kT), float(dt),
                                       None if W_r is None else _ptr(W_r), None if Z_w is None else _ptr(Z_w),
                                       float(tol), int(max_iter), _ptr(out), ctypes.byref(it)), self._h)
        return out, it.value

    def rfd_step(self, F, Q, dt, kT=1.0, delta=1e-3, seed=0, step=0, W_r=None, Z_w=None, W_t=None, tol=1e-6,
                 max_iter=500):
        """One EM-RFD step; Q (device [n_b, 3]) is updated in place.  Returns the GMRES iterations."""
        for t, k, name in ((F, 3 * self.n_b, "F"), (Q, 3 * self.n_b, "Q"), (W_r, 2 * self.n, "W_r"),
                           (Z_w, None, "Z_w"), (W_t, 3 * self.n_b, "W_t")):
            self._vec(t, k, name)
        it = ctypes.c_int(0)
        opt = lambda t: None if t is None else _ptr(t)
        _check(_lib.fbim_rfd_step(self._h, _ptr(F), float(dt), float(kT), float(delta), int(seed), int(step),
                                  opt(W_r), opt(Z_w), opt(W_t), float(tol), int(max_iter), _ptr(Q),
                                  ctypes.byref(it)), self._h)
        return it.value

    def bd_step(self, F, Q, dt, kT=1.0, delta=1e-3, scheme="em", seed=0, step=0, W_r=None, Z_w=None, W_t=None,
                tol=1e-6, tol_rfd=None, NF=None, have_prev=False, max_iter=500):
        """One Brownian dynamics step (scheme "em", "ab2" or "em_no_rfd", the biased scheme
        without the stochastic drift); Q is updated in place.  For "ab2", NF (device [n_b, 3])
        carries N F between steps (read when have_prev, written always).  Returns the GMRES
        iterations of the step's solves."""
        for t, k, name in ((F, 3 * self.n_b, "F"), (Q, 3 * self.n_b, "Q"), (W_r, 2 * self.n, "W_r"),
                           (Z_w, None, "Z_w"), (W_t, 3 * self.n_b, "W_t"), (NF, 3 * self.n_b, "NF")):
            self._vec(t, k, name)
        it = ctypes.c_int(0)
        opt = lambda t: None if t is None else _ptr(t)
        sch = {"em": 0, "ab2": 1, "em_no_rfd": 2}[scheme]
        _check(_lib.fbim_bd_step(self._h, sch, _ptr(F), float(dt), float(kT), float(delta), int(seed), int(step),
                                 opt(W_r), opt(Z_w), opt(W_t), float(tol), float(tol if tol_rfd is None else tol_rfd),
                                 int(max_iter), opt(NF), 1 if have_prev else 0, _ptr(Q), ctypes.byref(it)), self._h)
        return it.value

    def philox_normals(self, n, seed=0, stream=0, counter=0, out=None):
        import torch
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=torch.device("cuda", self.device))
        elif out.numel() < n or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out: contiguous float64 with n entries")
        _check(_lib.fbim_philox_normals(self._h, int(seed), int(stream), int(counter), int(n), _ptr(out)), self._h)
        return out

    def set_timing(self, on: bool):
        _check(_lib.fbim_set_timing(self._h, 1 if on else 0), self._h)

    def stage_times(self):
        ms = np.zeros(len(STAGES))
        calls = (ctypes.c_longlong * len(STAGES))()
        _check(_lib.fbim_stage_times(self._h, _dptr(ms), calls, len(STAGES)), self._h)
        return {k: (float(ms[i]), int(calls[i])) for i, k in enumerate(STAGES)}

    def coarse_pairs(self, g_c, max_pairs=None):
        """Close pairs (gap < g_c) of the current configuration: (pairs int32 [n, 2], features float64 [n, 6])."""
        import torch
        n = ctypes.c_int(0)
        _check(_lib.fbim_coarse_pairs(self._h, float(g_c), 0, None, None, ctypes.byref(n)), self._h)
        cap = n.value if max_pairs is None else min(int(max_pairs), n.value)
        dev = torch.device("cuda", self.device)
        pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=dev)
        feats = torch.empty((max(cap, 1), 6), dtype=torch.float64, device=dev)
        _check(_lib.fbim_coarse_pairs(self._h, float(g_c), cap, _ptr(pairs), _ptr(feats), ctypes.byref(n)), self._h)
        return pairs[:cap], feats[:cap]

    def coarse_enable(self, model, g_c):
        """Turn the learned coarse level on with ``model`` (an MLP), or off with None."""
        self._coarse_model = model  # keeps the network alive while the handle uses it
        _check(_lib.fbim_coarse_enable(self._h, None if model is None else model._m, float(g_c)), self._h)

    def coarse_stats(self):
        n, r = ctypes.c_int(0), ctypes.c_int(0)
        _check(_lib.fbim_coarse_stats(self._h, ctypes.byref(n), ctypes.byref(r)), self._h)
        return n.value, r.value

    def precondition(self, r, out=None):
        """One application of the block-diagonal preconditioner to r = [r_mu; r_U] (2N + 3 n_b)."""
        o = out if out is not None else self._out(r, (2 * self.n + 3 * self.n_b,))
        _check(_lib.fbim_precondition(self._h, _ptr(r), _ptr(o)), self._h)
        return o

    def set_residual_audit(self, on: bool):
        """Make every mobility solve also measure its true FP64 residual (clears the records)."""
        _check(_lib.fbim_set_residual_audit(self._h, 1 if on else 0), self._h)

    def residual_audit(self, n=64):
        """The last audit records, oldest first: (reported residuals, measured residuals)."""
        rep = np.zeros(n)
        mea = np.zeros(n)
        k = ctypes.c_int(0)
        _check(_lib.fbim_residual_audit(self._h, int(n), _dptr(rep), _dptr(mea), ctypes.byref(k)), self._h)
        return rep[:k.value].tolist(), mea[:k.value].tolist()

    def update_config(self, Q_dev):
        _check(_lib.fbim_update_config(self._h, _ptr(Q_dev)), self._h)

    def second_kind_solve(self, F, tol=1e-12, max_iter=500, want_phi=False, check=True):
        """Second-kind reference solve (App. B): returns (U [n_b, 3], phi or None, iterations,
        measured relative residual)."""
        import torch
        U = torch.empty((self.n_b, 3), dtype=torch.float64, device=F.device)
        phi = torch.empty((self.n, 2), dtype=torch.float64, device=F.device) if want_phi else None
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        st = _lib.fbim_second_kind_solve(self._h, _ptr(F), float(tol), int(max_iter), _ptr(U),
                                         None if phi is None else _ptr(phi), ctypes.byref(it), ctypes.byref(res))
        if check or st not in (0, 6):
            _check(st, self._h)
        return U, phi, it.value, res.value

    def second_kind_apply(self, x):
        """y = A x of the second-kind system, x = [phi (2N); U (3 n_b)] flat float64 (device)."""
        import torch
        y = torch.empty_like(x)
        _check(_lib.fbim_second_kind_apply(self._h, _ptr(x), _ptr(y)), self._h)
        return y

    def second_kind_rhs(self, F):
        """b = [C F; 0] of the second-kind system for F [n_b, 3] (device)."""
        import torch
        b = torch.empty(2 * self.n + 3 * self.n_b, dtype=torch.float64, device=F.device)
        _check(_lib.fbim_second_kind_rhs(self._h, _ptr(F), _ptr(b)), self._h)
        return b

    def update_config_displaced(self, Q_dev, a, W_dev):
        """Move the bodies to Q + a W (device [n_b, 3] tensors)."""
        _check(_lib.fbim_update_config_displaced(self._h, _ptr(Q_dev), float(a), _ptr(W_dev)), self._h)

    def close(self):
        if getattr(self, "_h", None):
            _lib.fbim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched mobility solves over several handles (``FBIM`` objects).

    ``n_rhs[k]`` right-hand sides go with handle k; systems are ordered
    handle-major.  ``solve`` takes the systems' forces (and slips) as lists of
    tensors, or as stacked flat tensors, and returns the velocities as a list of
    [n_b, 3] tensors with the per-system iterations and FP64 relative residuals.
    """

    def __init__(self, ops, n_rhs=None):
        self.ops = list(ops)  # keeps the handles alive
        n = len(self.ops)
        self.n_rhs = [1] * n if n_rhs is None else [int(r) for r in n_rhs]
        hs = (_P * n)(*[o.handle.value if isinstance(o.handle, _P) else o.handle for o in self.ops])
        rr = (ctypes.c_int * n)(*self.n_rhs)
        b = _P()
        st = _lib.fbim_batch_create(ctypes.byref(b), n, hs, rr)
        if st != 0:
            msg = _lib.fbim_batch_last_error(None)
            raise FbimError(st, msg.decode() if msg else "")
        self._b = b
        self.systems = [(k, r) for k in range(n) for r in range(self.n_rhs[k])]

    def _check(self, st):
        if st != 0:
            msg = _lib.fbim_batch_last_error(self._b)
            raise FbimError(st, msg.decode() if msg else "")

    def info(self):
        i = BatchInfo()
        self._check(_lib.fbim_batch_get_info(self._b, ctypes.byref(i)))
        return i.as_dict()

    def solve(self, F, slip=None, tol=1e-6, max_iter=500, check=True, out=None):
        """out: optional flat float64 tensor for the stacked velocities (3 n_b per system)."""
        import torch
        Fs = torch.cat([f.reshape(-1) for f in F]) if isinstance(F, (list, tuple)) else F
        Ss = None
        if slip is not None:
            Ss = torch.cat([s.reshape(-1) for s in slip]) if isinstance(slip, (list, tuple)) else slip
        n_sys = len(self.systems)
        sizes = [3 * self.ops[k].n_b for k, _ in self.systems]
        if out is None:
            U = torch.empty(sum(sizes), dtype=torch.float64, device=Fs.device)
        elif out.numel() != sum(sizes) or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out: contiguous float64 with 3 n_b entries per system")
        else:
            U = out.view(-1)
        it = (ctypes.c_int * n_sys)()
        res = (ctypes.c_double * n_sys)()
        st = _lib.fbim_batch_solve(self._b, _ptr(Fs), None if Ss is None else _ptr(Ss), float(tol), int(max_iter),
                                   _ptr(U), it, res)
        if check or st not in (0, 6):
            self._check(st)
        Us = list(torch.split(U, sizes))
        return [u.view(-1, 3) for u in Us], list(it), list(res)

    def slip(self, seeds, counter=0, kT=1.0, dt=1.0, tol=1e-6, max_iter=200, out=None):
        """Brownian slip of every system: system i with Philox seed seeds[i] (an int gives
        seeds + i).  Returns the [N, 2] slips as views of one stacked tensor (``out`` if
        given, a flat float64 tensor of the systems' 2N entries) and the Lanczos steps."""
        import torch
        n_sys = len(self.systems)
        if isinstance(seeds, int):
            seeds = [seeds + i for i in range(n_sys)]
        if len(seeds) != n_sys:
            raise ValueError("one seed per system")
        sizes = [2 * self.ops[k].n for k, _ in self.systems]
        if out is None:
            out = torch.empty(sum(sizes), dtype=torch.float64, device=torch.device("cuda", self.ops[0].device))
        elif out.numel() < sum(sizes) or out.dtype != torch.float64 or not out.is_contiguous():
            raise ValueError("out: contiguous float64 with the systems' 2N entries")
        sd = (ctypes.c_uint64 * n_sys)(*[int(x) for x in seeds])
        it = (ctypes.c_int * n_sys)()
        self._check(_lib.fbim_batch_slip(self._b, sd, int(counter), float(kT), float(dt), float(tol),
                                         int(max_iter), _ptr(out), it))
        flat = out.reshape(-1)[:sum(sizes)]
        return [s.view(-1, 2) for s in torch.split(flat, sizes)], list(it)

    def close(self):
        if getattr(self, "_b", None):
            _lib.fbim_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_param_count() -> int:
    return _lib.fbim_mlp_param_count()


class MLP:
    """Pair-correction network 6-128-128-128-36 (bf16 tensor-core products, FP32 state)."""

    def __init__(self, max_batch=1024, device=0, stream=None):
        m = _P()
        st = _lib.fbim_mlp_create(ctypes.byref(m), int(max_batch), stream, int(device))
        if st != 0:
            msg = _lib.fbim_mlp_last_error(None)
            raise FbimError(st, msg.decode() if msg else "")
        self._m = m
        self.max_batch = int(max_batch)
        self.device = int(device)
        self.n_params = mlp_param_count()

    def _check(self, st):
        if st != 0:
            msg = _lib.fbim_mlp_last_error(self._m)
            raise FbimError(st, msg.decode() if msg else "")

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.n_params
        self._check(_lib.fbim_mlp_set_params(self._m, t.ctypes.data_as(_FP)))

    def get_params(self):
        t = np.empty(self.n_params, dtype=np.float32)
        self._check(_lib.fbim_mlp_get_params(self._m, t.ctypes.data_as(_FP)))
        return t

    def set_normalization(self, in_shift, in_scale, out_scale):
        a = [np.ascontiguousarray(x, dtype=np.float32) for x in (in_shift, in_scale, out_scale)]
        self._check(_lib.fbim_mlp_set_normalization(self._m, *[x.ctypes.data_as(_FP) for x in a]))
        self.normalization = a

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], 36), dtype=torch.float32, device=X.device)
        self._check(_lib.fbim_mlp_forward(self._m, int(X.shape[0]), _ptr(X), _ptr(Y)))
        return Y

    def gradient(self, X, T):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device=X.device)
        loss = ctypes.c_double(0.0)
        self._check(_lib.fbim_mlp_gradient(self._m, int(X.shape[0]), _ptr(X), _ptr(T), _ptr(g), ctypes.byref(loss)))
        return loss.value, g

    def adam_step(self, X, T, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        loss = ctypes.c_double(0.0)
        self._check(_lib.fbim_mlp_adam_step(self._m, int(X.shape[0]), _ptr(X), _ptr(T), float(lr), float(beta1),
                                            float(beta2), float(eps), ctypes.byref(loss)))
        return loss.value

    @property
    def launches(self):
        return _lib.fbim_mlp_launches(self._m)

    def close(self):
        if getattr(self, "_m", None):
            _lib.fbim_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
