"""Thin ctypes binding of the dd_nls C-ABI (include/dd_nls.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module only converts arguments.
Arrays may be numpy arrays (host memory) or CUDA torch tensors (device memory); the
pointer kind is passed to the library accordingly.  If the compiled library is missing the
import of a Solver fails loudly: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libddnls.so")

TC_ROBIN, TC_PADE = 0, 1
BC_SAME, BC_NEUMANN = 0, 1
CLASSICAL, PRECONDITIONED = 0, 1
FP64, FP32_INNER, FP32_DW = 0, 1, 2
GUESS_ZERO, GUESS_PREVIOUS = 0, 1
PTR_HOST, PTR_DEVICE = 0, 1
PSOLVE_GMRES, PSOLVE_MODAL = 0, 1

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENONFINITE",
          6: "ETIMEOUT", 7: "EBREAKDOWN"}


class Params(ctypes.Structure):
    _fields_ = [
        ("xl", ctypes.c_double), ("xr", ctypes.c_double), ("yb", ctypes.c_double), ("yu", ctypes.c_double),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("n_strips", ctypes.c_int),
        ("dt", ctypes.c_double), ("lap", ctypes.c_double), ("kappa", ctypes.c_double),
        ("tc", ctypes.c_int), ("p", ctypes.c_double), ("pade_m", ctypes.c_int), ("pade_theta", ctypes.c_double),
        ("bc", ctypes.c_int), ("algorithm", ctypes.c_int), ("precision", ctypes.c_int), ("guess", ctypes.c_int),
        ("tol", ctypes.c_double), ("tol_absolute", ctypes.c_int), ("max_schwarz", ctypes.c_int),
        ("nl_tol", ctypes.c_double), ("max_nl", ctypes.c_int),
        ("inner_tol", ctypes.c_double), ("max_inner", ctypes.c_int),
        ("gmres_tol", ctypes.c_double), ("gmres_restart", ctypes.c_int), ("gmres_max", ctypes.c_int),
        ("psolve", ctypes.c_int), ("nl_relax", ctypes.c_double), ("nl_picard", ctypes.c_int),
        ("nl_adapt", ctypes.c_double),
        ("omega_rot", ctypes.c_double), ("trap_gx", ctypes.c_double), ("trap_gy", ctypes.c_double),
        ("psolve_modes", ctypes.c_int), ("wait_limit_ms", ctypes.c_double), ("solver_layout", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int), ("schwarz_iterations", ctypes.c_int), ("last_schwarz_iterations", ctypes.c_int),
        ("nl_iterations", ctypes.c_longlong), ("krylov_iterations", ctypes.c_longlong),
        ("gmres_iterations", ctypes.c_longlong),
        ("residual", ctypes.c_double), ("residual_abs", ctypes.c_double),
        ("mass", ctypes.c_double), ("energy", ctypes.c_double), ("setup_ms", ctypes.c_double),
        ("lz", ctypes.c_double), ("energy_lab", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [
        ("strip_solve_ms", ctypes.c_double), ("strip_solve_launches", ctypes.c_longlong),
        ("strip_solve_bytes", ctypes.c_double), ("strip_solve_flops", ctypes.c_double),
        ("interface_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
        ("kernel_launches", ctypes.c_longlong),
        ("phase_cycles", ctypes.c_double * 5),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["phase_cycles"] = list(self.phase_cycles)
        return d


SYMBOLS = ["dd_nls_default_params", "dd_nls_create", "dd_nls_step", "dd_nls_solve_interface",
           "dd_nls_get_state", "dd_nls_set_state", "dd_nls_get_blocks", "dd_nls_get_modal", "dd_nls_set_profiling",
           "dd_nls_get_profile", "dd_nls_destroy", "dd_nls_last_error", "dd_nls_step_noalloc",
           "dd_nls_batch_create", "dd_nls_batch_step", "dd_nls_batch_get_u", "dd_nls_batch_tuning",
           "dd_nls_batch_set_profiling", "dd_nls_batch_get_profile", "dd_nls_batch_last_error",
           "dd_nls_batch_destroy", "dd_nls_step_guess", "dd_cnn_create", "dd_cnn_num_params",
           "dd_cnn_set_params", "dd_cnn_get_params", "dd_cnn_guess", "dd_cnn_train_step", "dd_cnn_loss_grad",
           "dd_cnn_last_error", "dd_cnn_destroy", "dd_nls_lab_frame", "dd_nls_batch_set_u", "dd_cnn_set_base"]

_lib = None


def load(path=LIB_PATH):
    """Load the compiled library (build it with paper_1603_05110_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"dd_nls CUDA library not built: {path} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.dd_nls_default_params.argtypes = [ctypes.POINTER(Params)]
    lib.dd_nls_default_params.restype = None
    lib.dd_nls_create.argtypes = [ctypes.POINTER(Params), vp, vp, ip, vp, ctypes.POINTER(vp)]
    lib.dd_nls_create.restype = ip
    lib.dd_nls_step.argtypes = [vp, ip, vp, ip, ctypes.POINTER(Stats)]
    lib.dd_nls_step.restype = ip
    lib.dd_nls_solve_interface.argtypes = [vp, vp, vp, vp, ip, ctypes.POINTER(Stats)]
    lib.dd_nls_solve_interface.restype = ip
    lib.dd_nls_get_state.argtypes = [vp, vp, vp, ctypes.POINTER(ctypes.c_int), ip]
    lib.dd_nls_get_state.restype = ip
    lib.dd_nls_set_state.argtypes = [vp, vp, vp, ip, ip]
    lib.dd_nls_set_state.restype = ip
    lib.dd_nls_get_blocks.argtypes = [vp, ip, vp, ip]
    lib.dd_nls_get_blocks.restype = ip
    lib.dd_nls_get_modal.argtypes = [vp, ip, vp, ip]
    lib.dd_nls_get_modal.restype = ip
    lib.dd_nls_lab_frame.argtypes = [vp, ip, ip, vp, ip]
    lib.dd_nls_lab_frame.restype = ip
    lib.dd_nls_set_profiling.argtypes = [vp, ip]
    lib.dd_nls_set_profiling.restype = ip
    lib.dd_nls_get_profile.argtypes = [vp, ctypes.POINTER(Profile)]
    lib.dd_nls_get_profile.restype = ip
    lib.dd_nls_destroy.argtypes = [vp]
    lib.dd_nls_destroy.restype = None
    lib.dd_nls_last_error.argtypes = [vp]
    lib.dd_nls_last_error.restype = ctypes.c_char_p
    lib.dd_nls_step_noalloc.argtypes = [ctypes.POINTER(Params), vp, vp, vp, vp, vp, ctypes.POINTER(Stats)]
    lib.dd_nls_step_noalloc.restype = ip
    pp = ctypes.POINTER(ctypes.c_void_p)
    lib.dd_nls_batch_create.argtypes = [ip, ctypes.POINTER(Params), pp, pp, ip, vp, ctypes.POINTER(vp)]
    lib.dd_nls_batch_create.restype = ip
    lib.dd_nls_batch_step.argtypes = [vp, ip, ctypes.POINTER(Stats)]
    lib.dd_nls_batch_step.restype = ip
    lib.dd_nls_batch_get_u.argtypes = [vp, ip, vp, ip]
    lib.dd_nls_batch_get_u.restype = ip
    lib.dd_nls_batch_set_u.argtypes = [vp, ip, vp, ip]
    lib.dd_nls_batch_set_u.restype = ip
    lib.dd_nls_batch_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.dd_nls_batch_tuning.restype = ip
    lib.dd_nls_batch_set_profiling.argtypes = [vp, ip]
    lib.dd_nls_batch_set_profiling.restype = ip
    lib.dd_nls_batch_get_profile.argtypes = [vp, ctypes.POINTER(Profile)]
    lib.dd_nls_batch_get_profile.restype = ip
    lib.dd_nls_batch_last_error.argtypes = [vp]
    lib.dd_nls_batch_last_error.restype = ctypes.c_char_p
    lib.dd_nls_batch_destroy.argtypes = [vp]
    lib.dd_nls_batch_destroy.restype = None
    lib.dd_nls_step_guess.argtypes = [vp, vp, vp, ip, ctypes.POINTER(Stats)]
    lib.dd_nls_step_guess.restype = ip
    lib.dd_cnn_create.argtypes = [ip, ip, vp, ctypes.POINTER(vp)]
    lib.dd_cnn_create.restype = ip
    lib.dd_cnn_num_params.argtypes = [vp]
    lib.dd_cnn_num_params.restype = ctypes.c_longlong
    lib.dd_cnn_set_base.argtypes = [vp, ip]
    lib.dd_cnn_set_base.restype = ip
    lib.dd_cnn_set_params.argtypes = [vp, vp, ip]
    lib.dd_cnn_set_params.restype = ip
    lib.dd_cnn_get_params.argtypes = [vp, vp, ip]
    lib.dd_cnn_get_params.restype = ip
    lib.dd_cnn_guess.argtypes = [vp, vp, vp, vp, vp]
    lib.dd_cnn_guess.restype = ip
    lib.dd_cnn_train_step.argtypes = [vp, vp, vp, vp, vp, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]
    lib.dd_cnn_train_step.restype = ip
    lib.dd_cnn_loss_grad.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double), ip]
    lib.dd_cnn_loss_grad.restype = ip
    lib.dd_cnn_last_error.argtypes = [vp]
    lib.dd_cnn_last_error.restype = ctypes.c_char_p
    lib.dd_cnn_destroy.argtypes = [vp]
    lib.dd_cnn_destroy.restype = None
    _ = dp
    _lib = lib
    return lib


class DDNLSError(RuntimeError):
    def __init__(self, code, msg, stats=None):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.stats = stats          # the call's statistics up to the failure, when it has any


def default_params(**kw):
    lib = load()
    p = Params()
    lib.dd_nls_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(a, writable=False):
    """(pointer, kind) of a numpy array or torch tensor, or (None, None)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):                      # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (PTR_DEVICE if a.is_cuda else PTR_HOST)
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous numpy array or a torch tensor")
    if writable and not a.flags.writeable:
        raise ValueError("output array is read-only")
    return a.ctypes.data, PTR_HOST


def _kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ks.pop() if ks else PTR_HOST


def step_noalloc(params, u, V=None, g0=None, g_out=None, stream=None):
    """One time step through dd_nls_step_noalloc (no device allocation inside the library).

    u (in/out), V, g0, g_out must be CUDA tensors (device pointers)."""
    lib = load()
    if isinstance(params, dict):
        params = default_params(**params)
    ptrs = []
    for a in (V, u, g0, g_out):
        pa, ka = _ptr(a)
        if pa is not None and ka != PTR_DEVICE:
            raise ValueError("dd_nls_step_noalloc takes device arrays only")
        ptrs.append(pa)
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = Stats()
    rc = lib.dd_nls_step_noalloc(ctypes.byref(params), ptrs[0], ptrs[1], ptrs[2], ptrs[3], s, ctypes.byref(st))
    if rc != 0:
        raise DDNLSError(rc, lib.dd_nls_last_error(None).decode(), st.as_dict())
    return st.as_dict()


class Solver:
    """A dd_nls handle.  ``params``: a Params or a dict of its fields."""

    def __init__(self, params, u0, V=None, stream=None):
        self.lib = load()
        if isinstance(params, dict):
            params = default_params(**params)
        self.params = params
        if isinstance(u0, np.ndarray):
            u0 = np.ascontiguousarray(u0, dtype=np.complex128)
        if isinstance(V, np.ndarray):
            V = np.ascontiguousarray(V, dtype=np.float64)
        pu, ku = _ptr(u0)
        pv, kv = _ptr(V)
        kind = _kind(ku, kv)
        self.shape = (params.ny + 1, params.nx + 1)
        self.n_traces = 2 * (params.n_strips - 1)
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        h = ctypes.c_void_p()
        rc = self.lib.dd_nls_create(ctypes.byref(params), pv, pu, kind, s, ctypes.byref(h))
        if rc != 0:
            raise DDNLSError(rc, self.lib.dd_nls_last_error(None).decode())
        self.h = h

    def _check(self, rc, stats=None):
        if rc != 0:
            raise DDNLSError(rc, self.lib.dd_nls_last_error(self.h).decode(),
                             stats.as_dict() if stats is not None else None)

    def step(self, nsteps=1, u_out=None):
        st = Stats()
        pu, ku = _ptr(u_out, writable=True)
        self._check(self.lib.dd_nls_step(self.h, nsteps, pu, _kind(ku), ctypes.byref(st)), st)
        return st.as_dict()

    def step_guess(self, g0, u_out=None):
        st = Stats()
        p0, k0 = _ptr(g0)
        pu, ku = _ptr(u_out, writable=True)
        self._check(self.lib.dd_nls_step_guess(self.h, p0, pu, _kind(k0, ku), ctypes.byref(st)), st)
        return st.as_dict()

    def solve_interface(self, g0=None, g_out=None, v_out=None):
        st = Stats()
        p0, k0 = _ptr(g0)
        pg, kg = _ptr(g_out, writable=True)
        pv, kv = _ptr(v_out, writable=True)
        self._check(self.lib.dd_nls_solve_interface(self.h, p0, pg, pv, _kind(k0, kg, kv), ctypes.byref(st)), st)
        return st.as_dict()

    def get_state(self, u=None, g=None):
        pu, ku = _ptr(u, writable=True)
        pg, kg = _ptr(g, writable=True)
        n = ctypes.c_int()
        self._check(self.lib.dd_nls_get_state(self.h, pu, pg, ctypes.byref(n), _kind(ku, kg)))
        return n.value

    def set_state(self, u=None, g=None, step=0):
        pu, ku = _ptr(u)
        pg, kg = _ptr(g)
        self._check(self.lib.dd_nls_set_state(self.h, pu, pg, step, _kind(ku, kg)))

    def blocks(self, strip):
        ne = self.params.ny + 1
        x = np.zeros((4, ne, ne), np.complex128)
        self._check(self.lib.dd_nls_get_blocks(self.h, strip, x.ctypes.data, PTR_HOST))
        return x

    def modal(self, strip):
        ne = self.params.ny + 1
        x = np.zeros((4, ne), np.complex128)
        self._check(self.lib.dd_nls_get_modal(self.h, strip, x.ctypes.data, PTR_HOST))
        return x

    def lab_frame(self, nx_out, ny_out, out=None):
        """u(t_n) in the lab frame on the valid zone, (ny_out+1, nx_out+1) complex values."""
        if out is None:
            out = np.zeros((ny_out + 1, nx_out + 1), np.complex128)
        po, ko = _ptr(out, writable=True)
        self._check(self.lib.dd_nls_lab_frame(self.h, nx_out, ny_out, po, _kind(ko)))
        return out

    def set_profiling(self, on=True):
        self._check(self.lib.dd_nls_set_profiling(self.h, 1 if on else 0))

    def profile(self):
        p = Profile()
        self._check(self.lib.dd_nls_get_profile(self.h, ctypes.byref(p)))
        return p.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.dd_nls_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """A dd_nls_batch handle: n independent instances stepped together.

    params: list of Params or dicts; u0, V: lists of arrays (numpy = host, CUDA tensors = device).
    """

    def __init__(self, params, u0, V=None, stream=None):
        self.lib = load()
        n = len(params)
        arr = (Params * n)()
        for i, p in enumerate(params):
            arr[i] = default_params(**p) if isinstance(p, dict) else p
        self.params = list(arr)
        keep = []
        kinds = []
        up = (ctypes.c_void_p * n)()
        vp_ = (ctypes.c_void_p * n)()
        for i in range(n):
            u = u0[i]
            if isinstance(u, np.ndarray):
                u = np.ascontiguousarray(u, dtype=np.complex128)
            keep.append(u)
            pu, ku = _ptr(u)
            up[i] = pu
            kinds.append(ku)
            if V is not None and V[i] is not None:
                v = V[i]
                if isinstance(v, np.ndarray):
                    v = np.ascontiguousarray(v, dtype=np.float64)
                keep.append(v)
                pv, kv = _ptr(v)
                vp_[i] = pv
                kinds.append(kv)
        kind = _kind(*kinds)
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        h = ctypes.c_void_p()
        rc = self.lib.dd_nls_batch_create(n, arr, vp_, up, kind, s, ctypes.byref(h))
        if rc != 0:
            raise DDNLSError(rc, self.lib.dd_nls_batch_last_error(None).decode())
        self.h = h
        self.n = n

    def _check(self, rc, stats=None):
        if rc != 0:
            raise DDNLSError(rc, self.lib.dd_nls_batch_last_error(self.h).decode(), stats)

    def step(self, nsteps=1):
        st = (Stats * self.n)()
        rc = self.lib.dd_nls_batch_step(self.h, nsteps, st)
        self._check(rc, [x.as_dict() for x in st])
        return [x.as_dict() for x in st]

    def get_u(self, i, out=None):
        p = self.params[i]
        if out is None:
            out = np.zeros((p.ny + 1, p.nx + 1), np.complex128)
        po, ko = _ptr(out, writable=True)
        self._check(self.lib.dd_nls_batch_get_u(self.h, i, po, ko))
        return out

    def set_u(self, i, u):
        if isinstance(u, np.ndarray):
            u = np.ascontiguousarray(u, dtype=np.complex128)
        pu, ku = _ptr(u)
        self._check(self.lib.dd_nls_batch_set_u(self.h, i, pu, ku))

    def tuning(self):
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.dd_nls_batch_tuning(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_profiling(self, on=True):
        self._check(self.lib.dd_nls_batch_set_profiling(self.h, 1 if on else 0))

    def profile(self):
        p = Profile()
        self._check(self.lib.dd_nls_batch_get_profile(self.h, ctypes.byref(p)))
        return p.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.dd_nls_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


CNN_LAYERS = ((6, 32), (32, 32), (32, 32), (32, 2))


class CNN:
    """A dd_cnn handle (learned interface guess).  Interface vectors are CUDA complex128
    tensors of shape (2(N-1), ny+1)."""

    BASE_PREVIOUS, BASE_EXTRAPOLATE = 0, 1

    def __init__(self, n_traces, nodes_per_trace, stream=None, base=1):
        self.lib = load()
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        h = ctypes.c_void_p()
        rc = self.lib.dd_cnn_create(n_traces, nodes_per_trace, s, ctypes.byref(h))
        if rc != 0:
            raise DDNLSError(rc, self.lib.dd_nls_last_error(None).decode())
        self.h = h
        self.n = int(self.lib.dd_cnn_num_params(h))
        if base != self.BASE_EXTRAPOLATE:
            self._check(self.lib.dd_cnn_set_base(h, int(base)))

    def _check(self, rc):
        if rc != 0:
            raise DDNLSError(rc, self.lib.dd_cnn_last_error(self.h).decode())

    @staticmethod
    def init_params(seed=0, last_scale=0.0):
        """He-normal weights, zero biases; the last layer scaled by last_scale (0: the network
        starts as linear extrapolation)."""
        rng = np.random.default_rng(seed)
        out = []
        for i, (ci, co) in enumerate(CNN_LAYERS):
            w = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (ci * 9))
            if i == len(CNN_LAYERS) - 1:
                w *= last_scale
            out += [w.ravel(), np.zeros(co)]
        return np.concatenate(out).astype(np.float32)

    def set_params(self, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.n
        self._check(self.lib.dd_cnn_set_params(self.h, w.ctypes.data, PTR_HOST))

    def get_params(self):
        w = np.zeros(self.n, np.float32)
        self._check(self.lib.dd_cnn_get_params(self.h, w.ctypes.data, PTR_HOST))
        return w

    def guess(self, g1, g2, g3, out):
        self._check(self.lib.dd_cnn_guess(self.h, g1.data_ptr(), g2.data_ptr(), g3.data_ptr(), out.data_ptr()))
        return out

    def train_step(self, g1, g2, g3, gt, lr=1e-3):
        loss = ctypes.c_double()
        self._check(self.lib.dd_cnn_train_step(self.h, g1.data_ptr(), g2.data_ptr(), g3.data_ptr(), gt.data_ptr(),
                                               lr, ctypes.byref(loss)))
        return loss.value

    def loss_grad(self, g1, g2, g3, gt):
        grad = np.zeros(self.n, np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.dd_cnn_loss_grad(self.h, g1.data_ptr(), g2.data_ptr(), g3.data_ptr(), gt.data_ptr(),
                                              grad.ctypes.data, ctypes.byref(loss), PTR_HOST))
        return loss.value, grad

    def close(self):
        if getattr(self, "h", None):
            self.lib.dd_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
