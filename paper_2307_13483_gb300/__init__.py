"""Python binding of libvbk (GB300 Krylov solver for vibronic dynamics in the electron continuum).

Thin ctypes marshalling over the C ABI declared in ``include/vbk.h``: every computation runs
in the CUDA library; this module only converts model dictionaries to the C structures,
passes torch tensors' device pointers and the current CUDA stream, and returns results.
The function names are those of the C ABI.  Importing the module loads ``libvbk.so`` and
raises if it has not been built (``python -m paper_2307_13483_gb300.build`` or
``__graft_entry__.build()``).
"""

from __future__ import annotations

import ctypes as C
from collections.abc import Sequence
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvbk.so")

VBK_MAX_MODES = 4
VBK_OK = 0
VBK_ERR_NOT_CONVERGED = 4
VBK_GMRES, VBK_COCG = 0, 1
VBK_FP64, VBK_MIXED = 0, 1
VBK_PRECOND_NONE = -1
VBK_MATVEC_NVARIANTS = 20
SYS_STATUS = {0: "converged", 1: "max_iter", 2: "breakdown", 3: "nan", 4: "pivot", 5: "zero_rhs"}


class vbk_term(C.Structure):
    _fields_ = [("d", C.c_int), ("dp", C.c_int), ("coef", C.c_double), ("pow", C.c_int * VBK_MAX_MODES),
                ("raise", C.c_int * VBK_MAX_MODES), ("lower", C.c_int * VBK_MAX_MODES)]


class vbk_channel(C.Structure):
    _fields_ = [("d", C.c_int), ("mu", C.c_int), ("a", C.c_double), ("b", C.c_double), ("l", C.c_int)]


class vbk_cterm(C.Structure):
    _fields_ = [("channel", C.c_int), ("coef", C.c_double), ("pow", C.c_int * VBK_MAX_MODES)]


class vbk_model_desc(C.Structure):
    _fields_ = [
        ("n_states", C.c_int),
        ("n_modes", C.c_int),
        ("n_basis", C.c_int * VBK_MAX_MODES),
        ("omega", C.c_double * VBK_MAX_MODES),
        ("n_terms", C.c_int),
        ("terms", C.POINTER(vbk_term)),
        ("n_channels", C.c_int),
        ("channels", C.POINTER(vbk_channel)),
        ("n_cterms", C.c_int),
        ("cterms", C.POINTER(vbk_cterm)),
    ]


class vbk_opts(C.Structure):
    _fields_ = [
        ("method", C.c_int),
        ("precision", C.c_int),
        ("precond_span", C.c_int),
        ("restart", C.c_int),
        ("max_iter", C.c_int),
        ("max_refine", C.c_int),
        ("tol", C.c_double),
        ("inner_tol", C.c_double),
        ("check_every", C.c_int),
        ("timing", C.c_int),
        ("autotune", C.c_int),
        ("resident", C.c_int),
        ("inner_max_iter", C.c_int),
        ("matvec_variant", C.c_int),
    ]


class vbk_stats(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("refinements", C.c_int), ("rel_residual", C.c_double)]


_STATS_DTYPE = np.dtype({"names": ["status", "iterations", "refinements", "rel_residual"],
                         "formats": ["<i4", "<i4", "<i4", "<f8"], "offsets": [0, 4, 8, 16], "itemsize": 24})


class SolveStats(Sequence):
    """Per-system results of a solve: item k is a dict (status name, iterations, refinements,
    rel_residual), built on access; the fields are also numpy arrays (``.status`` holds the
    VBK_SYS_* codes) over the library's own result buffer."""

    def __init__(self, buf):
        assert C.sizeof(vbk_stats) == _STATS_DTYPE.itemsize
        self._buf = buf
        self._a = np.frombuffer(buf, dtype=_STATS_DTYPE)

    def __len__(self):
        return self._a.size

    def __getitem__(self, k):
        if isinstance(k, slice):
            return [self[i] for i in range(*k.indices(len(self)))]
        r = self._a[k]
        code = int(r["status"])
        return dict(status=SYS_STATUS.get(code, code), iterations=int(r["iterations"]), refinements=int(r["refinements"]),
                    rel_residual=float(r["rel_residual"]))

    def __getattr__(self, name):
        if name in _STATS_DTYPE.names:
            return self._a[name]
        raise AttributeError(name)


EXPORTED = [
    "vbk_default_opts", "vbk_build_model", "vbk_free_model", "vbk_model_size", "vbk_solve",
    "vbk_cross_sections", "vbk_eels", "vbk_solve_adjoint", "vbk_matvec", "vbk_precond_apply",
    "vbk_kernel_timings", "vbk_last_launch_count", "vbk_level_shift", "vbk_status_str",
    "vbk_sys_status_str", "vbk_last_error", "vbk_matvec_noalloc", "vbk_matvec_variant", "vbk_set_op_timing",
    "vbk_level_shift_df", "vbk_debug_stream_delay",
]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvbk.so is not built ({LIB_PATH}); run paper_2307_13483_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    sig = {
        "vbk_default_opts": (None, [C.POINTER(vbk_opts)]),
        "vbk_build_model": (C.c_int, [C.POINTER(vbk_model_desc), C.POINTER(vp)]),
        "vbk_free_model": (None, [vp]),
        "vbk_model_size": (C.c_int, [vp, ip, ip]),
        "vbk_solve": (C.c_int, [vp, C.c_int, dp, C.c_int, ip, C.POINTER(vbk_opts), vp, C.POINTER(vbk_stats), vp]),
        "vbk_cross_sections": (C.c_int, [vp, C.c_int, dp, C.c_int, ip, vp, C.c_int, ip, vp, vp, vp]),
        "vbk_eels": (C.c_int, [vp, C.c_int, C.c_int, ip, C.c_int, ip, vp, C.c_int, dp, C.c_double, vp, vp]),
        "vbk_solve_adjoint": (C.c_int, [vp, C.c_int, dp, C.c_int, ip, C.POINTER(vbk_opts), vp, C.c_int, ip, vp,
                                        C.c_int, ip, dp, C.POINTER(vbk_stats), vp]),
        "vbk_matvec": (C.c_int, [vp, C.c_int, dp, C.c_int, vp, vp, C.c_int, C.c_int, vp]),
        "vbk_precond_apply": (C.c_int, [vp, C.c_int, dp, C.c_int, C.c_int, vp, vp, C.c_int, vp]),
        "vbk_matvec_noalloc": (C.c_int, [vp, C.c_int, dp, C.c_int, vp, vp, vp]),
        "vbk_kernel_timings": (C.c_int, [vp, C.c_int, C.POINTER(C.c_char_p), ip, dp]),
        "vbk_last_launch_count": (C.c_longlong, [vp]),
        "vbk_matvec_variant": (C.c_int, [vp, C.c_int]),
        "vbk_debug_stream_delay": (C.c_int, [C.c_int]),
        "vbk_set_op_timing": (C.c_int, [vp, C.c_int]),
        "vbk_level_shift": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int, dp, dp]),
        "vbk_level_shift_df": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int, dp, dp]),
        "vbk_status_str": (C.c_char_p, [C.c_int]),
        "vbk_sys_status_str": (C.c_char_p, [C.c_int]),
        "vbk_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


class VbkError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.vbk_last_error().decode()
        super().__init__(f"{where}: {_lib.vbk_status_str(code).decode()} ({code}) {msg}")


def _check(code, where, allow=()):
    if code != VBK_OK and code not in allow:
        raise VbkError(code, where)
    return code


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _stream(stream):
    if stream is None:
        import torch

        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def _tensor_ptr(t):
    return C.c_void_p(t.data_ptr())


class Model:
    """Owns a ``vbk_model*`` built from a model dictionary (see ``workloads``)."""

    def __init__(self, desc: dict):
        self.desc = desc
        modes = desc["modes"]
        d = vbk_model_desc()
        d.n_states = int(desc["n_states"])
        d.n_modes = len(modes)
        for k, mo in enumerate(modes):
            d.n_basis[k] = int(mo["n"])
            d.omega[k] = float(mo["omega"])
        terms = (vbk_term * max(1, len(desc["terms"])))()
        for k, t in enumerate(desc["terms"]):
            terms[k].d, terms[k].dp, terms[k].coef = int(t["d"]), int(t["dp"]), float(t["coef"])
            for j, pw in enumerate(t["pow"]):
                terms[k].pow[j] = int(pw)
            for j, v in enumerate(t.get("raise") or []):
                getattr(terms[k], "raise")[j] = int(v)  # (a Python keyword as a field name)
            for j, v in enumerate(t.get("lower") or []):
                terms[k].lower[j] = int(v)
        chans = (vbk_channel * max(1, len(desc["channels"])))()
        for k, c in enumerate(desc["channels"]):
            chans[k].d, chans[k].mu, chans[k].a, chans[k].b, chans[k].l = (
                int(c["d"]), int(c["mu"]), float(c["a"]), float(c["b"]), int(c["l"]))
        d.n_terms, d.terms = len(desc["terms"]), terms
        d.n_channels, d.channels = len(desc["channels"]), chans
        # coupling polynomials of q-dependent channels (Sec. II.C), channel by channel
        ct = [(k, t) for k, c in enumerate(desc["channels"]) for t in (c.get("terms") or [])]
        cterms = (vbk_cterm * max(1, len(ct)))()
        for j, (k, t) in enumerate(ct):
            cterms[j].channel, cterms[j].coef = k, float(t["coef"])
            for i, pw in enumerate(t["pow"]):
                cterms[j].pow[i] = int(pw)
        d.n_cterms, d.cterms = len(ct), cterms
        h = C.c_void_p()
        _check(_lib.vbk_build_model(C.byref(d), C.byref(h)), "vbk_build_model")
        self.handle = h
        n, nmu = C.c_int(), C.c_int()
        _check(_lib.vbk_model_size(h, C.byref(n), C.byref(nmu)), "vbk_model_size")
        self.N, self.n_mu = n.value, nmu.value
        self.n_modes = len(modes)

    def close(self):
        if getattr(self, "handle", None):
            _lib.vbk_free_model(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def vbk_build_model(desc: dict) -> Model:
    return Model(desc)


def vbk_default_opts(**kw) -> vbk_opts:
    o = vbk_opts()
    _lib.vbk_default_opts(C.byref(o))
    names = {"method": {"gmres": VBK_GMRES, "cocg": VBK_COCG}, "precision": {"fp64": VBK_FP64, "mixed": VBK_MIXED}}
    for k, v in kw.items():
        if k in names and isinstance(v, str):
            v = names[k][v]
        setattr(o, k, v)
    return o


def _multi(model: Model, states) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(states, dtype=np.int32).reshape(-1, model.n_modes))
    return a


def vbk_solve(model: Model, eps_i, vi, opts: vbk_opts | None = None, psi=None, stream=None, check=True):
    """Solves all (eps_i, v_i, mu) systems; returns (psi [n_eps, n_vi, n_mu, N] complex128, stats list)."""
    import torch

    eps = np.ascontiguousarray(np.asarray(eps_i, dtype=np.float64).ravel())
    vis = _multi(model, vi)
    nsys = eps.size * vis.shape[0] * model.n_mu
    if psi is None:
        psi = torch.empty((eps.size, vis.shape[0], model.n_mu, model.N), dtype=torch.complex128, device="cuda")
    st = (vbk_stats * nsys)()
    o = opts or vbk_default_opts()
    rc = _lib.vbk_solve(model.handle, eps.size, _dptr(eps), vis.shape[0], _iptr(vis), C.byref(o), _tensor_ptr(psi), st,
                        _stream(stream))
    _check(rc, "vbk_solve", allow=() if check else (VBK_ERR_NOT_CONVERGED,))
    return psi, SolveStats(st)


def vbk_cross_sections(model: Model, eps_i, vi, psi, vf, stream=None, want_t=False):
    """sigma [n_eps, n_vi, n_vf] (device float64) and optionally T."""
    import torch

    eps = np.ascontiguousarray(np.asarray(eps_i, dtype=np.float64).ravel())
    vis, vfs = _multi(model, vi), _multi(model, vf)
    sig = torch.empty((eps.size, vis.shape[0], vfs.shape[0]), dtype=torch.float64, device=psi.device)
    T = None
    if want_t:
        T = torch.empty((eps.size, vis.shape[0], model.n_mu, vfs.shape[0], model.n_mu), dtype=torch.complex128,
                        device=psi.device)
    _check(_lib.vbk_cross_sections(model.handle, eps.size, _dptr(eps), vis.shape[0], _iptr(vis), _tensor_ptr(psi),
                                   vfs.shape[0], _iptr(vfs), _tensor_ptr(sig),
                                   _tensor_ptr(T) if T is not None else None, _stream(stream)), "vbk_cross_sections")
    return (sig, T) if want_t else sig


def vbk_eels(model: Model, vi, vf, sigma, de_grid, fwhm=0.010, stream=None):
    import torch

    vis, vfs = _multi(model, vi), _multi(model, vf)
    de = np.ascontiguousarray(np.asarray(de_grid, dtype=np.float64).ravel())
    n_eps = sigma.shape[0]
    S = torch.empty((n_eps, vis.shape[0], de.size), dtype=torch.float64, device=sigma.device)
    _check(_lib.vbk_eels(model.handle, n_eps, vis.shape[0], _iptr(vis), vfs.shape[0], _iptr(vfs), _tensor_ptr(sigma),
                         de.size, _dptr(de), float(fwhm), _tensor_ptr(S), _stream(stream)), "vbk_eels")
    return S


def vbk_solve_adjoint(model: Model, eps_i, vi, psi, vf, dL_dsigma, theta_ids, opts=None, stream=None, check=True):
    eps = np.ascontiguousarray(np.asarray(eps_i, dtype=np.float64).ravel())
    vis, vfs = _multi(model, vi), _multi(model, vf)
    th = np.ascontiguousarray(np.asarray(theta_ids, dtype=np.int32).ravel())
    grad = np.zeros(th.size, dtype=np.float64)
    nsys = eps.size * vis.shape[0] * model.n_mu
    st = (vbk_stats * nsys)()
    o = opts or vbk_default_opts()
    dl = dL_dsigma.contiguous()
    rc = _lib.vbk_solve_adjoint(model.handle, eps.size, _dptr(eps), vis.shape[0], _iptr(vis), C.byref(o),
                                _tensor_ptr(psi), vfs.shape[0], _iptr(vfs), _tensor_ptr(dl), th.size, _iptr(th),
                                _dptr(grad), st, _stream(stream))
    _check(rc, "vbk_solve_adjoint", allow=() if check else (VBK_ERR_NOT_CONVERGED,))
    return grad, SolveStats(st)


def vbk_matvec(model: Model, E, x, precision=VBK_FP64, variant=-1, stream=None):
    """y = A(E_k) x for x of shape [n_E, n_vec, N] (complex128, CUDA); variant -1 = tuned choice."""
    import torch

    Ev = np.ascontiguousarray(np.asarray(E, dtype=np.float64).ravel())
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(_lib.vbk_matvec(model.handle, Ev.size, _dptr(Ev), x.shape[1], _tensor_ptr(x), _tensor_ptr(y), precision,
                           int(variant), _stream(stream)), "vbk_matvec")
    return y


def vbk_matvec_noalloc(model: Model, E, x, y, stream=None):
    """y = A(E_k) x in FP64 into the caller's ``y`` without any device allocation by the library
    (its scratch is a fixed 8 MiB device array; see include/vbk.h for the limits)."""
    Ev = np.ascontiguousarray(np.asarray(E, dtype=np.float64).ravel())
    _check(_lib.vbk_matvec_noalloc(model.handle, Ev.size, _dptr(Ev), x.shape[1], _tensor_ptr(x), _tensor_ptr(y),
                                   _stream(stream)), "vbk_matvec_noalloc")
    return y


def vbk_precond_apply(model: Model, E, r, span, precision=VBK_FP64, stream=None):
    import torch

    Ev = np.ascontiguousarray(np.asarray(E, dtype=np.float64).ravel())
    r = r.contiguous()
    z = torch.empty_like(r)
    _check(_lib.vbk_precond_apply(model.handle, Ev.size, _dptr(Ev), r.shape[1], int(span), _tensor_ptr(r),
                                  _tensor_ptr(z), precision, _stream(stream)), "vbk_precond_apply")
    return z


def vbk_kernel_timings(model: Model):
    cap = 64
    names = (C.c_char_p * cap)()
    launches = (C.c_int * cap)()
    ms = (C.c_double * cap)()
    n = _lib.vbk_kernel_timings(model.handle, cap, names, launches, ms)
    return {names[k].decode(): (launches[k], ms[k]) for k in range(min(n, cap))}


def vbk_set_op_timing(model: Model, on: bool = True):
    """Per-kernel CUDA-event timings of later vbk_matvec / vbk_precond_apply calls (see
    vbk_kernel_timings); those calls then synchronise their stream."""
    _check(_lib.vbk_set_op_timing(model.handle, 1 if on else 0), "vbk_set_op_timing")


def vbk_debug_stream_delay(ms: int) -> None:
    """Test hook: the next streaming-matvec launch holds its first copies back by `ms` ms."""
    _check(_lib.vbk_debug_stream_delay(int(ms)), "vbk_debug_stream_delay")


def vbk_matvec_variant(model: Model, precision=VBK_MIXED) -> int:
    return int(_lib.vbk_matvec_variant(model.handle, int(precision)))


def vbk_last_launch_count(model: Model) -> int:
    return int(_lib.vbk_last_launch_count(model.handle))


def vbk_level_shift(eps: float, a: float, b: float, l: int) -> complex:
    re, im = C.c_double(), C.c_double()
    _check(_lib.vbk_level_shift(float(eps), float(a), float(b), int(l), C.byref(re), C.byref(im)), "vbk_level_shift")
    return complex(re.value, im.value)


def vbk_level_shift_df(eps: float, a: float, b: float, l: int) -> complex:
    """The level shift in double-float arithmetic (the FP32 refinement path's table code), on the host."""
    re, im = C.c_double(), C.c_double()
    _check(_lib.vbk_level_shift_df(float(eps), float(a), float(b), int(l), C.byref(re), C.byref(im)),
           "vbk_level_shift_df")
    return complex(re.value, im.value)


def vbk_status_str(code: int) -> str:
    return _lib.vbk_status_str(int(code)).decode()


def vbk_sys_status_str(code: int) -> str:
    return _lib.vbk_sys_status_str(int(code)).decode()


def vbk_last_error() -> str:
    return _lib.vbk_last_error().decode()


from .autograd import CrossSectionFunction, cross_sections_torch  # noqa: E402,F401
