"""Thin ctypes binding of libdtr (C ABI in include/dtr.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch provides device memory (fields, workspaces) and the current
stream.  Fields are torch.complex128 CUDA tensors of shape (nrhs, N), i.e.
the C ABI's column-major N x nrhs block (column j = row j here), N = 12 V,
dof i = 12*site + 3*spin + colour.

There is no fallback: if the shared library is missing or fails to load,
importing this module raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libdtr.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libdtr.so not built: run `python -m paper_1603_05988_gb300.build` "
                      "(or __graft_entry__.build()) first")
_lib = ctypes.CDLL(LIB_PATH)

# ---------------------------------------------------------------- C structs
DTR_OK, DTR_EINVAL, DTR_ENOMEM, DTR_ECUDA, DTR_ENOTCONV, DTR_ENAN, DTR_ETIMEOUT = range(7)
DTR_F64, DTR_F32, DTR_BF16, DTR_F16, DTR_DF32 = range(5)
SOLVER_F64, SOLVER_MIXED_F32, SOLVER_FGMRES_NET, SOLVER_MIXED_F16, SOLVER_MIXED_BF16 = 0, 1, 2, 3, 4
_PREC = {"f64": DTR_F64, "f32": DTR_F32, "bf16": DTR_BF16, "f16": DTR_F16, "df32": DTR_DF32}
_SOLVER = {"f64": SOLVER_F64, "mixed_f32": SOLVER_MIXED_F32, "fgmres_net": SOLVER_FGMRES_NET,
           "mixed_f16": SOLVER_MIXED_F16, "mixed_bf16": SOLVER_MIXED_BF16}


class SolveParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("solver", ctypes.c_int),
                ("check_every", ctypes.c_int), ("inner_tol", ctypes.c_double), ("engine", ctypes.c_int),
                ("grid", ctypes.c_int), ("net", ctypes.c_void_p), ("gmres_m", ctypes.c_int), ("no_graph", ctypes.c_int)]


class SolveStat(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("converged", ctypes.c_int),
                ("pad_", ctypes.c_int), ("true_residual", ctypes.c_double)]


class TraceParams(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("z0_first", ctypes.c_int64), ("n_z0", ctypes.c_int),
                ("ncolors", ctypes.c_int), ("nvec", ctypes.c_int), ("dilute12", ctypes.c_int),
                ("block", ctypes.c_int), ("use_x0", ctypes.c_int), ("solve", SolveParams), ("lanes", ctypes.c_int),
                ("n_gamma", ctypes.c_int), ("gamma", ctypes.c_int * 16), ("vec_first", ctypes.c_int64)]


class TraceResult(ctypes.Structure):
    _fields_ = [("trace", ctypes.c_double * 2), ("T_D", ctypes.c_double * 2), ("var_runs", ctypes.c_double),
                ("jk_err", ctypes.c_double), ("var_samples", ctypes.c_double), ("n_solves", ctypes.c_int64),
                ("iterations", ctypes.c_int64), ("max_true_residual", ctypes.c_double),
                ("all_converged", ctypes.c_int), ("pad_", ctypes.c_int),
                ("samples", ctypes.POINTER(ctypes.c_double)), ("trace_runs", ctypes.POINTER(ctypes.c_double)),
                ("replay", ctypes.POINTER(ctypes.c_double)), ("gamma_samples", ctypes.POINTER(ctypes.c_double)),
                ("gamma_trace", ctypes.c_double * 32), ("gamma_T_D", ctypes.c_double * 32),
                ("gamma_var_runs", ctypes.c_double * 16), ("gamma_jk_err", ctypes.c_double * 16),
                ("frob2", ctypes.c_double), ("frob2_err", ctypes.c_double)]


class EigParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("p", ctypes.c_int), ("degree", ctypes.c_int), ("first_degree", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("chunk", ctypes.c_int), ("store", ctypes.c_int), ("tol_ref", ctypes.c_int),
                ("tol", ctypes.c_double), ("first_cut", ctypes.c_double), ("time_limit_s", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class EigStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("basis", ctypes.c_int),
                ("pad_", ctypes.c_int), ("max_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("cut", ctypes.c_double), ("bound", ctypes.c_double), ("t_filter", ctypes.c_double),
                ("t_gram", ctypes.c_double), ("t_host", ctypes.c_double), ("t_rotate", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int), ("block", ctypes.c_int), ("rhs_per_s", ctypes.c_double),
                ("n_tried", ctypes.c_int), ("cached", ctypes.c_int), ("table_lanes", ctypes.c_int * 16),
                ("table_block", ctypes.c_int * 16), ("table_rhs_per_s", ctypes.c_double * 16)]


_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i = ctypes.c_int
_d = ctypes.c_double
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("dtr_last_error", ctypes.c_char_p, [])
_sig("dtr_version", ctypes.c_char_p, [])
_sig("dtr_kernel_launches", ctypes.c_uint64, [])
_sig("dtr_half_link_rows", ctypes.c_int, [])
_sig("dtr_tensor_core_contractions", ctypes.c_uint64, [])
_sig("dtr_time_deflate_workspace_bytes", ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int])
_sig("dtr_time_deflate", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.c_size_t, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p])
_sig("dtr_graph_stats", ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)])
_sig("dtr_profile_persistent", _i, [_i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64),
                                    ctypes.POINTER(ctypes.c_double)])
_sig("dtr_time_dslash", _i, [_vp, _d, _i, _i, _i, _vp, _sz, ctypes.POINTER(ctypes.c_double), _vp])
_sig("dtr_selftest_barrier", _i, [_i64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _vp])
_sig("dtr_make_lattice", _i, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_vp)])
_sig("dtr_destroy_lattice", None, [_vp])
_sig("dtr_lattice_info", _i, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_i64), ctypes.POINTER(_i64)])
_sig("dtr_make_gauge", _i, [_vp, _d, _u64, ctypes.POINTER(_vp)])
_sig("dtr_gauge_from_host", _i, [_vp, _vp, ctypes.POINTER(_vp)])
_sig("dtr_gauge_to_host", _i, [_vp, _vp])
_sig("dtr_destroy_gauge", None, [_vp])
_sig("dtr_dslash_workspace_bytes", _sz, [_vp, _i])
_sig("dtr_dslash", _i, [_vp, _d, _vp, _vp, _i, _i, _i, _vp, _sz, _vp])
_sig("dtr_gen_noise", _i, [_vp, _u64, _i64, _i, _i, _i64, _i, _vp, _vp])
_sig("dtr_solve_params_default", None, [ctypes.POINTER(SolveParams)])
_sig("dtr_solve_workspace_bytes", _sz, [_vp, _i, ctypes.POINTER(SolveParams)])
_sig("dtr_solve_batch", _i, [_vp, _d, _vp, _vp, _i, ctypes.POINTER(SolveParams), _vp, _sz,
                             ctypes.POINTER(SolveStat), _vp])
_sig("dtr_defl_create", _i, [_vp, _i, _i, _vp, _vp, ctypes.POINTER(_vp)])
_sig("dtr_defl_trace", _i, [_vp, ctypes.POINTER(ctypes.c_double)])
_sig("dtr_destroy_defl", None, [_vp])
_sig("dtr_deflate_workspace_bytes", _sz, [_vp, _i])
_sig("dtr_deflate_project", _i, [_vp, _vp, _i, _vp, _vp, _vp, _vp, _sz, _vp])
_sig("dtr_deflate_project_static", _i, [_vp, _vp, _i, _vp, _vp, _vp])
_sig("dtr_net_create", _i, [_vp, _i, _vp, _d, _d, _u64, ctypes.POINTER(_vp)])
_sig("dtr_destroy_net", None, [_vp])
_sig("dtr_net_get_weights", _i, [_vp, _i, _vp])
_sig("dtr_net_set_precision", _i, [_vp, _i])
_sig("dtr_net_workspace_bytes", _sz, [_vp, _i])
_sig("dtr_net_apply", _i, [_vp, _vp, _vp, _i, _vp, _sz, _vp])
_sig("dtr_net_train_step", _i, [_vp, _vp, _d, _vp, _vp, _i, _d, _i, ctypes.POINTER(ctypes.c_double), _vp, _vp, _sz,
                                _vp])
_sig("dtr_trace_workspace_bytes", _sz, [_vp, _vp, ctypes.POINTER(TraceParams)])
_sig("dtr_trace_estimate", _i, [_vp, _d, _vp, ctypes.POINTER(TraceParams), _vp, _sz,
                                ctypes.POINTER(TraceResult), _vp])
_sig("dtr_wd", _i, [_vp, _vp, _vp, _i, _i, _i, _vp, _vp])
_sig("dtr_defl_gram", _i, [_vp, _vp, _d, _vp])
_sig("dtr_eig_params_default", None, [ctypes.POINTER(EigParams)])
_sig("dtr_eig_workspace_bytes", _sz, [_vp, ctypes.POINTER(EigParams)])
_sig("dtr_eig_deflation", _i, [_vp, _d, ctypes.POINTER(EigParams), _vp, _sz, _vp, ctypes.POINTER(EigStats),
                               ctypes.POINTER(_vp), _vp])
_sig("dtr_defl_to_host", _i, [_vp, _vp, _vp])
_sig("dtr_trace_autotune_workspace_bytes", _sz, [_vp, _vp, ctypes.POINTER(TraceParams)])
_sig("dtr_trace_autotune", _i, [_vp, _d, _vp, ctypes.POINTER(TraceParams), _i, _i, _vp, _sz,
                                ctypes.POINTER(TuneResult), _vp])


class DtrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dtr error %d: %s" % (code, msg))
        self.code = code


def _check(rc, allow=()):
    if rc != DTR_OK and rc not in allow:
        raise DtrError(rc, _lib.dtr_last_error().decode())
    return rc


def version():
    return _lib.dtr_version().decode()


def _torch():
    import torch
    return torch


def _stream():
    return _vp(_torch().cuda.current_stream().cuda_stream)


def _workspace(nbytes):
    torch = _torch()
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")


def _ptr(t):
    return _vp(t.data_ptr())


def _field(t, N, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.complex128):
        raise TypeError("%s must be a CUDA complex128 tensor" % name)
    if t.dim() == 1:
        t = t.reshape(1, -1)
    if t.shape[-1] != N or not t.is_contiguous():
        raise ValueError("%s must be contiguous with shape (nrhs, %d)" % (name, N))
    return t


# ------------------------------------------------------------------- handles
class Lattice:
    def __init__(self, dims):
        d = (ctypes.c_int * 4)(*[int(x) for x in dims])
        h = _vp()
        _check(_lib.dtr_make_lattice(d, ctypes.byref(h)))
        self._h = h
        self.dims = tuple(int(x) for x in dims)
        self.V = int(np.prod(self.dims))
        self.N = 12 * self.V

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.dtr_destroy_lattice(self._h)
            self._h = None


def make_lattice(dims):
    return Lattice(dims)


class Gauge:
    """Gauge field handle: links uploaded from host (`links`, shape (V, 4, 3, 3)
    complex128) or generated on the device from (eps, seed)."""

    def __init__(self, lat, links=None, eps=None, seed=None):
        h = _vp()
        if links is not None:
            links = np.ascontiguousarray(links, dtype=np.complex128)
            if links.shape != (lat.V, 4, 3, 3):
                raise ValueError("links must have shape (V, 4, 3, 3)")
            _check(_lib.dtr_gauge_from_host(lat._h, links.ctypes.data_as(_vp), ctypes.byref(h)))
        else:
            _check(_lib.dtr_make_gauge(lat._h, float(eps), int(seed), ctypes.byref(h)))
        self._h = h
        self.lat = lat

    def to_host(self):
        out = np.empty((self.lat.V, 4, 3, 3), dtype=np.complex128)
        _check(_lib.dtr_gauge_to_host(self._h, out.ctypes.data_as(_vp)))
        return out

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.dtr_destroy_gauge(self._h)
            self._h = None


def make_gauge(lat, eps, seed):
    """Random SU(3) field U = exp(i eps H) generated on the device (dtr_make_gauge)."""
    return Gauge(lat, eps=eps, seed=seed)


def gauge_from_host(lat, links):
    """Gauge field uploaded from host links of shape (V, 4, 3, 3) (dtr_gauge_from_host)."""
    return Gauge(lat, links=links)


def dslash(gauge, m0, x, dagger=False, prec="f64"):
    """out = A x (or A^H x) for x of shape (nrhs, N), nrhs <= 64."""
    torch = _torch()
    lat = gauge.lat
    x = _field(x, lat.N, "x")
    nrhs = x.shape[0]
    out = torch.empty_like(x)
    nb = _lib.dtr_dslash_workspace_bytes(lat._h, nrhs)
    w = _workspace(nb)
    _check(_lib.dtr_dslash(gauge._h, float(m0), _ptr(x), _ptr(out), nrhs, int(bool(dagger)), _PREC[prec],
                           _ptr(w), nb, _stream()))
    return out


def dslash_many(gauge, m0, X, dagger=False, prec="f64", chunk=64):
    """dslash over any number of rows of X (chunks of <= 64 right-hand sides)."""
    torch = _torch()
    out = torch.empty_like(X)
    for c0 in range(0, X.shape[0], chunk):
        out[c0:c0 + chunk] = dslash(gauge, m0, X[c0:c0 + chunk].contiguous(), dagger=dagger, prec=prec)
    return out


def selftest_barrier(budget_cycles=2_000_000):
    """Run the bounded-barrier self-test; returns (timed_out, error_word)."""
    t = ctypes.c_int()
    e = ctypes.c_int()
    _check(_lib.dtr_selftest_barrier(int(budget_cycles), ctypes.byref(t), ctypes.byref(e), _stream()))
    return t.value, e.value


def profile_persistent(enable=-1):
    """Read (and with enable 0/1 reset and switch) persistent-kernel accounting:
    returns dict(ms, launches, site_rhs_iterations)."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    w = ctypes.c_double()
    _check(_lib.dtr_profile_persistent(int(enable), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
    return {"ms": ms.value, "launches": n.value, "site_rhs_iterations": w.value}


def tensor_core_contractions():
    """Deflation contractions that ran on the tensor cores so far in this process."""
    return int(_lib.dtr_tensor_core_contractions())


def time_deflate(defl, nrhs, reps=20):
    """Average duration (ms) of one deflation contraction of an nrhs-column Z4 block
    (tensor cores for a BF16-stored deflation space), CUDA events on the current stream."""
    nb = _lib.dtr_time_deflate_workspace_bytes(defl._h, int(nrhs))
    w = _workspace(nb)
    ms = ctypes.c_double()
    _check(_lib.dtr_time_deflate(defl._h, int(nrhs), int(reps), _ptr(w), nb, ctypes.byref(ms), _stream()))
    return ms.value


def half_link_rows():
    """Rows per link the half-precision stencil stores (3, or 2 with the third rebuilt)."""
    return int(_lib.dtr_half_link_rows())


def kernel_launches():
    """Kernels the library launched so far in this process (host-launched kernels
    plus the kernels of device-driven graph loops, which the device counts)."""
    return int(_lib.dtr_kernel_launches())


def graph_stats():
    """(graphs captured, graph launches) of the graph-driven mixed solver."""
    c, l = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(_lib.dtr_graph_stats(ctypes.byref(c), ctypes.byref(l)))
    return int(c.value), int(l.value)


def time_dslash(gauge, m0, nrhs, prec="f32", reps=50):
    """Average duration (ms) of one internal dslash launch of width nrhs (CUDA events)."""
    nb = _lib.dtr_dslash_workspace_bytes(gauge.lat._h, nrhs)
    w = _workspace(nb)
    ms = ctypes.c_double()
    _check(_lib.dtr_time_dslash(gauge._h, float(m0), int(nrhs), _PREC[prec], int(reps), _ptr(w), nb,
                                ctypes.byref(ms), _stream()))
    return ms.value


def gen_noise(lat, seed, z0_index, ncolors, dilute12, q0, nrhs):
    """Probing vectors z = z0 .* z_h, shape (nrhs, N) complex128 on the GPU."""
    torch = _torch()
    out = torch.empty((nrhs, lat.N), dtype=torch.complex128, device="cuda")
    _check(_lib.dtr_gen_noise(lat._h, int(seed), int(z0_index), int(ncolors), int(bool(dilute12)), int(q0),
                              int(nrhs), _ptr(out), _stream()))
    return out


_ENGINE = {"persistent": 0, "kernels": 1}


def solve_params(tol=1e-10, maxiter=5000, solver="f64", check_every=8, inner_tol=1e-5, engine="persistent",
                 grid=0, net=None, gmres_m=16, graph=True):
    """dtr_solve_params.  solver: "f64" (plain FP64 BiCGStab), "mixed_f32",
    "mixed_f16", "mixed_bf16" (inner BiCGStab with FP32, FP16 or BF16 Krylov
    vectors in FP64 defect correction; the half-storage ones need the
    persistent engine) or "fgmres_net" (FGMRES(gmres_m) with the network `net`,
    None = unpreconditioned).  engine: "persistent" (one cooperative launch per
    (inner) solve) or "kernels" (one kernel per BiCGStab step).  graph: run the
    mixed defect-correction loop as one CUDA graph (persistent engine)."""
    p = SolveParams()
    _lib.dtr_solve_params_default(ctypes.byref(p))
    p.tol, p.maxiter, p.solver, p.check_every, p.inner_tol = tol, maxiter, _SOLVER[solver], check_every, inner_tol
    p.engine = _ENGINE[engine]
    p.grid = int(grid)
    p.net = net._h.value if net is not None else None
    p.gmres_m = int(gmres_m)
    p.no_graph = 0 if graph else 1
    return p


NET_WEIGHTS = 4 * 81 * 24 * 24


class Net:
    """Learned preconditioner network (4 layers, 3^4 stencil, 24 real channels).
    precision "bf16": BF16 layer inputs and gradients, tensor-core convolutions;
    "f32": FP32 fields, CUDA-core convolutions."""

    def __init__(self, lat, act=0, weights=None, init_scale=1.0, noise=0.0, seed=0, precision="bf16"):
        h = _vp()
        wp = None
        if weights is not None:
            wa = np.ascontiguousarray(weights, dtype=np.float32).reshape(-1)
            if wa.size != NET_WEIGHTS:
                raise ValueError("weights must have 4*81*24*24 entries")
            self._w = wa
            wp = wa.ctypes.data_as(_vp)
        _check(_lib.dtr_net_create(lat._h, int(act), wp, float(init_scale), float(noise), int(seed), ctypes.byref(h)))
        self._h = h
        self.lat = lat
        self.act = act
        self.set_precision(precision)

    def set_precision(self, precision):
        _check(_lib.dtr_net_set_precision(self._h, _PREC[precision]))
        self.precision = precision

    def weights(self, bf16_rounded=False):
        out = np.empty(NET_WEIGHTS, dtype=np.float32)
        _check(_lib.dtr_net_get_weights(self._h, int(bool(bf16_rounded)), out.ctypes.data_as(_vp)))
        return out.reshape(4, 81, 24, 24)

    def apply(self, x):
        torch = _torch()
        x = _field(x, self.lat.N, "x")
        out = torch.empty_like(x)
        nb = _lib.dtr_net_workspace_bytes(self._h, x.shape[0])
        w = _workspace(nb)
        _check(_lib.dtr_net_apply(self._h, _ptr(x), _ptr(out), x.shape[0], _ptr(w), nb, _stream()))
        return out

    def train_step(self, x, target, lr=1e-3, step=True, want_grad=False, gauge=None, m0=0.0):
        """One Adam step on pairs (x, target) with A target = x; residual-weighted
        loss |A M x - x|^2 / |x|^2 if a gauge field is given, else the error loss."""
        x = _field(x, self.lat.N, "x")
        target = _field(target, self.lat.N, "target")
        nb = _lib.dtr_net_workspace_bytes(self._h, x.shape[0])
        w = _workspace(nb)
        loss = ctypes.c_double()
        grad = np.empty(NET_WEIGHTS, dtype=np.float32) if want_grad else None
        _check(_lib.dtr_net_train_step(self._h, gauge._h if gauge is not None else None, float(m0), _ptr(x),
                                       _ptr(target), x.shape[0], float(lr), int(bool(step)), ctypes.byref(loss),
                                       grad.ctypes.data_as(_vp) if grad is not None else None, _ptr(w), nb,
                                       _stream()))
        return (loss.value, grad.reshape(4, 81, 24, 24)) if want_grad else loss.value

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.dtr_destroy_net(self._h)
            self._h = None


def solve_batch(gauge, m0, z, y0=None, params=None, allow_notconv=False):
    """Solve A y = z for z of shape (nrhs, N); returns (y, stats list of dicts)."""
    torch = _torch()
    lat = gauge.lat
    z = _field(z, lat.N, "z")
    nrhs = z.shape[0]
    y = torch.zeros_like(z) if y0 is None else _field(y0, lat.N, "y0").clone()
    p = params if params is not None else solve_params()
    nb = _lib.dtr_solve_workspace_bytes(lat._h, nrhs, ctypes.byref(p))
    w = _workspace(nb)
    st = (SolveStat * nrhs)()
    rc = _lib.dtr_solve_batch(gauge._h, float(m0), _ptr(z), _ptr(y), nrhs, ctypes.byref(p), _ptr(w), nb, st,
                              _stream())
    _check(rc, allow=(DTR_ENOTCONV,) if allow_notconv else ())
    stats = [dict(iterations=s.iterations, restarts=s.restarts, converged=bool(s.converged), flags=s.pad_,
                  true_residual=s.true_residual) for s in st]
    return y, stats


class Deflation:
    def __init__(self, lat, V, lam, prec="f64", handle=None, k=None):
        if handle is not None:            # a space the library built on the device
            self._h, self.lat, self.k = handle, lat, int(k)
            return
        V = np.asarray(V, dtype=np.complex128)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        if V.ndim != 2 or V.shape[0] != lat.N or V.shape[1] != lam.shape[0]:
            raise ValueError("V must be (N, k) and lambda (k,)")
        k = V.shape[1]
        Vc = np.asfortranarray(V)   # column-major N x k
        h = _vp()
        _check(_lib.dtr_defl_create(lat._h, k, _PREC[prec], Vc.ctypes.data_as(_vp), lam.ctypes.data_as(_vp),
                                    ctypes.byref(h)))
        self._h = h
        self.lat = lat
        self.k = k

    def gram(self, gauge, m0):
        """Switch to the Galerkin form D = V (V^H g5 A V)^-1 V^H g5 (computed on the GPU in FP64)."""
        _check(_lib.dtr_defl_gram(self._h, gauge._h, float(m0), _stream()))
        return self

    def to_host(self):
        """(V (N, k) complex128, lambda (k,)): the stored space, widened exactly."""
        V = np.empty((self.k, self.lat.N), dtype=np.complex128)
        lam = np.empty(self.k)
        _check(_lib.dtr_defl_to_host(self._h, V.ctypes.data_as(_vp), lam.ctypes.data_as(_vp)))
        return V.T, lam

    def lambdas(self):
        """The k signed eigenvalues (host), without copying V."""
        lam = np.empty(self.k)
        _check(_lib.dtr_defl_to_host(self._h, None, lam.ctypes.data_as(_vp)))
        return lam

    def T_D(self):
        td = (ctypes.c_double * 2)()
        _check(_lib.dtr_defl_trace(self._h, td))
        return complex(td[0], td[1])

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.dtr_destroy_defl(self._h)
            self._h = None


def defl_create(lat, V, lam, prec="f64"):
    return Deflation(lat, V, lam, prec)


def eig_params(k, p=0, degree=48, first_degree=0, max_iter=100, chunk=32, store="f64", tol=1e-2, first_cut=0.0,
               time_limit_s=0.0, seed=0, tol_ref="lambda"):
    """dtr_eig_params; tol_ref "lambda" (residual relative to |lambda_j|) or "norm" (relative to the
    bound on ||A||)."""
    q = EigParams()
    q.tol_ref = {"lambda": 0, "norm": 1}[tol_ref]
    _lib.dtr_eig_params_default(ctypes.byref(q))
    q.k, q.p, q.degree, q.first_degree, q.max_iter, q.chunk = int(k), int(p), int(degree), int(first_degree), \
        int(max_iter), int(chunk)
    q.store, q.tol, q.first_cut, q.time_limit_s, q.seed = _PREC[store], float(tol), float(first_cut), \
        float(time_limit_s), int(seed)
    return q


def eig_deflation(gauge, m0, params):
    """The k smallest-|lambda| eigenpairs of g5 A computed on the device (dtr_eig_deflation).
    Returns (Deflation, relative residuals (k,), stats dict)."""
    nb = _lib.dtr_eig_workspace_bytes(gauge.lat._h, ctypes.byref(params))
    if nb == 0:
        raise DtrError(DTR_EINVAL, "bad eigensolver parameters")
    w = _workspace(nb)
    res = np.zeros(params.k)
    st = EigStats()
    h = _vp()
    _check(_lib.dtr_eig_deflation(gauge._h, float(m0), ctypes.byref(params), _ptr(w), nb,
                                  res.ctypes.data_as(_vp), ctypes.byref(st), ctypes.byref(h), _stream()))
    del w
    stats = dict(iterations=st.iterations, converged=st.converged, basis=st.basis, max_residual=st.max_residual,
                 seconds=st.seconds, cut=st.cut, bound=st.bound, workspace_bytes=int(nb),
                 t_filter=st.t_filter, t_gram=st.t_gram, t_host=st.t_host, t_rotate=st.t_rotate)
    return Deflation(gauge.lat, None, None, handle=h, k=params.k), res, stats


def deflate_project(defl, z, want_coeff=False, want_x0=False):
    """Returns (d, C or None, x0 or None): d_j = z_j^H V diag(1/lambda) V^H g5 z_j."""
    torch = _torch()
    lat = defl.lat
    z = _field(z, lat.N, "z")
    nrhs = z.shape[0]
    d = torch.empty(nrhs, dtype=torch.complex128, device="cuda")
    C = torch.empty((2 * nrhs, defl.k), dtype=torch.complex128, device="cuda") if want_coeff else None
    x0 = torch.empty_like(z) if want_x0 else None
    nb = _lib.dtr_deflate_workspace_bytes(defl._h, nrhs)
    w = _workspace(nb)
    _check(_lib.dtr_deflate_project(defl._h, _ptr(z), nrhs, _ptr(d), _ptr(C) if C is not None else None,
                                    _ptr(x0) if x0 is not None else None, _ptr(w), nb, _stream()))
    return d, C, x0


STATIC_MAX_K, STATIC_MAX_RHS = 128, 16


def deflate_project_static(defl, z, want_coeff=False):
    """Allocation-free deflation projection (the library uses a fixed device
    array as scratch; no workspace, no device allocation by the library).
    Returns (d, C or None) like deflate_project.  nrhs <= 16, k <= 128."""
    torch = _torch()
    z = _field(z, defl.lat.N, "z")
    nrhs = z.shape[0]
    d = torch.empty(nrhs, dtype=torch.complex128, device="cuda")
    C = torch.empty((2 * nrhs, defl.k), dtype=torch.complex128, device="cuda") if want_coeff else None
    _check(_lib.dtr_deflate_project_static(defl._h, _ptr(z), nrhs, _ptr(d), _ptr(C) if C is not None else None,
                                           _stream()))
    return d, C


def trace_params(seed=0, z0_first=0, n_z0=1, ncolors=1, nvec=1, dilute12=False, block=16, use_x0=False,
                 solve=None, lanes=1, gammas=(), vec_first=0):
    """dtr_trace_params; vec_first: first probing (Hadamard) vector of each run used by this call."""
    p = TraceParams()
    p.vec_first = int(vec_first)
    p.seed, p.z0_first, p.n_z0, p.ncolors, p.nvec = int(seed), int(z0_first), int(n_z0), int(ncolors), int(nvec)
    p.dilute12, p.block, p.use_x0 = int(bool(dilute12)), int(block), int(bool(use_x0))
    p.solve = solve if solve is not None else solve_params()
    p.lanes = int(lanes)
    gammas = list(gammas)
    if len(gammas) > 16:
        raise ValueError("at most 16 Gamma matrices")
    p.n_gamma = len(gammas)
    for q, n in enumerate(gammas):
        p.gamma[q] = int(n)
    return p


class TraceWorkspace:
    """Reusable device workspace for repeated trace_estimate calls."""

    def __init__(self, gauge, defl, params):
        self.nbytes = _lib.dtr_trace_workspace_bytes(gauge._h, defl._h if defl else None, ctypes.byref(params))
        self.buf = _workspace(self.nbytes)


def wd(lat, cols, dofs, maxd, ncolors=0):
    """W_d (d = 0..maxd) of the matrix whose columns B e_i for the sampled dofs are
    `cols` (device, shape (ns, N) complex128, row q = column of dofs[q])."""
    cols = _field(cols, lat.N, "cols")
    dofs = np.ascontiguousarray(dofs, dtype=np.int64)
    if cols.shape[0] != dofs.shape[0]:
        raise ValueError("one column per sampled dof")
    W = np.zeros(int(maxd) + 1)
    _check(_lib.dtr_wd(lat._h, _ptr(cols), dofs.ctypes.data_as(_vp), int(dofs.shape[0]), int(maxd), int(ncolors),
                       W.ctypes.data_as(_vp), _stream()))
    return W


def trace_autotune(gauge, m0, defl, params, reps=3, force=False, max_workspace_bytes=None):
    """Time the candidate launch shapes (lanes; RHS block too if params.block <= 0)
    and return a dict with the fastest ("lanes", "block", "rhs_per_s") and the
    table of candidates; the choice is cached per problem shape.  With
    max_workspace_bytes the workspace is capped there and candidates that need
    more are skipped."""
    nb = _lib.dtr_trace_autotune_workspace_bytes(gauge._h, defl._h if defl else None, ctypes.byref(params))
    if nb == 0:
        raise DtrError(DTR_EINVAL, "bad autotune parameters")
    if max_workspace_bytes is not None:
        nb = min(nb, int(max_workspace_bytes))
    w = _workspace(nb)
    r = TuneResult()
    _check(_lib.dtr_trace_autotune(gauge._h, float(m0), defl._h if defl else None, ctypes.byref(params), int(reps),
                                   int(bool(force)), _ptr(w), nb, ctypes.byref(r), _stream()))
    table = [dict(lanes=r.table_lanes[i], block=r.table_block[i], rhs_per_s=r.table_rhs_per_s[i])
             for i in range(r.n_tried)]
    return dict(lanes=r.lanes, block=r.block, rhs_per_s=r.rhs_per_s, cached=bool(r.cached), table=table)


def trace_estimate(gauge, m0, defl, params, workspace=None, want_samples=True, want_replay=False,
                   allow_notconv=False):
    """Algorithm 1 over params.n_z0 runs; returns a dict of results."""
    R, s = params.n_z0, params.nvec
    k = defl.k if defl is not None else 0
    ws = workspace if workspace is not None else TraceWorkspace(gauge, defl, params)
    res = TraceResult()
    samples = np.zeros(2 * R * s) if want_samples else None
    runs = np.zeros(2 * R)
    replay = np.zeros(2 * R * s * max(k, 1)) if (want_replay and k) else None
    dp = ctypes.POINTER(ctypes.c_double)
    res.samples = samples.ctypes.data_as(dp) if samples is not None else None
    res.trace_runs = runs.ctypes.data_as(dp)
    res.replay = replay.ctypes.data_as(dp) if replay is not None else None
    ng = params.n_gamma
    gsamp = np.zeros(2 * ng * R * s) if (ng and want_samples) else None
    res.gamma_samples = gsamp.ctypes.data_as(dp) if gsamp is not None else None
    rc = _lib.dtr_trace_estimate(gauge._h, float(m0), defl._h if defl is not None else None, ctypes.byref(params),
                                 _ptr(ws.buf), ws.nbytes, ctypes.byref(res), _stream())
    _check(rc, allow=(DTR_ENOTCONV,) if allow_notconv else ())
    out = dict(trace=complex(res.trace[0], res.trace[1]), T_D=complex(res.T_D[0], res.T_D[1]),
               var_runs=res.var_runs, jk_err=res.jk_err, var_samples=res.var_samples, n_solves=res.n_solves,
               iterations=res.iterations, max_true_residual=res.max_true_residual,
               all_converged=bool(res.all_converged), status=rc,
               trace_runs=runs[0::2] + 1j * runs[1::2], frob2=res.frob2, frob2_err=res.frob2_err)
    if samples is not None:
        out["samples"] = (samples[0::2] + 1j * samples[1::2]).reshape(R, s)
    if replay is not None:
        out["replay"] = (replay[0::2] + 1j * replay[1::2]).reshape(R, s, k)
    if ng:
        gam = []
        for q in range(ng):
            d = dict(n=int(params.gamma[q]), trace=complex(res.gamma_trace[2 * q], res.gamma_trace[2 * q + 1]),
                     T_D=complex(res.gamma_T_D[2 * q], res.gamma_T_D[2 * q + 1]),
                     var_runs=res.gamma_var_runs[q], jk_err=res.gamma_jk_err[q])
            if gsamp is not None:
                g = gsamp[2 * q * R * s:2 * (q + 1) * R * s]
                d["samples"] = (g[0::2] + 1j * g[1::2]).reshape(R, s)
            gam.append(d)
        out["gamma"] = gam
    return out
