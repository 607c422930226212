"""Thin ctypes binding of the RT-TDA C ABI (include/rttda.h).

The functions below carry the ABI's names and only marshal arguments:
numpy arrays for host buffers, integer device addresses (e.g.
``tensor.data_ptr()``) for device buffers.  Every step of the propagation
runs in the library's CUDA kernels; if the shared library is missing this
module raises on import instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librttda.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"RT-TDA CUDA library not built: {LIB_PATH} is missing "
                      "(run paper_2601_16949_b300/build.py)")

lib = ct.CDLL(LIB_PATH)

# status codes (rttda_status)
OK, E_ARG, E_OOM, E_CUDA, E_TIMEOUT, E_STATE, E_BUSY = range(7)
STATUS_NAMES = {0: "OK", 1: "E_ARG", 2: "E_OOM", 3: "E_CUDA", 4: "E_TIMEOUT", 5: "E_STATE", 6: "E_BUSY"}
# precisions (rttda_prec)
FP64, FP32, TF32, BF16, BF16X3, BF16X2, FP64_OZ = 0, 1, 2, 3, 4, 5, 6
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16": BF16, "bf16x3": BF16X3, "bf16x2": BF16X2,
              "fp64oz": FP64_OZ}
# pulse kinds (rttda_pulse_kind)
KICK, CW, GAUSS_TL, CHIRP, SIN2 = 0, 1, 2, 3, 4


class rttda_pulse(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("E0", ct.c_double), ("omega", ct.c_double), ("t0", ct.c_double),
                ("fwhm", ct.c_double), ("beta", ct.c_double), ("duration", ct.c_double),
                ("dir", ct.c_double * 3)]


class rttda_request(ct.Structure):
    _fields_ = [("nocc", ct.c_int), ("nvirt", ct.c_int), ("naux", ct.c_int)] + \
               [(n, ct.POINTER(ct.c_double)) for n in ("eps_occ", "eps_virt", "B_ov", "B_oo", "B_vv", "mu_oo",
                                                        "mu_vv", "mu_0ov")] + \
               [("c_x", ct.c_double), ("prec", ct.c_int), ("pulse", rttda_pulse), ("dt", ct.c_double),
                ("nsteps", ct.c_long), ("gamma", ct.c_double), ("wmin", ct.c_double), ("wmax", ct.c_double),
                ("nfreq", ct.c_long), ("factors_on_device", ct.c_int)]


class rttda_server_stats(ct.Structure):
    _fields_ = [(n, ct.c_long) for n in ("submitted", "completed", "failed", "cancelled", "pending", "active")] + \
               [("max_concurrent", ct.c_int), ("trajectory_steps", ct.c_double), ("p50_latency_s", ct.c_double),
                ("p99_latency_s", ct.c_double), ("mean_latency_s", ct.c_double), ("busy_seconds", ct.c_double),
                ("bytes_in_use", ct.c_size_t), ("bytes_budget", ct.c_size_t), ("grouped", ct.c_long)]


class rttda_plan_info(ct.Structure):
    _fields_ = [(n, ct.c_int) for n in ("prec", "ntraj", "main_kernel", "main_bn", "main_mb", "main_kb",
                                        "main_splits", "z_chunk", "coulomb_kernel", "tuned", "ncand")] + \
               [("tune_ms", ct.c_double * 8), ("main_cluster", ct.c_int), ("main_grid", ct.c_int)]


REQ_PENDING, REQ_ACTIVE, REQ_DONE, REQ_FAILED, REQ_CANCELLED = range(5)


class RTTDAError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.rttda_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


_dp = ct.POINTER(ct.c_double)
_h = ct.c_void_p

lib.rttda_abi_version.restype = ct.c_int
lib.rttda_last_error.restype = ct.c_char_p
lib.rttda_create.argtypes = [ct.c_int, ct.c_int, ct.c_int] + [_dp] * 8 + [ct.c_double, ct.c_int, ct.POINTER(_h)]
lib.rttda_create.restype = ct.c_int
lib.rttda_memory_bytes.argtypes = [_h, ct.POINTER(ct.c_size_t)]
lib.rttda_create_device.argtypes = [ct.c_int, ct.c_int, ct.c_int] + [ct.c_void_p] * 8 + [ct.c_double, ct.c_int,
                                                                                          ct.POINTER(_h)]
lib.rttda_create_device.restype = ct.c_int
lib.rttda_set_field.argtypes = [_h, ct.POINTER(rttda_pulse), ct.c_int]
lib.rttda_propagate.argtypes = [_h, _dp, ct.c_double, ct.c_long, _dp, _dp, _dp]
lib.rttda_propagate_device.argtypes = [_h, ct.c_void_p, ct.c_double, ct.c_long, ct.c_void_p, ct.c_void_p,
                                       ct.c_void_p, ct.c_void_p]
lib.rttda_resume.argtypes = [_h, ct.c_double, ct.c_long, _dp, _dp, _dp]
lib.rttda_get_state.argtypes = [_h, _dp, _dp]
lib.rttda_set_state.argtypes = [_h, _dp, ct.c_double]
lib.rttda_sigma.argtypes = [_h, ct.c_void_p, ct.c_double, ct.c_void_p, ct.c_void_p]
lib.rttda_spectrum.argtypes = [_dp, ct.c_long, ct.c_long, ct.c_double, ct.c_double, ct.c_double, ct.c_double,
                               ct.c_double, ct.c_long, _dp, _dp]
lib.rttda_sync.argtypes = [_h, ct.c_void_p]
lib.rttda_profile.argtypes = [_h, ct.c_int]
lib.rttda_profile_read.argtypes = [_h, _dp, ct.POINTER(ct.c_longlong)]
lib.rttda_launch_stats.argtypes = [_h, ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong)]
lib.rttda_plan.argtypes = [_h, ct.POINTER(rttda_plan_info)]
lib.rttda_set_integrator.argtypes = [_h, ct.c_int]
lib.rttda_eigenstates.argtypes = [_h, ct.c_int, ct.c_double, ct.c_int, _dp, _dp, ct.POINTER(ct.c_int)]
lib.rttda_set_projectors.argtypes = [_h, ct.c_int, _dp]
lib.rttda_get_overlaps.argtypes = [_h, _dp, ct.c_long]
lib.rttda_set_autocorrelation.argtypes = [_h, ct.c_int]
lib.rttda_get_autocorrelation.argtypes = [_h, _dp, ct.c_long]
lib.rttda_spectrum_autocorr.argtypes = [_dp, ct.c_long, ct.c_long, ct.c_double, ct.c_long, ct.c_long, ct.c_int,
                                        _dp, _dp]
lib.rttda_coulomb_noalloc.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int,
                                      ct.c_void_p, ct.c_void_p]
lib.rttda_coulomb_noalloc.restype = ct.c_int
lib.rttda_server_create.argtypes = [ct.c_size_t, ct.c_int, ct.c_long, ct.POINTER(_h)]
lib.rttda_server_submit.argtypes = [_h, ct.POINTER(rttda_request), ct.POINTER(ct.c_long)]
lib.rttda_server_poll.argtypes = [_h, ct.c_long, ct.POINTER(ct.c_int), _dp, _dp, _dp, _dp]
lib.rttda_server_wait.argtypes = [_h, ct.c_long, ct.c_double]
lib.rttda_server_cancel.argtypes = [_h, ct.c_long]
lib.rttda_server_set_grouping.argtypes = [_h, ct.c_int]
lib.rttda_server_stats_get.argtypes = [_h, ct.POINTER(rttda_server_stats)]
lib.rttda_estimate_bytes.argtypes = [ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_long,
                                     ct.POINTER(ct.c_size_t)]
lib.rttda_server_destroy.argtypes = [_h]
lib.rttda_server_destroy.restype = None
for _name in ("rttda_server_create", "rttda_server_submit", "rttda_server_poll", "rttda_server_wait",
              "rttda_server_cancel", "rttda_server_set_grouping", "rttda_server_stats_get", "rttda_estimate_bytes"):
    getattr(lib, _name).restype = ct.c_int
lib.rttda_selftest_wait.argtypes = [ct.c_double]
lib.rttda_selftest_wait.restype = ct.c_int
lib.rttda_destroy.argtypes = [_h]
lib.rttda_destroy.restype = None
for _name in ("rttda_create", "rttda_memory_bytes", "rttda_set_field", "rttda_propagate", "rttda_propagate_device",
              "rttda_resume", "rttda_get_state", "rttda_set_state", "rttda_sigma", "rttda_spectrum",
              "rttda_profile", "rttda_profile_read", "rttda_launch_stats", "rttda_sync", "rttda_plan",
              "rttda_set_integrator", "rttda_eigenstates", "rttda_set_projectors", "rttda_get_overlaps",
              "rttda_set_autocorrelation", "rttda_get_autocorrelation", "rttda_spectrum_autocorr"):
    getattr(lib, _name).restype = ct.c_int


def _check(status: int, where: str) -> None:
    if status != OK:
        raise RTTDAError(status, where)


def _ptr(a):
    """Host pointer of a C-contiguous float64 numpy array (None -> NULL).
    An int is taken as a raw address (e.g. a pinned torch tensor's data_ptr())."""
    if a is None:
        return None
    if isinstance(a, int):
        return ct.cast(ct.c_void_p(a), _dp) if a else None
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("expected a C-contiguous float64 numpy array")
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def rttda_abi_version() -> int:
    return lib.rttda_abi_version()


def rttda_last_error() -> str:
    return lib.rttda_last_error().decode(errors="replace")


def rttda_create(nocc, nvirt, naux, eps_occ, eps_virt, B_ov, B_oo, B_vv, mu_oo, mu_vv, mu_0ov, c_x, prec):
    arrs = [_f64(x) for x in (eps_occ, eps_virt, B_ov, B_oo, B_vv, mu_oo, mu_vv, mu_0ov)]
    h = _h()
    prec = PRECISIONS.get(prec, prec) if isinstance(prec, str) else prec
    _check(lib.rttda_create(nocc, nvirt, naux, *[_ptr(a) for a in arrs], float(c_x), int(prec), ct.byref(h)),
           "rttda_create")
    return h


def rttda_create_device(nocc, nvirt, naux, ptrs, c_x, prec):
    """ptrs: device addresses of eps_occ, eps_virt, B_ov, B_oo, B_vv, mu_oo, mu_vv, mu_0ov (FP64)."""
    h = _h()
    prec = PRECISIONS.get(prec, prec) if isinstance(prec, str) else prec
    _check(lib.rttda_create_device(nocc, nvirt, naux, *[ct.c_void_p(int(p)) for p in ptrs], float(c_x), int(prec),
                                   ct.byref(h)), "rttda_create_device")
    return h


def rttda_memory_bytes(h) -> int:
    n = ct.c_size_t()
    _check(lib.rttda_memory_bytes(h, ct.byref(n)), "rttda_memory_bytes")
    return n.value


def make_pulses(pulses) -> ct.Array:
    arr = (rttda_pulse * len(pulses))()
    for k, p in enumerate(pulses):
        get = (lambda name, d=0.0: p.get(name, d)) if isinstance(p, dict) else (lambda name, d=0.0: getattr(p, name, d))
        arr[k].kind = int(get("kind", KICK))
        arr[k].E0 = float(get("E0", 0.0))
        arr[k].omega = float(get("omega", 0.0))
        arr[k].t0 = float(get("t0", 0.0))
        arr[k].fwhm = float(get("fwhm", 1.0))
        arr[k].beta = float(get("beta", 0.0))
        arr[k].duration = float(get("duration", 0.0))
        d = get("direction", None)
        if d is None:
            d = get("dir", (0.0, 0.0, 1.0))
        for x in range(3):
            arr[k].dir[x] = float(d[x])
    return arr


def rttda_set_field(h, pulses) -> None:
    arr = make_pulses(pulses)
    _check(lib.rttda_set_field(h, arr, len(pulses)), "rttda_set_field")


def rttda_propagate(h, c0, dt, nsteps, c_out=None, dipole_trace=None, norm_trace=None) -> None:
    _check(lib.rttda_propagate(h, _ptr(c0), float(dt), int(nsteps), _ptr(c_out), _ptr(dipole_trace),
                               _ptr(norm_trace)), "rttda_propagate")


def rttda_propagate_ptr(h, c0_ptr, dt, nsteps, c_out_ptr, dip_ptr, nrm_ptr) -> None:
    """rttda_propagate with raw host addresses (e.g. pinned torch tensors)."""
    cast = lambda p: None if not p else ct.cast(ct.c_void_p(p), _dp)
    _check(lib.rttda_propagate(h, cast(c0_ptr), float(dt), int(nsteps), cast(c_out_ptr), cast(dip_ptr),
                               cast(nrm_ptr)), "rttda_propagate")


def rttda_propagate_device(h, c0_dev, dt, nsteps, c_out_dev, dipole_dev, norm_dev, stream=0) -> None:
    _check(lib.rttda_propagate_device(h, c0_dev or None, float(dt), int(nsteps), c_out_dev or None,
                                      dipole_dev or None, norm_dev or None, stream or None),
           "rttda_propagate_device")


def rttda_resume(h, dt, nsteps, c_out=None, dipole_trace=None, norm_trace=None) -> None:
    _check(lib.rttda_resume(h, float(dt), int(nsteps), _ptr(c_out), _ptr(dipole_trace), _ptr(norm_trace)),
           "rttda_resume")


def rttda_get_state(h, c) -> float:
    t = ct.c_double()
    _check(lib.rttda_get_state(h, _ptr(c), ct.byref(t)), "rttda_get_state")
    return t.value


def rttda_set_state(h, c, t) -> None:
    _check(lib.rttda_set_state(h, _ptr(c), float(t)), "rttda_set_state")


def rttda_sync(h, stream=0) -> None:
    _check(lib.rttda_sync(h, stream or None), "rttda_sync")


def rttda_sigma(h, c_dev, t, sigma_dev, stream=0) -> None:
    _check(lib.rttda_sigma(h, c_dev, float(t), sigma_dev, stream or None), "rttda_sigma")


def rttda_spectrum(trace, dt, kappa, gamma, wmin, wmax, nfreq):
    tr = np.atleast_2d(_f64(trace))
    om = np.zeros(nfreq)
    S = np.zeros(nfreq)
    _check(lib.rttda_spectrum(_ptr(tr), tr.shape[0], tr.shape[1], float(dt), float(kappa), float(gamma),
                              float(wmin), float(wmax), int(nfreq), _ptr(om), _ptr(S)), "rttda_spectrum")
    return om, S


KERNEL_CLASSES = ("field", "coulomb", "exchange_z", "exchange_main", "combine", "observe", "kick")


def rttda_profile(h, enable: bool) -> None:
    _check(lib.rttda_profile(h, 1 if enable else 0), "rttda_profile")


def rttda_profile_read(h) -> dict:
    n = len(KERNEL_CLASSES)
    ms = (ct.c_double * n)()
    cnt = (ct.c_longlong * n)()
    _check(lib.rttda_profile_read(h, ms, cnt), "rttda_profile_read")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}


def rttda_launch_stats(h) -> tuple:
    tot = ct.c_longlong()
    per = ct.c_longlong()
    _check(lib.rttda_launch_stats(h, ct.byref(tot), ct.byref(per)), "rttda_launch_stats")
    return tot.value, per.value


INTEGRATORS = {"rk4": 0, "sso": 1}


def rttda_set_integrator(h, integrator) -> None:
    """'rk4' (default) or 'sso' (symplectic split operator), or the enum value."""
    code = INTEGRATORS[integrator] if isinstance(integrator, str) else int(integrator)
    _check(lib.rttda_set_integrator(h, code), "rttda_set_integrator")


def rttda_eigenstates(h, k: int, dim: int = 0, tol: float = 1e-8, max_iter: int = 200,
                      allow_unconverged: bool = False):
    """(evals[k], evecs[k][dim] or None when dim = 0, iterations): the k
    lowest TI-TDA states of A (dim = 1 + nocc * nvirt).  With
    allow_unconverged, RTTDA_E_STATE (tolerance not reached within max_iter)
    returns the last estimates and iterations = -max_iter instead of raising."""
    n = ct.c_int()
    ev = np.zeros(k)
    vecs = np.zeros((k, dim)) if dim else None
    st = lib.rttda_eigenstates(h, int(k), float(tol), int(max_iter), _ptr(ev),
                               _ptr(vecs) if vecs is not None else None, ct.byref(n))
    if allow_unconverged and st == E_STATE:
        return ev, vecs, -int(max_iter)
    _check(st, "rttda_eigenstates")
    return ev, vecs, n.value


def rttda_set_projectors(h, X) -> None:
    """Real projector vectors X[k][N] (numpy); None or an empty array removes them."""
    if X is None or len(X) == 0:
        _check(lib.rttda_set_projectors(h, 0, None), "rttda_set_projectors")
        return
    X = _f64(np.atleast_2d(X))
    _check(lib.rttda_set_projectors(h, X.shape[0], _ptr(X)), "rttda_set_projectors")


def rttda_get_overlaps(h, ntraj: int, npts: int, k: int) -> np.ndarray:
    """Complex overlaps [ntraj][npts][k] of the last propagation."""
    out = np.zeros((ntraj, npts, k, 2))
    _check(lib.rttda_get_overlaps(h, _ptr(out), int(npts)), "rttda_get_overlaps")
    return out[..., 0] + 1j * out[..., 1]


def rttda_set_autocorrelation(h, enable: bool = True) -> None:
    _check(lib.rttda_set_autocorrelation(h, 1 if enable else 0), "rttda_set_autocorrelation")


def rttda_get_autocorrelation(h, ntraj: int, npts: int) -> np.ndarray:
    """Complex R[ntraj][npts] of the last propagation."""
    out = np.zeros((ntraj, npts, 2))
    _check(lib.rttda_get_autocorrelation(h, _ptr(out), int(npts)), "rttda_get_autocorrelation")
    return out[..., 0] + 1j * out[..., 1]


def rttda_spectrum_autocorr(R, dt: float, npad: int = 50000, nfreq: int = 1024, normalize: bool = True):
    """(omega[nfreq], S[nfreq]) from complex autocorrelation records R[ntr][npts]."""
    R = np.atleast_2d(np.asarray(R))
    Rri = _f64(np.stack([R.real, R.imag], axis=-1))
    om = np.zeros(nfreq)
    S = np.zeros(nfreq)
    _check(lib.rttda_spectrum_autocorr(_ptr(Rri), Rri.shape[0], Rri.shape[1], float(dt), int(npad), int(nfreq),
                                       1 if normalize else 0, _ptr(om), _ptr(S)), "rttda_spectrum_autocorr")
    return om, S


def rttda_plan(h) -> dict:
    """The sigma build's execution plan for the current batch (see rttda.h)."""
    pi = rttda_plan_info()
    _check(lib.rttda_plan(h, ct.byref(pi)), "rttda_plan")
    d = {name: getattr(pi, name) for name, _ in rttda_plan_info._fields_ if name != "tune_ms"}
    d["tune_ms"] = [pi.tune_ms[k] for k in range(min(pi.ncand, 8))]
    return d


def rttda_coulomb_noalloc(nocc, nvirt, naux, B_ov_dev, c_dev, ntraj, sigma_dev, stream=0) -> None:
    """Coulomb part of sigma with no device allocation (device addresses in)."""
    _check(lib.rttda_coulomb_noalloc(int(nocc), int(nvirt), int(naux), B_ov_dev, c_dev, int(ntraj), sigma_dev,
                                     stream or None), "rttda_coulomb_noalloc")


def rttda_selftest_wait(limit_s) -> int:
    """Status of the bounded-device-wait self-test (RTTDA_E_TIMEOUT expected)."""
    return lib.rttda_selftest_wait(float(limit_s))


def rttda_destroy(h) -> None:
    lib.rttda_destroy(h)


def rttda_estimate_bytes(nocc, nvirt, naux, ntraj, prec, nsteps) -> int:
    n = ct.c_size_t()
    prec = PRECISIONS.get(prec, prec) if isinstance(prec, str) else prec
    _check(lib.rttda_estimate_bytes(nocc, nvirt, naux, ntraj, int(prec), int(nsteps), ct.byref(n)),
           "rttda_estimate_bytes")
    return n.value


def rttda_server_create(hbm_budget, max_active, chunk_steps):
    h = _h()
    _check(lib.rttda_server_create(int(hbm_budget), int(max_active), int(chunk_steps), ct.byref(h)),
           "rttda_server_create")
    return h


def make_request(mol, c_x, prec, pulse, dt, nsteps, gamma, wmin, wmax, nfreq):
    """Build an rttda_request; the returned tuple keeps the arrays alive.
    A molecule of torch CUDA tensors (float64, contiguous) makes a request
    with factors_on_device = 1: the tensors must stay alive until the request
    is no longer pending."""
    names = ("eps_occ", "eps_virt", "B_ov", "B_oo", "B_vv", "mu_oo", "mu_vv", "mu_0ov")
    q = rttda_request()
    q.nocc, q.nvirt, q.naux = mol["nocc"], mol["nvirt"], mol["naux"]
    if getattr(mol["B_vv"], "is_cuda", False):
        arrs = [mol[k] for k in names]
        for name, a in zip(names, arrs):
            setattr(q, name, ct.cast(ct.c_void_p(a.data_ptr()), ct.POINTER(ct.c_double)))
        q.factors_on_device = 1
    else:
        arrs = [_f64(mol[k]) for k in names]
        for name, a in zip(names, arrs):
            setattr(q, name, _ptr(a))
        q.factors_on_device = 0
    q.c_x = float(c_x)
    q.prec = PRECISIONS.get(prec, prec) if isinstance(prec, str) else int(prec)
    q.pulse = make_pulses([pulse])[0]
    q.dt, q.nsteps = float(dt), int(nsteps)
    q.gamma, q.wmin, q.wmax, q.nfreq = float(gamma), float(wmin), float(wmax), int(nfreq)
    return q, arrs


def rttda_server_submit(srv, request) -> int:
    q = request[0] if isinstance(request, tuple) else request
    rid = ct.c_long()
    _check(lib.rttda_server_submit(srv, ct.byref(q), ct.byref(rid)), "rttda_server_submit")
    return rid.value


def rttda_server_poll(srv, rid, nfreq=0, nsteps=-1):
    st = ct.c_int()
    S = np.zeros(max(nfreq, 1))
    om = np.zeros(max(nfreq, 1))
    dip = np.zeros(max(nsteps + 1, 1))
    lat = ct.c_double()
    _check(lib.rttda_server_poll(srv, int(rid), ct.byref(st), _ptr(S) if nfreq else None,
                                 _ptr(om) if nfreq else None, _ptr(dip) if nsteps >= 0 else None,
                                 ct.byref(lat)), "rttda_server_poll")
    return st.value, (S if nfreq else None), (om if nfreq else None), (dip if nsteps >= 0 else None), lat.value


def rttda_server_wait(srv, rid, timeout_s) -> None:
    _check(lib.rttda_server_wait(srv, int(rid), float(timeout_s)), "rttda_server_wait")


def rttda_server_cancel(srv, rid) -> None:
    _check(lib.rttda_server_cancel(srv, int(rid)), "rttda_server_cancel")


def rttda_server_set_grouping(srv, mode) -> None:
    """0: off, 1 (or True): by work (the default), 2: every eligible request."""
    _check(lib.rttda_server_set_grouping(srv, int(mode)), "rttda_server_set_grouping")


def rttda_server_stats_get(srv) -> dict:
    st = rttda_server_stats()
    _check(lib.rttda_server_stats_get(srv, ct.byref(st)), "rttda_server_stats_get")
    return {name: getattr(st, name) for name, _ in rttda_server_stats._fields_}


def rttda_server_destroy(srv) -> None:
    lib.rttda_server_destroy(srv)


# ---------------------------------------------------------------------------
# Convenience wrapper (still only marshalling)
# ---------------------------------------------------------------------------
class Propagator:
    """Owns one handle; numpy in, numpy out."""

    KEYS = ("eps_occ", "eps_virt", "B_ov", "B_oo", "B_vv", "mu_oo", "mu_vv", "mu_0ov")

    def __init__(self, mol: dict, c_x: float, prec="fp64", integrator="rk4"):
        self.nocc, self.nvirt, self.naux = mol["nocc"], mol["nvirt"], mol["naux"]
        self.n = 1 + self.nocc * self.nvirt
        first = mol["B_vv"]
        if hasattr(first, "data_ptr") and getattr(first, "is_cuda", False):
            # torch CUDA tensors (float64, contiguous): factors made on the GPU
            self.h = rttda_create_device(self.nocc, self.nvirt, self.naux,
                                         [mol[k].data_ptr() for k in self.KEYS], c_x, prec)
        else:
            self.h = rttda_create(self.nocc, self.nvirt, self.naux, *[mol[k] for k in self.KEYS], c_x, prec)
        self.ntraj = 0
        if integrator != "rk4":
            rttda_set_integrator(self.h, integrator)

    def set_field(self, pulses):
        rttda_set_field(self.h, pulses)
        self.ntraj = len(pulses)

    def propagate(self, dt, nsteps, c0=None, want_state=True, want_trace=True):
        c_out = np.zeros((self.ntraj, self.n, 2)) if want_state else None
        dip = np.zeros((self.ntraj, nsteps + 1)) if want_trace else None
        nrm = np.zeros((self.ntraj, nsteps + 1)) if want_trace else None
        c0a = None
        if c0 is not None:
            c0 = np.asarray(c0)
            if np.iscomplexobj(c0):
                c0 = np.stack([c0.real, c0.imag], axis=-1)
            c0a = _f64(c0.reshape(self.ntraj, self.n, 2))
        rttda_propagate(self.h, c0a, dt, nsteps, c_out, dip, nrm)
        c = None if c_out is None else c_out[..., 0] + 1j * c_out[..., 1]
        return c, dip, nrm

    def eigenstates(self, k, tol=1e-8, max_iter=200, allow_unconverged=False):
        return rttda_eigenstates(self.h, k, self.n, tol, max_iter, allow_unconverged)

    def set_projectors(self, X):
        rttda_set_projectors(self.h, X)
        self.nproj = 0 if X is None else len(X)

    def overlaps(self, nsteps):
        return rttda_get_overlaps(self.h, self.ntraj, nsteps + 1, self.nproj)

    def autocorrelation(self, nsteps):
        return rttda_get_autocorrelation(self.h, self.ntraj, nsteps + 1)

    def resume(self, dt, nsteps):
        c_out = np.zeros((self.ntraj, self.n, 2))
        dip = np.zeros((self.ntraj, nsteps + 1))
        nrm = np.zeros((self.ntraj, nsteps + 1))
        rttda_resume(self.h, dt, nsteps, c_out, dip, nrm)
        return c_out[..., 0] + 1j * c_out[..., 1], dip, nrm

    def get_state(self):
        c = np.zeros((self.ntraj, self.n, 2))
        t = rttda_get_state(self.h, c)
        return c[..., 0] + 1j * c[..., 1], t

    def set_state(self, c, t):
        c = np.asarray(c)
        rttda_set_state(self.h, _f64(np.stack([c.real, c.imag], axis=-1)), t)

    def memory_bytes(self):
        return rttda_memory_bytes(self.h)

    def close(self):
        if self.h:
            rttda_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
