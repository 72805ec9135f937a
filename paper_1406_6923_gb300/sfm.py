"""Thin ctypes binding of ``libsfm`` (``include/sfm.h``).

The functions carry the C names and only marshal arguments: every step of
the method runs in the library's CUDA kernels.  A failing call raises
:class:`SfmError` with the library's status code and message.  Loading fails
loudly when ``libsfm.so`` has not been built: there is no fallback."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsfm.so")

SFM_OK = 0
SFM_ERR_ARG = -1
SFM_ERR_CUDA = -2
SFM_ERR_NOT_SPD = -3
SFM_ERR_BREAKDOWN = -4
SFM_ERR_UNSTABLE = -5
SFM_ERR_TIMEOUT = -6
SFM_ERR_NOMEM = -7
SFM_ERR_STATE = -8

SFM_FP64 = 0
SFM_FP32 = 1
SFM_FP32X2 = 2
SFM_FP32F = 3
SFM_TF32X3 = 4
SFM_TF32 = 5
SFM_BF16 = 6
SFM_FP32FX2 = 7
SFM_FP32X2P = 8

SFM_DEVICE_PTR = 1
SFM_ENERGY = 2

# every symbol include/sfm.h declares
EXPORTS = ["sfm_create", "sfm_destroy", "sfm_last_error", "sfm_set_stream", "sfm_set_topology",
           "sfm_set_coeffs", "sfm_get_coeffs", "sfm_set_sources", "sfm_set_receivers",
           "sfm_run", "sfm_cfl_dt", "sfm_last_launches", "sfm_debug_set", "sfm_set_model",
           "sfm_build_roms", "sfm_project_sources", "sfm_project_receivers", "sfm_free_build", "sfm_run_static",
           "sfm_autotune", "sfm_set_initial", "sfm_plan_pieces", "sfm_usable_depths",
           "sfm_cut_depth", "sfm_checkpoint", "sfm_restore", "sfm_run_report",
           "sfm_net_create", "sfm_net_destroy", "sfm_net_last_error", "sfm_net_params",
           "sfm_net_grad", "sfm_net_adam", "sfm_net_forward", "sfm_raw_encode",
           "sfm_net_fit_decoder", "sfm_net_decode", "sfm_ntd_error", "sfm_build_roms_surrogate", "sfm_build_roms_shifts",
           "sfm_probe_read_gbs"]


class sfm_build_report(C.Structure):
    _fields_ = [("seconds", C.c_double), ("cg_iterations_max", C.c_int),
                ("cg_residual_max", C.c_double), ("krylov_min_ratio", C.c_double),
                ("nclasses", C.c_int), ("nregularized", C.c_int)]


class sfm_run_info(C.Structure):
    _fields_ = [("precision", C.c_int), ("nsteps", C.c_int), ("nshots", C.c_int),
                ("launches", C.c_int), ("kernel_ms", C.c_double), ("total_ms", C.c_double),
                ("status", C.c_int), ("unstable_step", C.c_int), ("energy", C.c_int)]


class sfm_surrogate_report(C.Structure):
    _fields_ = [("eligible", C.c_int), ("accepted", C.c_int), ("fallback", C.c_int),
                ("sigma_err_median", C.c_double), ("sigma_err_max_accepted", C.c_double),
                ("seconds_surrogate", C.c_double), ("seconds_exact", C.c_double)]


class SfmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libsfm error {code}: {msg}")
        self.code = code


_lib = None

_i = C.c_int
_p = C.c_void_p
_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)


def load(path=LIB_PATH):
    """Load ``libsfm.so`` (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libsfm.so not built at {path}; run paper_1406_6923_gb300._build")
    lib = C.CDLL(path)
    sig = {
        "sfm_create": (_i, [C.POINTER(_p), _i]),
        "sfm_destroy": (_i, [_p]),
        "sfm_last_error": (C.c_char_p, [_p]),
        "sfm_set_stream": (_i, [_p, _p]),
        "sfm_set_topology": (_i, [_p, _i, _ip, _ip, _ip]),
        "sfm_set_coeffs": (_i, [_p, _dp, C.c_size_t]),
        "sfm_get_coeffs": (_i, [_p, _dp, C.c_size_t, C.POINTER(C.c_size_t)]),
        "sfm_set_sources": (_i, [_p, _i, _i, _ip, _ip, _dp]),
        "sfm_set_receivers": (_i, [_p, _i, _i, _ip, _ip, _dp]),
        "sfm_run": (_i, [_p, _i, C.c_double, _i, _p, _p, _i, _dp]),
        "sfm_cfl_dt": (_i, [_p, _i, _dp, _dp]),
        "sfm_last_launches": (_i, [_p, _ip]),
        "sfm_debug_set": (_i, [_p, _i, C.c_longlong]),
        "sfm_set_model": (_i, [_p, _i, _i, _i, C.c_double, _dp, _i, _ip, _i, _ip, _i, _ip]),
        "sfm_build_roms": (_i, [_p, _ip, _ip, C.c_double, C.c_double,
                                C.POINTER(sfm_build_report)]),
        "sfm_project_sources": (_i, [_p, _i, _dp, C.c_double]),
        "sfm_project_receivers": (_i, [_p, _i, _dp]),
        "sfm_free_build": (_i, [_p]),
        "sfm_run_static": (_i, [_i, _p, _i, _ip, _ip, _ip, _p, _i, _i, _ip, _ip, _p, _i, _i, _ip,
                                _ip, _p, C.c_double, _i, _p, _p]),
        "sfm_autotune": (_i, [_p, _i, _i, _ip, _ip, _dp]),
        "sfm_set_initial": (_i, [_p, _i, _i, _ip, _ip, _dp, _dp]),
        "sfm_plan_pieces": (_i, [_i, _i, _ip, _i, _ip, _ip, _i, _ip]),
        "sfm_usable_depths": (_i, [_i, _ip, _i, _dp, C.c_double, _ip]),
        "sfm_cut_depth": (_i, [_p, C.c_double, _ip, _i, _ip]),
        "sfm_checkpoint": (_i, [_p, _p, C.POINTER(C.c_size_t)]),
        "sfm_restore": (_i, [_p, _p, C.c_size_t]),
        "sfm_run_report": (_i, [_p, C.POINTER(sfm_run_info), _dp, _i]),
        "sfm_net_create": (_i, [C.POINTER(_p), _i, _i, _i, _i, _i, _i, _i, C.c_ulonglong]),
        "sfm_net_destroy": (_i, [_p]),
        "sfm_net_last_error": (C.c_char_p, [_p]),
        "sfm_net_params": (_i, [_p, _fp, C.c_size_t, C.POINTER(C.c_size_t), _i]),
        "sfm_net_grad": (_i, [_p, _p, _p, _i, _fp, _fp]),
        "sfm_net_adam": (_i, [_p, C.c_float]),
        "sfm_net_forward": (_i, [_p, _p, _i, _p, _i]),
        "sfm_raw_encode": (_i, [_i, _i, _i, _i, _p, _p]),
        "sfm_net_fit_decoder": (_i, [_p, _i, _i, _p, _i, _i, C.c_ulonglong, _p]),
        "sfm_net_decode": (_i, [_p, _p, _i, _p]),
        "sfm_ntd_error": (_i, [_i, _i, _i, _i, _p, _p, _i, _dp, _dp]),
        "sfm_build_roms_shifts": (_i, [_p, _ip, _ip, _dp, _i, C.c_double, C.POINTER(sfm_build_report)]),
        "sfm_build_roms_surrogate": (_i, [_p, _p, _ip, _ip, C.c_double, C.c_double, C.c_double, _ip,
                                          C.POINTER(sfm_surrogate_report), C.POINTER(sfm_build_report)]),
        "sfm_probe_read_gbs": (_i, [_i, C.c_size_t, _i, _dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(h, rc):
    if rc != SFM_OK:
        msg = _lib.sfm_last_error(h)
        raise SfmError(rc, msg.decode() if msg else "")


def _iarr(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _darr(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def sfm_create(device=0):
    lib = load()
    h = _p()
    rc = lib.sfm_create(C.byref(h), int(device))
    _check(None, rc)
    return h


def sfm_destroy(h):
    load().sfm_destroy(h)


def sfm_last_error(h):
    return load().sfm_last_error(h).decode()


def sfm_set_stream(h, stream_ptr):
    _check(h, load().sfm_set_stream(h, _p(int(stream_ptr)) if stream_ptr else None))


def sfm_set_topology(h, k_sub, m_face, nbr):
    k, kp = _iarr(k_sub)
    m, mp = _iarr(np.asarray(m_face).reshape(-1))
    n, np_ = _iarr(np.asarray(nbr).reshape(-1))
    _check(h, load().sfm_set_topology(h, len(k), kp, mp, np_))


def sfm_set_coeffs(h, coeffs):
    c, cp = _darr(np.asarray(coeffs).reshape(-1))
    _check(h, load().sfm_set_coeffs(h, cp, c.size))


def sfm_get_coeffs(h):
    need = C.c_size_t(0)
    _check(h, load().sfm_get_coeffs(h, None, 0, C.byref(need)))
    out = np.empty(need.value, dtype=np.float64)
    _check(h, load().sfm_get_coeffs(h, out.ctypes.data_as(_dp), out.size, C.byref(need)))
    return out


def sfm_set_sources(h, nshots, pair_shot, pair_sub, rows):
    a, ap = _iarr(pair_shot)
    b, bp = _iarr(pair_sub)
    r, rp = _darr(np.asarray(rows).reshape(-1))
    _check(h, load().sfm_set_sources(h, int(nshots), len(a), ap, bp, rp))


def sfm_set_initial(h, nshots, pair_shot, pair_sub, u0_rows, v0_rows=None):
    a, ap = _iarr(pair_shot)
    b, bp = _iarr(pair_sub)
    u, up = _darr(np.asarray(u0_rows).reshape(-1))
    if v0_rows is None:
        vp = None
    else:
        v, vp = _darr(np.asarray(v0_rows).reshape(-1))
    _check(h, load().sfm_set_initial(h, int(nshots), len(a), ap, bp, up, vp))


def sfm_set_receivers(h, nrec, pair_rec, pair_sub, rows):
    a, ap = _iarr(pair_rec)
    b, bp = _iarr(pair_sub)
    r, rp = _darr(np.asarray(rows).reshape(-1))
    _check(h, load().sfm_set_receivers(h, int(nrec), len(a), ap, bp, rp))


def sfm_run(h, precision, dt, nsteps, wavelet, nshots, nrec, traces=None, device_ptrs=None,
            energy=False):
    """Step the coupled ROMs.  Host form: ``wavelet`` is a [nshots, nsteps]
    array and the traces [nshots, nrec, nsteps+1] are returned.  Device form:
    ``device_ptrs=(wavelet_ptr, traces_ptr)`` (FP64 device buffers).
    ``energy``: also evaluate the discrete energy (see sfm_run_report).
    Returns ``(traces, kernel_ms)``."""
    ms = C.c_double(0.0)
    extra = SFM_ENERGY if energy else 0
    if device_ptrs is not None:
        wp, tp = device_ptrs
        _check(h, load().sfm_run(h, int(precision), float(dt), int(nsteps), _p(int(wp)),
                                 _p(int(tp)), SFM_DEVICE_PTR | extra, C.byref(ms)))
        return None, ms.value
    w, _ = _darr(np.asarray(wavelet).reshape(nshots, nsteps))
    out = np.empty((nshots, nrec, nsteps + 1)) if traces is None else traces
    _check(h, load().sfm_run(h, int(precision), float(dt), int(nsteps),
                             _p(w.ctypes.data), _p(out.ctypes.data), extra, C.byref(ms)))
    return out, ms.value


def sfm_run_report(h):
    """Report of the last sfm_run: a dict of the sfm_run_info fields, plus
    ``energy_start``/``energy_end`` arrays (per shot) when it evaluated them."""
    info = sfm_run_info()
    _check(h, load().sfm_run_report(h, C.byref(info), None, 0))
    out = {name: getattr(info, name) for name, _ in sfm_run_info._fields_}
    if info.energy:
        e = np.zeros(2 * info.nshots)
        _check(h, load().sfm_run_report(h, C.byref(info), e.ctypes.data_as(_dp), e.size))
        out["energy_start"] = e[:info.nshots].copy()
        out["energy_end"] = e[info.nshots:].copy()
    return out


def sfm_checkpoint(h):
    """The stepping state of the last sfm_run as a bytes blob."""
    need = C.c_size_t(0)
    _check(h, load().sfm_checkpoint(h, None, C.byref(need)))
    buf = np.zeros(need.value // 8, dtype=np.int64)     # 8-byte aligned
    cap = C.c_size_t(buf.nbytes)
    _check(h, load().sfm_checkpoint(h, buf.ctypes.data_as(_p), C.byref(cap)))
    return buf.tobytes()


def sfm_restore(h, blob):
    buf = np.frombuffer(blob, dtype=np.int64).copy()
    _check(h, load().sfm_restore(h, buf.ctypes.data_as(_p), buf.nbytes))


def sfm_cfl_dt(h, iters=300):
    lam = C.c_double(0.0)
    dt = C.c_double(0.0)
    _check(h, load().sfm_cfl_dt(h, int(iters), C.byref(lam), C.byref(dt)))
    return lam.value, dt.value


def sfm_autotune(h, precision, nsteps=200):
    """Returns (consumer warps, ring stages, microseconds per time step)."""
    ncw = C.c_int(0)
    nst = C.c_int(0)
    us = C.c_double(0.0)
    _check(h, load().sfm_autotune(h, int(precision), int(nsteps), C.byref(ncw), C.byref(nst),
                                  C.byref(us)))
    return ncw.value, nst.value, us.value


def sfm_plan_pieces(nunits, k_sub, grid):
    """Returns (ptr[grid+1], pieces[n][3] as (unit, j0, j1))."""
    k, kp = _iarr(k_sub)
    ptr = np.zeros(grid + 1, dtype=np.int32)
    n = C.c_int(0)
    rc = load().sfm_plan_pieces(int(nunits), len(k), kp, int(grid), ptr.ctypes.data_as(_ip), None, 0,
                                C.byref(n))
    if rc not in (SFM_OK, SFM_ERR_ARG) or n.value <= 0:
        _check(None, rc)
    pieces = np.zeros((n.value, 3), dtype=np.int32)
    _check(None, load().sfm_plan_pieces(int(nunits), len(k), kp, int(grid), ptr.ctypes.data_as(_ip),
                                        pieces.ctypes.data_as(_ip), n.value, C.byref(n)))
    return ptr, pieces


def sfm_probe_read_gbs(device, nbytes, repeats):
    """Read bandwidth (GB/s) of ``nbytes`` streamed ``repeats`` times in one
    launch (L2-resident when ``nbytes`` fits in L2)."""
    v = C.c_double()
    _check(None, load().sfm_probe_read_gbs(int(device), int(nbytes), int(repeats), C.byref(v)))
    return v.value


def sfm_last_launches(h):
    n = C.c_int(0)
    _check(h, load().sfm_last_launches(h, C.byref(n)))
    return n.value


def sfm_debug_set(h, key, value):
    _check(h, load().sfm_debug_set(h, int(key), int(value)))


def sfm_set_model(h, c, hgrid, xcuts, ycuts, zcuts):
    """``c``: [nz, ny, nx] cell velocities; cuts: node indices 0..n per axis."""
    c = np.ascontiguousarray(c, dtype=np.float64)
    nz, ny, nx = c.shape
    x, xp = _iarr(xcuts)
    y, yp = _iarr(ycuts)
    z, zp = _iarr(zcuts)
    _check(h, load().sfm_set_model(h, nx, ny, nz, float(hgrid), c.ctypes.data_as(_dp),
                                   len(x) - 1, xp, len(y) - 1, yp, len(z) - 1, zp))


def sfm_build_roms(h, m_sub, k_sub, sigma, cg_tol=1e-14):
    m, mp = _iarr(m_sub)
    k, kp = _iarr(k_sub)
    rep = sfm_build_report()
    _check(h, load().sfm_build_roms(h, mp, kp, float(sigma), float(cg_tol), C.byref(rep)))
    return {f: getattr(rep, f) for f, _ in sfm_build_report._fields_}


def sfm_build_roms_shifts(h, m_sub, k_sub, shifts, cg_tol=1e-14):
    """The offline build with distinct Krylov shifts (Eq. 6)."""
    m, mp = _iarr(m_sub)
    k, kp = _iarr(k_sub)
    sh, sp = _darr(np.asarray(shifts, dtype=np.float64))
    rep = sfm_build_report()
    _check(h, load().sfm_build_roms_shifts(h, mp, kp, sp, len(sh), float(cg_tol), C.byref(rep)))
    return {f: getattr(rep, f) for f, _ in sfm_build_report._fields_}


def sfm_project_sources(h, xyz, width):
    x, xp = _darr(np.asarray(xyz).reshape(-1, 3))
    _check(h, load().sfm_project_sources(h, x.shape[0], xp, float(width)))


def sfm_project_receivers(h, xyz):
    x, xp = _darr(np.asarray(xyz).reshape(-1, 3))
    _check(h, load().sfm_project_receivers(h, x.shape[0], xp))


def sfm_free_build(h):
    _check(h, load().sfm_free_build(h))


def sfm_usable_depths(k_sub, range_, tau=1e-13):
    """Depth decision alone (host): ``range_`` [nsub][2*kmax][2] of
    (lambda_min, lambda_max) per block, kmax = range_.shape[1] // 2."""
    k, kp = _iarr(k_sub)
    r, rp = _darr(np.asarray(range_).reshape(len(k), -1, 2))
    depth = np.zeros(len(k), dtype=np.int32)
    _check(None, load().sfm_usable_depths(len(k), kp, r.shape[1] // 2, rp, float(tau),
                                          depth.ctypes.data_as(_ip)))
    return depth


def sfm_cut_depth(h, nsub, tau=1e-13):
    """Cut every subdomain's fraction to its usable depth; returns (depths,
    levels removed)."""
    depth = np.zeros(int(nsub), dtype=np.int32)
    n = C.c_int(0)
    _check(h, load().sfm_cut_depth(h, float(tau), depth.ctypes.data_as(_ip), len(depth),
                                   C.byref(n)))
    return depth, n.value


def sfm_run_static(device, stream_ptr, k_sub, m_face, nbr, coeffs_ptr, nshots, src_shot, src_sub,
                   src_rows_ptr, nrec, rec_id, rec_sub, rec_rows_ptr, dt, nsteps, wavelet_ptr,
                   traces_ptr):
    """FP64 stepping with no device allocation: the ``*_ptr`` arguments are
    device addresses owned by the caller; the topology and pair lists are
    host arrays."""
    k, kp = _iarr(k_sub)
    m, mp = _iarr(np.asarray(m_face).reshape(-1))
    n, np_ = _iarr(np.asarray(nbr).reshape(-1))
    a, ap = _iarr(src_shot)
    b, bp = _iarr(src_sub)
    c, cp = _iarr(rec_id)
    d, dp = _iarr(rec_sub)
    rc = load().sfm_run_static(int(device), _p(int(stream_ptr)) if stream_ptr else None, len(k),
                               kp, mp, np_, _p(int(coeffs_ptr)), int(nshots), len(a), ap, bp,
                               _p(int(src_rows_ptr)), int(nrec), len(c), cp, dp,
                               _p(int(rec_rows_ptr)), float(dt), int(nsteps), _p(int(wavelet_ptr)),
                               _p(int(traces_ptr)))
    _check(None, rc)


# ---------------------------------------------------------------------------
# learned surrogate (network object)

def _ncheck(net, rc):
    if rc != SFM_OK:
        msg = _lib.sfm_net_last_error(net) if net else _lib.sfm_last_error(None)
        raise SfmError(rc, msg.decode() if msg else "")


def sfm_net_create(device, n, c1, c2, c3, hidden, code, seed=0):
    net = _p()
    _ncheck(None, load().sfm_net_create(C.byref(net), int(device), int(n), int(c1), int(c2), int(c3),
                                        int(hidden), int(code), int(seed)))
    return net


def sfm_net_destroy(net):
    load().sfm_net_destroy(net)


def sfm_net_params(net, values=None):
    """Without ``values``: the parameters as an FP32 array; with: replace them."""
    cnt = C.c_size_t(0)
    _ncheck(net, load().sfm_net_params(net, None, 0, C.byref(cnt), 0))
    if values is None:
        out = np.empty(cnt.value, dtype=np.float32)
        _ncheck(net, load().sfm_net_params(net, out.ctypes.data_as(_fp), out.size, C.byref(cnt), 0))
        return out
    v = np.ascontiguousarray(values, dtype=np.float32)
    _ncheck(net, load().sfm_net_params(net, v.ctypes.data_as(_fp), v.size, C.byref(cnt), 1))
    return None


def sfm_net_grad(net, c_ptr, zt_ptr, batch, want_grad=False):
    """Loss of a batch (device pointers) and, with ``want_grad``, the
    gradient of every parameter as an FP32 array; returns (loss, grad)."""
    loss = C.c_float(0.0)
    g = None
    if want_grad:
        g = np.empty(sfm_net_params(net).size, dtype=np.float32)
    _ncheck(net, load().sfm_net_grad(net, _p(int(c_ptr)), _p(int(zt_ptr)), int(batch), C.byref(loss),
                                     g.ctypes.data_as(_fp) if g is not None else None))
    return loss.value, g


def sfm_net_adam(net, lr):
    _ncheck(net, load().sfm_net_adam(net, float(lr)))


def sfm_net_forward(net, c_ptr, batch, z_ptr, bf16=False):
    _ncheck(net, load().sfm_net_forward(net, _p(int(c_ptr)), int(batch), _p(int(z_ptr)), 1 if bf16 else 0))


def raw_size(b, k):
    return 2 * (k - 1) * (b * (b - 1) // 2 + b)


def sfm_raw_encode(device, count, b, k, coef_ptr, raw_ptr):
    _ncheck(None, load().sfm_raw_encode(int(device), int(count), int(b), int(k), _p(int(coef_ptr)),
                                        _p(int(raw_ptr))))


def sfm_net_fit_decoder(net, b, k, raw_ptr, N, iters=4, seed=0, codes_ptr=None):
    _ncheck(net, load().sfm_net_fit_decoder(net, int(b), int(k), _p(int(raw_ptr)), int(N), int(iters),
                                            int(seed), _p(int(codes_ptr)) if codes_ptr else None))


def sfm_net_decode(net, z_ptr, batch, coef_ptr):
    _ncheck(net, load().sfm_net_decode(net, _p(int(z_ptr)), int(batch), _p(int(coef_ptr))))


def sfm_ntd_error(device, count, b, k, coef_a_ptr, coef_r_ptr, lams):
    """Relative NtD-map errors [count][len(lams)] of two coefficient families
    (device pointers) at the complex ``lams``."""
    lam = np.ascontiguousarray(np.stack([np.real(lams), np.imag(lams)], axis=1), dtype=np.float64)
    err = np.empty((count, len(lams)))
    _ncheck(None, load().sfm_ntd_error(int(device), int(count), int(b), int(k), _p(int(coef_a_ptr)),
                                       _p(int(coef_r_ptr)), len(lams), lam.ctypes.data_as(_dp),
                                       err.ctypes.data_as(_dp)))
    return err


def sfm_build_roms_surrogate(h, net, m_sub, k_sub, sigma, nt_tol, exact=None, cg_tol=1e-14):
    """Offline stage with the surrogate and exact fallback; returns
    (surrogate report dict, exact-build report dict)."""
    m, mp = _iarr(m_sub)
    k, kp = _iarr(k_sub)
    ep = None
    if exact is not None:
        e, ep = _iarr(np.asarray(exact, dtype=np.int32))
    srep = sfm_surrogate_report()
    rep = sfm_build_report()
    _check(h, load().sfm_build_roms_surrogate(h, net, mp, kp, float(sigma), float(cg_tol), float(nt_tol),
                                              ep, C.byref(srep), C.byref(rep)))
    return ({n: getattr(srep, n) for n, _ in sfm_surrogate_report._fields_},
            {n: getattr(rep, n) for n, _ in sfm_build_report._fields_})
