"""Thin ctypes binding of include/of.h: the same entry points, argument marshalling only.

Field arguments may be torch CUDA tensors (their data_ptr is passed) or integer device
addresses; host arrays (ion positions, charges, forces) are numpy float64 arrays.  Every
computation happens in libof.so; this module never falls back to anything else and raises
if the library cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_lib

OF_OK, OF_EINVAL, OF_ENOMEM, OF_ECUDA, OF_ENOCONV, OF_EBREAKDOWN, OF_ETIMEOUT = range(7)
OF_F64, OF_F32 = 0, 1
OF_LINE_BRENT, OF_LINE_SLOPE = 0, 1
OF_FP_VLR, OF_FP_U = 0, 1
OF_VW_LAPLACIAN, OF_VW_GRADIENT = 0, 1
STATUS_NAMES = {0: "OF_OK", 1: "OF_EINVAL", 2: "OF_ENOMEM", 3: "OF_ECUDA", 4: "OF_ENOCONV",
                5: "OF_EBREAKDOWN", 6: "OF_ETIMEOUT"}


class of_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("precision", C.c_int),
                ("inner_tol", C.c_double), ("check_every", C.c_int), ("no_multigrid", C.c_int),
                ("precond", C.c_void_p), ("precond_theta", C.c_double)]


class of_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int),
                ("rel_residual", C.c_double), ("net_steps", C.c_int)]


class of_system(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("R", C.POINTER(C.c_double)),
                ("Z", C.POINTER(C.c_double)), ("sigma", C.c_double), ("rc", C.c_double),
                ("b_from_potential", C.c_int), ("sigma_ref", C.c_double), ("rc_ref", C.c_double)]


class of_functional(C.Structure):
    _fields_ = [("lambda_", C.c_double), ("mu", C.c_double), ("alpha", C.c_double),
                ("beta", C.c_double), ("n_terms", C.c_int), ("P", C.c_double * 16),
                ("Q", C.c_double * 16), ("L", C.c_int),
                ("P10", C.c_double * 16), ("Q10", C.c_double * 16),
                ("P20", C.c_double * 16), ("Q20", C.c_double * 16),
                ("P11", C.c_double * 16), ("Q11", C.c_double * 16)]


class of_scf_opts(C.Structure):
    _fields_ = [("nlcg_tol", C.c_double), ("nlcg_max_iter", C.c_int),
                ("nlcg_restart", C.c_int), ("fp_tol", C.c_double), ("fp_max_iter", C.c_int),
                ("anderson_m", C.c_int), ("anderson_zeta", C.c_double),
                ("precision", C.c_int), ("poisson", of_solve_opts), ("kernel", of_solve_opts),
                ("verbose", C.c_int), ("line_tol", C.c_double), ("nlcg_tol_rel", C.c_double),
                ("line_search", C.c_int), ("fixed_point", C.c_int), ("vw_energy", C.c_int),
                ("nlcg_precond_shift", C.c_double),
                ("nlcg_precond_low", C.c_double)]


class of_scf_result(C.Structure):
    _fields_ = [("energy", C.c_double), ("e_tf", C.c_double), ("e_vw", C.c_double),
                ("e_lr", C.c_double), ("e_xc", C.c_double), ("e_es", C.c_double),
                ("e_self", C.c_double), ("e_corr", C.c_double), ("fp_error", C.c_double),
                ("nlcg_residual", C.c_double), ("outer_iterations", C.c_int),
                ("nlcg_iterations", C.c_int), ("poisson_iterations", C.c_int),
                ("kernel_iterations", C.c_int), ("line_evaluations", C.c_int),
                ("converged", C.c_int)]


class of_relax_opts(C.Structure):
    _fields_ = [("ftol", C.c_double), ("max_steps", C.c_int), ("step0", C.c_double),
                ("line_tol", C.c_double), ("max_line", C.c_int)]


class of_relax_result(C.Structure):
    _fields_ = [("energy", C.c_double), ("max_force", C.c_double), ("steps", C.c_int),
                ("evaluations", C.c_int), ("converged", C.c_int)]


class of_vacancy_result(C.Structure):
    _fields_ = [("e_perfect", C.c_double), ("e_unrelaxed", C.c_double),
                ("e_relaxed", C.c_double), ("evf_unrelaxed", C.c_double),
                ("evf_relaxed", C.c_double), ("max_force", C.c_double),
                ("relax_steps", C.c_int), ("evaluations", C.c_int)]


class of_kernel_stat(C.Structure):
    _fields_ = [("kernel_class", C.c_int), ("launches", C.c_longlong), ("timed", C.c_longlong),
                ("total_ms", C.c_double), ("mean_ms", C.c_double),
                ("bytes_per_launch", C.c_double)]


_P = C.c_void_p
_D = C.c_double
_I = C.c_int
_SIGNATURES = {
    "of_default_solve_opts": (None, [C.POINTER(of_solve_opts)]),
    "of_default_scf_opts": (None, [C.POINTER(of_scf_opts)]),
    "of_grid_create": (_I, [_I, _I, _I, _D, _D, _D, _I, _P, C.POINTER(_P)]),
    "of_grid_destroy": (_I, [_P]),
    "of_laplacian_apply": (_I, [_P, _I, _P, _P]),
    "of_poisson_solve": (_I, [_P, _P, _P, C.POINTER(of_solve_opts), C.POINTER(of_solve_info)]),
    "of_kernel_solve": (_I, [_P, _P, _I, C.POINTER(_D), C.POINTER(_D), _D, _P,
                             C.POINTER(of_solve_opts), C.POINTER(of_solve_info)]),
    "of_pseudocharge": (_I, [_P, C.POINTER(of_system), _P, C.POINTER(_D)]),
    "of_hamiltonian_apply": (_I, [_P, C.POINTER(of_functional), _P, _P, _P, _P]),
    "of_lr_potential": (_I, [_P, C.POINTER(of_functional), _D, _P, _P, C.POINTER(_D), _P,
                             C.POINTER(of_solve_opts), C.POINTER(of_solve_info)]),
    "of_lr_workspace_fields": (_I, [C.POINTER(of_functional)]),
    "of_default_relax_opts": (None, [C.POINTER(of_relax_opts)]),
    "of_relax": (_I, [_P, C.POINTER(of_system), C.POINTER(of_functional), C.POINTER(of_scf_opts),
                      C.POINTER(of_relax_opts), _P, _P, C.POINTER(_D), C.POINTER(_D),
                      C.POINTER(of_relax_result)]),
    "of_vacancy_formation": (_I, [_P, _P, C.POINTER(of_system), _I, C.POINTER(of_functional),
                                  C.POINTER(of_scf_opts), C.POINTER(of_relax_opts), _P, _P, _P,
                                  _P, C.POINTER(_D), C.POINTER(of_vacancy_result)]),
    "of_scf_ground_state": (_I, [_P, C.POINTER(of_system), C.POINTER(of_functional),
                                 C.POINTER(of_scf_opts), _P, _P, C.POINTER(of_scf_result)]),
    "of_forces": (_I, [_P, C.POINTER(of_system), _P, _P, C.POINTER(_D)]),
    "of_scf_ground_state_batched": (_I, [_I, C.POINTER(_P), C.POINTER(of_system),
                                         C.POINTER(of_functional), C.POINTER(of_scf_opts),
                                         C.POINTER(_P), C.POINTER(_P), C.POINTER(of_scf_result)]),
    "of_last_error": (C.c_char_p, []),
    "of_poisson_solve_noalloc": (_I, [_I, _I, _I, _D, _D, _D, _I, _P, _P, _P,
                                      C.POINTER(of_solve_opts), C.POINTER(of_solve_info)]),
    "of_poisson_solve_batched": (_I, [_I, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                      C.POINTER(of_solve_opts), C.POINTER(of_solve_info)]),
    "of_precond_num_params": (_I, []),
    "of_precond_create": (_I, [C.POINTER(C.c_float), _I, C.POINTER(_P)]),
    "of_precond_destroy": (_I, [_P]),
    "of_precond_set_wait_limit": (_I, [_P, _D]),
    "of_precond_get_params": (_I, [_P, C.POINTER(C.c_float), _I]),
    "of_precond_apply": (_I, [_P, _P, _P, _P]),
    "of_precond_loss_grad": (_I, [_P, _P, _P, C.POINTER(_D), C.POINTER(C.c_float)]),
    "of_precond_train": (_I, [_P, _P, _P, _I, C.POINTER(_I), _I, _I, C.c_float, C.POINTER(_D)]),
    "of_precond_collect": (_I, [_P, _P, _D, _I, _I, _P, C.POINTER(_I)]),
    "of_precond_set_shift": (_I, [_P, _D]),
    "of_launch_count": (C.c_ulonglong, []),
    "of_resource_count": (C.c_ulonglong, []),
    "of_alu_peak": (_I, [_I, _P, C.POINTER(_D)]),
    "of_kernel_class_name": (C.c_char_p, [_I]),
    "of_profile_enable": (_I, [_P, _I]),
    "of_profile_read": (_I, [_P, C.POINTER(of_kernel_stat), _I]),
}

_lib = None


def load(build_if_missing: bool = True):
    """Load libof.so (building it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        build_lib.build()
    if not os.path.exists(build_lib.LIB):
        raise RuntimeError(f"{build_lib.LIB} is missing: build the CUDA library first")
    lib = C.CDLL(build_lib.LIB)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGNATURES)


class OfError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = load().of_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")


def _check(status, where, allow=()):
    if status != OF_OK and status not in allow:
        raise OfError(status, where)
    return status


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("field arguments must be contiguous CUDA tensors")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------- the entry points
def of_default_solve_opts():
    o = of_solve_opts()
    load().of_default_solve_opts(C.byref(o))
    return o


def of_default_scf_opts():
    o = of_scf_opts()
    load().of_default_scf_opts(C.byref(o))
    return o


def of_grid_create(n, L, fd_half_order=6, stream=None):
    h = _P()
    _check(load().of_grid_create(int(n[0]), int(n[1]), int(n[2]), float(L[0]), float(L[1]),
                                 float(L[2]), int(fd_half_order), _stream_ptr(stream),
                                 C.byref(h)), "of_grid_create")
    return h


def of_grid_destroy(h):
    return _check(load().of_grid_destroy(h), "of_grid_destroy")


def of_laplacian_apply(h, dtype, x, y):
    return _check(load().of_laplacian_apply(h, int(dtype), _ptr(x), _ptr(y)),
                  "of_laplacian_apply")


def of_poisson_solve(h, rho, phi, opts=None, allow=()):
    info = of_solve_info()
    st = load().of_poisson_solve(h, _ptr(rho), _ptr(phi), C.byref(opts) if opts else None,
                                 C.byref(info))
    _check(st, "of_poisson_solve", allow)
    return info


def of_kernel_solve(h, f, P, Q, kf2, W, opts=None, allow=()):
    P = np.ascontiguousarray(np.asarray(P, dtype=np.complex128))
    Q = np.ascontiguousarray(np.asarray(Q, dtype=np.complex128))
    Pd = P.view(np.float64)
    Qd = Q.view(np.float64)
    info = of_solve_info()
    st = load().of_kernel_solve(h, _ptr(f), int(P.size), Pd.ctypes.data_as(C.POINTER(_D)),
                                Qd.ctypes.data_as(C.POINTER(_D)), float(kf2), _ptr(W),
                                C.byref(opts) if opts else None, C.byref(info))
    _check(st, "of_kernel_solve", allow)
    return info


def make_system(R, Z, sigma, rc, b_from_potential=False, sigma_ref=0.0, rc_ref=0.0):
    """of_system from numpy arrays (kept alive on the returned object).  sigma_ref > 0: the
    overlap correction on the grid with reference charges of that width within rc_ref."""
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(-1, 3))
    Z = np.ascontiguousarray(np.asarray(Z, dtype=np.float64).reshape(-1))
    s = of_system(int(Z.size), R.ctypes.data_as(C.POINTER(_D)), Z.ctypes.data_as(C.POINTER(_D)),
                  float(sigma), float(rc), int(bool(b_from_potential)), float(sigma_ref),
                  float(rc_ref))
    s._keep = (R, Z)
    return s


def make_functional(lam, mu, alpha=0.0, beta=0.0, P=(), Q=(), L=0, K=None):
    """of_functional record.  P, Q: the K_00 terms; L = 2 with K = {"10": (P, Q), "20": ...,
    "11": ...}: the density-dependent classes (same number of terms each)."""
    f = of_functional()
    f.lambda_, f.mu, f.alpha, f.beta = float(lam), float(mu), float(alpha), float(beta)
    f.n_terms = len(P)
    f.L = int(L)

    def fill(dstP, dstQ, P, Q):
        for k, (p, q) in enumerate(zip(P, Q)):
            dstP[2 * k], dstP[2 * k + 1] = complex(p).real, complex(p).imag
            dstQ[2 * k], dstQ[2 * k + 1] = complex(q).real, complex(q).imag

    fill(f.P, f.Q, P, Q)
    for c, (Pc, Qc) in (K or {}).items():
        if len(Pc) != len(P):
            raise ValueError(f"class {c}: {len(Pc)} terms, K_00 has {len(P)}")
        fill(getattr(f, "P" + c), getattr(f, "Q" + c), Pc, Qc)
    return f


def of_pseudocharge(h, sys, b):
    e = _D()
    _check(load().of_pseudocharge(h, C.byref(sys), _ptr(b), C.byref(e)), "of_pseudocharge")
    return e.value


def of_hamiltonian_apply(h, fn, u, phi, vlr, hu):
    return _check(load().of_hamiltonian_apply(h, C.byref(fn), _ptr(u), _ptr(phi), _ptr(vlr),
                                              _ptr(hu)), "of_hamiltonian_apply")


def of_default_relax_opts():
    o = of_relax_opts()
    load().of_default_relax_opts(C.byref(o))
    return o


def of_relax(h, sys, fn, scf_opts, relax_opts, u, phi, allow=()):
    """Relaxes the geometry of sys; returns (R (n, 3), F (n, 3), of_relax_result)."""
    n = sys.n_atoms
    R = (C.c_double * (3 * n))()
    F = (C.c_double * (3 * n))()
    res = of_relax_result()
    st = load().of_relax(h, C.byref(sys), C.byref(fn), C.byref(scf_opts) if scf_opts else None,
                         C.byref(relax_opts) if relax_opts else None, _ptr(u), _ptr(phi), R, F,
                         C.byref(res))
    if st != OF_OK and st not in allow:
        _check(st, "of_relax")
    return (np.array(R[:]).reshape(n, 3), np.array(F[:]).reshape(n, 3), res)


def vacancy_cell_lengths(L, n_atoms):
    """Sides of the vacancy cell of a perfect cell with sides L and n_atoms ions: L scaled by
    ((M - 1)/M)^(1/3), the volume per atom kept (Sec. 5.6)."""
    s = ((n_atoms - 1) / n_atoms) ** (1.0 / 3.0)
    return tuple(s * float(x) for x in L)


def of_vacancy_formation(hp, hv, sys, site, fn, scf_opts, relax_opts, u_perfect, phi_perfect,
                         u_vacancy, phi_vacancy, allow=()):
    """Vacancy formation energy; returns (R of the vacancy cell (M - 1, 3), of_vacancy_result).
    relax_opts None: unrelaxed only."""
    m = sys.n_atoms - 1
    R = (C.c_double * (3 * max(m, 1)))()
    res = of_vacancy_result()
    st = load().of_vacancy_formation(hp, hv, C.byref(sys), int(site), C.byref(fn),
                                     C.byref(scf_opts) if scf_opts else None,
                                     C.byref(relax_opts) if relax_opts else None,
                                     _ptr(u_perfect), _ptr(phi_perfect), _ptr(u_vacancy),
                                     _ptr(phi_vacancy), R, C.byref(res))
    if st != OF_OK and st not in allow:
        _check(st, "of_vacancy_formation")
    return np.array(R[:3 * m]).reshape(m, 3), res


def of_lr_workspace_fields(fn):
    return int(load().of_lr_workspace_fields(C.byref(fn)))


def of_lr_potential(h, fn, kf2, u, vlr, W=None, opts=None):
    t = _D()
    info = of_solve_info()
    _check(load().of_lr_potential(h, C.byref(fn), float(kf2), _ptr(u), _ptr(vlr), C.byref(t),
                                  _ptr(W), C.byref(opts) if opts else None, C.byref(info)),
           "of_lr_potential")
    return t.value, info


def of_scf_ground_state(h, sys, fn, opts, u, phi, allow=()):
    res = of_scf_result()
    st = load().of_scf_ground_state(h, C.byref(sys), C.byref(fn), C.byref(opts), _ptr(u),
                                    _ptr(phi), C.byref(res))
    _check(st, "of_scf_ground_state", allow)
    return res


def of_scf_ground_state_batched(grids, systems, fn, opts, us, phis, allow=()):
    """Ground states of several cells in one call (see include/of.h); returns their results."""
    nc = len(grids)
    G = (_P * nc)(*[g.value if isinstance(g, _P) else g for g in grids])
    S = (of_system * nc)(*systems)
    U = (_P * nc)(*[_ptr(x) for x in us])
    Ph = (_P * nc)(*[_ptr(x) for x in phis])
    res = (of_scf_result * nc)()
    st = load().of_scf_ground_state_batched(nc, G, S, C.byref(fn), C.byref(opts), U, Ph, res)
    _check(st, "of_scf_ground_state_batched", allow)
    return list(res)


def of_forces(h, sys, u, phi):
    F = np.zeros((sys.n_atoms, 3))
    _check(load().of_forces(h, C.byref(sys), _ptr(u), _ptr(phi),
                            F.ctypes.data_as(C.POINTER(_D))), "of_forces")
    return F


def of_last_error():
    return load().of_last_error().decode(errors="replace")


def of_launch_count():
    return int(load().of_launch_count())


def of_resource_count():
    return int(load().of_resource_count())


OF_PEAK_F64, OF_PEAK_F32, OF_PEAK_F32X2 = 0, 1, 2


def of_alu_peak(kind, stream=None):
    """Measured FMA rate of the CUDA cores in FLOP/s (kind: OF_PEAK_F64 / F32 / F32X2)."""
    out = _D(0.0)
    _check(load().of_alu_peak(int(kind), _stream_ptr(stream), C.byref(out)), "of_alu_peak")
    return out.value


def of_kernel_class_name(cls):
    return load().of_kernel_class_name(int(cls)).decode()


def of_profile_enable(h, sample_every=1):
    return _check(load().of_profile_enable(h, int(sample_every)), "of_profile_enable")


def of_profile_read(h):
    """Per-kernel-class statistics as a list of dicts (synchronises the grid's stream)."""
    buf = (of_kernel_stat * 32)()
    k = load().of_profile_read(h, buf, 32)
    if k < 0:
        raise OfError(OF_ECUDA, "of_profile_read")
    return [dict(kernel=of_kernel_class_name(buf[i].kernel_class), launches=buf[i].launches,
                 timed=buf[i].timed, total_ms=buf[i].total_ms, mean_ms=buf[i].mean_ms,
                 bytes_per_launch=buf[i].bytes_per_launch) for i in range(k)]


def of_poisson_solve_noalloc(n, L, fd_half_order, stream, rho, phi, opts=None, allow=()):
    """Poisson solve that allocates no device memory (see include/of.h)."""
    info = of_solve_info()
    st = load().of_poisson_solve_noalloc(int(n[0]), int(n[1]), int(n[2]), float(L[0]),
                                         float(L[1]), float(L[2]), int(fd_half_order),
                                         _stream_ptr(stream), _ptr(rho), _ptr(phi),
                                         C.byref(opts) if opts else None, C.byref(info))
    _check(st, "of_poisson_solve_noalloc", allow)
    return info


def of_poisson_solve_batched(grids, rhos, phis, opts=None, allow=()):
    """Batched Poisson solves of independent cells (see include/of.h); returns the infos."""
    nc = len(grids)
    G = (_P * nc)(*[g.value if isinstance(g, _P) else g for g in grids])
    R = (_P * nc)(*[_ptr(x) for x in rhos])
    F = (_P * nc)(*[_ptr(x) for x in phis])
    infos = (of_solve_info * nc)()
    st = load().of_poisson_solve_batched(nc, G, R, F, C.byref(opts) if opts else None, infos)
    _check(st, "of_poisson_solve_batched", allow)
    return list(infos)


# ------------------------------------------------------------- learned preconditioner
def of_precond_num_params():
    return int(load().of_precond_num_params())


def of_precond_create(params):
    """New network handle from host FP32 parameters (W1, b1, W2, b2, W3, b3 flattened)."""
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
    h = _P()
    _check(load().of_precond_create(p.ctypes.data_as(C.POINTER(C.c_float)), int(p.size),
                                    C.byref(h)), "of_precond_create")
    return h


def of_precond_destroy(P):
    return _check(load().of_precond_destroy(P), "of_precond_destroy")


def of_precond_get_params(P):
    out = np.zeros(of_precond_num_params(), dtype=np.float32)
    _check(load().of_precond_get_params(P, out.ctypes.data_as(C.POINTER(C.c_float)), int(out.size)),
           "of_precond_get_params")
    return out


def of_precond_set_wait_limit(P, seconds):
    return _check(load().of_precond_set_wait_limit(P, float(seconds)), "of_precond_set_wait_limit")


def of_precond_set_shift(P, shift):
    return _check(load().of_precond_set_shift(P, float(shift)), "of_precond_set_shift")


def of_precond_apply(h, P, r, z):
    return _check(load().of_precond_apply(h, P, _ptr(r), _ptr(z)), "of_precond_apply")


def of_precond_loss_grad(h, P, r):
    loss = _D()
    grad = np.zeros(of_precond_num_params(), dtype=np.float32)
    _check(load().of_precond_loss_grad(h, P, _ptr(r), C.byref(loss),
                                       grad.ctypes.data_as(C.POINTER(C.c_float))),
           "of_precond_loss_grad")
    return loss.value, grad


def of_precond_train(h, P, samples, nsamples, order, steps, batch, lr):
    o = np.ascontiguousarray(np.asarray(order, dtype=np.int32).ravel())
    if o.size < steps * batch:
        raise ValueError("order needs steps * batch entries")
    loss = _D()
    _check(load().of_precond_train(h, P, _ptr(samples), int(nsamples),
                                   o.ctypes.data_as(C.POINTER(_I)), int(steps), int(batch),
                                   float(lr), C.byref(loss)), "of_precond_train")
    return loss.value


def of_precond_collect(h, rho, stride, max_samples, samples, shift=0.0):
    count = _I()
    _check(load().of_precond_collect(h, _ptr(rho), float(shift), int(stride), int(max_samples),
                                     _ptr(samples), C.byref(count)), "of_precond_collect")
    return count.value
