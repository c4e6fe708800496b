"""Thin ctypes binding of libsmr.so (C ABI in include/smr.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Function names are the C names.  Device buffers are passed as
torch tensors (complex128, CUDA, contiguous) or as raw integer pointers; the
stream defaults to torch's current stream on the tensor's device.  A non-zero
status raises ``SmrError`` with the library's message.  There is no fallback:
if libsmr.so has not been built the first call raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libsmr.so")
_lib = None

SMR_PREC_FP64, SMR_PREC_FP32 = 0, 1
SMR_LRULE_FORMULA, SMR_LRULE_DOUBLE = 0, 1
SMR_PRECOND_NONE, SMR_PRECOND_BLOCKDIAG, SMR_PRECOND_LEARNED, SMR_PRECOND_NEAR, SMR_PRECOND_CLUSTER = 0, 1, 2, 3, 4
SMR_OK, SMR_E_INVALID_ARG, SMR_E_SHAPE, SMR_E_NOT_CONVERGED = 0, -1, -2, -5
SMR_E_BREAKDOWN, SMR_E_TIMEOUT = -6, -8
ERRORS = {-1: "INVALID_ARG", -2: "SHAPE", -3: "OOM", -4: "CUDA", -5: "NOT_CONVERGED",
          -6: "BREAKDOWN", -7: "NAN", -8: "TIMEOUT", -9: "STATE"}


class SmrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"SMR_E_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class smr_opts(C.Structure):
    _fields_ = [("device", C.c_int), ("wavelength", C.c_double), ("pitch", C.c_double),
                ("L0", C.c_int), ("level_rule", C.c_int), ("digits", C.c_double),
                ("n_theta", C.c_int), ("n_phi", C.c_int)]


class smr_info_t(C.Structure):
    _fields_ = [("p", C.c_int), ("n_psi", C.c_int), ("n_shapes", C.c_int), ("n_levels", C.c_int),
                ("n_arrays", C.c_int),
                ("n_unknowns", C.c_longlong), ("L", C.c_int * 16), ("K", C.c_int * 16),
                ("n_box", C.c_int * 16), ("n_il", C.c_int * 16), ("n_near_pairs", C.c_longlong),
                ("n_near_blocks", C.c_int), ("device_bytes", C.c_double),
                ("column_lanes", C.c_int)]


class smr_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("restart", C.c_int), ("precond", C.c_int),
                ("precision", C.c_int), ("max_outer", C.c_int), ("use_x0", C.c_int),
                ("fallback_iters", C.c_int), ("near_sweeps", C.c_int), ("poly_degree", C.c_int)]


class smr_solve_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("matvecs_fp64", C.c_int), ("matvecs_fp32", C.c_int),
                ("outer", C.c_int), ("reorth", C.c_int), ("resid_true", C.c_double),
                ("seconds", C.c_double), ("seconds_product", C.c_double),
                ("seconds_precond", C.c_double), ("seconds_orth", C.c_double),
                ("fallback_x0", C.c_int), ("fallback_precond", C.c_int), ("iters_learned", C.c_int)]


class smr_launch_t(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("level", C.c_int), ("bytes", C.c_double),
                ("flops", C.c_double), ("ms", C.c_double)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_SIGS = {
    "smr_default_opts": (None, [C.POINTER(smr_opts)]),
    "smr_default_solve_opts": (None, [C.POINTER(smr_solve_opts)]),
    "smr_create": (C.c_int, [C.POINTER(_P), C.POINTER(smr_opts)]),
    "smr_destroy": (C.c_int, [_P]),
    "smr_last_error": (C.c_char_p, [_P]),
    "smr_add_sphere": (C.c_int, [_P, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "smr_set_scene": (C.c_int, [_P, C.c_int, _D, C.POINTER(C.c_int), _D, _D, _D, _D]),
    "smr_set_scene_arrays": (C.c_int, [_P, C.c_int, _D, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       _D, _D, _D, _D]),
    "smr_info": (C.c_int, [_P, C.POINTER(smr_info_t)]),
    "smr_rhs_plane_waves": (C.c_int, [_P, C.c_int, _D, _D, _P, _P]),
    "smr_rhs_plane_waves_static": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "smr_matvec": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "smr_matvec_graph": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "smr_matvec_parts": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int, _P]),
    "smr_matvec_host": (C.c_int, [_P, C.c_int, _D, _D, C.c_int, _P]),
    "smr_precond": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "smr_solve": (C.c_int, [_P, C.c_int, _P, _P, C.POINTER(smr_solve_opts),
                            C.POINTER(smr_solve_stats), _P]),
    "smr_far_field": (C.c_int, [_P, C.c_int, _P, C.c_int, _D, _P, _P]),
    "smr_cross_sections": (C.c_int, [_P, C.c_int, _P, C.c_int, _D, _D, _D, _D, _P]),
    "smr_near_field": (C.c_int, [_P, C.c_int, _P, C.c_int, _D, _P, _P]),
    "smr_profile_matvec": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, C.POINTER(smr_launch_t), C.c_int,
                                     C.POINTER(C.c_int), _P]),
    "smr_rhs_plane_waves_arrays": (C.c_int, [_P, _D, _D, _P, _P]),
    "smr_nn_init": (C.c_int, [_P, C.c_int, C.c_ulonglong]),
    "smr_nn_num_params": (C.c_longlong, [_P]),
    "smr_nn_get_params": (C.c_int, [_P, C.POINTER(C.c_float), C.c_longlong]),
    "smr_nn_set_params": (C.c_int, [_P, C.POINTER(C.c_float), C.c_longlong]),
    "smr_nn_features": (C.c_int, [_P, _D, _D, _P, _P]),
    "smr_nn_targets": (C.c_int, [_P, _D, _P, C.c_double, _P, _P]),
    "smr_nn_train_step": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_float, _D, _P]),
    "smr_nn_loss_grad": (C.c_int, [_P, C.c_int, _P, _P, _P, _D, C.POINTER(C.c_float), _P]),
    "smr_nn_predict": (C.c_int, [_P, _D, _D, C.c_double, _P, _P]),
    "smr_copy_pattern": (C.c_int, [_P, C.c_int, _D]),
    "smr_copy_translation": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _D]),
    "smr_copy_near_block": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, _D]),
    "smr_copy_pair_block": (C.c_int, [_P, C.c_int, C.c_int, _D]),
    "smr_copy_level": (C.c_int, [_P, C.c_int, C.c_int, _D, C.c_size_t]),
    "smr_set_tensor_cores": (C.c_int, [_P, C.c_int]),
    "smr_add_shape_sampled": (C.c_int, [_P, C.c_int, _D, _D, C.c_int, C.c_int, _D, _D, C.POINTER(C.c_int)]),
    "smr_measure_peak": (C.c_int, [C.c_int, _D]),
    "smr_add_shape_rotated": (C.c_int, [_P, C.c_int, C.c_double, C.POINTER(C.c_int)]),
    "smr_add_shape_mesh": (C.c_int, [_P, C.c_int, _D, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int,
                                     C.POINTER(C.c_int)]),
    "smr_shape_modes": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _D, _D]),
    "smr_self_block": (C.c_int, [_P, C.c_int, _D]),
    "smr_mesh_static_modes": (C.c_int, [C.c_int, _D, C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int,
                                        C.POINTER(C.c_int), _D, _D]),
    "smr_nn_precond": (C.c_int, [_P, _D, _D, C.c_double, _P, _P]),
    "smr_autotune": (C.c_int, [_P, C.c_int, C.c_int, _P]),
    "smr_sync": (C.c_int, [_P, _P]),
    "smr_set_wait_limit": (C.c_int, [_P, C.c_longlong]),
    "smr_set_column_lanes": (C.c_int, [_P, C.c_int]),
    "smr_set_overlap": (C.c_int, [_P, C.c_int]),
    "smr_precond_cluster": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, _P]),
    "smr_set_variant": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int]),
}


def exported_symbols():
    """Names this binding expects the library to export."""
    return sorted(_SIGS)


def lib():
    """Load libsmr.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIBPATH):
            raise ImportError(f"{_LIBPATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(_LIBPATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(ctx, rc):
    if rc != 0:
        msg = lib().smr_last_error(ctx).decode() if ctx else ""
        raise SmrError(rc, msg)


def _dptr(a):
    return a.ctypes.data_as(_D)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    if not (t.is_cuda and t.is_contiguous() and t.dtype == torch.complex128):
        raise ValueError("device buffers must be contiguous complex128 CUDA tensors")
    return t.data_ptr()


def _stream(stream, t=None):
    if stream is None:
        import torch
        dev = t.device if t is not None and hasattr(t, "device") else None
        return torch.cuda.current_stream(dev).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _R(t, n):
    if isinstance(t, int):
        raise ValueError("pass R explicitly with raw pointers")
    return t.numel() // n


# ------------------------------------------------------------------ context
def smr_default_opts(**kw):
    o = smr_opts()
    lib().smr_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def smr_create(**kw):
    """Create a context; keyword arguments override smr_default_opts."""
    o = smr_default_opts(**kw)
    h = _P()
    rc = lib().smr_create(C.byref(h), C.byref(o))
    if rc != 0:
        raise SmrError(rc, "smr_create failed (device or options)")
    return h


def smr_destroy(ctx):
    lib().smr_destroy(ctx)


def smr_add_sphere(ctx, radius, n_perp, n_par):
    sid = C.c_int()
    _check(ctx, lib().smr_add_sphere(ctx, float(radius), int(n_perp), int(n_par), C.byref(sid)))
    return sid.value


def smr_set_scene(ctx, centres, shape_ids, eps_in, eps_out=1.0, mu_in=1.0, mu_out=1.0):
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(shape_ids, dtype=np.int32).ravel()
    cx = lambda v: np.array([np.real(v), np.imag(v)], dtype=np.float64)
    ei, mi, eo, mo = cx(eps_in), cx(mu_in), cx(eps_out), cx(mu_out)
    _check(ctx, lib().smr_set_scene(ctx, c.shape[0], _dptr(c), s.ctypes.data_as(C.POINTER(C.c_int)),
                                    _dptr(ei), _dptr(mi), _dptr(eo), _dptr(mo)))


def smr_set_scene_arrays(ctx, centres, shape_ids, array_ids, eps_in, eps_out=1.0, mu_in=1.0, mu_out=1.0):
    c = np.ascontiguousarray(centres, dtype=np.float64).reshape(-1, 3)
    s = np.ascontiguousarray(shape_ids, dtype=np.int32).ravel()
    a = np.ascontiguousarray(array_ids, dtype=np.int32).ravel()
    cx = lambda v: np.array([np.real(v), np.imag(v)], dtype=np.float64)
    ei, mi, eo, mo = cx(eps_in), cx(mu_in), cx(eps_out), cx(mu_out)
    ip = C.POINTER(C.c_int)
    _check(ctx, lib().smr_set_scene_arrays(ctx, c.shape[0], _dptr(c), s.ctypes.data_as(ip),
                                           a.ctypes.data_as(ip), _dptr(ei), _dptr(mi), _dptr(eo),
                                           _dptr(mo)))


def scene_from_arrays(ws, **opts):
    """One context holding several workload dicts as independent arrays."""
    w0 = ws[0]
    ctx = smr_create(pitch=w0["pitch"], **opts)
    add_shapes(ctx, w0["shapes"])
    C_ = np.concatenate([w["centres"] for w in ws])
    S_ = np.concatenate([w["shape_ids"] for w in ws])
    A_ = np.concatenate([np.full(len(w["centres"]), i, dtype=np.int32) for i, w in enumerate(ws)])
    smr_set_scene_arrays(ctx, C_, S_, A_, w0["eps_in"])
    return ctx


def smr_info(ctx):
    i = smr_info_t()
    _check(ctx, lib().smr_info(ctx, C.byref(i)))
    n = i.n_levels
    return dict(p=i.p, n_psi=i.n_psi, n_shapes=i.n_shapes, n_levels=n, n_arrays=i.n_arrays,
                n_unknowns=i.n_unknowns,
                L=list(i.L[:n]), K=list(i.K[:n]), n_box=list(i.n_box[:n]), n_il=list(i.n_il[:n]),
                n_near_pairs=i.n_near_pairs, n_near_blocks=i.n_near_blocks,
                device_bytes=i.device_bytes, column_lanes=i.column_lanes)


def smr_rhs_plane_waves(ctx, khat, pol, b, stream=None):
    kh = np.ascontiguousarray(khat, dtype=np.float64).reshape(-1, 3)
    pl = np.ascontiguousarray(np.asarray(pol, dtype=np.complex128).reshape(-1, 3))
    pv = pl.view(np.float64)
    _check(ctx, lib().smr_rhs_plane_waves(ctx, kh.shape[0], _dptr(kh), _dptr(pv), _ptr(b),
                                          _stream(stream, b)))


def smr_rhs_plane_waves_static(ctx, khat, pol, b, R=None, stream=None):
    """No-allocation variant: khat (R,3) float64 and pol (R,3) complex128 are
    device tensors (or raw pointers with R given); b is the device output."""
    if R is None:
        R = khat.shape[0]
    for t, dt, what in ((khat, "float64", "khat"), (pol, "complex128", "pol")):
        if isinstance(t, int):
            continue
        # the library reads these as raw device pointers and cannot check them
        if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch." + dt
                and tuple(t.shape) == (R, 3)):
            raise ValueError(f"{what} must be a contiguous ({R}, 3) {dt} CUDA tensor")
        if hasattr(b, "device") and t.device != b.device:
            raise ValueError(f"{what} is on {t.device}, the output on {b.device}")
    kp = khat if isinstance(khat, int) else khat.data_ptr()
    pp = pol if isinstance(pol, int) else pol.data_ptr()
    _check(ctx, lib().smr_rhs_plane_waves_static(ctx, R, kp, pp, _ptr(b), _stream(stream, b)))


def smr_matvec(ctx, x, y, precision=SMR_PREC_FP64, R=None, stream=None):
    n = smr_info(ctx)["n_unknowns"] if R is None else None
    R = R if R is not None else _R(x, n)
    _check(ctx, lib().smr_matvec(ctx, R, _ptr(x), _ptr(y), precision, _stream(stream, x)))


def smr_matvec_graph(ctx, x, y, precision=SMR_PREC_FP64, R=None, stream=None):
    R = R if R is not None else _R(x, smr_info(ctx)["n_unknowns"])
    _check(ctx, lib().smr_matvec_graph(ctx, R, _ptr(x), _ptr(y), precision, _stream(stream, x)))


def smr_matvec_parts(ctx, x, y_near, y_far, precision=SMR_PREC_FP64, R=None, stream=None):
    R = R if R is not None else _R(x, smr_info(ctx)["n_unknowns"])
    _check(ctx, lib().smr_matvec_parts(ctx, R, _ptr(x), _ptr(y_near), _ptr(y_far), precision,
                                       _stream(stream, x)))


def smr_matvec_host(ctx, x, precision=SMR_PREC_FP64, stream=None):
    """x: host complex128 array [N] or [N, R]; returns y (host)."""
    xx = np.ascontiguousarray(x, dtype=np.complex128)
    n = smr_info(ctx)["n_unknowns"]
    R = xx.size // n
    y = np.empty_like(xx)
    _check(ctx, lib().smr_matvec_host(ctx, R, _dptr(xx.view(np.float64)), _dptr(y.view(np.float64)),
                                      precision, _stream(stream)))
    return y


def smr_precond(ctx, r, z, precision=SMR_PREC_FP64, R=None, stream=None):
    R = R if R is not None else _R(r, smr_info(ctx)["n_unknowns"])
    _check(ctx, lib().smr_precond(ctx, R, _ptr(r), _ptr(z), precision, _stream(stream, r)))


def smr_default_solve_opts(**kw):
    o = smr_solve_opts()
    lib().smr_default_solve_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def smr_solve(ctx, b, x, R=None, stream=None, **kw):
    """Returns (status, stats dict); SMR_E_NOT_CONVERGED is returned, not raised."""
    R = R if R is not None else _R(b, smr_info(ctx)["n_unknowns"])
    o = smr_default_solve_opts(**kw)
    st = smr_solve_stats()
    rc = lib().smr_solve(ctx, R, _ptr(b), _ptr(x), C.byref(o), C.byref(st), _stream(stream, b))
    if rc not in (0, -5):
        _check(ctx, rc)
    return rc, dict(iters=st.iters, matvecs_fp64=st.matvecs_fp64, matvecs_fp32=st.matvecs_fp32,
                    outer=st.outer, reorth=st.reorth, resid_true=st.resid_true, seconds=st.seconds,
                    seconds_product=st.seconds_product, seconds_precond=st.seconds_precond,
                    seconds_orth=st.seconds_orth, fallback_x0=st.fallback_x0,
                    fallback_precond=st.fallback_precond, iters_learned=st.iters_learned)


def smr_set_tensor_cores(ctx, enable):
    _check(ctx, lib().smr_set_tensor_cores(ctx, 1 if enable else 0))


def smr_autotune(ctx, precision=SMR_PREC_FP32, stream=None, R=1):
    _check(ctx, lib().smr_autotune(ctx, int(R), precision, _stream(stream, None)))


def smr_sync(ctx, stream=None):
    _check(ctx, lib().smr_sync(ctx, _stream(stream, None)))


SMR_STEP_TRANSLATE, SMR_STEP_INTERPOLATE, SMR_STEP_ANTERPOLATE = 0, 1, 2


def smr_set_variant(ctx, step, level, precision, variant):
    """Select a launch variant of a level step (level -1: every level)."""
    _check(ctx, lib().smr_set_variant(ctx, int(step), int(level), int(precision), int(variant)))


def smr_set_wait_limit(ctx, rounds):
    """Polling limit of the tensor-core pipeline waits; rounds < 0 restores the default."""
    _check(ctx, lib().smr_set_wait_limit(ctx, int(rounds)))


def smr_precond_cluster(ctx, r, z, precision=SMR_PREC_FP64, R=None, stream=None):
    """z = (2 x 2 cluster block-Jacobi matrix)^-1 r."""
    R = R if R is not None else _R(r, smr_info(ctx)["n_unknowns"])
    _check(ctx, lib().smr_precond_cluster(ctx, R, _ptr(r), _ptr(z), precision, _stream(stream, r)))


def smr_set_overlap(ctx, enable):
    """Overlap the near product and the translations with the rest (1) or not (0)."""
    _check(ctx, lib().smr_set_overlap(ctx, int(bool(enable))))


def smr_set_column_lanes(ctx, lanes):
    """Columns in flight in an FP32 product with several right-hand sides (1..16)."""
    _check(ctx, lib().smr_set_column_lanes(ctx, int(lanes)))


def smr_far_field(ctx, x, dirs, F, R=None, stream=None):
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    R = R if R is not None else _R(x, smr_info(ctx)["n_unknowns"])
    _check(ctx, lib().smr_far_field(ctx, R, _ptr(x), d.shape[0], _dptr(d), _ptr(F), _stream(stream, x)))


def smr_cross_sections(ctx, x, khat, pol, n_theta=48, R=None, stream=None):
    """(C_sca[R], C_ext[R]) for plane-wave excitations khat[R][3], pol[R][3]."""
    R = R if R is not None else _R(x, smr_info(ctx)["n_unknowns"])
    kh = np.ascontiguousarray(khat, dtype=np.float64).reshape(-1, 3)
    pc = np.ascontiguousarray(pol, dtype=np.complex128).reshape(-1, 3)
    if kh.shape[0] != R or pc.shape[0] != R:
        raise ValueError(f"khat and pol need {R} rows, got {kh.shape[0]} and {pc.shape[0]}")
    pv = np.ascontiguousarray(pc.view(np.float64))
    csca = np.zeros(R)
    cext = np.zeros(R)
    _check(ctx, lib().smr_cross_sections(ctx, R, _ptr(x), int(n_theta), _dptr(kh), _dptr(pv),
                                         _dptr(csca), _dptr(cext), _stream(stream, x)))
    return csca, cext


def smr_near_field(ctx, x, pts, EH, R=None, stream=None):
    d = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    R = R if R is not None else _R(x, smr_info(ctx)["n_unknowns"])
    _check(ctx, lib().smr_near_field(ctx, R, _ptr(x), d.shape[0], _dptr(d), _ptr(EH), _stream(stream, x)))


def smr_profile_matvec(ctx, x, y, precision=SMR_PREC_FP64, R=None, stream=None):
    """One product with per-launch (name, level, bytes, flops, ms) records."""
    R = R if R is not None else _R(x, smr_info(ctx)["n_unknowns"])
    cap = 8192
    arr = (smr_launch_t * cap)()
    n = C.c_int()
    _check(ctx, lib().smr_profile_matvec(ctx, R, _ptr(x), _ptr(y), precision, arr, cap, C.byref(n),
                                         _stream(stream, x)))
    return [dict(name=arr[i].name.decode(), level=arr[i].level, bytes=arr[i].bytes,
                 flops=arr[i].flops, ms=arr[i].ms) for i in range(min(n.value, cap))]


def _inc(khat, pol):
    kh = np.ascontiguousarray(khat, dtype=np.float64).reshape(-1, 3)
    pl = np.ascontiguousarray(np.asarray(pol, dtype=np.complex128).reshape(-1, 3))
    return kh, pl, pl.view(np.float64)


def _fptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def smr_rhs_plane_waves_arrays(ctx, khat, pol, b, stream=None):
    kh, pl, pv = _inc(khat, pol)
    _check(ctx, lib().smr_rhs_plane_waves_arrays(ctx, _dptr(kh), _dptr(pv), _ptr(b), _stream(stream, b)))


def smr_nn_init(ctx, width=256, seed=0):
    _check(ctx, lib().smr_nn_init(ctx, int(width), int(seed)))


def smr_nn_num_params(ctx):
    return int(lib().smr_nn_num_params(ctx))


def smr_nn_get_params(ctx):
    n = smr_nn_num_params(ctx)
    out = np.empty(n, dtype=np.float32)
    _check(ctx, lib().smr_nn_get_params(ctx, out.ctypes.data_as(C.POINTER(C.c_float)), n))
    return out


def smr_nn_set_params(ctx, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(ctx, lib().smr_nn_set_params(ctx, p.ctypes.data_as(C.POINTER(C.c_float)), p.size))


def _need(t, n, what):
    if hasattr(t, "numel") and t.numel() != n:
        raise ValueError(f"{what}: {t.numel()} elements given, {n} required")


def smr_nn_features(ctx, khat, pol, feat, stream=None):
    _need(feat, smr_info(ctx)["p"] * 448, "features [p][448]")
    kh, pl, pv = _inc(khat, pol)
    _check(ctx, lib().smr_nn_features(ctx, _dptr(kh), _dptr(pv), _fptr(feat), _stream(stream, feat)))


def smr_nn_targets(ctx, khat, x, scale, tgt, stream=None):
    i = smr_info(ctx)
    _need(tgt, i["p"] * 4 * i["n_psi"], "targets [p][4 n_psi]")
    kh = np.ascontiguousarray(khat, dtype=np.float64).reshape(-1, 3)
    _check(ctx, lib().smr_nn_targets(ctx, _dptr(kh), _ptr(x), float(scale), _fptr(tgt), _stream(stream, x)))


def smr_nn_train_step(ctx, n, feat, tgt, lr, idx=None, stream=None):
    loss = C.c_double()
    _check(ctx, lib().smr_nn_train_step(ctx, int(n), _fptr(feat), _fptr(idx), _fptr(tgt), float(lr),
                                        C.byref(loss), _stream(stream, feat)))
    return loss.value


def smr_nn_loss_grad(ctx, n, feat, tgt, idx=None, stream=None):
    loss = C.c_double()
    g = np.empty(smr_nn_num_params(ctx), dtype=np.float32)
    _check(ctx, lib().smr_nn_loss_grad(ctx, int(n), _fptr(feat), _fptr(idx), _fptr(tgt), C.byref(loss),
                                       g.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream, feat)))
    return loss.value, g


def smr_nn_predict(ctx, khat, pol, scale, x0, stream=None):
    kh, pl, pv = _inc(khat, pol)
    _check(ctx, lib().smr_nn_predict(ctx, _dptr(kh), _dptr(pv), float(scale), _ptr(x0), _stream(stream, x0)))


def smr_nn_precond(ctx, khat, pol, scale, b, stream=None):
    kh, pl, pv = _inc(khat, pol)
    _check(ctx, lib().smr_nn_precond(ctx, _dptr(kh), _dptr(pv), float(scale), _ptr(b), _stream(stream, b)))


def smr_copy_pattern(ctx, shape):
    i = smr_info(ctx)
    out = np.empty((i["n_psi"], 2, i["K"][0]), dtype=np.complex128)
    _check(ctx, lib().smr_copy_pattern(ctx, shape, _dptr(out.view(np.float64))))
    return out


def smr_copy_translation(ctx, level, dx, dy):
    K = smr_info(ctx)["K"][level]
    out = np.empty(K, dtype=np.complex128)
    _check(ctx, lib().smr_copy_translation(ctx, level, dx, dy, _dptr(out.view(np.float64))))
    return out


def smr_copy_near_block(ctx, sm, sn, dx, dy):
    n2 = 2 * smr_info(ctx)["n_psi"]
    out = np.empty((n2, n2), dtype=np.complex128)
    _check(ctx, lib().smr_copy_near_block(ctx, sm, sn, dx, dy, _dptr(out.view(np.float64))))
    return out


def smr_copy_pair_block(ctx, mu, nu):
    n2 = 2 * smr_info(ctx)["n_psi"]
    out = np.empty((n2, n2), dtype=np.complex128)
    _check(ctx, lib().smr_copy_pair_block(ctx, mu, nu, _dptr(out.view(np.float64))))
    return out


def smr_copy_level(ctx, level, kind, R=1):
    i = smr_info(ctx)
    out = np.empty((i["n_box"][level], i["K"][level], 4, R), dtype=np.complex128)
    _check(ctx, lib().smr_copy_level(ctx, level, kind, _dptr(out.view(np.float64)), out.size * 2))
    return out


def add_shapes(ctx, shapes):
    """Register shapes: (radius, n_perp, n_par) tuples are closed-form spheres;
    dicts with kind 'mesh' (verts, tris, n_perp, n_par) are meshed shapes;
    dicts with kind 'rotated' (base, angle) are an earlier shape rotated about
    z; objects with r, w, psi, div, Zs, n_perp, n_par are shapes given as data."""
    for sh in shapes:
        if isinstance(sh, dict) and sh.get("kind") == "mesh":
            smr_add_shape_mesh(ctx, sh["verts"], sh["tris"], sh["n_perp"], sh["n_par"])
        elif isinstance(sh, dict) and sh.get("kind") == "rotated":
            smr_add_shape_rotated(ctx, sh["base"], sh["angle"])
        elif hasattr(sh, "psi"):
            smr_add_shape_sampled(ctx, sh.r, sh.w, sh.n_perp, sh.n_par, sh.psi, sh.div, sh.Zs)
        else:
            a, npp, npl = sh
            smr_add_sphere(ctx, a, npp, npl)


def smr_add_shape_sampled(ctx, pts, wts, n_perp, n_par, psi, div, self_block):
    """pts (Q,3), wts (Q,), psi (n_psi,Q,3), div (n_psi,Q), self_block
    (2 n_psi, 2 n_psi) complex; returns the shape id."""
    P = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    W = np.ascontiguousarray(wts, dtype=np.float64).ravel()
    M = np.ascontiguousarray(np.concatenate([np.asarray(psi, dtype=np.float64),
                                             np.asarray(div, dtype=np.float64)[..., None]], axis=2))
    Z = np.ascontiguousarray(self_block, dtype=np.complex128)
    sid = C.c_int()
    _check(ctx, lib().smr_add_shape_sampled(ctx, P.shape[0], _dptr(P), _dptr(W), n_perp, n_par, _dptr(M),
                                            _dptr(Z.view(np.float64)), C.byref(sid)))
    return sid.value


def _mesh_args(verts, tris):
    V = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1, 3)
    T = np.ascontiguousarray(tris, dtype=np.int32).reshape(-1, 3)
    return V, T, T.ctypes.data_as(C.POINTER(C.c_int))


def smr_add_shape_mesh(ctx, verts, tris, n_perp, n_par):
    """verts (nv,3), tris (nt,3) outward; returns the shape id."""
    V, T, tp = _mesh_args(verts, tris)
    sid = C.c_int()
    _check(ctx, lib().smr_add_shape_mesh(ctx, V.shape[0], _dptr(V), T.shape[0], tp, n_perp, n_par,
                                         C.byref(sid)))
    return sid.value


def smr_measure_peak(kind):
    """Measured TFLOP/s of the current device: 0 FP32 FMA, 1 packed FP32x2
    FMA, 2 FP64 FMA."""
    v = C.c_double()
    rc = lib().smr_measure_peak(int(kind), C.byref(v))
    if rc:
        raise SmrError(rc, "smr_measure_peak failed")
    return v.value


def smr_add_shape_rotated(ctx, base, angle):
    """Shape `base` rotated by `angle` radians about z; returns the shape id."""
    sid = C.c_int()
    _check(ctx, lib().smr_add_shape_rotated(ctx, int(base), float(angle), C.byref(sid)))
    return sid.value


def smr_shape_modes(ctx, shape_id):
    """(M [n_psi][n_edges], gamma [n_psi]) of a meshed shape."""
    n, ne = C.c_int(), C.c_int()
    _check(ctx, lib().smr_shape_modes(ctx, shape_id, C.byref(n), C.byref(ne), None, None))
    M = np.empty((n.value, ne.value))
    g = np.empty(n.value)
    _check(ctx, lib().smr_shape_modes(ctx, shape_id, None, None, _dptr(M), _dptr(g)))
    return M, g


def smr_self_block(ctx, shape_id):
    """The self block (2 n_psi, 2 n_psi) complex the scene uses for a shape."""
    n2 = 2 * smr_info(ctx)["n_psi"]
    Z = np.empty((n2, n2), dtype=np.complex128)
    _check(ctx, lib().smr_self_block(ctx, shape_id, _dptr(Z.view(np.float64))))
    return Z


def smr_mesh_static_modes(verts, tris, n_perp, n_par):
    """Host static-mode solve of a mesh: (M [n_psi][n_edges], gamma [n_psi])."""
    V, T, tp = _mesh_args(verts, tris)
    ne = C.c_int()
    n = n_perp + n_par
    # edges of a closed genus-0 mesh: 3 nt / 2
    M = np.empty((n, 3 * T.shape[0] // 2))
    g = np.empty(n)
    rc = lib().smr_mesh_static_modes(V.shape[0], _dptr(V), T.shape[0], tp, n_perp, n_par, C.byref(ne),
                                     _dptr(M), _dptr(g))
    if rc != 0:
        raise SmrError(rc, "smr_mesh_static_modes rejected the mesh or the mode counts")
    return M[:, :ne.value], g


def scene_from_workload(w, **opts):
    """Create a context and set the scene of a workload dict (workloads.make);
    the workload's L0, if it names one, unless opts overrides it."""
    o = {"L0": w["L0"]} if "L0" in w else {}
    o.update(opts)
    ctx = smr_create(pitch=w["pitch"], **o)
    add_shapes(ctx, w["shapes"])
    smr_set_scene(ctx, w["centres"], w["shape_ids"], w["eps_in"])
    return ctx
