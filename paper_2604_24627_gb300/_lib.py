"""ctypes binding of libaxpic's C ABI (include/axpic.h).

Argument marshalling only: every entry point forwards to the CUDA library with
the same name. The library must have been built (``build.py``); importing this
module on a machine where it is missing raises instead of falling back to
anything else.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libaxpic.so")

AXPIC_OK, AXPIC_E_INVALID, AXPIC_E_CAPACITY, AXPIC_E_CUDA, AXPIC_E_TIMEOUT, AXPIC_E_NUMERIC = range(6)
STATUS_NAMES = {0: "AXPIC_OK", 1: "AXPIC_E_INVALID", 2: "AXPIC_E_CAPACITY", 3: "AXPIC_E_CUDA",
                4: "AXPIC_E_TIMEOUT", 5: "AXPIC_E_NUMERIC"}
CH_PRIMAKOFF, CH_COMPTON, CH_BREMS, CH_ALL = 1, 2, 4, 7

TOTALS_LEN = 32
TOTALS_NAMES = ["nemit_p", "nemit_c", "nemit_b", "uemit_p", "uemit_c", "uemit_b", "events_p", "events_c",
                "events_b", "events_pinv", "absorbed_c", "absorbed_b", "cap_hits", "clamp_hits", "dropped",
                "n_axions", "u_axions", "macro_axions", "macro_photons", "residual_e", "n_photons", "u_photons",
                "u_electrons", "remaps", "part_e", "part_g", "part_a", "remap_e", "cell_steps"]
CELL_INFO_LEN = 16
CELL_INFO_NAMES = ["rho", "X_H", "n_e", "n_eff", "S_Z", "kappa", "Q_C", "Q_B", "Gamma_C", "Gamma_B",
                   "Gamma0_P", "eta", "T"]
CELL_DIAG_LEN = 16
CELL_DIAG_NAMES = ["dE", "dPx", "dPy", "dPz", "S_minus_1", "bx", "by", "bz", "var", "var_new", "W",
                   "applied_E", "res_E", "res_Px", "res_Py", "res_Pz"]


class Species(ctypes.Structure):
    """axpic_species: wp and xyz hold 4 binary32 values a slot, {w, px, py,
    pz} and {x, y, z, unused}."""
    _fields_ = [("wp", ctypes.c_void_p), ("xyz", ctypes.c_void_p), ("count", ctypes.c_void_p),
                ("capacity", ctypes.c_int32)]


class PlasmaDesc(ctypes.Structure):
    _fields_ = [("ncells", ctypes.c_int32), ("nspecies", ctypes.c_int32), ("cell_index_base", ctypes.c_int64),
                ("T_keV", ctypes.c_void_p), ("n_ion", ctypes.c_void_p), ("Z", ctypes.POINTER(ctypes.c_double)),
                ("A", ctypes.POINTER(ctypes.c_double)), ("cell_volume_cm3", ctypes.c_double),
                ("electrons", Species), ("photons", Species), ("axions", Species)]


class Params(ctypes.Structure):
    _fields_ = [("g_agg_GeV_inv", ctypes.c_double), ("g_ae", ctypes.c_double), ("dt_phys_s", ctypes.c_double),
                ("w_a", ctypes.c_double), ("w_gamma_ref", ctypes.c_double), ("lambda_cap", ctypes.c_double),
                ("kappa_mode", ctypes.c_int32), ("kappa_fixed_keV", ctypes.c_double),
                ("prim_targets", ctypes.c_int32), ("prim_inverse_mult", ctypes.c_double),
                ("eq_stats", ctypes.c_int32), ("brems_ee", ctypes.c_int32), ("absorb_mode", ctypes.c_int32),
                ("brems_gamma_shape", ctypes.c_double), ("relax_r", ctypes.c_double),
                ("T_floor_keV", ctypes.c_double), ("T_ceil_keV", ctypes.c_double), ("T_mode", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("tally_nbins", ctypes.c_int32), ("tally_Emax_keV", ctypes.c_double),
                ("tally_enable", ctypes.c_int32), ("diag_enable", ctypes.c_int32),
                ("threads_per_block", ctypes.c_int32), ("decide_chunk", ctypes.c_int32),
                ("rate_model", ctypes.c_int32), ("sr_table_nkt", ctypes.c_int32), ("sr_table_nne", ctypes.c_int32),
                ("step_branches", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2),
                ("axion_mass_keV", ctypes.c_double)]


class AxpicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None

EXPORTS = {
    "axpic_mlp_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "axpic_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "axpic_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "axpic_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "axpic_mlp_gradients": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)]),
    "axpic_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
    "axpic_mlp_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "axpic_set_surrogate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float]),
    "axpic_get_cell_records": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_float), ctypes.c_void_p]),
    "axpic_get_spectral_records": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                                  ctypes.POINTER(ctypes.c_float)]),
    "axpic_mlp_set_norm": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float)]),
    "axpic_mlp_get_norm": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float)]),
    "axpic_mlp_set_skip": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "axpic_mlp_get_skip": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    "axpic_surrogate_targets": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_double,
                                               ctypes.POINTER(ctypes.c_double)]),
    "axpic_surrogate_features": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                                ctypes.POINTER(ctypes.c_float)]),
    "axpic_surrogate_fit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double)]),
    "axpic_surrogate_validate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                ctypes.POINTER(ctypes.c_float)]),
    "axpic_mlp_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "axpic_default_params": (None, [ctypes.POINTER(Params)]),
    "axpic_init_plasma": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(PlasmaDesc),
                                         ctypes.POINTER(Params), ctypes.c_void_p]),
    "axpic_sample_plasma": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "axpic_update_cells": (ctypes.c_int, [ctypes.c_void_p]),
    "axpic_step_cells": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32]),
    "axpic_absorb": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]),
    "axpic_emit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]),
    "axpic_feedback": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "axpic_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32]),
    "axpic_run_steps": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]),
    "axpic_launch_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "axpic_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "axpic_tally_spectrum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]),
    "axpic_eval_rates": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_void_p]),
    "axpic_get_cell_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double)]),
    "axpic_get_cell_diag": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double)]),
    "axpic_get_residuals": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double)]),
    "axpic_step_noalloc": (ctypes.c_int, [ctypes.POINTER(PlasmaDesc), ctypes.POINTER(Params), ctypes.c_int64,
                                          ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "axpic_profile_begin": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "axpic_profile_end": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int32)]),
    "axpic_step_kernel_names": (ctypes.c_char_p, [ctypes.c_void_p]),
    "axpic_stream_axions": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32]),
    "axpic_stream_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "axpic_merge_axions": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_float)]),
    "axpic_merge_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "axpic_deposit_composition": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                                 ctypes.c_void_p]),
    "axpic_state_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]),
    "axpic_save_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "axpic_load_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "axpic_run_steps_streamed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                ctypes.c_double, ctypes.c_double, ctypes.c_int32]),
    "axpic_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "axpic_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "axpic_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "axpic_version": (ctypes.c_char_p, []),
}


def lib():
    """Load libaxpic.so (once). Raises if the CUDA library has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libaxpic.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


def _check(ctx, status):
    if status != AXPIC_OK:
        msg = lib().axpic_last_error(ctx)
        raise AxpicError(status, msg.decode() if msg else "")


def default_params():
    p = Params()
    lib().axpic_default_params(ctypes.byref(p))
    return p


def axpic_init_plasma(desc, params, stream=0):
    ctx = ctypes.c_void_p()
    st = lib().axpic_init_plasma(ctypes.byref(ctx), ctypes.byref(desc), ctypes.byref(params),
                                 ctypes.c_void_p(stream))
    if st != AXPIC_OK:
        raise AxpicError(st, "axpic_init_plasma failed (see stderr)")
    return ctx


def axpic_sample_plasma(ctx, n_el, n_ph, n_ax):
    _check(ctx, lib().axpic_sample_plasma(ctx, n_el, n_ph, n_ax))


def axpic_step_cells(ctx, step, mask, first_cell, ncells):
    _check(ctx, lib().axpic_step_cells(ctx, step, mask, first_cell, ncells))


def axpic_update_cells(ctx):
    _check(ctx, lib().axpic_update_cells(ctx))


def axpic_absorb(ctx, step, mask):
    _check(ctx, lib().axpic_absorb(ctx, step, mask))


def axpic_emit(ctx, step, mask):
    _check(ctx, lib().axpic_emit(ctx, step, mask))


def axpic_feedback(ctx, step):
    _check(ctx, lib().axpic_feedback(ctx, step))


def axpic_step(ctx, step, mask):
    _check(ctx, lib().axpic_step(ctx, step, mask))


def axpic_run_steps(ctx, first_step, nsteps, mask):
    _check(ctx, lib().axpic_run_steps(ctx, first_step, nsteps, mask))


def axpic_launch_shape(ctx):
    """(decide_chunk, event warps per CTA, branches of a replayed step)."""
    v = [ctypes.c_int32() for _ in range(3)]
    _check(ctx, lib().axpic_launch_shape(ctx, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def axpic_autotune(ctx, step, trial_steps, mask):
    """(best ms per step, decide_chunk, event warps per CTA)."""
    ms = ctypes.c_double()
    chunk = ctypes.c_int32()
    warps = ctypes.c_int32()
    _check(ctx, lib().axpic_autotune(ctx, step, trial_steps, mask, ctypes.byref(ms), ctypes.byref(chunk),
                                     ctypes.byref(warps)))
    return ms.value, chunk.value, warps.value


def axpic_tally_spectrum(ctx, nbins, H_out, totals_out):
    """H_out and totals_out: ctypes double arrays (or None)."""
    _check(ctx, lib().axpic_tally_spectrum(ctx, nbins, H_out, totals_out))


def axpic_eval_rates(ctx, cell, E_ptr, n, out_ptr):
    _check(ctx, lib().axpic_eval_rates(ctx, cell, ctypes.c_void_p(E_ptr), n, ctypes.c_void_p(out_ptr)))


def axpic_get_cell_info(ctx, first, count, out):
    _check(ctx, lib().axpic_get_cell_info(ctx, first, count, out))


def axpic_get_cell_diag(ctx, first, count, out):
    _check(ctx, lib().axpic_get_cell_diag(ctx, first, count, out))


def axpic_get_residuals(ctx, first, count, out):
    _check(ctx, lib().axpic_get_residuals(ctx, first, count, out))


def axpic_step_noalloc(desc, params, step, mask, carry_ptr, stream=0):
    """One fused step without a context or any allocation (carry: device
    pointer to ncells*4 doubles, caller-owned)."""
    st = lib().axpic_step_noalloc(ctypes.byref(desc), ctypes.byref(params), step, mask,
                                  ctypes.c_void_p(carry_ptr), ctypes.c_void_p(stream))
    if st != AXPIC_OK:
        raise AxpicError(st, "axpic_step_noalloc failed (see stderr)")


PROFILE_SLOTS = 4


def axpic_step_kernel_names(ctx):
    """Names of the kernels one axpic_step launches, in order."""
    return tuple(n for n in lib().axpic_step_kernel_names(ctx).decode().split(",") if n)


def axpic_profile_begin(ctx, max_steps):
    _check(ctx, lib().axpic_profile_begin(ctx, max_steps))


def axpic_profile_end(ctx):
    """(dict kernel -> summed ms, number of steps recorded)."""
    ms = (ctypes.c_double * PROFILE_SLOTS)()
    n = ctypes.c_int32()
    _check(ctx, lib().axpic_profile_end(ctx, ms, ctypes.byref(n)))
    return dict(zip(axpic_step_kernel_names(ctx), list(ms))), n.value


def axpic_sync(ctx):
    _check(ctx, lib().axpic_sync(ctx))


def axpic_destroy(ctx):
    st = lib().axpic_destroy(ctx)
    if st != AXPIC_OK:
        raise AxpicError(st, "axpic_destroy reported a latched error")


def axpic_version():
    return lib().axpic_version().decode()


# ---------------------------------------------------------------- surrogate network
MLP_PARAMS = 10720


def _mlp_check(h, status):
    if status != AXPIC_OK:
        msg = lib().axpic_mlp_last_error(h)
        raise AxpicError(status, msg.decode() if msg else "")


def axpic_mlp_create(stream):
    h = ctypes.c_void_p()
    st = lib().axpic_mlp_create(ctypes.byref(h), stream)
    if st != AXPIC_OK:
        raise AxpicError(st, "axpic_mlp_create failed")
    return h


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def axpic_mlp_set_params(h, params):
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == MLP_PARAMS
    _mlp_check(h, lib().axpic_mlp_set_params(h, _fptr(p)))


def axpic_mlp_get_params(h):
    import numpy as np
    p = np.empty(MLP_PARAMS, dtype=np.float32)
    _mlp_check(h, lib().axpic_mlp_get_params(h, _fptr(p)))
    return p


def axpic_mlp_forward(h, X_ptr, n, Z_ptr):
    _mlp_check(h, lib().axpic_mlp_forward(h, X_ptr, n, Z_ptr))


def axpic_mlp_gradients(h, X_ptr, Zt_ptr, n):
    import numpy as np
    g = np.empty(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_double()
    _mlp_check(h, lib().axpic_mlp_gradients(h, X_ptr, Zt_ptr, n, ctypes.byref(loss), _fptr(g)))
    return loss.value, g


def axpic_mlp_train_step(h, X_ptr, Zt_ptr, n, lr, want_loss=True):
    loss = ctypes.c_double()
    _mlp_check(h, lib().axpic_mlp_train_step(h, X_ptr, Zt_ptr, n, lr, ctypes.byref(loss) if want_loss else None))
    return loss.value if want_loss else None


def axpic_mlp_destroy(h):
    _mlp_check(h, lib().axpic_mlp_destroy(h))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def axpic_surrogate_targets(rows, brems_shape=1.70):
    """rows: (n, 4) of (x, kappa/T, n_e, Z) -> (n, 96) float64."""
    import numpy as np
    r = np.ascontiguousarray(rows, dtype=np.float64).reshape(-1, 4)
    out = np.empty((len(r), 96))
    st = lib().axpic_surrogate_targets(_dptr(r), len(r), brems_shape, _dptr(out))
    if st != AXPIC_OK:
        raise AxpicError(st, "axpic_surrogate_targets")
    return out


def axpic_surrogate_features(rows):
    import numpy as np
    r = np.ascontiguousarray(rows, dtype=np.float64).reshape(-1, 4)
    out = np.empty((len(r), 4), dtype=np.float32)
    st = lib().axpic_surrogate_features(_dptr(r), len(r), _fptr(out))
    if st != AXPIC_OK:
        raise AxpicError(st, "axpic_surrogate_features")
    return out


def axpic_mlp_set_norm(h, mu, sigma):
    import numpy as np
    m = np.ascontiguousarray(mu, dtype=np.float32)
    s = np.ascontiguousarray(sigma, dtype=np.float32)
    _mlp_check(h, lib().axpic_mlp_set_norm(h, _fptr(m), _fptr(s)))


def axpic_mlp_get_norm(h):
    import numpy as np
    m = np.empty(96, dtype=np.float32)
    s = np.empty(96, dtype=np.float32)
    _mlp_check(h, lib().axpic_mlp_get_norm(h, _fptr(m), _fptr(s)))
    return m, s


def axpic_mlp_set_skip(h, skip):
    """The model's FP32 linear map S[96][4]."""
    import numpy as np
    a = np.ascontiguousarray(skip, dtype=np.float32).reshape(96 * 4)
    _mlp_check(h, lib().axpic_mlp_set_skip(h, _fptr(a)))


def axpic_mlp_get_skip(h):
    import numpy as np
    a = np.empty(96 * 4, dtype=np.float32)
    _mlp_check(h, lib().axpic_mlp_get_skip(h, _fptr(a)))
    return a.reshape(96, 4)


def axpic_surrogate_fit(h, ncells, x_per_cell, steps, batch, lr, seed=0, brems_shape=1.70):
    loss = ctypes.c_double()
    _mlp_check(h, lib().axpic_surrogate_fit(h, ncells, x_per_cell, steps, batch, lr, seed, brems_shape,
                                            ctypes.byref(loss)))
    return loss.value


def axpic_surrogate_validate(h, nT, nne, brems_shape=1.70):
    """(2, nne, nT, 3) array per grid node, indexed [Z - 1, j, i]: largest
    ln-rate error, largest relative error of the Compton-like and
    bremsstrahlung quantiles, and of the Primakoff quantiles."""
    import numpy as np
    out = np.empty(nT * nne * 2 * 3, dtype=np.float32)
    _mlp_check(h, lib().axpic_surrogate_validate(h, nT, nne, brems_shape, _fptr(out)))
    return out.reshape(2, nne, nT, 3)


def axpic_set_surrogate(ctx, net_handle, err_map, nT, nne, tol_rate, tol_quantile=1e-3):
    """err_map: axpic_surrogate_validate's array for the same (nT, nne)."""
    import numpy as np
    e = np.ascontiguousarray(err_map, dtype=np.float32).reshape(-1)
    assert e.size == 2 * nT * nne * 3
    _check(ctx, lib().axpic_set_surrogate(ctx, net_handle, _fptr(e), nT, nne, tol_rate, tol_quantile))


def axpic_get_cell_records(ctx, first, count):
    """(records [count, 16] float32, sources [count] uint8: 1 = the cell's
    rates come from its spectral record)."""
    import numpy as np
    rec = np.empty((max(count, 1), 16), dtype=np.float32)
    src = np.empty(max(count, 1), dtype=np.uint8)
    _check(ctx, lib().axpic_get_cell_records(ctx, first, count, _fptr(rec), src.ctypes.data_as(ctypes.c_void_p)))
    return rec[:count], src[:count]


def axpic_stream_axions(ctx, dims, h_cm, dt_s, boundary, mass_keV=0.0):
    nx, ny, nz = dims
    _check(ctx, lib().axpic_stream_axions(ctx, nx, ny, nz, h_cm, dt_s, mass_keV, boundary))


def axpic_run_steps_streamed(ctx, first, nsteps, mask, dims, h_cm, dt_s, boundary, mass_keV=0.0):
    nx, ny, nz = dims
    _check(ctx, lib().axpic_run_steps_streamed(ctx, first, nsteps, mask, nx, ny, nz, h_cm, dt_s, mass_keV, boundary))


def axpic_merge_axions(ctx, n_target, edges_p2):
    import numpy as np
    e = np.ascontiguousarray(edges_p2, dtype=np.float32)
    _check(ctx, lib().axpic_merge_axions(ctx, n_target, e.size, _fptr(e) if e.size else None))


def axpic_deposit_composition(ctx, bind_species, mass_frac, n_ion_out_ptr):
    import numpy as np
    x = None if mass_frac is None else np.ascontiguousarray(mass_frac, dtype=np.float64)
    xp = None if x is None else x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(ctx, lib().axpic_deposit_composition(ctx, bind_species, xp, n_ion_out_ptr))


def axpic_merge_stats(ctx):
    out = ctypes.c_double()
    _check(ctx, lib().axpic_merge_stats(ctx, ctypes.byref(out)))
    return out.value


def axpic_save_state(ctx):
    import numpy as np
    n = ctypes.c_uint64()
    _check(ctx, lib().axpic_state_bytes(ctx, ctypes.byref(n)))
    out = np.empty(max(n.value, 1), dtype=np.uint8)
    _check(ctx, lib().axpic_save_state(ctx, out.ctypes.data_as(ctypes.c_void_p), n.value))
    return out[:n.value]


def axpic_load_state(ctx, buf):
    import numpy as np
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(ctx, lib().axpic_load_state(ctx, buf.ctypes.data_as(ctypes.c_void_p), buf.size))


def axpic_stream_stats(ctx):
    import numpy as np
    out = np.zeros(4, dtype=np.float64)
    _check(ctx, lib().axpic_stream_stats(ctx, _dptr(out)))
    return out


def axpic_get_spectral_records(ctx, first, count):
    import numpy as np
    out = np.empty((max(count, 1), 192), dtype=np.float32)
    _check(ctx, lib().axpic_get_spectral_records(ctx, first, count, _fptr(out)))
    return out[:count]
