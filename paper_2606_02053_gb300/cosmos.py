"""Thin ctypes binding of libcosmos_gb300.so (declared in include/cosmos.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch CUDA tensors (float64); streams are torch
CUDA streams.  Functions keep the C names and return the C error code,
except that ``check`` raises ``CosmosError`` on a non-zero code.

If the shared library is missing this module raises on import of any entry
point: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcosmos_gb300.so")

COSMOS_OK = 0
COSMOS_EINVAL = -1
COSMOS_ECUDA = -2
COSMOS_EWORKSPACE = -3
COSMOS_EALIGN = -4
COSMOS_ENONFINITE = -5
COSMOS_EIO = -6
COSMOS_ECHECKPOINT = -7
COSMOS_OP_RHS, COSMOS_OP_RK4, COSMOS_OP_CONSTRAINTS, COSMOS_OP_INIT = 0, 1, 2, 3
COSMOS_OP_VJP, COSMOS_OP_ADJOINT, COSMOS_OP_INIT_VJP, COSMOS_OP_DIAG = 4, 5, 6, 7
COSMOS_OP_SCAN = 8


class cosmos_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("pitch", ctypes.c_int),
                ("h", ctypes.c_double * 3), ("x0", ctypes.c_double * 3)]


class cosmos_params(ctypes.Structure):
    _fields_ = [("slicing", ctypes.c_int), ("shift", ctypes.c_int), ("fluid", ctypes.c_int), ("scalar", ctypes.c_int),
                ("eta", ctypes.c_double), ("ko_sigma", ctypes.c_double), ("w", ctypes.c_double),
                ("H0", ctypes.c_double), ("t0", ctypes.c_double)]


class cosmos_id(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("A", ctypes.c_double), ("mu", ctypes.c_double), ("sigma", ctypes.c_double),
                ("q", ctypes.c_double * 3), ("center", ctypes.c_double * 3), ("a0", ctypes.c_double),
                ("t", ctypes.c_double)]


class cosmos_batch_tuning(ctypes.Structure):
    _fields_ = [("mapping", ctypes.c_int), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
                ("blocks_per_sm", ctypes.c_int)]


COSMOS_FMR_MAX_LEVELS = 8


class cosmos_fmr(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("grid", cosmos_grid * COSMOS_FMR_MAX_LEVELS),
                ("origin", (ctypes.c_int * 3) * COSMOS_FMR_MAX_LEVELS),
                ("lo", (ctypes.c_int * 3) * COSMOS_FMR_MAX_LEVELS),
                ("hi", (ctypes.c_int * 3) * COSMOS_FMR_MAX_LEVELS)]


class CosmosError(RuntimeError):
    pass


_lib = None
_P = ctypes.c_void_p
_G = ctypes.POINTER(cosmos_grid)
_PP = ctypes.POINTER(cosmos_params)
_IDP = ctypes.POINTER(cosmos_id)
_FP = ctypes.POINTER(cosmos_fmr)
_D = ctypes.c_double
_S = ctypes.c_size_t

_SIGS = {
    "cosmos_nfields": ([_PP], ctypes.c_int),
    "cosmos_field_stride": ([_G], ctypes.c_size_t),
    "cosmos_workspace_bytes": ([_G, _PP, ctypes.c_int], ctypes.c_size_t),
    "cosmos_init_grid": ([_G, _PP, _IDP, _P, _P, _S, _P], ctypes.c_int),
    "cosmos_rhs": ([_G, _PP, _P, _P, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_rk4_stage": ([_G, _PP, ctypes.c_int, _P, _P, _P, _P, _D, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_rk4_step": ([_G, _PP, _P, _D, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_rk4_step_stages": ([_G, _PP, _P, _D, _D, _P, _P, _P, _P, _S, _P], ctypes.c_int),
    "cosmos_field_exponents": ([_G, _PP, _P, _P, _P], ctypes.c_int),
    "cosmos_rk4_stage_slab": ([_G, _PP, ctypes.c_int, _P, _P, _P, _P, _D, _D, ctypes.c_int, ctypes.c_int, _P, _P, _S,
                               _P], ctypes.c_int),
    "cosmos_stage_pass": ([_G, _PP, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _D, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_evolve_host": ([_G, _PP, _P, _P, _P, ctypes.c_int, _D, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_evolve_host_many": ([_G, _PP, ctypes.c_int, _P, _P, _P, ctypes.c_int, ctypes.c_int, _D, _D, _P, _S, _P],
                                ctypes.c_int),
    "cosmos_constraints": ([_G, _PP, _P, _P, ctypes.POINTER(ctypes.c_double), _P, _S, _P], ctypes.c_int),
    "cosmos_constraints_noalloc": ([_G, _PP, _P, _P, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "cosmos_checkpoint_save": ([ctypes.c_char_p, _G, _PP, _P, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, _P],
                               ctypes.c_int),
    "cosmos_checkpoint_load": ([ctypes.c_char_p, _G, _PP, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_longlong), _P], ctypes.c_int),
    "cosmos_scan_state": ([_G, _PP, _P, ctypes.POINTER(ctypes.c_int), _P, _S, _P], ctypes.c_int),
    "cosmos_probe_fp64": ([_P, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "cosmos_adjoint_workspace_bytes": ([_G, _PP, ctypes.c_int], ctypes.c_size_t),
    "cosmos_rhs_vjp": ([_G, _PP, _P, _P, _P, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_adjoint_step": ([_G, _PP, _P, _P, _P, _D, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_adjoint_step_stages": ([_G, _PP, _P, _P, _P, _P, _P, _P, _D, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_init_zeta": ([_G, _PP, _P, _D, _P, _P, _S, _P], ctypes.c_int),
    "cosmos_init_zeta_vjp": ([_G, _PP, _P, _P, _P, _P, _S, _P], ctypes.c_int),
    "cosmos_compaction": ([_G, _PP, _P, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                           ctypes.POINTER(ctypes.c_double), _P, _S, _P], ctypes.c_int),
    "cosmos_compaction_vjp": ([_G, _PP, _P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _D, _P, _P],
                              ctypes.c_int),
    "cosmos_central_lapse": ([_G, _PP, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "cosmos_central_lapse_vjp": ([_G, _PP, _D, _P, _P], ctypes.c_int),
    "cosmos_series_argmin": ([_P, ctypes.c_int, _P, _P], ctypes.c_int),
    "cosmos_batch_workspace_bytes": ([ctypes.c_int, _G, _PP, ctypes.c_int], ctypes.c_size_t),
    "cosmos_batch_plan": ([ctypes.c_int, _G, _PP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(cosmos_batch_tuning), _P, _S,
                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "cosmos_batch_set_tuning": ([_P, ctypes.POINTER(cosmos_batch_tuning)], ctypes.c_int),
    "cosmos_batch_run": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P], ctypes.c_int),
    "cosmos_batch_time_stage": ([_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "cosmos_batch_default_candidates": ([ctypes.POINTER(cosmos_batch_tuning), ctypes.c_int], ctypes.c_int),
    "cosmos_batch_autotune": ([_P, ctypes.POINTER(cosmos_batch_tuning), ctypes.c_int, ctypes.c_int, ctypes.c_char_p,
                               ctypes.POINTER(cosmos_batch_tuning), ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_int), _P], ctypes.c_int),
    "cosmos_batch_free": ([_P], None),
    "cosmos_fmr_workspace_bytes": ([_FP, _PP], ctypes.c_size_t),
    "cosmos_fmr_init": ([_FP, _PP, _IDP, ctypes.POINTER(ctypes.c_void_p), _P, _S, _P], ctypes.c_int),
    "cosmos_fmr_step": ([_FP, _PP, ctypes.POINTER(ctypes.c_void_p), _D, _D, _P, _S, _P], ctypes.c_int),
    "cosmos_fmr_prolong": ([_FP, _PP, ctypes.c_int, _P, _P, _P, _S, _P], ctypes.c_int),
    "cosmos_fmr_restrict": ([_FP, _PP, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "cosmos_last_cuda_error": ([], ctypes.c_int),
    "cosmos_strerror": ([ctypes.c_int], ctypes.c_char_p),
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CosmosError(f"{LIB_PATH} is missing: build it with paper_2606_02053_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def check(code: int):
    if code != COSMOS_OK:
        msg = lib().cosmos_strerror(code).decode()
        extra = f" (cudaError {lib().cosmos_last_cuda_error()})" if code == COSMOS_ECUDA else ""
        raise CosmosError(f"cosmos error {code}: {msg}{extra}")
    return code


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ws(ws):
    if ws is None:
        return None, 0
    return _ptr(ws), ws.numel() * ws.element_size()


# ---- C entry points (same names) ----------------------------------------------
def cosmos_nfields(p: cosmos_params) -> int:
    return lib().cosmos_nfields(ctypes.byref(p))


def cosmos_field_stride(g: cosmos_grid) -> int:
    return lib().cosmos_field_stride(ctypes.byref(g))


def cosmos_workspace_bytes(g: cosmos_grid, p: cosmos_params, op: int) -> int:
    return lib().cosmos_workspace_bytes(ctypes.byref(g), ctypes.byref(p), op)


def cosmos_init_grid(g, p, ident, state, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_init_grid(ctypes.byref(g), ctypes.byref(p), ctypes.byref(ident), _ptr(state), w, nb,
                                  _stream(stream))


def cosmos_rhs(g, p, state, rhs, t, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_rhs(ctypes.byref(g), ctypes.byref(p), _ptr(state), _ptr(rhs), float(t), w, nb,
                            _stream(stream))


def cosmos_rk4_stage(g, p, stage, U_s, U_n, U_next, acc, t, dt, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_rk4_stage(ctypes.byref(g), ctypes.byref(p), int(stage), _ptr(U_s), _ptr(U_n), _ptr(U_next),
                                  _ptr(acc), float(t), float(dt), w, nb, _stream(stream))


def cosmos_field_exponents(g, p, state, E, stream=None) -> int:
    return lib().cosmos_field_exponents(ctypes.byref(g), ctypes.byref(p), _ptr(state), _ptr(E), _stream(stream))


def cosmos_rk4_stage_slab(g, p, stage, U_s, U_n, U_next, acc, t, dt, k_lo, k_cnt, E=None, ws=None,
                          stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_rk4_stage_slab(ctypes.byref(g), ctypes.byref(p), int(stage), _ptr(U_s), _ptr(U_n),
                                       _ptr(U_next), _ptr(acc), float(t), float(dt), int(k_lo), int(k_cnt), _ptr(E),
                                       w, nb, _stream(stream))


def cosmos_stage_pass(g, p, pss, stage, U_s, U_n, U_next, acc, t, dt, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_stage_pass(ctypes.byref(g), ctypes.byref(p), int(pss), int(stage), _ptr(U_s), _ptr(U_n),
                                   _ptr(U_next), _ptr(acc), float(t), float(dt), w, nb, _stream(stream))


def cosmos_rk4_step(g, p, state, t, dt, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_rk4_step(ctypes.byref(g), ctypes.byref(p), _ptr(state), float(t), float(dt), w, nb,
                                 _stream(stream))


def cosmos_rk4_step_stages(g, p, state, t, dt, U2, U3, U4, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_rk4_step_stages(ctypes.byref(g), ctypes.byref(p), _ptr(state), float(t), float(dt),
                                        _ptr(U2), _ptr(U3), _ptr(U4), w, nb, _stream(stream))


def cosmos_evolve_host(g, p, host_in, host_out, dev_state, steps, t, dt, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_evolve_host(ctypes.byref(g), ctypes.byref(p), _ptr(host_in), _ptr(host_out),
                                    _ptr(dev_state), int(steps), float(t), float(dt), w, nb, _stream(stream))


def cosmos_evolve_host_many(g, p, host_in, host_out, dev_states, steps, t, dt, ws=None, stream=None) -> int:
    """host_in, host_out: sequences of host tensors (one per state); dev_states: device buffers."""
    n = len(host_in)
    if len(host_out) != n:
        return COSMOS_EINVAL
    ins = (ctypes.c_void_p * max(n, 1))(*[_ptr(x) for x in host_in])
    outs = (ctypes.c_void_p * max(n, 1))(*[_ptr(x) for x in host_out])
    devs = (ctypes.c_void_p * max(len(dev_states), 1))(*[_ptr(x) for x in dev_states])
    w, nb = _ws(ws)
    return lib().cosmos_evolve_host_many(ctypes.byref(g), ctypes.byref(p), n, ins, outs, devs, len(dev_states),
                                         int(steps), float(t), float(dt), w, nb, _stream(stream))


def cosmos_constraints(g, p, state, ham_mom, norms_out, ws=None, stream=None) -> int:
    """norms_out: a ctypes double[8] (or anything exposing 8 writable doubles)."""
    w, nb = _ws(ws)
    return lib().cosmos_constraints(ctypes.byref(g), ctypes.byref(p), _ptr(state), _ptr(ham_mom), norms_out, w, nb,
                                    _stream(stream))


def cosmos_constraints_noalloc(g, p, state, ham_mom, norms_out, stream=None) -> int:
    """cosmos_constraints with the library's static scratch (no workspace argument)."""
    return lib().cosmos_constraints_noalloc(ctypes.byref(g), ctypes.byref(p), _ptr(state), _ptr(ham_mom), norms_out,
                                            _stream(stream))


def _state_arg(state):
    """(pointer, on_device) of a torch tensor (CUDA or CPU) or a C-contiguous numpy array."""
    if hasattr(state, "data_ptr"):
        return ctypes.c_void_p(state.data_ptr()), int(state.is_cuda)
    return ctypes.c_void_p(state.ctypes.data), 0


def cosmos_checkpoint_save(path, g, p, state, t, step, stream=None) -> int:
    """state: a device tensor, or a host tensor / numpy array, in the state layout."""
    ptr, dev = _state_arg(state)
    return lib().cosmos_checkpoint_save(os.fsencode(path), ctypes.byref(g), ctypes.byref(p), ptr, dev, float(t),
                                        int(step), _stream(stream) if dev else None)


def cosmos_checkpoint_load(path, g, p, state, stream=None):
    """Returns (code, t, step); state is overwritten only on success."""
    ptr, dev = _state_arg(state)
    t = ctypes.c_double(0.0)
    step = ctypes.c_longlong(0)
    code = lib().cosmos_checkpoint_load(os.fsencode(path), ctypes.byref(g), ctypes.byref(p), ptr, dev,
                                        ctypes.byref(t), ctypes.byref(step), _stream(stream) if dev else None)
    return code, t.value, step.value


def cosmos_scan_state(g, p, state, ws=None, stream=None):
    """Returns (code, per-field counts of non-finite values / tau~ <= 0)."""
    nf = cosmos_nfields(p)
    counts = (ctypes.c_int * nf)()
    w, nb = _ws(ws)
    code = lib().cosmos_scan_state(ctypes.byref(g), ctypes.byref(p), _ptr(state), counts, w, nb, _stream(stream))
    return code, list(counts)


def cosmos_probe_fp64(scratch, stream=None) -> float:
    out = ctypes.c_double(0.0)
    check(lib().cosmos_probe_fp64(_ptr(scratch), ctypes.byref(out), _stream(stream)))
    return out.value


def cosmos_adjoint_workspace_bytes(g, p, op) -> int:
    return lib().cosmos_adjoint_workspace_bytes(ctypes.byref(g), ctypes.byref(p), int(op))


def cosmos_rhs_vjp(g, p, U, w, v, t, ws=None, stream=None) -> int:
    wp, nb = _ws(ws)
    return lib().cosmos_rhs_vjp(ctypes.byref(g), ctypes.byref(p), _ptr(U), _ptr(w), _ptr(v), float(t), wp, nb,
                                _stream(stream))


def cosmos_adjoint_step(g, p, U_n, lam_np1, lam_n, t, dt, ws=None, stream=None) -> int:
    wp, nb = _ws(ws)
    return lib().cosmos_adjoint_step(ctypes.byref(g), ctypes.byref(p), _ptr(U_n), _ptr(lam_np1), _ptr(lam_n),
                                     float(t), float(dt), wp, nb, _stream(stream))


def cosmos_adjoint_step_stages(g, p, U_n, U2, U3, U4, lam_np1, lam_n, t, dt, ws=None, stream=None) -> int:
    wp, nb = _ws(ws)
    return lib().cosmos_adjoint_step_stages(ctypes.byref(g), ctypes.byref(p), _ptr(U_n), _ptr(U2), _ptr(U3),
                                            _ptr(U4), _ptr(lam_np1), _ptr(lam_n), float(t), float(dt), wp, nb,
                                            _stream(stream))


def cosmos_init_zeta(g, p, zeta, a0, state, ws=None, stream=None) -> int:
    wp, nb = _ws(ws)
    return lib().cosmos_init_zeta(ctypes.byref(g), ctypes.byref(p), _ptr(zeta), float(a0), _ptr(state), wp, nb,
                                  _stream(stream))


def cosmos_init_zeta_vjp(g, p, state0, lam0, zeta_bar, ws=None, stream=None) -> int:
    wp, nb = _ws(ws)
    return lib().cosmos_init_zeta_vjp(ctypes.byref(g), ctypes.byref(p), _ptr(state0), _ptr(lam0), _ptr(zeta_bar),
                                      wp, nb, _stream(stream))


def cosmos_compaction(g, p, state, kmax, ws=None, stream=None):
    """Returns (code, C[kmax] list, aux ctypes array)."""
    C = (ctypes.c_double * kmax)()
    aux = (ctypes.c_double * (4 * kmax + 2))()
    wp, nb = _ws(ws)
    code = lib().cosmos_compaction(ctypes.byref(g), ctypes.byref(p), _ptr(state), C, int(kmax), aux, wp, nb,
                                   _stream(stream))
    return code, list(C), aux


def cosmos_compaction_vjp(g, p, state, kstar, kmax, aux, cbar, lam, stream=None) -> int:
    return lib().cosmos_compaction_vjp(ctypes.byref(g), ctypes.byref(p), _ptr(state), int(kstar), int(kmax), aux,
                                       float(cbar), _ptr(lam), _stream(stream))


def cosmos_central_lapse(g, p, state, series, index, stream=None) -> int:
    return lib().cosmos_central_lapse(ctypes.byref(g), ctypes.byref(p), _ptr(state), _ptr(series), int(index),
                                      _stream(stream))


def cosmos_central_lapse_vjp(g, p, abar, lam, stream=None) -> int:
    return lib().cosmos_central_lapse_vjp(ctypes.byref(g), ctypes.byref(p), float(abar), _ptr(lam), _stream(stream))


def cosmos_series_argmin(series, count, result, stream=None) -> int:
    return lib().cosmos_series_argmin(_ptr(series), int(count), _ptr(result), _stream(stream))


def cosmos_batch_workspace_bytes(grids, p, max_steps) -> int:
    arr = (cosmos_grid * len(grids))(*grids)
    return lib().cosmos_batch_workspace_bytes(len(grids), arr, ctypes.byref(p), int(max_steps))


def cosmos_batch_plan(grids, p, dts, t0s, states, max_steps, tuning, ws):
    """Returns (code, plan handle as c_void_p)."""
    n = len(grids)
    arr = (cosmos_grid * n)(*grids)
    dt = (ctypes.c_double * n)(*dts)
    t0 = (ctypes.c_double * n)(*t0s)
    st = (ctypes.c_void_p * n)(*[s.data_ptr() for s in states])
    plan = ctypes.c_void_p()
    w, nb = _ws(ws)
    code = lib().cosmos_batch_plan(n, arr, ctypes.byref(p), dt, t0, st, int(max_steps),
                                   None if tuning is None else ctypes.byref(tuning), w, nb, ctypes.byref(plan))
    return code, plan


def cosmos_batch_set_tuning(plan, tuning) -> int:
    return lib().cosmos_batch_set_tuning(plan, ctypes.byref(tuning))


def cosmos_batch_run(plan, first_step, steps, use_graph, stream=None) -> int:
    return lib().cosmos_batch_run(plan, int(first_step), int(steps), int(use_graph), _stream(stream))


def cosmos_batch_time_stage(plan, reps, stream=None):
    ms = ctypes.c_double(0.0)
    code = lib().cosmos_batch_time_stage(plan, int(reps), ctypes.byref(ms), _stream(stream))
    return code, ms.value


def cosmos_batch_default_candidates():
    """The autotuner's built-in candidate tunings, as cosmos_batch_tuning structs."""
    n = lib().cosmos_batch_default_candidates(None, 0)
    arr = (cosmos_batch_tuning * n)()
    lib().cosmos_batch_default_candidates(arr, n)
    return list(arr)


def cosmos_batch_autotune(plan, candidates, reps, cache_path=None, stream=None):
    """Returns (code, best tuning, per-candidate ms, cache hit); candidates =
    None or [] takes the library's built-in list."""
    cands = list(candidates or [])
    arr = (cosmos_batch_tuning * len(cands))(*cands) if cands else None
    nms = len(cands) or lib().cosmos_batch_default_candidates(None, 0)
    ms = (ctypes.c_double * nms)()
    best = cosmos_batch_tuning()
    hit = ctypes.c_int(0)
    code = lib().cosmos_batch_autotune(plan, arr, len(cands), int(reps),
                                       None if cache_path is None else os.fsencode(cache_path), ctypes.byref(best),
                                       ms, ctypes.byref(hit), _stream(stream))
    return code, best, list(ms), bool(hit.value)


def cosmos_batch_free(plan) -> None:
    lib().cosmos_batch_free(plan)


def _state_ptrs(states):
    return (ctypes.c_void_p * len(states))(*[s.data_ptr() for s in states])


def cosmos_fmr_workspace_bytes(m, p) -> int:
    return lib().cosmos_fmr_workspace_bytes(ctypes.byref(m), ctypes.byref(p))


def cosmos_fmr_init(m, p, ident, states, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_fmr_init(ctypes.byref(m), ctypes.byref(p), ctypes.byref(ident), _state_ptrs(states), w, nb,
                                 _stream(stream))


def cosmos_fmr_step(m, p, states, t, dt0, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_fmr_step(ctypes.byref(m), ctypes.byref(p), _state_ptrs(states), float(t), float(dt0), w, nb,
                                 _stream(stream))


def cosmos_fmr_prolong(m, p, level, parent, child, ws=None, stream=None) -> int:
    w, nb = _ws(ws)
    return lib().cosmos_fmr_prolong(ctypes.byref(m), ctypes.byref(p), int(level), _ptr(parent), _ptr(child), w, nb,
                                    _stream(stream))


def cosmos_fmr_restrict(m, p, level, child, parent, stream=None) -> int:
    return lib().cosmos_fmr_restrict(ctypes.byref(m), ctypes.byref(p), int(level), _ptr(child), _ptr(parent),
                                     _stream(stream))


# ---- convenience constructors (plain data) -----------------------------------
def make_grid(n, h, x0=(0.0, 0.0, 0.0), pitch=None) -> cosmos_grid:
    nx, ny, nz = (n, n, n) if isinstance(n, int) else n
    hh = (h, h, h) if isinstance(h, (int, float)) else h
    g = cosmos_grid()
    g.nx, g.ny, g.nz = nx, ny, nz
    g.pitch = nx if pitch is None else pitch
    g.h[:] = list(hh)
    g.x0[:] = list(x0)
    return g


def make_params(slicing=0, shift=1, fluid=0, scalar=0, eta=2.0, ko_sigma=0.1, w=1.0 / 3.0, H0=0.0,
                t0=0.0) -> cosmos_params:
    p = cosmos_params()
    p.slicing, p.shift, p.fluid, p.scalar = slicing, shift, fluid, scalar
    p.eta, p.ko_sigma, p.w, p.H0, p.t0 = eta, ko_sigma, w, H0, t0
    return p


def make_id(kind, A=0.0, mu=0.0, sigma=0.125, q=(1.0, 1.0, 1.0), center=(0.0, 0.0, 0.0), a0=1.0, t=0.0) -> cosmos_id:
    d = cosmos_id()
    d.kind, d.A, d.mu, d.sigma = kind, A, mu, sigma
    d.q[:] = list(q)
    d.center[:] = list(center)
    d.a0, d.t = a0, t
    return d


def make_fmr(levels, pitch_align=1) -> cosmos_fmr:
    """cosmos_fmr from a list of per-level dicts (n, h, x0, origin, lo, hi), as
    inputs.nested_boxes returns; rows padded to a multiple of pitch_align."""
    if not 1 <= len(levels) <= COSMOS_FMR_MAX_LEVELS:
        raise ValueError("1 to %d levels" % COSMOS_FMR_MAX_LEVELS)
    m = cosmos_fmr()
    m.levels = len(levels)
    for l, lv in enumerate(levels):
        nx = int(lv["n"][0])
        pitch = -(-nx // pitch_align) * pitch_align
        m.grid[l] = make_grid(tuple(int(v) for v in lv["n"]), tuple(float(v) for v in lv["h"]),
                              tuple(float(v) for v in lv["x0"]), pitch=pitch)
        for d in range(3):
            m.origin[l][d] = int(lv["origin"][d])
            m.lo[l][d] = int(lv["lo"][d])
            m.hi[l][d] = int(lv["hi"][d])
    return m
