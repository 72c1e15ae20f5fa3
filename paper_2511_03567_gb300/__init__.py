"""Python binding of the GB300 spin-free RIC-MRCCSD library (libricmrcc.so).

Argument marshalling only: every step of the residual, energy and solver
runs in the library's CUDA kernels.  Host arrays are numpy float64; device
arrays are CUDA torch tensors (float64, contiguous) passed to the *_dev calls.
Importing works without a GPU; creating a handle needs the built library and
a CUDA device and raises if either is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libricmrcc.so")

OK, EINVAL, ENOMEM, ECUDA, NOT_CONVERGED, DIVERGED, ESTATE, ENOTSUP = range(8)
RDM, CUMULANT = 0, 1
FP64, MIXED, EMULATED = 0, 1, 2
METHOD_RIC, METHOD_FULL = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "NOT_CONVERGED",
                5: "DIVERGED", 6: "ESTATE", 7: "ENOTSUP"}

T1_NAMES = ("IA", "IT", "TA")
T2_NAMES = ("IJAB", "IJTA", "IJTU", "ITAB", "ITUA", "ITAU", "ITUV", "TUAB", "TUVA")


class Layout(ctypes.Structure):
    _fields_ = [("t1_size", ctypes.c_int64), ("t2_size", ctypes.c_int64),
                ("t1_offset", ctypes.c_int64 * 3), ("t1_shape", (ctypes.c_int32 * 2) * 3),
                ("t2_offset", ctypes.c_int64 * 9), ("t2_shape", (ctypes.c_int32 * 4) * 9)]


class Opts(ctypes.Structure):
    _fields_ = [("s", ctypes.c_double), ("max_iter", ctypes.c_int), ("e_tol", ctypes.c_double),
                ("t_tol", ctypes.c_double), ("diis_size", ctypes.c_int),
                ("diis_start", ctypes.c_int), ("precision", ctypes.c_int),
                ("refine_tol", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int),
                ("fp64_iterations", ctypes.c_int), ("mixed_iterations", ctypes.c_int),
                ("diverged", ctypes.c_int), ("energy", ctypes.c_double), ("e0", ctypes.c_double),
                ("max_dt", ctypes.c_double), ("seconds", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("residual_terms", ctypes.c_int64), ("residual_launches", ctypes.c_int64),
                ("step_launches", ctypes.c_int64), ("residual_flops", ctypes.c_double),
                ("arena_bytes", ctypes.c_double), ("table_bytes", ctypes.c_double),
                ("kind_launches", ctypes.c_int64 * 3), ("kind_flops", ctypes.c_double * 3),
                ("tc_contractions", ctypes.c_int64), ("tc_flops", ctypes.c_double),
                ("tc_pack_bytes", ctypes.c_double), ("graph_launches", ctypes.c_int64 * 2),
                ("kernel_ops", ctypes.c_int64 * 8), ("kernel_work", ctypes.c_double * 8),
                ("tc_gemm_bytes", ctypes.c_double), ("tc_grouped_ops", ctypes.c_int64),
                ("tc_weighted_ops", ctypes.c_int64), ("oz_contractions", ctypes.c_int64),
                ("oz_flops", ctypes.c_double)]


class TileRule(ctypes.Structure):
    _fields_ = [("tc_min_flops", ctypes.c_double), ("skinny", ctypes.c_int), ("tc_grouped", ctypes.c_int),
                ("tc_min_n", ctypes.c_int), ("oz_max_pad", ctypes.c_double)]


TUNE_MAX = 8


class Tuning(ctypes.Structure):
    _fields_ = [("n_candidates", ctypes.c_int), ("rule", TileRule * TUNE_MAX),
                ("ms", ctypes.c_double * TUNE_MAX), ("chosen", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("waves", ctypes.c_int), ("grouped_launches", ctypes.c_int64),
                ("tc_contractions", ctypes.c_int64), ("flops", ctypes.c_double),
                ("tc_flops", ctypes.c_double), ("kernel_launches", ctypes.c_int64)]


class LadderInfo(ctypes.Structure):
    _fields_ = [("slabs", ctypes.c_int), ("slab_rows", ctypes.c_int64), ("rebuild_flops", ctypes.c_double),
                ("ladder_flops", ctypes.c_double), ("rebuild_flops_executed", ctypes.c_double),
                ("ladder_flops_executed", ctypes.c_double), ("workspace_bytes", ctypes.c_double),
                ("ms_pack", ctypes.c_double), ("ms_rebuild", ctypes.c_double), ("ms_symmetrise", ctypes.c_double),
                ("ms_ladder", ctypes.c_double), ("ms_unpack", ctypes.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class AdjointInfo(ctypes.Structure):
    _fields_ = [("fp64_applications", ctypes.c_int), ("mixed_applications", ctypes.c_int),
                ("seconds", ctypes.c_double)]


class RicMrccError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_LIB = None
_DP = ctypes.POINTER(ctypes.c_double)


def library_path():
    return LIB_PATH


def load_library():
    """Load libricmrcc.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp = ctypes.c_void_p
    sig = {
        "ricmrcc_create": ([ctypes.c_int] * 4 + [ctypes.POINTER(vp)], ctypes.c_int),
        "ricmrcc_create_method": ([ctypes.c_int] * 5 + [ctypes.POINTER(vp)], ctypes.c_int),
        "ricmrcc_destroy": ([vp], None),
        "ricmrcc_last_error": ([vp], ctypes.c_char_p),
        "ricmrcc_set_stream": ([vp, vp], ctypes.c_int),
        "ricmrcc_set_precision": ([vp, ctypes.c_int], ctypes.c_int),
        "ricmrcc_set_integrals": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_set_integrals_dev": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_set_rdms": ([vp, vp, vp, vp, ctypes.c_int], ctypes.c_int),
        "ricmrcc_set_rdms_dev": ([vp, vp, vp, vp, ctypes.c_int], ctypes.c_int),
        "ricmrcc_semicanonicalize": ([vp, vp], ctypes.c_int),
        "ricmrcc_amplitude_layout": ([vp, ctypes.POINTER(Layout)], ctypes.c_int),
        "ricmrcc_reference": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_residual": ([vp] * 6, ctypes.c_int),
        "ricmrcc_residual_dev": ([vp] * 6, ctypes.c_int),
        "ricmrcc_opts_default": ([ctypes.POINTER(Opts)], ctypes.c_int),
        "ricmrcc_solve": ([vp, ctypes.c_double, ctypes.POINTER(Opts), vp, ctypes.POINTER(Stats)],
                          ctypes.c_int),
        "ricmrcc_get_amplitudes_dev": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_set_amplitudes_dev": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_get_amplitudes": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_step": ([vp, ctypes.POINTER(Opts), ctypes.c_int, ctypes.c_int, vp, vp], ctypes.c_int),
        "ricmrcc_plan_info": ([vp, ctypes.POINTER(PlanInfo)], ctypes.c_int),
        "ricmrcc_profile": ([vp, ctypes.c_int, ctypes.c_int, vp], ctypes.c_int),
        "ricmrcc_set_amplitudes": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_run_largest_ops": ([vp, ctypes.c_int], ctypes.c_int),
        "ricmrcc_energy_backward": ([vp, vp, vp, vp], ctypes.c_int),
        "ricmrcc_energy_backward_dev": ([vp, vp, vp, vp], ctypes.c_int),
        "ricmrcc_get_adjoint_info": ([vp, ctypes.POINTER(AdjointInfo)], ctypes.c_int),
        "ricmrcc_gemm_bf16x3": ([vp, ctypes.c_int64, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                 ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, vp],
                                ctypes.c_int),
        "ricmrcc_gemm_f64_emulated": ([vp, ctypes.c_int64, vp, ctypes.c_int64, vp, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_int, vp], ctypes.c_int),
        "ricmrcc_block_eigh_noalloc": ([vp, ctypes.c_int, vp, vp, vp], ctypes.c_int),
        "ricmrcc_ladder_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(vp)],
                                  ctypes.c_int),
        "ricmrcc_ladder_destroy": ([vp], None),
        "ricmrcc_ladder_last_error": ([vp], ctypes.c_char_p),
        "ricmrcc_ladder_set_stream": ([vp, vp], ctypes.c_int),
        "ricmrcc_ladder_set_factor_dev": ([vp, vp], ctypes.c_int),
        "ricmrcc_ladder_apply_dev": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_ladder_finish": ([vp, ctypes.POINTER(LadderInfo)], ctypes.c_int),
        "ricmrcc_ladder_info": ([vp, ctypes.POINTER(LadderInfo)], ctypes.c_int),
        "ricmrcc_ladder_set_factor": ([vp, vp], ctypes.c_int),
        "ricmrcc_ladder_apply": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_set_wait_limit": ([ctypes.c_double, ctypes.c_int], ctypes.c_int),
        "ricmrcc_get_residual": ([vp, vp, vp], ctypes.c_int),
        "ricmrcc_set_tile_rule": ([vp, ctypes.POINTER(TileRule)], ctypes.c_int),
        "ricmrcc_get_tile_rule": ([vp, ctypes.POINTER(TileRule)], ctypes.c_int),
        "ricmrcc_tune": ([vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Tuning)], ctypes.c_int),
        "ricmrcc_batch_create": ([ctypes.c_int, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "ricmrcc_batch_destroy": ([vp], None),
        "ricmrcc_batch_last_error": ([vp], ctypes.c_char_p),
        "ricmrcc_batch_instance": ([vp, ctypes.c_int, ctypes.POINTER(vp)], ctypes.c_int),
        "ricmrcc_batch_set_integrals": ([vp, ctypes.c_int, vp, vp], ctypes.c_int),
        "ricmrcc_batch_set_rdms": ([vp, ctypes.c_int, vp, vp, vp, ctypes.c_int], ctypes.c_int),
        "ricmrcc_batch_residual": ([vp, ctypes.c_int, vp], ctypes.c_int),
        "ricmrcc_batch_solve": ([vp, ctypes.POINTER(Opts), vp, vp], ctypes.c_int),
        "ricmrcc_batch_solve_flows": ([vp, vp, ctypes.POINTER(Opts), vp, vp], ctypes.c_int),
        "ricmrcc_batch_step": ([vp, ctypes.POINTER(Opts), ctypes.c_int, ctypes.c_int, vp, vp],
                               ctypes.c_int),
        "ricmrcc_batch_tune": ([vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Tuning)], ctypes.c_int),
        "ricmrcc_batch_info": ([vp, ctypes.POINTER(BatchInfo)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _LIB = lib
    return lib


def _ptr(x):
    """Address of a contiguous float64 numpy array or CUDA torch tensor (or None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"], "need contiguous float64"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "need a contiguous tensor"
        return x.data_ptr()
    raise TypeError(type(x))


def _host(x):
    return None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.float64))


class RicMrcc:
    """One problem (sizes fixed at creation) on the current CUDA device."""

    def __init__(self, n_core, n_act, n_virt, n_aux, _borrowed=None, method=METHOD_RIC):
        self.lib = load_library()
        self.dims = (n_core, n_act, n_virt, n_aux)
        self.method = method
        self._owner = None
        if _borrowed is not None:
            # handle owned by a RicMrccBatch (kept alive through _owner)
            h, self._owner = _borrowed
        else:
            h = ctypes.c_void_p()
            rc = self.lib.ricmrcc_create_method(n_core, n_act, n_virt, n_aux, int(method), ctypes.byref(h))
            if rc != OK:
                raise RicMrccError(rc, "ricmrcc_create failed")
        self.h = h
        lay = Layout()
        self._check(self.lib.ricmrcc_amplitude_layout(self.h, ctypes.byref(lay)))
        self.layout = lay

    def _check(self, rc, allow=(OK,)):
        if rc not in allow:
            msg = self.lib.ricmrcc_last_error(self.h).decode()
            raise RicMrccError(rc, msg)
        return rc

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owner", None) is None:
                self.lib.ricmrcc_destroy(self.h)
            self.h = None
            self._owner = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ setup
    def set_stream(self, stream_ptr):
        self._check(self.lib.ricmrcc_set_stream(self.h, stream_ptr))

    def set_precision(self, precision):
        self._check(self.lib.ricmrcc_set_precision(self.h, precision))

    def set_integrals(self, hmat, B):
        if hasattr(hmat, "is_cuda") and hmat.is_cuda:
            self._check(self.lib.ricmrcc_set_integrals_dev(self.h, _ptr(hmat), _ptr(B)))
        else:
            hm, b = _host(hmat), _host(B)
            self._check(self.lib.ricmrcc_set_integrals(self.h, _ptr(hm), _ptr(b)))

    def set_rdms(self, g1, g2, g3, kind=RDM):
        if hasattr(g1, "is_cuda") and g1.is_cuda:
            self._check(self.lib.ricmrcc_set_rdms_dev(self.h, _ptr(g1), _ptr(g2), _ptr(g3), kind))
        else:
            a, b, c = _host(g1), _host(g2), _host(g3)
            self._check(self.lib.ricmrcc_set_rdms(self.h, _ptr(a), _ptr(b), _ptr(c), kind))

    def semicanonicalize(self):
        n = sum(self.dims[:3])
        U = np.zeros((n, n))
        self._check(self.lib.ricmrcc_semicanonicalize(self.h, _ptr(U)))
        return U

    def reference(self):
        n = sum(self.dims[:3])
        e0 = ctypes.c_double()
        F = np.zeros((n, n))
        self._check(self.lib.ricmrcc_reference(self.h, ctypes.byref(e0), _ptr(F)))
        return e0.value, F

    # ------------------------------------------------------------- amplitudes
    def pack(self, T):
        """{class: array} -> (flat T1, flat T2) in the library layout."""
        lay = self.layout
        t1 = np.zeros(lay.t1_size)
        t2 = np.zeros(lay.t2_size)
        for i, nm in enumerate(T1_NAMES):
            shp = tuple(lay.t1_shape[i])
            t1[lay.t1_offset[i]:lay.t1_offset[i] + int(np.prod(shp))] = np.asarray(T[nm]).ravel()
        for i, nm in enumerate(T2_NAMES):
            shp = tuple(lay.t2_shape[i])
            t2[lay.t2_offset[i]:lay.t2_offset[i] + int(np.prod(shp))] = np.asarray(T[nm]).ravel()
        return t1, t2

    def unpack(self, t1, t2):
        lay = self.layout
        out = {}
        for i, nm in enumerate(T1_NAMES):
            shp = tuple(lay.t1_shape[i])
            out[nm] = np.asarray(t1[lay.t1_offset[i]:lay.t1_offset[i] + int(np.prod(shp))]).reshape(shp)
        for i, nm in enumerate(T2_NAMES):
            shp = tuple(lay.t2_shape[i])
            out[nm] = np.asarray(t2[lay.t2_offset[i]:lay.t2_offset[i] + int(np.prod(shp))]).reshape(shp)
        return out

    def residual(self, T):
        """Residual class blocks and energy for amplitudes T (dict or flat pair)."""
        t1, t2 = self.pack(T) if isinstance(T, dict) else (_host(T[0]), _host(T[1]))
        r1 = np.zeros(self.layout.t1_size)
        r2 = np.zeros(self.layout.t2_size)
        e = ctypes.c_double()
        self._check(self.lib.ricmrcc_residual(self.h, _ptr(t1), _ptr(t2), _ptr(r1), _ptr(r2),
                                              ctypes.byref(e)))
        return self.unpack(r1, r2), e.value

    def residual_dev(self, t1, t2, r1, r2, e_out=None):
        """Device-pointer variant: torch CUDA tensors, results written in place."""
        self._check(self.lib.ricmrcc_residual_dev(self.h, _ptr(t1), _ptr(t2), _ptr(r1), _ptr(r2),
                                                  _ptr(e_out)))

    def get_amplitudes(self):
        t1 = np.zeros(self.layout.t1_size)
        t2 = np.zeros(self.layout.t2_size)
        self._check(self.lib.ricmrcc_get_amplitudes(self.h, _ptr(t1), _ptr(t2)))
        return self.unpack(t1, t2)

    def set_amplitudes(self, T):
        t1, t2 = self.pack(T)
        self._check(self.lib.ricmrcc_set_amplitudes(self.h, _ptr(t1), _ptr(t2)))

    def get_amplitudes_dev(self, t1, t2):
        """Stored amplitudes into flat device arrays (torch CUDA float64 tensors)."""
        self._check(self.lib.ricmrcc_get_amplitudes_dev(self.h, _ptr(t1), _ptr(t2)))

    def set_amplitudes_dev(self, t1, t2):
        """Flat device arrays (torch CUDA float64 tensors) into the stored amplitudes."""
        self._check(self.lib.ricmrcc_set_amplitudes_dev(self.h, _ptr(t1), _ptr(t2)))

    # ------------------------------------------------------------------ solve
    @staticmethod
    def default_opts(**kw):
        o = Opts()
        load_library().ricmrcc_opts_default(ctypes.byref(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def solve(self, s=0.5, **kw):
        """Converge the amplitudes at flow s; keyword options as ricmrcc_opts
        (max_iter, e_tol, t_tol, diis_size, diis_start, precision, refine_tol).
        precision FP64: every iteration in FP64; MIXED: split-BF16 tensor-core
        iterations until max|dt| < refine_tol, then FP64 refinement;
        EMULATED: the same, with the refinement's large contractions as
        emulated-FP64 tensor-core products.  Returns (energy, Stats); a
        NOT_CONVERGED outcome is reported in Stats, other failures raise."""
        o = self.default_opts(s=s, **kw)
        st = Stats()
        e = ctypes.c_double()
        rc = self.lib.ricmrcc_solve(self.h, float(s), ctypes.byref(o), ctypes.byref(e), ctypes.byref(st))
        self._check(rc, allow=(OK, NOT_CONVERGED))
        return e.value, st


def _step(self, s=0.5, n_steps=1, restart=False, **kw):
    """n_steps solver iterations without the convergence test (see ricmrcc_step)."""
    o = self.default_opts(s=s, **kw)
    e = ctypes.c_double()
    dt = ctypes.c_double()
    self._check(self.lib.ricmrcc_step(self.h, ctypes.byref(o), n_steps, int(restart),
                                      ctypes.byref(e), ctypes.byref(dt)))
    return e.value, dt.value


def _plan_info(self):
    info = PlanInfo()
    self._check(self.lib.ricmrcc_plan_info(self.h, ctypes.byref(info)))
    return info


PROFILE_KINDS = ("tile_64x64", "tile_16x16", "dot", "tc_pack", "tc_gemm", "tile_128x16", "tile_64x32",
                 "small_long_k")


def _profile(self, reps=3, mixed=False):
    """Mean ms per residual per kernel (names in PROFILE_KINDS), launches serialised."""
    ms = np.zeros(len(PROFILE_KINDS))
    self._check(self.lib.ricmrcc_profile(self.h, reps, int(mixed), _ptr(ms)))
    return ms


def _energy_backward(self):
    """(dE/dh [n,n], dE/dB [n_aux,n,n], dE/ds) of the last converged solve."""
    n = sum(self.dims[:3])
    dh = np.zeros((n, n))
    dB = np.zeros((self.dims[3], n, n))
    ds = ctypes.c_double()
    self._check(self.lib.ricmrcc_energy_backward(self.h, _ptr(dh), _ptr(dB), ctypes.byref(ds)))
    return dh, dB, ds.value


def _energy_backward_dev(self, dh, dB, ds):
    """Device-output variant: CUDA float64 tensors [n,n], [n_aux,n,n], [1]."""
    self._check(self.lib.ricmrcc_energy_backward_dev(self.h, _ptr(dh), _ptr(dB), _ptr(ds)))


def _adjoint_info(self):
    """Applications of the multiplier map (FP64, mixed) and seconds of the last energy_backward."""
    info = AdjointInfo()
    self._check(self.lib.ricmrcc_get_adjoint_info(self.h, ctypes.byref(info)))
    return info


def _get_residual(self):
    """(R1, R2) flat class layout of the last residual evaluation."""
    r1 = np.zeros(self.layout.t1_size)
    r2 = np.zeros(self.layout.t2_size)
    self._check(self.lib.ricmrcc_get_residual(self.h, _ptr(r1), _ptr(r2)))
    return r1, r2


def _set_tile_rule(self, tc_min_flops=1e7, skinny=True, tc_grouped=True, tc_min_n=1, oz_max_pad=4.0):
    r = TileRule(float(tc_min_flops), int(bool(skinny)), int(bool(tc_grouped)), int(tc_min_n), float(oz_max_pad))
    self._check(self.lib.ricmrcc_set_tile_rule(self.h, ctypes.byref(r)))


def _get_tile_rule(self):
    r = TileRule()
    self._check(self.lib.ricmrcc_get_tile_rule(self.h, ctypes.byref(r)))
    return {"tc_min_flops": r.tc_min_flops, "skinny": bool(r.skinny), "tc_grouped": bool(r.tc_grouped),
            "tc_min_n": r.tc_min_n, "oz_max_pad": r.oz_max_pad}


def _tuning_dict(t):
    cands = [{"tc_min_flops": t.rule[i].tc_min_flops, "skinny": bool(t.rule[i].skinny),
              "tc_grouped": bool(t.rule[i].tc_grouped), "tc_min_n": t.rule[i].tc_min_n, "ms": t.ms[i]}
             for i in range(t.n_candidates)]
    return {"candidates": cands, "chosen": t.chosen}


def _tune(self, precision=MIXED, reps=3):
    """Time the captured residual under each candidate tile rule; keep the fastest."""
    t = Tuning()
    self._check(self.lib.ricmrcc_tune(self.h, precision, reps, ctypes.byref(t)))
    return _tuning_dict(t)


RicMrcc.get_residual = _get_residual
RicMrcc.set_tile_rule = _set_tile_rule
RicMrcc.get_tile_rule = _get_tile_rule
RicMrcc.tune = _tune
RicMrcc.energy_backward = _energy_backward
RicMrcc.energy_backward_dev = _energy_backward_dev
RicMrcc.adjoint_info = _adjoint_info
RicMrcc.step = _step
RicMrcc.plan_info = _plan_info
RicMrcc.profile = _profile


class RicMrccBatch:
    """Independent problems of uneven sizes solved together (ricmrcc_batch_*)."""

    def __init__(self, dims):
        self.lib = load_library()
        self.dims = [tuple(int(x) for x in d) for d in dims]
        arr = np.ascontiguousarray(np.array(self.dims, dtype=np.int32).reshape(-1, 4))
        b = ctypes.c_void_p()
        rc = self.lib.ricmrcc_batch_create(len(self.dims), arr.ctypes.data, ctypes.byref(b))
        if rc != OK:
            raise RicMrccError(rc, "ricmrcc_batch_create failed")
        self.b = b
        self.instances = []
        for i, d in enumerate(self.dims):
            h = ctypes.c_void_p()
            self._check(self.lib.ricmrcc_batch_instance(self.b, i, ctypes.byref(h)))
            self.instances.append(RicMrcc(*d, _borrowed=(h, self)))

    @property
    def count(self):
        return len(self.dims)

    def _check(self, rc, allow=(OK,)):
        if rc not in allow:
            raise RicMrccError(rc, self.lib.ricmrcc_batch_last_error(self.b).decode())
        return rc

    def close(self):
        if getattr(self, "b", None):
            for inst in self.instances:
                inst.h = None
                inst._owner = None
            self.lib.ricmrcc_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __getitem__(self, i):
        return self.instances[i]

    def residual(self, precision=FP64):
        """Energies of all instances at their current amplitudes (residuals: get_residual)."""
        e = np.zeros(self.count)
        self._check(self.lib.ricmrcc_batch_residual(self.b, precision, _ptr(e)))
        return e

    def solve(self, s=0.5, **kw):
        o = RicMrcc.default_opts(s=s, **kw)
        e = np.zeros(self.count)
        st = (Stats * self.count)()
        rc = self.lib.ricmrcc_batch_solve(self.b, ctypes.byref(o), _ptr(e), ctypes.cast(st, ctypes.c_void_p))
        self._check(rc, allow=(OK, NOT_CONVERGED, DIVERGED))
        return e, list(st), rc

    def solve_flows(self, s_values, **kw):
        """Solve instance i with flow s_values[i] (a flow scan as one batch)."""
        s_arr = np.ascontiguousarray(np.asarray(s_values, dtype=np.float64))
        assert s_arr.size == self.count
        o = RicMrcc.default_opts(**kw)
        e = np.zeros(self.count)
        st = (Stats * self.count)()
        rc = self.lib.ricmrcc_batch_solve_flows(self.b, _ptr(s_arr), ctypes.byref(o), _ptr(e),
                                                ctypes.cast(st, ctypes.c_void_p))
        self._check(rc, allow=(OK, NOT_CONVERGED, DIVERGED))
        return e, list(st), rc

    def step(self, s=0.5, n_steps=1, restart=False, **kw):
        o = RicMrcc.default_opts(s=s, **kw)
        e = np.zeros(self.count)
        dt = np.zeros(self.count)
        self._check(self.lib.ricmrcc_batch_step(self.b, ctypes.byref(o), n_steps, int(restart),
                                                _ptr(e), _ptr(dt)))
        return e, dt

    def tune(self, precision=MIXED, reps=3):
        t = Tuning()
        self._check(self.lib.ricmrcc_batch_tune(self.b, precision, reps, ctypes.byref(t)))
        return _tuning_dict(t)

    def info(self):
        i = BatchInfo()
        self._check(self.lib.ricmrcc_batch_info(self.b, ctypes.byref(i)))
        return {"waves": i.waves, "grouped_launches": i.grouped_launches,
                "tc_contractions": i.tc_contractions, "flops": i.flops, "tc_flops": i.tc_flops,
                "kernel_launches": i.kernel_launches}


class Ladder:
    """Density-fitted particle-particle ladder (ricmrcc_ladder_*):
    R[k,l,a,b] += sum_{e,f} (ae|bf) T[k,l,e,f] with (ae|bf) = sum_Q B[Q,a,e] B[Q,b,f]."""

    def __init__(self, n_hole, n_virt, n_aux, slab_rows=0):
        self.lib = load_library()
        self.dims = (n_hole, n_virt, n_aux)
        L = ctypes.c_void_p()
        rc = self.lib.ricmrcc_ladder_create(n_hole, n_virt, n_aux, int(slab_rows), ctypes.byref(L))
        if rc != OK:
            raise RicMrccError(rc, "ricmrcc_ladder_create failed")
        self.L = L

    def _check(self, rc, allow=(OK,)):
        if rc not in allow:
            raise RicMrccError(rc, self.lib.ricmrcc_ladder_last_error(self.L).decode())
        return rc

    def close(self):
        if getattr(self, "L", None):
            self.lib.ricmrcc_ladder_destroy(self.L)
            self.L = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        self._check(self.lib.ricmrcc_ladder_set_stream(self.L, stream_ptr))

    def set_factor(self, Bvv):
        """Bvv [n_aux, n_virt, n_virt]: a CUDA float64 tensor or a host array."""
        if hasattr(Bvv, "is_cuda") and Bvv.is_cuda:
            self._check(self.lib.ricmrcc_ladder_set_factor_dev(self.L, _ptr(Bvv)))
        else:
            b = _host(Bvv)
            self._check(self.lib.ricmrcc_ladder_set_factor(self.L, _ptr(b)))

    def apply_dev(self, T, R):
        """R += ladder(T) for CUDA float64 tensors [n_hole, n_hole, n_virt, n_virt] (enqueued)."""
        self._check(self.lib.ricmrcc_ladder_apply_dev(self.L, _ptr(T), _ptr(R)))

    def finish(self):
        """Wait for the enqueued work; sizes and phase times of the last application."""
        info = LadderInfo()
        self._check(self.lib.ricmrcc_ladder_finish(self.L, ctypes.byref(info)))
        return info.as_dict()

    def apply(self, T, R):
        """Host arrays: returns R + ladder(T) (R is not modified)."""
        t = _host(T)
        r = _host(R).copy()
        self._check(self.lib.ricmrcc_ladder_apply(self.L, _ptr(t), _ptr(r)))
        return r

    def info(self):
        info = LadderInfo()
        self._check(self.lib.ricmrcc_ladder_info(self.L, ctypes.byref(info)))
        return info.as_dict()


def gemm_f64_emulated(A, B, C, alpha=1.0, slices=0, stream=None):
    """C += alpha * A @ B.T on the tensor cores with FP64 accuracy (digit
    slicing, see ricmrcc_gemm_f64_emulated).  A [M,K], B [N,K], C [M,N]:
    CUDA float64 tensors with unit stride along the last axis."""
    M, K = A.shape
    N = B.shape[0]
    assert B.shape[1] == K and tuple(C.shape) == (M, N)
    for x in (A, B, C):
        assert x.dtype.is_floating_point and x.element_size() == 8 and x.is_cuda and x.stride(1) == 1
    rc = load_library().ricmrcc_gemm_f64_emulated(
        A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), C.data_ptr(), C.stride(0), M, N, K,
        float(alpha), int(slices), None if stream is None else stream.cuda_stream)
    if rc != OK:
        raise RicMrccError(rc, "ricmrcc_gemm_f64_emulated failed")


def set_wait_limit(seconds, stall_test=False):
    """Time bound of every wait inside the tensor-core kernels (default 4 s);
    stall_test makes each kernel wait once on a barrier nothing completes."""
    rc = load_library().ricmrcc_set_wait_limit(float(seconds), int(bool(stall_test)))
    if rc != OK:
        raise RicMrccError(rc, "ricmrcc_set_wait_limit failed")


def header_symbols(header=None):
    """Entry points declared in include/ricmrcc.h."""
    import re
    header = header or os.path.join(os.path.dirname(HERE), "include", "ricmrcc.h")
    return re.findall(r"RICMRCC_API [\w\s\*]*?\b(ricmrcc_\w+)\(", open(header).read())
