"""Python binding of librh15d_gpu.so (the C ABI in include/rh15d.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  Arrays are numpy (host) or torch CUDA tensors (device, passed by
pointer with ``on_device=True``).  There is no CPU fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import LIB, build

RH_OK, RH_EINVAL, RH_ENOMEM, RH_ECUDA, RH_ESTATE, RH_ETIMEOUT, RH_ENOTCONV = range(7)
COL_CONVERGED, COL_MAXITER, COL_NONFINITE, COL_SINGULAR, COL_NOTRUN = range(5)

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lib = None

EXPORTS = ("rh_create", "rh_destroy", "rh_last_error", "rh_setup_atom", "rh_nlambda", "rh_get_grid",
           "rh_load_columns", "rh_iterate", "rh_get_populations", "rh_get_lte", "rh_set_populations",
           "rh_emergent_spectrum", "rh_iterate_noalloc", "rh_surrogate_init", "rh_surrogate_state_size",
           "rh_surrogate_get_state", "rh_surrogate_set_state", "rh_surrogate_train", "rh_surrogate_loss_grad",
           "rh_surrogate_predict", "rh_solve", "rh_autotune", "rh_start_populations",
           "rh_emergent_stokes", "rh_surrogate_save", "rh_surrogate_load", "rh_surrogate_file_info",
           "rh_fma_peak", "rh_regrid", "rh_get_columns", "rh_column_smem_layout")

MAX_RERUN = 4
MAX_TUNE = 8


class AtomDesc(C.Structure):
    _fields_ = [("nlev", C.c_int32), ("E_J", _dp), ("g", _dp),
                ("nline", C.c_int32), ("line_l", _ip), ("line_u", _ip),
                ("line_f", _dp), ("line_a_top", _dp), ("line_a_bot", _dp),
                ("line_nlambda", _ip), ("line_qwing", _dp),
                ("ncont", C.c_int32), ("cont_l", _ip), ("cont_alpha0", _dp),
                ("cont_nlambda", _ip), ("cont_ratio", _dp),
                ("mass_amu", C.c_double), ("T_ref", C.c_double), ("nmu", C.c_int32),
                ("metal_floor", C.c_double), ("line_prd", _ip)]


class GridOpts(C.Structure):
    _fields_ = [("dlog_colden", C.c_double), ("dlnT", C.c_double), ("dvz", C.c_double),
                ("spacing_factor", C.c_double), ("z_top", C.c_double), ("use_z_top", C.c_int32)]


class IterOpts(C.Structure):
    _fields_ = [("maxiter", C.c_int32), ("tol", C.c_double), ("ng_order", C.c_int32),
                ("ng_delay", C.c_int32), ("ng_period", C.c_int32), ("start", C.c_int32),
                ("precision", C.c_int32), ("persistent", C.c_int32), ("block_warps", C.c_int32),
                ("crsw_init", C.c_double), ("only_unconverged", C.c_int32), ("prd_eps0", C.c_double),
                ("prd_hybrid", C.c_int32), ("formal", C.c_int32)]


class IterStats(C.Structure):
    _fields_ = [("n_converged", C.c_int64), ("n_maxiter", C.c_int64), ("n_failed", C.c_int64),
                ("n_processed", C.c_int64), ("iterations_total", C.c_int64), ("seconds", C.c_double),
                ("pts", C.c_double), ("max_dn_final", C.c_double), ("guess_fallback_depths", C.c_int64),
                ("guess_seconds", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("pass1", IterOpts), ("nrerun", C.c_int32), ("rerun_maxiter", C.c_int32),
                ("rerun_crsw", C.c_double * MAX_RERUN), ("use_graph", C.c_int32), ("autotune", C.c_int32),
                ("rerun_ng", C.c_int32 * MAX_RERUN), ("fused_rerun", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("n_converged", C.c_int64), ("n_maxiter", C.c_int64), ("n_failed", C.c_int64),
                ("iterations_total", C.c_int64), ("pass_columns", C.c_int64 * (1 + MAX_RERUN)),
                ("pass_iterations", C.c_int64 * (1 + MAX_RERUN)), ("seconds", C.c_double),
                ("pass_seconds", C.c_double * (1 + MAX_RERUN)), ("pts", C.c_double),
                ("guess_fallback_depths", C.c_int64), ("kernel_launches", C.c_int32),
                ("graph_replayed", C.c_int32), ("block_warps", C.c_int32), ("ctas_per_sm", C.c_int32)]


class TuneResult(C.Structure):
    _fields_ = [("best_block_warps", C.c_int32), ("best_ctas_per_sm", C.c_int32), ("ncand", C.c_int32),
                ("cand_block_warps", C.c_int32 * MAX_TUNE), ("cand_ctas_per_sm", C.c_int32 * MAX_TUNE),
                ("cand_ms", C.c_double * MAX_TUNE), ("sample_columns", C.c_int64)]


class TrainOpts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("seed", C.c_uint64), ("standardise", C.c_int32)]


class TrainStats(C.Structure):
    _fields_ = [("loss_first_epoch", C.c_double), ("loss_last_epoch", C.c_double), ("steps", C.c_int64),
                ("samples", C.c_int64), ("seconds", C.c_double)]


def lib(path: str | None = None):
    """Load the CUDA library (raises if it is missing or fails to load)."""
    global _lib
    if _lib is None:
        p = path or LIB
        if not os.path.exists(p):
            raise RuntimeError("librh15d_gpu.so is not built (run paper_1411_1079_gb300._build.build())")
        L = C.CDLL(p)
        vp = C.c_void_p
        L.rh_create.argtypes = [C.POINTER(vp), C.c_int, vp]
        L.rh_destroy.argtypes = [vp]
        L.rh_destroy.restype = None
        L.rh_last_error.argtypes = [vp]
        L.rh_last_error.restype = C.c_char_p
        L.rh_setup_atom.argtypes = [vp, C.POINTER(AtomDesc)]
        L.rh_nlambda.argtypes = [vp]
        L.rh_nlambda.restype = C.c_int64
        L.rh_get_grid.argtypes = [vp, _dp]
        L.rh_load_columns.argtypes = [vp, C.c_int64, C.c_int32, vp, vp, vp, vp, vp, C.c_int32]
        L.rh_iterate.argtypes = [vp, C.POINTER(IterOpts), C.POINTER(IterStats)]
        L.rh_get_populations.argtypes = [vp, vp, _ip, C.POINTER(C.c_uint8), _dp, C.c_int32]
        L.rh_get_lte.argtypes = [vp, _dp, _dp]
        L.rh_set_populations.argtypes = [vp, _dp]
        L.rh_emergent_spectrum.argtypes = [vp, C.c_double, C.c_int64, _dp, vp, C.c_int32, C.c_int32]
        L.rh_iterate_noalloc.argtypes = [vp, C.POINTER(IterOpts), vp, vp, vp, vp, C.POINTER(IterStats)]
        L.rh_solve.argtypes = [vp, C.POINTER(SolveOpts), C.POINTER(SolveStats)]
        L.rh_autotune.argtypes = [vp, C.c_int32, C.POINTER(TuneResult)]
        L.rh_start_populations.argtypes = [vp, C.c_int32]
        L.rh_emergent_stokes.argtypes = [vp, C.c_int32, C.c_double, vp, vp, vp, C.c_int64, _dp, vp, C.c_int32,
                                         C.c_int32]
        _fp = C.POINTER(C.c_float)
        L.rh_surrogate_init.argtypes = [vp, C.c_int32, C.c_int32, C.c_uint64]
        L.rh_surrogate_state_size.argtypes = [vp]
        L.rh_surrogate_state_size.restype = C.c_int64
        L.rh_surrogate_get_state.argtypes = [vp, _fp]
        L.rh_surrogate_set_state.argtypes = [vp, _fp]
        L.rh_surrogate_train.argtypes = [vp, C.POINTER(TrainOpts), C.POINTER(TrainStats)]
        L.rh_surrogate_loss_grad.argtypes = [vp, C.c_int64, _ip, C.POINTER(C.c_double), _fp]
        L.rh_surrogate_predict.argtypes = [vp, _fp]
        L.rh_surrogate_save.argtypes = [vp, C.c_char_p]
        L.rh_surrogate_load.argtypes = [vp, C.c_char_p]
        L.rh_surrogate_file_info.argtypes = [C.c_char_p, _ip, C.POINTER(C.c_int64), C.c_char_p, C.c_size_t]
        L.rh_regrid.argtypes = [vp, C.c_int32, C.POINTER(GridOpts)]
        L.rh_get_columns.argtypes = [vp, _dp, _dp, _dp, _dp]
        L.rh_column_smem_layout.argtypes = [C.c_int32] * 8 + [C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        L.rh_fma_peak.argtypes = [C.c_int32, C.c_int32, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _ptr(x):
    """Pointer of a numpy array or a torch tensor (device)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def column_smem_layout(precision, nlev, ndep, ntr, ncont, nline, macc, ring_warps=0):
    """rh_column_smem_layout (host only): ([16] region offsets in carve
    order, the carve's end last; allocated bytes)."""
    off = (C.c_size_t * 16)()
    b = C.c_size_t()
    rc = lib().rh_column_smem_layout(precision, nlev, ndep, ntr, ncont, nline, macc, ring_warps, off, C.byref(b))
    if rc:
        raise RhError(rc, "rh_column_smem_layout: invalid sizes")
    return list(off), b.value


def fma_peak(device: int = 0, precision: int = 1, seconds: float = 0.5) -> dict:
    """rh_fma_peak: measured FMA rate of the device (FP32: precision 1, FP64:
    0), FLOP/s, and the timed launch's duration."""
    f = C.c_double()
    t = C.c_double()
    rc = lib().rh_fma_peak(device, precision, seconds, C.byref(f), C.byref(t))
    if rc:
        raise RhError(rc, "rh_fma_peak failed")
    return {"flop_s": f.value, "seconds": t.value}


class RhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("rh error %d: %s" % (code, msg))
        self.code = code


def surrogate_file_info(path) -> dict:
    """rh_surrogate_file_info: check a network checkpoint file (no context,
    no GPU); its sizes and state length, or RhError(RH_EINVAL, reason)."""
    sizes = np.zeros(4, np.int32)
    npar = C.c_int64()
    msg = C.create_string_buffer(256)
    rc = lib().rh_surrogate_file_info(os.fsencode(path), _i(sizes), C.byref(npar), msg, 256)
    if rc:
        raise RhError(rc, msg.value.decode())
    return {"nin": int(sizes[0]), "hidden": int(sizes[1]), "nhidden": int(sizes[2]), "nout": int(sizes[3]),
            "nparam": int(npar.value)}


class Context:
    """One rh_ctx: an atom, a set of columns and their MALI state on one GPU."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = lib()
        p = C.c_void_p()
        rc = self._lib.rh_create(C.byref(p), device, C.c_void_p(stream) if stream else None)
        self._p = p
        if rc:
            msg = self._lib.rh_last_error(p).decode() if p else "rh_create failed"
            raise RhError(rc, msg)
        self._keep = None
        self.device = device
        self.ncol = 0

    def close(self):
        if getattr(self, "_p", None):
            self._lib.rh_destroy(self._p)
            self._p = None

    __del__ = close

    def _check(self, rc, allow=()):
        if rc and rc not in allow:
            raise RhError(rc, self._lib.rh_last_error(self._p).decode())
        return rc

    def setup_atom(self, atom: dict):
        a = {k: (np.ascontiguousarray(v) if isinstance(v, np.ndarray) else v) for k, v in atom.items()}
        self._keep = a
        d = AtomDesc(nlev=a["nlev"], E_J=_d(a["E_J"]), g=_d(a["g"]), nline=len(a["line_l"]),
                     line_l=_i(a["line_l"]), line_u=_i(a["line_u"]), line_f=_d(a["line_f"]),
                     line_a_top=_d(a["line_a_top"]), line_a_bot=_d(a["line_a_bot"]),
                     line_nlambda=_i(a["line_nlambda"]), line_qwing=_d(a["line_qwing"]),
                     ncont=len(a["cont_l"]), cont_l=_i(a["cont_l"]), cont_alpha0=_d(a["cont_alpha0"]),
                     cont_nlambda=_i(a["cont_nlambda"]), cont_ratio=_d(a["cont_ratio"]),
                     mass_amu=a["mass_amu"], T_ref=a["T_ref"], nmu=a["nmu"],
                     metal_floor=a["metal_floor"])
        if "line_prd" in a:
            a["line_prd"] = np.ascontiguousarray(a["line_prd"], dtype=np.int32)
            d.line_prd = _i(a["line_prd"])
        self._check(self._lib.rh_setup_atom(self._p, C.byref(d)))
        self.nlev = a["nlev"]
        self.nmu = a["nmu"]
        self.has_prd = bool("line_prd" in a and np.any(a["line_prd"]))

    @property
    def nlambda(self) -> int:
        return int(self._lib.rh_nlambda(self._p))

    def grid(self):
        nu = np.zeros(self.nlambda)
        self._check(self._lib.rh_get_grid(self._p, _d(nu)))
        return nu

    def load_columns(self, cols: dict, ne=None, on_device: bool = False):
        """``cols``: z, T, nH, vz arrays [ncol][ndep] (numpy; or torch tensors,
        CUDA with on_device=True, or CPU/pinned with on_device=False)."""
        if on_device or hasattr(cols["T"], "data_ptr"):
            arrs = [cols["z"], cols["T"], ne, cols["nH"], cols["vz"]]
            ncol, ndep = cols["T"].shape
        else:
            arrs = [None if x is None else np.ascontiguousarray(x, dtype=np.float64)
                    for x in (cols["z"], cols["T"], ne, cols["nH"], cols["vz"])]
            ncol, ndep = arrs[1].shape
        self._cols_keep = arrs
        self._check(self._lib.rh_load_columns(self._p, ncol, ndep, *[_ptr(x) for x in arrs], int(on_device)))
        self.ncol, self.ndep = int(ncol), int(ndep)

    def iterate(self, maxiter=500, tol=1e-3, ng_order=2, ng_delay=5, ng_period=3, start=0,
                precision=1, persistent=1, block_warps=0, crsw_init=1.0, only_unconverged=0,
                prd_eps0=0.0, prd_hybrid=0, formal=0) -> dict:
        o = IterOpts(maxiter=maxiter, tol=tol, ng_order=ng_order, ng_delay=ng_delay,
                     ng_period=ng_period, start=start, precision=precision, persistent=persistent,
                     block_warps=block_warps, crsw_init=crsw_init, only_unconverged=only_unconverged,
                     prd_eps0=prd_eps0, prd_hybrid=prd_hybrid, formal=formal)
        s = IterStats()
        rc = self._check(self._lib.rh_iterate(self._p, C.byref(o), C.byref(s)), allow=(RH_ENOTCONV,))
        out = {f: getattr(s, f) for f, _ in IterStats._fields_}
        out["rc"] = rc
        return out

    # Sect. 2.3: run all columns with an aggressive choice of options, then
    # re-run the columns that did not converge with other options.
    RERUN_CRSW = (1e3, 1e5, 1e7)
    # with PRD lines the rungs keep Ng (its Jacobi step on rho) first -- the
    # damped rho update without it diverges on strongly moving columns -- and
    # end with rungs without Ng, which converge columns where Ng's
    # extrapolation of rho does not
    RERUN_PRD = ((1e3, 1), (1e5, 1), (1e3, 0), (1e5, 0))

    def solve(self, precision=1, maxiter=500, tol=1e-3, persistent=1, block_warps=0, rescue=True, start=0,
              ng_order=2, ng_delay=5, ng_period=3, use_graph=1, autotune=1, fused_rerun=1,
              prd_eps0=0.0, rungs=None, prd_hybrid=0, rerun_maxiter=None, formal=0, rescue_formal=None) -> dict:
        """rh_solve: every column from LTE (start=0), the learned guess
        (start=1), the current populations (start=2), zero radiation (3) or
        escape probabilities (4) with Ng acceleration, then the columns that
        did not converge again from LTE -- first with the same options when
        pass 1 started elsewhere, then with collisional-radiative switching
        (x1e3, x1e5, then x1e7) and without Ng (the paper's two-stage
        strategy): by the column kernel itself as
        soon as a column fails (fused_rerun=1) or as separate passes over a
        device-selected list; the sequence is replayed as a CUDA graph.
        With PRD lines the default ladder is LTE with the same options (when
        pass 1 started elsewhere), switching x1e3 and x1e5 with Ng, then
        x1e3 and x1e5 without Ng, at most MAX_RERUN rungs, and re-runs take
        up to 3 x maxiter iterations.  rungs: the re-run ladder as (collisional-radiative
        factor, Ng on) pairs, at most MAX_RERUN of them, in place of the
        default; rerun_maxiter: the re-runs' iteration limit.  rescue_formal
        (default: 1 with PRD lines, none otherwise): after the ladder, one
        more pass (rh_iterate, only_unconverged) over the columns still not
        converged, from LTE with Ng and that formal solver -- the Bezier
        solver converges most PRD columns on which every linear-solver rung
        diverges; its counts are merged into the result under "rescue"."""
        o = SolveOpts()
        o.pass1 = IterOpts(maxiter=maxiter, tol=tol, ng_order=ng_order, ng_delay=ng_delay, ng_period=ng_period,
                           start=start, precision=precision, persistent=persistent, block_warps=block_warps,
                           crsw_init=1.0, only_unconverged=0, prd_eps0=prd_eps0, prd_hybrid=prd_hybrid,
                           formal=formal)
        # the ladder: from a start other than LTE, first LTE with the same
        # options; then stronger and stronger switching without Ng
        prd = getattr(self, "has_prd", False)
        if rungs is None:
            if prd:
                rungs = (([(1.0, 1)] if start != 0 else []) + list(self.RERUN_PRD))[:MAX_RERUN]
            else:
                rungs = ([(1.0, 1)] if start != 0 else []) + [(f, 0) for f in self.RERUN_CRSW]
        if rerun_maxiter is None:
            rerun_maxiter = 3 * maxiter if prd else maxiter
        rungs = [(float(f), int(bool(ng))) for f, ng in rungs]
        if len(rungs) > len(o.rerun_crsw) or any(not f >= 1.0 for f, _ in rungs):
            raise ValueError("rungs: at most %d pairs with factors >= 1" % len(o.rerun_crsw))
        o.nrerun = len(rungs) if rescue else 0
        o.rerun_maxiter = int(rerun_maxiter)
        for i, (f, ng) in enumerate(rungs[:o.nrerun]):
            o.rerun_crsw[i] = f
            o.rerun_ng[i] = ng
        o.use_graph = int(use_graph)
        o.autotune = int(autotune)
        o.fused_rerun = int(fused_rerun)
        st = SolveStats()
        r = self._lib.rh_solve(self._p, C.byref(o), C.byref(st))
        if r not in (0, 6):
            self._check(r)
        npass = 1 + o.nrerun
        out = {"n_converged": st.n_converged, "n_maxiter": st.n_maxiter, "n_failed": st.n_failed,
                "seconds": st.seconds, "pts": st.pts, "iterations_total": st.iterations_total,
                "pass_columns": list(st.pass_columns)[:npass], "pass_iterations": list(st.pass_iterations)[:npass],
                "pass_seconds": list(st.pass_seconds)[:npass],
                "rerun_columns": int(sum(list(st.pass_columns)[1:npass])),
                "guess_fallback_depths": st.guess_fallback_depths, "launches": st.kernel_launches,
                "graph_replayed": bool(st.graph_replayed), "block_warps": st.block_warps,
                "ctas_per_sm": st.ctas_per_sm}
        if rescue_formal is None and prd and formal == 0:
            rescue_formal = 1
        if rescue and rescue_formal is not None and out["n_converged"] < self.ncol:
            r2 = self.iterate(maxiter=int(rerun_maxiter), tol=tol, ng_order=ng_order, ng_delay=ng_delay,
                              ng_period=ng_period, start=0, precision=precision, persistent=persistent,
                              block_warps=block_warps, only_unconverged=1, prd_eps0=prd_eps0,
                              prd_hybrid=prd_hybrid, formal=int(rescue_formal))
            out["rescue"] = {"formal": int(rescue_formal), "columns": r2["n_processed"],
                             "iterations": r2["iterations_total"], "seconds": r2["seconds"],
                             "converged_before": out["n_converged"], "converged_after": r2["n_converged"]}
            for k in ("n_converged", "n_maxiter", "n_failed"):
                out[k] = r2[k]
            out["iterations_total"] += r2["iterations_total"]
            out["seconds"] += r2["seconds"]
            out["pts"] += r2["pts"]
        return out

    def emergent_stokes(self, line, g_eff, B_T, theta, chi, lam_m, precision=0, out=None):
        """rh_emergent_stokes: (I, Q, U, V) at mu = 1 of line `line` with Zeeman
        splitting; B_T, theta, chi [ncol][ndep] (numpy, or CUDA tensors with
        out a CUDA tensor [ncol][nlam][4]); returns [ncol][nlam][4]."""
        lam_m = np.ascontiguousarray(lam_m, dtype=np.float64)
        if out is not None:
            self._check(self._lib.rh_emergent_stokes(self._p, line, g_eff, _ptr(B_T), _ptr(theta), _ptr(chi),
                                                     lam_m.size, _d(lam_m), _ptr(out), precision, 1))
            return out
        B_T, theta, chi = (np.ascontiguousarray(x, dtype=np.float64) for x in (B_T, theta, chi))
        res = np.zeros((self.ncol, lam_m.size, 4))
        self._check(self._lib.rh_emergent_stokes(self._p, line, g_eff, _ptr(B_T), _ptr(theta), _ptr(chi),
                                                 lam_m.size, _d(lam_m), _ptr(res), precision, 0))
        return res

    START_LTE, START_LEARNED, START_CURRENT, START_ZERO_RADIATION, START_ESCAPE = 0, 1, 2, 3, 4

    def regrid(self, ndep_out, dlog_colden=0.1, dlnT=0.02, dvz=1e3, spacing_factor=4.0, z_top=None):
        """rh_regrid: depth-grid optimisation of every loaded column onto
        ndep_out points; z_top (m) removes the layers above it."""
        o = GridOpts(dlog_colden=dlog_colden, dlnT=dlnT, dvz=dvz, spacing_factor=spacing_factor,
                     z_top=0.0 if z_top is None else z_top, use_z_top=0 if z_top is None else 1)
        self._check(self._lib.rh_regrid(self._p, ndep_out, C.byref(o)))
        self.ndep = int(ndep_out)

    def columns(self):
        """The loaded atmosphere: dict of z, T, nH, vz [ncol][ndep]."""
        out = {k: np.zeros((self.ncol, self.ndep)) for k in ("z", "T", "nH", "vz")}
        self._check(self._lib.rh_get_columns(self._p, _d(out["z"]), _d(out["T"]), _d(out["nH"]), _d(out["vz"])))
        return out

    def start_populations(self, kind):
        """rh_start_populations: write the LTE (0), learned (1), zero-radiation
        (3) or escape-probability (4) start into the current populations."""
        self._check(self._lib.rh_start_populations(self._p, kind))

    def autotune(self, precision=1) -> dict:
        """rh_autotune: time the column kernel's launch shapes on a sample of
        the loaded columns and keep the fastest for this precision."""
        t = TuneResult()
        self._check(self._lib.rh_autotune(self._p, precision, C.byref(t)))
        n = t.ncand
        return {"block_warps": t.best_block_warps, "ctas_per_sm": t.best_ctas_per_sm,
                "sample_columns": t.sample_columns,
                "candidates": [(t.cand_block_warps[i], t.cand_ctas_per_sm[i], t.cand_ms[i]) for i in range(n)]}

    # ---- learned initial guess
    def surrogate_init(self, hidden=512, nhidden=3, seed=0):
        self._check(self._lib.rh_surrogate_init(self._p, hidden, nhidden, seed))

    def surrogate_state(self):
        n = int(self._lib.rh_surrogate_state_size(self._p))
        out = np.zeros(n, np.float32)
        self._check(self._lib.rh_surrogate_get_state(self._p, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def surrogate_set_state(self, state):
        state = np.ascontiguousarray(state, dtype=np.float32)
        self._check(self._lib.rh_surrogate_set_state(self._p, state.ctypes.data_as(C.POINTER(C.c_float))))

    def surrogate_train(self, epochs=20, batch=512, lr=2e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=0,
                        standardise=1) -> dict:
        o = TrainOpts(epochs=epochs, batch=batch, lr=lr, beta1=beta1, beta2=beta2, eps=eps, seed=seed,
                      standardise=standardise)
        s = TrainStats()
        self._check(self._lib.rh_surrogate_train(self._p, C.byref(o), C.byref(s)))
        return {f: getattr(s, f) for f, _ in TrainStats._fields_}

    def surrogate_loss_grad(self, cols):
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        loss = C.c_double()
        grad = np.zeros(int(self._lib.rh_surrogate_state_size(self._p)), np.float32)
        self._check(self._lib.rh_surrogate_loss_grad(self._p, cols.size, _i(cols), C.byref(loss),
                                                     grad.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, grad

    def surrogate_save(self, path):
        self._check(self._lib.rh_surrogate_save(self._p, os.fsencode(path)))

    def surrogate_load(self, path):
        self._check(self._lib.rh_surrogate_load(self._p, os.fsencode(path)))

    def surrogate_predict(self):
        out = np.zeros((self.ncol, self.nlev, self.ndep), np.float32)
        self._check(self._lib.rh_surrogate_predict(self._p, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def iterate_noalloc(self, n_out, iters_out, status_out, dmax_out, maxiter=500, tol=1e-3, ng_order=2,
                        ng_delay=5, ng_period=3, start=0, precision=1, persistent=1, block_warps=0,
                        crsw_init=1.0, formal=0) -> dict:
        """rh_iterate_noalloc: results into caller-owned CUDA tensors (float64
        [ncol][nlev][ndep], int32 [ncol], uint8 [ncol], float64 [ncol]) on the
        context's device, contiguous; the library allocates nothing during the
        call.  Anything else is refused here, before the call."""
        if not self.ncol:          # nothing loaded: the library reports RH_ESTATE
            want = ()
        else:
            want = ((n_out, "float64", self.ncol * self.nlev * self.ndep, "n_out"),
                    (iters_out, "int32", self.ncol, "iters_out"), (status_out, "uint8", self.ncol, "status_out"),
                    (dmax_out, "float64", self.ncol, "dmax_out"))
        for t, dt, numel, name in want:
            if not (hasattr(t, "is_cuda") and t.is_cuda):
                raise ValueError("%s must be a CUDA tensor" % name)
            if t.device.index != self.device:
                raise ValueError("%s is on cuda:%s, the context on cuda:%d" % (name, t.device.index, self.device))
            if str(t.dtype) != "torch." + dt:
                raise ValueError("%s must be %s, got %s" % (name, dt, t.dtype))
            if not t.is_contiguous():
                raise ValueError("%s must be contiguous" % name)
            if t.numel() < numel:
                raise ValueError("%s holds %d elements, needs %d" % (name, t.numel(), numel))
        o = IterOpts(maxiter=maxiter, tol=tol, ng_order=ng_order, ng_delay=ng_delay,
                     ng_period=ng_period, start=start, precision=precision, persistent=persistent,
                     block_warps=block_warps, crsw_init=crsw_init, only_unconverged=0, formal=formal)
        s = IterStats()
        rc = self._check(self._lib.rh_iterate_noalloc(self._p, C.byref(o), _ptr(n_out), _ptr(iters_out),
                                                      _ptr(status_out), _ptr(dmax_out), C.byref(s)),
                         allow=(RH_ENOTCONV,))
        out = {f: getattr(s, f) for f, _ in IterStats._fields_}
        out["rc"] = rc
        return out

    def populations(self, out=None):
        """(n [ncol][nlev][ndep], iters, status, dmax).  ``out`` may be a torch
        tensor (CUDA: device copy; CPU, e.g. pinned: host copy)."""
        it = np.zeros(self.ncol, np.int32)
        st = np.zeros(self.ncol, np.uint8)
        dm = np.zeros(self.ncol)
        if out is not None:
            dev = int(bool(getattr(out, "is_cuda", False)))
            self._check(self._lib.rh_get_populations(self._p, _ptr(out), _i(it),
                                                     st.ctypes.data_as(C.POINTER(C.c_uint8)), _d(dm), dev))
            return out, it, st, dm
        n = np.zeros((self.ncol, self.nlev, self.ndep))
        self._check(self._lib.rh_get_populations(self._p, _ptr(n), _i(it),
                                                 st.ctypes.data_as(C.POINTER(C.c_uint8)), _d(dm), 0))
        return n, it, st, dm

    def lte(self):
        ns = np.zeros((self.ncol, self.nlev, self.ndep))
        ne = np.zeros((self.ncol, self.ndep))
        self._check(self._lib.rh_get_lte(self._p, _d(ns), _d(ne)))
        return ns, ne

    def set_populations(self, n):
        n = np.ascontiguousarray(n, dtype=np.float64)
        self._check(self._lib.rh_set_populations(self._p, _d(n)))

    def emergent_spectrum(self, mu, lam_m, precision=0, out=None):
        lam_m = np.ascontiguousarray(lam_m, dtype=np.float64)
        if out is not None:
            self._check(self._lib.rh_emergent_spectrum(self._p, float(mu), lam_m.size, _d(lam_m), _ptr(out),
                                                       precision, 1))
            return out
        I = np.zeros((self.ncol, lam_m.size))
        self._check(self._lib.rh_emergent_spectrum(self._p, float(mu), lam_m.size, _d(lam_m), _ptr(I),
                                                   precision, 0))
        return I


__all__ = ["Context", "RhError", "build", "lib", "EXPORTS"]
