"""ctypes binding of the FP64 CPU oracle (``rh_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this
module.  It shares no code with the CUDA library and never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rh_oracle.c")
_LIB = os.path.join(_HERE, "librh15d_oracle.so")

ST_CONV, ST_MAXITER, ST_NONFINITE, ST_SINGULAR, ST_NOTRUN = range(5)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only: it also builds on Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.rho_voigt.restype = C.c_double
        L.rho_voigt.argtypes = [C.c_double, C.c_double]
        L.rho_expE1.restype = C.c_double
        L.rho_expE1.argtypes = [C.c_double]
        L.rho_planck.restype = C.c_double
        L.rho_planck.argtypes = [C.c_double, C.c_double]
        L.rho_cff.restype = C.c_double
        L.rho_cff.argtypes = []
        L.rho_sc_sweep.restype = None
        L.rho_sc_sweep.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_int, _dp, _dp]
        L.rho_sc_sweep_bezier.restype = None
        L.rho_sc_sweep_bezier.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_int, _dp, _dp]
        L.rho_bez_weights.restype = None
        L.rho_bez_weights.argtypes = [C.c_double, _dp]
        L.rho_ng2.restype = C.c_int
        L.rho_ng2.argtypes = [C.c_int64, _dp, _dp, _dp, _dp, _dp, C.c_int32]
        L.rho_gauss_legendre01.argtypes = [C.c_int, _dp, _dp]
        L.rho_two_level_jbar.argtypes = [C.c_int, _dp, C.c_int, C.c_double, C.c_int, C.c_double,
                                         _dp, _dp, _dp]
        L.rho_two_level_solve.argtypes = [C.c_int, _dp, C.c_int, C.c_double, C.c_int, C.c_double,
                                          C.c_double, C.c_int, C.c_double, C.c_int, C.c_int,
                                          C.c_int, _dp, _ip]
        L.rho_create.argtypes = [C.POINTER(C.c_void_p)]
        L.rho_destroy.argtypes = [C.c_void_p]
        L.rho_destroy.restype = None
        L.rho_last_error.argtypes = [C.c_void_p]
        L.rho_last_error.restype = C.c_char_p
        L.rho_setup_atom.argtypes = [C.c_void_p, C.c_void_p]
        L.rho_nlambda.argtypes = [C.c_void_p]
        L.rho_nlambda.restype = C.c_int64
        L.rho_get_grid.argtypes = [C.c_void_p, _dp, _ip, _ip, _dp]
        L.rho_atom_info.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp]
        L.rho_load_columns.argtypes = [C.c_void_p, C.c_int64, C.c_int32, _dp, _dp, _dp, _dp, _dp]
        L.rho_get_lte.argtypes = [C.c_void_p, _dp, _dp]
        L.rho_get_populations.argtypes = [C.c_void_p, _dp, _ip, C.POINTER(C.c_uint8), _dp]
        L.rho_set_populations.argtypes = [C.c_void_p, _dp]
        L.rho_iterate.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]
        L.rho_rate_matrix.argtypes = [C.c_void_p, C.c_int64, _dp, C.c_int32, _dp]
        L.rho_collision_rates.argtypes = [C.c_void_p, C.c_int64, _dp]
        L.rho_escape_probabilities.argtypes = [C.c_void_p, C.c_int64, _dp, _dp]
        L.rho_column_background.argtypes = [C.c_void_p, C.c_int64, _dp]
        L.rho_prd_update_ratio.argtypes = [C.c_void_p, C.c_int64, _dp, C.c_int32, _dp]
        L.rho_prd_kernel.argtypes = [C.c_void_p, C.c_int64, C.c_int32, _ip, _ip, _dp, _dp, _dp]
        L.rho_start_populations.argtypes = [C.c_void_p, C.c_int32]
        L.rho_emergent_spectrum.argtypes = [C.c_void_p, C.c_double, C.c_int64, _dp, _dp, C.c_int32]
        L.rho_electron_density.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.rho_electron_density.restype = C.c_double
        L.rho_hminus_sigma.restype = C.c_double
        L.rho_hminus_sigma.argtypes = [C.c_double]
        L.rho_r2a.restype = C.c_double
        L.rho_r2a.argtypes = [C.c_double, C.c_double, C.c_double]
        L.rho_faddeeva.restype = None
        L.rho_faddeeva.argtypes = [C.c_double, C.c_double, _dp, _dp]
        L.rho_stokes_sweep.restype = None
        L.rho_stokes_sweep.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp]
        L.rho_emergent_stokes.argtypes = [C.c_void_p, C.c_int32, C.c_double, _dp, _dp, _dp, C.c_int64, _dp, _dp]
        L.rho_regrid.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
        L.rho_get_columns.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.rho_prd_switch_eps.restype = C.c_double
        L.rho_prd_switch_eps.argtypes = [C.c_double, C.c_int32]
        L.rho_crsw_factor.restype = C.c_double
        L.rho_crsw_factor.argtypes = [C.c_double, C.c_int32]
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


class AtomDesc(C.Structure):
    _fields_ = [("nlev", C.c_int32), ("E_J", _dp), ("g", _dp),
                ("nline", C.c_int32), ("line_l", _ip), ("line_u", _ip),
                ("line_f", _dp), ("line_a_top", _dp), ("line_a_bot", _dp),
                ("line_nlambda", _ip), ("line_qwing", _dp),
                ("ncont", C.c_int32), ("cont_l", _ip), ("cont_alpha0", _dp),
                ("cont_nlambda", _ip), ("cont_ratio", _dp),
                ("mass_amu", C.c_double), ("T_ref", C.c_double), ("nmu", C.c_int32),
                ("metal_floor", C.c_double), ("line_prd", _ip)]


class IterOpts(C.Structure):
    _fields_ = [("maxiter", C.c_int32), ("tol", C.c_double), ("ng_order", C.c_int32),
                ("ng_delay", C.c_int32), ("ng_period", C.c_int32), ("start", C.c_int32),
                ("crsw_init", C.c_double), ("prd_eps0", C.c_double), ("prd_hybrid", C.c_int32),
                ("formal", C.c_int32)]


class GridOpts(C.Structure):
    _fields_ = [("dlog_colden", C.c_double), ("dlnT", C.c_double), ("dvz", C.c_double),
                ("spacing_factor", C.c_double), ("z_top", C.c_double), ("use_z_top", C.c_int32)]


class IterStats(C.Structure):
    _fields_ = [("n_converged", C.c_int64), ("n_maxiter", C.c_int64), ("n_failed", C.c_int64),
                ("iterations_total", C.c_int64), ("seconds", C.c_double), ("pts", C.c_double),
                ("max_dn_final", C.c_double)]


def voigt(a, v):
    L = lib()
    return float(L.rho_voigt(float(a), float(v)))


def r2a(a, xp, x):
    """Angle-averaged redistribution function R_II-A(x', x), Doppler units."""
    return float(lib().rho_r2a(float(a), float(xp), float(x)))


def faddeeva(a, v):
    """(H, L) = (Re, Im) of w(v + i a)."""
    h = C.c_double()
    l_ = C.c_double()
    lib().rho_faddeeva(float(a), float(v), C.byref(h), C.byref(l_))
    return h.value, l_.value


def stokes_sweep(dtau, Kp, S, Ib):
    """DELO-linear polarised sweep from k = N-1 to k = 0; returns the Stokes
    vector at k = 0.  dtau [N-1], Kp [N][6] = (eQ, eU, eV, rQ, rU, rV)/eI,
    S [N][4] emission / eI, Ib [4]."""
    dtau = np.ascontiguousarray(dtau, dtype=np.float64)
    Kp = np.ascontiguousarray(Kp, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    Ib = np.ascontiguousarray(Ib, dtype=np.float64)
    out = np.zeros(4)
    lib().rho_stokes_sweep(S.shape[0], _d(dtau), _d(Kp), _d(S), _d(Ib), _d(out))
    return out


def prd_switch_eps(eps0, it):
    """PRD switching factor eps of iteration it (Sect. 2.3, Eq. 1)."""
    return lib().rho_prd_switch_eps(float(eps0), int(it))


def crsw_factor(f0, it):
    """Collisional-radiative switching factor of iteration it (Sect. 2.3)."""
    return lib().rho_crsw_factor(float(f0), int(it))


def expE1(y):
    return float(lib().rho_expE1(float(y)))


def planck(nu, T):
    return float(lib().rho_planck(float(nu), float(T)))


def cff():
    return float(lib().rho_cff())


def gauss_legendre01(n):
    x = np.zeros(n)
    w = np.zeros(n)
    if lib().rho_gauss_legendre01(n, _d(x), _d(w)):
        raise ValueError("n out of range")
    return x, w


def sc_sweep(dtau, S, I0, direction, bezier=False):
    """Linear (or quadratic Bezier) short-characteristics sweep; returns
    (I, dI/dS_local)."""
    dtau = np.ascontiguousarray(dtau, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    N = S.size
    I = np.zeros(N)
    lam = np.zeros(N)
    f = lib().rho_sc_sweep_bezier if bezier else lib().rho_sc_sweep
    f(N, _d(dtau), _d(S), float(I0), int(direction), _d(I), _d(lam))
    return I, lam


def bez_weights(d):
    """Quadratic Bezier step weights (e^-d, w_u, w_o, w_c, 1 - w_o - w_c)."""
    out = np.zeros(5)
    lib().rho_bez_weights(float(d), _d(out))
    return out


def ng2(x0, x1, x2, x3, relative=True):
    x = [np.ascontiguousarray(v, dtype=np.float64) for v in (x0, x1, x2, x3)]
    out = np.zeros_like(x[0])
    if lib().rho_ng2(x[0].size, _d(x[0]), _d(x[1]), _d(x[2]), _d(x[3]), _d(out), int(relative)):
        raise ArithmeticError("singular Ng system")
    return out


def two_level_jbar(tau0, nfreq, xmax, nmu, B, S):
    tau0 = np.ascontiguousarray(tau0, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    J = np.zeros_like(S)
    Ls = np.zeros_like(S)
    lib().rho_two_level_jbar(tau0.size, _d(tau0), nfreq, xmax, nmu, B, _d(S), _d(J), _d(Ls))
    return J, Ls


def two_level_solve(tau0, nfreq, xmax, nmu, eps, B, maxiter=2000, tol=1e-10, ng_order=2,
                    ng_delay=5, ng_period=3):
    tau0 = np.ascontiguousarray(tau0, dtype=np.float64)
    S = np.zeros_like(tau0)
    it = np.zeros(1, np.int32)
    lib().rho_two_level_solve(tau0.size, _d(tau0), nfreq, xmax, nmu, eps, B, maxiter, tol,
                              ng_order, ng_delay, ng_period, _d(S), _i(it))
    return S, int(it[0])


class Oracle:
    """The oracle behind the same calls as the CUDA library (``rho_*``)."""

    def __init__(self):
        self._lib = lib()
        p = C.c_void_p()
        if self._lib.rho_create(C.byref(p)):
            raise MemoryError("rho_create failed")
        self._p = p
        self._keep = []

    def __del__(self):
        if getattr(self, "_p", None):
            self._lib.rho_destroy(self._p)
            self._p = None

    def _check(self, rc):
        if rc:
            raise RuntimeError("oracle: " + self._lib.rho_last_error(self._p).decode())

    def setup_atom(self, atom: dict):
        a = {k: (np.ascontiguousarray(v) if isinstance(v, np.ndarray) else v) for k, v in atom.items()}
        self._keep = [a]
        d = AtomDesc(nlev=a["nlev"], E_J=_d(a["E_J"]), g=_d(a["g"]), nline=len(a["line_l"]),
                     line_l=_i(a["line_l"]), line_u=_i(a["line_u"]), line_f=_d(a["line_f"]),
                     line_a_top=_d(a["line_a_top"]), line_a_bot=_d(a["line_a_bot"]),
                     line_nlambda=_i(a["line_nlambda"]), line_qwing=_d(a["line_qwing"]),
                     ncont=len(a["cont_l"]), cont_l=_i(a["cont_l"]),
                     cont_alpha0=_d(a["cont_alpha0"]), cont_nlambda=_i(a["cont_nlambda"]),
                     cont_ratio=_d(a["cont_ratio"]), mass_amu=a["mass_amu"], T_ref=a["T_ref"],
                     nmu=a["nmu"], metal_floor=a["metal_floor"])
        if "line_prd" in a:
            a["line_prd"] = np.ascontiguousarray(a["line_prd"], dtype=np.int32)
            d.line_prd = _i(a["line_prd"])
        self._check(self._lib.rho_setup_atom(self._p, C.byref(d)))
        self.nlev = a["nlev"]
        self.ntr = len(a["line_l"]) + len(a["cont_l"])
        self.nmu = a["nmu"]

    @property
    def nlambda(self):
        return int(self._lib.rho_nlambda(self._p))

    def grid(self):
        n = self.nlambda
        nu = np.zeros(n)
        nact = np.zeros(n, np.int32)
        act = np.zeros((n, 8), np.int32)
        wq = np.zeros((n, 8))
        self._lib.rho_get_grid(self._p, _d(nu), _i(nact), _i(act), _d(wq))
        return dict(nu=nu, nact=nact, act=act, wq=wq)

    def atom_info(self):
        t = self.ntr
        out = {k: np.zeros(t) for k in ("nu0", "A", "Blu", "Bul")}
        mu = np.zeros(self.nmu)
        wmu = np.zeros(self.nmu)
        self._lib.rho_atom_info(self._p, _d(out["nu0"]), _d(out["A"]), _d(out["Blu"]),
                                _d(out["Bul"]), _d(mu), _d(wmu))
        out["mu"] = mu
        out["wmu"] = wmu
        return out

    def load_columns(self, cols: dict, ne=None):
        z = np.ascontiguousarray(cols["z"], dtype=np.float64)
        T = np.ascontiguousarray(cols["T"], dtype=np.float64)
        nH = np.ascontiguousarray(cols["nH"], dtype=np.float64)
        vz = np.ascontiguousarray(cols["vz"], dtype=np.float64)
        ncol, ndep = T.shape
        nep = None
        if ne is not None:
            ne = np.ascontiguousarray(ne, dtype=np.float64)
            nep = _d(ne)
        self._check(self._lib.rho_load_columns(self._p, ncol, ndep, _d(z), _d(T), nep, _d(nH), _d(vz)))
        self.ncol, self.ndep = ncol, ndep

    def regrid(self, ndep_out, dlog_colden=0.1, dlnT=0.02, dvz=1e3, spacing_factor=4.0, z_top=None):
        """Depth-grid optimisation (Sect. 2.3) of every loaded column onto
        ndep_out points; z_top (m) removes the layers above it."""
        o = GridOpts(dlog_colden=dlog_colden, dlnT=dlnT, dvz=dvz, spacing_factor=spacing_factor,
                     z_top=0.0 if z_top is None else z_top, use_z_top=0 if z_top is None else 1)
        self._check(self._lib.rho_regrid(self._p, ndep_out, C.byref(o)))
        self.ndep = ndep_out

    def columns(self):
        """The loaded atmosphere: dict of z, T, nH, vz [ncol][ndep]."""
        out = {k: np.zeros((self.ncol, self.ndep)) for k in ("z", "T", "nH", "vz")}
        self._check(self._lib.rho_get_columns(self._p, _d(out["z"]), _d(out["T"]), _d(out["nH"]), _d(out["vz"])))
        return out

    def electron_density(self, T, nH):
        return float(self._lib.rho_electron_density(self._p, float(T), float(nH)))

    def lte(self):
        ns = np.zeros((self.ncol, self.nlev, self.ndep))
        ne = np.zeros((self.ncol, self.ndep))
        self._lib.rho_get_lte(self._p, _d(ns), _d(ne))
        return ns, ne

    def populations(self):
        n = np.zeros((self.ncol, self.nlev, self.ndep))
        it = np.zeros(self.ncol, np.int32)
        st = np.zeros(self.ncol, np.uint8)
        dm = np.zeros(self.ncol)
        self._lib.rho_get_populations(self._p, _d(n), _i(it), st.ctypes.data_as(C.POINTER(C.c_uint8)),
                                      _d(dm))
        return n, it, st, dm

    def set_populations(self, n):
        n = np.ascontiguousarray(n, dtype=np.float64)
        self._check(self._lib.rho_set_populations(self._p, _d(n)))

    def iterate(self, maxiter=500, tol=1e-3, ng_order=2, ng_delay=5, ng_period=3, start=0,
                crsw_init=1.0, nthreads=None, prd_eps0=0.0, prd_hybrid=0, formal=0):
        o = IterOpts(maxiter=maxiter, tol=tol, ng_order=ng_order, ng_delay=ng_delay,
                     ng_period=ng_period, start=start, crsw_init=crsw_init, prd_eps0=prd_eps0,
                     prd_hybrid=prd_hybrid, formal=formal)
        s = IterStats()
        if nthreads is None:
            nthreads = os.cpu_count() or 1
        self._check(self._lib.rho_iterate(self._p, C.byref(o), C.byref(s), nthreads))
        self.last_threads = nthreads
        return {f: getattr(s, f) for f, _ in IterStats._fields_}

    def rate_matrix(self, col, n, mode=0):
        n = np.ascontiguousarray(n, dtype=np.float64)
        A = np.zeros((self.ndep, self.nlev, self.nlev))
        self._check(self._lib.rho_rate_matrix(self._p, col, _d(n), mode, _d(A)))
        return A

    def escape_probabilities(self, col, n):
        """p[t][k] of the escape-probability start for populations n of one column."""
        n = np.ascontiguousarray(n, dtype=np.float64)
        e = np.zeros((self.ntr, self.ndep))
        self._check(self._lib.rho_escape_probabilities(self._p, col, _d(n), _d(e)))
        return e

    def column_background(self, col):
        """Background opacity [nlambda][ndep] (m^-1) of column col on the grid."""
        chi = np.zeros((self.nlambda, self.ndep))
        self._check(self._lib.rho_column_background(self._p, col, _d(chi)))
        return chi

    def prd_update_ratio(self, col, n, q):
        """One PRD update of line q from rho = 1 with populations n: the
        plain ratio before switching and before the Jacobi step, [ndep][np],
        points in frequency order."""
        n = np.ascontiguousarray(n, dtype=np.float64)
        m = np.zeros(1, np.int32)
        self._check(self._lib.rho_prd_kernel(self._p, col, q, _i(m), None, None, None, None))
        r = np.zeros((self.ndep, int(m[0])))
        self._check(self._lib.rho_prd_update_ratio(self._p, col, _d(n), q, _d(r)))
        return r

    def prd_kernel(self, col, q):
        """Redistribution kernel of PRD line q in column col: grid indices
        and quadrature weights of its points, K [ndep][np][np], f [ndep][np]."""
        m = np.zeros(1, np.int32)
        self._check(self._lib.rho_prd_kernel(self._p, col, q, _i(m), None, None, None, None))
        n = int(m[0])
        pts = np.zeros(n, np.int32)
        w = np.zeros(n)
        K = np.zeros((self.ndep, n, n))
        f = np.zeros((self.ndep, n))
        self._check(self._lib.rho_prd_kernel(self._p, col, q, _i(m), _i(pts), _d(w), _d(K), _d(f)))
        return pts, w, K, f

    def start_populations(self, kind):
        """Write the start populations (0 LTE, 3 zero radiation, 4 escape
        probability) of every column into the current populations."""
        self._check(self._lib.rho_start_populations(self._p, kind))

    def emergent_stokes(self, line, geff, B_T, theta, chi, lam_m):
        """Stokes (I, Q, U, V) at mu = 1 of line `line` with Zeeman splitting;
        B_T, theta, chi [ncol][ndep]; returns [ncol][nlam][4]."""
        B_T, theta, chi, lam_m = (np.ascontiguousarray(x, dtype=np.float64) for x in (B_T, theta, chi, lam_m))
        out = np.zeros((self.ncol, lam_m.size, 4))
        self._check(self._lib.rho_emergent_stokes(self._p, line, geff, _d(B_T), _d(theta), _d(chi), lam_m.size,
                                                  _d(lam_m), _d(out)))
        return out

    def collision_rates(self, col):
        Cm = np.zeros((self.ndep, self.nlev, self.nlev))
        self._check(self._lib.rho_collision_rates(self._p, col, _d(Cm)))
        return Cm

    def emergent_spectrum(self, mu, lam_m, nthreads=None):
        lam_m = np.ascontiguousarray(lam_m, dtype=np.float64)
        out = np.zeros((self.ncol, lam_m.size))
        if nthreads is None:
            nthreads = os.cpu_count() or 1
        self._check(self._lib.rho_emergent_spectrum(self._p, float(mu), lam_m.size, _d(lam_m),
                                                    _d(out), nthreads))
        return out
