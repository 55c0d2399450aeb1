"""ctypes wrapper of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  Nothing here imports the
GPU package, and the GPU package never imports this.

Variable vector layout: ``[pg(G) | qg(G) | w(B) | theta(B) | wR(L) | wI(L)]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

DP = C.POINTER(C.c_double)
IP = C.POINTER(C.c_int32)
HIST_W = 13


def build(force: bool = False) -> str:
    """Compile liboracle.so in place with gcc (-O2, no target-specific flags)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


class _Grid(C.Structure):
    _fields_ = [("nbus", C.c_int32), ("nbranch", C.c_int32), ("ngen", C.c_int32),
                ("bus_type", IP), ("pd", DP), ("qd", DP), ("gs", DP), ("bs", DP), ("vmin", DP), ("vmax", DP),
                ("f", IP), ("t", IP), ("r", DP), ("x", DP), ("b", DP), ("rate", DP), ("angmin", DP),
                ("angmax", DP), ("tap", DP), ("shift", DP), ("gbus", IP), ("pmin", DP), ("pmax", DP),
                ("qmin", DP), ("qmax", DP), ("c2", DP), ("c1", DP), ("c0", DP), ("base_mva", C.c_double)]


_QP_FIELDS = [("flow", 4, "L"), ("H", 36, "L"), ("aR", 4, "L"), ("aI", 4, "L"), ("bR", 1, "L"), ("bI", 1, "L"),
              ("QH", 16, "L"), ("gH", 4, "L"), ("F", 16, "L"), ("f0", 4, "L"), ("lo", 4, "L"), ("hi", 4, "L"),
              ("G", 8, "L"), ("grhs", 2, "L"), ("alo", 1, "L"), ("ahi", 1, "L"),
              ("gd1", 1, "G"), ("gd2", 1, "G"), ("glp", 1, "G"), ("gup", 1, "G"), ("glq", 1, "G"), ("guq", 1, "G"),
              ("pdk", 1, "B"), ("qdk", 1, "B")]


class _QP(C.Structure):
    _fields_ = [(n, DP) for n, _, _ in _QP_FIELDS]


_ST_FIELDS = [("xl", 8, "L"), ("zl", 8, "L"), ("ll", 8, "L"), ("xg", 2, "G"), ("zg", 2, "G"), ("lg", 2, "G"),
              ("rl", 8, "L"), ("rg", 2, "G"), ("zb", 2, "B"), ("nu", 2, "B"), ("ul", 4, "L")]


class _State(C.Structure):
    _fields_ = [(n, DP) for n, _, _ in _ST_FIELDS] + [("aset", IP)]


class _AdmmOpts(C.Structure):
    _fields_ = [("eps", C.c_double), ("max_iter", C.c_int32), ("use_angle", C.c_int32), ("rb_period", C.c_int32),
                ("rb_mu", C.c_double), ("rb_tau", C.c_double)]


class _AdmmInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("r_inf", C.c_double), ("s_inf", C.c_double),
                ("line_fail", C.c_int32), ("line_reg", C.c_int32)]


class _SqpOpts(C.Structure):
    _fields_ = [("mu", C.c_double), ("tol", C.c_double), ("step_tol", C.c_double), ("delta0", C.c_double),
                ("delta_max", C.c_double), ("delta_min", C.c_double), ("rho", C.c_double),
                ("max_sqp", C.c_int32), ("warm_lambda", C.c_int32), ("admm", _AdmmOpts),
                ("soc", C.c_int32), ("restore", C.c_int32)]


class _SqpInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("accepted", C.c_int32), ("status", C.c_int32), ("admm_total", C.c_int32),
                ("obj", C.c_double), ("primal", C.c_double), ("dual", C.c_double), ("delta", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        L.og_model_create.argtypes = [C.POINTER(_Grid), C.POINTER(C.c_void_p)]
        L.og_model_destroy.argtypes = [C.c_void_p]
        L.og_n_vars.argtypes = [C.c_void_p]
        L.og_admittance.argtypes = [C.c_void_p, DP]
        L.og_flat_start.argtypes = [C.c_void_p, DP]
        L.og_flows.argtypes = [C.c_void_p, DP, DP]
        L.og_constraints.argtypes = [C.c_void_p, DP, DP, DP]
        L.og_objective.argtypes = [C.c_void_p, DP]
        L.og_objective.restype = C.c_double
        L.og_build.argtypes = [C.c_void_p, DP, DP, C.c_double, C.c_int, C.POINTER(_QP)]
        L.og_build_ex.argtypes = [C.c_void_p, DP, DP, C.c_double, C.c_int, DP, C.c_double, C.POINTER(_QP)]
        L.og_merit_ex.argtypes = [C.c_void_p, C.POINTER(_QP), DP, DP, C.c_double, C.c_int, C.c_double, DP, DP, DP]
        L.og_gen_update.argtypes = [C.c_double] * 6 + [DP, DP, DP, DP]
        L.og_line_qp.argtypes = [DP, DP, DP, DP, DP, DP, C.c_double, C.c_double, C.c_int, DP, DP]
        L.og_line_update.argtypes = [C.c_void_p, C.POINTER(_QP), C.c_int, DP, DP, DP, C.c_int, DP, DP, IP]
        L.og_admm_cold.argtypes = [C.c_void_p, C.POINTER(_State), C.c_double, C.c_int]
        L.og_admm.argtypes = [C.c_void_p, C.POINTER(_QP), C.POINTER(_AdmmOpts), C.POINTER(_State),
                              C.POINTER(_AdmmInfo)]
        L.og_step.argtypes = [C.c_void_p, C.POINTER(_QP), C.POINTER(_State), DP, DP, DP]
        L.og_merit.argtypes = [C.c_void_p, C.POINTER(_QP), DP, DP, C.c_double, C.c_int, DP, DP, DP]
        L.og_kkt.argtypes = [C.c_void_p, DP, DP, DP, DP, C.c_int, DP, DP]
        L.og_sqp.argtypes = [C.c_void_p, C.POINTER(_SqpOpts), DP, DP, DP, C.POINTER(_SqpInfo), DP, C.c_int]
        L.og_tr_update.argtypes = [C.POINTER(_SqpOpts), C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.POINTER(C.c_int)]
        L.og_tr_update.restype = C.c_double
        L.og_violations.argtypes = [C.c_void_p, DP, C.c_int, DP, DP]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(DP)


def _ip(a):
    return a.ctypes.data_as(IP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class SqpOptions:
    mu: float = 1e5
    tol: float = 1e-4
    step_tol: float = 1e-9
    delta0: float = 1.0
    delta_max: float = 10.0
    delta_min: float = 1e-8
    rho: float = 2e4
    max_sqp: int = 30
    warm_lambda: int = 1
    eps: float = 1e-4
    max_iter: int = 20000
    use_angle: int = 1
    rb_period: int = 0
    rb_mu: float = 10.0
    rb_tau: float = 2.0
    soc: int = 0
    restore: int = 0


def _sqp_opts(o: SqpOptions):
    return _SqpOpts(o.mu, o.tol, o.step_tol, o.delta0, o.delta_max, o.delta_min, o.rho, o.max_sqp,
                    o.warm_lambda, _AdmmOpts(o.eps, o.max_iter, o.use_angle, o.rb_period, o.rb_mu, o.rb_tau),
                    o.soc, o.restore)


def tr_update(opts: SqpOptions, delta, dnorm, ared, pred):
    """Ratio test and trust-region update of Alg. 1: (accepted, new radius)."""
    acc = C.c_int()
    nd = lib().og_tr_update(C.byref(_sqp_opts(opts)), float(delta), float(dnorm), float(ared), float(pred),
                            C.byref(acc))
    return bool(acc.value), nd


class Model:
    """One grid loaded into the oracle."""

    def __init__(self, grid):
        self._keep = []
        g = _Grid()
        g.nbus, g.nbranch, g.ngen = grid.nbus, grid.nbranch, grid.ngen
        for name in ("pd", "qd", "gs", "bs", "vmin", "vmax", "r", "x", "b", "rate", "angmin", "angmax",
                     "tap", "shift", "pmin", "pmax", "qmin", "qmax", "c2", "c1", "c0"):
            a = _f64(getattr(grid, name))
            self._keep.append(a)
            setattr(g, name, _dp(a))
        for name in ("bus_type", "f", "t", "gbus"):
            a = np.ascontiguousarray(getattr(grid, name), dtype=np.int32)
            self._keep.append(a)
            setattr(g, name, _ip(a))
        g.base_mva = float(grid.base_mva)
        self._g = g
        h = C.c_void_p()
        rc = lib().og_model_create(C.byref(g), C.byref(h))
        if rc != 0:
            raise ValueError(f"oracle rejected the grid (code {rc})")
        self._h = h
        self.grid = grid
        self.B, self.L, self.G = grid.nbus, grid.nbranch, grid.ngen
        self.n = lib().og_n_vars(h)

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().og_model_destroy(self._h)
                self._h = None
        except Exception:
            pass

    # ---------------------------------------------------------------- views
    def split(self, v):
        G, B, L = self.G, self.B, self.L
        o = np.cumsum([0, G, G, B, B, L, L])
        names = ("pg", "qg", "w", "th", "wr", "wi")
        return {k: v[o[i]:o[i + 1]] for i, k in enumerate(names)}

    def _count(self, which):
        return {"L": self.L, "G": self.G, "B": self.B}[which]

    # ------------------------------------------------------------- model fns
    def admittance(self):
        Y = np.zeros(8 * self.L)
        lib().og_admittance(self._h, _dp(Y))
        return Y.reshape(self.L, 8)

    def flat_start(self):
        x = np.zeros(self.n)
        lib().og_flat_start(self._h, _dp(x))
        return x

    def flows(self, x):
        x = _f64(x)
        fl = np.zeros(4 * self.L)
        lib().og_flows(self._h, _dp(x), _dp(fl))
        return fl.reshape(self.L, 4)

    def constraints(self, x):
        x = _f64(x)
        c4 = np.zeros(4 * self.L + 1)
        bal = np.zeros(2 * self.B)
        lib().og_constraints(self._h, _dp(x), _dp(c4), _dp(bal))
        return c4[:4 * self.L].reshape(self.L, 4), bal.reshape(self.B, 2)

    def objective(self, x):
        return lib().og_objective(self._h, _dp(_f64(x)))

    def violations(self, x, use_angle=1):
        """(l1 sum, l_inf maximum) of every constraint violation at x."""
        a, b = C.c_double(), C.c_double()
        lib().og_violations(self._h, _dp(_f64(x)), int(use_angle), C.byref(a), C.byref(b))
        return a.value, b.value

    # --------------------------------------------------------------- QP data
    def new_qp(self):
        arrs = {n: np.zeros(w * max(self._count(c), 1)) for n, w, c in _QP_FIELDS}
        s = _QP(**{n: _dp(arrs[n]) for n in arrs})
        return arrs, s

    def build(self, x, pi=None, delta=1.0, use_angle=1, dsoc=None, fscale=1.0):
        """QP of eq. QPsub at x; with dsoc, the second-order correction QP of
        that step; fscale weights the objective (0: restoration)."""
        x = _f64(x)
        pi = np.zeros(4 * self.L) if pi is None else _f64(pi).ravel()
        arrs, s = self.new_qp()
        if dsoc is None and fscale == 1.0:
            lib().og_build(self._h, _dp(x), _dp(pi), float(delta), int(use_angle), C.byref(s))
        else:
            ds = None if dsoc is None else _dp(_f64(dsoc))
            lib().og_build_ex(self._h, _dp(x), _dp(pi), float(delta), int(use_angle), ds, float(fscale), C.byref(s))
        return QP(self, arrs, s)

    # ------------------------------------------------------------------ ADMM
    def new_state(self, rho=2e4):
        arrs = {n: np.zeros(w * max(self._count(c), 1)) for n, w, c in _ST_FIELDS}
        st = AdmmState(self, arrs)
        lib().og_admm_cold(self._h, C.byref(st.s), float(rho), 0)
        return st

    def cold(self, state, rho=2e4, keep_lambda=0):
        """ADMM restart for a new QP: d, z = 0; multipliers reset unless kept."""
        lib().og_admm_cold(self._h, C.byref(state.s), float(rho), int(keep_lambda))
        return state

    def admm(self, qp, state=None, rho=2e4, eps=1e-4, max_iter=20000, use_angle=1, rb_period=0, rb_mu=10.0,
             rb_tau=2.0):
        st = self.new_state(rho) if state is None else state
        o = _AdmmOpts(float(eps), int(max_iter), int(use_angle), int(rb_period), float(rb_mu), float(rb_tau))
        info = _AdmmInfo()
        lib().og_admm(self._h, C.byref(qp.s), C.byref(o), C.byref(st.s), C.byref(info))
        return st, dict(iters=info.iters, r=info.r_inf, s=info.s_inf, line_fail=info.line_fail,
                        line_reg=info.line_reg)

    def step(self, qp, state, x):
        d = np.zeros(self.n)
        pi = np.zeros(4 * self.L + 1)
        lib().og_step(self._h, C.byref(qp.s), C.byref(state.s), _dp(_f64(x)), _dp(d), _dp(pi))
        return d, pi[:4 * self.L]

    def merit(self, qp, x, d, mu=1e5, use_angle=1, fscale=1.0):
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        lib().og_merit_ex(self._h, C.byref(qp.s), _dp(_f64(x)), _dp(_f64(d)), float(mu), int(use_angle),
                          float(fscale), C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def kkt(self, x, pi, nu, ul, use_angle=1):
        p, dd = C.c_double(), C.c_double()
        pi = _f64(pi)
        pi = np.concatenate([pi, [0.0]])
        ul = np.concatenate([_f64(ul), [0.0]])
        lib().og_kkt(self._h, _dp(_f64(x)), _dp(pi), _dp(_f64(nu)), _dp(ul), int(use_angle),
                     C.byref(p), C.byref(dd))
        return p.value, dd.value

    def sqp(self, opts: SqpOptions | None = None, x0=None, hist_cap=200):
        o = opts or SqpOptions()
        so = _sqp_opts(o)
        x0 = self.flat_start() if x0 is None else _f64(x0)
        x = np.zeros(self.n)
        pi = np.zeros(4 * self.L + 1)
        info = _SqpInfo()
        hist = np.zeros(HIST_W * hist_cap)
        lib().og_sqp(self._h, C.byref(so), _dp(x0), _dp(x), _dp(pi), C.byref(info), _dp(hist), hist_cap)
        k = min(info.iters, hist_cap)
        return dict(x=x, pi=pi[:4 * self.L], status=info.status, iters=info.iters, accepted=info.accepted,
                    admm_total=info.admm_total, obj=info.obj, primal=info.primal, dual=info.dual,
                    delta=info.delta, hist=hist[:HIST_W * k].reshape(k, HIST_W))


class QP:
    def __init__(self, model, arrs, s):
        self.model, self.a, self.s = model, arrs, s

    def __getitem__(self, k):
        m = self.model
        w = dict((n, (wd, c)) for n, wd, c in _QP_FIELDS)[k]
        n = m._count(w[1])
        a = self.a[k][:w[0] * n]
        return a.reshape(n, w[0]) if w[0] > 1 else a


class AdmmState:
    def __init__(self, model, arrs):
        self.model, self.a = model, arrs
        self.aset = np.full(max(model.L, 1), -1, dtype=np.int32)
        self.s = _State(**{n: _dp(arrs[n]) for n in arrs}, aset=_ip(self.aset))

    def __getitem__(self, k):
        m = self.model
        w = dict((n, (wd, c)) for n, wd, c in _ST_FIELDS)[k]
        n = m._count(w[1])
        a = self.a[k][:w[0] * n]
        return a.reshape(n, w[0]) if w[0] > 1 else a


def line_qp(Q, c, lo, hi, G, grhs, alo, ahi, use_angle=1):
    """Exact minimiser of the 4-variable line QP; returns (x, mult[4], rc)."""
    x = np.zeros(4)
    mult = np.zeros(4)
    args = [_f64(np.asarray(Q).ravel()), _f64(c), _f64(lo), _f64(hi), _f64(np.asarray(G).ravel()), _f64(grhs)]
    rc = lib().og_line_qp(*[_dp(a) for a in args], float(alo), float(ahi), int(use_angle), _dp(x), _dp(mult))
    return x, mult, rc


def gen_update(gd1, gd2, lp, up, lq, uq, z, lam, rho):
    out = np.zeros(2)
    lib().og_gen_update(gd1, gd2, lp, up, lq, uq, _dp(_f64(z)), _dp(_f64(lam)), _dp(_f64(rho)), _dp(out))
    return out
