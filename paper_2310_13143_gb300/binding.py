"""ctypes binding of libacopf.so (include/acopf.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  There is no CPU fallback -- if the library is missing or no
CUDA device is usable the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libacopf.so")

DP = C.POINTER(C.c_double)
FP = C.POINTER(C.c_float)
IP = C.POINTER(C.c_int32)

ACOPF_FP64, ACOPF_MIXED = 0, 1
RESULTS = {0: "converged", 1: "max_iter", 2: "step_too_small", 3: "non_finite", 4: "running", 5: "infeasible"}
STATUS = {0: "ok", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTREADY"}


class AcopfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class acopf_grid(C.Structure):
    _fields_ = [("nbus", C.c_int32), ("bus_type", IP), ("pd", DP), ("qd", DP), ("gs", DP), ("bs", DP),
                ("vmin", DP), ("vmax", DP), ("nbranch", C.c_int32), ("f", IP), ("t", IP), ("r", DP), ("x", DP),
                ("b", DP), ("rate", DP), ("angmin", DP), ("angmax", DP), ("tap", DP), ("shift", DP),
                ("ngen", C.c_int32), ("gbus", IP), ("pmin", DP), ("pmax", DP), ("qmin", DP), ("qmax", DP),
                ("c2", DP), ("c1", DP), ("c0", DP), ("base_mva", C.c_double)]


class acopf_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("use_angle", C.c_int32), ("device", C.c_int32),
                ("block_threads", C.c_int32), ("ctas_per_sm", C.c_int32)]


class admm_options(C.Structure):
    _fields_ = [("rho", C.c_double), ("eps", C.c_double), ("eps_dual", C.c_double), ("max_iter", C.c_int32),
                ("warm", C.c_int32),
                ("alm_beta", C.c_double), ("alm_tol", C.c_double), ("alm_max_outer", C.c_int32),
                ("newton_max", C.c_int32), ("spin_limit", C.c_int64), ("rb_period", C.c_int32),
                ("rb_mu", C.c_double), ("rb_tau", C.c_double), ("line_solver", C.c_int32)]


class sqp_options(C.Structure):
    _fields_ = [("mu", C.c_double), ("tol", C.c_double), ("step_tol", C.c_double), ("delta0", C.c_double),
                ("delta_max", C.c_double), ("delta_min", C.c_double), ("max_sqp", C.c_int32),
                ("merit_linear", C.c_int32), ("admm", admm_options), ("soc", C.c_int32), ("restore", C.c_int32)]


class acopf_solution(C.Structure):
    _fields_ = [("pg", DP), ("qg", DP), ("vm", DP), ("va", DP), ("wr", DP), ("wi", DP), ("obj", C.c_double)]


class acopf_residuals(C.Structure):
    _fields_ = [("primal", C.c_double), ("dual", C.c_double), ("r_inf", C.c_double), ("s_inf", C.c_double),
                ("obj", C.c_double), ("delta", C.c_double), ("sqp_iter", C.c_int32), ("admm_iter", C.c_int32),
                ("accepted", C.c_int32), ("result", C.c_int32)]


QP_FIELDS = [("flow", 4), ("H", 36), ("aR", 4), ("aI", 4), ("bR", 1), ("bI", 1), ("QH", 16), ("gH", 4),
             ("F", 16), ("f0", 4), ("lo", 4), ("hi", 4), ("G", 8), ("grhs", 2), ("alo", 1), ("ahi", 1)]


class acopf_qp_view(C.Structure):
    _fields_ = [(n, DP) for n, _ in QP_FIELDS] + [("gen", DP), ("bus", DP)]


STATE_FIELDS = [("x", 8, "L"), ("z", 8, "L"), ("lam", 8, "L"), ("xg", 2, "G"), ("zg", 2, "G"), ("lg", 2, "G"),
                ("zb", 2, "B"), ("nu", 2, "B"), ("ul", 4, "L")]


class acopf_admm_state(C.Structure):
    _fields_ = [(n, DP) for n, _, _ in STATE_FIELDS]


_lib = None


# device allocator callbacks of acopf_set_allocator: alloc(bytes, ctx) -> ptr, release(ptr, ctx)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def lib():
    """Load libacopf.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2310_13143_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        H = C.c_void_p
        S = C.c_int
        sig = {
            "acopf_default_options": (None, [C.POINTER(acopf_options)]),
            "admm_default_options": (None, [C.POINTER(admm_options)]),
            "sqp_default_options": (None, [C.POINTER(sqp_options)]),
            "acopf_status_string": (C.c_char_p, [S]),
            "acopf_last_error": (S, [H, C.c_char_p, C.c_size_t]),
            "acopf_create": (S, [C.POINTER(acopf_grid), C.c_int32, C.POINTER(acopf_options), C.POINTER(H)]),
            "acopf_destroy": (S, [H]),
            "acopf_set_stream": (S, [H, C.c_void_p]),
            "acopf_set_allocator": (S, [H, ALLOC_FN, FREE_FN, C.c_void_p]),
            "acopf_set_loads": (S, [H, C.c_int32, DP, DP]),
            "sqp_solve": (S, [H, C.POINTER(sqp_options)]),
            "admm_solve_qp": (S, [H, C.c_double, C.POINTER(admm_options)]),
            "acopf_set_warm_start": (S, [H, C.c_int32, DP, DP, DP]),
            "acopf_get_solution": (S, [H, C.c_int32, C.POINTER(acopf_solution)]),
            "acopf_get_residuals": (S, [H, C.c_int32, C.POINTER(acopf_residuals)]),
            "acopf_set_iterate": (S, [H, C.c_int32, DP, DP]),
            "acopf_get_iterate": (S, [H, C.c_int32, DP, DP]),
            "acopf_build_qp": (S, [H, C.c_double, C.c_double, C.c_int32]),
            "acopf_get_qp": (S, [H, C.c_int32, C.POINTER(acopf_qp_view)]),
            "acopf_get_admm_state": (S, [H, C.c_int32, C.POINTER(acopf_admm_state)]),
            "acopf_set_admm_state": (S, [H, C.c_int32, C.POINTER(acopf_admm_state)]),
            "admm_iterate": (S, [H, C.c_int32, C.POINTER(admm_options)]),
            "acopf_get_step": (S, [H, C.c_int32, DP, DP]),
            "acopf_launch_count": (S, [H, C.POINTER(C.c_int64)]),
            "acopf_profile": (S, [H, C.c_int32]),
            "acopf_get_history": (S, [H, C.c_int32, DP, C.c_int32, IP]),
            "admm_iterate_static": (S, [H, C.c_int32, C.POINTER(admm_options), C.c_void_p, C.c_void_p]),
            "acopf_get_profile_phases": (S, [H, DP]),
            "acopf_tune": (S, [H, C.c_int32, C.c_int32, C.c_int32]),
            "acopf_get_profile": (S, [H, DP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
            "acopf_set_warm_start_device": (S, [H, C.c_void_p, C.c_int64, C.c_double, S, S, S, S]),
            "sqp_solve_graph": (S, [H, C.POINTER(sqp_options), C.c_int32]),
            "acopf_project_linear": (S, [H, C.c_double, C.c_double, C.c_int32, IP, DP]),
            "acopf_autotune": (S, [H, C.c_char_p, C.c_int32, IP, DP]),
            "acopf_mlp_create": (S, [IP, C.c_int32, C.c_int32, C.c_int32, C.POINTER(H)]),
            "acopf_mlp_destroy": (S, [H]),
            "acopf_mlp_set_stream": (S, [H, C.c_void_p]),
            "acopf_mlp_last_error": (S, [H, C.c_char_p, C.c_size_t]),
            "acopf_mlp_num_params": (S, [H, C.POINTER(C.c_int64)]),
            "acopf_mlp_set_params": (S, [H, FP, C.c_int64]),
            "acopf_mlp_get_params": (S, [H, FP, C.c_int64]),
            "acopf_mlp_get_grads": (S, [H, FP, C.c_int64]),
            "acopf_mlp_fit_standardiser": (S, [H, C.c_void_p, C.c_void_p, C.c_int32]),
            "acopf_mlp_get_standardiser": (S, [H, FP, FP, FP, FP]),
            "acopf_mlp_forward": (S, [H, C.c_void_p, C.c_int32, C.c_void_p]),
            "acopf_mlp_train_step": (S, [H, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_void_p]),
            "acopf_mlp_sync": (S, [H]),
            "acopf_gemm_bf16": (S, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                    C.c_void_p, FP]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


EXPORTED = ["acopf_default_options", "admm_default_options", "sqp_default_options", "acopf_status_string",
            "acopf_last_error", "acopf_create", "acopf_destroy", "acopf_set_stream", "acopf_set_allocator",
            "acopf_set_loads", "sqp_solve",
            "admm_solve_qp", "acopf_set_warm_start", "acopf_get_solution", "acopf_get_residuals",
            "acopf_set_iterate", "acopf_get_iterate", "acopf_build_qp", "acopf_get_qp", "acopf_get_admm_state",
            "acopf_set_admm_state", "admm_iterate", "acopf_get_step", "acopf_launch_count", "acopf_profile",
            "acopf_get_profile", "acopf_get_history", "admm_iterate_static", "acopf_get_profile_phases",
            "acopf_tune", "acopf_set_warm_start_device", "sqp_solve_graph", "acopf_autotune", "acopf_project_linear", "acopf_mlp_create", "acopf_mlp_destroy",
            "acopf_mlp_set_stream", "acopf_mlp_last_error", "acopf_mlp_num_params", "acopf_mlp_set_params",
            "acopf_mlp_get_params", "acopf_mlp_get_grads", "acopf_mlp_fit_standardiser",
            "acopf_mlp_get_standardiser", "acopf_mlp_forward", "acopf_mlp_train_step", "acopf_mlp_sync",
            "acopf_gemm_bf16"]


def _dp(a):
    return None if a is None else a.ctypes.data_as(DP)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_admm(**kw) -> admm_options:
    o = admm_options()
    lib().admm_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def default_sqp(admm: dict | None = None, **kw) -> sqp_options:
    o = sqp_options()
    lib().sqp_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    for k, v in (admm or {}).items():
        setattr(o.admm, k, v)
    return o


class Solver:
    """A handle over one or more grids (``gridgen.Grid``-like objects)."""

    def __init__(self, grids, precision: str = "fp64", use_angle: bool = True, device: int = 0,
                 block_threads: int = 256, ctas_per_sm: int = 0):
        if not isinstance(grids, (list, tuple)):
            grids = [grids]
        self.grids = list(grids)
        self._keep = []
        arr = (acopf_grid * len(grids))()
        for k, g in enumerate(grids):
            s = arr[k]
            s.nbus, s.nbranch, s.ngen = g.nbus, g.nbranch, g.ngen
            for name in ("pd", "qd", "gs", "bs", "vmin", "vmax", "r", "x", "b", "rate", "angmin", "angmax",
                         "tap", "shift", "pmin", "pmax", "qmin", "qmax", "c2", "c1", "c0"):
                a = _f64(getattr(g, name))
                self._keep.append(a)
                setattr(s, name, a.ctypes.data_as(DP))
            for name in ("bus_type", "f", "t", "gbus"):
                a = np.ascontiguousarray(getattr(g, name), dtype=np.int32)
                self._keep.append(a)
                setattr(s, name, a.ctypes.data_as(IP))
            s.base_mva = float(g.base_mva)
        o = acopf_options()
        lib().acopf_default_options(C.byref(o))
        o.precision = ACOPF_MIXED if precision == "mixed" else ACOPF_FP64
        o.use_angle = int(bool(use_angle))
        o.device = device
        o.block_threads = block_threads
        o.ctas_per_sm = ctas_per_sm
        h = C.c_void_p()
        st = lib().acopf_create(arr, len(grids), C.byref(o), C.byref(h))
        if st != 0:
            buf = C.create_string_buffer(512)
            lib().acopf_last_error(None, buf, 512)
            raise AcopfError(st, buf.value.decode())
        self.h = h
        self._keep_arr = arr
        self.precision = precision
        self.device = device
        self._alloc_cbs = None

    def close(self):
        if getattr(self, "h", None):
            lib().acopf_destroy(self.h)
            self.h = None
        self._alloc_cbs = None  # after destroy, which may still call them

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            buf = C.create_string_buffer(512)
            lib().acopf_last_error(self.h, buf, 512)
            raise AcopfError(st, buf.value.decode())

    def _dims(self, inst):
        g = self.grids[inst]
        return g.nbus, g.nbranch, g.ngen

    def nvars(self, inst=0):
        B, L, G = self._dims(inst)
        return 2 * G + 2 * B + 2 * L

    # ------------------------------------------------------------ solver calls
    def set_stream(self, stream_ptr: int):
        self._check(lib().acopf_set_stream(self.h, C.c_void_p(stream_ptr)))

    def set_allocator(self, alloc=None, free=None):
        """Move the handle's device memory to alloc(nbytes) -> int / free(ptr)
        and allocate through them from now on; no arguments: back to
        cudaMalloc.  The callbacks stay referenced until close()."""
        if (alloc is None) != (free is None):
            raise ValueError("give both alloc and free, or neither")
        if alloc is None:
            cbs = (ALLOC_FN(), FREE_FN())  # NULL function pointers
        else:
            cbs = (ALLOC_FN(lambda n, ctx: alloc(n)), FREE_FN(lambda p, ctx: free(p)))
        self._check(lib().acopf_set_allocator(self.h, cbs[0], cbs[1], None))
        # the old callbacks were last used inside the call above
        self._alloc_cbs = cbs if alloc is not None else None

    def use_torch_allocator(self):
        """Serve the handle's device memory from torch's caching allocator."""
        import torch

        dev = self.device
        self.set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n, device=dev),
                           torch.cuda.caching_allocator_delete)

    def set_loads(self, inst, pd, qd):
        pd, qd = _f64(pd), _f64(qd)
        self._check(lib().acopf_set_loads(self.h, inst, _dp(pd), _dp(qd)))

    def sqp_solve(self, opts: sqp_options | None = None):
        self._check(lib().sqp_solve(self.h, C.byref(opts or default_sqp())))

    def sqp_solve_graph(self, opts: sqp_options | None = None, check_every: int = 4):
        self._check(lib().sqp_solve_graph(self.h, C.byref(opts or default_sqp()), int(check_every)))

    def project_linear(self, rho=0.5, eps=1e-6, max_iter=20000):
        """Project every instance's iterate onto the linear constraints; returns
        (iterations, largest primal residual, largest dual residual)."""
        it = C.c_int32()
        rs = np.zeros(2)
        self._check(lib().acopf_project_linear(self.h, float(rho), float(eps), int(max_iter), C.byref(it), _dp(rs)))
        return it.value, rs[0], rs[1]

    def autotune(self, cache_path: str | None = None, iters: int = 50):
        """Returns ((threads, ctas_per_sm, stages), us_per_iter or -1 if cached)."""
        shape = np.zeros(3, dtype=np.int32)
        us = C.c_double()
        self._check(lib().acopf_autotune(self.h, cache_path.encode() if cache_path else None, int(iters),
                                         shape.ctypes.data_as(IP), C.byref(us)))
        return tuple(int(v) for v in shape), us.value

    def admm_solve_qp(self, delta=1.0, opts: admm_options | None = None):
        self._check(lib().admm_solve_qp(self.h, float(delta), C.byref(opts or default_admm())))

    def admm_iterate(self, n, opts: admm_options | None = None):
        self._check(lib().admm_iterate(self.h, int(n), C.byref(opts or default_admm())))

    def build_qp(self, delta=1.0, rho=2e4, use_angle=True):
        self._check(lib().acopf_build_qp(self.h, float(delta), float(rho), int(bool(use_angle))))

    def set_warm_start_device(self, pred_ptr: int, ld: int, base_rho=2e4, use_x=True, use_pi=True, use_lambda=True,
                              use_rho=True):
        """Warm start of every instance from device predictions (FP32 [K x ld] at pred_ptr)."""
        self._check(lib().acopf_set_warm_start_device(self.h, C.c_void_p(pred_ptr), int(ld), float(base_rho),
                                                      int(use_x), int(use_pi), int(use_lambda), int(use_rho)))

    def set_warm_start(self, inst, x0=None, lambda0=None, rho=None):
        a, b, c = (None if v is None else _f64(v) for v in (x0, lambda0, rho))
        self._check(lib().acopf_set_warm_start(self.h, inst, _dp(a), _dp(b), _dp(c)))

    # -------------------------------------------------------------- read-outs
    def set_iterate(self, inst, x, pi=None):
        x = _f64(x)
        pi = None if pi is None else _f64(pi)
        self._check(lib().acopf_set_iterate(self.h, inst, _dp(x), _dp(pi)))

    def get_iterate(self, inst=0):
        B, L, G = self._dims(inst)
        x = np.zeros(2 * G + 2 * B + 2 * L)
        pi = np.zeros(4 * max(L, 1))
        self._check(lib().acopf_get_iterate(self.h, inst, _dp(x), _dp(pi)))
        return x, pi[:4 * L]

    def get_qp(self, inst=0):
        B, L, G = self._dims(inst)
        out = {n: np.zeros(w * max(L, 1)) for n, w in QP_FIELDS}
        out["gen"] = np.zeros(6 * G)
        out["bus"] = np.zeros(2 * B)
        v = acopf_qp_view(**{n: _dp(a) for n, a in out.items()})
        self._check(lib().acopf_get_qp(self.h, inst, C.byref(v)))
        res = {}
        for n, w in QP_FIELDS:
            a = out[n][:w * L]
            res[n] = a.reshape(L, w) if w > 1 else a
        gen = out["gen"].reshape(G, 6)
        for k, n in enumerate(("gd1", "gd2", "glp", "gup", "glq", "guq")):
            res[n] = gen[:, k].copy()
        res["pdk"] = out["bus"][0::2].copy()
        res["qdk"] = out["bus"][1::2].copy()
        return res

    def get_admm_state(self, inst=0):
        B, L, G = self._dims(inst)
        cnt = {"L": max(L, 1), "G": G, "B": B}
        out = {n: np.zeros(w * cnt[c]) for n, w, c in STATE_FIELDS}
        s = acopf_admm_state(**{n: _dp(a) for n, a in out.items()})
        self._check(lib().acopf_get_admm_state(self.h, inst, C.byref(s)))
        real = {"L": L, "G": G, "B": B}
        return {n: out[n][:w * real[c]].reshape(real[c], w) for n, w, c in STATE_FIELDS}

    def set_admm_state(self, inst, state: dict):
        arrs = {n: (None if state.get(n) is None else _f64(np.asarray(state[n]).ravel())) for n, _, _ in STATE_FIELDS}
        s = acopf_admm_state(**{n: (_dp(a) if a is not None else None) for n, a in arrs.items()})
        self._check(lib().acopf_set_admm_state(self.h, inst, C.byref(s)))

    def get_step(self, inst=0):
        B, L, G = self._dims(inst)
        d = np.zeros(2 * G + 2 * B + 2 * L)
        pi = np.zeros(4 * max(L, 1))
        self._check(lib().acopf_get_step(self.h, inst, _dp(d), _dp(pi)))
        return d, pi[:4 * L]

    def get_solution(self, inst=0):
        B, L, G = self._dims(inst)
        arrs = {"pg": np.zeros(G), "qg": np.zeros(G), "vm": np.zeros(B), "va": np.zeros(B),
                "wr": np.zeros(max(L, 1)), "wi": np.zeros(max(L, 1))}
        s = acopf_solution(**{n: _dp(a) for n, a in arrs.items()})
        self._check(lib().acopf_get_solution(self.h, inst, C.byref(s)))
        arrs["wr"], arrs["wi"] = arrs["wr"][:L], arrs["wi"][:L]
        arrs["obj"] = s.obj
        return arrs

    def get_residuals(self, inst=0):
        r = acopf_residuals()
        self._check(lib().acopf_get_residuals(self.h, inst, C.byref(r)))
        d = {n: getattr(r, n) for n, _ in acopf_residuals._fields_}
        d["result_name"] = RESULTS.get(d["result"], str(d["result"]))
        return d

    HIST_COLS = ("obj", "primal", "dual", "admm_iters", "r", "s", "accepted", "delta", "dnorm", "ared", "pred",
                 "rho_factor", "soc", "restoring")

    def get_history(self, inst=0):
        w = len(self.HIST_COLS)
        out = np.zeros(64 * w)
        n = C.c_int32()
        self._check(lib().acopf_get_history(self.h, inst, _dp(out), 64, C.byref(n)))
        k = min(n.value, 64)
        return out[:w * k].reshape(k, w)

    def profile(self, on=True):
        self._check(lib().acopf_profile(self.h, int(bool(on))))

    def get_profile(self):
        ms = C.c_double()
        n, it = C.c_int64(), C.c_int64()
        self._check(lib().acopf_get_profile(self.h, C.byref(ms), C.byref(n), C.byref(it)))
        return dict(sweep_ms=ms.value, sweeps=n.value, admm_iters=it.value)

    def get_profile_phases(self):
        ns = np.zeros(4)
        self._check(lib().acopf_get_profile_phases(self.h, _dp(ns)))
        return dict(phase_a_ns=ns[0], wait1_ns=ns[1], phase_b_ns=ns[2], wait2_ns=ns[3])

    def tune(self, block_threads=0, ctas_per_sm=-1, sweep_stages=-1):
        self._check(lib().acopf_tune(self.h, block_threads, ctas_per_sm, sweep_stages))

    def launch_count(self):
        n = C.c_int64()
        self._check(lib().acopf_launch_count(self.h, C.byref(n)))
        return n.value


def gemm_bf16(a_ptr: int, b_ptr: int, c_ptr: int, M: int, N: int, K: int, splits: int = 1, stream: int = 0):
    """C [M x N] = A [M x K] B [N x K]^T on the tensor cores (device pointers:
    bfloat16 A and B, FP32 C).  Returns the kernels' device time in ms."""
    ms = C.c_float()
    st = lib().acopf_gemm_bf16(C.c_void_p(a_ptr), C.c_void_p(b_ptr), C.c_void_p(c_ptr), M, N, K, splits,
                               C.c_void_p(stream), C.byref(ms))
    if st != 0:
        raise AcopfError(st, "acopf_gemm_bf16 failed")
    return ms.value


class Mlp:
    """The warm-start network (include/acopf_mlp.h); device buffers are passed
    as integer device pointers."""

    def __init__(self, dims, max_batch: int, device: int = 0):
        self.dims = [int(d) for d in dims]
        arr = np.ascontiguousarray(self.dims, dtype=np.int32)
        h = C.c_void_p()
        st = lib().acopf_mlp_create(arr.ctypes.data_as(IP), len(self.dims) - 1, int(max_batch), device, C.byref(h))
        if st != 0:
            raise AcopfError(st, "acopf_mlp_create failed")
        self.h = h
        n = C.c_int64()
        self._check(lib().acopf_mlp_num_params(self.h, C.byref(n)))
        self.nparams = n.value

    def _check(self, st):
        if st != 0:
            buf = C.create_string_buffer(512)
            lib().acopf_mlp_last_error(self.h, buf, 512)
            raise AcopfError(st, buf.value.decode())

    def close(self):
        if getattr(self, "h", None):
            lib().acopf_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr: int):
        self._check(lib().acopf_mlp_set_stream(self.h, C.c_void_p(stream_ptr)))

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(lib().acopf_mlp_set_params(self.h, a.ctypes.data_as(FP), a.size))

    def get_params(self):
        a = np.zeros(self.nparams, dtype=np.float32)
        self._check(lib().acopf_mlp_get_params(self.h, a.ctypes.data_as(FP), a.size))
        return a

    def get_grads(self):
        a = np.zeros(self.nparams, dtype=np.float32)
        self._check(lib().acopf_mlp_get_grads(self.h, a.ctypes.data_as(FP), a.size))
        return a

    def fit_standardiser(self, x_ptr: int, y_ptr: int, rows: int):
        self._check(lib().acopf_mlp_fit_standardiser(self.h, C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(rows)))

    def get_standardiser(self):
        d0, dn = self.dims[0], self.dims[-1]
        out = [np.zeros(d, dtype=np.float32) for d in (d0, d0, dn, dn)]
        self._check(lib().acopf_mlp_get_standardiser(self.h, *[o.ctypes.data_as(FP) for o in out]))
        return out

    def forward(self, x_ptr: int, rows: int, y_ptr: int):
        self._check(lib().acopf_mlp_forward(self.h, C.c_void_p(x_ptr), int(rows), C.c_void_p(y_ptr)))

    def train_step(self, x_ptr: int, t_ptr: int, idx_ptr, rows: int, lr: float, loss_ptr=None):
        self._check(lib().acopf_mlp_train_step(self.h, C.c_void_p(x_ptr), C.c_void_p(t_ptr),
                                               C.c_void_p(idx_ptr or 0) if idx_ptr else None, int(rows),
                                               float(lr), C.c_void_p(loss_ptr) if loss_ptr else None))

    def sync(self):
        self._check(lib().acopf_mlp_sync(self.h))
