"""Thin ctypes binding of the TAPS C ABI (include/taps.h).

Argument marshalling only: every step of the method runs in the CUDA library
libtaps.so built from csrc/.  PyTorch is used for the current CUDA stream and for
device buffers handed to the evaluation entry points.  If the library is missing the
binding raises; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtaps.so")

MAX_DIMS = 8
MAX_TERMS = 128
MAX_SOURCES = 4096
OK, ERR_INVALID_ARG, ERR_SINGULAR, ERR_NONFINITE, ERR_NOT_CONVERGED = 0, -1, -2, -3, -4
ERR_TIMEOUT, ERR_CUDA, ERR_OOM, ERR_SCRATCH_LIMIT = -5, -6, -7, -8
NOALLOC_SCRATCH_BYTES = 4 << 20
SPACE, PARAM, TIME = 0, 1, 2
OP = {"K": 0, "M": 1, "G": 2, "W": 3, "Blo": 4, "Bhi": 5}
OP_WEIGHTED = 16   # 'w<j>' in a term: weighted operator j of that dim


def op_code(name):
    """'K', 'M', 'G', 'W', 'Blo', 'Bhi' or 'w<j>' (the dim's weighted operator j)."""
    return OP_WEIGHTED + int(name[1:]) if name.startswith("w") else OP[name]
NUM_OPS = 6
SRC = {"const": 0, "sin": 1, "gauss": 2, "poly": 3, "nodal": 4, "opvec": 5, "opvecfull": 6}
FP64, FP32, MIXED, BF16 = 0, 1, 2, 3
RES_ALS, RES_FULL = 0, 1
INIT_GIVEN, INIT_RANDOM, INIT_ZERO = 0, 1, 2
SOLVER_BLOCK_LU, SOLVER_FASTDIAG, SOLVER_MODEDIAG, SOLVER_AUTO = 0, 1, 2, 3


class DimDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("lo", ctypes.c_double),
                ("hi", ctypes.c_double), ("s", ctypes.c_int), ("a", ctypes.c_double),
                ("p", ctypes.c_int), ("n_quad", ctypes.c_int), ("dirichlet_lo", ctypes.c_int),
                ("dirichlet_hi", ctypes.c_int), ("weight_poly", ctypes.c_double * 4)]


class Term(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("op", ctypes.c_int * MAX_DIMS)]


class Source(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("kind", ctypes.c_int * MAX_DIMS),
                ("par", (ctypes.c_double * 4) * MAX_DIMS),
                ("nodal", ctypes.POINTER(ctypes.c_double) * MAX_DIMS)]


class SweepOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("solver", ctypes.c_int), ("normalize", ctypes.c_int)]


class SweepReport(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("change", ctypes.c_double), ("seconds", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("M0", ctypes.c_int), ("M_max", ctypes.c_int), ("als_tol", ctypes.c_double),
                ("res_tol", ctypes.c_double), ("res_kind", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("precision", ctypes.c_int),
                ("polish_sweeps", ctypes.c_int), ("solver", ctypes.c_int), ("init", ctypes.c_int),
                ("seed", ctypes.c_uint), ("history_cap", ctypes.c_int), ("graphs", ctypes.c_int),
                ("res_stall", ctypes.c_double), ("M_step", ctypes.c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("sweeps", ctypes.c_int), ("fp64_sweeps", ctypes.c_int),
                ("rho", ctypes.c_double), ("rho_full", ctypes.c_double),
                ("change", ctypes.c_double), ("seconds", ctypes.c_double),
                ("converged", ctypes.c_int), ("hist_M", ctypes.POINTER(ctypes.c_int)),
                ("hist_change", ctypes.POINTER(ctypes.c_double)),
                ("hist_rho", ctypes.POINTER(ctypes.c_double)), ("hist_len", ctypes.c_int)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)
_pi = ctypes.POINTER(ctypes.c_int)

# name -> (restype, argtypes); the full exported surface of include/taps.h
SIGNATURES = {
    "taps_status_string": (ctypes.c_char_p, [_i]),
    "taps_version": (_i, []),
    "taps_assemble_1d": (_i, [ctypes.POINTER(DimDesc), _vp, ctypes.POINTER(_vp)]),
    "taps_dim_info": (_i, [_vp, _pi, _pi, _pi]),
    "taps_dim_copy_band": (_i, [_vp, _i, _pd]),
    "taps_dim_copy_shape": (_i, [_vp, _pd, _pd, _pd]),
    "taps_dim_destroy": (None, [_vp]),
    "taps_problem_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(Term), _i,
                                 ctypes.POINTER(Source), _i, _vp, ctypes.POINTER(_vp)]),
    "taps_problem_copy_source": (_i, [_vp, _i, _i, _pd]),
    "taps_problem_set_weighted_ops": (_i, [_vp, _i, _i, ctypes.POINTER(_i), _pd]),
    "taps_problem_copy_op": (_i, [_vp, _i, _i, _pd]),
    "taps_factors_copy": (_i, [_vp, _vp]),
    "taps_factors_rel_change": (_i, [_vp, _vp, _pd]),
    "taps_problem_destroy": (None, [_vp]),
    "taps_factors_create": (_i, [_vp, _i, ctypes.POINTER(_vp)]),
    "taps_factors_set": (_i, [_vp, _i, ctypes.POINTER(_pd)]),
    "taps_factors_get": (_i, [_vp, ctypes.POINTER(_pd)]),
    "taps_factors_M": (_i, [_vp]),
    "taps_factors_device_ptr": (_vp, [_vp, _i]),
    "taps_factors_destroy": (None, [_vp]),
    "taps_sweep": (_i, [_vp, _vp, _i, ctypes.POINTER(SweepOpts), ctypes.POINTER(SweepReport)]),
    "taps_residual": (_i, [_vp, _vp, _i, _pd]),
    "taps_solve": (_i, [_vp, _vp, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveReport)]),
    "taps_eval_grid": (_i, [_vp, _vp, _pi, _pi, _pi, _vp, _i]),
    "taps_eval_points": (_i, [_vp, _vp, _i, _vp, _vp]),
    "taps_eval_grid_noalloc": (_i, [_vp, _vp, _pi, _pi, _pi, _vp, _i]),
    "taps_profile_reset": (_i, [_vp, _i]),
    "taps_batch_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _i, _i, ctypes.POINTER(_vp)]),
    "taps_batch_sweep": (_i, [_vp, _i, _i, _pd, _pi]),
    "taps_batch_info": (_i, [_vp, _pi, ctypes.POINTER(ctypes.c_float)]),
    "taps_batch_refresh_grams": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_float), _pd]),
    "taps_batch_gram_info": (_i, [_vp, _pi, _pi, ctypes.POINTER(ctypes.c_float)]),
    "taps_problem_refresh_grams": (_i, [_vp, _vp, _i]),
    "taps_problem_copy_grams": (_i, [_vp, _i, _i, _pd, _pd, _pi, _pi]),
    "taps_util_barrier_test": (_i, [_i, _i, ctypes.c_longlong, _vp]),
    "taps_batch_destroy": (None, [_vp]),
    "taps_mlp_create": (_i, [_i, _i, _i, _i, ctypes.c_uint, _vp, ctypes.POINTER(_vp)]),
    "taps_mlp_num_params": (ctypes.c_longlong, [_vp]),
    "taps_mlp_get_params": (_i, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_longlong]),
    "taps_mlp_set_params": (_i, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_longlong]),
    "taps_mlp_forward": (_i, [_vp, _vp, _i, _vp]),
    "taps_mlp_grad": (_i, [_vp, _vp, _vp, _i, ctypes.POINTER(ctypes.c_float),
                           ctypes.POINTER(ctypes.c_float)]),
    "taps_mlp_adam": (_i, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    "taps_mlp_train": (_i, [_vp, _vp, _vp, _i, _i, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]),
    "taps_mlp_destroy": (None, [_vp]),
    "taps_factors_from_profiles": (_i, [_vp, _vp, _i, _vp, _i, _d]),
    "taps_profile_get": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_longlong), _pd, _pd, _pd]),
    "taps_util_rcp": (_i, [_vp, _vp, ctypes.c_longlong, _vp]),
    "taps_util_md_pencil": (_i, [_vp, _vp, _i, _vp, _vp, _pi, _vp]),
}

PROF_CLASSES = ["gram", "coeff", "block_assemble", "block_lu", "backsub", "normalize",
                "residual", "eval", "other", "fastdiag", "fd_transform", "modediag"]

_LIB = None


def lib():
    """Load libtaps.so (raises if it has not been built: no fallback exists)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2503_13933_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class TapsError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().taps_status_string(status).decode()
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


def check(status, where):
    if status != OK:
        raise TapsError(status, where)
    return status


def current_stream():
    import torch
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def rcp(x, y):
    """y = 1 / x with the small solves' reciprocal (x, y: CUDA float64 tensors)."""
    check(lib().taps_util_rcp(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                              x.numel(), current_stream()), "taps_util_rcp")


def md_pencil(CX, CY, W, lam):
    """The mode-side eigen-solve on one pencil (taps_util_md_pencil): CX, CY (CY may be
    None), W CUDA float64 M x M tensors, lam CUDA float64 [M]; returns 1 if the FP64
    corrections were accepted, 0 if the FP64 rotation pass ran."""
    ref = ctypes.c_int()
    cy = ctypes.c_void_p(CY.data_ptr()) if CY is not None else ctypes.c_void_p(0)
    check(lib().taps_util_md_pencil(ctypes.c_void_p(CX.data_ptr()), cy, CX.shape[0], ctypes.c_void_p(W.data_ptr()),
                                    ctypes.c_void_p(lam.data_ptr()), ctypes.byref(ref), current_stream()),
          "taps_util_md_pencil")
    return ref.value


def dim_desc(dm):
    w = (ctypes.c_double * 4)(*[float(c) for c in dm["weight_poly"]][:4])
    return DimDesc(kind=dm["kind"], n=dm["n"], lo=dm["lo"], hi=dm["hi"], s=dm["s"], a=dm["a"],
                   p=dm["p"], n_quad=dm["n_quad"], dirichlet_lo=int(dm["dirichlet_lo"]),
                   dirichlet_hi=int(dm["dirichlet_hi"]), weight_poly=w)


class Dim:
    """An assembled dimension (taps_assemble_1d)."""

    def __init__(self, dm, stream=None):
        self.desc = dm
        self.stream = stream if stream is not None else current_stream()
        h = ctypes.c_void_p()
        d = dim_desc(dm)
        check(lib().taps_assemble_1d(ctypes.byref(d), self.stream, ctypes.byref(h)),
              "taps_assemble_1d")
        self.handle = h
        a, f, hb = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().taps_dim_info(h, ctypes.byref(a), ctypes.byref(f), ctypes.byref(hb)),
              "taps_dim_info")
        self.n_all, self.n_free, self.hb = a.value, f.value, hb.value

    def band(self, op):
        out = np.zeros((self.n_free, 2 * self.hb + 1))
        check(lib().taps_dim_copy_band(self.handle, OP[op] if isinstance(op, str) else op,
                                       out.ctypes.data_as(_pd)), "taps_dim_copy_band")
        return out

    def shape_tables(self):
        s, nq = self.desc["s"], self.desc["n_quad"]
        N = np.zeros((self.n_all - 1, nq, 2 * s + 2))
        B = np.zeros_like(N)
        X = np.zeros((self.n_all - 1, nq))
        check(lib().taps_dim_copy_shape(self.handle, N.ctypes.data_as(_pd), B.ctypes.data_as(_pd),
                                        X.ctypes.data_as(_pd)), "taps_dim_copy_shape")
        return N, B, X

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.taps_dim_destroy(self.handle)
            self.handle = None


class Problem:
    """A separated problem (taps_problem_create) built from a workload description."""

    def __init__(self, desc, stream=None, dim_cache=None):
        """dim_cache: an optional dict shared by problems on the same stream (slabs of a
        chain, their compression problems): identical dimension descriptions then share
        one assembled dimension and its cached pencil decompositions across problems."""
        self.desc = desc
        self.stream = stream if stream is not None else current_stream()
        # identical dimension descriptions share one assembled dimension (and its
        # cached pencil decomposition)
        uniq = dim_cache if dim_cache is not None else {}
        self.dims = []
        for dm in desc["dims"]:
            key = tuple(sorted((k, tuple(v) if isinstance(v, (list, tuple)) else v)
                               for k, v in dm.items()))
            if key not in uniq:
                uniq[key] = Dim(dm, self.stream)
            self.dims.append(uniq[key])
        D = len(self.dims)
        self.D = D
        terms = (Term * len(desc["terms"]))()
        for t, (alpha, ops) in enumerate(desc["terms"]):
            terms[t].alpha = float(alpha)
            for d, o in enumerate(ops):
                terms[t].op[d] = op_code(o)
        srcs = (Source * len(desc["sources"]))()
        self._keep = []
        for r, (beta, facs) in enumerate(desc["sources"]):
            srcs[r].beta = float(beta)
            for d, (kind, par) in enumerate(facs):
                srcs[r].kind[d] = SRC[kind]
                if kind == "nodal":
                    arr = np.ascontiguousarray(par, dtype=np.float64)
                    self._keep.append(arr)
                    srcs[r].nodal[d] = arr.ctypes.data_as(_pd)
                elif kind in ("opvec", "opvecfull"):   # (operator name, free- / all-node vector)
                    arr = np.ascontiguousarray(par[1], dtype=np.float64)
                    self._keep.append(arr)
                    srcs[r].nodal[d] = arr.ctypes.data_as(_pd)
                    srcs[r].par[d][0] = float(OP[par[0]])
                else:
                    vals = [float(v) for v in par] + [0.0] * (4 - len(par))
                    for j in range(4):
                        srcs[r].par[d][j] = vals[j]
        handles = (ctypes.c_void_p * D)(*[dm.handle.value for dm in self.dims])
        h = ctypes.c_void_p()
        check(lib().taps_problem_create(handles, D, terms, len(desc["terms"]), srcs,
                                        len(desc["sources"]), self.stream, ctypes.byref(h)),
              "taps_problem_create")
        self.handle = h
        self.n_free = [dm.n_free for dm in self.dims]
        for d, wl in enumerate(desc.get("weighted") or []):
            if wl:
                self.set_weighted(d, wl)

    def set_weighted(self, d, ops):
        """Define / update dim d's weighted operators: ops[j] = (base 'K'|'M'|'G',
        nodal weights at all nodes) is operator 'w<j>' (taps_problem_set_weighted_ops)."""
        base = (ctypes.c_int * len(ops))(*[OP[b] for b, _ in ops])
        w = np.ascontiguousarray(np.stack([np.asarray(v, dtype=np.float64) for _, v in ops]))
        check(lib().taps_problem_set_weighted_ops(self.handle, int(d), len(ops), base, w.ctypes.data_as(_pd)),
              "taps_problem_set_weighted_ops")

    def op_band(self, d, op):
        """The band [n_free][2 hb + 1] of operator `op` ('K', ..., 'w<j>') of dim d."""
        out = np.zeros((self.n_free[d], 2 * self.dims[d].hb + 1))
        check(lib().taps_problem_copy_op(self.handle, int(d), op_code(op), out.ctypes.data_as(_pd)),
              "taps_problem_copy_op")
        return out

    def source(self, r, d):
        out = np.zeros(self.n_free[d])
        check(lib().taps_problem_copy_source(self.handle, r, d, out.ctypes.data_as(_pd)),
              "taps_problem_copy_source")
        return out

    def factors(self, M_cap):
        return Factors(self, M_cap)

    def refresh_grams(self, U, precision=FP64):
        """Recompute every dim's Grams from U at `precision` (taps_problem_refresh_grams)."""
        check(lib().taps_problem_refresh_grams(self.handle, U.handle, precision), "taps_problem_refresh_grams")

    def grams(self, d, M):
        """(Gamma [nops][M][M], h [R_f][M], op codes) of dim d (taps_problem_copy_grams)."""
        nops = ctypes.c_int()
        ops = (ctypes.c_int * 64)()
        check(lib().taps_problem_copy_grams(self.handle, d, M, None, None, ops, ctypes.byref(nops)),
              "taps_problem_copy_grams")
        g = np.zeros((nops.value, M, M))
        h = np.zeros((len(self.desc["sources"]), M))
        check(lib().taps_problem_copy_grams(self.handle, d, M, g.ctypes.data_as(_pd), h.ctypes.data_as(_pd),
                                            None, None), "taps_problem_copy_grams")
        return g, h, [ops[k] for k in range(nops.value)]

    def sweep(self, U, n=1, precision=FP64, normalize=True, solver=SOLVER_BLOCK_LU):
        """Run n sweeps (Algorithm 1 inner loop)."""
        o = SweepOpts(precision=precision, solver=solver, normalize=int(normalize))
        rep = SweepReport()
        check(lib().taps_sweep(self.handle, U.handle, n, ctypes.byref(o), ctypes.byref(rep)),
              "taps_sweep")
        return dict(sweeps=rep.sweeps, change=rep.change, seconds=rep.seconds)

    def residual(self, U, kind=RES_ALS):
        v = ctypes.c_double()
        check(lib().taps_residual(self.handle, U.handle, kind, ctypes.byref(v)), "taps_residual")
        return v.value

    def solve(self, U, M0=1, M_max=8, als_tol=1e-10, res_tol=1e-6, res_kind=RES_ALS,
              max_sweeps=200, precision=FP64, polish_sweeps=20, init=INIT_ZERO, seed=0,
              history_cap=4096, raise_not_converged=False, solver=SOLVER_BLOCK_LU, graphs=True,
              res_stall=0.0, M_step=1):
        o = SolveOpts(M0=M0, M_max=M_max, als_tol=als_tol, res_tol=res_tol, res_kind=res_kind,
                      max_sweeps=max_sweeps, precision=precision, polish_sweeps=polish_sweeps,
                      solver=solver, init=init, seed=seed, history_cap=history_cap,
                      graphs=int(graphs), res_stall=res_stall, M_step=M_step)
        hM = (ctypes.c_int * max(history_cap, 1))()
        hc = (ctypes.c_double * max(history_cap, 1))()
        hr = (ctypes.c_double * max(history_cap, 1))()
        rep = SolveReport(hist_M=hM, hist_change=hc, hist_rho=hr)
        st = lib().taps_solve(self.handle, U.handle, ctypes.byref(o), ctypes.byref(rep))
        if st != OK and (st != ERR_NOT_CONVERGED or raise_not_converged):
            check(st, "taps_solve")
        n = rep.hist_len
        return dict(status=st, M=rep.M, sweeps=rep.sweeps, fp64_sweeps=rep.fp64_sweeps,
                    rho=rep.rho, rho_full=rep.rho_full, change=rep.change, seconds=rep.seconds,
                    converged=bool(rep.converged),
                    history=[(hM[i], hc[i], hr[i]) for i in range(n)])

    def eval_grid(self, U, start, count, step, out, dtype=FP32):
        """out: a CUDA tensor of prod(count) elements (float32 or float64)."""
        D = self.D
        a = (ctypes.c_int * D)(*start)
        c = (ctypes.c_int * D)(*count)
        s = (ctypes.c_int * D)(*step)
        check(lib().taps_eval_grid(self.handle, U.handle, a, c, s, ctypes.c_void_p(out.data_ptr()),
                                   dtype), "taps_eval_grid")
        return out

    def eval_grid_noalloc(self, U, start, count, step, out, dtype=FP32):
        """Allocation-free reconstruction (fixed library scratch; see include/taps.h)."""
        D = self.D
        a = (ctypes.c_int * D)(*start)
        c = (ctypes.c_int * D)(*count)
        s = (ctypes.c_int * D)(*step)
        check(lib().taps_eval_grid_noalloc(self.handle, U.handle, a, c, s,
                                           ctypes.c_void_p(out.data_ptr()), dtype),
              "taps_eval_grid_noalloc")
        return out

    def eval_points(self, U, pts, out):
        """pts: CUDA float64 tensor [n, D]; out: CUDA float64 tensor [n]."""
        check(lib().taps_eval_points(self.handle, U.handle, int(pts.shape[0]),
                                     ctypes.c_void_p(pts.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr())), "taps_eval_points")
        return out

    def profile_reset(self, events=True):
        check(lib().taps_profile_reset(self.handle, int(events)), "taps_profile_reset")

    def profile(self):
        """{class: dict(launches, ms, flops, bytes)} accumulated since profile_reset."""
        out = {}
        for c, name in enumerate(PROF_CLASSES):
            n = ctypes.c_longlong()
            ms, fl, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            check(lib().taps_profile_get(self.handle, c, ctypes.byref(n), ctypes.byref(ms),
                                         ctypes.byref(fl), ctypes.byref(by)), "taps_profile_get")
            out[name] = dict(launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value)
        return out

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.taps_problem_destroy(self.handle)
            self.handle = None


class Batch:
    """Independent instances swept together (taps_batch_*)."""

    def __init__(self, problems, factors, precision=FP64, solver=SOLVER_FASTDIAG):
        self.problems, self.factors = list(problems), list(factors)
        n = len(self.problems)
        ph = (ctypes.c_void_p * n)(*[p.handle.value for p in self.problems])
        uh = (ctypes.c_void_p * n)(*[u.handle.value for u in self.factors])
        h = ctypes.c_void_p()
        check(lib().taps_batch_create(ph, uh, n, precision, solver, ctypes.byref(h)), "taps_batch_create")
        self.handle = h

    def sweep(self, n_sweeps, graphs=True, statuses=False):
        """Returns each instance's last factor change; with statuses=True also each
        instance's status (the batch then runs to the end whatever the instances'
        numerical errors)."""
        ch = np.zeros(len(self.problems))
        st = np.zeros(len(self.problems), dtype=np.int32) if statuses else None
        check(lib().taps_batch_sweep(self.handle, n_sweeps, int(graphs), ch.ctypes.data_as(_pd),
                                     st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if statuses else None),
              "taps_batch_sweep")
        return (ch, st) if statuses else ch

    def info(self):
        """(solver used by the sweeps, [trial ms FASTDIAG, MODEDIAG] of the AUTO tuner)."""
        sv = ctypes.c_int()
        ms = (ctypes.c_float * 2)()
        check(lib().taps_batch_info(self.handle, ctypes.byref(sv), ms), "taps_batch_info")
        return sv.value, [ms[0], ms[1]]

    def refresh_grams(self, precision=BF16):
        """Every instance's Grams from its current factors (taps_batch_refresh_grams);
        returns (device ms, algorithmic bytes)."""
        ms = ctypes.c_float()
        by = ctypes.c_double()
        check(lib().taps_batch_refresh_grams(self.handle, precision, ctypes.byref(ms), ctypes.byref(by)),
              "taps_batch_refresh_grams")
        return ms.value, by.value

    GRAM_TILES = [(64, 1), (64, 2), (64, 3), (64, 4), (128, 1), (128, 2)]

    def gram_info(self):
        """(chunk rows, CTAs per SM, trial ms of each (rows, CTAs per SM) in GRAM_TILES)."""
        r, c = ctypes.c_int(), ctypes.c_int()
        t = (ctypes.c_float * 6)()
        check(lib().taps_batch_gram_info(self.handle, ctypes.byref(r), ctypes.byref(c), t), "taps_batch_gram_info")
        return r.value, c.value, [t[k] for k in range(6)]

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.taps_batch_destroy(self.handle)
            self.handle = None


class MLP:
    """The warm-start network (taps_mlp_*): FP32, tanh hidden layers, linear output."""

    def __init__(self, n_in, n_hidden, hidden_layers, n_out, seed=0, stream=None):
        self.stream = stream if stream is not None else current_stream()
        h = ctypes.c_void_p()
        check(lib().taps_mlp_create(n_in, n_hidden, hidden_layers, n_out, seed, self.stream,
                                    ctypes.byref(h)), "taps_mlp_create")
        self.handle = h
        self.n_in, self.n_out = n_in, n_out
        self.nparams = lib().taps_mlp_num_params(h)

    def params(self):
        out = np.zeros(self.nparams, dtype=np.float32)
        check(lib().taps_mlp_get_params(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        self.nparams), "taps_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        check(lib().taps_mlp_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                        self.nparams), "taps_mlp_set_params")

    def forward(self, x, y):
        """x, y: CUDA float32 tensors [batch, n_in], [batch, n_out]."""
        check(lib().taps_mlp_forward(self.handle, ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                     ctypes.c_void_p(y.data_ptr())), "taps_mlp_forward")
        return y

    def grad(self, x, t, want_grad=True):
        loss = ctypes.c_float()
        g = np.zeros(self.nparams, dtype=np.float32) if want_grad else None
        check(lib().taps_mlp_grad(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                  int(x.shape[0]), ctypes.byref(loss),
                                  g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) if want_grad else None),
              "taps_mlp_grad")
        return loss.value, g

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        check(lib().taps_mlp_adam(self.handle, lr, b1, b2, eps), "taps_mlp_adam")

    def train(self, x, t, steps, lr=1e-3):
        loss = ctypes.c_float()
        check(lib().taps_mlp_train(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                   int(x.shape[0]), steps, lr, ctypes.byref(loss)), "taps_mlp_train")
        return loss.value

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.taps_mlp_destroy(self.handle)
            self.handle = None


class Factors:
    """CP factor matrices U_d (n_free x M, column-major on the device)."""

    def __init__(self, prob, M_cap):
        self.prob = prob
        h = ctypes.c_void_p()
        check(lib().taps_factors_create(prob.handle, M_cap, ctypes.byref(h)), "taps_factors_create")
        self.handle = h
        self.M_cap = M_cap

    @property
    def M(self):
        return lib().taps_factors_M(self.handle)

    def set(self, Us):
        M = Us[0].shape[1]
        cols = [np.asfortranarray(u, dtype=np.float64) for u in Us]
        ptrs = (_pd * len(cols))(*[c.ctypes.data_as(_pd) for c in cols])
        check(lib().taps_factors_set(self.handle, M, ptrs), "taps_factors_set")

    def from_profiles(self, prof, M, n_ref, weight_scale=1.0):
        """Initial factors from predicted profiles (CUDA float32 [M, D*n_ref + 1])."""
        check(lib().taps_factors_from_profiles(self.prob.handle, self.handle, M,
                                               ctypes.c_void_p(prof.data_ptr()), n_ref,
                                               float(weight_scale)),
              "taps_factors_from_profiles")

    def copy_from(self, other):
        """These factors := other's (same problem; a device copy)."""
        check(lib().taps_factors_copy(self.handle, other.handle), "taps_factors_copy")

    def rel_change(self, other):
        """|u_self - u_other| / |u_self| of the CP tensors, on the device."""
        out = ctypes.c_double()
        check(lib().taps_factors_rel_change(self.handle, other.handle, ctypes.byref(out)),
              "taps_factors_rel_change")
        return out.value

    def get(self):
        M = self.M
        outs = [np.zeros((n, M), order="F") for n in self.prob.n_free]
        ptrs = (_pd * len(outs))(*[o.ctypes.data_as(_pd) for o in outs])
        check(lib().taps_factors_get(self.handle, ptrs), "taps_factors_get")
        return [np.ascontiguousarray(o) for o in outs]

    def __del__(self):
        if getattr(self, "handle", None) and _LIB is not None:
            _LIB.taps_factors_destroy(self.handle)
            self.handle = None


def barrier_test(ctas, missing, poll_limit, stream=None):
    """Status of the library's bounded grid barrier test (taps_util_barrier_test):
    OK with every CTA present, ERR_TIMEOUT with `missing` CTAs that never arrive."""
    return lib().taps_util_barrier_test(ctas, missing, poll_limit,
                                        stream if stream is not None else current_stream())
