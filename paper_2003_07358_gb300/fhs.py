"""Thin Python binding of the libfhs C ABI (include/fhs.h).

Argument marshalling only: every operator runs in the CUDA kernels of
libfhs.so.  Device arrays are torch tensors (float32 / complex64, contiguous,
on the context's device); PyTorch provides memory and streams, nothing else.
If libfhs.so is missing or cannot be loaded, every call raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfhs.so")

FHS_WIN = {"triangular": 0, "sine": 1}
_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "TIMEOUT", 5: "NONFINITE", 6: "UNSUPPORTED"}

SYMBOLS = [
    "fhs_create", "fhs_destroy", "fhs_get_sizes", "fhs_sync", "fhs_last_error", "fhs_vis_permutation",
    "fhs_vis_to_internal", "fhs_vis_to_user", "fhs_measure", "fhs_adjoint", "fhs_opnorm_sq",
    "fhs_sara_analysis", "fhs_sara_synthesis", "fhs_prox_l21_sara_facets", "fhs_prox_nuclear_facets",
    "fhs_proj_l2ball_blocks", "fhs_reweight", "fhs_pdfb_iter", "fhs_set_params", "fhs_kernel_launches",
    "fhs_proj_l2ball_noalloc", "fhs_noalloc_last_error", "fhs_set_path", "fhs_set_kernel_timer",
    "fhs_kernel_timer_read", "fhs_solve", "fhs_heuristic_params", "fhs_set_preconditioning",
    "fhs_pdfb_iter_host", "fhs_set_wait_limit", "fhs_set_alloc_limit",
    "fhs_checkpoint_save", "fhs_checkpoint_load", "fhs_set_dde", "fhs_set_autotune", "fhs_get_tuning",
    "fhs_set_lanes", "fhs_get_lanes",
]
MAX_SOLVE_CYCLES = 32
FHS_PATH = {"fast": 0, "plain": 1}
FHS_TIMER = {None: 0, "grid": 1, "degrid": 2}


class FhsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libfhs {_STATUS.get(status, status)}: {msg}")
        self.status = status


class fhs_cube_desc(C.Structure):
    _fields_ = [("n1", C.c_int32), ("n2", C.c_int32), ("L", C.c_int32), ("Qy", C.c_int32), ("Qx", C.c_int32),
                ("overlap", C.c_double), ("window", C.c_int32), ("B", C.c_int32),
                ("M", C.POINTER(C.c_int64)), ("uv", C.POINTER(C.c_float)),
                ("tau", C.c_double), ("zeta", C.c_double), ("kappa", C.c_double),
                ("eta", C.POINTER(C.c_double)), ("mu", C.c_double),
                ("mu_bar", C.POINTER(C.c_double)), ("eps", C.POINTER(C.c_double))]


class fhs_sizes(C.Structure):
    _fields_ = [("n_pix", C.c_int64), ("n_vis", C.c_int64), ("n_coef", C.c_int64), ("n_facet_pix", C.c_int64),
                ("n_facets", C.c_int32), ("n_blocks", C.c_int32)]


class fhs_state(C.Structure):
    _fields_ = [("W", C.c_void_p), ("theta", C.c_void_p), ("P", C.c_void_p), ("theta_bar", C.c_void_p),
                ("v", C.c_void_p), ("u_prev", C.c_void_p)]


class fhs_iterate(C.Structure):
    _fields_ = [("X", C.c_void_p), ("Xcheck", C.c_void_p), ("y", C.c_void_p), ("state", fhs_state)]


class fhs_iter_stats(C.Structure):
    _fields_ = [("xi", C.c_double), ("res_norm", C.c_double), ("eps_norm", C.c_double)]


class fhs_solve_params(C.Structure):
    _fields_ = [("p_min", C.c_int32), ("p_max", C.c_int32), ("xi_pdfb", C.c_double), ("res_factor", C.c_double),
                ("t_max", C.c_int32), ("xi_reweight", C.c_double)]


class fhs_solve_report(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("iterations", C.c_int32),
                ("iterations_per_cycle", C.c_int32 * MAX_SOLVE_CYCLES), ("xi", C.c_double),
                ("res_norm", C.c_double), ("xi_reweight", C.c_double), ("nonfinite", C.c_int32)]


class fhs_tuning(C.Structure):
    _fields_ = [("grid_tile", C.c_int32), ("degrid_tiled", C.c_int32), ("gram_tc", C.c_int32),
                ("sara_fast", C.c_int32), ("prox_ctas_per_sm", C.c_int32), ("source", C.c_int32),
                ("ms", C.c_double * 10)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfhs.so and declare its signatures (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FhsError(2, f"{path} not found: build it with __graft_entry__.build() (CUDA toolkit required)")
    lib = C.CDLL(path)
    vp, i32, i64p, dp = C.c_void_p, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_double)
    sig = {
        "fhs_create": ([C.POINTER(fhs_cube_desc), i32, vp, C.POINTER(vp)], i32),
        "fhs_destroy": ([vp], i32),
        "fhs_get_sizes": ([vp, i32, C.POINTER(fhs_sizes)], i32),
        "fhs_sync": ([vp], i32),
        "fhs_last_error": ([vp], C.c_char_p),
        "fhs_vis_permutation": ([vp, i32, i64p], i32),
        "fhs_vis_to_internal": ([vp, i32, vp, vp], i32),
        "fhs_vis_to_user": ([vp, i32, vp, vp], i32),
        "fhs_measure": ([vp, i32, vp, vp], i32),
        "fhs_adjoint": ([vp, i32, vp, vp], i32),
        "fhs_opnorm_sq": ([vp, i32, i32, C.c_double, dp], i32),
        "fhs_sara_analysis": ([vp, i32, vp, vp], i32),
        "fhs_sara_synthesis": ([vp, i32, vp, vp], i32),
        "fhs_prox_l21_sara_facets": ([vp, i32, vp, vp, vp, vp], i32),
        "fhs_prox_nuclear_facets": ([vp, i32, vp, vp, vp, vp], i32),
        "fhs_proj_l2ball_blocks": ([vp, i32, vp, vp, vp, dp], i32),
        "fhs_reweight": ([vp, i32, vp, vp, vp], i32),
        "fhs_pdfb_iter": ([vp, C.POINTER(fhs_iterate), i32, C.POINTER(fhs_iter_stats)], i32),
        "fhs_set_params": ([vp, i32, C.c_double, C.c_double, C.c_double, dp, C.c_double, dp, dp], i32),
        "fhs_kernel_launches": ([], C.c_uint64),
        "fhs_proj_l2ball_noalloc": ([vp, vp, i64p, i32, dp, vp, dp, vp], i32),
        "fhs_noalloc_last_error": ([], C.c_char_p),
        "fhs_set_path": ([vp, i32], i32),
        "fhs_set_kernel_timer": ([vp, i32], i32),
        "fhs_kernel_timer_read": ([vp, C.POINTER(C.c_double), C.POINTER(i32)], i32),
        "fhs_solve": ([vp, C.POINTER(fhs_iterate), C.POINTER(fhs_solve_params), C.POINTER(fhs_solve_report)], i32),
        "fhs_heuristic_params": ([vp, i32, dp, i32, C.c_double, dp, dp, dp, dp], i32),
        "fhs_set_preconditioning": ([vp, i32, i32, C.POINTER(C.c_float)], i32),
        "fhs_set_wait_limit": ([C.c_int64], i32),
        "fhs_checkpoint_save": ([vp, C.POINTER(fhs_iterate), C.c_char_p], i32),
        "fhs_checkpoint_load": ([vp, C.POINTER(fhs_iterate), C.c_char_p], i32),
        "fhs_set_alloc_limit": ([C.c_uint64], i32),
        "fhs_set_dde": ([vp, i32, i32, i32, C.POINTER(C.c_float), C.POINTER(C.c_int32)], i32),
        "fhs_set_autotune": ([i32, C.c_char_p], i32),
        "fhs_get_tuning": ([vp, i32, C.POINTER(fhs_tuning)], i32),
        "fhs_set_lanes": ([vp, i32], i32),
        "fhs_get_lanes": ([vp, C.POINTER(i32)], i32),
        "fhs_pdfb_iter_host": ([vp, C.POINTER(fhs_iterate), C.POINTER(vp), C.POINTER(vp), i32,
                                C.POINTER(fhs_iter_stats)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("libfhs takes contiguous CUDA tensors")
    return t.data_ptr()


def fhs_set_wait_limit(spins: int) -> None:
    """Fault-injection hook: first phase of the bounded device-side waits (0: default)."""
    rc = load().fhs_set_wait_limit(spins)
    if rc != 0:
        raise FhsError(rc, "fhs_set_wait_limit")


def fhs_set_alloc_limit(nbytes: int) -> None:
    """Fault-injection hook: cap on the device bytes one context may allocate (0: none)."""
    rc = load().fhs_set_alloc_limit(nbytes)
    if rc != 0:
        raise FhsError(rc, "fhs_set_alloc_limit")


def fhs_set_autotune(mode: int, cache_path: str | None = None) -> None:
    """Autotuning of the contexts created afterwards: 0 defaults, 1 cache then measure,
    2 always measure; cache_path a JSON file (or None)."""
    rc = load().fhs_set_autotune(mode, cache_path.encode() if cache_path else None)
    if rc != 0:
        raise FhsError(rc, "fhs_set_autotune")


def _host_ptr(a, dtype) -> int:
    """Address of a contiguous host array (torch CPU tensor or numpy array) of `dtype`."""
    if hasattr(a, "is_cuda"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("host buffers must be contiguous CPU tensors")
        if str(a.dtype).replace("torch.", "") != np.dtype(dtype).name:
            raise ValueError(f"host buffer must be {np.dtype(dtype).name}")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
        raise ValueError(f"host buffers must be contiguous {np.dtype(dtype).name} arrays")
    return a.ctypes.data


def _check_noalloc_args(z, y, seg_off: np.ndarray, eps: np.ndarray, v_out) -> None:
    """Checks the C side cannot make (it has no lengths): raises ValueError before any
    device work, so a wrong offset array can never read or write out of bounds."""
    if seg_off.ndim != 1 or seg_off.size < 2:
        raise ValueError("seg_off must be a 1-D array of nseg + 1 offsets")
    if eps.shape != (seg_off.size - 1,):
        raise ValueError(f"eps must have nseg = {seg_off.size - 1} entries, got shape {eps.shape}")
    if seg_off[0] < 0 or np.any(np.diff(seg_off) < 0):
        raise ValueError("seg_off must start at >= 0 and be non-decreasing")
    need = int(seg_off[-1])
    for name, t in (("z", z), ("y", y), ("v_out", v_out)):
        if t is None or not hasattr(t, "dtype"):
            raise ValueError(f"{name} must be a tensor")
        if str(t.dtype) != "torch.complex64":
            raise ValueError(f"{name} must be complex64, got {t.dtype}")
        if t.numel() < need:
            raise ValueError(f"{name} has {t.numel()} elements, the segments need {need}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if not (z.is_cuda and y.is_cuda and v_out.is_cuda):
        raise ValueError("z, y and v_out must be CUDA tensors")
    if not (z.device == y.device == v_out.device):
        raise ValueError("z, y and v_out must be on the same device")


def fhs_proj_l2ball_noalloc(z, y, seg_off, eps, v_out, want_norms: bool = True, stream=None):
    """Allocation-free l2-ball projection on plain arrays (no context): segment s
    of the caller's order gets v = (z - y)(1 - min(1, eps_s / ||z_s - y_s||)).
    For callers that may not allocate device memory; see include/fhs.h."""
    so = np.ascontiguousarray(seg_off, dtype=np.int64)
    ep = np.ascontiguousarray(eps, dtype=np.float64)
    _check_noalloc_args(z, y, so, ep, v_out)
    import torch
    lib = load()
    out = np.zeros(so.size - 1, dtype=np.float64) if want_norms else None
    st = stream if stream is not None else torch.cuda.current_stream(z.device)
    P = C.POINTER(C.c_double)
    with torch.cuda.device(z.device):    # the C side works on the current device
        rc = lib.fhs_proj_l2ball_noalloc(_ptr(z), _ptr(y), so.ctypes.data_as(C.POINTER(C.c_int64)), so.size - 1,
                                         ep.ctypes.data_as(P), _ptr(v_out),
                                         out.ctypes.data_as(P) if want_norms else None, C.c_void_p(st.cuda_stream))
    if rc != 0:
        raise FhsError(rc, lib.fhs_noalloc_last_error().decode())
    return out


@dataclass
class CubeParams:
    """One spectral sub-cube for fhs_create (host arrays, float64 parameters)."""
    n1: int
    n2: int
    L: int
    Qy: int
    Qx: int
    overlap: float
    window: str
    M_lb: np.ndarray          # [L][B] int64
    uv: np.ndarray            # [sum M][2] float32, channel-major, block-contiguous
    eta: np.ndarray           # [L]
    mu: float
    mu_bar: np.ndarray        # [Qy*Qx]
    eps: np.ndarray           # [L][B]
    tau: float = 0.33
    zeta: float = 1.0
    kappa: float = 1.0


class Context:
    """Owns an fhs_ctx; methods mirror the C-ABI calls one to one."""

    def __init__(self, cubes: list[CubeParams], stream=None):
        import torch
        self.lib = load()
        self._keep = []
        descs = (fhs_cube_desc * len(cubes))()
        for d, cp in zip(descs, cubes):
            M = np.ascontiguousarray(cp.M_lb, dtype=np.int64).ravel()
            uv = np.ascontiguousarray(cp.uv, dtype=np.float32).ravel()
            eta = np.ascontiguousarray(cp.eta, dtype=np.float64).ravel()
            mub = np.ascontiguousarray(cp.mu_bar, dtype=np.float64).ravel()
            eps = np.ascontiguousarray(cp.eps, dtype=np.float64).ravel()
            self._keep += [M, uv, eta, mub, eps]
            d.n1, d.n2, d.L, d.Qy, d.Qx = cp.n1, cp.n2, cp.L, cp.Qy, cp.Qx
            d.overlap, d.window, d.B = cp.overlap, FHS_WIN[cp.window], int(np.asarray(cp.M_lb).shape[1])
            d.M = M.ctypes.data_as(C.POINTER(C.c_int64))
            d.uv = uv.ctypes.data_as(C.POINTER(C.c_float))
            d.tau, d.zeta, d.kappa, d.mu = cp.tau, cp.zeta, cp.kappa, cp.mu
            d.eta = eta.ctypes.data_as(C.POINTER(C.c_double))
            d.mu_bar = mub.ctypes.data_as(C.POINTER(C.c_double))
            d.eps = eps.ctypes.data_as(C.POINTER(C.c_double))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        h = C.c_void_p()
        st = self.lib.fhs_create(descs, len(cubes), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise FhsError(st, self.lib.fhs_last_error(None).decode())
        self.h = h
        self.cubes = cubes
        self._keep = []

    # ---------------------------------------------------------------- utils
    def _check(self, st):
        if st != 0:
            raise FhsError(st, self.lib.fhs_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.fhs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self, cube: int = 0) -> dict:
        s = fhs_sizes()
        self._check(self.lib.fhs_get_sizes(self.h, cube, C.byref(s)))
        return {k: getattr(s, k) for k, _ in fhs_sizes._fields_}

    def sync(self):
        self._check(self.lib.fhs_sync(self.h))

    def fhs_vis_permutation(self, cube: int = 0) -> np.ndarray:
        n = self.sizes(cube)["n_vis"]
        out = np.zeros(n, dtype=np.int64)
        self._check(self.lib.fhs_vis_permutation(self.h, cube, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return out

    def fhs_vis_to_internal(self, cube, user, internal):
        self._check(self.lib.fhs_vis_to_internal(self.h, cube, _ptr(user), _ptr(internal)))

    def fhs_vis_to_user(self, cube, internal, user):
        self._check(self.lib.fhs_vis_to_user(self.h, cube, _ptr(internal), _ptr(user)))

    # ------------------------------------------------------------ operators
    def fhs_measure(self, cube, x, y):
        self._check(self.lib.fhs_measure(self.h, cube, _ptr(x), _ptr(y)))

    def fhs_adjoint(self, cube, v, x):
        self._check(self.lib.fhs_adjoint(self.h, cube, _ptr(v), _ptr(x)))

    def fhs_opnorm_sq(self, cube, max_iter=100, rel_tol=1e-4) -> np.ndarray:
        L = self.cubes[cube].L
        out = np.zeros(L, dtype=np.float64)
        self._check(self.lib.fhs_opnorm_sq(self.h, cube, max_iter, rel_tol,
                                           out.ctypes.data_as(C.POINTER(C.c_double))))
        return out

    def fhs_sara_analysis(self, cube, x, coef):
        self._check(self.lib.fhs_sara_analysis(self.h, cube, _ptr(x), _ptr(coef)))

    def fhs_sara_synthesis(self, cube, coef, x):
        self._check(self.lib.fhs_sara_synthesis(self.h, cube, _ptr(coef), _ptr(x)))

    def fhs_prox_l21_sara_facets(self, cube, xcheck, W, theta, A):
        self._check(self.lib.fhs_prox_l21_sara_facets(self.h, cube, _ptr(xcheck), _ptr(W), _ptr(theta), _ptr(A)))

    def fhs_prox_nuclear_facets(self, cube, xcheck, P, theta_bar, A):
        self._check(self.lib.fhs_prox_nuclear_facets(self.h, cube, _ptr(xcheck), _ptr(P), _ptr(theta_bar), _ptr(A)))

    def fhs_proj_l2ball_blocks(self, cube, z, y, v_out, want_norms=True):
        nb = self.sizes(cube)["n_blocks"]
        out = np.zeros(nb, dtype=np.float64) if want_norms else None
        self._check(self.lib.fhs_proj_l2ball_blocks(
            self.h, cube, _ptr(z), _ptr(y), _ptr(v_out),
            out.ctypes.data_as(C.POINTER(C.c_double)) if want_norms else None))
        return out

    def fhs_reweight(self, cube, x, theta, theta_bar):
        self._check(self.lib.fhs_reweight(self.h, cube, _ptr(x), _ptr(theta), _ptr(theta_bar)))

    @staticmethod
    def _iterates(iterates: list[dict]):
        arr = (fhs_iterate * len(iterates))()
        for a, it in zip(arr, iterates):
            a.X, a.Xcheck, a.y = _ptr(it["X"]), _ptr(it["Xcheck"]), _ptr(it["y"])
            s = it["state"]
            a.state.W, a.state.theta, a.state.P = _ptr(s["W"]), _ptr(s["theta"]), _ptr(s["P"])
            a.state.theta_bar, a.state.v, a.state.u_prev = _ptr(s["theta_bar"]), _ptr(s["v"]), _ptr(s["u_prev"])
        return arr

    def fhs_pdfb_iter(self, iterates: list[dict], n_iter: int, want_stats: bool = True):
        arr = self._iterates(iterates)
        stats = (fhs_iter_stats * len(iterates))() if want_stats else None
        self._check(self.lib.fhs_pdfb_iter(self.h, arr, n_iter, stats))
        if not want_stats:
            return None
        return [{"xi": s.xi, "res_norm": s.res_norm, "eps_norm": s.eps_norm} for s in stats]

    def fhs_solve(self, iterates: list[dict], p_min: int, p_max: int, xi_pdfb: float, res_factor: float,
                  t_max: int, xi_reweight: float) -> list[dict]:
        """Algorithm 1 around Algorithm 2 with their stopping rules, on the device (one
        graph with nested WHILE nodes per cube); returns one report per cube."""
        arr = self._iterates(iterates)
        prm = fhs_solve_params(p_min, p_max, xi_pdfb, res_factor, t_max, xi_reweight)
        reps = (fhs_solve_report * len(iterates))()
        self._check(self.lib.fhs_solve(self.h, arr, C.byref(prm), reps))
        return [{"cycles": r.cycles, "iterations": r.iterations,
                 "iterations_per_cycle": list(r.iterations_per_cycle)[:r.cycles], "xi": r.xi,
                 "res_norm": r.res_norm, "xi_reweight": r.xi_reweight, "nonfinite": bool(r.nonfinite)}
                for r in reps]

    def fhs_heuristic_params(self, cube, sigma, power_iters=100, rel_tol=1e-4) -> dict:
        """eta, eps, mu, mu_bar of a cube from its noise levels sigma [L], computed on the
        device (power method and the noise-based heuristics) and installed in the context."""
        cp = self.cubes[cube]
        L, B, Q = cp.L, int(np.asarray(cp.M_lb).shape[1]), cp.Qy * cp.Qx
        sig = np.ascontiguousarray(sigma, dtype=np.float64)
        if sig.shape != (L,):
            raise ValueError(f"sigma must have {L} entries")
        eta, eps, mu, mub = np.zeros(L), np.zeros(L * B), np.zeros(1), np.zeros(Q)
        P = C.POINTER(C.c_double)
        self._check(self.lib.fhs_heuristic_params(self.h, cube, sig.ctypes.data_as(P), power_iters, rel_tol,
                                                  eta.ctypes.data_as(P), eps.ctypes.data_as(P),
                                                  mu.ctypes.data_as(P), mub.ctypes.data_as(P)))
        return {"eta": eta, "eps": eps.reshape(L, B), "mu": float(mu[0]), "mu_bar": mub}

    def fhs_set_preconditioning(self, cube, n_sub: int, U=None):
        """Preconditioned data duals (n_sub forward-backward sub-iterations; U in the
        caller's visibility order, or None for the inverse sampling density); n_sub = 0
        returns to Euclidean projections."""
        if U is None:
            self._check(self.lib.fhs_set_preconditioning(self.h, cube, n_sub, None))
            return
        u = np.ascontiguousarray(U, dtype=np.float32).ravel()
        if u.size != self.sizes(cube)["n_vis"]:
            raise ValueError("U must have one entry per visibility of the cube")
        self._check(self.lib.fhs_set_preconditioning(self.h, cube, n_sub, u.ctypes.data_as(C.POINTER(C.c_float))))

    def fhs_get_tuning(self, cube) -> dict:
        t = fhs_tuning()
        self._check(self.lib.fhs_get_tuning(self.h, cube, C.byref(t)))
        return {"grid_tile": t.grid_tile, "degrid_tiled": t.degrid_tiled, "gram_tc": t.gram_tc,
                "sara_fast": t.sara_fast, "prox_ctas_per_sm": t.prox_ctas_per_sm,
                "source": {0: "defaults", 1: "measured", 2: "cache"}[t.source], "ms": list(t.ms)}

    def fhs_set_lanes(self, lanes: int) -> None:
        self._check(self.lib.fhs_set_lanes(self.h, lanes))

    def fhs_get_lanes(self) -> int:
        v = C.c_int32(0)
        self._check(self.lib.fhs_get_lanes(self.h, C.byref(v)))
        return v.value

    def fhs_set_dde(self, cube, kern=None, kidx=None):
        """DDE-extended de-gridding kernels: kern [n_kern][S_d][S_d] complex (first index
        along grid rows), kidx [n_vis] kernel of each visibility in the caller's order;
        kern None returns to the plain Kaiser-Bessel rows."""
        if kern is None:
            self._check(self.lib.fhs_set_dde(self.h, cube, 0, 0, None, None))
            return
        k = np.ascontiguousarray(kern, dtype=np.complex64)
        if k.ndim != 3 or k.shape[1] != k.shape[2]:
            raise ValueError("kern must be [n_kern][S_d][S_d]")
        idx = np.ascontiguousarray(kidx, dtype=np.int32).ravel()
        if idx.size != self.sizes(cube)["n_vis"]:
            raise ValueError("kidx must have one entry per visibility of the cube")
        kf = k.view(np.float32)
        self._check(self.lib.fhs_set_dde(self.h, cube, k.shape[1], k.shape[0], kf.ctypes.data_as(C.POINTER(C.c_float)),
                                         idx.ctypes.data_as(C.POINTER(C.c_int32))))

    def fhs_pdfb_iter_host(self, iterates: list[dict], y_host: list, X_host: list, n_iter: int,
                           want_stats: bool = True):
        """fhs_pdfb_iter with the data (complex64, caller's order) and the result (float32
        images) in host memory: CPU tensors or numpy arrays, contiguous."""
        arr = self._iterates(iterates)
        n = len(iterates)
        yp = (C.c_void_p * n)(*[_host_ptr(a, np.complex64) for a in y_host])
        xp = (C.c_void_p * n)(*[_host_ptr(a, np.float32) for a in X_host])
        stats = (fhs_iter_stats * n)() if want_stats else None
        self._check(self.lib.fhs_pdfb_iter_host(self.h, arr, yp, xp, n_iter, stats))
        if not want_stats:
            return None
        return [{"xi": s.xi, "res_norm": s.res_norm, "eps_norm": s.eps_norm} for s in stats]

    def fhs_checkpoint_save(self, iterates: list[dict], path: str):
        self._check(self.lib.fhs_checkpoint_save(self.h, self._iterates(iterates), os.fsencode(path)))

    def fhs_checkpoint_load(self, iterates: list[dict], path: str):
        self._check(self.lib.fhs_checkpoint_load(self.h, self._iterates(iterates), os.fsencode(path)))

    def fhs_set_params(self, cube, tau, zeta, kappa, eta, mu, mu_bar, eps):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).ravel() for a in (eta, mu_bar, eps)]
        P = C.POINTER(C.c_double)
        self._check(self.lib.fhs_set_params(self.h, cube, tau, zeta, kappa, arrs[0].ctypes.data_as(P), mu,
                                            arrs[1].ctypes.data_as(P), arrs[2].ctypes.data_as(P)))

    def fhs_set_path(self, path: str):
        """'fast' (fused kernels, default) or 'plain' (one launch per pass)."""
        self._check(self.lib.fhs_set_path(self.h, FHS_PATH[path]))

    def fhs_kernel_launches(self) -> int:
        return int(self.lib.fhs_kernel_launches())

    def fhs_set_kernel_timer(self, kernel):
        """Record CUDA events around one kernel of fhs_pdfb_iter: None, 'grid' or 'degrid'."""
        self._check(self.lib.fhs_set_kernel_timer(self.h, FHS_TIMER[kernel]))

    def fhs_kernel_timer_read(self):
        """(summed ms, launches) of the timed kernel in the most recent iteration."""
        ms = C.c_double()
        n = C.c_int32()
        self._check(self.lib.fhs_kernel_timer_read(self.h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    # ------------------------------------------------------------ helpers
    def new_state(self, cube: int = 0) -> dict:
        """Zero duals and unit weights (Algorithm 1 starts from X = 0, weights 1)."""
        import torch
        sz = self.sizes(cube)
        L = self.cubes[cube].L
        dev = self.device
        return {
            "W": torch.zeros(L * sz["n_coef"], device=dev),
            "theta": torch.ones(sz["n_coef"], device=dev),
            "P": torch.zeros(L * sz["n_facet_pix"], device=dev),
            "theta_bar": torch.ones(sz["n_facets"] * L, device=dev),
            "v": torch.zeros(sz["n_vis"], dtype=torch.complex64, device=dev),
            "u_prev": torch.zeros(sz["n_vis"], dtype=torch.complex64, device=dev),
        }
