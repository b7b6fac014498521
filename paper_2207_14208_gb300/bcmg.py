"""Thin ctypes binding of the GB300 BCMG C ABI (``include/bcmg.h``).

Argument marshalling only: every step of the solver runs in the CUDA library
``_build/libbcmg.so``.  Tensors are PyTorch CUDA tensors (float64,
contiguous, n^d entries, x fastest); work is ordered on the current PyTorch
stream.  If the library has not been built, loading raises.
"""

from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbcmg.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bcmg.h")

OK, EINVAL, ENOMEM, ECUDA, EGEOM, ENOCONV, ENONFINITE = range(7)
INACTIVE, INTERIOR, GHOST, BOXDIR = 0, 1, 2, 3
DTAU_EXP, DTAU_POLY, DTAU_CONST = 0, 1, 2
PREC_FP64, PREC_MIXED = 0, 1
BC_DIRICHLET, BC_NEUMANN = 0, 1
CYCLE_V, CYCLE_W, CYCLE_TG = 0, 1, 2
ORDER_RB, ORDER_LEX = 0, 1

_lib = None
_lock = threading.Lock()


class BcmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bcmg error %d: %s" % (code, msg))
        self.code = code


class Opts(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("dtau_mode", C.c_int),
                ("dtau_const", C.c_double), ("ext_sweeps", C.c_int), ("min_coarse", C.c_int),
                ("max_levels", C.c_int), ("use_graph", C.c_int), ("profile", C.c_int),
                ("precision", C.c_int), ("bc", C.c_int), ("reaction", C.c_double), ("cycle", C.c_int),
                ("ordering", C.c_int), ("tg_inner", C.c_int)]


def declared_functions():
    """Names of the functions declared in include/bcmg.h."""
    text = open(HEADER).read()
    return re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(bcmg_[a-z_0-9]+)\s*\(", text, re.M)


def load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("BCMG CUDA library missing (%s); build it with "
                               "paper_2207_14208_gb300.build.build()" % LIB_PATH)
        lib = C.CDLL(LIB_PATH)
        vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_int64, C.c_double
        sig = {
            "bcmg_default_opts": (None, [vp]),
            "bcmg_create_grid_hierarchy": (i32, [i32, i64, vp, vp, vp, vp, vp]),
            "bcmg_create_grid_hierarchy_ex": (i32, [i32, i64, f64, f64, vp, vp, vp, vp, C.c_size_t, vp, vp]),
            "bcmg_workspace_size": (i32, [vp, vp]),
            "bcmg_debug_fail_allocation": (i32, [i64]),
            "bcmg_debug_batch_shape": (i32, [i32, i32, i64]),
            "bcmg_vcycle_batch": (i32, [vp, vp, i32, i32]),
            "bcmg_batch_last_shape": (i32, [vp, vp, vp]),
            "bcmg_debug_live_blocks": (i32, [vp, vp]),
            "bcmg_destroy": (i32, [vp]),
            "bcmg_ghost_count": (i32, [vp, vp]),
            "bcmg_ghost_points": (i32, [vp, vp]),
            "bcmg_set_boundary_values": (i32, [vp, vp]),
            "bcmg_set_rhs": (i32, [vp, vp]),
            "bcmg_vcycle": (i32, [vp, vp, i32]),
            "bcmg_solve": (i32, [vp, vp, f64, i32, vp, vp]),
            "bcmg_residual_norm": (i32, [vp, vp, vp]),
            "bcmg_solve_batch": (i32, [vp, vp, i32, f64, i32, vp, vp, vp]),
            "bcmg_ghost_normals": (i32, [vp, vp]),
            "bcmg_dtau_opt": (i32, [i32, i32, i32, f64, f64, vp]),
            "bcmg_memory_footprint": (i32, [vp, vp]),
            "bcmg_footprint_estimate": (i32, [i32, i64, vp, vp]),
            "bcmg_footprint": (i32, [i32, vp, vp, vp]),
            "bcmg_last_error": (C.c_char_p, []),
            "bcmg_kernel_launches": (i64, []),
            "bcmg_profile_read": (i32, [vp, vp]),
            "bcmg_time_sweeps": (i32, [vp, i32, vp]),
            "bcmg_time_sweeps_bf16": (i32, [vp, i32, vp]),
            "bcmg_residual_norms_static": (i32, [vp, vp, i64, vp, vp]),
            "bcmg_selftest_div_wsum": (i32, [i32, vp, i64, vp]),
            "bcmg_num_levels": (i32, [vp, vp]),
            "bcmg_level_info": (i32, [vp, i32, vp]),
            "bcmg_level_lists": (i32, [vp, i32, vp]),
            "bcmg_get_class": (i32, [vp, i32, vp]),
            "bcmg_get_ghosts": (i32, [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
            "bcmg_get_band": (i32, [vp, i32, vp]),
            "bcmg_smooth": (i32, [vp, i32, vp, vp, i32]),
            "bcmg_residual": (i32, [vp, i32, vp, vp, vp]),
            "bcmg_extend": (i32, [vp, i32, vp]),
            "bcmg_restrict": (i32, [vp, i32, vp, vp]),
            "bcmg_prolong": (i32, [vp, i32, vp, vp]),
            "bcmg_coarsest_solve": (i32, [vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc):
    if rc != OK:
        raise BcmgError(rc, load().bcmg_last_error().decode())


def debug_batch_shape(block: int = 0, items: int = 1, tail_rows: int = 0) -> None:
    """Launch shape of the batched kernels for the following batched solves
    (block 0: the autotuner's choice again)."""
    _check(load().bcmg_debug_batch_shape(int(block), int(items), int(tail_rows)))


def batch_last_shape():
    """(block, items per thread, tail rows) the last batched solve used."""
    b, i, t = C.c_int(), C.c_int(), C.c_int64()
    _check(load().bcmg_batch_last_shape(C.byref(b), C.byref(i), C.byref(t)))
    return b.value, i.value, t.value


def debug_fail_allocation(k: int) -> None:
    """The k-th device allocation of the library from now on fails (0: off)."""
    _check(load().bcmg_debug_fail_allocation(int(k)))


def debug_live_blocks():
    """(blocks, bytes) of device memory live handles hold from the library."""
    b, n = C.c_int64(), C.c_int64()
    _check(load().bcmg_debug_live_blocks(C.byref(b), C.byref(n)))
    return b.value, n.value


def kernel_launches() -> int:
    return int(load().bcmg_kernel_launches())


def residual_norms_static(r, cls, out):
    """Norms of a residual without any device allocation by the library
    (bcmg_residual_norms_static): r float64 and cls uint8 CUDA tensors of the
    same length, out a float64 CUDA tensor of 4 entries.  Asynchronous on the
    current stream."""
    import torch
    if not (isinstance(cls, torch.Tensor) and cls.is_cuda and cls.dtype == torch.uint8 and cls.is_contiguous()):
        raise TypeError("cls must be a contiguous CUDA uint8 tensor")
    if cls.numel() != r.numel() or out.numel() < 4:
        raise ValueError("size mismatch")
    _check(load().bcmg_residual_norms_static(_dptr(r), C.c_void_p(cls.data_ptr()), r.numel(), _dptr(out),
                                             _stream()))


def selftest_div_wsum(a: np.ndarray, fp32: bool = False) -> np.ndarray:
    """a[i] / (1 + i % 64) as the library's restriction divides (host arrays)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.empty_like(a)
    _check(load().bcmg_selftest_div_wsum(int(fp32), _hptr(a), a.size, _hptr(out)))
    return out


def _dptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_opts(**kw) -> Opts:
    o = Opts()
    load().bcmg_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def dtau_opt(dim: int, theta: float, mode: int = DTAU_EXP, bc: int = BC_DIRICHLET, const: float = 1.75) -> float:
    """The library's Delta tau_OPT(theta) (Neumann: Delta tau_OPT / h)."""
    out = C.c_double()
    _check(load().bcmg_dtau_opt(int(dim), int(bc), int(mode), float(const), float(theta), C.byref(out)))
    return out.value


def footprint(dim: int, Ns, **opts) -> int:
    """bcmg_footprint: the estimate with the grid size per axis (cubic)."""
    o = default_opts(**opts)
    arr = (C.c_int64 * len(Ns))(*[int(n) for n in Ns])
    out = C.c_size_t()
    _check(load().bcmg_footprint(int(dim), arr, C.byref(o), C.byref(out)))
    return out.value


def footprint_estimate(dim: int, N: int, **opts) -> int:
    """A-priori device-memory estimate (bytes) of a hierarchy (bcmg_footprint_estimate)."""
    o = default_opts(**opts)
    out = C.c_int64()
    _check(load().bcmg_footprint_estimate(int(dim), int(N), C.byref(o), C.byref(out)))
    return out.value


def vcycle_batch(solvers, us, ncycles: int = 1) -> None:
    """ncycles V-cycles on many hierarchies at once (bcmg_vcycle_batch)."""
    n = len(solvers)
    if len(us) != n:
        raise ValueError("one u per solver")
    hs = (C.c_void_p * n)(*[s.h.value for s in solvers])
    ps = (C.c_void_p * n)(*[_dptr(u).value for u in us])
    _check(load().bcmg_vcycle_batch(hs, ps, n, int(ncycles)))


def solve_batch(solvers, us, rtol: float = 1e-10, max_cycles: int = 100):
    """Solve on many hierarchies at once (bcmg_solve_batch): the solves run
    concurrently on the device.  Returns (cycles, rel, statuses) lists; does
    not raise for a solve that stopped at max_cycles (its status says so)."""
    n = len(solvers)
    if len(us) != n:
        raise ValueError("one u per solver")
    hs = (C.c_void_p * n)(*[s.h.value for s in solvers])
    ps = (C.c_void_p * n)(*[_dptr(u).value for u in us])
    cyc = np.zeros(n, dtype=np.int32)
    rel = np.zeros(n)
    st = np.zeros(n, dtype=np.int32)
    rc = load().bcmg_solve_batch(hs, ps, n, float(rtol), int(max_cycles), _hptr(cyc), _hptr(rel), _hptr(st))
    if rc not in (OK, ENOCONV, ENONFINITE):
        _check(rc)
    return [int(c) for c in cyc], [float(r) for r in rel], [int(x) for x in st]


class Solver:
    """A BCMG hierarchy on the current CUDA device.

    phi, f: CUDA float64 tensors with (N+1)^dim entries (x fastest)."""

    def __init__(self, dim: int, N: int, phi, f=None, lo=None, h=None, workspace=None, **opts):
        """lo, h: the box [lo, lo + N h]^dim (default [-1, 1]^dim); workspace:
        a CUDA tensor whose storage holds every device array of the
        hierarchy (kept referenced by the solver)."""
        self.lib = load()
        self.dim, self.N = dim, N
        self.n = N + 1
        self.nn = self.n ** dim
        if phi.numel() != self.nn:
            raise ValueError("phi must have (N+1)^dim entries")
        o = default_opts(**opts)
        hd = C.c_void_p()
        fp = _dptr(f) if f is not None else None
        if lo is None and h is None and workspace is None:
            _check(self.lib.bcmg_create_grid_hierarchy(dim, N, _dptr(phi), fp, C.byref(o), _stream(),
                                                       C.byref(hd)))
        else:
            lo = -1.0 if lo is None else float(lo)
            h = 2.0 / N if h is None else float(h)
            wp, wb = (None, 0) if workspace is None else \
                (C.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size())
            _check(self.lib.bcmg_create_grid_hierarchy_ex(dim, N, lo, h, _dptr(phi), fp, C.byref(o), wp, wb,
                                                          _stream(), C.byref(hd)))
        self._workspace = workspace
        self.h = hd
        self.levels = self._num_levels()

    def workspace_size(self) -> int:
        v = C.c_int64()
        _check(self.lib.bcmg_workspace_size(self.h, C.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.bcmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- problem data ------------------------------------------------
    def ghost_count(self) -> int:
        n = C.c_int64()
        _check(self.lib.bcmg_ghost_count(self.h, C.byref(n)))
        return n.value

    def ghost_points(self, out=None):
        """Q of the finest-level ghosts (count x dim CUDA float64 tensor); with
        out (a contiguous tensor of that shape, e.g. a slice of one array that
        gathers the ghosts of many hierarchies, or a float64 numpy array of
        that shape in host memory) written there."""
        import torch
        ng = self.ghost_count()
        if isinstance(out, np.ndarray):
            if out.shape != (ng, self.dim) or out.dtype != np.float64 or not out.flags.c_contiguous:
                raise ValueError("out must be a C-contiguous float64 array of shape (ghost_count, dim)")
            if ng > 0:
                _check(self.lib.bcmg_ghost_points(self.h, _hptr(out)))
            return out
        if out is not None:
            if tuple(out.shape) != (ng, self.dim) or not out.is_contiguous() or out.dtype != torch.float64:
                raise ValueError("out must be a contiguous float64 tensor of shape (ghost_count, dim)")
            if ng > 0:
                _check(self.lib.bcmg_ghost_points(self.h, _dptr(out)))
            return out
        Q = torch.empty((max(ng, 1), self.dim), dtype=torch.float64, device="cuda")
        _check(self.lib.bcmg_ghost_points(self.h, _dptr(Q)))
        return Q[:ng]

    def ghost_normals(self):
        """Outward unit normals at the finest-level ghosts (count x dim CUDA
        tensor): the direction of Neumann data."""
        import torch
        ng = self.ghost_count()
        n = torch.empty((max(ng, 1), self.dim), dtype=torch.float64, device="cuda")
        _check(self.lib.bcmg_ghost_normals(self.h, _dptr(n)))
        return n[:ng]

    def set_boundary_values(self, g):
        """g: ghost_count float64 values, a CUDA tensor or a numpy array."""
        if isinstance(g, np.ndarray):
            g = np.ascontiguousarray(g, dtype=np.float64)
            if g.size != self.ghost_count():
                raise ValueError("g must have ghost_count entries")
            _check(self.lib.bcmg_set_boundary_values(self.h, _hptr(g)))
            return
        _check(self.lib.bcmg_set_boundary_values(self.h, _dptr(g)))

    def set_rhs(self, f):
        _check(self.lib.bcmg_set_rhs(self.h, _dptr(f) if f is not None else None))

    # ---- cycles ------------------------------------------------------
    def vcycle(self, u, ncycles: int = 1):
        _check(self.lib.bcmg_vcycle(self.h, _dptr(u), ncycles))

    def solve(self, u, rtol: float = 1e-10, max_cycles: int = 100, raise_noconv: bool = True):
        c = C.c_int()
        rel = C.c_double()
        rc = self.lib.bcmg_solve(self.h, _dptr(u), float(rtol), int(max_cycles), C.byref(c), C.byref(rel))
        if rc != OK and not (rc == ENOCONV and not raise_noconv):
            _check(rc)
        return c.value, rel.value

    def profile(self) -> dict:
        """Summed device time of the finest-level sweeps timed during solve()
        (needs profile=1 at creation)."""
        out = np.zeros(2)
        _check(self.lib.bcmg_profile_read(self.h, _hptr(out)))
        return {"smooth_ms": float(out[0]), "smooth_launches": int(out[1])}

    def time_sweeps(self, nsweeps: int) -> float:
        """Summed device time (ms) of nsweeps back-to-back finest-level sweeps."""
        v = C.c_double()
        _check(self.lib.bcmg_time_sweeps(self.h, int(nsweeps), C.byref(v)))
        return v.value

    def time_sweeps_bf16(self, nsweeps: int) -> float:
        """The same sweeps with bfloat16 storage of u and Fs (FP32 arithmetic),
        on temporary copies: summed device time (ms)."""
        v = C.c_double()
        _check(self.lib.bcmg_time_sweeps_bf16(self.h, int(nsweeps), C.byref(v)))
        return v.value

    def memory_footprint(self) -> int:
        """Device memory (bytes) this hierarchy holds."""
        out = C.c_int64()
        _check(self.lib.bcmg_memory_footprint(self.h, C.byref(out)))
        return out.value

    def residual_norm(self, u) -> np.ndarray:
        out = np.zeros(4)
        _check(self.lib.bcmg_residual_norm(self.h, _dptr(u), _hptr(out)))
        return out

    # ---- introspection -----------------------------------------------
    def _num_levels(self) -> int:
        v = C.c_int()
        _check(self.lib.bcmg_num_levels(self.h, C.byref(v)))
        return v.value

    def info(self, l: int = 0) -> dict:
        out = np.zeros(10, dtype=np.int64)
        _check(self.lib.bcmg_level_info(self.h, l, _hptr(out)))
        keys = ["N", "n", "nn", "n_interior", "n_ghost", "n_band", "n_boxdir", "n_clamped",
                "n_fallback", "n_active"]
        return dict(zip(keys, (int(v) for v in out)))

    def lists(self, l: int = 0) -> dict:
        """Sizes of the parts of the level's interior list: red rows, black
        rows with a neighbour that is not interior (ghost or box edge),
        black rows whose neighbours are all interior."""
        out = np.zeros(3, dtype=np.int64)
        _check(self.lib.bcmg_level_lists(self.h, l, _hptr(out)))
        return dict(zip(["red", "black_near", "black_inner"], (int(v) for v in out)))

    def cls(self, l: int = 0) -> np.ndarray:
        out = np.zeros(self.info(l)["nn"], dtype=np.uint8)
        _check(self.lib.bcmg_get_class(self.h, l, _hptr(out)))
        return out

    def ghosts(self, l: int = 0) -> dict:
        ng = self.info(l)["n_ghost"]
        idx = np.zeros(ng, dtype=np.int64)
        eta = np.zeros(ng)
        n3 = np.zeros((ng, 3))
        xi3 = np.zeros((ng, 3))
        s3 = np.zeros((ng, 3), dtype=np.int32)
        q3 = np.zeros((ng, 3), dtype=np.int32)
        dt = np.zeros(ng)
        Q3 = np.zeros((ng, 3))
        _check(self.lib.bcmg_get_ghosts(self.h, l, _hptr(idx), _hptr(eta), _hptr(n3), _hptr(xi3),
                                        _hptr(s3), _hptr(q3), _hptr(dt), _hptr(Q3)))
        d = self.dim
        return dict(idx=idx, eta=eta, n=n3[:, :d], xi=xi3[:, :d], s=s3[:, :d], q=q3[:, :d],
                    dtau=dt, Q=Q3[:, :d])

    def band(self, l: int = 0) -> np.ndarray:
        out = np.zeros(max(self.info(l)["n_band"], 1), dtype=np.int64)
        _check(self.lib.bcmg_get_band(self.h, l, _hptr(out)))
        return out[: self.info(l)["n_band"]]

    # ---- stage operators (device tensors of one level) -------------------
    def smooth(self, l, u, F, nsteps=1):
        _check(self.lib.bcmg_smooth(self.h, l, _dptr(u), _dptr(F), nsteps))

    def residual(self, l, u, F, r):
        _check(self.lib.bcmg_residual(self.h, l, _dptr(u), _dptr(F), _dptr(r)))

    def extend(self, l, a):
        _check(self.lib.bcmg_extend(self.h, l, _dptr(a)))

    def restrict(self, l, rf, Fc):
        _check(self.lib.bcmg_restrict(self.h, l, _dptr(rf), _dptr(Fc)))

    def prolong(self, l, ec, uf):
        _check(self.lib.bcmg_prolong(self.h, l, _dptr(ec), _dptr(uf)))

    def coarsest_solve(self, u, F):
        _check(self.lib.bcmg_coarsest_solve(self.h, _dptr(u), _dptr(F)))
