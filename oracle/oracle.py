"""ctypes wrapper of the C oracle (test infrastructure only).

The oracle is plain single-threaded FP64 C (``bcmg_oracle.c``); this module
compiles it with gcc into ``oracle/_build/liboracle.so`` and exposes it with
numpy arrays.  Nothing here is shared with the CUDA library.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bcmg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

# node classes (Sec. 3.3 partition of the grid)
INACTIVE, INTERIOR, GHOST, BOXDIR = 0, 1, 2, 3
# interior orderings: red-black, lexicographic GS (the paper's GS-LEX), and
# the exact interior block solve of REL-BC (eq. 2Ddiri:Pbc)
RB, LEX, BLOCK = 0, 1, 2
# Delta tau forms: exp form of G0 (Remark exptheta2D), polynomial form
# (eqs. G / G3D), constant
DT_EXP, DT_POLY, DT_CONST = 0, 1, 2
# boundary condition on Gamma
DIRICHLET, NEUMANN = 0, 1
# cycles: V (gamma = 1), two-grid correction scheme, W (gamma = 2)
CYC_V, CYC_TGCS, CYC_W = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, no FMA contraction) and return the path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp, i32, i64, f64 = C.c_void_p, C.c_int, C.c_long, C.c_double
        P = C.POINTER
        sig = {
            "orc_create": (vp, [i32, i32, vp, vp, vp]),
            "orc_destroy": (None, [vp]),
            "orc_num_levels": (i32, [vp]),
            "orc_direct_ok": (i32, [vp]),
            "orc_level_info": (None, [vp, i32, vp]),
            "orc_get_class": (None, [vp, i32, vp]),
            "orc_get_phi": (None, [vp, i32, vp]),
            "orc_get_ghosts": (None, [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
            "orc_get_band": (None, [vp, i32, vp]),
            "orc_set_rhs": (None, [vp, vp, vp]),
            "orc_get_F": (None, [vp, i32, vp]),
            "orc_set_F": (None, [vp, i32, vp]),
            "orc_smooth": (None, [vp, i32, vp, vp, i32]),
            "orc_interior_sweep": (None, [vp, i32, vp, vp]),
            "orc_interior_block": (i64, [vp, i32, vp, vp]),
            "orc_ghost_relax": (None, [vp, i32, vp, vp]),
            "orc_ghost_apply": (None, [vp, i32, vp, vp]),
            "orc_residual": (None, [vp, i32, vp, vp, vp]),
            "orc_extend": (None, [vp, i32, vp]),
            "orc_restrict": (None, [vp, i32, vp, vp]),
            "orc_prolong": (None, [vp, i32, vp, vp]),
            "orc_coarsest_solve": (None, [vp, vp, vp]),
            "orc_vcycle": (None, [vp, vp, i32]),
            "orc_norms": (None, [vp, vp, vp]),
            "orc_solve": (i32, [vp, vp, f64, i32, vp]),
            "orc_active_count": (i64, [vp, i32]),
            "orc_assemble": (None, [vp, i32, vp, vp, vp, vp, vp]),
            "orc_direct_solve": (i32, [vp, i32, vp, vp]),
            "orc_blfa_p": (f64, [i32, vp]),
            "orc_blfa_G0": (f64, [i32, i32, f64, f64]),
            "orc_dtau": (f64, [i32, i32, i32, f64, f64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        del P
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def blfa_p(d: int, alpha) -> float:
    """p(alpha) = acosh(d - sum cos alpha_i) (eqs. alphaNalpha / alphaNalpha3D)."""
    al = _f64(np.atleast_1d(alpha) if d > 1 else np.zeros(1))
    return _load().orc_blfa_p(d, _p(al))


def blfa_G0(bc: int, form: int, p: float, theta: float) -> float:
    """G0 of eqs. G / GN (form=1) or of Remark exptheta2D (form=0)."""
    return _load().orc_blfa_G0(bc, form, float(p), float(theta))


def dtau(d: int, theta: float, mode: int = DT_EXP, const: float = 1.75, bc: int = 0) -> float:
    """Delta tau_OPT(theta) of Props. 1-4 (or the constant)."""
    return _load().orc_dtau(d, bc, mode, float(const), float(theta))


class Oracle:
    """One BCMG hierarchy built by the oracle from grid values of phi."""

    def __init__(self, d: int, N: int, phi: np.ndarray, *, nu1: int = 2, nu2: int = 1,
                 ordering: int = RB, dtau_mode: int = DT_EXP, dtau_const: float = 1.75,
                 ext_sweeps: int = 4, cycle: int = CYC_V, min_coarse: int = 8,
                 max_levels: int = 24, tgcs_tol: float = 1e-13, tgcs_maxit: int = 200,
                 rmode: int = 3, ext_mode: int = 0, ext_cfl: float = 0.5, bc: int = 0,
                 reaction: float = 0.0, band_width: int = 2, gfam: int = 0,
                 cg_rhs: int = 0):
        self.lib = _load()
        self.d, self.N = d, N
        self.n = N + 1
        self.shape = (self.n,) * d
        phi = _f64(phi).reshape(-1)
        assert phi.size == self.n ** d
        iopts = np.array([nu1, nu2, ordering, dtau_mode, ext_sweeps, cycle, min_coarse,
                          max_levels, tgcs_maxit, rmode, ext_mode, bc, band_width, gfam,
                          cg_rhs], dtype=np.int32)
        dopts = np.array([dtau_const, tgcs_tol, ext_cfl, reaction], dtype=np.float64)
        self.h = self.lib.orc_create(d, N, _p(phi), _p(iopts), _p(dopts))
        if not self.h:
            raise ValueError("oracle: no interior node on the finest level")
        self.L = self.lib.orc_num_levels(self.h)

    def _need_direct(self):
        if not self.lib.orc_direct_ok(self.h):
            raise ValueError("oracle: coarsest system singular or too large for the dense solve")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    # ---- structure -------------------------------------------------
    def info(self, l: int = 0) -> dict:
        out = np.zeros(10, dtype=np.int64)
        self.lib.orc_level_info(self.h, l, _p(out))
        keys = ["N", "n", "nn", "n_interior", "n_ghost", "n_band", "n_boxdir",
                "n_clamped", "n_fallback", "n_active"]
        return dict(zip(keys, (int(v) for v in out)))

    def nn(self, l: int) -> int:
        return self.info(l)["nn"]

    def cls(self, l: int = 0) -> np.ndarray:
        out = np.zeros(self.nn(l), dtype=np.uint8)
        self.lib.orc_get_class(self.h, l, _p(out))
        return out

    def phi(self, l: int = 0) -> np.ndarray:
        out = np.zeros(self.nn(l), dtype=np.float64)
        self.lib.orc_get_phi(self.h, l, _p(out))
        return out

    def ghosts(self, l: int = 0) -> dict:
        ng = self.info(l)["n_ghost"]
        idx = np.zeros(ng, dtype=np.int64)
        eta = np.zeros(ng)
        n = np.zeros((ng, 3))
        xi = np.zeros((ng, 3))
        s = np.zeros((ng, 3), dtype=np.int32)
        q = np.zeros((ng, 3), dtype=np.int32)
        dt = np.zeros(ng)
        Q = np.zeros((ng, 3))
        self.lib.orc_get_ghosts(self.h, l, _p(idx), _p(eta), _p(n), _p(xi), _p(s), _p(q),
                                _p(dt), _p(Q))
        d = self.d
        return dict(idx=idx, eta=eta, n=n[:, :d], xi=xi[:, :d], s=s[:, :d], q=q[:, :d],
                    dtau=dt, Q=Q[:, :d])

    def band(self, l: int = 0) -> np.ndarray:
        nb = self.info(l)["n_band"]
        out = np.zeros(nb, dtype=np.int64)
        self.lib.orc_get_band(self.h, l, _p(out))
        return out

    # ---- data ------------------------------------------------------
    def set_rhs(self, f: np.ndarray, gQ: np.ndarray) -> None:
        f = _f64(f).reshape(-1)
        gQ = _f64(gQ).reshape(-1)
        assert gQ.size == self.info(0)["n_ghost"]
        self.lib.orc_set_rhs(self.h, _p(f), _p(gQ))

    def F(self, l: int = 0) -> np.ndarray:
        out = np.zeros(self.nn(l))
        self.lib.orc_get_F(self.h, l, _p(out))
        return out

    def set_F(self, l: int, F: np.ndarray) -> None:
        F = _f64(F).reshape(-1)
        self.lib.orc_set_F(self.h, l, _p(F))

    # ---- stage operators (in place on copies) --------------------------
    def smooth(self, l: int, u: np.ndarray, F: np.ndarray, nsteps: int = 1) -> np.ndarray:
        u = _f64(u).reshape(-1).copy()
        F = _f64(F).reshape(-1)
        self.lib.orc_smooth(self.h, l, _p(u), _p(F), nsteps)
        return u

    def interior_sweep(self, l: int, u: np.ndarray, F: np.ndarray) -> np.ndarray:
        u = _f64(u).reshape(-1).copy()
        self.lib.orc_interior_sweep(self.h, l, _p(u), _p(_f64(F).reshape(-1)))
        return u

    def interior_block(self, l: int, u: np.ndarray, F: np.ndarray) -> np.ndarray:
        u = _f64(u).reshape(-1).copy()
        self.lib.orc_interior_block(self.h, l, _p(u), _p(_f64(F).reshape(-1)))
        return u

    def ghost_relax(self, l: int, u: np.ndarray, F: np.ndarray) -> np.ndarray:
        u = _f64(u).reshape(-1).copy()
        self.lib.orc_ghost_relax(self.h, l, _p(u), _p(_f64(F).reshape(-1)))
        return u

    def ghost_apply(self, l: int, u: np.ndarray) -> np.ndarray:
        u = _f64(u).reshape(-1)
        out = np.zeros(self.info(l)["n_ghost"])
        self.lib.orc_ghost_apply(self.h, l, _p(u), _p(out))
        return out

    def residual(self, l: int, u: np.ndarray, F: np.ndarray) -> np.ndarray:
        u = _f64(u).reshape(-1)
        F = _f64(F).reshape(-1)
        r = np.zeros(self.nn(l))
        self.lib.orc_residual(self.h, l, _p(u), _p(F), _p(r))
        return r

    def extend(self, l: int, a: np.ndarray) -> np.ndarray:
        a = _f64(a).reshape(-1).copy()
        self.lib.orc_extend(self.h, l, _p(a))
        return a

    def restrict(self, l: int, rf: np.ndarray) -> np.ndarray:
        rf = _f64(rf).reshape(-1)
        Fc = np.zeros(self.nn(l + 1))
        self.lib.orc_restrict(self.h, l, _p(rf), _p(Fc))
        return Fc

    def prolong(self, l: int, ec: np.ndarray, uf: np.ndarray) -> np.ndarray:
        ec = _f64(ec).reshape(-1)
        uf = _f64(uf).reshape(-1).copy()
        self.lib.orc_prolong(self.h, l, _p(ec), _p(uf))
        return uf

    def coarsest_solve(self, u: np.ndarray, F: np.ndarray) -> np.ndarray:
        self._need_direct()
        u = _f64(u).reshape(-1).copy()
        self.lib.orc_coarsest_solve(self.h, _p(u), _p(_f64(F).reshape(-1)))
        return u

    # ---- cycles ----------------------------------------------------
    def vcycle(self, u: np.ndarray, ncycles: int = 1) -> np.ndarray:
        self._need_direct()
        u = _f64(u).reshape(-1).copy()
        self.lib.orc_vcycle(self.h, _p(u), ncycles)
        return u

    def norms(self, u: np.ndarray) -> np.ndarray:
        out = np.zeros(4)
        self.lib.orc_norms(self.h, _p(_f64(u).reshape(-1)), _p(out))
        return out

    def solve(self, u: np.ndarray, rtol: float = 1e-10, max_cycles: int = 100):
        self._need_direct()
        u = _f64(u).reshape(-1).copy()
        hist = np.zeros(max_cycles + 1)
        c = self.lib.orc_solve(self.h, _p(u), float(rtol), max_cycles, _p(hist))
        return u, c, hist[: c + 1]

    def assemble(self, l: int, u: np.ndarray, F: np.ndarray):
        nact = self.lib.orc_active_count(self.h, l)
        act = np.zeros(nact, dtype=np.int64)
        A = np.zeros((nact, nact))
        rhs = np.zeros(nact)
        self.lib.orc_assemble(self.h, l, _p(_f64(u).reshape(-1)), _p(_f64(F).reshape(-1)),
                              _p(act), _p(A), _p(rhs))
        return act, A, rhs

    def direct_solve(self, l: int, u: np.ndarray, F: np.ndarray) -> np.ndarray:
        u = _f64(u).reshape(-1).copy()
        rc = self.lib.orc_direct_solve(self.h, l, _p(u), _p(_f64(F).reshape(-1)))
        if rc != 0:
            raise np.linalg.LinAlgError("oracle: singular system")
        return u

    def rho(self, u0: np.ndarray, ncycles: int = 16):
        """Convergence-factor protocol of Sec. 2.2: rho = mean of
        ||r^(m+1)|| / ||r^(m)|| for m = 11..15 (homogeneous problem)."""
        u = _f64(u0).reshape(-1).copy()
        u[self.cls(0) == BOXDIR] = 0.0  # homogeneous eliminated Dirichlet data
        norms = []
        for m in range(ncycles + 1):
            nr = self.norms(u)
            norms.append(float(np.hypot(nr[0], nr[1])))
            if m < ncycles:
                self.lib.orc_vcycle(self.h, _p(u), 1)
        norms = np.array(norms)
        ratios = norms[1:] / np.where(norms[:-1] == 0, 1, norms[:-1])
        return float(np.mean(ratios[11:16])), norms
