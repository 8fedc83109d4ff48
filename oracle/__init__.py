"""CPU oracle of the TU-fRG hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_1710_08830_gb300``) never imports it and never falls
back to it.

``oracle/tufrg_oracle.c`` is a plain FP64 C implementation written from the
paper's equations; this module compiles it with gcc (``build()``) and wraps it
with ctypes.  ``oracle/bruteforce.py`` is a second, independent numpy
implementation of the full-momentum RGE used to pin the oracle.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tufrg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# The mutation test (tests/test_oracle_mutants.py) compiles copies of the oracle with one planted mistake
# each and runs the pin tests against them in a subprocess with this variable naming the copy; nothing
# else sets it.
MUTANT_ENV = "TUFRG_ORACLE_MUTANT_LIB"
_lock = threading.Lock()
_lib = None


def compile_source(src: str, out: str) -> str:
    """gcc -O2 -fopenmp (no -march) of one oracle source file into the shared library out."""
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (OpenMP, -O2, no -march)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [("ns", C.c_int), ("nhop", C.c_int), ("hopR", C.c_void_p), ("hopt", C.c_void_p),
                ("V0", C.c_void_p), ("nff", C.c_int), ("ffR", C.c_void_p),
                ("Lq", C.c_int), ("nc", C.c_int), ("mu", C.c_double), ("reg", C.c_int), ("T_reg", C.c_double),
                ("V0q", C.c_void_p)]


class FlowOpts(C.Structure):
    _fields_ = [("T0", C.c_double), ("T_end", C.c_double), ("rtol", C.c_double), ("atol", C.c_double),
                ("h0", C.c_double), ("stop", C.c_double), ("chmask", C.c_int), ("max_steps", C.c_int),
                ("fixed_n", C.c_int)]


class FlowResult(C.Structure):
    _fields_ = [("Tc", C.c_double), ("crossed", C.c_int), ("n_steps", C.c_int), ("n_reject", C.c_int),
                ("n_rhs", C.c_int), ("amax", C.c_double), ("T_last", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get(MUTANT_ENV) or build()
            L = C.CDLL(path)
            vp, d, i = C.c_void_p, C.c_double, C.c_int
            L.or_eigh.argtypes = [i, vp, vp, vp]
            L.or_bands.argtypes = [vp, vp, vp]
            L.or_density.argtypes = [vp, vp, d, d]
            L.or_density.restype = d
            L.or_find_mu.argtypes = [vp, vp, d, d]
            L.or_find_mu.restype = d
            L.or_fermi.argtypes = [d, d, vp, vp, vp]
            for fn in ("or_wm", "or_wp", "or_Fm", "or_Fp"):
                getattr(L, fn).argtypes = [d, d, d]
                getattr(L, fn).restype = d
            for fn in ("or_chi", "or_dchi"):
                getattr(L, fn).argtypes = [d, d]
                getattr(L, fn).restype = d
            for fn in ("or_wm_shell", "or_wp_shell"):
                getattr(L, fn).argtypes = [d, d, d, d]
                getattr(L, fn).restype = d
            L.or_delta_list.argtypes = [vp, vp]
            L.or_delta_list.restype = i
            L.or_loops.argtypes = [vp, vp, vp, d, i, i, vp]
            L.or_loops_at.argtypes = [vp, vp, vp, d, i, i, i, vp, vp]
            L.or_project.argtypes = [vp, vp, i, vp]
            L.or_project.restype = d
            L.or_vlv.argtypes = [vp, vp, vp, vp, i, vp]
            L.or_rhs.argtypes = [vp, vp, vp, d, vp, i, vp, vp]
            L.or_band_transform.argtypes = [vp, vp, vp, vp]
            L.or_bare_state.argtypes = [vp, vp]
            L.or_bare_state.restype = None
            L.or_band_transform.restype = None
            L.or_rhs.restype = d
            L.or_rhs_at.argtypes = [vp, vp, vp, d, vp, i, i, vp, vp]
            L.or_shard_classes.argtypes = [vp, vp]
            L.or_shard_classes.restype = i
            L.or_shard_transform.argtypes = [vp, vp, i, vp, i, vp]
            L.or_shard_transform.restype = None
            L.or_shard_finish.argtypes = [vp, vp, vp, d, vp, i, vp, vp, i, vp]
            L.or_shard_finish.restype = None
            L.or_flow.argtypes = [vp, vp, vp, vp, vp, vp]
            L.or_flow.restype = i
            L.or_num_threads.restype = i
            L.or_set_threads.argtypes = [i]
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def eigh(H: np.ndarray):
    """Eigen-decomposition of one Hermitian matrix by the oracle's Jacobi solver."""
    H = np.ascontiguousarray(H, np.complex128)
    n = H.shape[0]
    E = np.zeros(n)
    U = np.zeros((n, n), np.complex128)
    lib().or_eigh(n, _ptr(H), _ptr(E), _ptr(U))
    return E, U


def fermi(e: float, T: float):
    f, g, gp = C.c_double(), C.c_double(), C.c_double()
    lib().or_fermi(e, T, C.byref(f), C.byref(g), C.byref(gp))
    return f.value, g.value, gp.value


def wm(e1, e2, T):
    return lib().or_wm(e1, e2, T)


def wp(e1, e2, T):
    return lib().or_wp(e1, e2, T)


def Fm(e1, e2, T):
    return lib().or_Fm(e1, e2, T)


def Fp(e1, e2, T):
    return lib().or_Fp(e1, e2, T)


class Oracle:
    """The oracle bound to one model descriptor (``inputs.ModelSpec``).

    basis="band": the flow in the band basis (Sec. 3.2, Eqs. rge_Pmat, rge_Dmat): the loops are band-diagonal
    (the eigenvectors replaced by unit vectors, Eqs. loopminus, loopplus with Eqs. disc_2a, disc_2b) and the bare
    vertex enters through its band-basis projections, P^[V0](s) and C^[V0](u) transformed with Eqs. mat_trafo_P,
    mat_trafo_D from the orbital ones (V0 onsite, Sec. 4), with the eigenvectors band_U [Nk][N_s][N_s] (default:
    the oracle's own; the band basis depends on their gauge).  States, loops and right-hand sides are then
    band-basis objects in the layouts of the orbital ones with band indices in place of orbital indices."""

    def __init__(self, spec, mu: float | None = None, basis: str = "orbital", band_U=None):
        self.spec = spec
        self._hopR = np.ascontiguousarray(spec.hop_R, np.int32)
        self._hopt = np.ascontiguousarray(spec.hop_t, np.complex128)
        self._V0 = np.ascontiguousarray(spec.V0, np.complex128)
        self._ffR = np.ascontiguousarray(spec.ff_R, np.int32)
        self.m = _Model(spec.n_s, self._hopR.shape[0], _ptr(self._hopR), _ptr(self._hopt),
                        _ptr(self._V0), self._ffR.shape[0], _ptr(self._ffR), spec.Lq, spec.nc, 0.0,
                        int(getattr(spec, "regulator", 0)), float(getattr(spec, "T_reg", 0.05)), None)
        self.E, self.U = self.bands()
        if mu is not None:
            self.mu = float(mu)
        elif spec.filling > 0:
            self.mu = self.find_mu(spec.filling, spec.T_mu)
        else:
            self.mu = float(spec.mu)
        self.m.mu = self.mu
        dl = np.zeros((4096, 2), np.int32)
        nd = lib().or_delta_list(C.byref(self.m), _ptr(dl))
        self.deltas = dl[:nd].copy()
        self.basis = basis
        if basis == "band":
            Ub = self.U if band_U is None else np.ascontiguousarray(band_U, np.complex128).reshape(self.U.shape)
            s0 = np.zeros((2, spec.Nq, spec.M, spec.M), np.complex128)
            lib().or_bare_state(C.byref(self.m), _ptr(s0))
            self._V0q = np.ascontiguousarray(self.band_transform(Ub, s0))
            self.m.V0q = _ptr(self._V0q)
            self.U = np.ascontiguousarray(np.broadcast_to(np.eye(spec.n_s, dtype=np.complex128), self.U.shape))
        elif basis != "orbital":
            raise ValueError("basis must be 'orbital' or 'band'")

    def bare_state(self) -> np.ndarray:
        """The bare vertex as a state [2][Nq][M][M] (its projections at every momentum), orbital basis."""
        s = self.spec
        out = np.zeros((2, s.Nq, s.M, s.M), np.complex128)
        lib().or_bare_state(C.byref(self.m), _ptr(out))
        return out

    @property
    def nd(self) -> int:
        return int(self.deltas.shape[0])

    def bands(self):
        s = self.spec
        E = np.zeros((s.Nk, s.n_s))
        U = np.zeros((s.Nk, s.n_s, s.n_s), np.complex128)
        lib().or_bands(C.byref(self.m), _ptr(E), _ptr(U))
        return E, U

    def density(self, mu: float, T: float) -> float:
        return lib().or_density(C.byref(self.m), _ptr(self.E), mu, T)

    def find_mu(self, filling: float, T: float) -> float:
        return lib().or_find_mu(C.byref(self.m), _ptr(self.E), filling, T)

    def loops(self, T: float, which: int, kind: int = 0) -> np.ndarray:
        """Compact loops [Nq][nd][ns^2][ns^2]; which 0 = P (L^-), 1 = C (L^+); kind 1 = bubble F."""
        s = self.spec
        out = np.zeros((s.Nq, self.nd, s.n_s ** 2, s.n_s ** 2), np.complex128)
        lib().or_loops(C.byref(self.m), _ptr(self.E), _ptr(self.U), T, which, kind, _ptr(out))
        return out

    def loops_at(self, T: float, which: int, s_list, kind: int = 0) -> np.ndarray:
        """Compact loops for the listed transfer momenta only: [len(s_list)][nd][ns^2][ns^2]."""
        s = self.spec
        sl = np.ascontiguousarray(s_list, np.int32)
        out = np.zeros((sl.shape[0], self.nd, s.n_s ** 2, s.n_s ** 2), np.complex128)
        lib().or_loops_at(C.byref(self.m), _ptr(self.E), _ptr(self.U), T, which, kind, sl.shape[0], _ptr(sl),
                          _ptr(out))
        return out

    def project(self, state: np.ndarray, chmask: int = 3):
        s = self.spec
        state = np.ascontiguousarray(state, np.complex128)
        A = np.zeros_like(state)
        amax = lib().or_project(C.byref(self.m), _ptr(state), chmask, _ptr(A))
        return A, amax

    def vlv(self, A: np.ndarray, LcP: np.ndarray, LcC: np.ndarray, chmask: int = 3) -> np.ndarray:
        A = np.ascontiguousarray(A, np.complex128)
        LcP = np.ascontiguousarray(LcP, np.complex128)
        LcC = np.ascontiguousarray(LcC, np.complex128)
        out = np.zeros_like(A)
        lib().or_vlv(C.byref(self.m), _ptr(A), _ptr(LcP), _ptr(LcC), chmask, _ptr(out))
        return out

    def band_transform(self, Ub: np.ndarray, state: np.ndarray) -> np.ndarray:
        """Exchange propagators P, C of ``state`` in the band basis of the eigenvectors ``Ub[k][sigma][n]``
        (Sec. 3.4, Eqs. mat_trafo_P, mat_trafo_D)."""
        s = self.spec
        Ub = np.ascontiguousarray(Ub, np.complex128).reshape(s.Nk, s.n_s, s.n_s)
        st = np.ascontiguousarray(state, np.complex128).reshape(2, s.Nq, s.M, s.M)
        out = np.zeros_like(st)
        lib().or_band_transform(C.byref(self.m), _ptr(Ub), _ptr(st), _ptr(out))
        return out

    def rhs(self, T: float, state: np.ndarray, chmask: int = 3, want_A: bool = False):
        """dX/dT at temperature T; returns (dX, max|A|[, A])."""
        state = np.ascontiguousarray(state, np.complex128)
        d = np.zeros_like(state)
        A = np.zeros_like(state) if want_A else None
        amax = lib().or_rhs(C.byref(self.m), _ptr(self.E), _ptr(self.U), T, _ptr(state), chmask,
                            _ptr(d), _ptr(A) if want_A else None)
        return (d, amax, A) if want_A else (d, amax)

    def rhs_at(self, T: float, state: np.ndarray, s_list, chmask: int = 3) -> np.ndarray:
        """dX/dT restricted to the listed transfer momenta: [2][len(s_list)][M][M]."""
        s = self.spec
        state = np.ascontiguousarray(state, np.complex128)
        sl = np.ascontiguousarray(s_list, np.int32)
        out = np.zeros((2, sl.shape[0], s.M, s.M), np.complex128)
        lib().or_rhs_at(C.byref(self.m), _ptr(self.E), _ptr(self.U), T, _ptr(state), chmask, sl.shape[0], _ptr(sl),
                        _ptr(out))
        return out

    # ------------------------------------------------------------ the right-hand side split over shards of momenta
    def shard_classes(self) -> np.ndarray:
        """Bond classes R'' (mod Lq) of the shard transforms, [ncls][2]."""
        cls = np.zeros((4096, 2), np.int32)
        n = lib().or_shard_classes(C.byref(self.m), _ptr(cls))
        return cls[:n].copy()

    def shard_transform(self, state_local: np.ndarray, q_list, chmask: int = 3) -> np.ndarray:
        """This shard's part of the Fourier transform of Sec. 3.3: [2][ncls][M][M], summed over the listed momenta
        (state_local [2][n][M][M] holds their rows in list order)."""
        s = self.spec
        ql = np.ascontiguousarray(q_list, np.int32)
        st = np.ascontiguousarray(state_local, np.complex128)
        ncls = self.shard_classes().shape[0]
        out = np.zeros((2, ncls, s.M, s.M), np.complex128)
        lib().or_shard_transform(C.byref(self.m), _ptr(st), ql.shape[0], _ptr(ql), chmask, _ptr(out))
        return out

    def shard_finish(self, T: float, state_local: np.ndarray, q_list, xr: np.ndarray, chmask: int = 3) -> np.ndarray:
        """dX/dT of the listed momenta [2][n][M][M] from their rows and the transforms summed over all shards."""
        s = self.spec
        ql = np.ascontiguousarray(q_list, np.int32)
        st = np.ascontiguousarray(state_local, np.complex128)
        xr = np.ascontiguousarray(xr, np.complex128)
        out = np.zeros((2, ql.shape[0], s.M, s.M), np.complex128)
        lib().or_shard_finish(C.byref(self.m), _ptr(self.E), _ptr(self.U), T, _ptr(st), ql.shape[0], _ptr(ql), _ptr(xr),
                              chmask, _ptr(out))
        return out

    def flow(self, T0=10.0, T_end=0.02, rtol=1e-6, atol=1e-8, h0=-0.05, stop=50.0, chmask=3,
             max_steps=100000, fixed_n=0):
        s = self.spec
        state = np.zeros((2, s.Nq, s.M, s.M), np.complex128)
        o = FlowOpts(T0, T_end, rtol, atol, h0, stop, chmask, max_steps, fixed_n)
        r = FlowResult()
        st = lib().or_flow(C.byref(self.m), _ptr(self.E), _ptr(self.U), C.byref(o), _ptr(state), C.byref(r))
        res = {f: getattr(r, f) for f, _ in FlowResult._fields_}
        res["status"] = st
        return state, res
