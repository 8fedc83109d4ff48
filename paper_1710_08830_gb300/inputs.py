"""Seeded, synthetic model inputs shared by the CUDA path and the oracle.

This module only *describes* lattice models: hopping matrices t_R, the onsite
initial vertex V^(0), the form-factor bond set and the meshes.  It holds none
of the TU-fRG arithmetic (no eigensolve, no loops, no projections, no flow);
both the CUDA library and the CPU oracle consume the same descriptor and do
all of that on their own.

Conventions (shared by both consumers, stated once here):

* Square lattice, unit lattice constant.  The Bloch Hamiltonian is
  H(k)[tau][tau'] = sum_R t_R[tau][tau'] exp(i k.R)  (Sec. 4, Eq. gen_Ham for
  the two-band case); the descriptor stores every R with its own matrix, and
  t_{-R} = t_R^dagger so that H(k) is Hermitian.
* Spin-orbital index tau = 2*orbital + spin, spin 0 = up, 1 = down.
* Initial vertex V0[s1][s2][s3][s4]: onsite, antisymmetric, normalised as
  the paper's Hubbard vertex V^(0) = (U/2)(d13 d24 - d14 d23) (Sec. 4).  For
  multi-orbital interactions H_int = 1/2 sum W_1234 c+_1 c+_2 c_4 c_3 we set
  V0 = (W_1234 - W_1243)/2, which reproduces that normalisation.
* Form factors are plane waves f_R(k) = exp(-i k.R) labelled by bonds R
  (Sec. 2); the bond list always starts with R = (0,0).
* Transfer momenta live on an Lq x Lq mesh, loop momenta on the fine
  (Lq*nc) x (Lq*nc) mesh that contains it.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

SIGMA_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SIGMA_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SIGMA_Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


@dataclass
class ModelSpec:
    """One lattice model plus its TU-fRG discretisation."""
    name: str
    n_s: int
    hop_R: np.ndarray          # int32 [n_hop, 2]
    hop_t: np.ndarray          # complex128 [n_hop, n_s, n_s]
    V0: np.ndarray             # complex128 [n_s, n_s, n_s, n_s]
    ff_R: np.ndarray           # int32 [n_ff, 2], ff_R[0] == (0, 0)
    Lq: int
    nc: int
    mu: float = 0.0            # used when filling <= 0
    filling: float = 0.0       # electrons per site (all spin-orbitals); > 0 => mu is bisected
    T_mu: float = 0.02         # temperature at which mu is fixed by the filling
    params: dict = field(default_factory=dict)
    regulator: int = 0         # 0: temperature flow (scale = T); 1: momentum shell (scale = Lambda, Eq. def_lmp)
    T_reg: float = 0.05        # momentum shell: temperature of the Fermi functions in the bubbles

    @property
    def n_ff(self) -> int:
        return int(self.ff_R.shape[0])

    @property
    def M(self) -> int:
        return self.n_ff * self.n_s * self.n_s

    @property
    def Nq(self) -> int:
        return self.Lq * self.Lq

    @property
    def Lf(self) -> int:
        return self.Lq * self.nc

    @property
    def Nk(self) -> int:
        return self.Lf * self.Lf

    def with_(self, **kw) -> "ModelSpec":
        return replace(self, **kw)


# ----------------------------------------------------------------------------
# form-factor bond sets (Sec. 2: plane waves labelled by bonds, truncated at |R_c|)
# ----------------------------------------------------------------------------

def ff_set(n_ff: int) -> np.ndarray:
    """Bond sets used by the workloads: onsite + shells of the square lattice.

    5  = onsite + 4 nearest neighbours; 9 adds the 4 diagonal bonds;
    13 adds the 4 third-neighbour bonds (+-2, 0), (0, +-2).
    """
    shells = [
        [(0, 0)],
        [(1, 0), (0, 1), (-1, 0), (0, -1)],
        [(1, 1), (-1, 1), (-1, -1), (1, -1)],
        [(2, 0), (0, 2), (-2, 0), (0, -2)],
    ]
    out: List = []
    for sh in shells:
        if len(out) >= n_ff:
            break
        out.extend(sh)
    if len(out) != n_ff:
        raise ValueError(f"unsupported form-factor count {n_ff} (use 1, 5, 9 or 13)")
    return np.asarray(out, dtype=np.int32)


def ff_complete(L: int) -> np.ndarray:
    """All L*L bonds of an L x L torus (distinct mod L), onsite first.

    With this set the truncated unity of Eq. unity is the exact identity.
    """
    lo = -((L - 1) // 2)
    pts = [(x, y) for x in range(lo, lo + L) for y in range(lo, lo + L)]
    pts.sort(key=lambda p: (p[0] * p[0] + p[1] * p[1], p[0], p[1]))
    return np.asarray(pts, dtype=np.int32)


# ----------------------------------------------------------------------------
# hopping builders
# ----------------------------------------------------------------------------

class _Hops:
    def __init__(self, n_s: int):
        self.n_s = n_s
        self.d = {}

    def add(self, R, mat):
        R = (int(R[0]), int(R[1]))
        mat = np.asarray(mat, dtype=np.complex128)
        if R not in self.d:
            self.d[R] = np.zeros((self.n_s, self.n_s), np.complex128)
        self.d[R] = self.d[R] + mat

    def add_pair(self, R, mat):
        """Add t_R = mat and t_{-R} = mat^dagger (Hermitian H(k))."""
        self.add(R, mat)
        self.add((-R[0], -R[1]), np.conj(np.asarray(mat, np.complex128)).T)

    def arrays(self):
        keys = sorted(self.d.keys())
        R = np.asarray(keys, dtype=np.int32).reshape(-1, 2)
        t = np.stack([self.d[k] for k in keys]).astype(np.complex128)
        return R, t


def onsite_hubbard_vertex(U: float) -> np.ndarray:
    """V^(0) = (U/2)(d13 d24 - d14 d23) for one orbital with spin (Sec. 4)."""
    d = np.eye(2)
    return (U / 2.0) * (np.einsum("ac,bd->abcd", d, d) - np.einsum("ad,bc->abcd", d, d)).astype(np.complex128)


def kanamori_vertex(n_orb: int, U: float, J: float) -> np.ndarray:
    """Antisymmetrised onsite Kanamori vertex for n_orb orbitals with spin.

    H_int = 1/2 sum U_abcd c+_{a s} c+_{b s'} c_{d s'} c_{c s} with U_aaaa = U,
    U_abab = U' = U - 2J, U_abba = J (Hund), U_aabb = J (pair hopping);
    W_1234 = U_abcd d(s1,s3) d(s2,s4), V0 = (W_1234 - W_1243)/2.
    """
    Uo = np.zeros((n_orb,) * 4)
    Up = U - 2.0 * J
    for a in range(n_orb):
        Uo[a, a, a, a] = U
        for b in range(n_orb):
            if a != b:
                Uo[a, b, a, b] = Up
                Uo[a, b, b, a] = J
                Uo[a, a, b, b] = J
    ns = 2 * n_orb
    W = np.zeros((ns,) * 4, np.complex128)
    for t1 in range(ns):
        for t2 in range(ns):
            for t3 in range(ns):
                for t4 in range(ns):
                    a, s1 = divmod(t1, 2)
                    b, s2 = divmod(t2, 2)
                    c, s3 = divmod(t3, 2)
                    d_, s4 = divmod(t4, 2)
                    if s1 == s3 and s2 == s4:
                        W[t1, t2, t3, t4] = Uo[a, b, c, d_]
    return 0.5 * (W - W.transpose(0, 1, 3, 2))


# ----------------------------------------------------------------------------
# models
# ----------------------------------------------------------------------------

def hubbard_square(t=1.0, tp=-0.25, U=3.0, *, Lq=8, nc=16, n_ff=5, filling=0.9,
                   mu=0.0, T_mu=0.02, name="hubbard") -> ModelSpec:
    """Spinful single-band square-lattice Hubbard model without SOC.

    eps(k) = -2t(cos kx + cos ky) - 4t' cos kx cos ky, H(k) = eps(k) * 1_2.
    """
    h = _Hops(2)
    one = np.eye(2)
    for R in [(1, 0), (0, 1)]:
        h.add_pair(R, -t * one)
    for R in [(1, 1), (1, -1)]:
        h.add_pair(R, -tp * one)
    R, tt = h.arrays()
    return ModelSpec(name, 2, R, tt, onsite_hubbard_vertex(U), ff_set(n_ff), Lq, nc,
                     mu=mu, filling=filling, T_mu=T_mu,
                     params=dict(t=t, tp=tp, U=U))


def rashba_hubbard(t=1.0, tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, *, Lq=24, nc=8, n_ff=9,
                   filling=0.0, T_mu=0.02, name="rashba") -> ModelSpec:
    """Lattice Rashba-Hubbard model, H(k) = eps(k) 1 + g(k).sigma (Eq. gen_Ham).

    g(k) = alpha (-sin ky, sin kx, 0): the lattice form of the paper's
    continuum g = (-ky, kx, 0) (Sec. 4), time-reversal odd.
    """
    h = _Hops(2)
    one = np.eye(2)
    for R in [(1, 0), (0, 1)]:
        h.add_pair(R, -t * one)
    for R in [(1, 1), (1, -1)]:
        h.add_pair(R, -tp * one)
    # -alpha sin(ky) sigma_x : t_(0,1) = (i alpha / 2) sigma_x
    h.add_pair((0, 1), (1j * alpha / 2.0) * SIGMA_X)
    # +alpha sin(kx) sigma_y : t_(1,0) = (-i alpha / 2) sigma_y
    h.add_pair((1, 0), (-1j * alpha / 2.0) * SIGMA_Y)
    R, tt = h.arrays()
    return ModelSpec(name, 2, R, tt, onsite_hubbard_vertex(U), ff_set(n_ff), Lq, nc,
                     mu=mu, filling=filling, T_mu=T_mu,
                     params=dict(t=t, tp=tp, alpha=alpha, U=U, mu=mu))


def rashba_bilayer(t=1.0, tp=-0.2, alpha=0.3, t_perp=0.4, U=2.5, mu=-0.9, *, Lq=8, nc=4, n_ff=5,
                   filling=0.0, T_mu=0.02, name="rashba_bilayer") -> ModelSpec:
    """Two Rashba-Hubbard layers (N_s = 4, index layer * 2 + spin) with opposite Rashba couplings, so that the
    pair is inversion symmetric, coupled by an onsite interlayer hopping t_perp.

    Each layer: eps(k) 1 + (-1)^layer g(k).sigma with the lattice Rashba g(k) = alpha (-sin ky, sin kx, 0);
    between the layers -t_perp (sigma_x in layer space) (x) 1_spin; an onsite Hubbard U within each layer.
    """
    h = _Hops(4)
    one = np.eye(2)
    Lz = np.diag([1.0, -1.0])
    for R in [(1, 0), (0, 1)]:
        h.add_pair(R, -t * np.eye(4))
    for R in [(1, 1), (1, -1)]:
        h.add_pair(R, -tp * np.eye(4))
    h.add_pair((0, 1), np.kron(Lz, (1j * alpha / 2.0) * SIGMA_X))
    h.add_pair((1, 0), np.kron(Lz, (-1j * alpha / 2.0) * SIGMA_Y))
    h.add((0, 0), -t_perp * np.kron(np.array([[0.0, 1.0], [1.0, 0.0]]), one))
    R, tt = h.arrays()
    W = np.zeros((4,) * 4, np.complex128)
    for t1 in range(4):
        for t2 in range(4):
            l1, s1 = divmod(t1, 2)
            l2, s2 = divmod(t2, 2)
            if l1 == l2:
                W[t1, t2, t1, t2] = U              # U delta(s1 s3) delta(s2 s4) within one layer
    V0 = 0.5 * (W - W.transpose(0, 1, 3, 2))
    return ModelSpec(name, 4, R, tt, V0, ff_set(n_ff), Lq, nc, mu=mu, filling=filling, T_mu=T_mu,
                     params=dict(t=t, tp=tp, alpha=alpha, t_perp=t_perp, U=U, mu=mu))


def t2g_soc(seed=0, lam=0.2, U=2.0, J=0.4, *, Lq=32, nc=6, n_ff=9, filling=4.0,
            T_mu=0.02, name="t2g") -> ModelSpec:
    """Three-orbital (yz, xz, xy) square-lattice model with atomic SOC.

    Hoppings (t_par, t_perp, t_xy) ~ U[0.5, 1] drawn in that order; yz hops
    t_par along y and t_perp along x, xz the mirror image, xy hops t_xy both
    ways.  SOC = (lam/2) sum_i L_i (x) sigma_i, (L_i)_ab = -i eps_iab.
    Kanamori interaction with U' = U - 2J, J_H = J_P = J.
    """
    rng = np.random.default_rng(seed)
    t_par, t_perp, t_xy = rng.uniform(0.5, 1.0, size=3)
    n_orb = 3
    ns = 6
    h = _Hops(ns)
    # orbital hopping amplitudes along x and y: (yz, xz, xy)
    tx = [t_perp, t_par, t_xy]
    ty = [t_par, t_perp, t_xy]
    for o in range(n_orb):
        P = np.zeros((n_orb, n_orb))
        P[o, o] = 1.0
        h.add_pair((1, 0), -tx[o] * np.kron(P, np.eye(2)))
        h.add_pair((0, 1), -ty[o] * np.kron(P, np.eye(2)))
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    soc = np.zeros((ns, ns), np.complex128)
    for i, s in enumerate([SIGMA_X, SIGMA_Y, SIGMA_Z]):
        Li = -1j * eps[i]
        soc += 0.5 * lam * np.kron(Li, s)
    h.add((0, 0), soc)
    R, tt = h.arrays()
    return ModelSpec(name, ns, R, tt, kanamori_vertex(n_orb, U, J), ff_set(n_ff), Lq, nc,
                     filling=filling, T_mu=T_mu,
                     params=dict(t_par=float(t_par), t_perp=float(t_perp), t_xy=float(t_xy),
                                 lam=lam, U=U, J=J, seed=seed))


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

FLOW_T0 = 10.0
FLOW_T_END = 0.02
FLOW_RTOL = 1e-6
FLOW_ATOL = 1e-8
FLOW_STOP = 50.0


def hubbard_q8_k16_ff5() -> ModelSpec:
    """Single-band Hubbard, t'=-0.25, n=0.45 per spin, U=3, N_ff=5, 8x8 q, 16x16 k per cell."""
    return hubbard_square(1.0, -0.25, 3.0, Lq=8, nc=16, n_ff=5, filling=0.9, T_mu=FLOW_T_END,
                          name="hubbard_q8_k16_ff5")


def rashba_q24_k8_ff9(seed: int = 0) -> ModelSpec:
    """Rashba-Hubbard, t'=-0.2, alpha=0.3, mu~U[-1.2,-0.6], U=2.5, N_ff=9, 24x24 q, 8x8 k per cell."""
    rng = np.random.default_rng(seed)
    mu = float(rng.uniform(-1.2, -0.6))
    return rashba_hubbard(1.0, -0.2, 0.3, 2.5, mu, Lq=24, nc=8, n_ff=9, name=f"rashba_q24_k8_ff9_s{seed}")


def t2g_q32_k6_ff9(seed: int = 0) -> ModelSpec:
    """t2g + atomic SOC (lam=0.2), Kanamori U=2, J=0.4, N_ff=9, 32x32 q, 6x6 k per cell."""
    return t2g_soc(seed, 0.2, 2.0, 0.4, Lq=32, nc=6, n_ff=9, filling=4.0, T_mu=FLOW_T_END,
                   name=f"t2g_q32_k6_ff9_s{seed}")


def rashba_batch(seed: int = 0, n: int = 64, nc: int = 8) -> List[ModelSpec]:
    """64 uneven Rashba/Hubbard instances (t', alpha, U, Lq, N_ff, mu drawn per instance)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        tp = float(rng.uniform(-0.3, 0.0))
        alpha = float(rng.uniform(0.0, 0.4))
        U = float(rng.uniform(1.5, 3.5))
        Lq = int(rng.choice([16, 24, 32, 48]))
        n_ff = int(rng.choice([5, 9, 13]))
        mu = float(rng.uniform(-1.2, -0.6))
        out.append(rashba_hubbard(1.0, tp, alpha, U, mu, Lq=Lq, nc=nc, n_ff=n_ff,
                                  name=f"rashba_batch_{i}"))
    return out


def rashba_family_draw(rng: np.random.Generator, Lq: int = 24, nc: int = 8, n_ff: int = 9,
                   U: float = 2.5) -> ModelSpec:
    """One draw of the Rashba-Hubbard family (t', alpha, mu) used to train the loop surrogate."""
    tp = float(rng.uniform(-0.3, 0.0))
    alpha = float(rng.uniform(0.0, 0.4))
    mu = float(rng.uniform(-1.2, -0.6))
    return rashba_hubbard(1.0, tp, alpha, U, mu, Lq=Lq, nc=nc, n_ff=n_ff, name="rashba_family")


def random_state(spec: ModelSpec, seed: int, scale: float = 0.3, hermitian: bool = True) -> np.ndarray:
    """Seeded random exchange-propagator state [2][Nq][M][M] (P then C), Hermitian per q.

    Used only as a generic input for component parity (projections, V.L.V);
    it is not a physical state.
    """
    rng = np.random.default_rng(seed)
    M, Nq = spec.M, spec.Nq
    X = (rng.standard_normal((2, Nq, M, M)) + 1j * rng.standard_normal((2, Nq, M, M))) * scale
    if hermitian:
        X = 0.5 * (X + np.conj(np.swapaxes(X, -1, -2)))
    return np.ascontiguousarray(X, dtype=np.complex128)
