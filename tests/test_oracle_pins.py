"""Pins of the CPU oracle against things other than itself (CPU only).

Each test names the passage of the paper it follows and the class of mistake
it would catch.  The pins are:
  * library routines on special cases (numpy eigh, mpmath derivatives);
  * an independent full-momentum brute-force fRG (oracle/bruteforce.py), exact
    for the complete form-factor set on a 4x4 torus;
  * the paper's closed-form particle-particle solution (Sec. 4, Eq. sol_spin);
  * second-order perturbation theory (the bubble itself, not its derivative);
  * the q -> 0 compressibility of the single-band particle-hole loop;
  * hermiticity, SU(2) and bookkeeping invariants;
  * the momentum-shell regulator of Eq. def_lmp: its defining properties, finite differences in Lambda of
    chi chi F (F from Eqs. disc_2a/2b written out here), the closed forms with Lambda as the flow variable, and
    its Lambda -> 0 limit against the temperature-flow bubble.
"""
import numpy as np
import pytest

import oracle
from oracle import bruteforce
from paper_1710_08830_gb300 import inputs


# ---------------------------------------------------------------- eigensolver (step 1)

@pytest.mark.parametrize("n", [2, 3, 6])
def test_eigh_matches_numpy(n):
    rng = np.random.default_rng(n)
    for _ in range(20):
        A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        A = A + A.conj().T
        E, U = oracle.eigh(A)
        assert np.allclose(E, np.linalg.eigvalsh(A), atol=1e-13, rtol=0)
        assert np.abs(A @ U - U * E).max() < 1e-13 * max(1.0, np.abs(A).max())
        assert np.abs(U.conj().T @ U - np.eye(n)).max() < 1e-13


def test_eigh_degenerate_is_identity():
    """Spin-degenerate bands (no SOC): H = eps * 1 must give U = 1 exactly."""
    E, U = oracle.eigh(np.eye(2) * -1.3)
    assert np.array_equal(U, np.eye(2))
    assert np.array_equal(E, [-1.3, -1.3])


def test_bands_match_numpy():
    spec = inputs.t2g_soc(seed=3, Lq=4, nc=1)
    o = oracle.Oracle(spec, mu=0.0)
    L = spec.Lf
    kx, ky = np.divmod(np.arange(spec.Nk), L)
    H = np.zeros((spec.Nk, 6, 6), complex)
    for R, t in zip(spec.hop_R, spec.hop_t):
        H += np.exp(2j * np.pi * (kx * R[0] + ky * R[1]) / L)[:, None, None] * t
    assert np.allclose(o.E, np.linalg.eigvalsh(H), atol=1e-12)
    res = np.einsum("kij,kjl->kil", H, o.U) - o.U * o.E[:, None, :]
    assert np.abs(res).max() < 1e-12


# ---------------------------------------------------------------- Fermi weights (Eqs. disc_2a/2b)

mp = pytest.importorskip("mpmath")


def _mp_f(e, T):
    return 1 / (mp.exp(e / T) + 1)


@pytest.mark.parametrize("e,T", [(-0.3, 0.1), (0.05, 0.1), (0.2, 0.1), (1.0, 0.1), (0.01, 0.02), (-3.0, 0.05)])
def test_fermi_derivatives_vs_mpmath(e, T):
    mp.mp.dps = 40
    f, g, gp = oracle.fermi(e, T)
    ef, Tf = mp.mpf(e), mp.mpf(T)
    assert abs(f - float(_mp_f(ef, Tf))) < 1e-15
    g_ref = float(mp.diff(lambda t: _mp_f(ef, t), Tf))
    gp_ref = float(mp.diff(lambda x: mp.diff(lambda t: _mp_f(x, t), Tf), ef))
    assert abs(g - g_ref) <= 1e-12 * max(1.0, abs(g_ref))
    assert abs(gp - gp_ref) <= 1e-11 * max(1.0, abs(gp_ref))


@pytest.mark.parametrize("e1,e2,T", [(0.3, -0.1, 0.1), (0.05, 0.05 + 3e-7, 0.1), (0.05, 0.05 + 2e-6, 0.1),
                                     (-0.2, 0.2 + 1e-9, 0.05), (0.12, -0.12 + 4e-6, 0.05), (1.5, 1.5, 0.3)])
def test_pair_weights_vs_mpmath(e1, e2, T):
    """dF^-/dT and dF^+/dT, including the degenerate switch, against 40-digit arithmetic."""
    mp.mp.dps = 40
    a, b, t = mp.mpf(e1), mp.mpf(e2), mp.mpf(T)

    def Fm(tt):
        return (1 - _mp_f(a, tt) - _mp_f(b, tt)) / (a + b) if a + b != 0 else -mp.diff(lambda x: _mp_f(x, tt), a)

    def Fp(tt):
        return (_mp_f(a, tt) - _mp_f(b, tt)) / (a - b) if a != b else mp.diff(lambda x: _mp_f(x, tt), a)

    wm_ref = float(mp.diff(Fm, t))
    wp_ref = float(mp.diff(Fp, t))
    assert abs(oracle.wm(e1, e2, T) - wm_ref) <= 1e-9 * abs(wm_ref) + 1e-12
    assert abs(oracle.wp(e1, e2, T) - wp_ref) <= 1e-9 * abs(wp_ref) + 1e-12
    assert abs(oracle.Fm(e1, e2, T) - float(Fm(t))) <= 1e-10 * abs(float(Fm(t))) + 1e-13
    assert abs(oracle.Fp(e1, e2, T) - float(Fp(t))) <= 1e-10 * abs(float(Fp(t))) + 1e-13


# ---------------------------------------------------------------- bookkeeping (Sec. 2)

@pytest.mark.parametrize("nff,nd", [(5, 13), (9, 25), (13, 41)])
def test_delta_list_counts(nff, nd):
    spec = inputs.rashba_hubbard(Lq=16, nc=1, n_ff=nff)
    o = oracle.Oracle(spec)
    ff = spec.ff_R
    ref = sorted({(int(a[0] - b[0]), int(a[1] - b[1])) for a in ff for b in ff})
    assert o.nd == nd
    assert [tuple(d) for d in o.deltas] == ref


@pytest.mark.parametrize("L,nff", [(8, 5), (24, 9), (16, 13)])
def test_form_factor_orthonormality(L, nff):
    """(1/N) sum_k f_R(k) f*_R'(k) = delta_RR' on the meshes used (Sec. 2)."""
    ff = inputs.ff_set(nff)
    kx, ky = np.divmod(np.arange(L * L), L)
    f = np.exp(-2j * np.pi * (np.outer(kx, ff[:, 0]) + np.outer(ky, ff[:, 1])) / L)
    G = f.T @ f.conj() / (L * L)
    assert np.abs(G - np.eye(nff)).max() < 1e-13


def test_mu_bisection_hits_filling():
    """mu by bisection of the filling (reading R11), checked with a density computed here from numpy's eigenvalues
    of H(k) and the logistic form of f, n(mu) = (1/Nk) sum_{k,l} 1/(1 + e^{(E_l(k) - mu)/T}); also for the t2g
    model at 4 electrons in 6 states."""
    from scipy.special import expit
    for spec in (inputs.hubbard_square(Lq=4, nc=4, filling=0.9, T_mu=0.05),
                 inputs.t2g_soc(seed=2, Lq=4, nc=2, n_ff=1, filling=4.0, T_mu=0.05)):
        o = oracle.Oracle(spec)
        L = spec.Lf
        kx, ky = np.divmod(np.arange(spec.Nk), L)
        H = np.zeros((spec.Nk, spec.n_s, spec.n_s), complex)
        for R, t in zip(spec.hop_R, spec.hop_t):
            H += np.exp(2j * np.pi * (kx * R[0] + ky * R[1]) / L)[:, None, None] * t
        E = np.linalg.eigvalsh(H)
        n = lambda mu: float(expit(-(E - mu) / spec.T_mu).sum(axis=1).mean())
        assert abs(n(o.mu) - spec.filling) < 1e-12
        for mu in (o.mu - 0.3, o.mu + 0.2):
            assert abs(o.density(mu, spec.T_mu) - n(mu)) < 1e-12


# ---------------------------------------------------------------- brute-force exactness (Secs. 3.1-3.3)

def _complete_spec(model="rashba"):
    if model == "rashba":
        spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.4, U=2.0, mu=-0.7, Lq=4, nc=1)
    else:
        spec = inputs.hubbard_square(tp=-0.25, U=2.0, Lq=4, nc=1, filling=0.0, mu=-0.5)
    return spec.with_(ff_R=inputs.ff_complete(4))


@pytest.mark.parametrize("model,T", [("rashba", 0.5), ("rashba", 0.07), ("hubbard", 0.2)])
def test_rhs_equals_full_momentum_rge(model, T):
    """Complete form factors on a 4x4 torus: the channel-decomposed RHS (loops, all four
    projection formulas, V.L.V with c_P = 1, c_C = 2) equals the projections of the
    unprojected one-loop terms Phi^pp and Phi^{ph,c} (Eqs. eq_phipp, eq_phiphd)."""
    spec = _complete_spec(model)
    o = oracle.Oracle(spec)
    bf = bruteforce.Torus(spec, o.mu)
    P, C, _, _ = bf.random_consistent_state(np.random.default_rng(7))
    V = bf.vertex_from_channels(spec.V0, P, C)
    dP, dC = bf.channel_rhs(V, T)
    d, _ = o.rhs(T, np.stack([P, C]), 3)
    scale = max(np.abs(dP).max(), np.abs(dC).max())
    assert np.abs(d[0] - dP).max() < 1e-12 * scale
    assert np.abs(d[1] - dC).max() < 1e-12 * scale


@pytest.mark.parametrize("model", ["t2g", "bilayer"])
def test_rhs_equals_full_momentum_rge_multiorbital(model):
    """The same exactness with more than two spin-orbitals: the three-orbital t2g model with atomic SOC and the
    Kanamori vertex (N_s = 6, M = 324) and the Rashba bilayer (N_s = 4, M = 144); complete form factors on a 3x3
    torus, a consistent random state, T = 0.3.  It pins the oracle's loops, projections and products for
    N_s = 4 and 6."""
    if model == "t2g":
        spec = inputs.t2g_soc(seed=1, Lq=3, nc=1, n_ff=1, filling=4.0, T_mu=0.1)
    else:
        spec = inputs.rashba_bilayer(Lq=3, nc=1)
    spec = spec.with_(ff_R=inputs.ff_complete(3))
    o = oracle.Oracle(spec)
    bf = bruteforce.Torus(spec, o.mu)
    P, C, _, _ = bf.random_consistent_state(np.random.default_rng(7))
    dP, dC = bf.channel_rhs(bf.vertex_from_channels(spec.V0, P, C), 0.3)
    d, _ = o.rhs(0.3, np.stack([P, C]), 3)
    scale = max(np.abs(dP).max(), np.abs(dC).max())
    assert scale > 0.1
    assert np.abs(d[0] - dP).max() < 1e-12 * scale
    assert np.abs(d[1] - dC).max() < 1e-12 * scale


@pytest.mark.parametrize("model,mask", [("rashba", 3), ("rashba", 1), ("rashba", 2), ("t2g", 3)])
def test_rhs_at_equals_rows_of_the_full_rhs(model, mask):
    """The sampled right-hand side (the oracle's restriction of one evaluation to listed transfer momenta, used
    for bounded CPU timings) equals the listed rows of the full right-hand side, which the brute-force pins above
    tie to the paper's equations: loops at the listed momenta only, projections from the whole-mesh Fourier
    transform, c A L A with c_P = 1, c_C = 2 (Eq. RGE_spin and the C equation).  A swapped operand order, c_C = 1
    or a momentum taken from the list position instead of the list fails it."""
    if model == "rashba":
        spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=5, nc=2, n_ff=9)
        qs = [3, 0, 17, 24]
    else:
        spec = inputs.t2g_soc(seed=2, Lq=4, nc=1, n_ff=5, filling=4.0, T_mu=0.05)
        qs = [9, 1, 14]
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=11, scale=0.3)
    full, _ = o.rhs(0.2, st, mask)
    part = o.rhs_at(0.2, st, qs, mask)
    for ch in (0, 1):
        ref = full[ch][qs]
        if (mask >> ch) & 1:
            assert np.abs(ref).max() > 1e-3
            assert np.abs(part[ch] - ref).max() <= 1e-13 * np.abs(ref).max()
        else:
            assert not np.any(part[ch]) and not np.any(ref)


def test_flow_critical_at_start():
    """A flow whose bare vertex already exceeds the stop value (max|A| = U/2 at T0) is critical at T0: no step,
    Lambda_c = T0 (reading R14); just below that value it runs."""
    spec = inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=3.2, mu=-0.8, Lq=4, nc=2, n_ff=5)
    o = oracle.Oracle(spec)
    _, r = o.flow(T0=10.0, stop=1.5)
    assert r["crossed"] == 1 and r["n_steps"] == 0 and r["n_rhs"] == 1
    assert r["Tc"] == pytest.approx(10.0) and r["amax"] == pytest.approx(1.6)
    _, r2 = o.flow(T0=10.0, T_end=2.0, stop=1.7)
    assert r2["n_steps"] > 0 and r2["Tc"] < 10.0


def test_flow_equals_full_momentum_flow():
    """Same exactness for a whole flow: fixed-step RK4 of the full vertex vs the
    (P, C) flow, compared on the reconstructed vertex V0 + V^P + V^C + V^D."""
    spec = _complete_spec("rashba")
    o = oracle.Oracle(spec)
    bf = bruteforce.Torus(spec, o.mu)
    state, res = o.flow(T0=2.0, T_end=0.5, chmask=3, fixed_n=3)
    V_tu = bf.vertex_from_channels(spec.V0, state[0], state[1])
    V_bf = bf.flow_rk4(spec.V0, 2.0, 0.5, 3)
    assert np.abs(V_tu - V_bf).max() < 1e-12 * np.abs(V_bf).max()
    assert np.abs(V_bf - spec.V0[None, None, None]).max() > 1e-2   # the flow did something


@pytest.mark.parametrize("Lq,nff", [(8, 5), (6, 9)])
def test_truncated_projections_vs_double_k_sums(Lq, nff):
    """Eq. proj_PD and the D->P, P->C, D->C gathers against the defining double
    k-sums (Eq. def_P and analogues) for exchange propagators supported on a
    truncated bond set (8x8 and 6x6 coarse meshes; on the 6x6 torus shifted bonds
    with |x| = 3 wrap, so the modular R'' arithmetic is exercised too)."""
    spec = inputs.rashba_hubbard(Lq=Lq, nc=1, n_ff=nff, mu=-0.8)
    o = oracle.Oracle(spec)
    bf = bruteforce.Torus(spec, o.mu)
    st = inputs.random_state(spec, seed=11, hermitian=False)
    A, _ = o.project(st, 3)
    V0 = spec.V0
    zero = np.zeros_like(st[0])
    # P-channel: A_P - P = P^[V0] + P^[V^C + V^D]
    VCD = bf.vertex_from_channels(V0, zero, st[1], which="C") + bf.vertex_from_channels(V0, zero, st[1], which="CD")
    ref_P = bf.project_P(VCD + V0[None, None, None])
    assert np.abs(A[0] - st[0] - ref_P).max() < 1e-12
    # C-channel: A_C - C = C^[V0] + C^[V^P] + C^[V^D]
    VP = bf.vertex_from_channels(V0, st[0], zero, which="P")
    VD = bf.vertex_from_channels(V0, zero, st[1], which="CD")
    ref_C = bf.project_C(VP + VD + V0[None, None, None])
    assert np.abs(A[1] - st[1] - ref_C).max() < 1e-12


# ---------------------------------------------------------------- closed forms (Sec. 4)

def _pair_structure(ns):
    A = np.zeros((ns,) * 4)
    for a in range(ns):
        for b in range(ns):
            for c in range(ns):
                for d in range(ns):
                    A[a, b, c, d] = (a == c) * (b == d) - (a == d) * (b == c)
    return A


@pytest.mark.parametrize("alpha,tp,reg", [(0.3, -0.2, 0), (0.0, -0.25, 0), (0.3, -0.2, 1)])
def test_particle_particle_closed_form(alpha, tp, reg):
    """Eq. sol_spin: two-band TRS model, onsite U, P-only flow.  P stays local,
    P = -(g+U)/2 (d13 d24 - d14 d23) with g = -U/(1 + U [B(s) - B(s0)]), B from the
    bubble F^- itself (not its T-derivative), so the integrator is pinned too.  With the momentum-shell
    regulator (reg = 1) the scale s is Lambda and the bubble is chi chi F^- at the fixed temperature."""
    U = 2.5
    spec = inputs.rashba_hubbard(tp=tp, alpha=alpha, U=U, mu=-0.9, Lq=6, nc=2, n_ff=5).with_(regulator=reg, T_reg=0.1)
    o = oracle.Oracle(spec)
    T0, T1 = 10.0, 0.3
    state, res = o.flow(T0=T0, T_end=T1, rtol=1e-10, atol=1e-12, chmask=1, stop=1e9)
    assert res["T_last"] == pytest.approx(T1)
    ns = 2
    d0 = [i for i, (x, y) in enumerate(o.deltas) if x == 0 and y == 0][0]

    def Bbar(T):
        L = o.loops(T, 0, kind=1)[:, d0].reshape(spec.Nq, ns, ns, ns, ns)   # [s][t2][t1][t4][t3]
        B = np.zeros(spec.Nq, complex)
        for t1 in range(ns):
            for t2 in range(ns):
                B += 0.5 * (L[:, t2, t1, t2, t1] - L[:, t2, t1, t1, t2])
        return B

    g = -U / (1 + U * (Bbar(T1) - Bbar(T0)))
    A = _pair_structure(ns)
    expect = np.zeros((spec.Nq, spec.M, spec.M), complex)
    for s1 in range(ns):
        for s2 in range(ns):
            for s3 in range(ns):
                for s4 in range(ns):
                    expect[:, s1 * ns + s2, s4 * ns + s3] = -0.5 * (g + U) * A[s1, s2, s3, s4]
    assert np.abs(state[0] - expect).max() < 1e-9
    assert np.abs(state[1]).max() == 0.0


@pytest.mark.parametrize("stop", [2.0, 4.0])
def test_critical_scale_of_the_ladder(stop):
    """Lambda_c as reported (reading R14): for the P-only ladder with an attractive onsite U (the Cooper channel),
    A_P(s) = V0 + P = -(g_T(s) / 2) (d13 d24 - d14 d23) at R = R' = 0 by Eq. sol_spin, so max|A| = max_s |g_T(s)| / 2
    with g_T = -U / (1 + U [B(T) - B(T0)]).  The closed form's crossing of the stop value (bisection in ln T) equals the
    flow's Lambda_c, a linear interpolation in ln T between the accepted states around the crossing, to 1e-3 (one
    step is about 6% in T, so reporting either end of it fails)."""
    U, ns = -2.5, 2
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=U, mu=-0.9, Lq=6, nc=2, n_ff=5)
    o = oracle.Oracle(spec)
    d0 = [i for i, (x, y) in enumerate(o.deltas) if x == 0 and y == 0][0]

    def Bbar(T):
        L = o.loops(T, 0, kind=1)[:, d0].reshape(spec.Nq, ns, ns, ns, ns)   # [s][t2][t1][t4][t3]
        return sum(0.5 * (L[:, t2, t1, t2, t1] - L[:, t2, t1, t1, t2]) for t1 in range(ns) for t2 in range(ns))

    B0 = Bbar(10.0)
    amax = lambda lnT: np.abs(-U / (1 + U * (Bbar(np.exp(lnT)) - B0))).max() / 2
    lo, hi = np.log(1e-3), np.log(10.0)
    assert amax(lo) > stop > amax(hi)
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if amax(mid) > stop else (lo, mid)
    _, res = o.flow(T0=10.0, T_end=1e-3, rtol=1e-10, atol=1e-12, chmask=1, stop=stop)
    assert res["crossed"] == 1 and res["Tc"] == pytest.approx(np.exp(0.5 * (lo + hi)), rel=1e-3)


@pytest.mark.parametrize("reg", [0, 1])
def test_second_order_perturbation_theory(reg):
    """At O(U^2): P(T) = V0 [B^-(T) - B^-(T0)] V0 and C(T) = 2 V0 [B^+(T) - B^+(T0)] V0 with
    the bubble matrices built from F^-, F^+ directly (chi chi F^-/+ with the momentum shell, reg = 1);
    the remainder is O(U^3)."""
    base = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, mu=-0.8, Lq=4, nc=2, n_ff=5).with_(regulator=reg, T_reg=0.1)
    T0, T1 = 10.0, 0.4
    res = []
    for U in (0.2, 0.1):
        spec = base.with_(V0=inputs.onsite_hubbard_vertex(U))
        o = oracle.Oracle(spec)
        st, _ = o.flow(T0=T0, T_end=T1, rtol=1e-11, atol=1e-14, chmask=3, stop=1e9)
        ns, nff, M = spec.n_s, spec.n_ff, spec.M
        d_of = {tuple(d): i for i, d in enumerate(o.deltas)}
        V0P = np.zeros((M, M), complex)
        V0C = np.zeros((M, M), complex)
        for a in range(ns):
            for b in range(ns):
                for c in range(ns):
                    for d in range(ns):
                        V0P[a * ns + b, d * ns + c] = spec.V0[a, b, c, d]
                        V0C[a * ns + c, d * ns + b] = spec.V0[a, b, c, d]

        def expand(Lc):
            out = np.zeros((spec.Nq, M, M), complex)
            for i1 in range(nff):
                for i2 in range(nff):
                    di = d_of[tuple(spec.ff_R[i1] - spec.ff_R[i2])]
                    out[:, i1 * ns * ns:(i1 + 1) * ns * ns, i2 * ns * ns:(i2 + 1) * ns * ns] = Lc[:, di]
            return out

        BP = expand(o.loops(T1, 0, 1) - o.loops(T0, 0, 1))
        BC = expand(o.loops(T1, 1, 1) - o.loops(T0, 1, 1))
        P2 = V0P @ BP @ V0P
        C2 = 2 * V0C @ BC @ V0C
        res.append((np.abs(st[0] - P2).max(), np.abs(st[1] - C2).max(), np.abs(P2).max()))
    (p1, c1, s1), (p2, c2, s2) = res
    assert s1 / s2 == pytest.approx(4.0, rel=1e-6)        # the O(U^2) part itself
    assert 6.0 < p1 / p2 < 10.0 and 6.0 < c1 / c2 < 10.0  # the remainder is cubic
    assert p1 < 0.05 * s1


def test_compressibility_limit():
    """Single band: [L^+_{up up up up}(u=0)]_{R1=R2} = (1/Nk) sum_k d/dT F^+(e,e) = -d/dT d/dmu n_up(mu,T);
    pins the degenerate branch of the particle-hole weight."""
    spec = inputs.hubbard_square(tp=-0.25, Lq=4, nc=8, filling=0.0, mu=-0.6)
    o = oracle.Oracle(spec)
    T = 0.15
    Lc = o.loops(T, 1)
    d0 = [i for i, (x, y) in enumerate(o.deltas) if x == 0 and y == 0][0]
    lhs = Lc[0, d0, 0, 0].real
    L = spec.Lf
    kx, ky = np.divmod(np.arange(spec.Nk), L)
    kx, ky = 2 * np.pi * kx / L, 2 * np.pi * ky / L
    eps = -2 * (np.cos(kx) + np.cos(ky)) + 1.0 * np.cos(kx) * np.cos(ky)   # t=1, t'=-0.25

    def n(mu, T):
        return np.mean(1.0 / (np.exp((eps - mu) / T) + 1.0))

    h = 2e-3
    w = [1, -8, 8, -1]
    off = [-2, -1, 1, 2]
    dd = 0.0
    for wi, oi in zip(w, off):
        for wj, oj in zip(w, off):
            dd += wi * wj * n(-0.6 + oi * h, T + oj * h)
    dd /= (12 * h) ** 2
    assert lhs == pytest.approx(-dd, rel=1e-6)
    assert abs(Lc[0, d0, 0, 0].imag) < 1e-14


# ---------------------------------------------------------------- symmetries

def _expand_all(spec, o, Lc):
    ns2 = spec.n_s ** 2
    d_of = {tuple(d): i for i, d in enumerate(o.deltas)}
    out = np.zeros((spec.Nq, spec.M, spec.M), complex)
    for i1 in range(spec.n_ff):
        for i2 in range(spec.n_ff):
            out[:, i1 * ns2:(i1 + 1) * ns2, i2 * ns2:(i2 + 1) * ns2] = Lc[:, d_of[tuple(spec.ff_R[i1] - spec.ff_R[i2])]]
    return out


def test_hermiticity_of_loops_and_flow():
    """Sec. 2 (hermiticity of the projections): loop matrices, A and the flowing P, C are Hermitian."""
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=4, nc=2, n_ff=9)
    o = oracle.Oracle(spec)
    for which in (0, 1):
        Lm = _expand_all(spec, o, o.loops(0.2, which))
        assert np.abs(Lm - np.conj(np.swapaxes(Lm, 1, 2))).max() < 1e-14 * np.abs(Lm).max()
    st, _ = o.flow(T0=10.0, T_end=0.3, chmask=3, stop=1e9)
    A, _ = o.project(st, 3)
    for X in (st[0], st[1], A[0], A[1]):
        assert np.abs(X - np.conj(np.swapaxes(X, 1, 2))).max() < 1e-12 * np.abs(X).max()


def test_su2_relations_without_soc():
    """Zero SOC: X_{uuuu} = X_{udud} + X_{uddu}, spin conservation, up/down symmetry, and the decoupling of
    singlet and triplet pairs (P) and of charge and spin (C)."""
    spec = inputs.hubbard_square(tp=-0.25, U=3.0, Lq=4, nc=2, filling=0.0, mu=-0.7)
    o = oracle.Oracle(spec)
    st, _ = o.flow(T0=10.0, T_end=0.3, chmask=3, stop=1e9)
    nff = spec.n_ff
    P = st[0].reshape(spec.Nq, nff, 2, 2, nff, 2, 2)   # [q][R][s1][s2][R'][s4][s3]
    C = st[1].reshape(spec.Nq, nff, 2, 2, nff, 2, 2)   # [q][R][s1][s3][R'][s4][s2]
    Pt = lambda a, b, c, d: P[:, :, a, b, :, d, c]
    Ct = lambda a, b, c, d: C[:, :, a, c, :, d, b]
    for X in (Pt, Ct):
        assert np.abs(X(0, 0, 0, 0) - X(0, 1, 0, 1) - X(0, 1, 1, 0)).max() < 1e-12
        assert np.abs(X(0, 0, 0, 0) - X(1, 1, 1, 1)).max() < 1e-12
        for a in range(2):
            for b in range(2):
                for c in range(2):
                    for d in range(2):
                        if a + b != c + d:
                            assert np.abs(X(a, b, c, d)).max() < 1e-13
    assert np.abs(Pt(0, 1, 0, 1)).max() > 1e-3 and np.abs(Ct(0, 1, 0, 1)).max() > 1e-3
    # singlet and triplet pairs decouple in P; charge and spin decouple in C.  Pair index (a, b) = 2 a + b over
    # (up, down); P rows carry (s1, s2) and columns (s4, s3), C rows (s1, s3) and columns (s4, s2).
    r = 1 / np.sqrt(2)
    pp = np.array([[0, r, -r, 0],                       # singlet (ud - du) / sqrt 2
                   [1, 0, 0, 0], [0, r, r, 0], [0, 0, 0, 1]])   # triplets uu, (ud + du) / sqrt 2, dd
    ph = np.array([[r, 0, 0, r],                        # charge (uu + dd) / sqrt 2
                   [r, 0, 0, -r], [0, 1, 0, 0], [0, 0, 1, 0]])  # spin: (uu - dd) / sqrt 2, ud, du
    for X, B in ((st[0], pp), (st[1], ph)):
        Bf = np.kron(np.eye(nff), B)
        Y = (Bf @ X @ Bf.conj().T).reshape(spec.Nq, nff, 4, nff, 4)
        assert np.abs(Y[:, :, 0, :, 1:]).max() < 1e-13 and np.abs(Y[:, :, 1:, :, 0]).max() < 1e-13
        assert np.abs(Y[:, :, 0, :, 0]).max() > 1e-3 and np.abs(Y[:, :, 1:, :, 1:]).max() > 1e-3


# The square-lattice point group C4v as integer matrices acting on (x, y): the four rotations, then the four mirrors.
_C4V = [np.array(g) for g in (((1, 0), (0, 1)), ((0, -1), (1, 0)), ((-1, 0), (0, -1)), ((0, 1), (-1, 0)),
                              ((-1, 0), (0, 1)), ((1, 0), (0, -1)), ((0, 1), (1, 0)), ((0, -1), (-1, 0)))]
_SX = np.array([[0, 1], [1, 0]], complex)
_SY = np.array([[0, -1j], [1j, 0]])
_SZ = np.diag([1.0 + 0j, -1.0])


def _spin_rep(g):
    """SU(2) matrix of a C4v element acting on a spin (an axial vector): a rotation by theta about z is
    exp(-i theta/2 sigma_z); a mirror acts on an axial vector as the rotation by pi about its normal n."""
    if round(np.linalg.det(g)) == 1:
        th = np.arctan2(g[1, 0], g[0, 0])
        return np.diag([np.exp(-0.5j * th), np.exp(0.5j * th)])
    w, v = np.linalg.eigh(g.astype(float))
    n = v[:, np.argmin(w)]                                  # the mirror's normal (eigenvalue -1)
    return -1j * (n[0] * _SX + n[1] * _SY)


def _h_of_k(spec, k):
    return np.einsum("h,hab->ab", np.exp(1j * (spec.hop_R @ k)), spec.hop_t)


def _orbital_rep(g):
    """Representation of a C4v element on the t2g orbitals (yz, xz, xy), polar quadratic forms in (x, y, z):
    (O_g f)(r) = f(G^-1 r) with G = g (+) 1 maps the form Q_j to G Q_j G^T = sum_i D_ij Q_i."""
    G = np.eye(3)
    G[:2, :2] = g
    Q = []
    for a, b in ((1, 2), (0, 2), (0, 1)):
        q = np.zeros((3, 3))
        q[a, b] = q[b, a] = 1.0
        Q.append(q)
    return np.array([[np.sum(Qi * (G @ Qj @ G.T)) / 2.0 for Qj in Q] for Qi in Q])


def _check_setup(spec, o, reps, theta):
    """The Hamiltonian of the descriptor reproduces the oracle's bands and has the symmetries used below."""
    rng = np.random.default_rng(3)
    Lf = spec.Lq * spec.nc
    for idx in (0, 7, Lf + 2):
        k = 2 * np.pi * np.array([idx // Lf, idx % Lf]) / Lf
        assert np.allclose(np.linalg.eigvalsh(_h_of_k(spec, k)), o.E[idx], atol=1e-12)
    for g, W in zip(_C4V, reps):
        for _ in range(3):
            k = rng.uniform(-np.pi, np.pi, 2)
            assert np.allclose(_h_of_k(spec, g @ k), W @ _h_of_k(spec, k) @ W.conj().T, atol=1e-13)
    k = rng.uniform(-np.pi, np.pi, 2)
    assert np.allclose(_h_of_k(spec, -k), theta @ _h_of_k(spec, k).conj() @ theta.conj().T, atol=1e-13)


def _check_covariance(spec, Y, w, reps, theta):
    """Y: [Nq][M][M] of channel w (0 = P, 1 = C); the group action written out from the definitions:
        Y(g q)[(g R1, a), (g R2, b)] = (V Y(q) V^+)[(R1, a), (R2, b)],  Y(-q) = V' Y(q)^* V'^+,
    with the pair representation V = W (x) W for the P pair (t2, t1) (two eigenvector indices) and
    W (x) W^* for the C pair (t1, t2) (one U and one U^* index); V' likewise with Theta."""
    scale = np.abs(Y).max()
    assert scale > 1e-3
    bond = {tuple(r): i for i, r in enumerate(spec.ff_R)}
    Lq, ns2, one = spec.Lq, spec.n_s ** 2, np.eye(spec.n_ff)

    def qmap(q, g):
        x, y = g @ np.array([q // Lq, q % Lq])
        return (x % Lq) * Lq + (y % Lq)

    def pair_rep(Wm):
        return np.kron(Wm, Wm) if w == 0 else np.kron(Wm, Wm.conj())

    for g, W in zip(_C4V, reps):
        V = np.kron(one, pair_rep(W))                        # the pair representation on every bond block
        rows = [bond[tuple(g @ r)] * ns2 + a for r in spec.ff_R for a in range(ns2)]   # (R, a) -> (g R, a)
        for q in range(spec.Nq):
            lhs = Y[qmap(q, g)][np.ix_(rows, rows)]
            assert np.abs(lhs - V @ Y[q] @ V.conj().T).max() < 1e-12 * scale, (w, g.tolist(), q)
    Vt = np.kron(one, pair_rep(theta))
    for q in range(spec.Nq):
        rhs = Vt @ Y[q].conj() @ Vt.conj().T
        assert np.abs(Y[qmap(q, -np.eye(2, dtype=int))] - rhs).max() < 1e-12 * scale, (w, q)


def test_point_group_and_time_reversal_rashba():
    """The Rashba model (Sec. 4) has C4v with the spins rotating along, H(gk) = W_g H(k) W_g^+, and time
    reversal, H(-k) = Theta H(k)^* Theta^+ with Theta = i sigma_y.  With U(gk) = W_g U(k) in the projectors
    rho = U U^+ of Eq. loop_orbital and plain-wave form factors (g k . g R = k . R), both loop channels
    transform as stated in _check_covariance; the flowing P and C, built from them by Eq. RGE_spin and the
    projections, transform alike: checked at every momentum of a 5x5 mesh at T = 0.3 after a flow from T0 = 10.
    Swapping the C pair rule for the P rule, dropping the bond permutation or taking another element's W
    fails it."""
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=5, nc=2, n_ff=9)
    o = oracle.Oracle(spec)
    reps, theta = [_spin_rep(g) for g in _C4V], 1j * _SY
    _check_setup(spec, o, reps, theta)
    st, _ = o.flow(T0=10.0, T_end=0.3, chmask=3, stop=1e9)
    for w in (0, 1):
        _check_covariance(spec, _expand_all(spec, o, o.loops(0.3, w)), w, reps, theta)
        _check_covariance(spec, st[w], w, reps, theta)


def test_point_group_and_time_reversal_bilayer():
    """The N_s = 4 Rashba bilayer: C4v acts on the spins of both layers alike, W_g = 1_layer (x) S_g (the two
    layers' opposite Rashba couplings are each invariant), time reversal is 1 (x) i sigma_y.  Loops of both
    channels and the flowing P, C after a flow from T0 = 10 to T = 0.3 on a 5x5 mesh."""
    spec = inputs.rashba_bilayer(Lq=5, nc=2, n_ff=5)
    o = oracle.Oracle(spec)
    reps = [np.kron(np.eye(2), _spin_rep(g)) for g in _C4V]
    theta = np.kron(np.eye(2), 1j * _SY)
    _check_setup(spec, o, reps, theta)
    st, _ = o.flow(T0=10.0, T_end=0.3, chmask=3, stop=1e9)
    for w in (0, 1):
        _check_covariance(spec, _expand_all(spec, o, o.loops(0.3, w)), w, reps, theta)
        _check_covariance(spec, st[w], w, reps, theta)


def test_point_group_and_time_reversal_t2g():
    """The t2g model with atomic SOC: C4v acts on orbitals and spins, W_g = D_g (x) S_g (orbitals as polar
    quadratic forms, spins as an axial vector), and time reversal is 1 (x) i sigma_y on the real orbitals.
    Loops of both channels and two right-hand sides (at X = 0, where only the Kanamori vertex is projected,
    and at the covariant state X1 = 0.2 dX/dT(X = 0)) at every momentum of a 5x5 mesh."""
    spec = inputs.t2g_soc(seed=1, Lq=5, nc=1, n_ff=5, filling=4.0, T_mu=0.05)
    o = oracle.Oracle(spec)
    reps = [np.kron(_orbital_rep(g), _spin_rep(g)) for g in _C4V]
    theta = np.kron(np.eye(3), 1j * _SY)
    _check_setup(spec, o, reps, theta)
    zero = np.zeros((2, spec.Nq, spec.M, spec.M), complex)
    d1, _ = o.rhs(0.5, zero, 3)
    d2, _ = o.rhs(0.4, 0.2 * d1, 3)
    for w in (0, 1):
        _check_covariance(spec, _expand_all(spec, o, o.loops(0.5, w)), w, reps, theta)
        _check_covariance(spec, d1[w], w, reps, theta)
        _check_covariance(spec, d2[w], w, reps, theta)


# ---------------------------------------------------------------- momentum-shell regulator (Eq. def_lmp)

def _fermi(e, T):
    return 0.5 * (1.0 - np.tanh(0.5 * e / T))


def test_shell_regulator_definition():
    """chi_Lambda suppresses a shell of thickness Lambda around the Fermi surface: chi = 0 on it, 1/2 at
    |e| = Lambda, -> 1 far from it, monotone in |e|; d chi / d Lambda and the loop weight
    d/dLambda [chi(e1) chi(e2)] F^-/+(e1, e2) against central differences in Lambda, with F written out from
    Eqs. disc_2a/2b here (a dropped term of the product rule or a wrong sign fails)."""
    L = oracle.lib()
    for lam in (0.05, 0.7, 3.0):
        assert L.or_chi(0.0, lam) == 0.0
        assert L.or_chi(lam, lam) == pytest.approx(0.5, abs=1e-15)
        assert L.or_chi(-lam, lam) == pytest.approx(0.5, abs=1e-15)
        assert L.or_chi(1e4 * lam, lam) == pytest.approx(1.0, abs=1e-7)
        es = np.linspace(0, 5 * lam, 50)
        assert np.all(np.diff([L.or_chi(e, lam) for e in es]) > 0)
    rng = np.random.default_rng(3)
    T = 0.07
    for _ in range(40):
        e1, e2 = rng.uniform(-1.5, 1.5, 2)
        lam = rng.uniform(0.05, 2.0)
        h = 1e-5 * lam
        fd = (L.or_chi(e1, lam + h) - L.or_chi(e1, lam - h)) / (2 * h)
        assert L.or_dchi(e1, lam) == pytest.approx(fd, rel=1e-6, abs=1e-9)
        Fm = (1 - _fermi(e1, T) - _fermi(e2, T)) / (e1 + e2)
        Fp = (_fermi(e1, T) - _fermi(e2, T)) / (e1 - e2)

        def cc(l):
            return L.or_chi(e1, l) * L.or_chi(e2, l)

        dcc = (cc(lam + h) - cc(lam - h)) / (2 * h)
        assert L.or_wm_shell(e1, e2, lam, T) == pytest.approx(dcc * Fm, rel=1e-6, abs=1e-9)
        assert L.or_wp_shell(e1, e2, lam, T) == pytest.approx(dcc * Fp, rel=1e-6, abs=1e-9)


def test_shell_flow_reaches_temperature_bubble():
    """Lambda -> 0 with Lambda_0 -> infinity, chi chi F^- runs from 0 to F^- itself: the P-only shell flow
    (Eq. sol_spin structure) from Lambda_0 = 1e3 to 1e-5 must land on the closed form built from the
    temperature-flow bubble F^-(T_reg) of the same mesh (kind = 1 loops of a temperature-regulated oracle), a
    cross-check between the two regulators."""
    U, Treg = 2.5, 0.1
    base = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=U, mu=-0.9, Lq=6, nc=2, n_ff=5)
    o_sh = oracle.Oracle(base.with_(regulator=1, T_reg=Treg))
    state, res = o_sh.flow(T0=1e3, T_end=1e-5, rtol=1e-10, atol=1e-12, chmask=1, stop=1e9)
    o_t = oracle.Oracle(base)
    ns = 2
    d0 = [i for i, (x, y) in enumerate(o_t.deltas) if x == 0 and y == 0][0]
    Lb = o_t.loops(Treg, 0, kind=1)[:, d0].reshape(base.Nq, ns, ns, ns, ns)
    B = np.zeros(base.Nq, complex)
    for t1 in range(ns):
        for t2 in range(ns):
            B += 0.5 * (Lb[:, t2, t1, t2, t1] - Lb[:, t2, t1, t1, t2])
    g = -U / (1 + U * B)
    A = _pair_structure(ns)
    expect = np.zeros((base.Nq, base.M, base.M), complex)
    for s1 in range(ns):
        for s2 in range(ns):
            for s3 in range(ns):
                for s4 in range(ns):
                    expect[:, s1 * ns + s2, s4 * ns + s3] = -0.5 * (g + U) * A[s1, s2, s3, s4]
    assert np.abs(state[0] - expect).max() < 1e-6 * max(1.0, np.abs(expect).max())


# ---------------------------------------------------------------- band basis (Sec. 3.4)

def _schober_gauge(spec):
    """Two-band H = eps 1 + g.sigma (g_z = 0): U_{sigma n}(k) = (1, n e^{i phi(k)}) / sqrt(2), n = -1 (lower band,
    column 0) and +1 (upper, column 1), phi the polar angle of g(k) read off H(k) = sum_R t_R e^{i k.R}."""
    Lf = spec.Lf
    kx, ky = np.meshgrid(np.arange(Lf), np.arange(Lf), indexing="ij")
    H = np.zeros((Lf, Lf, 2, 2), complex)
    for R, t in zip(spec.hop_R, spec.hop_t):
        H += t[None, None] * np.exp(2j * np.pi * (kx * R[0] + ky * R[1]) / Lf)[:, :, None, None]
    gx, gy = H[..., 0, 1].real, -H[..., 0, 1].imag
    phi = np.arctan2(gy, gx).reshape(-1)
    Ub = np.zeros((Lf * Lf, 2, 2), complex)
    for j, n in enumerate((-1, 1)):
        Ub[:, 0, j] = 1 / np.sqrt(2)
        Ub[:, 1, j] = n * np.exp(1j * phi) / np.sqrt(2)
    # sanity: eigenvectors of H(k) with eigenvalues eps -/+ |g|
    Hf = H.reshape(-1, 2, 2)
    for j, n in enumerate((-1, 1)):
        lam = Hf[:, 0, 0] + n * np.hypot(gx, gy).reshape(-1)
        assert np.allclose(np.einsum("kab,kb->ka", Hf, Ub[:, :, j]), lam[:, None] * Ub[:, :, j], atol=1e-12)
    return Ub, phi


def test_band_basis_particle_particle_closed_form():
    """Eq. Pinband (P2): the local particle-particle propagator of Eq. sol_spin, P = -(g+U)/2 (d13 d24 - d14 d23)
    at R = R' = 0 with any g(s), transformed with Eq. mat_trafo_P in the gauge U_{sigma n} = (1, n e^{i phi})/sqrt 2,
    is -(g+U)/8 (1/N^2) sum_{k,k'} f_R(k) f*_R'(k') [n1 n3 e^{i phi(s-k') - i phi(k)} + n2 n4 e^{i phi(k') - i phi(s-k)}
    - n1 n4 e^{i phi(k') - i phi(k)} - n2 n3 e^{i phi(s-k') - i phi(s-k)}], written out here as factorised k-sums.
    A transposed pair index or a missing conjugation in the transformation law fails it."""
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=4, nc=3, n_ff=5)
    o = oracle.Oracle(spec)
    Ub, phi = _schober_gauge(spec)
    ns, M, Nq, Lq, nc, Lf = 2, spec.M, spec.Nq, spec.Lq, spec.nc, spec.Lf
    rng = np.random.default_rng(11)
    gU = rng.standard_normal(Nq) + 1j * rng.standard_normal(Nq)      # (g + U)(s), arbitrary
    A = _pair_structure(ns)
    st = np.zeros((2, Nq, M, M), complex)
    for s1 in range(ns):
        for s2 in range(ns):
            for s3 in range(ns):
                for s4 in range(ns):
                    st[0, :, s1 * ns + s2, s4 * ns + s3] = -0.5 * gU * A[s1, s2, s3, s4]
    out = o.band_transform(Ub, st)
    assert np.abs(out[1]).max() == 0.0
    k = np.arange(Lf * Lf)
    kx, ky = k // Lf, k % Lf
    ffR = spec.ff_R
    f = np.exp(-2j * np.pi * (kx[None, :] * ffR[:, 0:1] + ky[None, :] * ffR[:, 1:2]) / Lf)   # f_R(k), [nff][Nk]
    N = Lf * Lf
    nn = (-1, 1)
    for s in range(Nq):
        sx, sy = (s // Lq) * nc, (s % Lq) * nc
        smk = ((sx - kx) % Lf) * Lf + (sy - ky) % Lf                    # s - k on the fine mesh
        e_k, e_smk = np.exp(1j * phi), np.exp(1j * phi[smk])
        # (1/N) sum_k f_R(k) e^{-i phi(k)} etc. and (1/N) sum_k' f*_R'(k') e^{i phi(k')} etc.
        a_k = f @ e_k.conj() / N
        a_smk = f @ e_smk.conj() / N
        b_k = f.conj() @ e_k / N
        b_smk = f.conj() @ e_smk / N
        for i, n1 in enumerate(nn):
            for j, n2 in enumerate(nn):
                for p, n3 in enumerate(nn):
                    for q, n4 in enumerate(nn):
                        term = (n1 * n3 * np.outer(a_k, b_smk) + n2 * n4 * np.outer(a_smk, b_k)
                                - n1 * n4 * np.outer(a_k, b_k) - n2 * n3 * np.outer(a_smk, b_smk))
                        want = -gU[s] / 8 * term                        # [R][R']
                        got = out[0, s][np.ix_(np.arange(spec.n_ff) * 4 + i * 2 + j, np.arange(spec.n_ff) * 4 + q * 2 + p)]
                        assert np.abs(got - want).max() < 1e-12 * max(1.0, np.abs(want).max()), (s, n1, n2, n3, n4)


def test_band_basis_transformation_is_unitary_with_the_complete_set():
    """With the complete form-factor set of a 3x3 torus (N_ff = N_k = 9) the truncated unity is exact and U(s),
    X(u) are unitary: the transform of the identity is the identity in both channels, for the model's own
    (Jacobi) eigenvectors."""
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.35, U=2.0, mu=-0.7, Lq=3, nc=1).with_(ff_R=inputs.ff_complete(3))
    o = oracle.Oracle(spec)
    M, Nq = spec.M, spec.Nq
    eye = np.broadcast_to(np.eye(M), (2, Nq, M, M)).astype(complex)
    out = o.band_transform(o.U, eye)
    assert np.abs(out - eye).max() < 1e-12


def test_form_factor_convergence_orbital_vs_band_basis():
    """Sec. 3.4: the form-factor expansion converges faster in the orbital basis than in the band basis.  The
    local particle-particle propagator of the ladder (Eq. sol_spin: R = R' = 0 only) is captured completely by the
    onsite bond in the orbital basis; transformed to the band basis (Eq. mat_trafo_P, the paper's gauge, complete
    set of a 6x6 torus, so no weight is lost) it spreads over many bond shells.  Captured weight
    sum_{|R|^2, |R'|^2 <= r} |P^{RR'}|^2 / sum |P|^2 per cut r: the orbital basis is at 1 from r = 0, the band basis
    below 1e-2 at r = 0, below 0.9 with the nearest bonds and below 0.95 up to |R|^2 = 5, reaching 1 only with
    the complete set."""
    L = 6
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=L, nc=1).with_(ff_R=inputs.ff_complete(L))
    o = oracle.Oracle(spec)
    Ub, _ = _schober_gauge(spec)
    ns, M, Nq = 2, spec.M, spec.Nq
    A = _pair_structure(ns)
    st = np.zeros((2, Nq, M, M), complex)
    for s1 in range(ns):
        for s2 in range(ns):
            for s3 in range(ns):
                for s4 in range(ns):
                    st[0, :, s1 * ns + s2, s4 * ns + s3] = -0.5 * A[s1, s2, s3, s4]
    band = o.band_transform(Ub, st)[0]
    r2 = np.repeat([int(r[0]) ** 2 + int(r[1]) ** 2 for r in spec.ff_R], ns * ns)   # |R|^2 per row / column
    cuts = sorted(set(r2.tolist()))

    def captured(X):
        W = np.abs(X) ** 2
        return np.array([W[:, r2 <= c][:, :, r2 <= c].sum() for c in cuts]) / W.sum()

    orb, bnd = captured(st[0]), captured(band)
    print("\n|R|^2 cut, captured weight orbital / band: " +
          ", ".join(f"{c}: {a:.4f} / {b:.4f}" for c, a, b in zip(cuts, orb, bnd)))
    assert np.abs(band).max() > 0 and abs((np.abs(band) ** 2).sum() / (np.abs(st[0]) ** 2).sum() - 1) < 1e-12
    assert np.all(orb == 1.0)
    assert bnd[0] < 1e-2 and bnd[1] < 0.9 and bnd[cuts.index(5)] < 0.95
    assert np.all(np.diff(bnd) >= -1e-15) and abs(bnd[-1] - 1) < 1e-12


def test_band_basis_maps_orbital_loops_to_band_diagonal_loops():
    """Eq. loop_orbital is exact with the complete form-factor set: the transformation maps the orbital loop matrices
    (the oracle's direct k-sums with the U dressing, pinned above against the brute-force fRG) onto the band-basis
    loops, diagonal in the band pairs, [L_{l1 l2}]_{RR'}(s) = (1/N) sum_k f_R(k) f*_R'(k) w(e_l1(k1), e_l2(k2)) with
    (k1, k2) = (s - k, k) for P and (k, k - u) for C.  Every entry of U(s), X(u) enters, so a swapped or
    conjugated index fails it (the closed-form pin above is blind to the swap of the pair order, its state
    being antisymmetric in both pairs)."""
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.35, U=2.0, mu=-0.7, Lq=3, nc=1).with_(ff_R=inputs.ff_complete(3))
    o = oracle.Oracle(spec)
    T = 0.3
    ns, nff, M, Nq, Lf = 2, spec.n_ff, spec.M, spec.Nq, spec.Lf
    d_of = {tuple(d): i for i, d in enumerate(o.deltas)}
    X = np.zeros((2, Nq, M, M), complex)
    for ch in (0, 1):
        Lc = o.loops(T, ch)
        for i1 in range(nff):
            for i2 in range(nff):
                di = d_of[tuple(spec.ff_R[i1] - spec.ff_R[i2])]
                X[ch, :, i1 * 4:(i1 + 1) * 4, i2 * 4:(i2 + 1) * 4] = Lc[:, di]
    out = o.band_transform(o.U, X)
    e = o.E - o.mu                                             # [Nk][band]
    k = np.arange(Lf * Lf)
    kx, ky = k // Lf, k % Lf
    f = np.exp(-2j * np.pi * (kx[None, :] * spec.ff_R[:, 0:1] + ky[None, :] * spec.ff_R[:, 1:2]) / Lf)
    for ch, w in ((0, oracle.wm), (1, oracle.wp)):
        for s in range(Nq):
            sx, sy = s // spec.Lq, s % spec.Lq
            other = (((sx - kx) % Lf) * Lf + (sy - ky) % Lf) if ch == 0 else (((kx - sx) % Lf) * Lf + (ky - sy) % Lf)
            want = np.zeros((M, M), complex)
            for l1 in range(ns):
                for l2 in range(ns):
                    e1 = e[other, l1] if ch == 0 else e[k, l1]
                    e2 = e[k, l2] if ch == 0 else e[other, l2]
                    wk = np.array([w(a, b, T) for a, b in zip(e1, e2)])
                    B = (f * wk[None, :]) @ f.conj().T / (Lf * Lf)      # [R][R']
                    # band pair index of the layouts: P (l2, l1) in rows and columns, C (l1, l2)
                    p = l2 * ns + l1 if ch == 0 else l1 * ns + l2
                    want[np.ix_(np.arange(nff) * 4 + p, np.arange(nff) * 4 + p)] = B
            assert np.abs(out[ch, s] - want).max() < 1e-12 * max(1.0, np.abs(want).max()), (ch, s)


# ---------------------------------------------------------------- the flow in the band basis (Sec. 3.2, Sec. 3.4)

@pytest.mark.parametrize("model,mask", [("rashba", 3), ("rashba", 1), ("hubbard", 3)])
def test_band_basis_flow_equals_transformed_orbital_flow(model, mask):
    """Eqs. rge_Pmat, rge_Dmat in the band basis (band-diagonal loops of Eqs. loopminus, loopplus; the bare vertex
    through its band-basis projections) against the orbital flow: with the complete form-factor set of a 3x3
    torus both are exact reformulations of the same one-loop RGE, so the band-basis flow equals the orbital flow
    transformed with Eqs. mat_trafo_P, mat_trafo_D (pinned above by Eq. Pinband and unitarity), step by step
    (fixed-step RK4 from T0 = 2 to 0.4).  A wrong loop (orbital projectors left in), the bare vertex missing its
    momentum dependence, or a wrong prefactor fails it."""
    if model == "rashba":
        spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.4, U=2.0, mu=-0.7, Lq=3, nc=1)
    else:
        spec = inputs.hubbard_square(tp=-0.25, U=2.0, Lq=3, nc=1, filling=0.0, mu=-0.5)
    spec = spec.with_(ff_R=inputs.ff_complete(3))
    o = oracle.Oracle(spec)
    ob = oracle.Oracle(spec, basis="band", band_U=o.U)
    assert np.array_equal(ob.U[5], np.eye(2))
    y, _ = o.flow(T0=2.0, T_end=0.4, fixed_n=4, chmask=mask)
    yb, _ = ob.flow(T0=2.0, T_end=0.4, fixed_n=4, chmask=mask)
    yt = o.band_transform(o.U, y)
    assert np.abs(yt).max() > 1e-2
    assert np.abs(yb - yt).max() < 1e-12 * np.abs(yt).max()
    if model == "rashba":
        # with spin-orbit coupling the orbital-basis loops are not band-diagonal: a different computation
        assert np.abs(yb - y).max() > 1e-3 * np.abs(y).max()
    else:
        # without it the eigenvectors are the unit vectors (degenerate bands): the two bases coincide
        assert np.abs(yb - y).max() < 1e-12 * np.abs(y).max()


def test_form_factor_convergence_of_the_flows_orbital_vs_band():
    """Sec. 3.4: a form-factor expansion converges faster in the orbital basis than in the band basis.  The
    particle-particle flow of the onsite Rashba-Hubbard vertex (P only, a 6x6 torus, T0 = 2 -> 0.5) keeps its
    propagator in the onsite block in the orbital basis (Eq. sol_spin), so 5 bonds already give the complete set's
    result; in the band basis the bare vertex and the propagator spread over many bonds (Eq. Pinband), and the
    truncated flows approach the complete-set flow only as bonds are added."""
    base = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=6, nc=1)
    full = base.with_(ff_R=inputs.ff_complete(6))
    o_full = oracle.Oracle(full)
    ob_full = oracle.Oracle(full, basis="band", band_U=o_full.U)
    y_full, _ = o_full.flow(T0=2.0, T_end=0.5, fixed_n=3, chmask=1)
    yb_full, _ = ob_full.flow(T0=2.0, T_end=0.5, fixed_n=3, chmask=1)

    def onsite(y, spec):
        i0 = [i for i, r in enumerate(spec.ff_R) if r[0] == 0 and r[1] == 0][0]
        return y[0][:, i0 * 4:(i0 + 1) * 4, i0 * 4:(i0 + 1) * 4]

    err_orb, err_band = [], []
    for n_ff in (5, 9, 13):
        sp = base.with_(ff_R=inputs.ff_set(n_ff))
        o = oracle.Oracle(sp)
        ob = oracle.Oracle(sp, basis="band", band_U=o.U)
        y, _ = o.flow(T0=2.0, T_end=0.5, fixed_n=3, chmask=1)
        yb, _ = ob.flow(T0=2.0, T_end=0.5, fixed_n=3, chmask=1)
        ref_o, ref_b = onsite(y_full, full), onsite(yb_full, full)
        err_orb.append(np.abs(onsite(y, sp) - ref_o).max() / np.abs(ref_o).max())
        err_band.append(np.abs(onsite(yb, sp) - ref_b).max() / np.abs(ref_b).max())
    assert max(err_orb) < 1e-12                        # the orbital flow is local: any bond set holds it
    assert min(err_band) > 1e-4                        # the band flow needs more bonds
    assert err_band[-1] < err_band[0]                  # and approaches the complete set as they are added


# ---------------------------------------------------------------- irrep form factors (Sec. 2)

@pytest.mark.parametrize("n_ff", [5, 9, 13])
def test_irrep_form_factors_transform_under_the_point_group(n_ff):
    """Sec. 2: linear combinations of the plane waves that transform under an irreducible representation of the point
    group, orthonormal (the only property the method needs).  W is orthogonal; each A1 / A2 / B1 / B2 row is an
    eigenvector of every bond permutation D(g) with the character of its irrep as eigenvalue; each E space is
    invariant with the E character as trace; (1/N) sum_k f_i f_j* = delta_ij on a mesh."""
    from oracle import irreps
    ff = inputs.ff_set(n_ff)
    W, lab = irreps.basis(ff)
    assert W.shape == (n_ff, n_ff)
    assert np.abs(W @ W.T - np.eye(n_ff)).max() < 1e-13
    chi = {"A1": [1, 1, 1, 1, 1], "A2": [1, 1, 1, -1, -1], "B1": [1, -1, 1, 1, -1], "B2": [1, -1, 1, -1, 1],
           "E": [2, 0, -2, 0, 0]}
    cls = {"E": 0, "C4": 1, "C2": 2, "sv": 3, "sd": 4}
    for g, c in irreps.operations():
        D = irreps.perm_rep(ff, g)
        for s in sorted({l[0] for l in lab}):
            for gi, name in enumerate(irreps.IRREPS):
                rows = [i for i, l in enumerate(lab) if l[0] == s and l[1] == gi]
                if not rows:
                    continue
                B = W[rows]                                   # [d][n]
                img = B @ D.T                                 # rows D(g) w
                if name != "E":
                    assert np.abs(img - chi[name][cls[c]] * B).max() < 1e-12
                else:
                    rep = img @ B.T                           # the E space is invariant: img = rep B
                    assert np.abs(rep @ B - img).max() < 1e-12
                    assert np.trace(rep) == pytest.approx(chi["E"][cls[c]] * len(rows) / 2, abs=1e-12)
    L = 8
    kx, ky = np.divmod(np.arange(L * L), L)
    f = np.exp(-2j * np.pi * (np.outer(kx, ff[:, 0]) + np.outer(ky, ff[:, 1])) / L)   # [k][R]
    fi = f @ W.T
    assert np.abs(fi.T @ fi.conj() / (L * L) - np.eye(n_ff)).max() < 1e-13


def test_irrep_form_factors_closed_forms():
    """The familiar functions: on the nearest-neighbour shell the extended s-wave (cos kx + cos ky), d_{x^2-y^2}
    (cos kx - cos ky) and the p-waves (sin kx, sin ky); on the next-nearest shell cos kx cos ky (A1) and
    sin kx sin ky (B2, d_xy), each up to its normalisation and sign."""
    from oracle import irreps
    ff = inputs.ff_set(9)
    W, lab = irreps.basis(ff)
    k = np.random.default_rng(3).uniform(-np.pi, np.pi, (40, 2))
    f = np.exp(-1j * (np.outer(k[:, 0], ff[:, 0]) + np.outer(k[:, 1], ff[:, 1]))) @ W.T   # [k][i]
    cx, cy, sx, sy = np.cos(k[:, 0]), np.cos(k[:, 1]), np.sin(k[:, 0]), np.sin(k[:, 1])

    def proportional(a, b):
        c = np.vdot(b, a) / np.vdot(b, b)
        return abs(c) > 0.1 and np.abs(a - c * b).max() < 1e-12

    shells = {}
    for i, (s, gi, p) in enumerate(lab):
        shells.setdefault(s, {}).setdefault(irreps.IRREPS[gi], []).append(i)
    nn = [s for s in shells if len(shells[s].get("B1", [])) == 1 and len(shells[s]["A1"]) == 1
          and np.abs(ff[[i for i in range(9) if np.abs(W[shells[s]["A1"][0], i]) > 1e-9]]).sum(axis=1).max() == 1]
    nnn = [s for s in shells if "B2" in shells[s]]
    assert len(nn) == 1 and len(nnn) == 1
    s1, s2 = nn[0], nnn[0]
    assert proportional(f[:, shells[s1]["A1"][0]], cx + cy)
    assert proportional(f[:, shells[s1]["B1"][0]], cx - cy)
    E = f[:, shells[s1]["E"]]                                    # spans sin kx, sin ky
    for target in (sx, sy):
        c, *_ = np.linalg.lstsq(E, target.astype(complex), rcond=None)
        assert np.abs(E @ c - target).max() < 1e-12
    assert proportional(f[:, shells[s2]["A1"][0]], cx * cy)
    assert proportional(f[:, shells[s2]["B2"][0]], sx * sy)
