"""Band-basis exchange propagators (Sec. 3.4, Eqs. mat_trafo_P, mat_trafo_D) on the GPU against the oracle's, with
the GPU model's own eigenvectors (the band basis depends on their gauge), and the locality comparison the paper draws
from them: the particle-particle propagator of the ladder flow is local in the orbital basis (Eq. sol_spin) and
spreads over form factors in the band basis (Eq. Pinband)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1710_08830_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = {
    "rashba_ff5_Lf12": lambda: inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=4, nc=3, n_ff=5),
    "rashba_ff9_Lf25": lambda: inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=5, nc=5, n_ff=9),
    "complete_3x3": lambda: inputs.rashba_hubbard(tp=-0.2, alpha=0.35, U=2.0, mu=-0.7, Lq=3, nc=1).with_(
        ff_R=inputs.ff_complete(3)),
}


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08830_gb300 import api as _api, build
    build.build()
    return _api


@pytest.mark.gpu
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["FP64", "SPLIT32"])
def test_band_basis_matches_oracle(api, case, prec):
    spec = CASES[case]()
    m = api.Model(spec, getattr(api, prec))
    _, U = m.bands()
    st = inputs.random_state(spec, seed=9, scale=0.3)
    got = m.band_basis(st).cpu().numpy()
    want = oracle.Oracle(spec).band_transform(U.cpu().numpy(), st)
    assert rel(got, want) < (1e-11 if prec == "FP64" else 1e-5), rel(got, want)


@pytest.mark.gpu
def test_band_basis_of_the_ladder_is_not_local(api):
    """P-only flow (Eq. sol_spin): the orbital propagator lives in the R = R' = 0 block; in the band basis a large
    part of its weight sits at other bonds (the paper's argument that the orbital basis converges faster in form
    factors).  The complete set of a 3x3 torus makes the transformation unitary, so the total weight is kept."""
    spec = CASES["complete_3x3"]()
    m = api.Model(spec, api.FP64)
    st, _ = m.flow(T0=10.0, T_end=0.3, rtol=1e-10, atol=1e-12, stop=1e9, mask=1)
    P = st.cpu().numpy()[0]
    Pb = m.band_basis(st).cpu().numpy()[0]
    nff = spec.n_ff
    i0 = [i for i, R in enumerate(spec.ff_R) if R[0] == 0 and R[1] == 0][0]
    blk = np.zeros((nff, nff), bool)
    blk[i0, i0] = True
    mask = np.kron(blk, np.ones((4, 4), bool))
    w_orb = np.linalg.norm(P[:, mask]) ** 2 / np.linalg.norm(P) ** 2
    w_band = np.linalg.norm(Pb[:, mask]) ** 2 / np.linalg.norm(Pb) ** 2
    print(f"\nweight of the R = R' = 0 block: orbital {w_orb:.6f}, band {w_band:.6f}")
    assert w_orb > 1 - 1e-12
    assert w_band < 0.9
    assert np.linalg.norm(Pb) == pytest.approx(np.linalg.norm(P), rel=1e-10)


@pytest.mark.gpu
def test_band_basis_rejects_multi_orbital(api):
    spec = inputs.t2g_soc(seed=2, Lq=4, nc=2, n_ff=5, filling=4.0, T_mu=0.05)
    m = api.Model(spec, api.SPLIT32)
    with pytest.raises(api.TufrgError):
        m.band_basis(m.zeros_state())


# ------------------------------------------------------------------ the flow in the band basis (Eqs. rge_Pmat, rge_Dmat)

def _band_pair(api, spec, prec):
    """A band-basis model and the oracle in the band basis of the same eigenvectors (the GPU's)."""
    _, U = api.Model(spec, getattr(api, prec)).bands()
    mb = api.Model(spec, getattr(api, prec), basis=api.BASIS_BAND)
    ob = oracle.Oracle(spec, basis="band", band_U=U.cpu().numpy())
    return mb, ob


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["rashba_ff5_Lf12", "rashba_ff9_Lf25", "complete_3x3"])
@pytest.mark.parametrize("prec", ["FP64", "SPLIT32"])
def test_band_basis_rhs_matches_oracle(api, case, prec):
    """Loops (band-diagonal) and right-hand sides of the band-basis flow against the oracle's band-basis flow with
    the GPU's eigenvectors: FP64 <= 1e-10, split <= 2e-5 (loops) and 1e-4 (right-hand side), relative to the largest
    entry."""
    spec = CASES[case]()
    mb, ob = _band_pair(api, spec, prec)
    _, Ub = mb.bands()
    assert np.array_equal(Ub.cpu().numpy()[3], np.eye(2))       # the band basis: unit eigenvectors
    L = mb.loops(0.2).cpu().numpy()
    for ch in (0, 1):
        ref = ob.loops(0.2, ch)
        err = np.abs(L[ch] - ref).max() / np.abs(ref).max()
        assert err < (1e-10 if prec == "FP64" else 2e-5), (ch, err)
    st = inputs.random_state(spec, seed=4, scale=0.2)
    d = mb.rhs(0.3, st).cpu().numpy()
    ref, _ = ob.rhs(0.3, st, 3)
    err = np.abs(d - ref).max() / np.abs(ref).max()
    assert err < (1e-10 if prec == "FP64" else 1e-4), err


@pytest.mark.gpu
def test_band_basis_flow_matches_oracle(api):
    """The whole adaptive band-basis flow (FP64) takes the oracle's step sequence and ends on its state; the split
    flow reaches the same critical scale within 1%."""
    spec = CASES["rashba_ff5_Lf12"]().with_(V0=inputs.rashba_hubbard(U=3.3, Lq=4, nc=3, n_ff=5).V0)
    mb, ob = _band_pair(api, spec, "FP64")
    st, r = mb.flow(stop=5.0)
    st_ref, r_ref = ob.flow(stop=5.0)
    assert r["n_steps"] == r_ref["n_steps"] and r["n_reject"] == r_ref["n_reject"]
    assert r["crossed"] == r_ref["crossed"]
    assert r["Tc"] == pytest.approx(r_ref["Tc"], rel=1e-9)
    assert np.abs(st.cpu().numpy() - st_ref).max() < 1e-9 * np.abs(st_ref).max()
    mb32, _ = _band_pair(api, spec, "SPLIT32")
    _, r32 = mb32.flow(stop=5.0)
    assert r32["crossed"] == r["crossed"] and abs(r32["Tc"] / r["Tc"] - 1) < 0.01


@pytest.mark.gpu
def test_band_and_orbital_flows_agree_with_the_complete_set(api):
    """With the complete bond set of a 3x3 torus the band-basis flow on the GPU equals the orbital flow transformed
    to the band basis (tufrg_band_basis), both integrated tightly to the same temperature."""
    spec = CASES["complete_3x3"]()
    m = api.Model(spec, api.FP64)
    mb = api.Model(spec, api.FP64, basis=api.BASIS_BAND)
    kw = dict(T0=10.0, T_end=0.3, rtol=1e-11, atol=1e-13, stop=1e9)
    y, _ = m.flow(**kw)
    yb, _ = mb.flow(**kw)
    yt = m.band_basis(y).cpu().numpy()
    assert np.abs(yb.cpu().numpy() - yt).max() < 1e-8 * np.abs(yt).max()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["FP64", "SPLIT32"])
def test_form_factor_convergence_orbital_vs_band_on_the_gpu(api, prec):
    """Sec. 3.4 on the GPU: the particle-particle flow of the onsite Rashba-Hubbard vertex (P only, 4x4 torus, flow
    to T = 0.5) in the orbital basis is exact with 5 bonds already (its propagator is local), while the band-basis
    flow stays far from its complete-set result (16 bonds, M = 64, the largest the band transformation takes) with
    5 or 9 bonds.  Errors of the onsite block against the complete set are printed (pytest -s); the oracle's 6x6
    version of this comparison (tests/test_oracle_pins.py) shows the band-basis error falling as bonds are added."""
    base = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=4, nc=1)
    full = base.with_(ff_R=inputs.ff_complete(4))
    kw = dict(T0=2.0, T_end=0.5, rtol=1e-10, atol=1e-12, stop=1e9, mask=1)

    def onsite(y, spec):
        i0 = [i for i, r in enumerate(spec.ff_R) if r[0] == 0 and r[1] == 0][0]
        return y.cpu().numpy()[0][:, i0 * 4:(i0 + 1) * 4, i0 * 4:(i0 + 1) * 4]

    p = getattr(api, prec)
    ref_o = onsite(api.Model(full, p).flow(**kw)[0], full)
    ref_b = onsite(api.Model(full, p, basis=api.BASIS_BAND).flow(**kw)[0], full)
    eo, eb = [], []
    for n_ff in (5, 9):
        sp = base.with_(ff_R=inputs.ff_set(n_ff))
        eo.append(np.abs(onsite(api.Model(sp, p).flow(**kw)[0], sp) - ref_o).max() / np.abs(ref_o).max())
        eb.append(np.abs(onsite(api.Model(sp, p, basis=api.BASIS_BAND).flow(**kw)[0], sp) - ref_b).max() /
                  np.abs(ref_b).max())
    print(f"\n{prec} onsite-block error vs the complete set (N_ff = 5, 9): orbital "
          + ", ".join(f"{v:.2e}" for v in eo) + "; band " + ", ".join(f"{v:.2e}" for v in eb))
    tol = 1e-8 if prec == "FP64" else 1e-4
    assert max(eo) < tol
    assert min(eb) > 1e-2 and eb[1] <= eb[0] * (1 + 1e-9)   # (on the 4x4 torus the 9-bond set adds nothing onsite)
