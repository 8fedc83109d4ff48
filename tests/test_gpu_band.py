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
