"""Irrep form factors on the GPU (Sec. 2): the library's C4v basis against the oracle's independent construction
(through quantities that do not depend on the basis chosen inside an irreducible space: each (shell, irrep)
projector), the transformation of states against the oracle's, and a flow's leading form factor."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import irreps  # noqa: E402
from paper_1710_08830_gb300 import inputs  # noqa: E402


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08830_gb300 import api as _api, build
    build.build()
    return _api


def _projectors(W, lab):
    out = {}
    for s, gi, _ in lab:
        rows = [i for i, l in enumerate(lab) if l[0] == s and l[1] == gi]
        out[(int(s), int(gi))] = W[rows].T @ W[rows]
    return out


@pytest.mark.parametrize("n_ff,prec", [(5, "FP64"), (9, "SPLIT32"), (13, "FP64")])
def test_irrep_basis_matches_oracle(api, n_ff, prec):
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=6, nc=2, n_ff=n_ff)
    m = api.Model(spec, getattr(api, prec))
    W, lab = m.form_factors()
    Wo, labo = irreps.basis(spec.ff_R)
    assert np.abs(W @ W.T - np.eye(n_ff)).max() < 1e-13
    P, Po = _projectors(W, lab), _projectors(Wo, labo)
    # shells are numbered in order of first appearance in both constructions
    assert set(P) == set(Po)
    for key in P:
        assert np.abs(P[key] - Po[key]).max() < 1e-12, key
    st = inputs.random_state(spec, seed=2, scale=0.3)
    got = m.irrep_basis(st).cpu().numpy()
    want = irreps.transform(W, st, spec.n_s ** 2)
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    back = m.irrep_basis(torch.from_numpy(got).cuda(), inverse=True).cpu().numpy()
    assert np.abs(back - st).max() < 1e-12 * np.abs(st).max()


def test_irrep_basis_refuses_an_open_bond_set(api):
    spec = inputs.rashba_hubbard(Lq=5, nc=1, n_ff=5).with_(ff_R=np.array([(0, 0), (1, 0), (-1, 0)], np.int32))
    m = api.Model(spec, api.FP64)
    with pytest.raises(api.TufrgError) as e:
        m.form_factors()
    assert e.value.status == 8


def test_leading_form_factor_of_an_attractive_ladder(api):
    """The particle-particle flow of an attractive onsite interaction (P only) grows an onsite (A1 of the onsite
    shell) pairing propagator: the leading eigenvector of A_P(q = 0) at the end of the flow carries its weight in
    the onsite A1 form factor, in the irrep basis of the GPU's transformation."""
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=-2.0, mu=-0.9, Lq=6, nc=2, n_ff=9)
    m = api.Model(spec, api.FP64)
    st, r = m.flow(T0=10.0, T_end=0.05, stop=1e9, mask=1)
    A, _ = m.project(st, mask=1)
    Ai = m.irrep_basis(A).cpu().numpy()[0, 0]          # channel P, q = 0
    ev, vec = np.linalg.eigh(0.5 * (Ai + Ai.conj().T))
    v = vec[:, np.argmax(np.abs(ev))]
    W, lab = m.form_factors()
    w = (np.abs(v) ** 2).reshape(spec.n_ff, 4).sum(axis=1)
    lead = int(np.argmax(w))
    assert tuple(lab[lead][:2]) == (0, 0) and w[lead] > 0.9       # shell 0 (onsite), A1
