"""The momentum-shell regulator (Eq. def_lmp: L = d/dLambda [chi(e1) chi(e2)] F(e1, e2), chi_Lambda(e) =
e^2 / (e^2 + Lambda^2), F at a fixed temperature) on the GPU against the oracle: loops of every kernel family
(split two-band with symmetries, FP64 two-band, multi-orbital in both precisions), right-hand sides and flows
with Lambda as the flow variable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1710_08830_gb300 import inputs

T_REG = 0.05


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


CASES = {
    "rashba_ff9_Lf25": lambda: inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=5, nc=5, n_ff=9),
    "hubbard_ff5_Lf24": lambda: inputs.hubbard_square(U=3.0, Lq=6, nc=4, n_ff=5, filling=0.9, T_mu=0.02),
    "t2g_ff5_Lf8": lambda: inputs.t2g_soc(seed=2, Lq=4, nc=2, n_ff=5, filling=4.0, T_mu=0.05),
}


def _shell(spec):
    return spec.with_(regulator=1, T_reg=T_REG)


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
@pytest.mark.parametrize("lam", [1.5, 0.08])
def test_shell_loops(api, case, prec, lam):
    spec = _shell(CASES[case]())
    m = api.Model(spec, getattr(api, prec))
    o = oracle.Oracle(spec)
    L = m.loops(lam).cpu().numpy()
    for ch in (0, 1):
        ref = o.loops(lam, ch)
        assert rel(L[ch], ref) < (1e-10 if prec == "FP64" else 2e-5), (ch, rel(L[ch], ref))


@pytest.mark.gpu
@pytest.mark.parametrize("case,prec", [("rashba_ff9_Lf25", "SPLIT32"), ("rashba_ff9_Lf25", "FP64"),
                                       ("t2g_ff5_Lf8", "SPLIT32")])
def test_shell_rhs(api, case, prec):
    spec = _shell(CASES[case]())
    m = api.Model(spec, getattr(api, prec))
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=5, scale=0.2)
    d = m.rhs(0.3, st).cpu().numpy()
    ref, _ = o.rhs(0.3, st, 3)
    assert rel(d, ref) < (1e-10 if prec == "FP64" else 1e-4)


@pytest.mark.gpu
def test_shell_flow_fp64_matches_oracle(api):
    """The full P + C flow with Lambda as the flow variable: same step sequence, state and critical scale as the
    oracle's."""
    spec = _shell(CASES["hubbard_ff5_Lf24"]())
    o = oracle.Oracle(spec)
    st_ref, r_ref = o.flow(T0=10.0, T_end=1e-3, stop=6.0)
    m = api.Model(spec, api.FP64)
    st, r = m.flow(T0=10.0, T_end=1e-3, stop=6.0)
    assert r["n_steps"] == r_ref["n_steps"] and r["n_reject"] == r_ref["n_reject"]
    assert r["crossed"] == r_ref["crossed"]
    assert r["Tc"] == pytest.approx(r_ref["Tc"], rel=1e-9)
    assert rel(st.cpu().numpy(), st_ref) < 1e-9


@pytest.mark.gpu
def test_shell_flow_split_matches_fp64(api):
    """Split precision along the same Lambda flow (symmetric states and orbit products included): the critical
    scale within 1% of the FP64 flow's, same leading channel."""
    spec = _shell(CASES["hubbard_ff5_Lf24"]())
    _, r64 = api.Model(spec, api.FP64).flow(T0=10.0, T_end=1e-3, stop=6.0)
    _, r32 = api.Model(spec, api.SPLIT32).flow(T0=10.0, T_end=1e-3, stop=6.0)
    assert r32["crossed"] == r64["crossed"]
    assert abs(r32["Tc"] / r64["Tc"] - 1) < 0.01
    assert r32["lead_channel"] == r64["lead_channel"]


@pytest.mark.gpu
def test_shell_regulator_arguments(api):
    spec = CASES["rashba_ff9_Lf25"]()
    with pytest.raises(api.TufrgError):
        api.Model(spec.with_(regulator=1, T_reg=0.0), api.SPLIT32)
    with pytest.raises(api.TufrgError):
        api.Model(spec.with_(regulator=7), api.SPLIT32)
