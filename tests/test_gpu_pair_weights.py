"""Error of the split path's FP32 pair weights at the near-degenerate points, against the FP64 oracle.

The split-precision loop kernels evaluate the temperature derivatives of the bubbles (Eqs. disc_2a, disc_2b),
d/dT F^-(e1, e2) = -(g1 + g2) / (e1 + e2) and d/dT F^+(e1, e2) = (g1 - g2) / (e1 - e2), in FP32 from
e = E - mu rounded once, with the analytic limit (g'1 + g'2) / 2 below |e1 -+ e2| = 1e-2 T (the FP64 path and
the oracle switch at 1e-5 T).  Near the switch the FP32 divided difference loses about eps32 T / |e1 -+ e2| of
its accuracy and the limit misses the curvature term (e1 -+ e2)^2 g''' / 12; both stay near 1e-5 relative.

The transfer momenta where these branches carry weight are the zero momentum of each channel:
  * P at s = 0: the Cooper line, e(-k) + e(k) = 0 on the Fermi surface, hit by every pair of time-reversed
    states (F^- degenerate branch);
  * C at u = 0: the intra-momentum pairs, e1 = e2 exactly for the same band and, at zero spin-orbit coupling,
    for the two Kramers-degenerate bands (F^+ degenerate branch).
The test measures the loops there, and over all momenta, at the lowest flow temperature T = 0.02 (switch at
2e-4) and at T = 0.1, for the Hubbard model without spin-orbit coupling (degenerate bands) and the Rashba model,
and asserts the split-path parity bound of the loops (2e-5 relative to the largest entry of the channel at that
momentum).  The measured errors are printed (pytest -s) per case.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1710_08830_gb300 import inputs  # noqa: E402

MODELS = {
    "hubbard_no_soc": lambda: inputs.hubbard_square(tp=-0.25, U=3.0, Lq=8, nc=8, n_ff=5, filling=0.9, T_mu=0.02),
    "rashba": lambda: inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=8, nc=8, n_ff=9),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08830_gb300 import build
    build.build()
    oracle.build()


@pytest.mark.parametrize("model", list(MODELS))
@pytest.mark.parametrize("T", [0.02, 0.1])
def test_split_pair_weights_at_degenerate_points(model, T):
    from paper_1710_08830_gb300.api import SPLIT32, SYMMETRY_OFF, Model
    spec = MODELS[model]()
    m = Model(spec, SPLIT32, symmetry=SYMMETRY_OFF)   # every momentum summed directly
    o = oracle.Oracle(spec, mu=m.mu)
    L = m.loops(T).cpu().numpy()
    report = {}
    for ch, name in ((0, "P, s = 0 (Cooper line)"), (1, "C, u = 0 (degenerate pairs)")):
        ref = o.loops(T, ch)
        err_q0 = np.abs(L[ch][0] - ref[0]).max() / np.abs(ref[0]).max()
        err_all = max(np.abs(L[ch][q] - ref[q]).max() / np.abs(ref[q]).max() for q in range(spec.Nq))
        report[name] = (err_q0, err_all)
        assert err_q0 < 2e-5 and err_all < 2e-5, (name, err_q0, err_all)
    print(f"\n{model} T={T}: " + "; ".join(f"{k}: {a:.2e} (all q {b:.2e})" for k, (a, b) in report.items()))
