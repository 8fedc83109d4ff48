"""Flows driven step by step with per-step metrics and checkpoints (tufrg_flow_start / _step / _end, _save /
_resume): the stepwise flow is tufrg_flow's flow, and a flow resumed from a checkpoint in a fresh model continues
bit for bit (the controller, the state, the FSAL derivative and the launch shapes are restored)."""
import json
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu


def _api():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1710_08830_gb300 import api
    return api


def _spec():
    from paper_1710_08830_gb300 import inputs
    return inputs.rashba_hubbard(tp=-0.15, alpha=0.3, U=3.3, mu=-0.8, Lq=6, nc=3, n_ff=5)


@pytest.mark.parametrize("prec", ["SPLIT32", "FP64"])
def test_stepwise_flow_equals_flow_and_resume_is_bitwise(prec, tmp_path):
    api = _api()
    spec = _spec()
    p = getattr(api, prec)
    y_full, r_full = api.Model(spec, p).flow(stop=6.0)
    assert r_full["n_steps"] > 8
    # step by step with metrics: the same flow
    met = tmp_path / "steps.jsonl"
    y_step, r_step = api.Model(spec, p).flow(stop=6.0, metrics_path=str(met))
    assert torch.equal(y_step, y_full)
    for k in ("n_steps", "n_reject", "n_rhs", "crossed", "Tc", "amax", "lead_channel", "lead_q"):
        assert r_step[k] == r_full[k], k
    rows = [json.loads(line) for line in met.read_text().splitlines()]
    assert [r["step"] for r in rows] == list(range(1, r_full["n_steps"] + 1))
    Ts = [r["T"] for r in rows]
    assert all(a > b for a, b in zip(Ts, Ts[1:])) and Ts[-1] == pytest.approx(r_full["T_last"], rel=1e-12)
    for r in rows:
        assert r["amax"] == max(r["amax_P"], r["amax_C"])
    assert rows[-1]["n_reject"] == r_full["n_reject"]
    # interrupted after 7 accepted steps with a checkpoint every 3, resumed in a fresh model from step 6
    ck = tmp_path / "flow.ckpt"
    _, r_part = api.Model(spec, p).flow(stop=6.0, checkpoint_path=str(ck), checkpoint_every=3, stop_after=7)
    assert r_part["n_steps"] == 7 and ck.exists()
    m2 = api.Model(spec, p)
    y_res, r_res = m2.flow(stop=6.0, resume_from=str(ck))
    assert torch.equal(y_res, y_full)
    for k in ("n_steps", "n_reject", "n_rhs", "crossed", "Tc", "amax", "lead_channel", "lead_q"):
        assert r_res[k] == r_full[k], k
    # the model works normally afterwards
    y_again, r_again = m2.flow(stop=6.0)
    assert torch.equal(y_again, y_full) and r_again["n_steps"] == r_full["n_steps"]


def test_checkpoint_errors(tmp_path):
    api = _api()
    from paper_1710_08830_gb300 import inputs
    spec = _spec()
    ck = tmp_path / "a.ckpt"
    api.Model(spec, api.SPLIT32).flow(stop=6.0, checkpoint_path=str(ck), checkpoint_every=2, stop_after=2)
    # another mesh, another precision, another channel mask: refused
    other = inputs.rashba_hubbard(tp=-0.15, alpha=0.3, U=3.3, mu=-0.8, Lq=6, nc=4, n_ff=5)
    for model, mask in ((api.Model(other, api.SPLIT32), api.CH_P | api.CH_C), (api.Model(spec, api.FP64), api.CH_P | api.CH_C),
                        (api.Model(spec, api.SPLIT32), api.CH_P)):
        with pytest.raises(api.TufrgError, match="EINVAL"):
            model.flow(stop=6.0, mask=mask, resume_from=str(ck))
    # a truncated file is refused
    short = tmp_path / "short.ckpt"
    short.write_bytes(ck.read_bytes()[:100])
    with pytest.raises(api.TufrgError, match="EINVAL"):
        api.Model(spec, api.SPLIT32).flow(stop=6.0, resume_from=str(short))
