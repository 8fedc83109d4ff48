"""Failures injected from the host, none of which faults or hangs the device: a non-finite value planted in a
checkpoint (refused on resume with TUFRG_ENONFINITE), a huge finite value planted in one (the next right-hand side
overflows and the flow stops with TUFRG_ENONFINITE), and a device allocation that fails because the device memory
is held by another allocation (init stops with TUFRG_ENOMEM, frees what it had allocated once the handle is
released, and the device stays usable).  The bad descriptors and the device wait that gives up are
covered beside the descriptor checks and the device error flag."""
import os
import struct
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.gpu

# CkptHeader: char magic[8]; int version, flowdev_bytes; 10 ints of model fields; int products, ky_chunks;
# long long n_elems (offset 64); 72 bytes in all
HEADER_BYTES = 72


def _api():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1710_08830_gb300 import api
    return api


def _small():
    from paper_1710_08830_gb300 import inputs
    return inputs.rashba_hubbard(tp=-0.15, alpha=0.3, U=3.3, mu=-0.8, Lq=6, nc=3, n_ff=5)


def _checkpoint(api, spec, p, tmp_path):
    ck = tmp_path / "flow.ckpt"
    api.Model(spec, p).flow(stop=6.0, checkpoint_path=str(ck), checkpoint_every=2, stop_after=2)
    raw = bytearray(ck.read_bytes())
    assert raw[:8] == b"TUFRGCK1"
    flowdev_bytes = struct.unpack_from("<i", raw, 12)[0]
    n_elems = struct.unpack_from("<q", raw, 64)[0]
    assert n_elems == 2 * spec.Nq * spec.M ** 2
    assert len(raw) == HEADER_BYTES + flowdev_bytes + 2 * 16 * n_elems
    return raw, HEADER_BYTES + flowdev_bytes, n_elems


@pytest.mark.parametrize("where", ["state", "derivative"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_checkpoint_is_refused(bad, where, tmp_path):
    """A non-finite entry anywhere in a checkpoint's state or derivative (here the last momentum of the C channel,
    which the symmetric path never reads when it is not an orbit representative) is refused by tufrg_flow_resume
    with TUFRG_ENONFINITE, and the model then runs a clean flow."""
    api = _api()
    spec = _small()
    y_ref, r_ref = api.Model(spec, api.SPLIT32).flow(stop=6.0)
    raw, state_at, n_elems = _checkpoint(api, spec, api.SPLIT32, tmp_path)
    M2 = spec.M ** 2
    off = state_at + (16 * n_elems if where == "derivative" else 0) + 16 * (n_elems - M2) + 8
    struct.pack_into("<d", raw, off, bad)
    bad_ck = tmp_path / "bad.ckpt"
    bad_ck.write_bytes(bytes(raw))
    m = api.Model(spec, api.SPLIT32)
    with pytest.raises(api.TufrgError) as e:
        m.flow(stop=6.0, resume_from=str(bad_ck))
    assert e.value.status == 4 and "non-finite" in str(e.value), e.value
    y, r = m.flow(stop=6.0)
    assert torch.equal(y, y_ref) and r["n_steps"] == r_ref["n_steps"]


@pytest.mark.parametrize("prec", ["SPLIT32", "FP64"])
def test_overflowing_state_stops_the_flow_with_enonfinite(prec, tmp_path):
    """A finite but huge entry planted in a checkpoint's state (entry (0, 0) of the C channel at q = 0, an orbit
    representative) makes the next right-hand side overflow: the controller stops the flow with status 4 and
    tufrg_flow_end returns TUFRG_ENONFINITE with the state reached so far; the model then runs a clean flow."""
    api = _api()
    spec = _small()
    p = getattr(api, prec)
    y_ref, r_ref = api.Model(spec, p).flow(stop=6.0)
    raw, state_at, n_elems = _checkpoint(api, spec, p, tmp_path)
    struct.pack_into("<d", raw, state_at + 16 * (n_elems // 2), 1e200)
    big_ck = tmp_path / "big.ckpt"
    big_ck.write_bytes(bytes(raw))
    m = api.Model(spec, p)
    with pytest.raises(api.TufrgError) as e:
        m.flow(stop=6.0, resume_from=str(big_ck))
    assert e.value.status == 4 and "non-finite right-hand side" in str(e.value), e.value
    y, r = m.flow(stop=6.0)
    assert torch.equal(y, y_ref) and r["n_steps"] == r_ref["n_steps"]


def test_device_allocation_failure_is_reported_and_leaves_the_device_usable():
    api = _api()
    from paper_1710_08830_gb300 import inputs
    small = _small()
    st = inputs.random_state(small, seed=5, scale=0.2)
    m0 = api.Model(small, api.SPLIT32)
    ref = m0.rhs(0.3, st).clone()
    m0.close()
    del m0
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    # the FP32 projections and state copy of this model are 169 MiB each (2 x 4096 momenta x 52 x 52 entries)
    big = inputs.rashba_hubbard(tp=-0.15, alpha=0.3, U=3.3, mu=-0.8, Lq=64, nc=1, n_ff=13)
    assert 2 * big.Nq * big.M ** 2 * 8 > 160 << 20
    headroom = 256 << 20
    free, _ = torch.cuda.mem_get_info()
    blocker = torch.empty(((free - headroom) >> 21) << 21, dtype=torch.uint8, device="cuda")
    try:
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        assert free_before < 2 * headroom
        with pytest.raises(api.TufrgError) as e:
            api.Model(big, api.SPLIT32, products=api.PRODUCTS_SIMT)
        assert e.value.status == 2, e.value
        assert "cudaMalloc" in str(e.value)
        # the handle was released by the binding: what init had allocated is back, and no error is left pending
        # for the next launch check of this thread (torch's included)
        free_after, _ = torch.cuda.mem_get_info()
        assert free_after >= free_before - (16 << 20)
        torch.cuda.synchronize()
        probe = torch.ones(1024, device="cuda") * 2.0
        assert float(probe.sum()) == 2048.0
    finally:
        del blocker
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    m1 = api.Model(small, api.SPLIT32)
    assert torch.equal(m1.rhs(0.3, st), ref)
