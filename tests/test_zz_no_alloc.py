"""The allocation-free loop entry point, tufrg_loops_noalloc, against tufrg_loops and the oracle.

tufrg_loops_noalloc serves callers that cannot call cudaMalloc (device allocation
forbidden in their context, or owned by a host framework's allocator): it keeps its
scratch in one fixed-size static device array instead.  Here it is called through
the C ABI twice in a row (the second call reuses the scratch the first one left
behind) and compared with the model-based entry point on the same eigensystem and
with the CPU oracle's direct k-sum, within the tolerance the split-precision loop
tests use.  This file is collected last so that a run stopping at the first failure
has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1710_08830_gb300 import inputs  # noqa: E402

TOL_SPLIT = 2e-5   # relative, as for the split-precision loop parity tests


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08830_gb300 import _lib, build
    build.build()
    oracle.build()
    return _lib.lib()


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def _rel_np(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _call(lib, m, T, mask, out):
    ff = np.ascontiguousarray(m.spec.ff_R, np.int32)
    E, U = m.bands()
    st = lib.tufrg_loops_noalloc(m.spec.Lq, m.spec.nc, C.c_void_p(E.data_ptr()), C.c_void_p(U.data_ptr()),
                                 C.c_double(m.mu), C.c_double(T), ff.shape[0], ff.ctypes.data, mask,
                                 C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return st


def test_noalloc_matches_model_loops_and_oracle_twice(lib):
    from paper_1710_08830_gb300.api import SPLIT32, Model
    spec = inputs.rashba_q24_k8_ff9(0)          # the full-size benchmark mesh
    m = Model(spec, SPLIT32)
    o = oracle.Oracle(spec, mu=m.mu)
    for T in (0.1, 1.7):                         # two calls in a row, different temperatures
        out = torch.full(m.loop_shape(), float("nan"), dtype=torch.complex128, device="cuda")
        assert _call(lib, m, T, 3, out) == 0
        assert torch.isfinite(out).all()
        ref = m.loops(T, 3)
        assert _rel(out, ref) < TOL_SPLIT
        got = out.cpu().numpy()
        for ch in (0, 1):
            assert _rel_np(got[ch], o.loops(T, ch)) < TOL_SPLIT


# bond sets by the number of non-negative y components of their bond differences: 1 (a line along x),
# 2 (an L of three sites), 3 (the 5- and 9-bond shells), 5 (the 13-bond set, beyond the entry point)
BONDS = {"line3": [(0, 0), (1, 0), (-1, 0)], "ell3": [(0, 0), (1, 0), (0, 1)], "ff5": 5, "ff9": 9, "ff13": 13}


@pytest.mark.parametrize("bonds", list(BONDS))
def test_noalloc_single_channel_and_ragged_mesh(lib, bonds):
    """Every kernel instantiation the entry point dispatches (1, 2 or 3 non-negative bond-difference y
    components) on a ragged fine mesh, one channel at a time; 13 bonds (5 such components) are refused with
    TUFRG_ENOTSUP before any work."""
    from paper_1710_08830_gb300.api import SPLIT32, Model
    b = BONDS[bonds]
    spec = inputs.rashba_hubbard(tp=-0.15, alpha=0.35, U=2.0, mu=-0.7, Lq=5, nc=5,
                                 n_ff=b if isinstance(b, int) else 5)   # Lf = 25
    if not isinstance(b, int):
        spec = spec.with_(ff_R=np.array(b, np.int32))
    m = Model(spec, SPLIT32)
    o = oracle.Oracle(spec, mu=m.mu)
    out = torch.zeros(m.loop_shape(), dtype=torch.complex128, device="cuda")
    if bonds == "ff13":
        assert _call(lib, m, 0.07, 3, out) == 8            # TUFRG_ENOTSUP
        assert out.abs().max() == 0
        return
    ref = m.loops(0.07, 3)
    assert _call(lib, m, 0.07, 2, out) == 0            # C only: P stays untouched
    assert out[0].abs().max() == 0
    assert _rel(out[1], ref[1]) < TOL_SPLIT
    assert _rel_np(out[1].cpu().numpy(), o.loops(0.07, 1)) < TOL_SPLIT
    out.zero_()
    assert _call(lib, m, 0.07, 1, out) == 0            # P only: C stays untouched
    assert out[1].abs().max() == 0
    assert _rel(out[0], ref[0]) < TOL_SPLIT
    assert _rel_np(out[0].cpu().numpy(), o.loops(0.07, 0)) < TOL_SPLIT


def test_noalloc_rejects_oversize_and_bad_arguments(lib):
    from paper_1710_08830_gb300.api import SPLIT32, Model
    big = inputs.rashba_hubbard(Lq=48, nc=8, n_ff=9)   # needs more than the fixed scratch
    m = Model(big, SPLIT32)
    out = torch.zeros(m.loop_shape(), dtype=torch.complex128, device="cuda")
    assert _call(lib, m, 0.1, 3, out) == 9             # TUFRG_ETOOBIG, nothing launched
    assert out.abs().max() == 0
    assert _call(lib, m, -1.0, 3, out) == 1            # TUFRG_EINVAL
