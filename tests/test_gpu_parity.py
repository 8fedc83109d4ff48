"""GPU parity: every step of the CUDA path against the CPU oracle, through the C ABI.

Tolerances (stated per result):
  * integer gather tables: bit-exact;
  * FP64 path vs oracle: <= 1e-10 relative (max abs error / max abs value);
  * split path (FP32 loop sums and products, FP64 state) vs FP64 oracle: <= 1e-4 relative.
Sizes span several CTAs and a ragged tail of the fine mesh (Lf = 24, 25, 30, 120), the
degenerate bands of the SU(2) model, the complete 4x4 bond set and the full-size
24x24 / 8x8 Rashba workload.
"""
import contextlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_1710_08830_gb300 import inputs  # noqa: E402

TOL64 = 1e-10
TOL32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08830_gb300 import build
    build.build()
    oracle.build()


def _api():
    from paper_1710_08830_gb300 import api
    return api


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = {
    "rashba_ff5_Lf24": lambda: inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=6, nc=4, n_ff=5),
    "rashba_ff9_Lf25": lambda: inputs.rashba_hubbard(tp=-0.15, alpha=0.35, U=2.0, mu=-0.7, Lq=5, nc=5, n_ff=9),
    "hubbard_ff5_Lf24": lambda: inputs.hubbard_square(tp=-0.25, U=3.0, Lq=6, nc=4, n_ff=5, filling=0.9, T_mu=0.05),
    "rashba_ff13_Lf30": lambda: inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=2.0, mu=-1.0, Lq=10, nc=3, n_ff=13),
    "complete_4x4": lambda: inputs.rashba_hubbard(tp=-0.2, alpha=0.4, U=2.0, mu=-0.7, Lq=4, nc=1).with_(
        ff_R=inputs.ff_complete(4)),
    "rashba_ff9_Lf120": lambda: inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=12, nc=10, n_ff=9),
}


@pytest.mark.parametrize("case", ["rashba_ff5_Lf24", "hubbard_ff5_Lf24", "rashba_ff13_Lf30"])
def test_bands(case):
    api = _api()
    spec = CASES[case]()
    m = api.Model(spec, api.FP64)
    o = oracle.Oracle(spec)
    E, U = m.bands()
    E, U = E.cpu().numpy(), U.cpu().numpy()
    assert np.abs(E - o.E).max() < 1e-12
    L = spec.Lf
    kx, ky = np.divmod(np.arange(spec.Nk), L)
    H = np.zeros((spec.Nk, 2, 2), complex)
    for R, t in zip(spec.hop_R, spec.hop_t):
        H += np.exp(2j * np.pi * (kx * R[0] + ky * R[1]) / L)[:, None, None] * t
    assert np.abs(np.einsum("kij,kjl->kil", H, U) - U * E[:, None, :]).max() < 1e-12
    assert np.abs(np.einsum("kji,kjl->kil", U.conj(), U) - np.eye(2)).max() < 1e-13
    assert abs(m.mu - o.mu) < 1e-12


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("T", [2.0, 0.07])
def test_loops_fp64(case, T):
    api = _api()
    spec = CASES[case]()
    m = api.Model(spec, api.FP64)
    o = oracle.Oracle(spec)
    assert np.array_equal(m.deltas, o.deltas)
    L = m.loops(T).cpu().numpy()
    for ch in (0, 1):
        ref = o.loops(T, ch)
        assert rel(L[ch], ref) < TOL64, (ch, rel(L[ch], ref))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("T", [2.0, 0.07])
def test_loops_split(case, T):
    api = _api()
    spec = CASES[case]()
    m = api.Model(spec, api.SPLIT32)
    o = oracle.Oracle(spec)
    L = m.loops(T).cpu().numpy()
    for ch in (0, 1):
        ref = o.loops(T, ch)
        assert rel(L[ch], ref) < 2e-5, (ch, rel(L[ch], ref))


def _zeeman(spec, B=0.15):
    """The same model with an onsite Zeeman field B sigma_z (breaks time reversal)."""
    hop_R = np.array(spec.hop_R, np.int32)
    hop_t = np.array(spec.hop_t, np.complex128)
    z = B * np.diag([1.0, -1.0]).astype(np.complex128)
    onsite = [i for i, r in enumerate(hop_R) if r[0] == 0 and r[1] == 0]
    if onsite:
        hop_t[onsite[0]] += z
    else:
        hop_R = np.vstack([hop_R, [[0, 0]]]).astype(np.int32)
        hop_t = np.concatenate([hop_t, z[None]])
    return spec.with_(hop_R=hop_R, hop_t=hop_t)


C4V = [((1, 0), (0, 1)), ((0, -1), (1, 0)), ((-1, 0), (0, -1)), ((0, 1), (-1, 0)),
       ((-1, 0), (0, 1)), ((1, 0), (0, -1)), ((0, 1), (1, 0)), ((0, -1), (-1, 0))]


def _n_orbits(Lq, mats):
    """Orbits of the Lq x Lq transfer mesh under the given point operations (brute force)."""
    seen, n = set(), 0
    for qx in range(Lq):
        for qy in range(Lq):
            if (qx, qy) in seen:
                continue
            n += 1
            for (a, b), (c, d) in mats:
                seen.add(((a * qx + b * qy) % Lq, (c * qx + d * qy) % Lq))
    return n


@pytest.mark.parametrize("case", ["rashba_ff9_Lf25", "hubbard_ff5_Lf24", "rashba_ff13_Lf30"])
def test_loops_symmetry(case):
    """Models with the square-lattice point group (spin rotations included) sum the loops for one
    momentum per orbit and write the rest by symmetry; the result equals the full k-sum (to FP32
    rounding) and the oracle.  An out-of-plane Zeeman field leaves only the four rotations: the orbits
    of C4 are summed and the loops still match the oracle.  (Without spin-orbit coupling the field
    keeps all eight operations, with diagonal spin unitaries.)"""
    api = _api()
    spec = CASES[case]()
    Lq = spec.Lq
    m = api.Model(spec, api.SPLIT32)
    full = api.Model(spec, api.SPLIT32, symmetry=api.SYMMETRY_OFF)
    assert m.n_loop_q == _n_orbits(Lq, C4V) and full.n_loop_q == Lq * Lq
    for T in (2.0, 0.07):
        L, Lfull = m.loops(T).cpu().numpy(), full.loops(T).cpu().numpy()
        assert rel(L, Lfull) < 2e-6
    zs = _zeeman(spec)
    mz = api.Model(zs, api.SPLIT32)
    assert mz.n_loop_q == _n_orbits(Lq, C4V if case.startswith("hubbard") else C4V[:4])
    o = oracle.Oracle(zs)
    L = mz.loops(0.07).cpu().numpy()
    for ch in (0, 1):
        assert rel(L[ch], o.loops(0.07, ch)) < 2e-5


@pytest.mark.parametrize("case,prec", [("rashba_ff9_Lf25", "SPLIT32"), ("rashba_ff13_Lf30", "SPLIT32"),
                                       ("hubbard_ff5_Lf24", "FP64"), ("rashba_ff5_Lf24", "FP64"),
                                       ("t2g_ff5_Lf8", "SPLIT32"), ("t2g_ff9_Lf10", "FP64")])
def test_rhs_symmetric_state(case, prec):
    """A state one Euler step from X = 0 has the loop symmetries (X(G q) = W X(q) W^dagger); the right-hand
    side evaluated for the orbit representatives and written to the other momenta by symmetry equals the
    full evaluation, and the oracle's."""
    api = _api()
    spec = (CASES.get(case) or T2G[case])()
    m = api.Model(spec, getattr(api, prec), symmetry=api.SYMMETRY_STATES)   # representatives' path always
    zero = m.zeros_state()
    X1 = 0.05 * m.rhs(0.5, zero)
    full = m.rhs(0.4, X1).cpu().numpy()
    sym = m.rhs(0.4, X1, symmetric=True).cpu().numpy()
    assert rel(sym, full) < (1e-12 if prec == "FP64" else 2e-6)
    ref, _ = oracle.Oracle(spec).rhs(0.4, X1.cpu().numpy(), 3)
    assert rel(sym, ref) < (TOL64 if prec == "FP64" else TOL32)
    for mask in (api.CH_P, api.CH_C):   # one channel (the other's sources and dX/dT are zero)
        one = m.rhs(0.4, X1, mask=mask, symmetric=True).cpu().numpy()
        one_full = m.rhs(0.4, X1, mask=mask).cpu().numpy()
        ch = 0 if mask == api.CH_P else 1
        assert rel(one[ch], one_full[ch]) < (1e-12 if prec == "FP64" else 2e-6)
        assert not np.any(one[1 - ch])


@pytest.mark.parametrize("case,prec", [("rashba_ff9_Lf25", "SPLIT32"), ("hubbard_ff5_Lf24", "FP64")])
def test_flow_symmetric_state_path(case, prec):
    """Flows evaluate their (symmetric) states for the orbit representatives only; the result matches the flow
    with every symmetry off."""
    api = _api()
    spec = CASES[case]()
    y1, r1 = api.Model(spec, getattr(api, prec), symmetry=api.SYMMETRY_STATES).flow(stop=6.0)
    y0, r0 = api.Model(spec, getattr(api, prec), symmetry=api.SYMMETRY_OFF).flow(stop=6.0)
    assert r1["crossed"] == r0["crossed"]
    if prec == "FP64":
        assert r1["n_steps"] == r0["n_steps"]
    assert abs(r1["Tc"] / r0["Tc"] - 1) < (1e-9 if prec == "FP64" else 1e-4)
    assert rel(y1.cpu().numpy(), y0.cpu().numpy()) < (1e-9 if prec == "FP64" else 1e-4)


def _paper_gather_terms(spec):
    """Independent enumeration of the gather terms from the printed projection formulas."""
    L = spec.Lq
    ff = [tuple(map(int, r)) for r in spec.ff_R]
    idx = {((x % L), (y % L)): i for i, (x, y) in enumerate(ff)}
    classes = sorted({((a[0] - b[0]) % L, (a[1] - b[1]) % L) for a in ff for b in ff})
    P, C = set(), set()
    for iR, (Rx, Ry) in enumerate(ff):
        for iRp, (Px, Py) in enumerate(ff):
            for (cx, cy) in classes:
                i1 = idx.get(((Rx + cx) % L, (Ry + cy) % L))
                i2 = idx.get(((Px - cx) % L, (Py - cy) % L))
                j2 = idx.get(((-Px - cx) % L, (-Py - cy) % L))
                if i1 is not None and i2 is not None:
                    P.add((iR, iRp, 0, cx, cy, i1, i2, cx, cy))          # Eq. proj_PD
                    C.add((iR, iRp, 2, cx, cy, i1, i2, cx, cy))          # P -> C
                if i1 is not None and j2 is not None:
                    P.add((iR, iRp, 1, cx, cy, i1, j2, (Px + cx) % L, (Py + cy) % L))   # D -> P
            for i2, (Wx, Wy) in enumerate(ff):
                i1 = idx.get(((Rx - Px + Wx) % L, (Ry - Py + Wy) % L))
                if i1 is not None:
                    C.add((iR, iRp, 3, (-Px) % L, (-Py) % L, i1, i2, Wx % L, Wy % L))   # Eq. proj_DC
    return P, C


@pytest.mark.parametrize("case", ["rashba_ff5_Lf24", "rashba_ff9_Lf25", "rashba_ff13_Lf30", "complete_4x4"])
def test_gather_tables_bit_exact(case):
    api = _api()
    spec = CASES[case]()
    m = api.Model(spec, api.FP64)
    P, C = _paper_gather_terms(spec)
    gP = [tuple(int(v) for v in r) for r in m.gather_table(0)]
    gC = [tuple(int(v) for v in r) for r in m.gather_table(1)]
    assert len(gP) == len(set(gP)) and len(gC) == len(set(gC))
    assert set(gP) == P
    assert set(gC) == C


@pytest.mark.parametrize("case", ["rashba_ff5_Lf24", "rashba_ff9_Lf25", "rashba_ff13_Lf30", "complete_4x4"])
@pytest.mark.parametrize("mask", [3, 1, 2])
def test_projections(case, mask):
    api = _api()
    spec = CASES[case]()
    m = api.Model(spec, api.FP64)
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=5, scale=0.4)
    A, amax = m.project(st, mask)
    A = A.cpu().numpy()
    ref, amax_ref = o.project(st, mask)
    assert rel(A, ref) < 1e-13
    assert amax == pytest.approx(amax_ref, rel=1e-14)


@pytest.mark.parametrize("case", ["rashba_ff9_Lf25", "rashba_ff13_Lf30"])
def test_projections_split(case):
    """Split path: the projected vertices are formed in FP32 (max relative error per entry ~ 1e-7)."""
    api = _api()
    spec = CASES[case]()
    m = api.Model(spec, api.SPLIT32)
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=5, scale=0.4)
    A, amax = m.project(st, 3)
    ref, amax_ref = o.project(st, 3)
    assert rel(A.cpu().numpy(), ref) < 1e-6
    assert amax == pytest.approx(amax_ref, rel=1e-6)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("T", [5.0, 0.3, 0.05])
def test_rhs_fp64(case, T):
    api = _api()
    spec = CASES[case]()
    m = api.Model(spec, api.FP64)
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=9, scale=0.3)
    d = m.rhs(T, st).cpu().numpy()
    ref, _ = o.rhs(T, st, 3)
    assert rel(d, ref) < TOL64


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("T", [5.0, 0.05])
@pytest.mark.parametrize("products", ["PRODUCTS_TC", "PRODUCTS_SIMT"])
def test_rhs_split(case, T, products):
    """Split path with tensor-core (tcgen05, 3xTF32) or CUDA-core FP32 products."""
    api = _api()
    spec = CASES[case]()
    m = api.Model(spec, api.SPLIT32, products=getattr(api, products))
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=9, scale=0.3)
    d = m.rhs(T, st).cpu().numpy()
    ref, _ = o.rhs(T, st, 3)
    assert rel(d, ref) < TOL32


@pytest.mark.parametrize("mask", [1, 2])
def test_rhs_single_channel(mask):
    api = _api()
    spec = CASES["rashba_ff9_Lf25"]()
    m = api.Model(spec, api.FP64)
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=2, scale=0.3)
    st[2 - mask] = 0.0   # the channel that does not flow is zero
    d = m.rhs(0.2, st, mask).cpu().numpy()
    ref, _ = o.rhs(0.2, st, mask)
    assert rel(d, ref) < TOL64
    assert np.abs(d[2 - mask]).max() == 0.0


def test_rhs_host_buffers_match_device():
    api = _api()
    spec = CASES["rashba_ff5_Lf24"]()
    m = api.Model(spec, api.FP64)
    st = inputs.random_state(spec, seed=4, scale=0.3)
    d_dev = m.rhs(0.4, st).cpu()
    hs = torch.from_numpy(st).pin_memory()
    ho = torch.empty_like(hs).pin_memory()
    m.rhs_host(0.4, hs, ho)
    assert torch.equal(d_dev, ho)


@pytest.mark.parametrize("prec", ["FP64", "SPLIT32"])
def test_rhs_host_batch_matches_device(prec):
    """The pipelined host-buffer entry point (copies of neighbouring steps overlapped with the evaluations) gives,
    step by step, exactly the device right-hand side: distinct states and temperatures, a repeated input buffer,
    pinned and pageable host memory, odd and even batch lengths, the symmetric-state flag."""
    api = _api()
    spec = CASES["rashba_ff9_Lf25"]()
    m = api.Model(spec, getattr(api, prec))
    states = [torch.from_numpy(inputs.random_state(spec, seed=s, scale=0.3)) for s in (1, 2, 3)]
    Ts = [0.4, 0.25, 0.9, 0.4, 0.6]
    ins = [states[0].pin_memory(), states[1].pin_memory(), states[2], states[0].pin_memory(), states[1]]
    outs = [torch.empty_like(states[0]).pin_memory() for _ in range(4)] + [torch.empty_like(states[0])]
    for n in (1, 2, 5):
        m.rhs_host_batch(Ts[:n], ins[:n], outs[:n])
        for i in range(n):
            assert torch.equal(outs[i], m.rhs(Ts[i], ins[i]).cpu()), (n, i)
    zero = m.zeros_state()
    X1 = (0.05 * m.rhs(0.5, zero)).cpu().contiguous()     # a symmetric state (one Euler step from X = 0)
    hs = [X1.pin_memory(), X1.pin_memory()]
    ho = [torch.empty_like(X1).pin_memory() for _ in range(3)]
    m.rhs_host_batch(0.4, [hs[0], hs[1], hs[0]], ho, symmetric=True)
    want = m.rhs(0.4, X1, symmetric=True).cpu()
    for o in ho:
        assert torch.equal(o, want)
    with pytest.raises(api.TufrgError):
        m.rhs_host_batch([0.4, -1.0], ins[:2], outs[:2])


def test_rhs_deterministic():
    api = _api()
    spec = CASES["rashba_ff9_Lf120"]()
    for prec in (api.FP64, api.SPLIT32):
        m = api.Model(spec, prec)
        st = inputs.random_state(spec, seed=4, scale=0.3)
        a = m.rhs(0.1, st).cpu()
        b = m.rhs(0.1, st).cpu()
        assert torch.equal(a, b)


def test_flow_fp64_matches_oracle():
    api = _api()
    spec = inputs.hubbard_square(U=3.0, Lq=6, nc=4, n_ff=5, filling=0.9, T_mu=0.02)
    o = oracle.Oracle(spec)
    st_ref, r_ref = o.flow(stop=6.0)
    m = api.Model(spec, api.FP64)
    st, r = m.flow(stop=6.0)
    assert r_ref["crossed"] == 1 and r["crossed"] == 1
    assert r["n_steps"] == r_ref["n_steps"] and r["n_reject"] == r_ref["n_reject"]
    assert r["Tc"] == pytest.approx(r_ref["Tc"], rel=1e-9)
    assert rel(st.cpu().numpy(), st_ref) < 1e-9


def test_flow_split_critical_scale_within_one_percent():
    api = _api()
    spec = inputs.hubbard_square(U=3.0, Lq=6, nc=4, n_ff=5, filling=0.9, T_mu=0.02)
    o = oracle.Oracle(spec)
    _, r_ref = o.flow(stop=6.0)
    m = api.Model(spec, api.SPLIT32)
    st, r = m.flow(stop=6.0)
    assert r["crossed"] == 1
    assert abs(r["Tc"] / r_ref["Tc"] - 1) < 0.01


def test_flow_closed_form_particle_particle():
    """GPU flow in P-only mode reproduces the paper's closed form (Sec. 4, Eq. sol_spin)."""
    api = _api()
    U = 2.5
    spec = inputs.rashba_hubbard(tp=-0.2, alpha=0.3, U=U, mu=-0.9, Lq=6, nc=2, n_ff=5)
    m = api.Model(spec, api.FP64)
    st, r = m.flow(T0=10.0, T_end=0.3, rtol=1e-10, atol=1e-12, stop=1e9, mask=1)
    o = oracle.Oracle(spec)
    st_ref, _ = o.flow(T0=10.0, T_end=0.3, rtol=1e-10, atol=1e-12, stop=1e9, chmask=1)
    assert rel(st.cpu().numpy(), st_ref) < 1e-9


@pytest.mark.parametrize("prec", ["FP64", "SPLIT32"])
def test_rhs_full_size_rashba_24x24(prec):
    """The benchmark workload itself (Lq = 24, nc = 8, N_ff = 9, M = 36): full right-hand side."""
    api = _api()
    spec = inputs.rashba_q24_k8_ff9(0)
    m = api.Model(spec, getattr(api, prec))
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=1, scale=0.2)
    d = m.rhs(0.1, st).cpu().numpy()
    ref, _ = o.rhs(0.1, st, 3)
    assert rel(d, ref) < (TOL64 if prec == "FP64" else TOL32)


@pytest.fixture(scope="module")
def full_size_flow_state():
    """The state the benchmark evaluates: the split flow of the 24x24 / 8x8 Rashba workload from T0 = 10 down to
    T = 0.1.  Every state of a flow from X = 0 carries the loop symmetries exactly (dX/dT of the other momenta
    is written from the orbit representatives), so it may be evaluated with TUFRG_SYMMETRIC_STATE."""
    api = _api()
    spec = inputs.rashba_q24_k8_ff9(0)
    m = api.Model(spec, api.SPLIT32)
    st, r = m.flow(T_end=0.1, stop=1e9)
    assert r["T_last"] == pytest.approx(0.1) and m.symmetric_state_path
    return spec, st


@pytest.mark.parametrize("prec", ["FP64", "SPLIT32"])
def test_rhs_full_size_symmetric_state_path(full_size_flow_state, prec):
    """The benchmark's timed call itself at full size (Lq = 24, nc = 8, N_ff = 9, M = 36, T = 0.1): tufrg_rhs with
    TUFRG_SYMMETRIC_STATE on the mid-flow state - loop k-sums at the 91 orbit representatives (split path), their
    reduction, projections and orbit products at the representatives, dX/dT of all 576 momenta written through the orbit
    index maps - against the oracle's full right-hand side, element by element: FP64 <= 1e-10, split <= 1e-4."""
    api = _api()
    spec, st = full_size_flow_state
    m = api.Model(spec, getattr(api, prec))
    if prec == "SPLIT32":
        # the FP64 two-band path sums every momentum directly and ignores the flag (its general path is checked)
        assert m.n_loop_q == 91 and m.symmetric_state_path
    d = m.rhs(0.1, st, symmetric=True).cpu().numpy()
    ref, _ = oracle.Oracle(spec).rhs(0.1, st.cpu().numpy(), 3)
    assert np.abs(ref).max() > 1.0
    assert rel(d, ref) < (TOL64 if prec == "FP64" else TOL32), rel(d, ref)


def test_flow_full_size_hubbard_fp64_matches_oracle():
    """The single-band Hubbard workload at full size (8x8 transfer mesh, 16x16 fine points per cell, N_ff = 5,
    filling 0.45 per spin, U = 3): the FP64 GPU flow from T0 = 10 to T_end = 0.02 (the integration of the flow
    equations, Sec. 3.1) takes the oracle's step sequence - the same accepted and rejected steps - and ends on
    the oracle's state within 1e-9."""
    api = _api()
    spec = inputs.hubbard_q8_k16_ff5()
    o = oracle.Oracle(spec)
    st_ref, r_ref = o.flow()
    m = api.Model(spec, api.FP64)
    assert abs(m.mu - o.mu) < 1e-12
    st, r = m.flow()
    assert r["n_steps"] == r_ref["n_steps"] and r["n_reject"] == r_ref["n_reject"]
    assert r["crossed"] == r_ref["crossed"]
    assert r["Tc"] == pytest.approx(r_ref["Tc"], rel=1e-9)
    assert r["amax"] == pytest.approx(r_ref["amax"], rel=1e-9)
    assert rel(st.cpu().numpy(), st_ref) < 1e-9


def test_invalid_temperature_is_rejected():
    api = _api()
    m = api.Model(CASES["rashba_ff5_Lf24"](), api.FP64)
    with pytest.raises(api.TufrgError) as e:
        m.rhs(-1.0, m.zeros_state())
    assert e.value.status == 1


# ------------------------------------------------------------------ N_s = 6: three orbitals with atomic SOC

T2G = {
    "t2g_ff1_Lf8": lambda: inputs.t2g_soc(seed=1, Lq=4, nc=2, n_ff=1, filling=4.0, T_mu=0.05),          # M = 36
    "t2g_ff5_Lf8": lambda: inputs.t2g_soc(seed=2, Lq=4, nc=2, n_ff=5, filling=4.0, T_mu=0.05),          # M = 180
    "t2g_ff9_Lf10": lambda: inputs.t2g_soc(seed=3, Lq=5, nc=2, n_ff=9, filling=4.0, T_mu=0.05),         # M = 324
}


@pytest.mark.parametrize("case", list(T2G))
def test_t2g_bands_and_mu(case):
    api = _api()
    spec = T2G[case]()
    m = api.Model(spec, api.FP64)
    o = oracle.Oracle(spec)
    E, U = m.bands()
    E, U = E.cpu().numpy(), U.cpu().numpy()
    assert np.abs(E - o.E).max() < 1e-12
    assert np.abs(np.einsum("kji,kjl->kil", U.conj(), U) - np.eye(6)).max() < 1e-12
    assert abs(m.mu - o.mu) < 1e-11


def _t2g_model(api, spec, prec, **kw):
    """FP64, split precision with the tensor-core loop k-sum (the default where it applies) or with the
    CUDA-core loop k-sum."""
    if prec == "SPLIT32_SIMTLOOPS":
        m = api.Model(spec, api.SPLIT32, loops=api.LOOPS_SIMT, **kw)
        assert m.loops_backend == "simt"
        return m
    m = api.Model(spec, getattr(api, prec), **kw)
    assert m.loops_backend == ("tc" if prec == "SPLIT32" else "simt")
    return m


@pytest.mark.parametrize("case", list(T2G))
@pytest.mark.parametrize("prec", ["FP64", "SPLIT32", "SPLIT32_SIMTLOOPS"])
def test_t2g_loops(case, prec):
    """Loops of the t2g model (N_s = 6) against the oracle: FP64 on the CUDA cores, and the split path with the
    per-column orbital sums as 3xTF32 GEMMs on the tensor cores (Lf = 8 and the ragged Lf = 10, a last stage of
    two rows) or as FP32 FMAs on the CUDA cores."""
    api = _api()
    spec = T2G[case]()
    m = _t2g_model(api, spec, prec)
    o = oracle.Oracle(spec)
    for T in (0.15, 1.3):
        L = m.loops(T).cpu().numpy()
        for ch in (0, 1):
            ref = o.loops(T, ch)
            assert rel(L[ch], ref) < (TOL64 if prec == "FP64" else 2e-5), (ch, rel(L[ch], ref))


@pytest.mark.parametrize("case", list(T2G))
@pytest.mark.parametrize("prec", ["FP64", "SPLIT32", "SPLIT32_SIMTLOOPS"])
def test_t2g_loops_symmetry(case, prec):
    """The t2g model (orbitals yz, xz, xy with atomic SOC) has the point group with orbital x spin
    unitaries: one momentum per orbit is summed and the result equals the full k-sum (with every momentum
    summed the tensor-core kernel's last group of three momenta is incomplete: 16 or 25 momenta)."""
    api = _api()
    spec = T2G[case]()
    m = _t2g_model(api, spec, prec)
    full = _t2g_model(api, spec, prec, symmetry=api.SYMMETRY_OFF)
    assert m.n_loop_q == _n_orbits(spec.Lq, C4V) and full.n_loop_q == spec.Lq ** 2
    L, Lfull = m.loops(0.15).cpu().numpy(), full.loops(0.15).cpu().numpy()
    assert rel(L, Lfull) < (1e-13 if prec == "FP64" else 2e-6)
    o = oracle.Oracle(spec)
    for ch in (0, 1):
        assert rel(Lfull[ch], o.loops(0.15, ch)) < (TOL64 if prec == "FP64" else 2e-5)


def test_t2g_loops_tc_matches_cuda_cores_ragged():
    """Tensor-core and CUDA-core loop k-sums of the same split model on a ragged fine mesh (Lf = 15: the last
    stage of each column holds three rows) with 9 bonds, both channels, two temperatures."""
    api = _api()
    spec = inputs.t2g_soc(seed=4, Lq=5, nc=3, n_ff=9, filling=4.0, T_mu=0.05)
    mt = _t2g_model(api, spec, "SPLIT32")
    ms = _t2g_model(api, spec, "SPLIT32_SIMTLOOPS")
    o = oracle.Oracle(spec)
    for T in (0.08, 0.6):
        Lt, Ls = mt.loops(T).cpu().numpy(), ms.loops(T).cpu().numpy()
        assert rel(Lt, Ls) < 4e-6
        for ch in (0, 1):
            assert rel(Lt[ch], o.loops(T, ch)) < 2e-5


@pytest.mark.parametrize("case", list(T2G))
@pytest.mark.parametrize("prec", ["FP64", "SPLIT32", "SPLIT32_SIMT"])
def test_t2g_rhs(case, prec):
    api = _api()
    spec = T2G[case]()
    if prec == "SPLIT32_SIMT":
        m = api.Model(spec, api.SPLIT32, products=api.PRODUCTS_SIMT)
    elif prec == "SPLIT32":
        m = api.Model(spec, api.SPLIT32, products=api.PRODUCTS_TC)
    else:
        m = api.Model(spec, api.FP64)
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=13, scale=0.15)
    d = m.rhs(0.2, st).cpu().numpy()
    ref, _ = o.rhs(0.2, st, 3)
    assert rel(d, ref) < (TOL64 if prec == "FP64" else TOL32)


@pytest.mark.parametrize("shape", ["t2g_ff13", "bilayer_ff5", "rashba_ff5"])
def test_tc_products_tile_shapes(shape):
    """The tensor-core products at the tile shapes their work list takes: M = 468 (N_s = 6, 4 row tiles x 5 column
    tiles of 96), M = 80 (N_s = 4, one row tile, 80-column tile), M = 20 (N_s = 2, a 32-column tile), against the
    oracle's right-hand side, on both the general and the symmetric-state path."""
    api = _api()
    spec = {"t2g_ff13": lambda: inputs.t2g_soc(seed=4, Lq=5, nc=2, n_ff=13, filling=4.0, T_mu=0.05),
            "bilayer_ff5": lambda: inputs.rashba_bilayer(Lq=5, nc=2, n_ff=5),
            "rashba_ff5": lambda: inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=2.5, mu=-0.8, Lq=6, nc=4, n_ff=5)}[shape]()
    m = api.Model(spec, api.SPLIT32, products=api.PRODUCTS_TC)
    assert m.products == "tc"
    o = oracle.Oracle(spec)
    st = inputs.random_state(spec, seed=21, scale=0.15)
    d = m.rhs(0.2, st).cpu().numpy()
    ref, _ = o.rhs(0.2, st, 3)
    assert rel(d, ref) < TOL32
    # a symmetric state through the representatives' products (the orbit copy writes the other momenta)
    X1 = 0.05 * m.rhs(0.5, m.zeros_state())
    sym = m.rhs(0.3, X1, symmetric=True).cpu().numpy()
    ref1, _ = o.rhs(0.3, X1.cpu().numpy(), 3)
    assert rel(sym, ref1) < TOL32


def test_tc_products_tile_autotune():
    """With the products backend on AUTO the tensor cores are timed at two column-tile widths (M = 180: 96 and 64
    columns) and the faster kept; the tiling changes no output element's summation order, so the products equal
    those at the default width bit for bit."""
    api = _api()
    spec = T2G["t2g_ff5_Lf8"]()
    m = api.Model(spec, api.SPLIT32)
    t = m.products_tiles_tuning_ms
    assert len(t) == 2 and all(v > 0 for v in t)
    assert m.products_tile_width == (96 if t[0] <= t[1] else 64)
    ref = api.Model(spec, api.SPLIT32, products=api.PRODUCTS_TC)
    assert ref.products_tile_width == 96 and ref.products_tiles_tuning_ms == []
    st = inputs.random_state(spec, seed=5, scale=0.15)
    if m.products == "tc":
        assert torch.equal(m.rhs(0.2, st), ref.rhs(0.2, st))
    assert api.Model(spec, api.FP64).products_tile_width == 0


BILAYER = {   # N_s = 4: two Rashba layers with opposite couplings, interlayer hopping, onsite U per layer
    "bilayer_ff5_Lf10": lambda: inputs.rashba_bilayer(Lq=5, nc=2, n_ff=5),                            # M = 80
    "bilayer_ff9_Lf8": lambda: inputs.rashba_bilayer(Lq=4, nc=2, n_ff=9, alpha=0.25, t_perp=0.3),    # M = 144
}


@pytest.mark.parametrize("case", list(BILAYER))
@pytest.mark.parametrize("prec", ["FP64", "SPLIT32"])
def test_bilayer_loops_and_rhs(case, prec):
    """N_s = 4 (the multi-orbital loop kernel with 2 x 2 tiles, products at M = 16 N_ff, symmetry tables for a
    4-state unitary): loops and right-hand sides against the oracle."""
    api = _api()
    spec = BILAYER[case]()
    m = api.Model(spec, getattr(api, prec))
    o = oracle.Oracle(spec)
    L = m.loops(0.15).cpu().numpy()
    for ch in (0, 1):
        assert rel(L[ch], o.loops(0.15, ch)) < (TOL64 if prec == "FP64" else 2e-5), ch
    st = inputs.random_state(spec, seed=13, scale=0.15)
    ref, _ = o.rhs(0.2, st, 3)
    assert rel(m.rhs(0.2, st).cpu().numpy(), ref) < (TOL64 if prec == "FP64" else TOL32)


def test_bilayer_flows():
    """N_s = 4 flows: the FP64 flow takes the oracle's step sequence and reaches its state and critical scale to
    1e-9; the split flow (symmetric states, representatives and scatter) stays within 1% of the FP64 critical
    scale with the same leading channel."""
    api = _api()
    spec = BILAYER["bilayer_ff5_Lf10"]()
    st_ref, r_ref = oracle.Oracle(spec).flow(T0=10.0, T_end=1e-3, stop=6.0)
    st, r = api.Model(spec, api.FP64).flow(T0=10.0, T_end=1e-3, stop=6.0)
    assert r["n_steps"] == r_ref["n_steps"] and r["n_reject"] == r_ref["n_reject"] and r["crossed"] == r_ref["crossed"]
    assert r["Tc"] == pytest.approx(r_ref["Tc"], rel=1e-9)
    assert rel(st.cpu().numpy(), st_ref) < 1e-9
    _, r32 = api.Model(spec, api.SPLIT32).flow(T0=10.0, T_end=1e-3, stop=6.0)
    assert r32["crossed"] == r["crossed"] and abs(r32["Tc"] / r["Tc"] - 1) < 0.01
    assert r32["lead_channel"] == r["lead_channel"]


@pytest.mark.parametrize("prec", ["FP64", "SPLIT32"])
def test_t2g_full_size_sampled_loops(prec):
    """The 32x32 / 6x6-per-cell t2g workload (N_s = 6, M = 324): loops at sampled transfer momenta."""
    api = _api()
    spec = inputs.t2g_q32_k6_ff9(0)
    m = api.Model(spec, getattr(api, prec))
    o = oracle.Oracle(spec, mu=m.mu)
    L = m.loops(0.1).cpu().numpy()
    qs = [0, 33, 517]
    for ch in (0, 1):
        ref = o.loops_at(0.1, ch, qs)
        assert rel(L[ch][qs], ref) < (TOL64 if prec == "FP64" else 2e-5)


# ------------------------------------------------------------------ batched uneven flows

def test_flow_batch_matches_single_flows():
    """Uneven Rashba/Hubbard instances (different meshes and bond sets) run together through
    tufrg_flow_batch give exactly the flows tufrg_flow gives one at a time."""
    api = _api()
    specs = [inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=3.2, mu=-0.8, Lq=6, nc=4, n_ff=5),
             inputs.rashba_hubbard(tp=-0.25, alpha=0.35, U=3.4, mu=-1.0, Lq=8, nc=3, n_ff=9),
             inputs.hubbard_square(U=3.0, Lq=6, nc=4, n_ff=5, filling=0.9, T_mu=0.02),
             inputs.rashba_hubbard(tp=-0.05, alpha=0.1, U=2.8, mu=-0.7, Lq=10, nc=2, n_ff=13)]
    for prec in (api.FP64, api.SPLIT32):
        single = []
        for sp in specs:
            m = api.Model(sp, prec)
            _, r = m.flow(stop=6.0)
            single.append(r)
        streams = [torch.cuda.Stream() for _ in specs]
        models = [api.Model(sp, prec, stream=s) for sp, s in zip(specs, streams)]
        batch = api.flow_batch(models, stop=6.0)
        for r1, r2 in zip(single, batch):
            assert r1["n_steps"] == r2["n_steps"] and r1["n_reject"] == r2["n_reject"]
            assert r1["crossed"] == r2["crossed"]
            assert r1["Tc"] == r2["Tc"]


def test_rhs_graph_replay_matches_direct_launches():
    """tufrg_rhs replays a captured graph per (input, output, mask); the results equal the direct launches (taken
    while the phases are timed) bit for bit, for both precisions, both state flags, new buffers and more buffer
    pairs than the graph cache holds, on the legacy default stream (graphs on a private stream) and on a stream of
    the caller's."""
    api = _api()
    spec = CASES["rashba_ff9_Lf25"]()
    for prec, stream in ((api.SPLIT32, None), (api.FP64, None), (api.SPLIT32, torch.cuda.Stream())):
        with (torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext()):
            m = api.Model(spec, prec, stream=stream)
            X1 = 0.05 * m.rhs(0.5, m.zeros_state())
            for sym in (False, True):
                for T in (0.4, 0.13):
                    m.timing_begin()
                    want = m.rhs(T, X1, symmetric=sym).clone()
                    m.timing_end()
                    outs = [m.zeros_state() for _ in range(6)]
                    for rep in range(2):
                        for o in outs:
                            m.rhs(T, X1, out=o, symmetric=sym)
                            assert torch.equal(o, want)
            one = m.rhs(0.2, X1, mask=api.CH_P)
            m.timing_begin()
            ref = m.rhs(0.2, X1, mask=api.CH_P)
            m.timing_end()
            assert torch.equal(one, ref) and not torch.any(one[1])
        torch.cuda.synchronize()


def test_loop_tile_autotune():
    """The two-band split loop kernel's launch shape (ky ranges per column) is timed at set-up over every candidate
    and the fastest kept; a second model of the same shape reuses the choice (the same summation order), and the
    loops at the chosen shape match the oracle."""
    api = _api()
    spec = CASES["rashba_ff9_Lf25"]()
    m = api.Model(spec, api.SPLIT32)
    t = m.loop_tiles_tuning_ms
    assert len(t) >= 2 and all(v > 0 for v in t.values())
    assert m.loop_ky_chunks == min(t, key=t.get)
    assert all((spec.Lq * spec.nc + c - 1) // c >= 8 for c in t)
    m2 = api.Model(spec, api.SPLIT32)
    assert m2.loop_ky_chunks == m.loop_ky_chunks and m2.loop_tiles_tuning_ms == t
    o = oracle.Oracle(spec)
    L = m.loops(0.07).cpu().numpy()
    for ch in (0, 1):
        assert rel(L[ch], o.loops(0.07, ch)) < 2e-5
    # the FP64 path keeps its heuristic shape
    assert api.Model(spec, api.FP64).loop_tiles_tuning_ms == {}


def test_flow_batch_mixed_spin_orbitals():
    """A batch that mixes two-band (N_s = 2) and bilayer (N_s = 4) instances, with different meshes and bond sets,
    gives exactly the flows tufrg_flow gives one at a time, in both precisions."""
    api = _api()
    specs = [inputs.rashba_bilayer(tp=-0.2, alpha=0.3, t_perp=0.4, U=3.0, mu=-0.9, Lq=6, nc=3, n_ff=5),
             inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=3.2, mu=-0.8, Lq=8, nc=3, n_ff=9),
             inputs.rashba_bilayer(tp=-0.1, alpha=0.2, t_perp=0.3, U=2.8, mu=-0.7, Lq=4, nc=4, n_ff=9),
             inputs.hubbard_square(U=3.0, Lq=6, nc=4, n_ff=5, filling=0.9, T_mu=0.02)]
    assert sorted({sp.n_s for sp in specs}) == [2, 4]
    for prec in (api.FP64, api.SPLIT32):
        single = [api.Model(sp, prec).flow(stop=6.0)[1] for sp in specs]
        streams = [torch.cuda.Stream() for _ in specs]
        models = [api.Model(sp, prec, stream=s) for sp, s in zip(specs, streams)]
        batch = api.flow_batch(models, stop=6.0)
        for r1, r2 in zip(single, batch):
            assert r1["n_steps"] == r2["n_steps"] and r1["n_reject"] == r2["n_reject"]
            assert r1["crossed"] == r2["crossed"]
            assert r1["Tc"] == r2["Tc"]


def test_flow_critical_at_start():
    """max|A| of the bare vertex already above the stop value: the flow is critical at T0 (Lambda_c = T0, no
    step, one evaluation), alone and inside a batch next to a flow that runs; the oracle agrees."""
    api = _api()
    specs = [inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=3.2, mu=-0.8, Lq=6, nc=2, n_ff=5),     # max|V0| = 1.6
             inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=2.8, mu=-0.8, Lq=6, nc=2, n_ff=5)]     # max|V0| = 1.4
    _, ref = oracle.Oracle(specs[0]).flow(stop=1.5)
    assert ref["crossed"] == 1 and ref["n_steps"] == 0 and ref["Tc"] == pytest.approx(10.0)
    for prec in (api.FP64, api.SPLIT32):
        _, r = api.Model(specs[0], prec).flow(stop=1.5)
        assert r["crossed"] == 1 and r["n_steps"] == 0 and r["n_rhs"] == 1 and r["Tc"] == pytest.approx(10.0)
        assert r["amax"] == pytest.approx(1.6, rel=1e-6)
        streams = [torch.cuda.Stream() for _ in specs]
        models = [api.Model(sp, prec, stream=s) for sp, s in zip(specs, streams)]
        batch = api.flow_batch(models, stop=1.5)
        assert batch[0]["crossed"] == 1 and batch[0]["n_steps"] == 0 and batch[0]["Tc"] == pytest.approx(10.0)
        _, r1 = api.Model(specs[1], prec).flow(stop=1.5)
        assert batch[1]["n_steps"] == r1["n_steps"] > 0 and batch[1]["Tc"] == r1["Tc"]


def test_flow_step_limit_and_bad_options():
    """The step limit (accepted + rejected attempts) ends a flow with TUFRG_ENOTCONV; options outside their
    ranges are rejected with TUFRG_EINVAL before any work; the model stays usable after both."""
    api = _api()
    spec = inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=2.8, mu=-0.8, Lq=6, nc=2, n_ff=5)
    m = api.Model(spec, api.FP64)
    with pytest.raises(api.TufrgError) as e:
        m.flow(stop=50.0, max_steps=2)
    assert e.value.status == 5
    for bad in (dict(T0=0.1, T_end=0.2), dict(rtol=0.0), dict(h0=0.05), dict(mask=0), dict(max_steps=0)):
        with pytest.raises(api.TufrgError) as e:
            m.flow(**bad)
        assert e.value.status == 1, bad
    _, r = m.flow(T0=10.0, T_end=1.0, stop=50.0)
    _, ref = oracle.Oracle(spec).flow(T0=10.0, T_end=1.0, stop=50.0)
    assert r["n_steps"] == ref["n_steps"] and r["Tc"] == pytest.approx(ref["Tc"], rel=1e-12)


def test_flow_batch_matches_oracle():
    api = _api()
    specs = [inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=3.2, mu=-0.8, Lq=6, nc=2, n_ff=5),
             inputs.hubbard_square(U=3.0, Lq=4, nc=4, n_ff=5, filling=0.9, T_mu=0.02)]
    streams = [torch.cuda.Stream() for _ in specs]
    models = [api.Model(sp, api.FP64, stream=s) for sp, s in zip(specs, streams)]
    batch = api.flow_batch(models, stop=4.0)
    for sp, r in zip(specs, batch):
        _, ref = oracle.Oracle(sp).flow(stop=4.0)
        assert r["n_steps"] == ref["n_steps"]
        assert r["Tc"] == pytest.approx(ref["Tc"], rel=1e-9)


def test_device_timeout_flag_propagates_to_the_host():
    """TUFRG_ETIMEOUT reaches the caller of every entry point that reads the device error flag, raised from the
    host (tufrg_set_device_error writes the flag a bounded device wait sets when it gives up; no device wait is
    made to run out), and the model works again once the flag is cleared."""
    api = _api()
    spec = inputs.rashba_hubbard(tp=-0.1, alpha=0.2, U=2.8, mu=-0.8, Lq=6, nc=2, n_ff=5)
    m = api.Model(spec, api.SPLIT32)
    hs = m.zeros_state().cpu().pin_memory()
    ho = torch.empty_like(hs).pin_memory()
    assert m._L.tufrg_set_device_error(m._h, 1) == 0
    with pytest.raises(api.TufrgError) as e:
        m.rhs_host(0.4, hs, ho)
    assert e.value.status == 6
    with pytest.raises(api.TufrgError) as e:
        m.rhs_host_batch(0.4, [hs, hs], [ho, ho])
    assert e.value.status == 6
    with pytest.raises(api.TufrgError) as e:
        m.flow(T0=10.0, T_end=5.0)
    assert e.value.status == 6
    assert m._L.tufrg_set_device_error(m._h, 0) == 0
    m.rhs_host(0.4, hs, ho)
    _, r = m.flow(T0=10.0, T_end=5.0)
    assert r["T_last"] == pytest.approx(5.0)


@pytest.mark.parametrize("case,prec", [("rashba_ff9_Lf25", "SPLIT32"), ("rashba_ff5_Lf24", "FP64"),
                                       ("t2g_ff5_Lf8", "SPLIT32"), ("t2g_ff9_Lf10", "FP64"), ("hubbard_ff5_Lf24", "SPLIT32")])
def test_rhs_shards_emulated_on_one_gpu(case, prec):
    """The right-hand side split over shards of transfer momenta through the C ABI (tufrg_rhs_shard_transform, the
    sum of the parts, tufrg_rhs_shard_finish), three uneven shards run one after the other on one GPU (the sum
    stands in for the all-reduce between GPUs): every shard's rows equal those of tufrg_rhs and of the oracle.
    With loop symmetries the loop scratch holds fewer momenta than a shard lists (t2g: 6 orbit representatives),
    so the listed loops run in chunks."""
    from paper_1710_08830_gb300 import shard
    api = _api()
    spec = (CASES.get(case) or T2G[case])()
    m = api.Model(spec, getattr(api, prec))
    st = inputs.random_state(spec, seed=21, scale=0.25)
    rng = np.random.default_rng(3)
    perm = rng.permutation(spec.Nq)
    cut = [0, spec.Nq // 4, (2 * spec.Nq) // 3, spec.Nq]
    shards = [np.sort(perm[cut[i]:cut[i + 1]]) if i != 1 else perm[cut[i]:cut[i + 1]] for i in range(3)]
    xr = sum(m.shard_transform(st[:, s], s) for s in shards)
    full = m.rhs(0.3, st).cpu().numpy()
    ref, _ = oracle.Oracle(spec).rhs(0.3, st, 3)
    tol = TOL64 if prec == "FP64" else TOL32
    for s in shards:
        d = m.shard_finish(0.3, st[:, s], s, xr).cpu().numpy()
        assert rel(d, full[:, s]) < (1e-12 if prec == "FP64" else 2e-6)
        assert np.abs(d - ref[:, s]).max() < tol * np.abs(ref).max()
    # the partition helper's shards give the same rows
    q0 = shard.partition(spec.Nq, 2, 0)
    q1 = shard.partition(spec.Nq, 2, 1)
    xr2 = m.shard_transform(st[:, q0], q0) + m.shard_transform(st[:, q1], q1)
    d1 = m.shard_finish(0.3, st[:, q1], q1, xr2).cpu().numpy()
    assert np.abs(d1 - ref[:, q1]).max() < tol * np.abs(ref).max()
    with pytest.raises(api.TufrgError) as e:
        m.shard_transform(st[:, [0, 0]], [0, 0])                 # repeated momentum
    assert e.value.status == 1
