"""The seeded workload descriptors against the model definitions they state: lattice sizes, bond sets, the
dispersion and spin-orbit terms of H(k) evaluated here from their textbook forms, the bare vertices, the seeded
draws and their ranges, and reproducibility (CPU, no GPU)."""
import numpy as np
import pytest

from paper_1710_08830_gb300 import inputs

SX = np.array([[0, 1], [1, 0]], complex)
SY = np.array([[0, -1j], [1j, 0]])


def h_of_k(spec, k):
    return np.einsum("h,hab->ab", np.exp(1j * (spec.hop_R @ k)), spec.hop_t)


def _ks(n=5, seed=0):
    return np.random.default_rng(seed).uniform(-np.pi, np.pi, (n, 2))


def eps(k, t, tp):
    return -2 * t * (np.cos(k[0]) + np.cos(k[1])) - 4 * tp * np.cos(k[0]) * np.cos(k[1])


def test_hubbard_workload():
    """Single band with spin, t = 1, t' = -0.25, 0.45 electrons per spin, U = 3, 5 bonds, 8x8 q, 16x16 k per
    cell: H(k) = eps(k) 1, V0 = (U/2)(d13 d24 - d14 d23)."""
    s = inputs.hubbard_q8_k16_ff5()
    assert (s.n_s, s.n_ff, s.M, s.Lq, s.nc, s.Nq, s.Nk) == (2, 5, 20, 8, 16, 64, 16384)
    assert s.filling == pytest.approx(0.9)
    assert sorted(map(tuple, s.ff_R.tolist())) == [(-1, 0), (0, -1), (0, 0), (0, 1), (1, 0)]
    for k in _ks():
        assert np.allclose(h_of_k(s, k), eps(k, 1.0, -0.25) * np.eye(2), atol=1e-14)
    V = s.V0
    assert V[0, 1, 0, 1] == pytest.approx(1.5) and V[0, 1, 1, 0] == pytest.approx(-1.5)
    assert np.allclose(V, -V.transpose(1, 0, 2, 3)) and np.allclose(V, -V.transpose(0, 1, 3, 2))


@pytest.mark.parametrize("seed", [0, 1, 4])
def test_rashba_workload(seed):
    """Rashba-Hubbard: t = 1, t' = -0.2, alpha = 0.3, U = 2.5, mu ~ U[-1.2, -0.6] from the seed, 9 bonds (up
    to second neighbours), 24x24 q, 8x8 k per cell: H(k) = eps(k) + alpha (-sin ky sigma_x + sin kx sigma_y)."""
    s = inputs.rashba_q24_k8_ff9(seed)
    assert (s.n_s, s.n_ff, s.M, s.Lq, s.nc, s.Nq, s.Nk) == (2, 9, 36, 24, 8, 576, 36864)
    assert -1.2 <= s.mu <= -0.6 and s.filling == 0
    assert s.mu == inputs.rashba_q24_k8_ff9(seed).mu                        # reproducible
    assert s.mu == pytest.approx(np.random.default_rng(seed).uniform(-1.2, -0.6))
    assert {tuple(r) for r in s.ff_R.tolist()} == {(x, y) for x in (-1, 0, 1) for y in (-1, 0, 1)}
    for k in _ks(seed=seed):
        want = eps(k, 1.0, -0.2) * np.eye(2) + 0.3 * (-np.sin(k[1]) * SX + np.sin(k[0]) * SY)
        assert np.allclose(h_of_k(s, k), want, atol=1e-14)
    assert s.V0[0, 1, 0, 1] == pytest.approx(1.25)


def test_t2g_workload():
    """t2g + SOC: N_s = 6, 9 bonds (M = 324), 32x32 q, 6x6 k per cell, hoppings from the seed in [0.5, 1],
    atomic SOC with lambda = 0.2 (a doublet at -lambda and a quartet at lambda / 2), Kanamori
    U = 2, J = 0.4 (U' = U - 2J), four electrons in six states."""
    s = inputs.t2g_q32_k6_ff9(0)
    assert (s.n_s, s.n_ff, s.M, s.Lq, s.nc, s.Nq, s.Nk) == (6, 9, 324, 32, 6, 1024, 36864)
    assert s.filling == pytest.approx(4.0)
    p = s.params
    assert all(0.5 <= p[x] <= 1.0 for x in ("t_par", "t_perp", "t_xy"))
    assert (p["t_par"], p["t_perp"], p["t_xy"]) == tuple(np.random.default_rng(0).uniform(0.5, 1.0, 3))
    # onsite block: the SOC spectrum
    onsite = [t for R, t in zip(s.hop_R.tolist(), s.hop_t) if R == [0, 0]]
    assert len(onsite) == 1
    # (lambda/2) sum_i L_i (x) sigma_i with (L_i)_ab = -i eps_iab: L.sigma is -2 on the doublet, +1 on the quartet
    ev = np.sort(np.linalg.eigvalsh(onsite[0]))
    assert np.allclose(ev, [-0.2, -0.2, 0.1, 0.1, 0.1, 0.1], atol=1e-14)
    # the orbital hoppings: yz along y t_par, along x t_perp; xz mirrored; xy t_xy both ways (spin diagonal)
    k = np.array([0.37, -1.21])
    H = h_of_k(s, k) - onsite[0]
    diag = [-2 * (p["t_perp"] * np.cos(k[0]) + p["t_par"] * np.cos(k[1])),
            -2 * (p["t_par"] * np.cos(k[0]) + p["t_perp"] * np.cos(k[1])),
            -2 * p["t_xy"] * (np.cos(k[0]) + np.cos(k[1]))]
    assert np.allclose(H, np.kron(np.diag(diag), np.eye(2)), atol=1e-14)
    # Kanamori: intra-orbital U between opposite spins, U' between orbitals, Hund J
    V = s.V0
    up, dn = 0, 1
    assert V[0 * 2 + up, 0 * 2 + dn, 0 * 2 + up, 0 * 2 + dn] == pytest.approx(1.0)        # U / 2
    assert V[0 * 2 + up, 1 * 2 + dn, 0 * 2 + up, 1 * 2 + dn] == pytest.approx(0.6)        # U' / 2
    assert np.allclose(V, -V.transpose(0, 1, 3, 2))


def test_bilayer_model():
    """The N_s = 4 Rashba bilayer: each layer eps(k) + (-1)^layer alpha (-sin ky sigma_x + sin kx sigma_y),
    -t_perp between the layers at the same site, an onsite Hubbard U within each layer and none between them."""
    s = inputs.rashba_bilayer(tp=-0.2, alpha=0.3, t_perp=0.4, U=2.5, Lq=4, nc=2, n_ff=5)
    assert (s.n_s, s.M) == (4, 80)
    for k in _ks(seed=3):
        g = 0.3 * (-np.sin(k[1]) * SX + np.sin(k[0]) * SY)
        want = eps(k, 1.0, -0.2) * np.eye(4) + np.kron(np.diag([1.0, -1.0]), g) \
            - 0.4 * np.kron(np.array([[0, 1], [1, 0]]), np.eye(2))
        assert np.allclose(h_of_k(s, k), want, atol=1e-14)
    one = inputs.onsite_hubbard_vertex(2.5)
    assert np.allclose(s.V0[:2, :2, :2, :2], one) and np.allclose(s.V0[2:, 2:, 2:, 2:], one)
    assert np.abs(s.V0[0, 2, 0, 2]) == 0 and np.abs(s.V0[0, 3, 0, 3]) == 0


def test_batch_workload():
    """64 uneven Rashba/Hubbard instances: t' in [-0.3, 0], alpha in [0, 0.4], U in [1.5, 3.5],
    Lq in {16, 24, 32, 48}, N_ff in {5, 9, 13}, mu in [-1.2, -0.6]; reproducible from the seed."""
    b = inputs.rashba_batch(0)
    assert len(b) == 64
    for s in b:
        p = s.params
        assert -0.3 <= p["tp"] <= 0 and 0 <= p["alpha"] <= 0.4 and 1.5 <= p["U"] <= 3.5 and -1.2 <= p["mu"] <= -0.6
        assert s.Lq in (16, 24, 32, 48) and s.n_ff in (5, 9, 13) and s.nc == 8
    assert len({s.Lq for s in b}) == 4 and len({s.n_ff for s in b}) == 3
    b2 = inputs.rashba_batch(0)
    assert all(x.params == y.params and x.Lq == y.Lq and x.n_ff == y.n_ff for x, y in zip(b, b2))
