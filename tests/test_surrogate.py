"""Learned loop surrogate: the network kernels against a CPU FP64 network, the surrogate wiring inside
the right-hand side, and the trained surrogate inside a flow (accuracy and gain)."""
import numpy as np
import pytest

from oracle import mlp as cpu_mlp


def _bf16(x):
    """Round float32 values to bfloat16 (nearest even) and back."""
    a = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def leading_form_factor(ff_R, n_s, A):
    """Form-factor content of the leading instability: the eigenspace of the projected vertex A_X(q*) (M x M,
    rows (R, pair)) of the eigenvalue of largest modulus (eigenvalues within 1% of it; with time reversal and
    C4v it is often degenerate, so single eigenvectors are not unique), its weight per bond
    w_R = (1/d) sum_{v in the space} sum_pair |v_(R,pair)|^2, and the bond shell (|R|^2 class: onsite, nearest,
    next-nearest, ...) holding the largest weight."""
    lam, vec = np.linalg.eigh(A)
    top = lam[np.argmax(np.abs(lam))]
    V = vec[:, np.abs(lam - top) <= 1e-2 * abs(top)]
    w = (np.abs(V) ** 2).sum(axis=1).reshape(len(ff_R), n_s * n_s).sum(axis=1) / V.shape[1]
    r2 = np.array([int(r[0]) ** 2 + int(r[1]) ** 2 for r in ff_R])
    shells = sorted(set(r2.tolist()))
    per_shell = np.array([w[r2 == s].sum() for s in shells])
    return shells[int(np.argmax(per_shell))], w


def test_leading_form_factor_of_a_planted_vertex():
    """The helper on vertices with a known leading eigenspace: a d pattern on the four nearest bonds, an onsite
    and a next-nearest one, each over a background of smaller eigenvalues, and a doubly degenerate leading pair
    (p_x, p_y on the nearest bonds) whose eigenspace weights do not depend on the basis inside it."""
    ff_R = np.array([(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (1, -1), (-1, 1), (-1, -1)])
    ns, M = 2, 9 * 4
    rng = np.random.default_rng(4)
    B = rng.normal(size=(M, M)) + 1j * rng.normal(size=(M, M))
    B = 0.05 * (B + B.conj().T) / np.sqrt(M)
    for pattern, shell in (((0, 1, -1, 1, -1, 0, 0, 0, 0), 1), ((1, 0, 0, 0, 0, 0, 0, 0, 0), 0),
                           ((0, 0, 0, 0, 0, 1, 1, 1, 1), 2)):
        v = np.kron(np.array(pattern, float), np.array([0, 1, -1, 0]) / np.sqrt(2))
        v /= np.linalg.norm(v)
        A = B - 3.0 * np.outer(v, v)                       # an attractive leading eigenvalue
        got, w = leading_form_factor(ff_R, ns, A)
        assert got == shell
        assert np.allclose(w, np.array(pattern, float) ** 2 / np.sum(np.array(pattern, float) ** 2), atol=0.02)
    px = np.kron(np.array((0, 1, -1, 0, 0, 0, 0, 0, 0), float), np.array([1, 0, 0, 0])) / np.sqrt(2)
    py = np.kron(np.array((0, 0, 0, 1, -1, 0, 0, 0, 0), float), np.array([0, 0, 0, 1])) / np.sqrt(2)
    for c, s in ((1.0, 0.0), (0.6, 0.8)):                  # two bases of the same degenerate pair
        a, b = c * px + s * py, -s * px + c * py
        got, w = leading_form_factor(ff_R, ns, B - 3.0 * (np.outer(a, a) + np.outer(b, b)))
        assert got == 1 and np.allclose(w, [0, 0.25, 0.25, 0.25, 0.25, 0, 0, 0, 0], atol=0.02)


def test_cpu_network_gradient_vs_finite_differences():
    """The FP64 reference network's backward pass against central differences (relative 1e-7)."""
    rng = np.random.default_rng(0)
    shapes = cpu_mlp.layer_shapes(5, 7, 3, 4)
    n = sum(a * b + b for a, b in shapes)
    p = rng.standard_normal(n) * 0.5
    X = rng.standard_normal((6, 5))
    T = rng.standard_normal((6, 4))
    _, g = cpu_mlp.loss_and_grad(p, shapes, X, T)
    h = 1e-6
    for i in rng.choice(n, 40, replace=False):
        e = np.zeros(n)
        e[i] = h
        fd = (cpu_mlp.loss_and_grad(p + e, shapes, X, T)[0] - cpu_mlp.loss_and_grad(p - e, shapes, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9


torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_08830_gb300 import build
    build.build()


@pytest.mark.gpu
def test_gpu_network_gradients_vs_cpu(gpu):
    """BF16 weights/activations with FP32 accumulation against the FP64 network at the same (BF16-rounded)
    weights and inputs.  Each of the depth + 1 layers rounds two operands to BF16 (its input activation
    on the way forward, its upstream gradient on the way back), each a relative perturbation of at most
    2^-8; the bound on every block's relative L2 error is their linear sum, 2 (depth + 1) 2^-8."""
    from paper_1710_08830_gb300.surrogate import Net
    net = Net(20, 256, 4, 1600, seed=5)
    rng = np.random.default_rng(1)
    p = _bf16(net.get_params())
    net.set_params(p)
    X = _bf16(rng.standard_normal((256, 20)).astype(np.float32))
    T = rng.standard_normal((256, 1600)).astype(np.float32)
    loss, g = net.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    g = g.cpu().numpy()
    shapes = cpu_mlp.layer_shapes(20, 256, 4, 1600)
    loss_ref, g_ref = cpu_mlp.loss_and_grad(p.astype(np.float64), shapes, X.astype(np.float64), T.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-2)
    bound = 2 * len(shapes) * 2.0 ** -8
    o = 0
    for din, dout in shapes:
        for size in (din * dout, dout):
            a, b = g[o:o + size], g_ref[o:o + size]
            o += size
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert rel < bound, (din, dout, size, rel)
    # inference keeps the activations in FP32: only FP32 rounding separates it from the FP64 network
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Y_ref, _ = cpu_mlp.forward(p.astype(np.float64), shapes, X.astype(np.float64))
    assert np.linalg.norm(Y - Y_ref) / np.linalg.norm(Y_ref) < 1e-5


@pytest.mark.gpu
def test_gpu_training_reduces_loss(gpu):
    """300 Adam steps on a smooth synthetic regression (tanh of a random projection of 20 inputs):
    the FP64 network with the same recipe reaches 3% of its initial loss, BF16 training must reach 10%."""
    from paper_1710_08830_gb300.surrogate import Net
    rng = np.random.default_rng(2)
    X = torch.from_numpy(rng.uniform(-1, 1, (4096, 20)).astype(np.float32)).cuda()
    W = torch.from_numpy(rng.standard_normal((20, 64)).astype(np.float32)).cuda()
    Y = torch.tanh(0.3 * (X @ W)).contiguous()
    net = Net(20, 128, 3, 64, seed=1)
    first = None
    for it in range(300):
        idx = torch.from_numpy(rng.integers(0, 4096, 512)).cuda()
        l = net.train_step(X[idx].contiguous(), Y[idx].contiguous(), 3e-3, want_loss=(it % 50 == 0 or it == 299))
        if first is None:
            first = l
    assert l < 0.1 * first


@pytest.mark.gpu
def test_surrogate_wiring_accept_and_reject(gpu):
    """With an infinite tolerance the right-hand side runs on the network's loops; with a zero one it
    falls back to the direct k-sum and equals the plain right-hand side exactly."""
    from paper_1710_08830_gb300 import inputs, surrogate
    from paper_1710_08830_gb300.api import PRODUCTS_SIMT, SPLIT32, Model
    data = surrogate.generate(2 * 36, seed=4, Lq=6, nc=4, n_ff=9, temps_per_model=2)
    tr = surrogate.train(data, epochs=3, batch=24)
    tp, alpha, mu = -0.1, 0.25, -0.8
    spec = inputs.rashba_hubbard(1.0, tp, alpha, 2.5, mu, Lq=6, nc=4, n_ff=9)
    st = inputs.random_state(spec, seed=3, scale=0.2)
    plain = Model(spec, SPLIT32, products=PRODUCTS_SIMT)
    d_plain = plain.rhs(0.3, st).cpu()
    m = Model(spec, SPLIT32, products=PRODUCTS_SIMT)
    surrogate.attach(m, tr, alpha, tp, mu, tol=1e-300)
    d_rej = m.rhs(0.3, st).cpu()
    assert torch.equal(d_rej, d_plain)
    assert surrogate.stats(m) == (0, 1, 0)
    m.rhs(0.3, st)                       # every call re-arms the surrogate: checked and rejected again
    assert surrogate.stats(m) == (0, 2, 0)
    # inside a flow the first failed check switches it off: the flow is the direct flow, bit for bit
    y_plain, r_plain = plain.flow(stop=5.0)
    y_sur, r_sur = m.flow(stop=5.0)
    assert torch.equal(y_plain, y_sur)
    assert (r_sur["n_steps"], r_sur["n_rhs"], r_sur["Tc"]) == (r_plain["n_steps"], r_plain["n_rhs"], r_plain["Tc"])
    assert surrogate.stats(m) == (0, 3, r_sur["n_rhs"] - 1)
    surrogate.attach(m, tr, alpha, tp, mu, tol=1e300)
    L_sur = m.loops(0.3).cpu().reshape(2, 36, -1, 16)
    X = torch.from_numpy(surrogate.features(6, 0.3, alpha, tp, mu)).cuda()
    y = tr.net.forward(X).cpu().double() * torch.from_numpy(tr.std).double() + torch.from_numpy(tr.mean).double()
    y = torch.view_as_complex(y.reshape(36, 2, -1, 16, 2).contiguous()).permute(1, 0, 2, 3) / 0.3
    # the library forms the features on the device; they agree with the host's to FP32 rounding
    assert float(torch.linalg.norm(L_sur - y) / torch.linalg.norm(y)) < 1e-5
    L_direct = plain.loops(0.3).cpu().reshape(2, 36, -1, 16)
    assert float(torch.linalg.norm(L_sur - L_direct) / torch.linalg.norm(L_direct)) > 1e-2
    assert surrogate.stats(m) == (1, 0, 0)
    surrogate.detach(m)
    assert torch.equal(m.rhs(0.3, st).cpu(), d_plain)


@pytest.mark.gpu
def test_surrogate_trained_on_the_family_inside_a_flow(gpu):
    """Train on 2e5 direct loops of the Rashba-Hubbard family (24x24 / 8x8, 9 bonds; t' in [-0.3, 0],
    alpha in [0, 0.4], mu in [-1.2, -0.6], log-uniform T in [0.02, 10]), measure the held-out error per
    temperature band, and run the flow of a family member with the surrogate against the direct flow.

    No family member at U = 2.5 reaches 50 t above T = 0.02, so the critical scale here is the
    crossing of max|V| = 3 t.  At the residual tolerance 1e-3 the first check fails (the network's
    error is at the percent level), the surrogate switches off and the flow is the direct flow exactly;
    the cost is the one network evaluation plus device-side early exits.  At tolerance 0.1 the network
    serves the high-temperature stretch; the figures (critical scale, evaluations, wall time) are
    printed, the critical scale must stay within 2% with the same leading channel, transfer momentum and form
    factor (the bond shell carrying most of the leading eigenvector of the projected vertex, per-bond weights
    within 0.05)."""
    from paper_1710_08830_gb300 import inputs, surrogate
    from paper_1710_08830_gb300.api import PRODUCTS_SIMT, SPLIT32, Model
    train = surrogate.generate(200_000, seed=1)
    held = surrogate.generate(30 * 576, seed=2, q_per_block=576, temps_per_model=3)
    tr = surrogate.train(train, epochs=40)
    err = surrogate.relative_errors(tr, held)
    Ts = np.array([d[3] for d in held.draws])
    print(f"\ntraining: {train.X.shape[0]} samples, {tr.seconds:.1f} s; held-out relative error, median {np.median(err):.3e}")
    for lo, hi in ((0.02, 0.1), (0.1, 1.0), (1.0, 10.01)):
        sel = (Ts >= lo) & (Ts < hi)
        print(f"  T in [{lo}, {hi}): {sel.sum()} blocks, median {np.median(err[sel]):.3e}, max {err[sel].max():.3e}")
    assert np.median(err[Ts >= 1.0]) < 0.1

    tp, alpha, mu, stop = -0.2, 0.3, -0.7, 3.0
    spec = inputs.rashba_hubbard(1.0, tp, alpha, 2.5, mu, Lq=24, nc=8, n_ff=9)
    direct = Model(spec, SPLIT32, products=PRODUCTS_SIMT)
    direct.flow(stop=stop)                      # warm-up (graph capture)
    y0, r0 = direct.flow(stop=stop)
    assert r0["crossed"]
    print(f"direct: Tc {r0['Tc']:.5f}, {r0['n_rhs']} evaluations, {r0['wall_s'] * 1e3:.1f} ms")

    def form_factor(model, y, r):
        A, _ = model.project(y, want_max=False)
        return leading_form_factor(spec.ff_R, spec.n_s, A[r["lead_channel"], r["lead_q"]].cpu().numpy())

    ff0, w0 = form_factor(direct, y0, r0)
    print(f"direct: leading form factor shell |R|^2 = {ff0}, bond weights {np.round(w0, 3).tolist()}")
    for tol in (1e-3, 1e-1):
        m = Model(spec, SPLIT32, products=PRODUCTS_SIMT)
        surrogate.attach(m, tr, alpha, tp, mu, tol=tol)
        m.flow(stop=stop)
        surrogate.attach(m, tr, alpha, tp, mu, tol=tol)   # fresh counters
        y1, r1 = m.flow(stop=stop)
        acc, rej, skip = surrogate.stats(m)
        print(f"surrogate, tolerance {tol:g}: Tc {r1['Tc']:.5f} ({r1['Tc'] / r0['Tc'] - 1:+.2%}), {r1['n_rhs']} evaluations, "
              f"{r1['wall_s'] * 1e3:.1f} ms (direct / surrogate wall time {r0['wall_s'] / r1['wall_s']:.3f}); "
              f"kept {acc}, rejected {rej}, skipped {skip}")
        assert r1["crossed"] and r1["lead_channel"] == r0["lead_channel"] and r1["lead_q"] == r0["lead_q"]
        assert abs(r1["Tc"] / r0["Tc"] - 1) < 0.02
        ff1, w1 = form_factor(m, y1, r1)
        assert ff1 == ff0 and np.abs(w1 - w0).max() < 0.05, (ff1, w1, w0)
        if tol == 1e-3:
            assert (acc, rej, skip) == (0, 1, r1["n_rhs"] - 1)
            assert torch.equal(y0, y1) and r1["Tc"] == r0["Tc"]
        else:
            assert acc > 0
        m.close()
    # the configuration as it is stated: residual tolerance 1e-3, the stop value 50, down to T_end = 0.02 (no member
    # of the family crosses: a time to T_end); what the network gains or loses in wall time against the direct flow
    direct.flow(stop=50.0)
    y50, r50 = direct.flow(stop=50.0)
    m = Model(spec, SPLIT32, products=PRODUCTS_SIMT)
    surrogate.attach(m, tr, alpha, tp, mu, tol=1e-3)
    m.flow(stop=50.0)
    surrogate.attach(m, tr, alpha, tp, mu, tol=1e-3)
    y51, r51 = m.flow(stop=50.0)
    acc, rej, skip = surrogate.stats(m)
    print(f"as stated (tolerance 1e-3, stop 50, T_end 0.02): direct {r50['wall_s'] * 1e3:.1f} ms, with the network "
          f"{r51['wall_s'] * 1e3:.1f} ms (gain {r50['wall_s'] / r51['wall_s'] - 1:+.1%}); kept {acc}, rejected {rej}, "
          f"skipped {skip}")
    assert torch.equal(y50, y51) and (acc, rej) == (0, 1)
    m.close()
