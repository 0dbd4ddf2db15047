"""Learned initial guess of the plane positioning.

The tensor-core forward and backward passes are checked against the plain
FP64 reference network in oracle/mlp_ref.py run on the same BF16-rounded
operands; the features against a host computation; the training targets
(from the FP64 GPU reconstruction) against the oracle's own reconstruction;
and the trained network against the method without it: fewer positioning
iterations, the same planes (fill residual within the 1e-13 stop, checked by
the oracle's clipper) and the same step.
"""
import numpy as np
import pytest

from paper_1305_3417_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1305_3417_gb300 import build
    build.build()
    return torch


def _params(seed):
    from oracle import mlp_ref as M
    rng = np.random.default_rng(seed)
    p = np.zeros(M.N_PARAM)
    o = 0
    for s in M.SHAPES:
        n = int(np.prod(s))
        p[o:o + n] = rng.normal(0.0, (2.0 / s[0]) ** 0.5 if len(s) == 2 else 0.1, n)
        o += n
    return p.astype(np.float32).astype(np.float64)


# FP32 accumulation of exact BF16 products (k-steps of 16 on the tensor cores,
# then the bias): within ACC * 2^-24 of the sum of the terms' magnitudes
ACC = 16.0


def _bf16_margin(z):
    """Distance of each value to the nearest BF16 rounding boundary (midway
    between consecutive BF16 numbers; both neighbouring exponent ranges)."""
    a = np.abs(np.asarray(z, np.float64))
    e = np.floor(np.log2(np.maximum(a, 1e-300)))
    out = np.full(a.shape, np.inf)
    for de in (-1, 0):
        ulp = 2.0 ** (e + de - 7)
        t = a / ulp
        out = np.minimum(out, np.abs(t - np.floor(t) - 0.5) * ulp)
    return np.where(a == 0, np.inf, out)


def _bf16_ulp(a):
    return 2.0 ** (np.floor(np.log2(np.maximum(np.abs(a), 1e-300))) - 7)


def _forward_bound(M, p, X):
    """An elementwise bound on |Y_gpu - Y_ref| for the tensor-core forward
    against the reference on the same BF16 operands, carried through the
    layers: a pre-activation accumulated in FP32 is within r = ACC 2^-24
    (sum of |terms| + |bias|) of the exact one (plus what the earlier layer's
    error brings); its BF16 rounding then agrees with the reference's unless
    a rounding boundary (or zero, for the ReLU) lies within that distance, in
    which case the activation may differ by one BF16 unit (or by up to 2r near
    zero).  Also returns which samples had no such undecided activation."""
    W1, b1, W2, b2, W3, b3 = M.unpack(p)
    q = M.bf16
    c = ACC * 2.0 ** -24
    X0 = q(X)
    A1 = np.abs(q(W1)); A2 = np.abs(q(W2)); A3 = np.abs(q(W3))
    Z1 = X0 @ q(W1) + b1
    r1 = c * (np.abs(X0) @ A1 + np.abs(b1))
    u1 = (Z1 > -r1) & (_bf16_margin(Z1) <= r1)
    e1 = np.where(u1, _bf16_ulp(np.abs(Z1) + r1) + 2 * r1, 0.0)
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ q(W2) + b2
    r2 = c * ((np.abs(H1) + e1) @ A2 + np.abs(b2)) + e1 @ A2
    u2 = (Z2 > -r2) & (_bf16_margin(Z2) <= r2)
    e2 = np.where(u2, _bf16_ulp(np.abs(Z2) + r2) + 2 * r2, 0.0)
    H2 = q(np.maximum(Z2, 0.0))
    yb = c * ((np.abs(H2) + e2) @ A3 + np.abs(b3)) + e2 @ A3
    return yb, ~(u1.any(1) | u2.any(1))


def test_mlp_forward_matches_reference(torch):
    """Where no BF16 rounding of a hidden activation is within the FP32
    accumulation bound of its boundary (most samples), the tensor-core
    forward equals the reference on the same BF16 operands up to the output
    layer's accumulation bound; elsewhere a hidden activation may round to the
    neighbouring BF16 number, and the output moves by about that one unit."""
    from oracle import mlp_ref as M
    from paper_1305_3417_gb300 import vof
    p = _params(3)
    rng = np.random.default_rng(4)
    X = rng.uniform(0.0, 1.2, (203, M.N_IN)).astype(np.float32)
    net = vof.Mlp(p, max_batch=256)
    Y = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    Yr, _ = M.forward(p, X.astype(np.float64))
    yb, ok = _forward_bound(M, p, X.astype(np.float64))
    d = np.abs(Y - Yr)
    print(f"forward: max |dY| {d.max():.2e} of max |Y| {np.abs(Yr).max():.2e}; on the {ok.sum()} of {ok.size} "
          f"samples with every rounding decided {d[ok].max():.2e} (bound {yb[ok].max():.2e})")
    assert np.all(d <= yb)
    assert d[ok].max() <= 1e-5 * np.abs(Yr).max()


def test_mlp_gradient_matches_reference(torch):
    """The gradient on a batch of samples whose forward roundings are all
    decided (see the forward test): against the reference backward on the same BF16
    operands within 1e-3 of its norm (the backward's own BF16 roundings of the
    upstream gradients can still flip); loss to 1e-5."""
    from oracle import mlp_ref as M
    from paper_1305_3417_gb300 import vof
    p = _params(5)
    rng = np.random.default_rng(6)
    X = rng.uniform(0.0, 1.2, (3000, M.N_IN)).astype(np.float32)
    T = rng.normal(0.0, 1.0, (3000, M.N_OUT)).astype(np.float32)
    _, ok = _forward_bound(M, p, X.astype(np.float64))
    X, T = X[ok][:700], T[ok][:700]
    assert X.shape[0] >= 300
    net = vof.Mlp(p, max_batch=1024)
    loss, g = net.gradient(torch.from_numpy(X).cuda(), torch.from_numpy(T).cuda())
    lr, gr = M.backward(p, X.astype(np.float64), T.astype(np.float64))
    g = g.cpu().numpy()
    rel = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    print(f"gradient: |dg| / |g| = {rel:.2e}, loss {loss:.7f} vs {lr:.7f}")
    assert abs(loss - lr) <= 1e-5 * abs(lr)
    assert rel < 1e-3
    big = np.abs(gr) > 0.1 * np.abs(gr).max()
    assert np.all(np.abs(g[big] - gr[big]) <= 5e-3 * np.abs(gr[big]))


def test_mlp_adam_steps(torch):
    """Two training steps against Adam written out in numpy (beta1 0.9, beta2
    0.999, eps 1e-8, bias-corrected moments) from the device's own gradients
    at the same parameters: the update arithmetic, not the gradient, is under
    test here."""
    from oracle import mlp_ref as M
    from paper_1305_3417_gb300 import vof
    p0 = _params(7)
    rng = np.random.default_rng(8)
    X = torch.from_numpy(rng.uniform(0.0, 1.2, (512, M.N_IN)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.normal(0.0, 1.0, (512, M.N_OUT)).astype(np.float32)).cuda()
    net = vof.Mlp(p0, max_batch=1024)
    lr = 1e-3
    m = np.zeros(M.N_PARAM)
    v = np.zeros(M.N_PARAM)
    p = net.params().astype(np.float64)
    for t in (1, 2):
        _, g = net.gradient(X, T)
        g = g.cpu().numpy().astype(np.float64)
        net.train_step(X, T, lr)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        want = p - lr * (m / (1 - 0.9 ** t)) / (np.sqrt(v / (1 - 0.999 ** t)) + 1e-8)
        got = net.params().astype(np.float64)
        err = np.abs(got - want)
        print(f"Adam step {t}: max |p - p_numpy| = {err.max():.2e} (lr {lr})")
        assert np.all(err <= 2e-3 * lr + 2e-7 * np.abs(want))
        p = got
    net.close()


def test_mlp_features(torch):
    from paper_1305_3417_gb300 import vof
    m = I.hex_mesh((6, 5, 4), jitter=0.15, seed=8)
    a = np.random.default_rng(9).uniform(0, 1, m.n_cells)
    ctx = vof.VofContext(m, precision=1)
    f = torch.empty((m.n_cells, vof.MLP_IN), dtype=torch.float32, device="cuda")
    vof.vof_mlp_features(ctx.h, torch.from_numpy(a).cuda(), None, m.n_cells, f)
    f = f.cpu().numpy()
    nx, ny, nz = m.shape
    for c in [0, 7, 33, m.n_cells - 1, 61]:
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        want = np.full(27, a[c])
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    ii, jj, kk = i + dx, j + dy, k + dz
                    if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                        want[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] = a[ii + nx * (jj + ny * kk)]
        np.testing.assert_allclose(f[c, :27], want.astype(np.float32), rtol=0, atol=0)
        assert f[c, 31] == pytest.approx(6 / 24) and f[c, 32] == pytest.approx(1.0)


def test_mlp_training_gain(torch, oracle_lib):
    from paper_1305_3417_gb300 import mlp, vof
    m = I.hex_mesh((24, 24, 24), jitter=0.2, seed=11)
    c64 = vof.VofContext(m, precision=0)
    train_f = mlp.random_fields(m, 24, seed=12)
    test_f = mlp.random_fields(m, 4, seed=13)
    X, Y = mlp.samples(c64, m, train_f)
    # targets: the FP64 GPU reconstruction is the oracle's
    om = oracle_lib.OracleMesh(m)
    on, od, ofl, _, _ = om.reconstruct(train_f[0])
    cells = np.flatnonzero(ofl & oracle_lib.ORIENTED)[:200]
    Xc, Yc = mlp.samples(c64, m, train_f[:1])
    pts = m.points[m.cell_verts[cells]]
    proj = np.einsum("ckd,dc->ck", pts, on[:, cells])
    s = (od[cells] - proj.min(1)) / (proj.max(1) - proj.min(1))
    allc = np.flatnonzero(ofl & oracle_lib.ORIENTED)
    pos = np.searchsorted(allc, cells)
    Yc = Yc.cpu().numpy()
    assert np.abs(Yc[pos, :3] - on[:, cells].T).max() < 1e-6      # FP32 targets
    assert np.abs(Yc[pos, 3] - s).max() < 1e-6
    # training lowers the loss
    net = vof.Mlp(mlp.init_params(1306), max_batch=1 << 15)
    hist = mlp.train(net, X, Y, epochs=25, batch=2048, lr=3e-3)
    print("training loss", hist[0], "->", hist[-1])
    assert hist[-1] < 0.2 * hist[0]
    # the guess saves iterations; the planes and the step are the method's
    c32 = vof.VofContext(m, precision=1)
    tot0 = tot1 = 0
    for a in test_f:
        ta = torch.from_numpy(a).cuda()
        n0_, d0, fl0, it0 = (t.cpu().numpy() for t in c32.reconstruct(ta))
        vof.vof_set_guess(c32.h, net)
        n1, d1, fl1, it1 = (t.cpu().numpy() for t in c32.reconstruct(ta))
        vof.vof_set_guess(c32.h, None)
        assert np.array_equal(fl0, fl1) and np.array_equal(n0_, n1)
        ori = np.flatnonzero(fl1 & 2)
        tot0 += int(it0[ori].sum())
        tot1 += int(it1[ori].sum())
        nn = n1.reshape(3, -1)
        _, vc, _, _ = om.geometry()
        for c in ori[:: max(1, ori.size // 60)]:
            g = om.cut_volume(c, nn[:, c], d1[c]) / vc[c] - a[c]
            assert abs(g) <= 3e-13, (c, g)
    print(f"positioning iterations without / with the network: {tot0} / {tot1}")
    assert tot1 < tot0


def test_guess_batch_smaller_than_interface(torch):
    """A network whose batch is smaller than the interface list guesses the
    first cells only; every plane is still the method's (same flags and
    normals, offsets within the positioning stop), and detaching restores the
    plain start exactly."""
    from paper_1305_3417_gb300 import mlp, vof
    m = I.hex_mesh((20, 20, 20), jitter=0.2, seed=31)
    a = mlp.random_fields(m, 1, seed=32)[0]
    ctx = vof.VofContext(m, precision=1)
    ta = torch.from_numpy(a).cuda()
    n0, d0, f0, i0 = (t.cpu().numpy() for t in ctx.reconstruct(ta))
    assert int((f0 & 2).sum()) > 64
    net = vof.Mlp(mlp.init_params(7), max_batch=64)
    vof.vof_set_guess(ctx.h, net)
    n1, d1, f1, i1 = (t.cpu().numpy() for t in ctx.reconstruct(ta))
    vof.vof_set_guess(ctx.h, None)
    n2, d2, f2, i2 = (t.cpu().numpy() for t in ctx.reconstruct(ta))
    assert np.array_equal(f0, f1) and np.array_equal(n0, n1)
    assert np.abs(d1 - d0).max() < 1e-11 * m.h
    assert np.array_equal(d2, d0) and np.array_equal(i2, i0)
