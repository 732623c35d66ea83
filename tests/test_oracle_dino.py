"""Pins of the oracle's reduced-basis neural operator (Sec. 3.3-3.4), CPU only.

* KL projection returns exactly the whitened normals of a synthesised field (also with
  a nonzero mean field); its BF16 form rounds the centred field and the basis, each to
  the nearest bfloat16 (hand-computed values of the format), and sums in FP64.
* POD: M-orthonormal basis, reconstruction error = tail eigenvalue sum,
  rank-one data gives one mode.
* MLP: forward-mode control Jacobian against finite differences in z; the
  analytic DINO-loss gradient against finite differences in the weights;
  GELU derivatives against finite differences.
* Reduced loss (Sec. 3.4): full-space loss minus reduced loss does not depend
  on the network.
* Reduced quadratic QoI (Sec. 3.3): decoded Q equals 1/2 ||phi + c||^2 + const.
* Jacobian data (Sec. 3.4, implicit function theorem): Phi^T M J^-1 G against
  finite differences of the projected state.
* Hand-computed forward pass and forward-mode Jacobian of a 2 -> 3 -> 3 -> 3 -> 2 net whose
  pre-activations sit where GELU has a closed form (erf(1), erf(2) written out).
* Adam against hand-unrolled first and second steps (bias corrections at t = 2).
"""
import numpy as np
import pytest

from oracle import dino, field, pde, philox
from synthetic_inputs import controls, glorot_uniform_mlp


def test_kl_projection_returns_normals():
    n, r_m = 12, 30
    xi = philox.field_normals(9, 0, 3, n * n)
    m = field.synthesize(xi.reshape(3, n, n), n, 0.1, 1.0, 0.0)
    W, order = dino.kl_projection_matrix(n, r_m)
    got = m.reshape(3, -1) @ W
    np.testing.assert_allclose(got, xi[:, order[:r_m]], atol=1e-12)
    lam = field.kl_eigenvalues(n, 0.1, 1.0).ravel()[order]
    assert np.all(np.diff(lam) >= 0)
    assert order[0] == 0 and set(order[1:3]) == {1, n}
    m1 = field.synthesize(xi.reshape(3, n, n), n, 0.1, 1.0, -1.5)
    np.testing.assert_allclose(dino.project_fields(m1.reshape(3, -1), W, m_mean=-1.5), xi[:, order[:r_m]],
                               atol=1e-12)


def test_kl_projection_bf16_operands():
    # 1 + 2^-8 + 2^-12 lies above the midpoint of the bfloat16 neighbours 1 and 1 + 2^-7
    x = 1.0 + 2.0 ** -8 + 2.0 ** -12
    up = 1.0 + 2.0 ** -7
    m = np.array([[3.0 + x, 3.0 + 2.0, 3.0 - 0.5]])
    W = np.array([[x], [0.25], [-3.0]])
    got = dino.project_fields(m, W, m_mean=3.0, bf16=True)
    assert got[0, 0] == up * up + 2.0 * 0.25 + (-0.5) * (-3.0)
    exact = dino.project_fields(m, W, m_mean=3.0)
    np.testing.assert_allclose(exact[0, 0], x * x + 0.5 + 1.5, rtol=1e-15)
    # operands already in bfloat16: the sum is exact
    rng = np.random.default_rng(5)
    a = rng.integers(-64, 64, (4, 50)) * 2.0 ** -6
    B = rng.integers(-64, 64, (50, 3)) * 2.0 ** -4
    assert np.array_equal(dino.project_fields(a, B, bf16=True), a @ B)


def test_pod_properties():
    rng = np.random.default_rng(0)
    d, Ns, h = 50, 30, 0.1
    U = rng.standard_normal((Ns, 6)) @ rng.standard_normal((6, d)) + 0.01 * rng.standard_normal((Ns, d))
    Phi, ubar, ev = dino.pod(U, 5, h)
    np.testing.assert_allclose(h * h * Phi.T @ Phi, np.eye(5), atol=1e-10)
    D = U - ubar
    R = D - (h * h * (D @ Phi)) @ Phi.T
    np.testing.assert_allclose(h * h * np.sum(R * R), np.sum(ev[5:]), rtol=1e-8)
    v = rng.standard_normal(d)
    U1 = np.outer(rng.standard_normal(Ns), v) + 3.0
    Phi1, ubar1, ev1 = dino.pod(U1, 1, h)
    assert ev1[1] < 1e-10 * ev1[0]
    np.testing.assert_allclose(np.abs(Phi1[:, 0]), np.abs(v) / (h * np.linalg.norm(v)), rtol=1e-10)
    assert Phi1[np.argmax(np.abs(Phi1[:, 0])), 0] > 0


def test_gelu_derivatives():
    x = np.linspace(-4, 4, 17)
    d = 1e-6
    np.testing.assert_allclose((dino.gelu(x + d) - dino.gelu(x - d)) / (2 * d), dino.gelu_d1(x), atol=1e-9)
    np.testing.assert_allclose((dino.gelu_d1(x + d) - dino.gelu_d1(x - d)) / (2 * d), dino.gelu_d2(x), atol=1e-9)
    np.testing.assert_allclose(dino.gelu(np.array([0.0, 1.0])), [0.0, 0.8413447460685429], rtol=1e-14)


def _small_net(r_m=3, d_z=2, widths=(5, 6, 4), r_u=3, seed=1, scaled=True):
    Ws, bs = glorot_uniform_mlp([r_m + d_z, *widths, r_u], seed=seed)
    rng = np.random.default_rng(seed)
    bs = [0.1 * rng.standard_normal(b.shape) for b in bs]
    s = rng.uniform(0.2, 2.0, r_u) if scaled else None
    return dino.MLP(Ws, bs, r_m, out_scale=s)


@pytest.mark.parametrize("scaled", [True, False])
def test_forward_jacobian_finite_difference(scaled):
    net = _small_net(scaled=scaled)
    rng = np.random.default_rng(3)
    xi, z = rng.standard_normal((4, 3)), rng.uniform(-1, 1, (4, 2))
    J = net.forward(xi, z)["J"]
    step = 1e-6
    for j in range(2):
        e = np.zeros(2)
        e[j] = step
        fd = (net.forward(xi, z + e, jacobian=False)["phi"] - net.forward(xi, z - e, jacobian=False)["phi"]) / (2 * step)
        np.testing.assert_allclose(J[:, :, j], fd, rtol=1e-7, atol=1e-9)


@pytest.mark.parametrize("w_j,scaled", [(1.0, True), (0.0, True), (1.0, False)])
def test_loss_gradient_finite_difference(w_j, scaled):
    net = _small_net(scaled=scaled)
    rng = np.random.default_rng(5)
    B = 4
    xi, z = rng.standard_normal((B, 3)), rng.uniform(-1, 1, (B, 2))
    y, Y = rng.standard_normal((B, 3)), rng.standard_normal((B, 3, 2))
    loss, dW, db = net.loss_and_grad(xi, z, y, Y, w_j=w_j)
    step = 1e-6
    for l in range(len(net.Ws)):
        for (i, j) in [(0, 0), (1, net.Ws[l].shape[1] - 1), (net.Ws[l].shape[0] - 1, 1)]:
            a, b = net.copy(), net.copy()
            a.Ws[l][i, j] += step
            b.Ws[l][i, j] -= step
            fd = (a.loss_and_grad(xi, z, y, Y, w_j)[0] - b.loss_and_grad(xi, z, y, Y, w_j)[0]) / (2 * step)
            np.testing.assert_allclose(dW[l][i, j], fd, rtol=1e-7, atol=1e-9)
        a, b = net.copy(), net.copy()
        a.bs[l][0] += step
        b.bs[l][0] -= step
        fd = (a.loss_and_grad(xi, z, y, Y, w_j)[0] - b.loss_and_grad(xi, z, y, Y, w_j)[0]) / (2 * step)
        np.testing.assert_allclose(db[l][0], fd, rtol=1e-7, atol=1e-9)


def test_reduced_loss_equivalence_and_reduced_qoi():
    rng = np.random.default_rng(8)
    d, Ns, r_u, h, d_z = 40, 25, 3, 0.2, 2
    U = rng.standard_normal((Ns, 5)) @ rng.standard_normal((5, d))
    Phi, ubar, _ = dino.pod(U, r_u, h)
    B = 3
    u = U[:B]
    du = rng.standard_normal((B, d, d_z))
    xi = rng.standard_normal((B, 3))
    z = rng.uniform(-1, 1, (B, d_z))
    y = h * h * (u - ubar) @ Phi
    Y = h * h * np.einsum("dr,bdj->brj", Phi, du)
    gaps = []
    for seed in (1, 2):
        net = _small_net(r_u=r_u, seed=seed)
        st = net.forward(xi, z)
        uw = st["phi"] @ Phi.T + ubar
        duw = np.einsum("dr,brj->bdj", Phi, st["J"])
        full = (h * h * np.sum((uw - u) ** 2) + h * h * np.sum((duw - du) ** 2)) / B
        red = net.loss_and_grad(xi, z, y, Y)[0]
        gaps.append(full - red)
    np.testing.assert_allclose(gaps[0], gaps[1], rtol=1e-10)
    # reduced QoI equals the decoded one
    ut = rng.standard_normal(d)
    net = _small_net(r_u=r_u, seed=4)
    Q1, g1, _, _ = dino.eval_surrogate(net, xi, z, Phi, ubar, ut, h, decode=True)
    Q2, g2, _, _ = dino.eval_surrogate(net, xi, z, Phi, ubar, ut, h, decode=False)
    np.testing.assert_allclose(Q1, Q2, rtol=1e-10)
    np.testing.assert_allclose(g1, g2, rtol=1e-10)
    # and the surrogate gradient is the z-derivative of its Q
    step = 1e-6
    for j in range(d_z):
        e = np.zeros(d_z)
        e[j] = step
        qp = dino.eval_surrogate(net, xi, z + e, Phi, ubar, ut, h)[0]
        qm = dino.eval_surrogate(net, xi, z - e, Phi, ubar, ut, h)[0]
        np.testing.assert_allclose(g1[:, j], (qp - qm) / (2 * step), rtol=1e-6, atol=1e-10)


def test_jacobian_data_finite_difference():
    n = 17
    prob = pde.Problem(n=n, L=3)
    G = field.control_sources(n, prob.L, prob.width)
    m = field.sample_fields(3, 0, 1, n)[0]
    z = controls(4, 1, prob.d_z)[0]
    kx, ky = pde.face_coefficients(m)
    f = (G @ z).reshape(n, n)
    u, chol = pde.newton_solve(kx, ky, f, prob.r, prob.h)
    dudz = pde.state_jacobian_columns(chol, pde.interior_rows(G, n), n)
    step = 1e-5
    for k in (0, 4, 8):
        zp, zm = z.copy(), z.copy()
        zp[k] += step
        zm[k] -= step
        up = pde.newton_solve(kx, ky, (G @ zp).reshape(n, n), prob.r, prob.h)[0]
        um = pde.newton_solve(kx, ky, (G @ zm).reshape(n, n), prob.r, prob.h)[0]
        fd = ((up - um) / (2 * step))[1:-1, 1:-1].ravel()
        np.testing.assert_allclose(dudz[:, k], fd, rtol=1e-6, atol=1e-9 * np.abs(fd).max())


def test_adam_first_step():
    p = [np.array([1.0, -2.0])]
    g = [np.array([0.5, -0.1])]
    opt = dino.Adam(p)
    out = opt.step(p, g, 1e-3)
    # first step: m_hat = g, v_hat = g^2 -> p - lr * g / (|g| + eps)
    np.testing.assert_allclose(out[0], p[0] - 1e-3 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-14)
    assert dino.lr_schedule(99, 200) == 1e-3 and dino.lr_schedule(100, 200) == 2.5e-4


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159])
    r = dino.round_bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7
    assert abs(r[3] + 3.14159) < 2 ** -7 * 4


def test_output_scale_is_a_reparametrisation():
    """phi = s * (W h + b) equals the unscaled net whose last layer is diag(s) W, diag(s) b."""
    net = _small_net(scaled=True)
    plain = net.copy()
    plain.s = None
    plain.Ws[-1] = net.s[:, None] * net.Ws[-1]
    plain.bs[-1] = net.s * net.bs[-1]
    rng = np.random.default_rng(9)
    xi, z = rng.standard_normal((4, 3)), rng.uniform(-1, 1, (4, 2))
    a, b = net.forward(xi, z), plain.forward(xi, z)
    np.testing.assert_allclose(a["phi"], b["phi"], rtol=1e-13)
    np.testing.assert_allclose(a["J"], b["J"], rtol=1e-13)


# erf(1) and erf(2) to 31 digits (Abramowitz & Stegun, Table 7.1)
ERF1 = 0.8427007929497148693412206350826
ERF2 = 0.9953222650189527341620692563672
SQ2 = 1.4142135623730950488016887242097
INV_SQRT_2PI = 0.3989422804014326779399460599344


def _hand_net():
    """A 2 -> 3 -> 3 -> 3 -> 2 net (r_m = 1, d_z = 1) whose weights and biases put every
    hidden pre-activation at 12, -12, 0, sqrt 2, -sqrt 2 or 2 sqrt 2 for the input
    [xi, z] = [1, 2], where GELU(x) = x (1 + erf(x / sqrt 2)) / 2 is known in closed form:
    GELU(12) = 12 and GELU(-12) = 0 to double precision, GELU(0) = 0,
    GELU(+-sqrt 2) = +-(sqrt 2 / 2)(1 +- erf 1), GELU(2 sqrt 2) = sqrt 2 (1 + erf 2)."""
    g1 = SQ2 / 2 * (1 + ERF1)                      # GELU(sqrt 2)
    W0 = [[3.0, 1.5], [-1.0, -5.5], [1.0, 0.0]]
    b0 = [6.0, 0.0, SQ2 - 1.0]                     # a0 = [12, -12, sqrt 2]
    W1 = [[1.0, 5.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.0, SQ2 / g1]]
    b1 = [-12.0, 6.0, 0.0]                         # a1 = [0, 12, sqrt 2]
    W2 = [[7.0, 1.0, 0.0], [0.0, 0.0, -SQ2 / g1], [3.0, -1.0, 0.0]]
    b2 = [2 * SQ2 - 12.0, 0.0, 12.0]               # a2 = [2 sqrt 2, -sqrt 2, 0]
    W3 = [[1.0, 2.0, 5.0], [-1.0, 0.0, 3.0]]
    b3 = [0.25, -0.5]
    s = [2.0, 0.5]
    return dino.MLP([W0, W1, W2, W3], [b0, b1, b2, b3], 1, out_scale=s)


def test_forward_hand_computed():
    """Sec. 3.3: phi = s * (W3 GELU(W2 GELU(W1 GELU(W0 [xi; z] + b0) + b1) + b2) + b3), linear
    output layer, KL coordinates before the controls.  A dropped hidden bias, a GELU on the
    output layer, the inputs in the order [z; xi], or a missing output scale each change phi."""
    net = _hand_net()
    st = net.forward(np.array([[1.0]]), np.array([2.0]))
    g3 = SQ2 * (1 + ERF2)                          # GELU(2 sqrt 2)
    g2 = -SQ2 / 2 * (1 - ERF1)                     # GELU(-sqrt 2)
    # h3 = [g3, g2, 0]
    want = [2.0 * (g3 + 2.0 * g2 + 0.25), 0.5 * (-g3 - 0.5)]
    np.testing.assert_allclose(st["phi"][0], want, rtol=1e-14)
    np.testing.assert_allclose(st["a"][0][0], [12.0, -12.0, SQ2], rtol=1e-15)
    np.testing.assert_allclose(st["a"][1][0], [0.0, 12.0, SQ2], atol=1e-14)
    np.testing.assert_allclose(st["a"][2][0], [2 * SQ2, -SQ2, 0.0], atol=1e-14)


def test_forward_tangent_hand_computed():
    """Sec. 3.2: the forward-mode control Jacobian d phi / d z through the same net.
    GELU'(x) = Phi(x) + x phi(x): 1 at 12, 0 at -12, 1/2 at 0, and
    (1 + erf 2)/2 + 2 sqrt 2 e^-4 / sqrt(2 pi) at 2 sqrt 2.  With d a0/dz = W0[:, 1] = [1.5, -5.5, 0]:
    d h1 = [1.5, 0, 0], d a1 = [1.5, 0.75, 0], d h2 = [0.75, 0.75, 0], d a2 = [6, 0, 1.5],
    d h3 = [6 GELU'(2 sqrt 2), 0, 0.75], J = s * (W3 d h3)."""
    net = _hand_net()
    J = net.forward(np.array([[1.0]]), np.array([2.0]))["J"][0, :, 0]
    gp = (1 + ERF2) / 2 + 2 * SQ2 * np.exp(-4.0) * INV_SQRT_2PI
    want = [2.0 * (6 * gp + 5 * 0.75), 0.5 * (-6 * gp + 3 * 0.75)]
    np.testing.assert_allclose(J, want, rtol=1e-13)


def test_adam_second_step():
    """Adam's bias corrections at t = 2: m2 = 0.9 (0.1 g1) + 0.1 g2, v2 = 0.999 (0.001 g1^2) + 0.001 g2^2,
    divided by 1 - 0.9^2 = 0.19 and 1 - 0.999^2 = 0.001999.  With g1 = 3, g2 = -1:
    m_hat = 0.17 / 0.19 = 17/19 and v_hat = 0.009991 / 0.001999 = 9991/1999."""
    lr = 1e-3
    p0 = [np.array([0.5])]
    opt = dino.Adam(p0)
    p1 = opt.step(p0, [np.array([3.0])], lr)
    np.testing.assert_allclose(p1[0], [0.5 - lr * 3.0 / (3.0 + 1e-8)], rtol=1e-15)
    p2 = opt.step(p1, [np.array([-1.0])], lr)
    want = p1[0][0] - lr * (17.0 / 19.0) / (np.sqrt(9991.0 / 1999.0) + 1e-8)
    np.testing.assert_allclose(p2[0], [want], rtol=1e-14)
    assert opt.t == 2


def test_decode_reconstructs_states_in_the_basis_span():
    """Sec. 3.3: for u = ubar + Phi a (a state the POD basis represents exactly), the reduced
    coordinates Phi^T M (u - ubar) are a (M-orthonormal Phi), and decoding them returns u; the
    decoded QoI is 1/2 h^2 ||u - u_t||^2 written out over the interior nodes."""
    rng = np.random.default_rng(12)
    d, r_u, h = 30, 4, 0.25
    Phi = np.linalg.qr(rng.standard_normal((d, r_u)))[0] / h        # h^2 Phi^T Phi = I
    ubar = rng.standard_normal(d)
    a = rng.standard_normal((3, r_u))
    u = ubar + a @ Phi.T
    y = h * h * (u - ubar) @ Phi
    np.testing.assert_allclose(y, a, atol=1e-12)
    np.testing.assert_allclose(dino.decode_states(y, Phi, ubar), u, atol=1e-12)
    ut = rng.standard_normal(d)
    q = dino.decoded_qoi(u, ut, h)
    for i in range(3):
        assert q[i] == pytest.approx(0.5 * h * h * sum((u[i, k] - ut[k]) ** 2 for k in range(d)), rel=1e-14)


def test_projected_jacobian_routes_agree():
    """Sec. 3.4: Phi^T M J^-1 G by d_z forward solves equals (J^-1 M Phi)^T G by r_u adjoint
    solves (J symmetric), and both equal the projection of finite differences of the state."""
    n = 13
    prob = pde.Problem(n=n, L=2)
    G = field.control_sources(n, prob.L, prob.width)
    m = field.sample_fields(3, 5, 1, n)[0]
    z = controls(4, 1, prob.d_z)[0]
    kx, ky = pde.face_coefficients(m)
    u, chol = pde.newton_solve(kx, ky, (G @ z).reshape(n, n), prob.r, prob.h)
    G_int = pde.interior_rows(G, n)
    rng = np.random.default_rng(2)
    Phi = rng.standard_normal(((n - 2) ** 2, 6))
    Yf = pde.projected_jacobian(chol, G_int, Phi, prob.h, "forward")
    Ya = pde.projected_jacobian(chol, G_int, Phi, prob.h, "adjoint")
    np.testing.assert_allclose(Ya, Yf, rtol=1e-11, atol=1e-13 * np.abs(Yf).max())
    step = 1e-5
    for k in range(prob.d_z):
        e = np.zeros(prob.d_z)
        e[k] = step
        up = pde.newton_solve(kx, ky, (G @ (z + e)).reshape(n, n), prob.r, prob.h)[0]
        um = pde.newton_solve(kx, ky, (G @ (z - e)).reshape(n, n), prob.r, prob.h)[0]
        fd = ((up - um) / (2 * step))[1:-1, 1:-1].ravel()
        np.testing.assert_allclose(Yf[:, k], prob.h ** 2 * Phi.T @ fd, rtol=1e-6, atol=1e-10)
