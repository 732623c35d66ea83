"""Reduced-basis derivative-informed neural operator (oracle, test infrastructure only).

Architecture (Sec. 3.3):  u_w(m, z) = Phi phi_w(m_r, z) + b,  m_r = Psi^T m.
  * Psi: the leading r_M Karhunen-Loeve modes of the prior (Sec. 3.3, KLE),
    ordered by decreasing prior variance (increasing lambda; ties broken by
    (k1 + k2, k1)).  The network input is the whitened coordinate
    xi_k = lambda_k <psi_k, m - mbar>_M, which returns the standard normal
    that synthesised a KL draw.
  * Phi: mass-weighted POD of training states (Sec. 3.3): eigenvectors of the
    snapshot covariance in the M inner product (M = h^2 I on the interior
    nodes), Phi^T M Phi = I, bias b = mean state ubar.
  * phi_w: dense net [xi; z] -> 400 -> 400 -> 400 -> r_U with exact-erf GELU
    on the hidden layers and a linear output layer.
Control Jacobian by forward-mode differentiation in z (Sec. 3.2: d_z u_w).
DINO loss in the reduced output space (Sec. 3.4):
  L = (1/B) sum_i ||phi_i - Phi^T M (u_i - ubar)||^2 + w_J ||d_z phi_i - Phi^T M d_z u_i||_F^2
(w_J = 1 for MR-DINO, 0 for MR-NO).  Reduced quadratic QoI (Sec. 3.3):
Q(u_w) = 1/2 ||phi + c||^2 + const with c = Phi^T M (ubar - u_t).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

from .field import dct2_basis, kl_eigenvalues


# ----------------------------------------------------------------------------- KL basis
def kl_mode_order(n, gamma, delta):
    """Flat mode indices q = k2 n + k1 sorted by (lambda, k1 + k2, k1)."""
    lam = kl_eigenvalues(n, gamma, delta).ravel()
    q = np.arange(n * n)
    k1, k2 = q % n, q // n
    return np.lexsort((k1, k1 + k2, lam))


def kl_projection_matrix(n, r_m, gamma=0.1, delta=1.0):
    """W[node, j] such that xi_hat = (m - mbar)_flat @ W: W = (lambda_q / n) v_k1(ix) v_k2(iy)
    for the r_m leading modes q (mass 1/n^2 per node, psi_q = n v_k1 v_k2)."""
    order = kl_mode_order(n, gamma, delta)[:r_m]
    lam = kl_eigenvalues(n, gamma, delta).ravel()
    V = dct2_basis(n)
    W = np.empty((n * n, r_m))
    for j, q in enumerate(order):
        k1, k2 = q % n, q // n
        W[:, j] = (lam[q] / n) * np.outer(V[k2], V[k1]).ravel()
    return W, order


def project_fields(m_flat, W, m_mean=0.0, bf16=False):
    """Whitened KL coordinates xi_hat = (m - mbar) @ W.  With bf16=True both factors
    are rounded to bfloat16 first (the tensor-core projection's operands); the sum
    stays float64."""
    a = np.asarray(m_flat, dtype=np.float64) - m_mean
    if bf16:
        a, W = round_bf16(a), round_bf16(W)
    return a @ W


# ----------------------------------------------------------------------------- POD
def pod(U_int, r_u, h):
    """Mass-weighted POD of snapshots U_int (Ns, d) with M = h^2 I.
    Returns (Phi (d, r_u), ubar (d,), eigenvalues of the snapshot operator (all))."""
    ubar = U_int.mean(axis=0)
    D = U_int - ubar
    C = (h * h) * (D @ D.T)
    ev, V = np.linalg.eigh(C)
    ev, V = ev[::-1], V[:, ::-1]
    Phi = D.T @ V[:, :r_u] / np.sqrt(ev[:r_u])
    idx = np.argmax(np.abs(Phi), axis=0)
    Phi *= np.sign(Phi[idx, np.arange(r_u)])
    return Phi, ubar, ev


# ----------------------------------------------------------------------------- activation
SQRT1_2 = 1.0 / np.sqrt(2.0)
INV_SQRT_2PI = 1.0 / np.sqrt(2.0 * np.pi)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x * SQRT1_2))


def gelu_d1(x):
    return 0.5 * (1.0 + erf(x * SQRT1_2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def gelu_d2(x):
    return INV_SQRT_2PI * np.exp(-0.5 * x * x) * (2.0 - x * x)


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------- network
class MLP:
    """Weights Ws[l] (out, in), biases bs[l]; layer 0 input is [xi (r_m); z (d_z)].
    out_scale s (r_u,): a fixed per-mode scaling of the output layer,
    phi = s * (W h + b), so that every reduced coordinate is learned at unit scale
    (s_r = RMS of mode r over the training states); None means s = 1."""

    def __init__(self, Ws, bs, r_m, out_scale=None):
        self.Ws = [np.array(W, dtype=np.float64) for W in Ws]
        self.bs = [np.array(b, dtype=np.float64) for b in bs]
        self.r_m = r_m
        self.s = None if out_scale is None else np.array(out_scale, dtype=np.float64)

    def copy(self):
        return MLP(self.Ws, self.bs, self.r_m, self.s)

    def forward(self, xi, z, jacobian=True, bf16=False):
        """xi (B, r_m), z (B, d_z) or (d_z,).  Returns dict with a_l, h_l, phi, and (if jacobian)
        the tangents Ad_l (B, width, d_z), Hd_l and J = d phi / d z (B, r_u, d_z).
        With bf16=True the GEMM operands (weights, layer inputs, tangents) are rounded to
        bfloat16 where the CUDA path rounds them; accumulation stays float64."""
        rnd = round_bf16 if bf16 else (lambda a: a)
        B = xi.shape[0]
        z = np.broadcast_to(z, (B, z.shape[-1]))
        h0 = np.concatenate([xi, z], axis=1)
        Ws = [rnd(W) for W in self.Ws]
        st = {"h": [h0], "a": [], "Ad": [], "Hd": []}
        h = h0
        Hd = None
        nl = len(Ws)
        for l in range(nl):
            a = rnd(h) @ Ws[l].T + self.bs[l]
            if jacobian:
                if l == 0:
                    Ad = np.broadcast_to(Ws[0][:, self.r_m:], (B,) + Ws[0][:, self.r_m:].shape)
                else:
                    Ad = np.matmul(Ws[l], rnd(Hd))            # (o, i) @ (b, i, j) -> (b, o, j)
            if l < nl - 1:
                st["a"].append(a)
                h = gelu(a)
                st["h"].append(h)
                if jacobian:
                    st["Ad"].append(Ad)
                    Hd = gelu_d1(a)[:, :, None] * Ad
                    st["Hd"].append(Hd)
            else:
                sc = 1.0 if self.s is None else self.s
                st["phi"] = sc * a
                if jacobian:
                    st["J"] = (sc if self.s is None else self.s[None, :, None]) * Ad
        return st

    def loss_and_grad(self, xi, z, y, Y, w_j=1.0):
        """DINO loss over a batch and its gradient with respect to every weight and bias."""
        B = xi.shape[0]
        st = self.forward(xi, z, jacobian=True)
        ephi = st["phi"] - y
        eJ = st["J"] - Y
        loss = (np.sum(ephi ** 2) + w_j * np.sum(eJ ** 2)) / B
        g_phi = 2.0 * ephi / B
        G_J = 2.0 * w_j * eJ / B
        if self.s is not None:          # back through the fixed output scaling
            g_phi = g_phi * self.s
            G_J = G_J * self.s[None, :, None]
        nl = len(self.Ws)
        dW = [None] * nl
        db = [None] * nl
        # output layer
        h_in, Hd_in = st["h"][nl - 1], st["Hd"][nl - 2]
        dW[nl - 1] = g_phi.T @ h_in + np.einsum("boj,bij->oi", G_J, Hd_in)
        db[nl - 1] = g_phi.sum(axis=0)
        gh = g_phi @ self.Ws[nl - 1]
        GHd = np.einsum("oi,boj->bij", self.Ws[nl - 1], G_J)
        for l in range(nl - 2, -1, -1):
            a, Ad = st["a"][l], st["Ad"][l]
            s1, s2 = gelu_d1(a), gelu_d2(a)
            ga = gh * s1 + s2 * np.einsum("bij,bij->bi", GHd, Ad)
            GAd = GHd * s1[:, :, None]
            dW[l] = ga.T @ st["h"][l]
            db[l] = ga.sum(axis=0)
            if l == 0:
                dW[0][:, self.r_m:] += GAd.sum(axis=0)
            else:
                dW[l] += np.einsum("boj,bij->oi", GAd, st["Hd"][l - 1])
                gh = ga @ self.Ws[l]
                GHd = np.einsum("oi,boj->bij", self.Ws[l], GAd)
        return loss, dW, db


class Adam:
    """Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8) on float64 copies of the parameters."""

    def __init__(self, params, b1=0.9, b2=0.999, eps=1e-8):
        self.m = [np.zeros_like(p) for p in params]
        self.v = [np.zeros_like(p) for p in params]
        self.t = 0
        self.b1, self.b2, self.eps = b1, b2, eps

    def step(self, params, grads, lr):
        self.t += 1
        c1 = 1.0 - self.b1 ** self.t
        c2 = 1.0 - self.b2 ** self.t
        out = []
        for i, (p, g) in enumerate(zip(params, grads)):
            self.m[i] = self.b1 * self.m[i] + (1.0 - self.b1) * g
            self.v[i] = self.b2 * self.v[i] + (1.0 - self.b2) * g * g
            out.append(p - lr * (self.m[i] / c1) / (np.sqrt(self.v[i] / c2) + self.eps))
        return out


def lr_schedule(epoch, epochs, lr0=1e-3, lr1=2.5e-4):
    """Sec. 4.2: the initial rate is lowered to a quarter of it at half of the epochs."""
    return lr0 if epoch < epochs // 2 else lr1


# ----------------------------------------------------------------------------- evaluation
def reduced_qoi_constant(Phi, ubar, ut_int, h):
    """c = Phi^T M (ubar - u_t) and the constant so that Q(u_w) = 1/2 ||phi + c||^2 + const."""
    dv = ubar - ut_int
    c = h * h * (Phi.T @ dv)
    const = 0.5 * (h * h * float(dv @ dv) - float(c @ c))
    return c, const


def decode_states(phi, Phi, ubar):
    """Decoded interior states u_w = Phi phi + ubar (Sec. 3.3) of coefficient rows phi (B, r_u)."""
    return phi @ Phi.T + ubar


def decoded_qoi(u_int, ut_int, h):
    """Q(u) = 1/2 h^2 sum over the interior nodes of (u - u_t)^2 (the tracking QoI of Sec. 4.2)."""
    diff = u_int - ut_int
    return 0.5 * h * h * np.sum(diff * diff, axis=-1)


def eval_surrogate(net: MLP, xi, z, Phi, ubar, ut_int, h, decode=True, bf16=False):
    """Per-sample Q_i and grad_z Q_i of the surrogate.  With decode=True the state
    u_w = Phi phi + ubar is formed and Q, dQ/du are taken on it (the chain rule of
    Sec. 3.2: grad_z Q = dQ/du(u_w) Phi d_z phi); else the reduced form is used."""
    st = net.forward(xi, z, jacobian=True, bf16=bf16)
    phi, J = st["phi"], st["J"]
    if decode:
        uw = decode_states(phi, Phi, ubar)
        Q = decoded_qoi(uw, ut_int, h)
        dq_red = h * h * ((uw - ut_int) @ Phi)         # (dQ/du) Phi
    else:
        c, const = reduced_qoi_constant(Phi, ubar, ut_int, h)
        Q = 0.5 * np.sum((phi + c) ** 2, axis=1) + const
        dq_red = phi + c
    grads = np.einsum("br,brj->bj", dq_red, J)
    return Q, grads, phi, J
