"""Neural pair term of the Jastrow factor: the oracle's network, its radial
derivatives, the node table that the lattice projection interpolates, and
the variance-minimisation objective with its gradient.

TEST INFRASTRUCTURE ONLY: imported by the tests and by the smoke check. The
product package never imports it, and it imports nothing from the product.

All arithmetic is float64 on the CPU in plain PyTorch ops; the gradient of
the objective is taken by torch.autograd (a library primitive), which makes
it independent of the product's hand-written backward kernel.

The term (a radial pair network; the paper itself uses a fixed JAGP guiding
function, so this is the extension the workload adds on top of it):
  features    f_k(r) = r^2 / (r^2 + ell_k^2), plus a one-hot channel code
  network     h1 = silu(W1 z + b1), h2 = silu(W2 h1 + b2), m = w3 . h2 + b3
  cut-off     g_c(r) = m(r, c) s(r / r_cut_c),
              s(t) = 1 - 10 t^3 + 15 t^4 - 6 t^5 for t < 1, 0 beyond,
so g'(0) = 0 (every feature is flat at r = 0 and s'(0) = 0: the Pade cusp
conditions are untouched) and g, g', g'' vanish at r_cut. With ``bf16``
the weights enter as their bfloat16 roundings (to nearest, ties to even).

Local energy with the term (continuous E_L of psi_G = D exp(J_P + J_NN)):
  E_L = E_base - 1/2 sum_i [2 a_i . G_i + |G_i|^2 + L_i],
with a_i = grad_i log|D exp(J_P)| and E_base the local energy without the
term, G_i = grad_i J_NN and L_i = lap_i J_NN from the pair derivatives
(grad_i g(r_ij) = g'(r) (r_i - r_j)/r, lap_i g(r_ij) = g'' + 2 g'/r).

Objective: the variance of E_L over a fixed sample of configurations,
each reweighted by |psi(theta)/psi_0|^2 = exp(2 J_NN) (the sample was drawn
without the term):  L = sum_x w_x (E_x - Ebar)^2 / sum_x w_x.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

DT = torch.float64


def bf16_round(t: torch.Tensor) -> torch.Tensor:
    """float32 value of t rounded to bfloat16, nearest with ties to even (bit
    arithmetic on the float32 pattern: add 0x7FFF plus the lowest kept bit,
    then clear the 16 low bits); returned as float64."""
    f = t.detach().to(torch.float32).contiguous()
    u = f.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
    keep = (u >> 16) & 1
    u = (((u + 0x7FFF + keep) >> 16) << 16) & 0xFFFFFFFF
    u = torch.where(u >= 2 ** 31, u - 2 ** 32, u).to(torch.int32)
    return u.view(torch.float32).to(DT)


def unpack(theta: torch.Tensor, spec):
    H, D = spec.hidden, spec.n_in
    o = 0
    W1 = theta[o:o + H * D].view(H, D); o += H * D
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].view(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o:o + 1]
    return W1, b1, W2, b2, w3, b3


def used_weights(theta, bf16: bool):
    """The weights the network computes with; with bf16 their values are the
    bfloat16 roundings and the gradient passes straight through to theta."""
    theta = torch.as_tensor(theta, dtype=DT)
    if not bf16:
        return theta
    return bf16_round(theta) + (theta - theta.detach())


def _silu_chain(z, z1, z2):
    """silu applied to z with the first and second derivative chains of z."""
    sg = torch.sigmoid(z)
    a = z * sg
    d1 = sg * (1.0 + z * (1.0 - sg))
    d2 = sg * (1.0 - sg) * (2.0 + z * (1.0 - 2.0 * sg))
    return a, d1 * z1, d2 * z1 * z1 + d1 * z2


def network(theta, spec, r, ch, bf16=True):
    """m(r, c), dm/dr, d2m/dr2 for radii r [P] and channels ch [P]."""
    th = used_weights(theta, bf16)
    W1, b1, W2, b2, w3, b3 = unpack(th, spec)
    r = torch.as_tensor(r, dtype=DT)
    ch = torch.as_tensor(ch, dtype=torch.long)
    l2 = torch.tensor(spec.ell, dtype=DT) ** 2
    r2 = (r * r)[:, None]
    den = r2 + l2[None, :]
    f0 = r2 / den
    f1 = 2.0 * r[:, None] * l2 / den ** 2
    f2 = 2.0 * l2 * (l2 - 3.0 * r2) / den ** 3
    onehot = torch.nn.functional.one_hot(ch, spec.n_ch).to(DT)
    zero = torch.zeros_like(onehot)
    x0 = torch.cat([f0, onehot], 1)
    x1 = torch.cat([f1, zero], 1)
    x2 = torch.cat([f2, zero], 1)
    h, h1, h2 = _silu_chain(x0 @ W1.T + b1, x1 @ W1.T, x2 @ W1.T)
    h, h1, h2 = _silu_chain(h @ W2.T + b2, h1 @ W2.T, h2 @ W2.T)
    return h @ w3 + b3, h1 @ w3, h2 @ w3


def radial(theta, spec, r, ch, bf16=True):
    """g_c(r), g_c'(r), g_c''(r): the network times the smooth cut-off."""
    r = torch.as_tensor(r, dtype=DT)
    ch = torch.as_tensor(ch, dtype=torch.long)
    m, m1, m2 = network(theta, spec, r, ch, bf16)
    rc = torch.tensor(spec.r_cut, dtype=DT)[ch]
    t = r / rc
    inside = t < 1.0
    s = torch.where(inside, 1 - 10 * t ** 3 + 15 * t ** 4 - 6 * t ** 5, torch.zeros_like(t))
    s1 = torch.where(inside, (-30 * t ** 2 + 60 * t ** 3 - 30 * t ** 4) / rc, torch.zeros_like(t))
    s2 = torch.where(inside, (-60 * t + 180 * t ** 2 - 120 * t ** 3) / rc ** 2, torch.zeros_like(t))
    return m * s, m1 * s + m * s1, m2 * s + 2 * m1 * s1 + m * s2


@dataclass
class Table:
    r_cut: np.ndarray   # [n_ch]
    species: np.ndarray  # [n_nuc]
    n_cells: int
    nodes: np.ndarray   # [n_ch][n_cells + 1][3]: g, g', g'' at r_k = r_cut (k/n)^2


def table(theta, spec, n_cells=None, bf16=True) -> Table:
    """Node data of the interpolated term: g, g', g'' of every channel at
    r_k = r_cut (k/n)^2, k = 0..n."""
    n = spec.n_cells if n_cells is None else n_cells
    k = np.arange(n + 1, dtype=np.float64)
    nodes = np.zeros((spec.n_ch, n + 1, 3))
    with torch.no_grad():
        for c in range(spec.n_ch):
            r = spec.r_cut[c] * (k / n) ** 2
            g, g1, g2 = radial(theta, spec, r, np.full(n + 1, c), bf16)
            nodes[c, :, 0], nodes[c, :, 1], nodes[c, :, 2] = g.numpy(), g1.numpy(), g2.numpy()
    return Table(np.array(spec.r_cut, dtype=np.float64), np.array(spec.species, dtype=np.int32), n, nodes)


def pair_lists(N, n_up, n_nuc, species):
    """Electron pairs (i < j, channel 0 equal spin / 1 opposite) and
    electron-nucleus pairs (i, I, channel 2 + species[I])."""
    ee = [(i, j, 0 if (i < n_up) == (j < n_up) else 1) for i in range(N) for j in range(i + 1, N)]
    en = [(i, I, 2 + int(species[I])) for i in range(N) for I in range(n_nuc)]
    return ee, en


def energy_terms(theta, spec, x, n_up, nuc_xyz, grad_base, e_base, bf16=True):
    """E_L(theta) and J_NN(theta) of every configuration x [n][N][3], from the
    base terms (grad_base [n][N][3] = grad_i log|D exp(J_P)|, e_base [n])."""
    x = torch.as_tensor(x, dtype=DT)
    n, N, _ = x.shape
    nuc = torch.as_tensor(nuc_xyz, dtype=DT)
    ee, en = pair_lists(N, n_up, len(nuc), spec.species)
    G = torch.zeros(n, N, 3, dtype=DT)
    L = torch.zeros(n, N, dtype=DT)
    J = torch.zeros(n, dtype=DT)
    if ee:
        i = torch.tensor([p[0] for p in ee]); j = torch.tensor([p[1] for p in ee])
        c = torch.tensor([p[2] for p in ee])
        d = x[:, i] - x[:, j]                      # [n][P][3]
        r = torch.linalg.norm(d, dim=2)
        g, g1, g2 = radial(theta, spec, r.reshape(-1), c.repeat(n), bf16)
        g, g1, g2 = g.view(n, -1), g1.view(n, -1), g2.view(n, -1)
        gv = (g1 / r)[..., None] * d
        G = G.index_add(1, i, gv).index_add(1, j, -gv)
        lap = g2 + 2.0 * g1 / r
        L = L.index_add(1, i, lap).index_add(1, j, lap)
        J = J + g.sum(1)
    if en:
        i = torch.tensor([p[0] for p in en]); I = torch.tensor([p[1] for p in en])
        c = torch.tensor([p[2] for p in en])
        d = x[:, i] - nuc[I][None]
        r = torch.linalg.norm(d, dim=2)
        g, g1, g2 = radial(theta, spec, r.reshape(-1), c.repeat(n), bf16)
        g, g1, g2 = g.view(n, -1), g1.view(n, -1), g2.view(n, -1)
        G = G.index_add(1, i, (g1 / r)[..., None] * d)
        L = L.index_add(1, i, g2 + 2.0 * g1 / r)
        J = J + g.sum(1)
    a = torch.as_tensor(grad_base, dtype=DT)
    e0 = torch.as_tensor(e_base, dtype=DT)
    EL = e0 - 0.5 * (2.0 * (a * G).sum((1, 2)) + (G * G).sum((1, 2)) + L.sum(1))
    return EL, J


def variance_loss(EL, J):
    """Reweighted variance sum w (E - Ebar)^2 / sum w, w = exp(2 J) (shifted
    by max J, which cancels)."""
    w = torch.exp(2.0 * (J - J.max().detach()))
    sw = w.sum()
    ebar = (w * EL).sum() / sw
    return (w * (EL - ebar) ** 2).sum() / sw


def loss_and_grad(theta, spec, x, n_up, nuc_xyz, grad_base, e_base, bf16=True):
    th = torch.tensor(np.asarray(theta, dtype=np.float64), requires_grad=True)
    EL, J = energy_terms(th, spec, x, n_up, nuc_xyz, grad_base, e_base, bf16)
    loss = variance_loss(EL, J)
    loss.backward()
    return float(loss.detach()), th.grad.numpy().copy(), EL.detach().numpy(), J.detach().numpy()


def base_terms(osys, x):
    """grad_i log|psi_G| and E_L of the oracle system (without a neural term)
    for every configuration: the base terms of energy_terms."""
    n = len(x)
    grad = np.zeros((n, osys.N, 3))
    e = np.zeros(n)
    for w in range(n):
        Au, Ad = osys.inverses(x[w])
        grad[w] = osys.grad_log_psi(x[w], Au, Ad)
        e[w] = osys.local_energy(x[w], Au, Ad)
    return grad, e
