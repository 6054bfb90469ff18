"""Training of the neural pair term of the Jastrow factor on the GPU.

The network and its radial derivatives run in the library's own kernels
(lrdmc_nj_forward / lrdmc_nj_backward behind ``NeuralJastrowTerms``, a
torch.autograd.Function); PyTorch supplies the device memory, the reduction
of the per-configuration values to the objective and the Adam update.

Objective (variance minimisation with correlated-sampling reweighting): a
fixed sample of configurations x, drawn from a projection run without the
term, is reweighted by |psi_theta / psi_0|^2 = exp(2 J_NN(x)), and
  L(theta) = sum_x w_x (E_L(x) - Ebar)^2 / sum_x w_x,  Ebar = sum w E_L / sum w.
E_L(x) = e_base - 1/2 sum_i [2 a_i . G_i + |G_i|^2 + L_i] combines the base
terms of the trial function without the term (lrdmc_base_terms, FP64) with
the term's gradient G_i and Laplacian L_i.

After training, ``LrdmcSystem.set_neural_jastrow`` tabulates the network for
the projection (quintic Hermite cells, FP64 node values).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch


class NeuralJastrowTerms(torch.autograd.Function):
    """(params) -> (E_L [n], J_NN [n]) for configurations fixed at apply time."""

    @staticmethod
    def forward(ctx, params, lsys, spec, x, grad_base, e_base, bf16):
        el, j, q, _ = lsys.nj_forward(spec, params, x, grad_base, e_base, bf16)
        ctx.save_for_backward(params, q)
        ctx.lsys, ctx.spec, ctx.x, ctx.bf16 = lsys, spec, x, bf16
        return el, j

    @staticmethod
    def backward(ctx, d_el, d_j):
        params, q = ctx.saved_tensors
        n = ctx.x.shape[0]
        if d_el is None:
            d_el = torch.zeros(n, dtype=torch.float32, device=params.device)
        if d_j is None:
            d_j = torch.zeros(n, dtype=torch.float32, device=params.device)
        grad = ctx.lsys.nj_backward(ctx.spec, params, ctx.x, q, d_el.float(), d_j.float(), ctx.bf16)
        return grad, None, None, None, None, None, None


def variance_loss(el, j, reweight=True, clip=0.0):
    """Variance of E_L over the sample (float64 reduction of float32 values),
    each configuration weighted by exp(2 J_NN) when ``reweight``. With
    clip = k > 0 the local energies are first limited to the median
    +- k times the mean absolute deviation from the median (fixed per
    batch), which keeps the rare near-node values of the heavy-tailed
    distribution from dominating the estimate and its gradient."""
    el = el.double()
    j = j.double()
    if clip > 0:
        med = el.detach().median()
        mad = (el.detach() - med).abs().mean()
        el = torch.minimum(torch.maximum(el, med - clip * mad), med + clip * mad)
    if reweight:
        w = torch.exp(2.0 * (j - j.max().detach()))
    else:
        w = torch.ones_like(el)
    sw = w.sum()
    ebar = (w * el).sum() / sw
    return (w * (el - ebar) ** 2).sum() / sw


def effective_sample_fraction(j):
    """(sum w)^2 / (n sum w^2) of the reweighting factors exp(2 J)."""
    w = torch.exp(2.0 * (j.double() - j.double().max()))
    return float(w.sum() ** 2 / (len(w) * (w * w).sum()))


def evaluate(lsys, spec, params, x, grad_base, e_base, bf16=True, chunk=1 << 17):
    """E_L and J_NN of every configuration, in chunks."""
    els, js = [], []
    with torch.no_grad():
        for s in range(0, x.shape[0], chunk):
            el, j, _, _ = lsys.nj_forward(spec, params, x[s:s + chunk], grad_base[s:s + chunk], e_base[s:s + chunk],
                                          bf16)
            els.append(el)
            js.append(j)
    return torch.cat(els), torch.cat(js)


def train(lsys, spec, params0, x, grad_base, e_base, steps=400, batch=1 << 14, lr=1e-3, seed=0, bf16=True,
          log_every=0, min_ess=0.3, reweight=True, clip=5.0):
    """Adam on the (reweighted, clipped) variance over random minibatches
    of the sample. With reweighting, steps whose batch has an effective
    sample fraction below ``min_ess`` are skipped (the sample no longer
    represents |psi_theta|^2 there). Returns (params, history of (step,
    loss))."""
    dev = x.device
    params = torch.tensor(np.asarray(params0, dtype=np.float32), device=dev, requires_grad=True)
    opt = torch.optim.Adam([params], lr=lr)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    n = x.shape[0]
    hist = []
    for it in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), generator=gen, device=dev)
        el, j = NeuralJastrowTerms.apply(params, lsys, spec, x[idx], grad_base[idx], e_base[idx], bf16)
        if reweight and effective_sample_fraction(j.detach()) < min_ess:
            continue
        loss = variance_loss(el, j, reweight, clip)
        opt.zero_grad()
        loss.backward()
        opt.step()
        if log_every and it % log_every == 0:
            hist.append((it, float(loss.detach())))
    return params.detach(), hist


def sample_configurations(lsys_plain, x0, n_configs, a, spacing, tau, e_trial, seed=1, every=4, equil=50):
    """Configurations from a projection run without the term: the
    population after ``equil`` intervals, then every ``every`` intervals
    until n_configs are collected (float64 CUDA tensor [n][N][3])."""
    W = x0.shape[0]
    snaps = math.ceil(n_configs / W)
    lsys_plain.init_walkers(torch.as_tensor(x0, device="cuda"), seed=seed, tau=tau, e_trial=e_trial,
                            recompute_every=5, trace_capacity=equil + snaps * every + 4)
    lsys_plain.step(equil, a, spacing)
    out = []
    for _ in range(snaps):
        lsys_plain.step(every, a, spacing)
        out.append(torch.as_tensor(lsys_plain.walkers()["x"], device="cuda"))
    return torch.cat(out)[:n_configs].contiguous()


def timed(fn, *args, **kw):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = fn(*args, **kw)
    torch.cuda.synchronize()
    return r, time.perf_counter() - t0
