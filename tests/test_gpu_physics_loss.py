"""The physics terms of the training loss (Sec. 3.2: mass-fraction unity, energy
and heat release; the forms are the readings of oracle/physics_loss.py) in the
device's training step, against the oracle.

* chem_mlp_fit_physics_scales against oracle/physics_loss.py::scales (FP32
  enthalpy rows on the device): 1e-5 relative.
* One training step with lam_m = lam_q = 0.5: the loss within 2e-2 of the
  oracle's, and every gradient element within 8 standard deviations of the
  device's BF16 rounding (tests/grad_bounds.py) of the oracle's backward from
  the oracle's dL/du. The targets keep every residual, and each sample's bath
  and heat-release residuals, far from zero, so both sides take the same signs.
* The terms change the gradients: with weights 0 the step's gradients differ
  from these by far more than the bound (the terms are not silently dropped).
"""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from oracle import physics_loss as PL
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def _case(B, seed):
    mech = synth.get_mech("c2")
    T, p, Y = synth.states_profiles(mech, B, seed, synth.padded_ld(B))
    widths = [mech.N + 2, 256, 128, 64, mech.N - 1]
    layers = synth.mlp_layers(widths, 3000 + seed)
    mu_x, sd_x = M.zscore_stats(M.features(T[:B], p[:B], Y[:, :B]))
    rng = np.random.default_rng(seed + 7)
    stats = (mu_x, sd_x, rng.uniform(-1e-5, 1e-5, mech.N - 1), 10.0 ** rng.uniform(-6, -3, mech.N - 1))
    return mech, T, p, Y, widths, layers, stats


def _targets(uq, c, sd_u, rng):
    """u* = uq - r with |r_j| >= 0.5 rms(uq) and, per sample, |sum_j sd_j r_j| and
    |sum_j c_j sd_j r_j| at least 0.3 of their absolute sums (random signs, resampled)."""
    rms = np.sqrt(np.mean(uq ** 2))
    r = np.zeros_like(uq)
    for i in range(uq.shape[0]):
        for _ in range(1000):
            ri = rng.choice([-1.0, 1.0], size=uq.shape[1]) * (0.5 + np.abs(rng.normal(size=uq.shape[1]))) * rms
            m, am = np.sum(sd_u * ri), np.sum(sd_u * np.abs(ri))
            q, aq = np.sum(c[i] * sd_u * ri), np.sum(np.abs(c[i]) * sd_u * np.abs(ri))
            if abs(m) >= 0.3 * am and abs(q) >= 0.3 * aq:
                break
        else:
            raise AssertionError("no separated residual for sample %d" % i)
        r[i] = ri
    return uq - r


def _net(widths, layers, stats, B):
    from paper_2312_05800_gb300 import binding
    net = binding.Mlp(dev_mech("c2"), hidden=widths[1:4], max_batch=B)
    net.set_params(synth.flatten_layers(layers))
    net.set_norm(*stats)
    return net


def test_physics_scales_match_oracle():
    mech, T, p, Y, widths, layers, stats = _case(5000, 2091)
    n, ld = 5000, T.shape[0]
    sp = A.out_species(mech)
    dY = np.zeros_like(Y)
    dY[sp, :n] = np.random.default_rng(3).normal(size=(len(sp), n)) * stats[3][:, None]
    net = _net(widths, layers, stats, 256)
    sm, sq = net.fit_physics_scales(n, ld, to_dev(T), to_dev(Y), to_dev(Y + dY))
    om, oq = PL.scales(mech, T[:n], ((Y + dY) - Y)[sp, :n].T, sp)
    assert abs(sm - om) <= 1e-5 * om and abs(sq - oq) <= 1e-5 * oq, (sm, om, sq, oq)
    net.free()


def test_train_step_with_physics_terms_matches_oracle():
    import torch
    from paper_2312_05800_gb300 import binding
    from tests.grad_bounds import check, gradients_with_sigma
    B = 256
    mech, T, p, Y, widths, layers, stats = _case(B, 2092)
    mu_x, sd_x, mu_u, sd_u = stats
    sp = A.out_species(mech)
    z = (M.features(T[:B], p[:B], Y[:, :B]) - mu_x) / sd_x
    uq = A.network(layers, np.asarray(z, np.float32).astype(np.float64), round_bf16=True)
    _, c = PL.heat_release(mech, T[:B], np.zeros_like(uq), sp)           # c [B, G] = h_k - h_bath
    target = _targets(uq, c, sd_u, np.random.default_rng(2093))
    Y1 = Y.copy()
    Y1[sp, :B] += (target * sd_u + mu_u).T
    s_m, s_q = PL.scales(mech, T[:B], (target * sd_u + mu_u), sp)
    lam = (0.5, 0.5)
    # oracle: the loss on the FP64 forward, dL/du with its signs from the forward at the device's
    # rounding points (the residuals are far from zero, so the signs agree)
    u64 = A.network(layers, z)
    lo, _ = PL.loss(mech, u64, target, T[:B], stats, sp, lam[0], lam[1], s_m, s_q)
    _, dout = PL.loss(mech, uq, target, T[:B], stats, sp, lam[0], lam[1], s_m, s_q)
    _, go, sig, _ = gradients_with_sigma(layers, z, target, uq, dout=dout)
    net = _net(widths, layers, stats, B)
    net.set_physics_loss(lam[0], lam[1], s_m, s_q)
    ld = T.shape[0]
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    args = (B, None, ld, to_dev(T), to_dev(p), to_dev(Y), to_dev(Y1), 0.0, loss)
    binding.mlp_train_step(net, *args)
    torch.cuda.synchronize()
    assert net.error() == 0
    assert abs(float(loss[0].item()) - lo) <= 2e-2 * lo, (float(loss[0].item()), lo)
    g = synth.unflatten(net.get_grads(), widths)
    for l in range(4):
        for j, key in ((0, "W"), (1, "b")):
            check(g[l][j], go[l][j], sig[l][j], "layer %d d%s" % (l + 1, key))
    # the same step without the terms moves the top layer's bias gradient far outside the bound
    net.set_physics_loss(0.0, 0.0, s_m, s_q)
    binding.mlp_train_step(net, *args)
    torch.cuda.synchronize()
    g0 = synth.unflatten(net.get_grads(), widths)
    assert np.any(np.abs(g0[3][1] - go[3][1]) > 8 * sig[3][1] + 1e-12)
    net.free()
