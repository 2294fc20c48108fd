"""The per-species ensemble (Sec. 3.2: one network per species mass fraction, hidden
layers 1600, 800, 400, each trained on its own output) on the GPU against the oracle.

* Forward: against oracle.ann.network_ensemble with the device's BF16 rounding points,
  at the paper's widths and at ragged widths whose per-network K and N end inside a
  tile (the grouped maps must clip at each network's own bound, not the next one's),
  several chunks and a ragged tail. Bound as for the multi-output network: 99.99 %
  within 1e-2 (|u| + rms u), all within 3e-2 (|u| + rms u).
* chem_step_ann on an ensemble: Y', T' against the oracle step.
* Training: the gradients of one step against the oracle's per-network backward,
  element by element within 8 standard deviations of the device's BF16 rounding
  (tests/grad_bounds.py), with the norms as a summary.
* The autotuner's tile widths change no output bit; a checkpoint restores the ensemble
  exactly; E4M3 requests are refused.
Weights, statistics and states come from the seeded generator, never from the GPU.
"""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def _problem(n, hidden=(1600, 800, 400), seed=2042):
    mech = synth.get_mech("c2")
    T, p, Y = synth.states_profiles(mech, n, seed, synth.padded_ld(n))
    widths = [mech.N + 2, *hidden, mech.N - 1]
    nets = synth.mlp_ensemble(widths, 3000 + seed)
    x = M.features(T[:n], p[:n], Y[:, :n])
    mu_x, sd_x = M.zscore_stats(x)
    rng = np.random.default_rng(seed + 7)
    mu_u = rng.uniform(-1e-5, 1e-5, mech.N - 1)
    sd_u = 10.0 ** rng.uniform(-6, -3, mech.N - 1)
    return mech, T, p, Y, widths, nets, (mu_x, sd_x, mu_u, sd_u)


def _ens(widths, nets, stats, **kw):
    from paper_2312_05800_gb300 import binding
    net = binding.Mlp(dev_mech("c2"), hidden=widths[1:4], ensemble=True, **kw)
    assert net.groups == widths[4] and net.widths == widths
    net.set_params(synth.flatten_layers(synth.stack_ensemble(nets)))
    net.set_norm(*stats)
    return net


def _gpu_u(net, T, p, Y, n):
    import torch
    from paper_2312_05800_gb300 import binding
    u = torch.full((n, 32), float("nan"), dtype=torch.float32, device="cuda")
    binding.chem_mlp_forward(net, n, T.shape[0], to_dev(T), to_dev(p), to_dev(Y), u, 32)
    torch.cuda.synchronize()
    assert net.error() == 0
    return u.double().cpu().numpy()[:, :net.widths[4]]


def _check_u(u, uq):
    rms = np.sqrt(np.mean(uq ** 2))
    err = np.abs(u - uq)
    assert np.mean(err <= 1e-2 * (np.abs(uq) + rms)) >= 0.9999
    bound = 3e-2 * (np.abs(uq) + rms)
    if not np.all(err <= bound):
        i, j = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError("%d of %d outside; worst cell %d network %d: gpu %.6g oracle %.6g (rms %.3g)"
                             % ((err > bound).sum(), err.size, i, j, u[i, j], uq[i, j], rms))


@pytest.mark.parametrize("n,hidden,chunk", [(600, (1600, 800, 400), 256),
                                            (3001, (104, 56, 24), 1024),
                                            (3001, (160, 80, 48), 1024)])
def test_ensemble_forward_parity(n, hidden, chunk):
    mech, T, p, Y, widths, nets, stats = _problem(n, hidden)
    net = _ens(widths, nets, stats, chunk=chunk)
    u = _gpu_u(net, T, p, Y, n)
    uq = A.forward_u(mech, nets, stats, T[:n], p[:n], Y[:, :n], round_bf16=True, ensemble=True)
    _check_u(u, uq)
    u64 = A.forward_u(mech, nets, stats, T[:n], p[:n], Y[:, :n], ensemble=True)
    assert np.sqrt(np.mean((u - u64) ** 2)) <= 3e-2 * np.sqrt(np.mean(u64 ** 2))
    net.free()


def test_ensemble_tiles_change_no_bit():
    from paper_2312_05800_gb300 import binding
    n = 2000
    mech, T, p, Y, widths, nets, stats = _problem(n, (160, 80, 48), seed=2043)
    net = _ens(widths, nets, stats, chunk=1024)
    u0 = _gpu_u(net, T, p, Y, n)
    tiles = binding.chem_mlp_autotune(net, 1024)
    assert tiles[3] == 0
    assert np.array_equal(_gpu_u(net, T, p, Y, n), u0)
    net.free()


def test_ensemble_step_ann_parity():
    import torch
    from paper_2312_05800_gb300 import binding
    n = 1001
    mech, T, p, Y, widths, nets, stats = _problem(n, (256, 128, 64), seed=2044)
    net = _ens(widths, nets, stats, chunk=512)
    ld = T.shape[0]
    Td, pd, Yd = to_dev(T), to_dev(p), to_dev(Y)
    st = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
    binding.chem_step_ann(dev_mech("c2"), net, n, ld, 1e-6, binding.CHEM_PREC_BF16, None, Td, pd, Yd, st)
    torch.cuda.synchronize()
    Tg, Yg = Td.cpu().numpy(), Yd.cpu().numpy()
    To, Yo = A.step_ann(mech, nets, stats, T[:n], p[:n], Y[:, :n], round_bf16=True, ensemble=True)
    assert np.all(st.cpu().numpy()[:n] == 0)
    assert np.abs(Yg[:, :n].sum(axis=0) - 1).max() < 1e-12 and Yg[:, :n].min() >= 0
    sd_u = stats[3]
    uq = A.forward_u(mech, nets, stats, T[:n], p[:n], Y[:, :n], round_bf16=True, ensemble=True)
    bdy = (3e-2 * (np.abs(uq) + np.sqrt(np.mean(uq ** 2))) * sd_u).T
    sp = A.out_species(mech)
    btot = np.zeros_like(Yo)
    btot[sp, :] = bdy
    btot[mech.bath, :] = bdy.sum(axis=0)
    bound = btot + Yo * 2.0 * bdy.sum(axis=0)[None, :] + 1e-12
    err = np.abs(Yg[:, :n] - Yo)
    assert np.all(err <= bound), (err / bound).max()
    assert np.all(np.abs(Tg[:n] - To) <= 0.5 + 1e-5 * To), np.abs(Tg[:n] - To).max()
    assert np.array_equal(Tg[n:], T[n:])
    with pytest.raises(binding.ChemError):
        binding.chem_step_ann(dev_mech("c2"), net, n, ld, 1e-6, binding.CHEM_PREC_FP8, None, Td, pd, Yd, st)
    with pytest.raises(binding.ChemError):
        binding.chem_mlp_set_fp8_scales(net, [1.0, 1.0])
    net.free()


@pytest.mark.parametrize("hidden", [(256, 128, 64), (104, 56, 24)])
def test_ensemble_train_gradients_match_oracle(hidden):
    # Each network's gradients against the oracle's backward of its own Eq. 5 term, element by
    # element within 8 standard deviations of the device's BF16 rounding (tests/grad_bounds.py),
    # norms as a summary; targets keep every residual at least 0.5 rms(u) from zero.
    import torch
    from paper_2312_05800_gb300 import binding
    from tests.grad_bounds import check, gradients_with_sigma, separated_targets
    B = 512
    mech, T, p, Y, widths, nets, stats = _problem(B, hidden, seed=2045)
    mu_x, sd_x, mu_u, sd_u = stats
    z = (M.features(T[:B], p[:B], Y[:, :B]) - mu_x) / sd_x
    uq = A.network_ensemble(nets, np.asarray(z, np.float32).astype(np.float64), round_bf16=True)
    target = separated_targets(uq, np.random.default_rng(5))
    sp = A.out_species(mech)
    Y1 = Y.copy()
    Y1[sp, :B] += (target * sd_u + mu_u).T
    net = _ens(widths, nets, stats, max_batch=B)
    ld = T.shape[0]
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    binding.mlp_train_step(net, B, None, ld, to_dev(T), to_dev(p), to_dev(Y), to_dev(Y1), 0.0, loss)
    torch.cuda.synchronize()
    assert net.error() == 0
    G = widths[4]
    grads = synth.unstack_ensemble(_restack(net.get_grads(), widths, G), G)
    total = 0.0
    ga, gb = [[] for _ in range(4)], [[] for _ in range(4)]
    for g in range(G):
        lo, go, sig, min_res = gradients_with_sigma(nets[g], z, target[:, g:g + 1], uq[:, g:g + 1])
        total += lo
        for l in range(4):
            for j in range(2):
                check(grads[g][l][j], go[l][j], sig[l][j], "network %d layer %d %s" % (g, l + 1, "dW" if j == 0 else "db"))
            ga[l].append(grads[g][l][0].ravel())
            gb[l].append(go[l][0].ravel())
    assert abs(float(loss[0].item()) - total) <= 2e-2 * total
    for l in range(4):
        a, b = np.concatenate(ga[l]), np.concatenate(gb[l])
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert cos >= 0.9999 and rel <= 1e-2, (l, cos, rel)
    net.free()


def _restack(flat, widths, G):
    """The C ABI's flat ensemble parameters as stacked (W [G out_l][in_l], b [G out_l]) per layer."""
    out, o = [], 0
    outs = [widths[1], widths[2], widths[3], 1]
    for l in range(4):
        fi, fo = widths[l], G * outs[l]
        W = flat[o:o + fo * fi].reshape(fo, fi).astype(np.float64)
        o += fo * fi
        b = flat[o:o + fo].astype(np.float64)
        o += fo
        out.append((W, b))
    assert o == flat.size
    return out


def test_ensemble_checkpoint_roundtrip(tmp_path):
    import torch
    from paper_2312_05800_gb300 import binding
    B = 256
    mech, T, p, Y, widths, nets, stats = _problem(B, (104, 56, 24), seed=2046)
    dY = np.random.default_rng(6).normal(size=Y.shape) * stats[3].mean()
    ld = T.shape[0]
    Td, pd, Yd, dYd = to_dev(T), to_dev(p), to_dev(Y), to_dev(Y + dY)
    a = _ens(widths, nets, stats, max_batch=B)
    for _ in range(2):
        binding.mlp_train_step(a, B, None, ld, Td, pd, Yd, dYd, 1e-3)
    path = str(tmp_path / "ens.bin")
    a.save(path)
    b = binding.Mlp.load(dev_mech("c2"), path)
    assert b.ensemble and b.groups == widths[4] and b.nparams == a.nparams
    for _ in range(2):
        binding.mlp_train_step(a, B, None, ld, Td, pd, Yd, dYd, 1e-3)
        binding.mlp_train_step(b, B, None, ld, Td, pd, Yd, dYd, 1e-3)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    assert np.array_equal(_gpu_u(a, T, p, Y, B), _gpu_u(b, T, p, Y, B))
    a.free()
    b.free()
