"""The learned step on the GPU (Sec. 3.2; Eq. 5) against the FP64 oracle.

* Forward: against the oracle with BF16 rounding at the points where the device
  stores BF16 (input rows, weights, hidden activations; FP64 accumulation):
  99.99 % of outputs within 1e-2 (|u| + rms u) and all within 3e-2 (|u| + rms u)
  (a rounding flip of one hidden unit moves an output by one BF16 step of that
  unit). Against the plain FP64 oracle, relative RMS <= 3e-2.
* Z-score statistics (FP64 on both sides): 1e-10 relative.
* chem_step_ann: Y' and T' against the oracle step with the same BF16 points.
* Training: gradients of one step against the oracle's backward pass, element
  by element within 8 standard deviations of the device's BF16 rounding
  (tests/grad_bounds.py), with cosine >= 0.9999 and relative L2 <= 1e-2 per
  layer as a summary; Adam's first step moves every parameter by at most lr,
  opposite to the gradient's sign.
Weights, statistics and states come from the seeded generator, never from the GPU.
"""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def _problem(n, seed=2002, name="c2"):
    mech = synth.get_mech(name)
    T, p, Y = synth.states_profiles(mech, n, seed, synth.padded_ld(n))
    widths = [mech.N + 2, 1600, 800, 400, mech.N - 1]
    layers = synth.mlp_layers(widths, 3000 + seed)
    x = M.features(T[:n], p[:n], Y[:, :n])
    mu_x, sd_x = M.zscore_stats(x)
    rng = np.random.default_rng(seed + 7)
    mu_u = rng.uniform(-1e-5, 1e-5, mech.N - 1)
    sd_u = 10.0 ** rng.uniform(-6, -3, mech.N - 1)
    return mech, T, p, Y, widths, layers, (mu_x, sd_x, mu_u, sd_u)


def _mlp(mech_name, widths, layers, stats, **kw):
    from paper_2312_05800_gb300 import binding
    net = binding.Mlp(dev_mech(mech_name), hidden=widths[1:4], **kw)
    assert net.widths == widths
    net.set_params(synth.flatten_layers(layers))
    net.set_norm(*stats)
    return net


def _gpu_u(net, T, p, Y, n):
    import torch
    from paper_2312_05800_gb300 import binding
    ld = T.shape[0]
    u = torch.full((n, 32), float("nan"), dtype=torch.float32, device="cuda")
    binding.chem_mlp_forward(net, n, ld, to_dev(T), to_dev(p), to_dev(Y), u, 32)
    torch.cuda.synchronize()
    assert net.error() == 0
    return u.double().cpu().numpy()[:, :net.widths[4]]


def test_bf16_rounding_matches_torch():
    import torch
    x = np.random.default_rng(0).normal(size=10000) * 10.0 ** np.random.default_rng(1).uniform(-5, 5, 10000)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).double().numpy()
    assert np.array_equal(A.to_bf16(x), ref)


@pytest.mark.parametrize("n", [1000, 20000])
def test_forward_parity(n):
    mech, T, p, Y, widths, layers, stats = _problem(n)
    net = _mlp("c2", widths, layers, stats, chunk=8192)   # several chunks and a ragged tail
    u = _gpu_u(net, T, p, Y, n)
    uq = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n], round_bf16=True)
    rms = np.sqrt(np.mean(uq ** 2))
    err = np.abs(u - uq)
    # a hidden activation whose FP32 and FP64 sums fall on opposite sides of a
    # BF16 rounding boundary moves the output by one BF16 step of that unit
    assert np.mean(err <= 1e-2 * (np.abs(uq) + rms)) >= 0.9999
    bound = 3e-2 * (np.abs(uq) + rms)
    if not np.all(err <= bound):
        i, j = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError("%d of %d outside; worst cell %d out %d: gpu %.6g oracle %.6g (rms %.3g, rel rms %.3g)"
                             % ((err > bound).sum(), err.size, i, j, u[i, j], uq[i, j], rms,
                                np.sqrt(np.mean(err ** 2)) / rms))
    u64 = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n])
    assert np.sqrt(np.mean((u - u64) ** 2)) <= 3e-2 * np.sqrt(np.mean(u64 ** 2))
    net.free()


def test_fit_norm_matches_oracle():
    import torch
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y, widths, layers, stats = _problem(5000)
    n, ld = 5000, T.shape[0]
    dY = np.random.default_rng(5).normal(size=Y.shape) * 1e-4
    net = _mlp("c2", widths, layers, stats)
    binding.chem_mlp_fit_norm(net, n, ld, to_dev(T), to_dev(p), to_dev(Y), to_dev(Y + dY))
    mx, sx, mu, su = net.get_norm()
    omx, osx = M.zscore_stats(M.features(T[:n], p[:n], Y[:, :n]))
    sp = A.out_species(mech)
    du = (Y + dY) - Y
    omu, osu = du[sp, :n].mean(axis=1), du[sp, :n].std(axis=1)
    assert np.allclose(mx, omx, rtol=1e-10, atol=1e-12)
    assert np.allclose(sx, np.where(osx < 1e-12, 1.0, osx), rtol=1e-10, atol=0)
    assert np.allclose(mu, omu, rtol=1e-9, atol=1e-18)
    assert np.allclose(su, osu, rtol=1e-10, atol=0)
    net.free()


def test_step_ann_parity(oracle):
    import torch
    from paper_2312_05800_gb300 import binding
    n = 3001
    mech, T, p, Y, widths, layers, stats = _problem(n, seed=2012)
    net = _mlp("c2", widths, layers, stats, chunk=1024)
    ld = T.shape[0]
    Td, pd, Yd = to_dev(T), to_dev(p), to_dev(Y)
    st = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
    binding.chem_step_ann(dev_mech("c2"), net, n, ld, 1e-6, binding.CHEM_PREC_BF16, None, Td, pd, Yd, st)
    torch.cuda.synchronize()
    Tg, Yg = Td.cpu().numpy(), Yd.cpu().numpy()
    To, Yo = A.step_ann(mech, layers, stats, T[:n], p[:n], Y[:, :n], round_bf16=True)
    assert np.all(st.cpu().numpy()[:n] == 0)
    assert np.abs(Yg[:, :n].sum(axis=0) - 1).max() < 1e-12 and Yg[:, :n].min() >= 0
    # the forward parity bounds on u (99.95 % within 1e-2 (|u| + rms u), all within 3e-2: a BF16
    # rounding flip of one hidden unit moves an output by one BF16 step of it), carried through
    # dY = sd_u u + mu_u
    sd_u = stats[3]
    uq = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n], round_bf16=True)
    sp = A.out_species(mech)
    err = np.abs(Yg[:, :n] - Yo)

    def bound(tol):
        bdy = (tol * (np.abs(uq) + np.sqrt(np.mean(uq ** 2))) * sd_u).T      # [n_out, n] bound on dY
        # Y' = y / sum(y): an error in any dY moves every species through the sum
        btot = np.zeros_like(Yo)
        btot[sp, :] = bdy
        btot[mech.bath, :] = bdy.sum(axis=0)
        return btot + Yo * 2.0 * bdy.sum(axis=0)[None, :] + 1e-12

    b1, b3 = bound(1e-2), bound(3e-2)
    assert np.mean(err <= b1) >= 0.9995, np.mean(err <= b1)
    if not np.all(err <= b3):
        k, i = np.unravel_index(np.argmax(err / b3), err.shape)
        raise AssertionError("%d outside; worst species %d cell %d: %.3g vs bound %.3g"
                             % ((err > b3).sum(), k, i, err[k, i], b3[k, i]))
    assert np.all(np.abs(Tg[:n] - To) <= 0.2 + 1e-5 * To), np.abs(Tg[:n] - To).max()
    # nothing past ncells is touched
    assert np.array_equal(Tg[n:], T[n:])
    with pytest.raises(binding.ChemError):
        binding.chem_step_ann(dev_mech("c2"), net, n, ld, 2e-6, 0, None, Td, pd, Yd, st)
    net.free()


def _train_case(B=512, seed=2022):
    mech, T, p, Y, widths, layers, stats = _problem(B, seed=seed)
    dY = np.random.default_rng(seed).normal(size=Y.shape) * stats[3].mean()
    return mech, T, p, Y, dY, widths, layers, stats


def test_train_gradients_match_oracle():
    # One training step's gradients against the oracle's FP64 backward, element by element,
    # within 8 standard deviations of the device's BF16 rounding (tests/grad_bounds.py); the
    # norms stay as a summary. The targets keep every residual u - u* at least 0.5 rms(u)
    # from zero, so the L1 subgradient's sign is the same on both sides.
    import torch
    from paper_2312_05800_gb300 import binding
    from tests.grad_bounds import check, gradients_with_sigma, separated_targets
    B = 512
    mech, T, p, Y, _, widths, layers, stats = _train_case(B)
    mu_x, sd_x, mu_u, sd_u = stats
    z = (M.features(T[:B], p[:B], Y[:, :B]) - mu_x) / sd_x
    uq = A.network(layers, np.asarray(z, np.float32).astype(np.float64), round_bf16=True)
    target = separated_targets(uq, np.random.default_rng(2022))
    sp = A.out_species(mech)
    Y1 = Y.copy()
    Y1[sp, :B] += (target * sd_u + mu_u).T
    net = _mlp("c2", widths, layers, stats, max_batch=B)
    ld = T.shape[0]
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    binding.mlp_train_step(net, B, None, ld, to_dev(T), to_dev(p), to_dev(Y), to_dev(Y1), 0.0, loss)
    torch.cuda.synchronize()
    assert net.error() == 0
    g = synth.unflatten(net.get_grads(), widths)
    lo, go, sig, min_res = gradients_with_sigma(layers, z, target, uq)
    assert min_res >= 0.4 * np.sqrt(np.mean(uq ** 2))
    assert abs(float(loss[0].item()) - lo) <= 2e-2 * lo
    for l in range(4):
        for j, key in ((0, "W"), (1, "b")):
            check(g[l][j], go[l][j], sig[l][j], "layer %d d%s" % (l + 1, key))
            a, b = g[l][j].ravel(), go[l][j].ravel()
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b))
            rel = np.linalg.norm(a - b) / np.linalg.norm(b)
            assert cos >= 0.9999 and rel <= 1e-2, (l, key, cos, rel)
    net.free()


def test_adam_first_step():
    import torch
    from paper_2312_05800_gb300 import binding
    B = 256
    mech, T, p, Y, dY, widths, layers, stats = _train_case(B, seed=2023)
    net = _mlp("c2", widths, layers, stats, max_batch=B)
    ld = T.shape[0]
    p0 = net.get_params().astype(np.float64)
    lr = 1e-3
    binding.mlp_train_step(net, B, None, ld, to_dev(T), to_dev(p), to_dev(Y), to_dev(Y + dY), lr)
    torch.cuda.synchronize()
    g = net.get_grads().astype(np.float64)
    d = net.get_params().astype(np.float64) - p0
    # Adam's first step is -lr g / (|g| + eps): magnitude <= lr, sign opposite to g
    assert np.all(np.abs(d) <= lr * (1 + 1e-3) + 1e-7)
    big = np.abs(g) > 1e-6
    assert np.all(np.sign(d[big]) == -np.sign(g[big]))
    net.free()


def test_training_reduces_the_loss():
    import torch
    from paper_2312_05800_gb300 import binding
    B = 1024
    mech, T, p, Y, dY, widths, layers, stats = _train_case(B, seed=2024)
    # a learnable target: dY a smooth function of the state
    sp = A.out_species(mech)
    dY = np.zeros_like(Y)
    dY[sp, :B] = (np.sin(T[:B] / 300.0)[None, :] * stats[3][:, None] + 0.3 * Y[sp, :B] * stats[3][:, None] * 1e3)
    net = _mlp("c2", widths, layers, stats, max_batch=B)
    ld = T.shape[0]
    Td, pd, Yd, dYd = to_dev(T), to_dev(p), to_dev(Y), to_dev(Y + dY)
    loss = torch.zeros(4, dtype=torch.float32, device="cuda")
    losses = []
    for it in range(60):
        binding.mlp_train_step(net, B, None, ld, Td, pd, Yd, dYd, 3e-4, loss)
        losses.append(float(loss[0].item()))
    assert net.error() == 0
    assert losses[-1] < 0.5 * losses[0], losses[::10]
    net.free()


def test_checkpoint_resume_is_bit_identical(tmp_path):
    import torch
    from paper_2312_05800_gb300 import binding
    B = 256
    mech, T, p, Y, dY, widths, layers, stats = _train_case(B, seed=2025)
    ld = T.shape[0]
    Td, pd, Yd, dYd = to_dev(T), to_dev(p), to_dev(Y), to_dev(Y + dY)
    a = _mlp("c2", widths, layers, stats, max_batch=B)
    for _ in range(3):
        binding.mlp_train_step(a, B, None, ld, Td, pd, Yd, dYd, 1e-3)
    path = str(tmp_path / "net.bin")
    a.save(path)
    b = binding.Mlp.load(dev_mech("c2"), path)
    for _ in range(2):
        binding.mlp_train_step(a, B, None, ld, Td, pd, Yd, dYd, 1e-3)
        binding.mlp_train_step(b, B, None, ld, Td, pd, Yd, dYd, 1e-3)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    assert [np.array_equal(x, y) for x, y in zip(a.get_norm(), b.get_norm())] == [True] * 4
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 1
    open(path, "wb").write(bytes(raw))
    with pytest.raises(binding.ChemError):
        binding.Mlp.load(dev_mech("c2"), path)
    a.free()
    b.free()
