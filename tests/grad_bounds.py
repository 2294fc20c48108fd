"""Per-element error bounds of the device's training gradients against the FP64
oracle's backward pass (oracle/mlp.py), from the rounding points of the device's
arithmetic (test helper).

The device forward and backward round at these points, each a relative error of
at most 2^-9 (BF16, round to nearest), and otherwise accumulate in FP32, whose
error over K <= 2048 terms (about K 2^-24 relative) is far below one BF16
rounding:
  forward   W -> bf16(W), the first layer's W as two BF16 terms (16 significant
            bits); h_l = bf16(GELU(pre_l)); pre_l in FP32; the network input as
            two BF16 terms (16 significant bits);
  backward  dL/du = sign(u - u*)/B exactly; dX = g bf16(W); g_{l-1} =
            bf16(dX GELU'(pre_{l-1})) with the device's own FP32 pre-activation;
            dW = g^T h with the stored BF16 h (the first layer: the input's hi
            term only); db = column sums of g.
The roundings are independent, so their effect on a sum of K products grows
like sqrt(K), not K (probabilistic rounding-error analysis, as in Higham and
Mary 2019). The helper propagates standard deviations s (each rounding taken
as s = 2^-9 |value|, above the 2^-9 |value| / sqrt 3 of a uniform error) with
squares, through the FP64 values of the oracle:
  s_pre(l)^2 = s_h(l-1)^2 (W_l^2)^T + r_W (h_{l-1}^2)(W_l^2)^T   (r_W = 2^-18; 2^-32 for l = 1)
  s_h(l)^2   = GELU'(pre_l)^2 s_pre(l)^2 + 2^-18 h_l^2
  s_dX^2     = s_g^2 W^2 + 2^-18 g^2 W^2
  s_g(l-1)^2 = s_dX^2 GELU'^2 + dX^2 GELU''(pre)^2 s_pre^2 + 2^-18 g_{l-1}^2
  s_dW^2     = (s_g^2)^T h^2 + (g^2)^T s_h^2 + 2^-18 (g^2)^T h^2
  s_db^2     = sum over rows of s_g^2
and a test accepts |device - oracle| <= k s per element. The L1 subgradient's
sign is exact on both sides only if no residual u - u* is within the forward's
error of zero; the tests choose targets whose residuals are bounded away from it.
"""
import numpy as np

from oracle import mlp as M

R2 = 2.0 ** -18     # (one BF16 rounding)^2


def gelu_grad2(z):
    """d^2 GELU / dz^2 = phi(z) (2 - z^2)."""
    return np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi) * (2.0 - z * z)


def gradients_with_sigma(layers, z, target, sign_from, dout=None):
    """FP64 gradients of Eq. 5 for one network (layers: [(W [out, in], b)], inputs z [B, n_in],
    targets [B, n_out]), the L1 sign taken on sign_from, and the standard deviations above.
    dout (optional, [B, n_out]): dL/du of another loss (the physics terms), which the device
    stores as BF16 (one rounding, s = 2^-9 |dout|). Returns (loss, grads, sigmas,
    min |sign_from - target|) with grads and sigmas as [(dW, db)]; loss is Eq. 5's."""
    z = np.asarray(z, np.float64)
    Bn = z.shape[0]
    nl = len(layers)
    hs, vhs, pres, vpres = [z], [R2 * z * z], [], []
    h = z
    vh = 2.0 ** -32 * z * z             # the forward's hi + lo input
    for i, (W, b) in enumerate(layers):
        W2 = W * W
        pre = h @ W.T + b
        vpre = vh @ W2.T + (R2 if i > 0 else 2.0 ** -32) * ((h * h) @ W2.T)
        pres.append(pre)
        vpres.append(vpre)
        if i < nl - 1:
            h = M.gelu(pre)
            vh = M.gelu_grad(pre) ** 2 * vpre + R2 * h * h
            hs.append(h)
            vhs.append(vh)
    u = pres[-1]
    res = np.asarray(sign_from, np.float64) - target
    loss = float(np.abs(u - target).sum() / Bn)
    if dout is None:
        g = np.sign(res) / Bn
        vg = np.zeros_like(g)
    else:
        g = np.asarray(dout, np.float64)
        vg = R2 * g * g
    grads, sig = [None] * nl, [None] * nl
    for i in range(nl - 1, -1, -1):
        W = layers[i][0]
        W2 = W * W
        hin, vhin = hs[i], vhs[i]
        g2 = g * g
        grads[i] = (g.T @ hin, g.sum(axis=0))
        sig[i] = (np.sqrt(vg.T @ (hin * hin) + g2.T @ vhin + R2 * (g2.T @ (hin * hin))),
                  np.sqrt(vg.sum(axis=0) + 1e-12 * g2.sum(axis=0)))
        if i > 0:
            dX = g @ W
            vdX = vg @ W2 + R2 * (g2 @ W2)
            gp = M.gelu_grad(pres[i - 1])
            gn = dX * gp
            vg = vdX * gp * gp + dX * dX * gelu_grad2(pres[i - 1]) ** 2 * vpres[i - 1] + R2 * gn * gn
            g = gn
    return loss, grads, sig, float(np.abs(res).min())


def check(gpu, ref, sigma, what, k=8.0):
    """|gpu - ref| <= k sigma + 1e-12 max|ref| element by element; returns max |gpu - ref| / (k sigma)."""
    gpu = np.asarray(gpu, np.float64)
    err = np.abs(gpu - ref)
    lim = k * sigma + 1e-12 * np.abs(ref).max()
    if not np.all(err <= lim):
        idx = np.unravel_index(np.argmax(err / lim), err.shape)
        raise AssertionError("%s: %d of %d elements outside %g sigma; worst %s: gpu %.6g oracle %.6g sigma %.3g"
                             % (what, int((err > lim).sum()), err.size, k, idx, gpu[idx], ref[idx], sigma[idx]))
    return float((err / lim).max())


def separated_targets(uq, rng, margin=0.5):
    """Targets u* = uq - s (margin + |xi|) rms(uq) with random signs s: every residual uq - u* is
    at least margin rms(uq) from zero, far outside the forward's rounding errors, so both sides
    take the same L1 sign."""
    rms = np.sqrt(np.mean(uq ** 2))
    s = rng.choice([-1.0, 1.0], size=uq.shape)
    return uq - s * (margin + np.abs(rng.normal(size=uq.shape))) * rms
