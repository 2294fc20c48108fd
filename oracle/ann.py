"""FP64 oracle of the learned step (TEST INFRASTRUCTURE ONLY), Sec. 3.2.

prologue -> network -> epilogue, written out plainly:
  x = (T, p, F(Y)),  z = (x - mu_x) / sd_x            (Box-Cox and Z-score, Sec. 3.2)
  u = network(z)                                       (GELU hidden layers)
  dY_k = sd_u u_k + mu_u  for the non-bath species      (u* = Y(t+dt) - Y(t), Sec. 3.2)
  dY_bath = -sum_k dY_k                                 (mass conservation)
  Y' = max(Y + dY, 0) / sum(max(Y + dY, 0))
  T' : h(T', Y') = h(T, Y)  (adiabatic, constant p), Newton to |dT| < 1e-10 K.
round_bf16 rounds the operands at the points where the GPU stores BF16 (the
weights and each hidden activation; the network input, formed in FP32, as the
sum of two BF16 terms hi + lo, and the first layer's weights likewise, with the
product taken as z_hi W_hi + z_lo W_hi + z_hi W_lo); accumulation stays FP64.
"""
from __future__ import annotations

import numpy as np

from . import mlp as M


def to_bf16(x):
    """Round-to-nearest-even to BF16 (returned as float64)."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


# FP8 E4M3 (the "fn" variant: 4 exponent bits, bias 7, 3 mantissa bits, no
# infinities, one NaN pattern per sign): finite values are 0, m 2^-9 (m = 1..7,
# subnormal) and (1 + m/8) 2^e (e = -6..8, m = 0..7, except m = 7 at e = 8),
# the largest 448.
E4M3_MAX = 448.0


def e4m3_decode(codes):
    """Values of E4M3 codes (uint8) from the format definition; NaN for 0x7f / 0xff."""
    c = np.asarray(codes, np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    m = c & 0x7
    mag = np.where(e == 0, m * 2.0 ** -9, (1.0 + m / 8.0) * 2.0 ** (e - 7.0))
    mag = np.where((e == 0xF) & (m == 7), np.nan, mag)
    return sign * mag


def to_e4m3(x):
    """Round to the nearest E4M3 value, ties to even, saturating at +-448 (also for
    infinities); NaN stays NaN. Returned as float64."""
    x = np.asarray(x, np.float64)
    a = np.abs(x)
    _, ex = np.frexp(np.where(np.isfinite(a) & (a > 0), a, 1.0))
    e = np.maximum(ex.astype(np.float64) - 1.0, -6.0)   # floor(log2 a); below 2^-6 the spacing is 2^-9
    q = 2.0 ** (e - 3.0)
    r = np.rint(a / q) * q               # np.rint rounds halves to even; a / q is exact
    r = np.minimum(r, E4M3_MAX)
    r = np.where(np.isnan(x), np.nan, r)
    return np.copysign(r, x)


def quantize_rows(W):
    """Per output row: sw = fl32(max |W| / 448) (1 for a zero row) and the E4M3
    values of fl32(W / sw). W holds FP32 values."""
    W = np.asarray(W, np.float64)
    amax = np.abs(W).max(axis=1)
    sw = np.where(amax > 0, (amax / E4M3_MAX).astype(np.float32).astype(np.float64), 1.0)
    Wq = to_e4m3((W / sw[:, None]).astype(np.float32).astype(np.float64))
    return Wq, sw


def calibrate_fp8(layers, z):
    """E4M3 activation scales s_i = fl32(max |h_i| / 448) of the BF16 forward's h1, h2."""
    h = split_bf16(z)
    s = []
    for i, (W, b) in enumerate(layers[:2]):
        if i == 0:
            Wh = to_bf16(W)
            pre = h @ Wh.T + to_bf16(h) @ to_bf16(W - Wh).T + b
        else:
            pre = h @ to_bf16(W).T + b
        h = to_bf16(M.gelu(pre))
        s.append(float(np.float32(np.abs(h).max() / E4M3_MAX)))
    return s


def split_bf16(z):
    """z (FP32 values) as the sum of two BF16 terms: hi = bf16(z), lo = bf16(z - hi)."""
    z = np.asarray(z, np.float64)
    hi = to_bf16(z)
    return hi + to_bf16(z - hi)


def out_species(mech):
    return [k for k in range(mech.N) if k != mech.bath]


def network(layers, z, round_bf16=False, fp8_scales=None):
    """The MLP on normalised inputs z [n, n_in]. round_bf16: BF16 operands as
    stored by the device. fp8_scales = (s_1, s_2): additionally the two
    hidden-to-hidden layers take E4M3 operands, h_q = E4M3(h / s) and the weights
    of quantize_rows, with z = (h_q . Wq) fl32(sw s) + b (accumulation exact)."""
    h = np.asarray(z, np.float64)
    if round_bf16 or fp8_scales is not None:
        h = split_bf16(h)
    nl = len(layers)
    for i, (W, b) in enumerate(layers):
        if fp8_scales is not None and i in (1, 2):
            Wq, sw = quantize_rows(W)
            cs = (sw * np.float64(np.float32(fp8_scales[i - 1]))).astype(np.float32).astype(np.float64)
            pre = (h @ Wq.T) * cs + b
        elif i == 0 and (round_bf16 or fp8_scales is not None):
            Wh = to_bf16(W)
            pre = h @ Wh.T + to_bf16(h) @ to_bf16(W - Wh).T + b
        else:
            Wq = to_bf16(W) if (round_bf16 or fp8_scales is not None) else W
            pre = h @ Wq.T + b
        if i < nl - 1:
            h = M.gelu(pre)
            if fp8_scales is not None and i in (0, 1):
                h = to_e4m3(h / np.float64(np.float32(fp8_scales[i])))
            elif round_bf16 or fp8_scales is not None:
                h = to_bf16(h)
        else:
            h = pre
    return h


def network_ensemble(nets, z, round_bf16=False):
    """The per-species model of Sec. 3.2 (each species mass fraction has a network of its own):
    nets[g] holds the (W, b) layers of output g's network (widths n_in -> h1 -> h2 -> h3 -> 1), all
    reading the same input z. Column g of the result is network g's output."""
    return np.concatenate([network(layers, z, round_bf16) for layers in nets], axis=1)


def forward_u(mech, layers, stats, T, p, Y, round_bf16=False, fp8_scales=None, ensemble=False):
    """ensemble: layers is a list of per-output networks (network_ensemble)."""
    mu_x, sd_x, mu_u, sd_u = stats
    x = M.features(T, p, Y)
    z = (x - mu_x) / sd_x
    if round_bf16 or fp8_scales is not None:
        # the device forms z in FP32
        z = np.asarray(z, np.float32).astype(np.float64)
    if ensemble:
        if fp8_scales is not None:
            raise ValueError("the per-species ensemble has no E4M3 variant")
        return network_ensemble(layers, z, round_bf16)
    return network(layers, z, round_bf16, fp8_scales)


def step_ann(mech, layers, stats, T, p, Y, round_bf16=False, fp8_scales=None, ensemble=False):
    """Returns (T', Y') for SoA inputs T[n], p[n], Y[N, n]."""
    import oracle as O
    mu_x, sd_x, mu_u, sd_u = stats
    u = forward_u(mech, layers, stats, T, p, Y, round_bf16, fp8_scales, ensemble)
    dY = u * sd_u + mu_u
    Yn = np.array(Y, dtype=np.float64)
    sp = out_species(mech)
    Yn[sp, :] += dY.T
    Yn[mech.bath, :] -= dY.sum(axis=1)
    Yn = np.maximum(Yn, 0.0)
    Yn /= Yn.sum(axis=0, keepdims=True)
    n = T.shape[0]
    h0 = O.props(mech, T, p, Y)[1]
    Tn = np.array(T, dtype=np.float64)
    for _ in range(50):
        cp, h, *_ = O.props(mech, Tn, p, Yn)
        d = (h - h0) / cp
        Tn = Tn - d
        if np.all(np.abs(d[:n]) < 1e-10):
            break
    return Tn, Yn


# ---------------------------------------------------------------------------
# out-of-distribution test (not in the paper): occupancy grid over (T, h/R, Y_s)
# ---------------------------------------------------------------------------

def ood_features(mech, T, p, Y, species):
    """(T, h/R, Y_species) per cell, FP64; h is the NASA-7 mixture enthalpy (J/kg)."""
    import oracle as O
    from paper_2312_05800_gb300 import synth
    n = T.shape[0]
    h = O.props(mech, T, p, Y)[1]
    return np.stack([np.asarray(T, np.float64), h / synth.R_GAS, np.asarray(Y[species], np.float64)], axis=1)[:n]


def ood_fit(features, nbins=64, kmin=4, margin=0.05):
    """Grid over the training range +/- margin; mask[i, j, k] = the 3x3x3 block
    around bin (i, j, k) holds at least kmin training samples."""
    lo = features.min(axis=0)
    hi = features.max(axis=0)
    w = hi - lo
    lo, hi = lo - margin * w, hi + margin * w
    b = np.floor((features - lo) / (hi - lo) * nbins).astype(np.int64)
    counts = np.zeros((nbins,) * 3, np.int64)
    np.add.at(counts, (b[:, 0], b[:, 1], b[:, 2]), 1)
    padded = np.pad(counts, 1)
    nb = nbins
    block = sum(padded[1 + a:1 + a + nb, 1 + c:1 + c + nb, 1 + d:1 + d + nb]
                for a in (-1, 0, 1) for c in (-1, 0, 1) for d in (-1, 0, 1))
    return {"lo": lo, "hi": hi, "nbins": nbins, "mask": block >= kmin, "counts": counts}


def ood_flags(fit, features):
    """True where a cell is outside the training distribution."""
    nb = fit["nbins"]
    u = (features - fit["lo"]) / (fit["hi"] - fit["lo"]) * nb
    outside = ~np.all((u >= 0) & (u < nb), axis=1)
    b = np.clip(np.floor(u).astype(np.int64), 0, nb - 1)
    return outside | ~fit["mask"][b[:, 0], b[:, 1], b[:, 2]]


def ood_flags_multi(fits, features):
    """Several grids (one per feature species): a cell is outside if any grid puts it outside."""
    out = np.zeros(features[0].shape[0], bool)
    for fit, f in zip(fits, features):
        out |= ood_flags(fit, f)
    return out
