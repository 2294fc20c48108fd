"""Pins of the oracle's out-of-distribution grid (no counterpart in the paper):
every training state is in the distribution, a state far outside the
training range is not, the mask follows its 3x3x3 definition on a hand-built
sample, and on the perturbed workload it flags most moved cells and few others."""
import numpy as np

from oracle import ann as A
from paper_2312_05800_gb300 import synth


def test_training_states_are_in_distribution(oracle):
    m = synth.mech_c2()
    T, p, Y = synth.states_profiles(m, 20000, 5)
    F = A.ood_features(m, T[:20000], p[:20000], Y[:, :20000], m.roles["water"])
    fit = A.ood_fit(F, nbins=32, kmin=1)
    assert not A.ood_flags(fit, F).any()
    far = F[:3].copy()
    far[:, 0] += 10 * (fit["hi"][0] - fit["lo"][0])
    assert A.ood_flags(fit, far).all()


def test_mask_definition_on_a_hand_built_sample():
    # 5 samples in the corner bin (0, 0, 0), 1 in bin (9, 9, 9) (range [-0.05, 1.05], 10 bins):
    # with kmin 5 only the 2 x 2 x 2 bins whose 3x3x3 block reaches the corner are in
    F = np.array([[0.0, 0.0, 0.0]] * 5 + [[1.0, 1.0, 1.0]])
    fit = A.ood_fit(F, nbins=10, kmin=5)
    m = fit["mask"]
    assert fit["counts"][0, 0, 0] == 5 and fit["counts"][9, 9, 9] == 1
    assert m[0, 0, 0] and m[1, 1, 1] and not m[2, 0, 0] and m.sum() == 8


def test_perturbed_cells_are_flagged(oracle):
    m = synth.mech_c2()
    ntr, ne = 100000, 40000
    T, p, Y = synth.states_profiles(m, ntr, 2103)
    F = A.ood_features(m, T[:ntr], p[:ntr], Y[:, :ntr], m.roles["water"])
    fit = A.ood_fit(F)
    Te, pe, Ye = synth.states_profiles(m, ne, 2003)
    T2, Y2, moved = synth.perturb_off_manifold(Te, Ye, ne, 0.02, 2004)
    flags = A.ood_flags(fit, A.ood_features(m, T2[:ne], pe[:ne], Y2[:, :ne], m.roles["water"]))
    assert flags[moved[:ne]].mean() > 0.7
    assert flags[~moved[:ne]].mean() < 0.01


def test_two_grids_flag_the_union(oracle):
    # a cell is outside two grids' distribution when either grid puts it outside: the flags are
    # the union, so recall never drops and the false positives stay within the sum of both
    m = synth.mech_c2()
    ntr, ne = 100000, 40000
    T, p, Y = synth.states_profiles(m, ntr, 2103)
    Te, pe, Ye = synth.states_profiles(m, ne, 2003)
    T2, Y2, moved = synth.perturb_off_manifold(Te, Ye, ne, 0.02, 2004)
    fits, feats = [], []
    for sp in (m.roles["oxidizer"], m.roles["water"]):
        fits.append(A.ood_fit(A.ood_features(m, T[:ntr], p[:ntr], Y[:, :ntr], sp)))
        feats.append(A.ood_features(m, T2[:ne], pe[:ne], Y2[:, :ne], sp))
    single = [A.ood_flags(f, x) for f, x in zip(fits, feats)]
    both = A.ood_flags_multi(fits, feats)
    assert np.array_equal(both, single[0] | single[1])
    mv = moved[:ne]
    assert both[mv].mean() >= max(s[mv].mean() for s in single)
    assert both[~mv].mean() <= single[0][~mv].mean() + single[1][~mv].mean()
