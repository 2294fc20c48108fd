"""What the learned part gains (Sec. 3.2's a-priori test on a fresh random
data set): a network trained on the GPU with the library's own forward,
backward and Adam kernels, on pairs the GPU stiff integrator generated, is
compared on held-out cells with the FP64 oracle's tight integration, against
the methods without it: no chemistry (dY = 0) and one explicit Euler step with
the oracle's source terms at t."""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth

pytestmark = pytest.mark.gpu


def test_trained_network_beats_the_methods_without_it(oracle):
    import torch
    from paper_2312_05800_gb300 import binding, train
    from tests.gpu_util import dev_mech
    m = synth.mech_c2()
    dm = dev_mech("c2")
    data = train.make_training_set(dm, m, 131072, seed=2103)
    net = binding.Mlp(dm, hidden=(1600, 800, 400), dt=1e-6, seed=3003, chunk=65536, max_batch=4096)
    train.fit_norm(net, data)
    hist = train.train(net, data, epochs=24, batch=4096, lr0=1e-3)
    assert hist[-1] < 0.25 * hist[0]
    # held-out cells, a fresh seed of the same distribution
    n = 384
    T, p, Y = synth.states_profiles(m, n, 2003)
    ld = T.shape[0]
    Td, pd, Yd = (torch.from_numpy(a).cuda() for a in (T, p, Y))
    binding.chem_step_ann(dm, net, n, ld, 1e-6, binding.CHEM_PREC_BF16, None, Td, pd, Yd)
    torch.cuda.synchronize()
    Ta, Ya = Td.cpu().numpy()[:n], Yd.cpu().numpy()[:, :n]
    Tr, Yr, st, _ = oracle.step_stiff(m, T, p, Y, 1e-6, ncells=n, rtol=1e-7, atol_Y=1e-14, atol_T=1e-7,
                                      max_steps=50000)
    assert np.all(st[:n] == 0)
    dr = Yr[:, :n] - Y[:, :n]
    # explicit Euler with the oracle's right-hand side at t
    de = np.zeros_like(dr)
    for i in range(n):
        f = oracle.rhs(m, p[i], np.concatenate([[T[i]], Y[:, i]]))
        de[:, i] = 1e-6 * f[1:]
    major = [k for k in range(m.N) if k != m.bath and Y[k, :n].mean() >= 1e-2]
    for k in major:
        ref = np.linalg.norm(dr[k])
        e_ann = np.linalg.norm((Ya[k] - Y[k, :n]) - dr[k]) / ref
        e_euler = np.linalg.norm(de[k] - dr[k]) / ref
        assert e_ann < 0.1, (k, e_ann)          # dY = 0 has relative error 1 by definition
        assert e_ann < e_euler, (k, e_ann, e_euler)
    assert np.abs(Ta - Tr[:n]).max() < 2.0
    net.free()
