"""chem_step_stiff on the GPU against the FP64 oracle (Sec. 3.1: integration
of the reaction ODEs over dt = 1 us; Sec. 4.2: the direct-integration baseline).

Both sides run the same Rodas3 algorithm with the same controller; at the
parity tolerances (rtol 1e-9) the results agree within 1e-8 relative on Y and T
(|dY| <= 1e-8 |Y| + 1e-14). Sizes span several blocks and a ragged tail; the
full 2M-cell workload is checked on sampled cells.
"""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu
DT = 1.0e-6
PARITY = dict(rtol=1e-9, atol_Y=1e-15, atol_T=1e-9, h0=1e-9, max_steps=10000)


def _gpu(name, T, p, Y, n, ld, **opts):
    import torch
    from paper_2312_05800_gb300 import binding
    m = dev_mech(name)
    Td, pd, Yd = to_dev(T), to_dev(p), to_dev(Y)
    st = torch.full((ld,), -7, dtype=torch.int32, device="cuda")
    ns = torch.zeros(ld, dtype=torch.int32, device="cuda")
    binding.chem_step_stiff(m, n, ld, DT, binding.make_opts(**opts), Td, pd, Yd, st, ns)
    torch.cuda.synchronize()
    return Td.cpu().numpy(), Yd.cpu().numpy(), st.cpu().numpy(), ns.cpu().numpy()


def _check(name, T, p, Y, n, ld, rel=1e-8, absY=1e-14, **opts):
    import oracle as O
    mech = synth.get_mech(name)
    Tg, Yg, sg, ng = _gpu(name, T, p, Y, n, ld, **opts)
    To, Yo, so, no = O.step_stiff(mech, T, p, Y, DT, ncells=n, **opts)
    assert np.array_equal(sg[:n], so[:n])
    ok = sg[:n] == 0
    assert np.all(np.abs(Tg[:n] - To[:n])[ok] <= rel * To[:n][ok])
    assert np.all((np.abs(Yg[:, :n] - Yo[:, :n]) <= rel * np.abs(Yo[:, :n]) + absY)[:, ok])
    return sg, ng, no


def test_c1_full_parity(oracle):
    m = synth.mech_c1()
    T, p, Y = synth.states_dirichlet(m, 4096, 2001)
    sg, ng, no = _check("c1", T, p, Y, 4096, 4096, **PARITY)
    assert np.all(sg == 0)
    # identical step sequences in the vast majority of cells
    assert np.mean(ng == no) > 0.9


def test_c2_subset_ragged(oracle):
    m = synth.mech_c2()
    n = 203
    ld = 212
    T, p, Y = synth.states_profiles(m, n, 2002, ld)
    _check("c2", T, p, Y, n, ld, **PARITY)


def test_c5_subset(oracle):
    m = synth.mech_c5()
    n = 37
    T, p, Y = synth.states_profiles(m, n, 2005)
    _check("c5", T, p, Y, n, synth.padded_ld(n), **PARITY)


def test_status_codes_and_edges(oracle):
    import torch
    from paper_2312_05800_gb300 import binding
    m = synth.mech_c1()
    T, p, Y = synth.states_dirichlet(m, 64, 3)
    T[5] = np.nan
    Tg, Yg, sg, ng = _gpu("c1", T, p, Y, 64, 64, **dict(PARITY, max_steps=1))
    assert sg[5] == binding.CELL_NONFINITE
    assert np.all(sg[np.arange(64) != 5] == binding.CELL_MAXSTEPS) and np.all(ng[np.arange(64) != 5] == 1)
    # zero cells is a no-op; bad sizes are rejected
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    s = torch.zeros(8, dtype=torch.int32, device="cuda")
    binding.chem_step_stiff(dev_mech("c1"), 0, 8, DT, None, x, x, torch.zeros(9, 8, dtype=torch.float64,
                                                                              device="cuda"), s)
    with pytest.raises(binding.ChemError):
        binding.chem_step_stiff(dev_mech("c1"), 8, 6, DT, None, x, x, x, s)


def test_full_size_sampled(oracle):
    # 2,097,152 cells at the bench's throughput setting; sampled cells vs the oracle
    m = synth.mech_c2()
    n = 2097152
    T, p, Y = synth.states_profiles(m, n, 2002)
    rtol = 1e-2
    opts = dict(rtol=rtol, atol_Y=1e-8, atol_T=1e-2, h0=1e-9, max_steps=10000)
    Tg, Yg, sg, ng = _gpu("c2", T, p, Y, n, n, **opts)
    assert np.all(sg == 0)
    import oracle as O
    idx = np.concatenate([np.random.default_rng(1).choice(n, 96, replace=False), [0, n - 1]])
    To, Yo, so, no = O.step_stiff(m, T[idx].copy(), p[idx].copy(), Y[:, idx].copy(), DT, **opts)
    # same algorithm: where the accept/reject decisions agree the results agree to round-off;
    # a rare differing decision moves the result by about the tolerance
    assert np.all(np.abs(Tg[idx] - To) <= rtol * To)
    assert np.all(np.abs(Yg[:, idx] - Yo) <= rtol * np.abs(Yo) + 1e-6)
    same = ng[idx] == no
    assert np.mean(same) > 0.8
    close = (np.abs(Tg[idx] - To) <= 1e-6 * To) & np.all(np.abs(Yg[:, idx] - Yo) <= 1e-6 * np.abs(Yo) + 1e-12, axis=0)
    assert np.mean(close[same]) > 0.9


@pytest.mark.parametrize("name", ["c2", "c5"])
def test_team_mode_is_bitwise_warp_mode(name):
    # up to one cell per SM, a team of warps integrates each cell; the results are bitwise those
    # of one warp per cell (the same operations in the same order), for every status and step count
    m = synth.get_mech(name)
    n_big = 2000
    T, p, Y = synth.states_profiles(m, n_big, 31, synth.padded_ld(n_big))
    for opts in (PARITY, dict(rtol=1e-2, atol_Y=1e-8, atol_T=1e-2, h0=1e-9, max_steps=10000),
                 dict(rtol=1e-6, atol_Y=1e-12, atol_T=1e-6, h0=1e-9, max_steps=3)):
        Tw, Yw, sw, nw = _gpu(name, T, p, Y, n_big, T.shape[0], **opts)        # warps
        n = 100
        Tt, Yt, st, nt = _gpu(name, T, p, Y, n, T.shape[0], **opts)            # teams
        assert np.array_equal(st[:n], sw[:n]) and np.array_equal(nt[:n], nw[:n])
        assert np.array_equal(Tt[:n], Tw[:n]) and np.array_equal(Yt[:, :n], Yw[:, :n])
        assert np.array_equal(Tt[n:], T[n:])                                   # cells past n untouched
