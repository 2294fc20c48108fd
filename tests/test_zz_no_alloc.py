"""chem_step_stiff_noalloc: the stiff step for callers that must not allocate
device memory while they step (for example a host code that owns the whole
device budget in its own pool). Called through the C ABI, its results must
match the regular chem_step_stiff entry point within the parity tolerance of
the stiff tests, on two calls in a row (the second reuses the library's static
scratch left by the first)."""
import numpy as np
import pytest

from paper_2312_05800_gb300 import synth

pytestmark = pytest.mark.gpu
DT = 1.0e-6
OPTS = dict(rtol=1e-9, atol_Y=1e-15, atol_T=1e-9, h0=1e-9, max_steps=10000)


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_regular_entry_point_on_two_calls():
    import torch
    from paper_2312_05800_gb300 import binding
    mech = synth.mech_c1()
    n = 1001
    ld = synth.padded_ld(n)
    T, p, Y = synth.states_dirichlet(mech, n, 4242, ld)
    m = binding.Mech(mech)
    opts = binding.make_opts(**OPTS)

    def run(entry):
        Td, pd, Yd = _dev(T), _dev(p), _dev(Y)
        st = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
        ns = torch.zeros(ld, dtype=torch.int32, device="cuda")
        entry(m, n, ld, DT, opts, Td, pd, Yd, st, ns)
        torch.cuda.synchronize()
        return Td.cpu().numpy(), Yd.cpu().numpy(), st.cpu().numpy(), ns.cpu().numpy()

    Tr, Yr, sr, nr = run(binding.chem_step_stiff)
    for _ in range(2):
        Ta, Ya, sa, na = run(binding.chem_step_stiff_noalloc)
        assert np.array_equal(sa[:n], sr[:n]) and np.all(sa[:n] == 0)
        assert np.all(np.abs(Ta[:n] - Tr[:n]) <= 1e-8 * Tr[:n])
        assert np.all(np.abs(Ya[:, :n] - Yr[:, :n]) <= 1e-8 * np.abs(Yr[:, :n]) + 1e-14)
        assert np.array_equal(na[:n], nr[:n])
    # the size limit of the static scratch is reported, not run
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    s = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(binding.ChemError) as e:
        binding.chem_step_stiff_noalloc(m, (1 << 30) + 1, (1 << 30) + 4, DT, opts, x, x, x, s)
    assert "2^30" in str(e.value)
    m.free()
