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
    m.free()


def test_noalloc_leaves_device_memory_unchanged():
    # The device's free memory (cudaMemGetInfo through torch) is the same before and after the
    # first and second calls on a freshly loaded mechanism handle. The regular entry point runs
    # first so that loading the library's kernels and sizing their stack happen before the
    # measurement; every tensor the calls use exists before it.
    import torch
    from paper_2312_05800_gb300 import binding
    mech = synth.mech_c1()
    n = 515
    ld = synth.padded_ld(n)
    T, p, Y = synth.states_dirichlet(mech, n, 4243, ld)
    opts = binding.make_opts(**OPTS)
    warm = binding.Mech(mech)
    Td, pd, Yd = _dev(T), _dev(p), _dev(Y)
    st = torch.zeros(ld, dtype=torch.int32, device="cuda")
    binding.chem_step_stiff(warm, n, ld, DT, opts, Td, pd, Yd, st)
    torch.cuda.synchronize()
    warm.free()
    fresh = binding.Mech(mech)
    ins = [(_dev(T), _dev(Y)) for _ in range(2)]
    outs = [torch.full((ld,), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    for (Ti, Yi), si in zip(ins, outs):
        free0 = torch.cuda.mem_get_info()[0]
        binding.chem_step_stiff_noalloc(fresh, n, ld, DT, opts, Ti, pd, Yi, si)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert bool((si[:n] == 0).all())
    fresh.free()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2312_05800_gb300 import binding
    m = binding.Mech(synth.mech_c1())
    opts = binding.make_opts(**OPTS)
    # the size limit of the static scratch is reported, not run
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    s = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(binding.ChemError) as e:
        binding.chem_step_stiff_noalloc(m, (1 << 30) + 1, (1 << 30) + 4, DT, opts, x, x, x, s)
    assert "2^30" in str(e.value)
    m.free()
