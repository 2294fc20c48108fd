"""The C oracle under AddressSanitizer and UndefinedBehaviorSanitizer: thermo, transport,
rates, the analytic Jacobian and the stiff integrator (including a non-finite state and a
one-step budget) on the 9- and 30-species mechanisms, in a child process that preloads the
ASan runtime. Any finding aborts the child."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np
import oracle as O
from paper_2312_05800_gb300 import synth
for name, n in (("c1", 37), ("c2", 21)):
    m = synth.get_mech(name)
    T, p, Y = synth.states_profiles(m, n, 5) if name == "c2" else synth.states_dirichlet(m, n, 5)
    O.props(m, T, p, Y, ncells=n)
    y = np.concatenate([[T[0]], Y[:, 0]])
    O.rates(m, T[0], p[0], Y[:, 0])
    O.rhs(m, p[0], y)
    O.jac(m, p[0], y)
    T[3] = np.nan
    T1, Y1, st, ns = O.step_stiff(m, T, p, Y, 1e-6, ncells=n, rtol=1e-6, atol_Y=1e-13, atol_T=1e-6, h0=1e-9,
                                  max_steps=2000)
    assert st[3] == 4
    O.step_stiff(m, T, p, Y, 1e-6, ncells=n, rtol=1e-9, atol_Y=1e-15, atol_T=1e-9, h0=1e-9, max_steps=1)
print("clean")
"""


def test_oracle_is_clean_under_asan_and_ubsan():
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not asan or not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("no ASan runtime for gcc here")
    import oracle
    oracle.build(sanitize=True)
    env = dict(os.environ, ORACLE_SANITIZE="1", LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0",
               PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0 and "clean" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
