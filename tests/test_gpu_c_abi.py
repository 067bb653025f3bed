"""The C ABI used from C alone: tests/c_abi/lcde_step.c, compiled with gcc against include/mmfd.h
and linked to the in-tree libmmfd.so (no Python, no PyTorch in the process), advances a D2Q9
linear CDE; its output must equal the FP64 oracle to 1e-12 and conserve mass."""
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as orc
from oracle import params as P

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_program_matches_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_17057_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "lcde_step")
    subprocess.run(["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi", "lcde_step.c"), "-o", exe,
                    "-L", os.path.dirname(lib), "-lmmfd", "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    nx, ny, steps = 300, 70, 25
    rng = np.random.default_rng(123)
    phi0 = 1.0 + 0.3 * rng.standard_normal((ny, nx))
    phi0.tofile(tmp_path / "in.bin")
    r = subprocess.run([exe, str(tmp_path / "in.bin"), str(tmp_path / "out.bin"), str(nx), str(ny), str(steps)],
                       capture_output=True, text=True, env={**os.environ, "CUDA_VISIBLE_DEVICES": "0"})
    assert r.returncode == 0, r.stderr
    words = r.stdout.split()
    assert words[1] == "k_march2d", r.stdout
    m0, m1 = float(words[3]), float(words[4])
    out = np.fromfile(tmp_path / "out.bin").reshape(ny, nx)
    prob = P.problem_lcde("D2Q9", 2, [nx, ny], 1.0, [1.0, 1.0], [[0.02, 0.005], [0.005, 0.01]], [0.1, 0.05],
                          P.two_level_from_a0(0.0))
    ref, _ = orc.run(prob, [phi0], None, nsteps=steps)
    assert np.abs(out - ref[0]).max() < 1e-12 * np.abs(ref[0]).max()
    assert abs(m1 - m0) < 1e-12 * np.abs(phi0).sum()
