"""The C ABI from plain C: tests/c_example/solve_rof.c compiles against
include/lift.h alone (C99, warnings as errors) and links the library; on a
GPU it runs and matches the oracle."""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1512_01383_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_example", "solve_rof.c")


def _build(tmp_path):
    from paper_1512_01383_gb300 import lift as G
    if not os.path.exists(G.LIB_PATH):
        from paper_1512_01383_gb300 import build
        build.build()
    libdir = os.path.dirname(G.LIB_PATH)
    exe = str(tmp_path / "solve_rof")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-O2",
                    "-I", os.path.join(ROOT, "include"), SRC, "-o", exe,
                    "-L", libdir, "-l:" + os.path.basename(G.LIB_PATH),
                    "-Wl,-rpath," + libdir], check=True)
    return exe


def test_c_program_compiles_and_links(tmp_path):
    assert os.access(_build(tmp_path), os.X_OK)


@pytest.mark.gpu
def test_c_program_matches_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    exe = _build(tmp_path)
    H, W, iters = 37, 41, 300
    f = synth.as_f32(synth.gaussian_blobs(H, W, 2600))
    fp, up = tmp_path / "f.raw", tmp_path / "u.raw"
    f.tofile(fp)
    out = subprocess.run([exe, str(fp), str(up), str(H), str(W), str(iters)], check=True,
                         capture_output=True, text=True).stdout.split()
    Pg, Dg, Eg = (float(v) for v in out)
    u = np.fromfile(up, dtype=np.float32)
    P = O.Problem(O.QUAD, H, W, 2, 0.0, 1.0, lam=0.2, alpha=1.0, f=f.astype(np.float64))
    X = O.State(P)
    O.pdhg(P, X, iters)
    assert np.abs(u - O.unlift(P, X.u)).max() <= 1e-4
    for g, o in zip((Pg, Dg, Eg), O.energy(P, X)):
        assert abs(g - o) <= 1e-5 * max(abs(o), 1.0), (g, o)
