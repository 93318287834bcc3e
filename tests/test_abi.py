"""The C-ABI library loads and exports every entry point that include/lift.h
declares; argument and spec validation happens before any CUDA call, so it is
checked here without a GPU."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lift.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lift_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1512_01383_gb300 import lift as G
    if not os.path.exists(G.LIB_PATH):
        from paper_1512_01383_gb300 import build
        build.build()
    return G


def test_header_declares_the_binding(lib):
    assert declared_functions() == sorted(lib.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    syms = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in declared_functions():
        assert name in syms, name
    raw = C.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(raw, name)


def test_strerror_names_every_code(lib):
    codes = [lib.LIFT_OK, lib.LIFT_ERR_SPEC, lib.LIFT_ERR_OOM, lib.LIFT_ERR_CUDA,
             lib.LIFT_ERR_NAN, lib.LIFT_ERR_NOT_CONVERGED, lib.LIFT_ERR_ARG]
    names = {lib.strerror(c) for c in codes}
    assert len(names) == len(codes)
    assert "unknown" in lib.strerror(99)


def _spec(lib, **kw):
    f = np.zeros(12, np.float32)
    d = dict(kind=lib.LIFT_TRUNC_QUAD, H=3, W=4, L=5, gamma_min=0.0, gamma_max=1.0, lam=0.25,
             alpha=25.0, nu=0.1, f=f)
    d.update(kw)
    keep = d.pop("f")
    s = lib.make_spec(d.pop("kind"), d.pop("H"), d.pop("W"), d.pop("L"), d.pop("gamma_min"),
                      d.pop("gamma_max"), d.pop("lam"), d.pop("alpha"), d.pop("nu"), f=keep, **d)
    return s, keep


@pytest.mark.parametrize("bad", [
    dict(kind=7), dict(H=0), dict(W=-1), dict(L=1), dict(L=66), dict(gamma_max=0.0),
    dict(lam=-1.0), dict(alpha=0.0), dict(nu=0.0), dict(lam=float("nan")),
    dict(alpha=float("inf")), dict(f=None), dict(depth=-1),
    dict(H=4096, W=4096, L=65, depth=2),          # N*k beyond 2^31
])
def test_invalid_spec_rejected_before_any_cuda_call(lib, bad):
    s, keep = _spec(lib, **bad)
    h = C.c_void_p()
    rc = lib.load().lift_create(C.byref(s), None, C.byref(h))
    assert rc == lib.LIFT_ERR_SPEC and not h.value


def test_pl_spec_must_cover_the_label_range(lib):
    cost = np.zeros((2, 2, 9), np.float32)
    s = lib.make_spec(lib.LIFT_PL_SAMPLED, 2, 2, 3, 0.0, 8.0, 0.1, cost=cost, sample_min=0.0,
                      sample_max=6.0)
    h = C.c_void_p()
    assert lib.load().lift_create(C.byref(s), None, C.byref(h)) == lib.LIFT_ERR_SPEC
    one = np.ascontiguousarray(cost[..., :1])
    s = lib.make_spec(lib.LIFT_PL_SAMPLED, 2, 2, 3, 0.0, 8.0, 0.1, cost=one,
                      sample_min=0.0, sample_max=8.0)
    assert lib.load().lift_create(C.byref(s), None, C.byref(h)) == lib.LIFT_ERR_SPEC


def test_null_arguments(lib):
    L = lib.load()
    assert L.lift_create(None, None, None) == lib.LIFT_ERR_ARG
    assert L.lift_iterate(None, 3) == lib.LIFT_ERR_ARG
    assert L.lift_energy(None, None, None, None) == lib.LIFT_ERR_ARG
    assert L.lift_unlift(None, None, 0) == lib.LIFT_ERR_ARG
    assert L.lift_state_bytes(None) == 0
    L.lift_destroy(None)
    assert L.lift_create_batch(None, 0, None, None) == lib.LIFT_ERR_ARG
    assert L.lift_batch_iterate(None, 3) == lib.LIFT_ERR_ARG
    assert L.lift_batch_set_schedule(None, 256, 0) == lib.LIFT_ERR_ARG
    assert L.lift_batch_schedule(None, None, None, None) == lib.LIFT_ERR_ARG
    assert L.lift_batch_size(None) == 0
    L.lift_batch_destroy(None)
    assert L.lift_set_bands(None, 0, None) == lib.LIFT_ERR_ARG
    assert L.lift_set_resident(None, 1, None) == lib.LIFT_ERR_ARG
    assert L.lift_average(None, 1) == lib.LIFT_ERR_ARG
    assert L.lift_average_count(None) == -1
    assert L.lift_energy_average(None, None, None, None) == lib.LIFT_ERR_ARG
    assert L.lift_unlift_average(None, None, 0) == lib.LIFT_ERR_ARG
    assert L.lift_average_restart(None) == lib.LIFT_ERR_ARG
    assert L.lift_solve_averaged(None, 10, 1e-3, 10, 1, None, None) == lib.LIFT_ERR_ARG


def test_volume_batch_rejected_before_any_cuda_call(lib):
    s, keep = _spec(lib, depth=2)
    arr = (lib.lift_spec * 1)(s)
    b = C.c_void_p()
    assert lib.load().lift_create_batch(arr, 1, None, C.byref(b)) == lib.LIFT_ERR_SPEC
    assert not b.value
