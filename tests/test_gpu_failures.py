"""Failure detection on the GPU, without faulting, trapping or hanging it.

* A bounded device wait that runs out: block 1 of a strip skips its first barrier arrival (test
  hook DD_NLS_TEST_SKIP_ARRIVAL, one launch only) and the wait limit is 5 ms; every block gives up,
  the call returns DD_NLS_ETIMEOUT, nothing is committed, and the next call on the same handle
  steps normally.  In FP64 the wait is the cooperative launch's global-memory barrier; in FP32
  with the double-word residual it is the exchange of a thread-block cluster (CTA 1 of strip 0's
  cluster pushes nothing).
* An exact breakdown of the inner COCG: a strip whose first residual r satisfies r^T D^{-1} r = 0
  exactly (two edge nodes of equal diagonal with residuals -3 and -3i, made exact by a mesh of
  hy = 6 where the edge mass is the integer matrix [[2, 1], [1, 2]]); the recurrence cannot form
  beta and the call returns DD_NLS_EBREAKDOWN.
* A device allocation that fails inside create (test hook DD_NLS_TEST_FAIL_ALLOC): create returns
  DD_NLS_ENOMEM and releases what it had allocated.
* An unknown ptr_kind: DD_NLS_EINVAL before any copy, and the handle steps on.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1603_05110_gb300 import binding, workloads as wl  # noqa: E402
from tests.helpers import gpu_params  # noqa: E402

pytestmark = pytest.mark.gpu

SMALL = wl.scaled(wl.NLS_SMALL, 48, 37, n_strips=3, xl=-6.0, xr=6.0, yb=-5.0, yu=5.0, dt=0.02)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05110_gb300 import build
    build.build()
    binding.load()


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_DW])
def test_a_wait_that_runs_out_returns_etimeout_and_the_handle_stays_usable(monkeypatch, precision):
    w = SMALL
    prm = gpu_params(w, tol=1e-12, wait_limit_ms=5.0, precision=precision)
    ref = np.zeros_like(w.u0())
    with binding.Solver(prm, w.u0(), w.V()) as s:
        s.step(1, ref)
    monkeypatch.setenv("DD_NLS_TEST_SKIP_ARRIVAL", "2")          # block 1 (of strip 0's blocks)
    s = binding.Solver(prm, w.u0(), w.V())
    monkeypatch.delenv("DD_NLS_TEST_SKIP_ARRIVAL")
    try:
        with pytest.raises(binding.DDNLSError) as e:
            s.step(1)
        assert e.value.code == 6 and "timed out" in str(e.value)
        assert s.get_state() == 0                                 # not committed
        out = np.zeros_like(w.u0())
        st = s.step(1, out)                                       # the hook applied to one launch
        assert st["steps"] == 1
        assert np.array_equal(out, ref)
    finally:
        s.close()


def breakdown_case(precision):
    """Two strips of one cell, ny = 1, hy = 6, u0 = 0, V = 0, kappa = 0: strip 0's right-edge rows
    carry -M^Gamma r with r = (2 - i, -1 + 2i), i.e. residuals (-3, -3i) on two nodes of equal
    diagonal, so r^T D^{-1} r = 9 d^{-1} - 9 d^{-1} = 0 exactly."""
    prm = dict(xl=0.0, xr=2.0, yb=0.0, yu=6.0, nx=2, ny=1, n_strips=2, dt=0.1, lap=1.0, kappa=0.0, p=1.0,
               tol=1e-12, nl_tol=1e-13, precision=precision)
    u0 = np.zeros((2, 3), np.complex128)
    g0 = np.zeros((2, 2), np.complex128)
    g0[0] = [2 - 1j, -1 + 2j]
    return prm, u0, g0


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_INNER])
def test_an_exact_cocg_breakdown_returns_ebreakdown(precision):
    prm, u0, g0 = breakdown_case(precision)
    with binding.Solver(prm, u0) as s:
        with pytest.raises(binding.DDNLSError) as e:
            s.solve_interface(g0)
        assert e.value.code == 7, str(e.value)
        assert s.get_state() == 0


def test_a_failed_device_allocation_in_create_returns_enomem_and_releases(monkeypatch):
    w = SMALL
    torch.cuda.synchronize()
    with binding.Solver(gpu_params(w), w.u0(), w.V()) as s:      # first create: context, module load
        s.step(1)
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 5, 12):
        monkeypatch.setenv("DD_NLS_TEST_FAIL_ALLOC", str(k))
        with pytest.raises(binding.DDNLSError) as e:
            binding.Solver(gpu_params(w), w.u0(), w.V())
        assert e.value.code == 2 and "memory" in str(e.value).lower()
    monkeypatch.delenv("DD_NLS_TEST_FAIL_ALLOC")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (2 << 20)
    with binding.Solver(gpu_params(w), w.u0(), w.V()) as s:
        assert s.step(1)["steps"] == 1


def test_an_unknown_ptr_kind_is_einval_and_the_handle_stays_usable():
    """Every entry point that takes caller memory checks ptr_kind before it copies."""
    w = SMALL
    out = np.zeros((w.ny + 1, w.nx + 1), np.complex128)
    with binding.Solver(gpu_params(w), w.u0(), w.V()) as s:
        ptr = ctypes.c_void_p(out.ctypes.data)
        assert s.lib.dd_nls_step(s.h, 1, ptr, 7, None) == 1
        assert "ptr_kind" in s.lib.dd_nls_last_error(s.h).decode()
        assert s.lib.dd_nls_get_state(s.h, ptr, None, None, -1) == 1
        assert s.step(1, out)["steps"] == 1
        assert np.isfinite(out).all()
