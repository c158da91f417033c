"""dd_nls_step_noalloc against dd_nls_step.

The no-allocation entry point serves callers that cannot call cudaMalloc while they step (a
pool or arena that owns the device, a shared context whose allocation state must not
change).  It takes all of its working memory from a fixed array inside the library.  Two
consecutive time steps through it must match two steps of the ordinary entry point within
the parity tolerance of the FP64 path (both iterate to the same interface tolerance).

This file is collected last on purpose: a failure here leaves every other test already run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1603_05110_gb300 import binding, workloads as wl  # noqa: E402
from tests.helpers import gpu_params, rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05110_gb300 import build
    build.build()
    binding.load()


@pytest.mark.parametrize("precision", [binding.FP64, binding.FP32_INNER])
def test_two_noalloc_steps_match_the_ordinary_step(precision):
    w = wl.scaled(wl.NLS_SMALL, 48, 37, n_strips=3, xl=-6.0, xr=6.0, yb=-5.0, yu=5.0, dt=0.02)
    prm = gpu_params(w, tol=1e-12, precision=precision)
    u0 = w.u0()
    V = w.V()
    # ordinary entry point: a handle, two steps
    ref = []
    out = np.zeros_like(u0)
    with binding.Solver(prm, u0, V) as s:
        for _ in range(2):
            s.step(1, out)
            ref.append(out.copy())
    # no-allocation entry point: state on the caller's side, two calls in a row
    dev = torch.device("cuda:0")
    u = torch.from_numpy(u0.copy()).to(dev)
    Vd = torch.from_numpy(V.copy()).to(dev)
    ntr = 2 * (w.n_strips - 1)
    g = torch.zeros(ntr, w.ny + 1, dtype=torch.complex128, device=dev)
    g_next = torch.zeros_like(g)
    for k in range(2):
        st = binding.step_noalloc(prm, u, Vd, g0=g if k else None, g_out=g_next)
        assert st["steps"] == 1 and st["schwarz_iterations"] > 0
        torch.cuda.synchronize()
        assert rel(u.cpu().numpy(), ref[k]) < 1e-11
        g.copy_(g_next)
    # the property the entry point exists for: further steps change neither the device's free
    # memory nor torch's pool
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(3):
        binding.step_noalloc(prm, u, Vd, g0=g, g_out=g_next)
        g.copy_(g_next)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_the_double_word_form_by_name():
    w = wl.scaled(wl.NLS_SMALL, 48, 37, n_strips=3)
    u = torch.zeros(w.ny + 1, w.nx + 1, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(binding.DDNLSError) as e:
        binding.step_noalloc(gpu_params(w, precision=binding.FP32_DW), u)
    assert e.value.code == 1 and "FP32_DW" in str(e.value)


def test_noalloc_rejects_a_problem_beyond_its_memory():
    w = wl.scaled(wl.NLS_SMALL, 1024, 1024, n_strips=16)
    u = torch.zeros(w.ny + 1, w.nx + 1, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(binding.DDNLSError) as e:
        binding.step_noalloc(gpu_params(w), u)
    assert e.value.code == 1 and "limit" in str(e.value)
