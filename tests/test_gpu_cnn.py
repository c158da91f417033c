"""The learned interface guess on the GPU (dd_cnn_*): gradients against the FP64 oracle, and
what the trained network gains over the previous-step guess of the paper (Sec. 5)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn as ocnn  # noqa: E402
from paper_1603_05110_gb300 import binding, workloads as wl  # noqa: E402
from tests.helpers import gpu_params  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1603_05110_gb300 import build
    build.build()
    binding.load()


def bf16(a):
    """Round to the nearest BF16 value (ties to even), as the device does."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex128)).to("cuda:0")


def test_gradients_match_fp64_oracle():
    rng = np.random.default_rng(4)
    H, W = 6, 37
    net = binding.CNN(H, W)
    params = binding.CNN.init_params(seed=5, last_scale=0.5)
    params[np.arange(params.size) % 7 == 0] += 0.05          # nonzero biases too
    net.set_params(params)
    g = [rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W)) for _ in range(4)]
    loss_gpu, grad_gpu = net.loss_grad(*[dev(x) for x in g])
    # the oracle on the values the device sees: BF16 parameters and features
    x, tgt, _, _ = ocnn.features(g[0], g[1], g[2], g[3])
    loss_ref, grad_ref = ocnn.loss_grad(bf16(params), bf16(x), tgt)
    assert abs(loss_gpu - loss_ref) < 2e-2 * loss_ref
    err = np.linalg.norm(grad_gpu - grad_ref) / np.linalg.norm(grad_ref)
    cos = grad_gpu @ grad_ref / (np.linalg.norm(grad_gpu) * np.linalg.norm(grad_ref))
    assert err < 5e-2 and cos > 0.998, (err, cos)
    # forward: the predicted guess
    g0 = torch.empty_like(dev(g[0]))
    net.guess(dev(g[0]), dev(g[1]), dev(g[2]), g0)
    ref = ocnn.guess(bf16(params), g[0], g[1], g[2])
    corr_gpu = g0.cpu().numpy() - (2 * g[0] - g[1])
    corr_ref = ref - (2 * g[0] - g[1])
    assert np.linalg.norm(corr_gpu - corr_ref) < 3e-2 * np.linalg.norm(corr_ref)
    net.close()


def trajectory(w, steps, prm):
    """Converged interface vectors and states of the plain solver, steps 0..steps."""
    us, gs = [w.u0()], []
    ntr = 2 * (w.n_strips - 1)
    with binding.Solver(prm, w.u0(), w.V()) as s:
        for _ in range(steps):
            out = np.zeros_like(w.u0())
            s.step(1, out)
            g = np.zeros((ntr, w.ny + 1), np.complex128)
            s.get_state(None, g)
            us.append(out)
            gs.append(g)
    return us, gs


def test_trained_guess_needs_fewer_schwarz_iterations():
    w = wl.Workload("learn", -8.0, 8.0, -8.0, 8.0, 64, 64, 4, 0.005, 60, lap=0.5, kappa=-300.0,
                    p=float(np.sqrt(4 / 0.005)), potential="trap", datum="ground_noise", seed=2000)
    prm = gpu_params(w, tol=1e-10, nl_tol=1e-13)
    us, gs = trajectory(w, 56, prm)          # gs[n-1] = converged g of step n
    H, Wd = gs[0].shape
    net = binding.CNN(H, Wd)
    net.set_params(binding.CNN.init_params(seed=7, last_scale=0.1))
    train = range(3, 40)                     # predict g of step n+1 from steps n, n-1, n-2
    for epoch in range(60):
        for n in train:
            net.train_step(dev(gs[n - 1]), dev(gs[n - 2]), dev(gs[n - 3]), dev(gs[n]), lr=3e-4)

    def iterations(n, g0):
        """Schwarz iterations of step n+1 started from g0 (state u after step n)."""
        with binding.Solver(prm, us[n], w.V()) as s:
            st = s.solve_interface(np.ascontiguousarray(g0))
        return st["last_schwarz_iterations"]

    prev, extrap, learned = [], [], []
    g0 = torch.empty(H, Wd, dtype=torch.complex128, device="cuda:0")
    for n in range(42, 55):                  # held out
        prev.append(iterations(n + 1, gs[n]))
        extrap.append(iterations(n + 1, 2 * gs[n] - gs[n - 1]))
        net.guess(dev(gs[n]), dev(gs[n - 1]), dev(gs[n - 2]), g0)
        learned.append(iterations(n + 1, g0.cpu().numpy()))
    net.close()
    print(f"Schwarz iterations per step, held out: previous {np.mean(prev):.1f}, "
          f"extrapolation {np.mean(extrap):.1f}, learned {np.mean(learned):.1f}")
    assert np.mean(learned) < np.mean(prev)
