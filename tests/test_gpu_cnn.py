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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.complex128)).to("cuda:0")


@pytest.mark.parametrize("base", [binding.CNN.BASE_EXTRAPOLATE, binding.CNN.BASE_PREVIOUS])
def test_gradients_match_fp64_oracle_elementwise(base):
    """Loss, every gradient entry and every predicted value against the oracle with its BF16
    operand rounding switched on (the rounding points of the definition: features, weights, ReLU
    activations, back-propagated output gradients); what remains is FP32 against FP64 accumulation
    and the rare BF16 rounding it flips.  Both base guesses (extrapolation, previous vector)."""
    rng = np.random.default_rng(4)
    H, W = 6, 37
    e = 1.0 if base == binding.CNN.BASE_EXTRAPOLATE else 0.0
    net = binding.CNN(H, W, base=base)
    params = binding.CNN.init_params(seed=5, last_scale=0.5)
    params[np.arange(params.size) % 7 == 0] += 0.05          # nonzero biases too
    net.set_params(params)
    g = [rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W)) for _ in range(4)]
    loss_gpu, grad_gpu = net.loss_grad(*[dev(x) for x in g])
    x, tgt, _, _ = ocnn.features(g[0], g[1], g[2], g[3], e=e)
    loss_ref, grad_ref = ocnn.loss_grad(params.astype(np.float64), x, tgt, bf16_ops=True)
    assert abs(loss_gpu - loss_ref) < 1e-4 * loss_ref
    scale = np.max(np.abs(grad_ref))
    np.testing.assert_allclose(grad_gpu, grad_ref, rtol=2e-2, atol=2e-3 * scale)
    # forward: the predicted guess, node by node
    g0 = torch.empty_like(dev(g[0]))
    net.guess(dev(g[0]), dev(g[1]), dev(g[2]), g0)
    ref = ocnn.guess(params.astype(np.float64), g[0], g[1], g[2], bf16_ops=True, e=e)
    corr_gpu = g0.cpu().numpy() - (g[0] + e * (g[0] - g[1]))
    corr_ref = ref - (g[0] + e * (g[0] - g[1]))
    np.testing.assert_allclose(corr_gpu, corr_ref, rtol=2e-2, atol=2e-3 * np.max(np.abs(corr_ref)))
    net.close()


def test_adam_steps_match_the_oracle_update():
    """Three dd_cnn_train_step calls against the oracle's Adam (FP64) applied to the gradients the
    device computes at the same parameters (dd_cnn_loss_grad), from zero moments."""
    rng = np.random.default_rng(11)
    H, W = 4, 29
    net = binding.CNN(H, W)
    net.set_params(binding.CNN.init_params(seed=3, last_scale=0.3))
    g = [dev(rng.standard_normal((H, W)) + 1j * rng.standard_normal((H, W))) for _ in range(4)]
    w = net.get_params().astype(np.float64)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    lr = 1e-3
    for t in range(1, 4):
        _, grad = net.loss_grad(*g)
        net.train_step(*g, lr=lr)
        w, m, v = ocnn.adam_step(w, grad.astype(np.float64), m, v, t, lr)
        got = net.get_params().astype(np.float64)
        np.testing.assert_allclose(got, w, rtol=1e-6, atol=1e-3 * lr)
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
