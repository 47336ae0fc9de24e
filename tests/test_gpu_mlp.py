"""The surrogate network's tensor-core kernels against the FP64 oracle MLP:
forward and gradients with seeded weights, and training (needs a GB300)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import surrogate as S

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2604_24627_gb300.mlp import SurrogateNet  # noqa: E402


def seeded(seed, n):
    rng = np.random.default_rng(seed)
    P = S.init_params(rng)
    for k in P:
        if k.startswith("b"):
            P[k] = rng.normal(0, 0.2, P[k].shape)
    P = {k: np.asarray(v, np.float32).astype(np.float64) for k, v in P.items()}   # the FP32 values sent
    X = rng.uniform(-1, 1, (n, 4)).astype(np.float32).astype(np.float64)
    Zt = rng.normal(0, 1, (n, 96)).astype(np.float32).astype(np.float64)
    return P, X, Zt


def dev(a):
    return torch.tensor(np.asarray(a, np.float32), device="cuda:0")


@pytest.mark.parametrize("n", [1, 127, 128, 300, 4096])
def test_forward_matches_oracle(n):
    P, X, _ = seeded(1, n)
    net = SurrogateNet()
    net.set_params(P)
    got = net.forward(dev(X)).cpu().numpy().astype(np.float64)
    want, _ = S.forward(P, X, bf16_mma=True)
    err = np.abs(got - want)
    # FP32 accumulation against FP64; an occasional bfloat16 rounding flip of
    # a hidden activation moves one output by ~1e-3
    assert np.median(err) <= 2e-5 * max(1.0, np.abs(want).max()), np.median(err)
    assert err.max() <= 4e-3 * max(1.0, np.abs(want).max()), err.max()
    net.close()


@pytest.mark.parametrize("n", [200, 1000])
def test_gradients_match_oracle(n):
    P, X, Zt = seeded(2, n)
    net = SurrogateNet()
    net.set_params(P)
    loss, G = net.gradients(dev(X), dev(Zt))
    want = S.backward(P, X, Zt, bf16_mma=True)
    assert abs(loss - S.loss(P, X, Zt, bf16_mma=True)) <= 1e-4 * loss
    for k in want:
        d = np.linalg.norm(G[k] - want[k])
        assert d <= 5e-3 * np.linalg.norm(want[k]) + 1e-7, (k, d, np.linalg.norm(want[k]))
    net.close()


def test_training_reduces_loss():
    rng = np.random.default_rng(3)
    n = 8192
    X = rng.uniform(-1, 1, (n, 4))
    # a smooth 96-output target of the four features
    k = rng.normal(0, 1.0, (4, 96))
    Zt = np.tanh(X @ k) + 0.3 * np.sin(2.0 * X[:, :1] + X[:, 1:2])
    P = S.init_params(np.random.default_rng(4))
    net = SurrogateNet()
    net.set_params(P)
    Xd, Zd = dev(X), dev(Zt)
    l0 = net.train_step(Xd, Zd, 3e-3, want_loss=True)
    for _ in range(400):
        net.train_step(Xd, Zd, 3e-3)
    l1 = net.train_step(Xd, Zd, 3e-3, want_loss=True)
    assert l1 < 0.05 * l0, (l0, l1)
    net.close()


def test_batches_that_grow_reuse_the_network():
    """Work buffers are re-reserved when a batch outgrows them: every call,
    small then larger, still matches the oracle."""
    net = SurrogateNet()
    for n in (200, 5000, 300, 9000):
        P, X, Zt = seeded(10 + n, n)
        net.set_params(P)
        loss, G = net.gradients(dev(X), dev(Zt))
        want = S.backward(P, X, Zt, bf16_mma=True)
        for k in want:
            assert np.linalg.norm(G[k] - want[k]) <= 5e-3 * np.linalg.norm(want[k]) + 1e-7, (n, k)
        z = net.forward(dev(X)).cpu().numpy()
        zw, _ = S.forward(P, X, bf16_mma=True)
        assert np.median(np.abs(z - zw)) <= 2e-5 * max(1.0, np.abs(zw).max()), n
    net.close()
