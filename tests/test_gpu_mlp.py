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


U = 2.0 ** -7   # one bfloat16 unit, relative (7 stored mantissa bits)


def tanh_err(h):
    """Bound on the kernels' activation error at |tanh| = h: the hardware
    approximation's relative error (below 1e-5 over a sweep of 16.8 M
    points on a GB300) with a factor 3 of margin, plus 1e-6."""
    return 2.0 ** -15 * h + 1e-6


def forward_bound(P, X):
    """Element-wise bound on |GPU output - oracle output| (see
    gradient_bounds): the hidden activations one bfloat16 unit off, the tanh
    error, FP32 accumulation, carried through |W2| and |W3|."""
    q = S.bf16
    acc = 64 * 2.0 ** -24
    aW2, aW3 = np.abs(q(P["W2"])), np.abs(q(P["W3"]))
    ah1 = np.abs(np.tanh(X @ P["W1"] + P["b1"]))
    ah2 = np.abs(np.tanh(q(np.tanh(X @ P["W1"] + P["b1"])) @ q(P["W2"]) + P["b2"]))
    dh2 = (U * ah1 + tanh_err(ah1)) @ aW2 + acc * (ah1 @ aW2) + tanh_err(ah2)
    return (U * ah2 + dh2) @ aW3 + acc * (ah2 @ aW3)


@pytest.mark.parametrize("n", [1, 127, 128, 300, 4096])
def test_forward_matches_oracle(n):
    """Every output within its bound (forward_bound), and the typical output
    well inside it (median error below a quarter of its bound: the bound
    takes every activation a full bfloat16 unit off in the same direction,
    while the tanh approximation moves only some of them across a rounding
    boundary, in either direction)."""
    P, X, _ = seeded(1, n)
    net = SurrogateNet()
    net.set_params(P)
    got = net.forward(dev(X)).cpu().numpy().astype(np.float64)
    want, _ = S.forward(P, X, bf16_mma=True)
    err = np.abs(got - want)
    B = forward_bound(P, X) + 1e-7
    assert np.all(err <= B), float((err - B).max())
    assert np.median(err / B) < 0.25, np.median(err / B)
    net.close()


def gradient_bounds(P, X, Zt):
    """Element-wise bounds on |GPU gradient - oracle gradient| that the
    arithmetic allows, to first order: every rounded activation or gradient
    operand of a tensor-core product one bfloat16 unit off on one side (the
    sides round slightly different binary32 and FP64 values; the weights
    round identically), every FP32 sum off by n 2^-24 of its absolute sum,
    and the kernels' tanh off by tanh_err, carried through forward and
    backward with absolute values."""
    q = S.bf16
    n = len(X)
    acc = lambda m: m * 2.0 ** -24
    W1, W2, W3 = P["W1"], P["W2"], P["W3"]
    aW2, aW3 = np.abs(q(W2)), np.abs(q(W3))
    h1 = np.tanh(X @ W1 + P["b1"])
    a2 = q(h1) @ q(W2) + P["b2"]
    h2 = np.tanh(a2)
    ah1, ah2 = np.abs(h1), np.abs(h2)
    dh1 = tanh_err(ah1)
    dh2 = (U * ah1 + dh1) @ aW2 + acc(64) * (ah1 @ aW2) + tanh_err(ah2)
    z = q(h2) @ q(W3) + P["b3"]
    dzv = (U * ah2 + dh2) @ aW3 + acc(64) * (ah2 @ aW3)
    g = 2.0 * (z - Zt) / n
    ag = np.abs(g)
    dg = 2.0 * dzv / n + 2.0 ** -23 * ag
    B = {}
    B["W3"] = (U * ah2 + dh2).T @ ag + ah2.T @ (U * ag + dg) + acc(n) * (ah2.T @ ag)
    B["b3"] = dg.sum(0) + acc(n) * ag.sum(0)
    d_h2 = q(g) @ q(W3).T
    dd_h2 = (U * ag + dg) @ aW3.T + acc(96) * (ag @ aW3.T)
    da2 = d_h2 * (1 - h2 ** 2)
    ada2 = np.abs(da2)
    dda2 = dd_h2 + np.abs(d_h2) * 2 * ah2 * dh2
    B["W2"] = (U * ah1 + dh1).T @ ada2 + ah1.T @ (U * ada2 + dda2) + acc(n) * (ah1.T @ ada2)
    B["b2"] = dda2.sum(0) + acc(n) * ada2.sum(0)
    d_h1 = q(da2) @ q(W2).T
    dd_h1 = (U * ada2 + dda2) @ aW2.T + acc(64) * (ada2 @ aW2.T)
    da1 = d_h1 * (1 - h1 ** 2)
    ada1 = np.abs(da1)
    dda1 = dd_h1 + np.abs(d_h1) * 2 * ah1 * dh1
    aX = np.abs(X)
    B["W1"] = aX.T @ dda1 + acc(n) * (aX.T @ ada1)
    B["b1"] = dda1.sum(0) + acc(n) * ada1.sum(0)
    return B


@pytest.mark.parametrize("n", [200, 1000])
def test_gradients_match_oracle(n):
    """Every gradient element within its bound from gradient_bounds, and the
    typical element well inside it (median below a quarter of its bound)."""
    P, X, Zt = seeded(2, n)
    net = SurrogateNet()
    net.set_params(P)
    loss, G = net.gradients(dev(X), dev(Zt))
    want = S.backward(P, X, Zt, bf16_mma=True)
    B = gradient_bounds(P, X, Zt)
    assert abs(loss - S.loss(P, X, Zt, bf16_mma=True)) <= 1e-4 * loss
    rel = []
    for k in want:
        d = np.abs(G[k] - want[k])
        bad = d > B[k] + 1e-12
        assert not bad.any(), (k, int(bad.sum()), float((d - B[k]).max()))
        rel.append((d / (B[k] + 1e-12)).ravel())
    assert np.median(np.concatenate(rel)) < 0.25, np.median(np.concatenate(rel))
    net.close()


def test_adam_steps_match_oracle():
    """Three training steps (gradients, then Adam with bias-corrected moments,
    beta 0.9 and 0.999, eps 1e-8) from the same parameters as the oracle's
    Adam (oracle.surrogate.adam) on the oracle's gradients. A step moves an
    element by lr m/(sqrt(v) + eps), insensitive to the gradient's scale:
    where each step's oracle gradient exceeds its rounding bound B (from
    gradient_bounds) the GPU's element stays within lr sum_t 4 B_t / |G_t| of
    the oracle's (plus binary32 rounding), elsewhere within 2 lr a step; and
    the typical element is well inside that (median below a quarter)."""
    P, X, Zt = seeded(5, 512)
    net = SurrogateNet()
    net.set_params(P)   # resets the Adam state
    lr = 1e-3
    Po = {k: v.copy() for k, v in P.items()}
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    tol = {k: np.zeros_like(v) for k, v in P.items()}
    Xd, Zd = dev(X), dev(Zt)
    for t in range(1, 4):
        G = S.backward(Po, X, Zt, bf16_mma=True)
        B = gradient_bounds(Po, X, Zt)
        for k in G:
            r = B[k] / np.maximum(np.abs(G[k]), 1e-300)
            tol[k] += lr * np.where(r < 0.5, 4.0 * r, 2.0)
        S.adam(Po, G, M, V, t, lr)
        net.train_step(Xd, Zd, lr)
    got = net.get_params()
    rel = []
    for k in got:
        d = np.abs(got[k] - Po[k])
        ulp = 4 * np.spacing(np.abs(Po[k]).astype(np.float32)).astype(np.float64)
        bad = d > tol[k] + ulp
        assert not bad.any(), (k, int(bad.sum()), float((d - tol[k] - ulp).max()))
        rel.append((d / (tol[k] + ulp)).ravel())
    assert np.median(np.concatenate(rel)) < 0.25, np.median(np.concatenate(rel))
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
        B = gradient_bounds(P, X, Zt)
        for k in want:
            assert np.all(np.abs(G[k] - want[k]) <= B[k] + 1e-12), (n, k)
        z = net.forward(dev(X)).cpu().numpy()
        zw, _ = S.forward(P, X, bf16_mma=True)
        Bz = forward_bound(P, X) + 1e-7
        assert np.all(np.abs(z - zw) <= Bz), n
        assert np.median(np.abs(z - zw) / Bz) < 0.25, n
    net.close()
