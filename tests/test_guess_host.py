"""CPU tests of the learned guess's host logic (paper_2304_07386_gb300/guess.py):
the element grid <-> channel layout of features and targets, the proposal's
inverse mapping back to the library's nodal varphi layout, the per-channel
normalization, and the training loop's mini-batches and learning-rate
schedule.  The network itself is replaced by a stand-in object with the same
methods (its kernels are checked on the GPU and host-emulated elsewhere)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_07386_gb300 import guess as G  # noqa: E402


def test_features_put_each_element_at_its_grid_position():
    nx = 5
    rng = np.random.default_rng(0)
    st = np.exp(rng.standard_normal(nx * nx))
    ss = st * rng.uniform(0.5, 0.99, nx * nx)
    q = rng.integers(0, 2, nx * nx).astype(float)
    f = G.features(st, ss, q, nx)
    assert f.shape == (3, nx, nx) and f.dtype == np.float32
    for e in range(nx * nx):
        iy, ix = divmod(e, nx)
        assert np.allclose(f[:, iy, ix], [np.log(st[e]), ss[e] / st[e], q[e]], rtol=1e-6)


def test_targets_and_the_proposal_mapping_are_inverse():
    """targets() turns nodal varphi [element][node] into channels [node][y][x];
    predict_phi() must map the network's output in that layout back to the
    library's [element][node] vector, through the normalizer's inverse."""
    nx, n = 4, 9
    rng = np.random.default_rng(1)
    phi = rng.standard_normal(nx * nx * n)
    y = G.targets(phi, nx, n)
    assert y.shape == (n, nx, nx)
    assert y[3, 2, 1] == np.float32(phi[(2 * nx + 1) * n + 3])
    norm = G.Normalizer(np.stack([y, 2 * y + 1]))

    class EchoNet:
        """forward() writes the normalized targets, as a perfect network would."""

        def forward(self, x, out):
            out.copy_(torch.as_tensor(norm.fwd(y[None])))

    x = torch.zeros((1, 3, nx, nx), dtype=torch.float32)
    got = G.predict_phi(EchoNet(), x, norm, nx, n)
    assert got.dtype == np.float64 and got.shape == phi.shape
    assert np.allclose(got, phi, rtol=1e-5, atol=1e-5)


def test_normalizer_is_per_channel_and_invertible():
    rng = np.random.default_rng(2)
    data = rng.standard_normal((6, 3, 4, 4)) * np.array([1.0, 10.0, 0.1])[None, :, None, None] + 5.0
    norm = G.Normalizer(data)
    z = norm.fwd(data)
    assert np.allclose(z.mean(axis=(0, 2, 3)), 0.0, atol=1e-5)
    assert np.allclose(z.std(axis=(0, 2, 3)), 1.0, atol=1e-4)
    assert np.allclose(norm.inv(z), data, rtol=1e-5, atol=1e-5)


def test_training_loop_draws_distinct_samples_and_decays_the_rate():
    """Each step is one Adam step on a batch of distinct samples; the rate falls
    geometrically from lr to lr / 10 over the run."""
    N, steps, batch, lr = 40, 50, 8, 3e-3
    X = torch.arange(N, dtype=torch.float32).reshape(N, 1, 1, 1).repeat(1, 3, 2, 2)
    Y = torch.zeros((N, 9, 2, 2))

    class Recorder:
        def __init__(self):
            self.calls = []

        def train_step(self, xb, yb, rate):
            self.calls.append((xb[:, 0, 0, 0].tolist(), rate))
            return float(len(self.calls))

    net = Recorder()
    losses = G.train(net, X, Y, steps=steps, batch=batch, lr=lr, seed=3)
    assert losses == [float(i + 1) for i in range(steps)]
    seen = set()
    for s, (ids, rate) in enumerate(net.calls):
        assert len(ids) == batch and len(set(ids)) == batch and all(0 <= i < N for i in ids)
        assert rate == pytest.approx(lr * 0.1 ** (s / steps))
        seen.update(ids)
    assert len(seen) == N
