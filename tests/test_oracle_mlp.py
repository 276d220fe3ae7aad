"""Pins of the FP64 reference of the learned initial-guess network (oracle/mlp.py)."""

import numpy as np

from workloads import square_mesh, channel_cylinder_mesh
from oracle import mlp
from oracle.mesh import csr_pattern


def _setup(seed=0, n=6):
    m = square_mesh(n)
    rp, col = csr_pattern(m.n_vert, m.tri)
    rng = np.random.default_rng(seed)
    W, b = mlp.init_weights(seed)
    b = [x + 0.05 * rng.standard_normal(x.shape) for x in b]
    samples = []
    for _ in range(2):
        r = rng.standard_normal(m.n_vert)
        q = rng.standard_normal(m.n_vert)
        t = q + 0.3 * rng.standard_normal(m.n_vert)
        samples.append((r, q, t))
    return m, rp, col, W, b, samples


def test_forward_matches_per_vertex_loop():
    # written independently: every vertex, every neuron, plain Python loops
    m, rp, col, W, b, samples = _setup(1, 4)
    r, q, _ = samples[0]
    pred, _ = mlp.forward(W, b, r, q, m.xy, rp, col)
    n = m.n_vert
    sr, sq = np.sqrt(np.mean(r ** 2)), np.sqrt(np.mean(q ** 2))
    h = [[r[i] / sr, q[i] / sq, m.xy[i, 0], m.xy[i, 1]] for i in range(n)]
    for l in range(3):
        nxt = []
        for i in range(n):
            nb = [j for j in col[rp[i]:rp[i + 1]] if j != i]
            mean = [sum(h[j][f] for j in nb) / len(nb) for f in range(len(h[0]))]
            x = h[i] + mean
            row = []
            for o in range(W[l].shape[0]):
                a = b[l][o] + sum(W[l][o, k] * x[k] for k in range(len(x)))
                row.append(max(a, 0.0) if l < 2 else a)
            nxt.append(row)
        h = nxt
    ref = np.array([q[i] + sq * h[i][0] for i in range(n)])
    np.testing.assert_allclose(pred, ref, rtol=1e-12, atol=1e-12)


def test_gradients_match_central_differences():
    m, rp, col, W, b, samples = _setup(2, 4)
    L, gW, gb = mlp.loss_and_grads(W, b, samples, m.xy, rp, col)
    rng = np.random.default_rng(3)
    eps = 1e-6
    for l in range(3):
        for _ in range(6):
            o = rng.integers(W[l].shape[0])
            k = rng.integers(W[l].shape[1])
            Wp = [w.copy() for w in W]
            Wm = [w.copy() for w in W]
            Wp[l][o, k] += eps
            Wm[l][o, k] -= eps
            fd = (mlp.loss_and_grads(Wp, b, samples, m.xy, rp, col)[0]
                  - mlp.loss_and_grads(Wm, b, samples, m.xy, rp, col)[0]) / (2 * eps)
            assert abs(fd - gW[l][o, k]) <= 1e-6 * max(1.0, abs(fd)), (l, o, k, fd, gW[l][o, k])
        o = rng.integers(b[l].shape[0])
        bp = [x.copy() for x in b]
        bm = [x.copy() for x in b]
        bp[l][o] += eps
        bm[l][o] -= eps
        fd = (mlp.loss_and_grads(W, bp, samples, m.xy, rp, col)[0]
              - mlp.loss_and_grads(W, bm, samples, m.xy, rp, col)[0]) / (2 * eps)
        assert abs(fd - gb[l][o]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_reduces_loss_on_a_fixed_batch():
    m, rp, col, W, b, samples = _setup(4, 4)
    state = {"m": [np.zeros_like(x) for x in W + b], "v": [np.zeros_like(x) for x in W + b], "t": 0}
    l0 = mlp.loss_and_grads(W, b, samples, m.xy, rp, col)[0]
    for _ in range(30):
        _, gW, gb = mlp.loss_and_grads(W, b, samples, m.xy, rp, col)
        mlp.adam_step(W, b, gW, gb, state, 1e-2)
    assert mlp.loss_and_grads(W, b, samples, m.xy, rp, col)[0] < 0.5 * l0


def test_zero_network_returns_previous_increment():
    # with zero weights the prediction is the previous increment itself
    m = channel_cylinder_mesh(seed=5, h=0.08)
    rp, col = csr_pattern(m.n_vert, m.tri)
    W = [np.zeros((o, 2 * i)) for i, o in zip(mlp.WIDTHS[:-1], mlp.WIDTHS[1:])]
    b = [np.zeros(o) for o in mlp.WIDTHS[1:]]
    q = np.random.default_rng(6).standard_normal(m.n_vert)
    pred, _ = mlp.forward(W, b, np.ones(m.n_vert), q, m.xy, rp, col)
    np.testing.assert_array_equal(pred, q)
