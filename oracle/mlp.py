"""Learned initial guess for the coarse Poisson solve: FP64 reference (test infrastructure only).

Not in the paper: the network of the learned-guess form is defined here and followed
by the CUDA kernels.  It is a per-vertex MLP on the pressure-increment mesh with 1-ring
mean aggregation:

* inputs per vertex i: f_i = (r_i / s_r, q_i / s_q, x_i, y_i), r the (projected) coarse
  right-hand side of Eq. 23, q the previous step's increment Phi_c, s_r and s_q their root
  mean squares over the mesh (1 if zero);
* layer l = 1, 2, 3: a_l,i = W_l [h_{l-1,i}; m_{l-1,i}] + b_l with m_{l-1,i} the mean of
  h_{l-1,j} over the neighbours j != i of i; h_l = relu(a_l) for l = 1, 2; widths 4 -> 64
  -> 64 -> 1;
* prediction: Phi0_i = q_i + s_q * a_3,i (a correction of the previous increment);
* training loss for a target Phi*: mean_i (a_3,i - clip((Phi*_i - q_i) / s_q, -10, 10))^2,
  averaged over the samples of a batch (the clip bounds the regression target on
  transient steps where Phi changes by many times its own size).

Weights are stored as W_l (out, 2*in) and b_l (out,).  The CUDA forward uses bfloat16
copies of W and FP32 arithmetic; this reference takes whatever weights it is given in
FP64, so a test passes it the bfloat16-rounded weights.

Parity: backward pinned by central finite differences of the loss in
tests/test_oracle_mlp.py; the forward by a per-vertex loop written out independently;
adam_step (Kingma and Ba 2015, Algorithm 1) by its first bias-corrected step,
-lr g / (|g| + eps), and two scalar steps worked out by hand (tests/test_oracle_pins.py).
"""

import numpy as np

WIDTHS = (4, 64, 64, 1)
TARGET_CLIP = 10.0


def init_weights(seed=0):
    """He-style initialisation from a seeded generator (the same recipe the library uses
    is not required: tests pass weights explicitly)."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for fin, fout in zip(WIDTHS[:-1], WIDTHS[1:]):
        W.append(rng.standard_normal((fout, 2 * fin)) * np.sqrt(2.0 / (2 * fin)))
        b.append(np.zeros(fout))
    return W, b


def neighbour_mean(h, rowptr, col):
    """m_i = mean of h_j over j in the 1-ring of i, i excluded."""
    n = h.shape[0]
    m = np.zeros_like(h)
    for i in range(n):
        js = [j for j in col[rowptr[i]:rowptr[i + 1]] if j != i]
        m[i] = h[js].mean(axis=0)
    return m


def features(r, q, xy):
    sr = np.sqrt(np.mean(r * r))
    sq = np.sqrt(np.mean(q * q))
    sr = sr if sr > 0 else 1.0
    sq = sq if sq > 0 else 1.0
    return np.stack([r / sr, q / sq, xy[:, 0], xy[:, 1]], 1), sr, sq


def forward(W, b, r, q, xy, rowptr, col):
    """Returns (prediction Phi0, cache for backward)."""
    h, sr, sq = features(r, q, xy)
    hs, ms, As = [h], [], []
    for l in range(3):
        m = neighbour_mean(hs[-1], rowptr, col)
        a = np.concatenate([hs[-1], m], 1) @ W[l].T + b[l]
        ms.append(m)
        As.append(a)
        hs.append(np.maximum(a, 0.0) if l < 2 else a)
    out = As[2][:, 0]
    return q + sq * out, {"hs": hs, "ms": ms, "As": As, "sq": sq}


def loss_and_grads(W, b, samples, xy, rowptr, col):
    """samples: list of (r, q, target).  Mean loss over samples and its gradients."""
    n = xy.shape[0]
    gW = [np.zeros_like(w) for w in W]
    gb = [np.zeros_like(x) for x in b]
    total = 0.0
    for r, q, tgt in samples:
        _, c = forward(W, b, r, q, xy, rowptr, col)
        out = c["As"][2][:, 0]
        t = np.clip((tgt - q) / c["sq"], -TARGET_CLIP, TARGET_CLIP)
        d = out - t
        total += np.mean(d * d)
        ga = (2.0 / n) * d[:, None] / len(samples)          # dL/da_3
        for l in (2, 1, 0):
            x = np.concatenate([c["hs"][l], c["ms"][l]], 1)
            gW[l] += ga.T @ x
            gb[l] += ga.sum(axis=0)
            if l == 0:
                break
            gx = ga @ W[l]                                    # (n, 2*fin)
            fin = W[l].shape[1] // 2
            gh = gx[:, :fin].copy()
            gm = gx[:, fin:]
            # transpose of the neighbour mean: h_j feeds m_i of every neighbour i with 1/deg_i
            for i in range(n):
                js = [j for j in col[rowptr[i]:rowptr[i + 1]] if j != i]
                gh[js] += gm[i] / len(js)
            ga = gh * (c["As"][l - 1] > 0)
    return total / len(samples), gW, gb


def adam_step(W, b, gW, gb, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of the FP32 master weights (in place); state = dict with 'm', 'v', 't'."""
    state["t"] += 1
    t = state["t"]
    params = W + b
    grads = gW + gb
    for k, (p, g) in enumerate(zip(params, grads)):
        m = state["m"][k] = beta1 * state["m"][k] + (1 - beta1) * g
        v = state["v"][k] = beta2 * state["v"][k] + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p -= lr * mh / (np.sqrt(vh) + eps)
