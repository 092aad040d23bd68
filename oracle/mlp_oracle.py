"""FP64 reference of the learned parameter initializer.

TEST INFRASTRUCTURE ONLY (see the package docstring): the tests,
``__graft_entry__.smoke()`` and the CPU baseline leg of ``bench.py`` may use
it; the product library never does, and it shares no code with the CUDA path.

The initializer has no counterpart in the paper (which fits from a fixed
zero-knowledge guess, Sec. IV-A, and is training-free, Sec. V-C).  What is
computed here is the plain definition of the network and its training loss:

  features   80 per vehicle from the initial state and the observed
             prefix: positions relative to the vehicle's own start / 100 m
             and speeds / 30 m/s (central differences of the observations,
             the known initial speed at j = 0), for the vehicle and its
             leader; a lane head gets a virtual leader 200 m ahead at its own
             speed;
  network    h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2),
             h3 = gelu(W3 h2 + b3), o = W4 h3 + b4, s = sigmoid(o), with the
             exact (erf) GELU;
  loss       L = sum over the batch and 5 outputs of (s - label)^2 / (5 B);
  gradient   reverse-mode chain rule written out layer by layer;
  Adam       beta 0.9 / 0.999, eps 1e-8, bias-corrected.

All arithmetic is float64 on whatever values the caller passes (the GPU
tests pass the bf16-rounded weights and inputs the kernels use).
"""
import numpy as np
from scipy.special import erf

IN, HID, OUT, PREFIX = 80, 256, 5, 20
SHAPES = (("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)), ("W3", (HID, HID)),
          ("b3", (HID,)), ("W4", (OUT, HID)), ("b4", (OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(w):
    """Flat parameter vector -> dict of arrays (views)."""
    w = np.asarray(w, dtype=np.float64)
    assert w.shape == (N_PARAMS,)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def sigmoid(o):
    return 1.0 / (1.0 + np.exp(-o))


def features(lane_off, p_init, v_init, targets, obs_stride, dt, perm=None):
    """(n_rows, 80) float64 features of vehicles perm (default: all, in order).

    targets: (n_obs, N), row j-1 observed at step j*obs_stride; needs
    n_obs >= 20.
    """
    lane_off = np.asarray(lane_off, dtype=np.int64)
    N = int(lane_off[-1])
    p_init = np.asarray(p_init, dtype=np.float64)
    v_init = np.asarray(v_init, dtype=np.float64)
    Y = np.asarray(targets, dtype=np.float64).reshape(-1, N)
    assert Y.shape[0] >= PREFIX
    idx = np.arange(N) if perm is None else np.asarray(perm, dtype=np.int64)
    heads = np.zeros(N, dtype=bool)
    heads[lane_off[:-1][np.diff(lane_off) > 0]] = True
    obs = np.vstack([p_init[None, :], Y[:PREFIX]])           # (21, N): y_0 .. y_20
    span = 2.0 * obs_stride * dt
    X = np.empty((len(idx), 4 * PREFIX))
    for r, i in enumerate(idx):
        y0 = obs[0, i]
        for who, k in enumerate((i, i - 1)):
            xs = X[r, 2 * PREFIX * who:2 * PREFIX * who + PREFIX]
            vs = X[r, 2 * PREFIX * who + PREFIX:2 * PREFIX * (who + 1)]
            if who == 1 and heads[i]:
                xs[:] = X[r, :PREFIX] + 2.0
                vs[:] = X[r, PREFIX:2 * PREFIX]
                continue
            xs[:] = (obs[:PREFIX, k] - y0) / 100.0
            vs[0] = v_init[k] / 30.0
            vs[1:] = (obs[2:PREFIX + 1, k] - obs[0:PREFIX - 1, k]) / span / 30.0
    return X


def labels(theta, lo, hi, perm=None):
    """(n_rows, 5) normalized parameters (theta_q - lo_q) / (hi_q - lo_q)."""
    th = np.asarray(theta, dtype=np.float64)[:5]
    if perm is not None:
        th = th[:, np.asarray(perm, dtype=np.int64)]
    lo = np.asarray(lo, dtype=np.float64)[:, None]
    hi = np.asarray(hi, dtype=np.float64)[:, None]
    return ((th - lo) / (hi - lo)).T.copy()


def forward(w, X):
    """Activations of the batch X (B, 80): dict with z1..z3, h1..h3, o, s."""
    p = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    a = {"x": X}
    h = X
    for l in (1, 2, 3):
        z = h @ p["W%d" % l].T + p["b%d" % l]
        h = gelu(z)
        a["z%d" % l], a["h%d" % l] = z, h
    a["o"] = h @ p["W4"].T + p["b4"]
    a["s"] = sigmoid(a["o"])
    return a


def loss(w, X, T):
    s = forward(w, X)["s"]
    return float(np.sum((s - T) ** 2) / (5.0 * X.shape[0]))


def loss_grad(w, X, T):
    """(L, flat gradient) of the training loss."""
    p = unpack(w)
    a = forward(w, X)
    B = X.shape[0]
    s = a["s"]
    L = float(np.sum((s - T) ** 2) / (5.0 * B))
    g = {}
    d = 2.0 * (s - T) * s * (1.0 - s) / (5.0 * B)          # dL/do, (B, 5)
    g["W4"] = d.T @ a["h3"]
    g["b4"] = d.sum(axis=0)
    up, W_up = d, p["W4"]
    for l in (3, 2, 1):
        dz = (up @ W_up) * gelu_grad(a["z%d" % l])          # dL/dz_l
        below = a["h%d" % (l - 1)] if l > 1 else a["x"]
        g["W%d" % l] = dz.T @ below
        g["b%d" % l] = dz.sum(axis=0)
        up, W_up = dz, p["W%d" % l]
    return L, pack(g)


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t 1-based); returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def predict_params(w, X, lo, hi):
    """(5, B) parameters lo + (hi - lo) sigmoid(o) in (v0, T, s0, a_max, b) order."""
    s = forward(w, X)["s"]
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return (lo + (hi - lo) * s).T.copy()
