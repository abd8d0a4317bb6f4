"""FP64 reference of the far-field coordinate network (forward, loss, backward).

TEST INFRASTRUCTURE ONLY.  The network is the learned stand-in for the
far-far part of the deflection field (no counterpart in arXiv:2204.10871; the
paper interpolates the whole far field on its level-2 grid):

  input    x in R^2 (position scaled to [-1, 1] by the plane's half-extent)
  features f = [sin(pi B x), cos(pi B x)],  B a fixed 32 x 2 matrix -> 64 values
  layers   h1 = tanh(W1 f + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3)
           (64 -> 64 each), y = W4 h3 + b4 (64 -> 8)
  loss     L = mean over the batch and the 8 outputs of (y - t)^2

Parameters are packed in one flat vector in the order W1, b1, W2, b2, W3, b3,
W4, b4 (row-major W[out][in]), 13,000 values.  The backward pass is written
out by the chain rule; the tests pin it to central finite differences of the
loss, so it does not rely on itself.
"""
import numpy as np

N_FREQ = 32
WIDTH = 64
N_OUT = 8
SHAPES = [("W1", (WIDTH, 2 * N_FREQ)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
          ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("W4", (N_OUT, WIDTH)), ("b4", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def features(x, B):
    a = np.pi * (x @ B.T)
    return np.concatenate([np.sin(a), np.cos(a)], axis=1)


def forward(theta, B, x):
    """Returns the output (n, 8) and the activations needed by backward."""
    p = unpack(theta)
    f = features(x, B)
    h1 = np.tanh(f @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    h3 = np.tanh(h2 @ p["W3"].T + p["b3"])
    y = h3 @ p["W4"].T + p["b4"]
    return y, (f, h1, h2, h3)


def loss(theta, B, x, t):
    y, _ = forward(theta, B, x)
    return float(np.mean((y - t) ** 2))


def backward(theta, B, x, t):
    """Gradient of the loss with respect to the packed parameters."""
    p = unpack(theta)
    y, (f, h1, h2, h3) = forward(theta, B, x)
    n = x.shape[0]
    dy = 2.0 * (y - t) / (n * N_OUT)
    g = {"W4": dy.T @ h3, "b4": dy.sum(0)}
    dz3 = (dy @ p["W4"]) * (1.0 - h3 * h3)
    g["W3"], g["b3"] = dz3.T @ h2, dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * (1.0 - h2 * h2)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (1.0 - h1 * h1)
    g["W1"], g["b1"] = dz1.T @ f, dz1.sum(0)
    return pack(g)


def init_params(seed):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            bound = 1.0 / np.sqrt(shape[1])
            p[name] = rng.uniform(-bound, bound, shape)
        else:
            p[name] = np.zeros(shape)
    return pack(p)
