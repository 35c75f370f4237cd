"""Pair-selector network: FP64 forward / backward, FP32 inference, features.

TEST INFRASTRUCTURE ONLY.  The learned pair selector is not in the paper: it
only orders the certified actions of a node pair ahead of Fig. 6's bestMethod
rule, so its arithmetic here is the textbook multilayer perceptron with a
softmax cross-entropy loss and the Adam update (Kingma & Ba 2015), written
out plainly.

Network (12 -> 64 -> 64 -> 5):
  z  = (x - mu) * sc                      input normalisation (not trained)
  h1 = relu(W1^T z  + b1)                 W1: 12 x 64
  h2 = relu(W2^T h1 + b2)                 W2: 64 x 64
  o  = W3^T h2 + b3                       W3: 64 x 5, one score per action
  L  = mean_n  s_n (logsumexp(o_n) - o_n[y_n])

Parameter blob (float32, this order): mu[12], sc[12], W1[12][64], b1[64],
W2[64][64], b2[64], W3[64][5], b3[5]  -- 5341 values.

`infer_f32` restates the FP32 inference of the frontier kernel operation by
operation (each product and sum rounded to FP32 separately, inputs taken in
ascending order), so selector decisions can be compared bit for bit.
`features_f32` gives the piecewise-linear log2 used by the pair features.
"""
import numpy as np

NIN, NH, NOUT = 12, 64, 5
SHAPES = (("mu", (NIN,)), ("sc", (NIN,)), ("W1", (NIN, NH)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)),
          ("W3", (NH, NOUT)), ("b3", (NOUT,)))
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)
TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3")


def unpack(blob):
    """Blob -> dict of arrays (views, same dtype as the blob)."""
    blob = np.asarray(blob)
    assert blob.shape == (NPARAM,)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = blob[o:o + n].reshape(shp)
        o += n
    return out


def pack(params, dtype=np.float32):
    return np.concatenate([np.asarray(params[name], np.float64).reshape(-1) for name, _ in SHAPES]).astype(dtype)


def init(seed=0, mu=None, sc=None):
    """He-style random initial parameters (float32 blob)."""
    g = np.random.default_rng(seed)
    p = {"mu": np.zeros(NIN) if mu is None else mu, "sc": np.ones(NIN) if sc is None else sc,
         "W1": g.normal(0, np.sqrt(2.0 / NIN), (NIN, NH)), "b1": np.zeros(NH),
         "W2": g.normal(0, np.sqrt(2.0 / NH), (NH, NH)), "b2": np.zeros(NH),
         "W3": g.normal(0, np.sqrt(1.0 / NH), (NH, NOUT)), "b3": np.zeros(NOUT)}
    return pack(p)


def forward(blob, x):
    """FP64 forward.  x: n x 12.  Returns logits (n x 5) and the cache."""
    p = {k: np.asarray(v, np.float64) for k, v in unpack(blob).items()}
    x = np.asarray(x, np.float64)
    z = (x - p["mu"]) * p["sc"]
    a1 = z @ p["W1"] + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(a2, 0.0)
    o = h2 @ p["W3"] + p["b3"]
    return o, (p, z, a1, h1, a2, h2)


def loss(blob, x, y, s=None):
    """Mean weighted softmax cross entropy (FP64)."""
    o, _ = forward(blob, x)
    y = np.asarray(y, np.int64)
    s = np.ones(len(y)) if s is None else np.asarray(s, np.float64)
    m = o.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.exp(o - m).sum(axis=1))
    return float(np.mean(s * (lse - o[np.arange(len(y)), y])))


def grad(blob, x, y, s=None):
    """FP64 gradient of `loss` with respect to every blob entry (mu, sc get 0)."""
    o, (p, z, a1, h1, a2, h2) = forward(blob, x)
    n = len(y)
    y = np.asarray(y, np.int64)
    s = np.ones(n) if s is None else np.asarray(s, np.float64)
    e = np.exp(o - o.max(axis=1, keepdims=True))
    prob = e / e.sum(axis=1, keepdims=True)
    do = prob.copy()
    do[np.arange(n), y] -= 1.0
    do *= (s / n)[:, None]
    g = {"mu": np.zeros(NIN), "sc": np.zeros(NIN)}
    g["W3"] = h2.T @ do
    g["b3"] = do.sum(axis=0)
    dh2 = do @ p["W3"].T
    da2 = dh2 * (a2 > 0)
    g["W2"] = h1.T @ da2
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ p["W2"].T
    da1 = dh1 * (a1 > 0)
    g["W1"] = z.T @ da1
    g["b1"] = da1.sum(axis=0)
    return pack(g, np.float64)


def adam_step(blob, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step t >= 1) of the trained entries, FP64; returns (blob, m, v)."""
    blob = np.asarray(blob, np.float64).copy()
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    step = lr * mh / (np.sqrt(vh) + eps)
    mask = np.zeros(NPARAM, bool)
    o = 0
    for name, shp in SHAPES:
        k = int(np.prod(shp))
        mask[o:o + k] = name in TRAINED
        o += k
    blob[mask] -= step[mask]
    return blob, m, v


# ---------------------------------------------------------------------------
# FP32 restatements used by the selector in the traversal
# ---------------------------------------------------------------------------
def plog2_f32(x):
    """Piecewise-linear log2 in FP32: x = m 2^e, m in [1, 2) -> e + (m - 1).

    0 and subnormals give -150, +inf gives 128."""
    x = np.asarray(x, np.float32)
    out = np.empty(x.shape, np.float32)
    tiny = ~(x >= np.float32(2.0 ** -126))
    inf = np.isinf(x) & (x > 0)
    fr, ex = np.frexp(np.where(tiny | inf, np.float32(1), x))   # x = fr 2^ex, fr in [0.5, 1)
    m = (fr * np.float32(2)).astype(np.float32)
    e = (ex - 1).astype(np.float32)
    out[...] = e + (m - np.float32(1))
    out[tiny] = np.float32(-150)
    out[inf] = np.float32(128)
    return out


def infer_f32(blob, x):
    """FP32 scores, every product and sum rounded separately, inputs in order."""
    p = unpack(np.asarray(blob, np.float32))
    x = np.asarray(x, np.float32)
    f = np.float32
    z = ((x - p["mu"]).astype(f) * p["sc"]).astype(f)
    n = x.shape[0]
    a1 = np.broadcast_to(p["b1"], (n, NH)).astype(f).copy()
    for k in range(NIN):
        a1 = (a1 + (z[:, k:k + 1] * p["W1"][k]).astype(f)).astype(f)
    h1 = np.where(a1 > 0, a1, f(0)).astype(f)
    a2 = np.broadcast_to(p["b2"], (n, NH)).astype(f).copy()
    for i in range(NH):
        a2 = (a2 + (h1[:, i:i + 1] * p["W2"][i]).astype(f)).astype(f)
    h2 = np.where(a2 > 0, a2, f(0)).astype(f)
    o = np.broadcast_to(p["b3"], (n, NOUT)).astype(f).copy()
    for j in range(NH):
        o = (o + (h2[:, j:j + 1] * p["W3"][j]).astype(f)).astype(f)
    return o
