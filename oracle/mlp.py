"""FP64 reference of the per-tile termination MLP (test infrastructure only).

48 -> 64 -> 64 -> 1 with ReLU.  Parameters are the packed vector
w1t [64][48] | b1 [64] | w2t [64][64] | b2 [64] | w3 [64] | b3 [1]
(w1t, w2t stored [out][in]).  With `fp16=True` it models the method's
precision: weights and every layer input (x, h1, h2, and the back-propagated
dh2, dh1 that feed products) are rounded to IEEE half, while sums are exact
(FP64), so a GPU with FP32 accumulation must agree to accumulation error;
with `fp16=False` it is the plain real-valued network that finite
differences pin.  The loss is the mean asymmetric squared error
(1/m) sum w_r (y_r - t_r)^2 with w_r = under_weight when y_r < t_r.
"""
import numpy as np

IN, HID = 48, 64
NPARAM = HID * IN + HID + HID * HID + HID + HID + 1
OFF = dict(w1t=0, b1=HID * IN, w2t=HID * IN + HID, b2=HID * IN + HID + HID * HID,
           w3=HID * IN + 2 * HID + HID * HID, b3=HID * IN + 3 * HID + HID * HID)


def _h(a, on):
    return a.astype(np.float16).astype(np.float64) if on else np.asarray(a, np.float64)


def unpack(p, fp16=True):
    p = np.asarray(p, np.float64)
    w1t = _h(p[OFF["w1t"]:OFF["b1"]].reshape(HID, IN), fp16)
    b1 = p[OFF["b1"]:OFF["w2t"]]
    w2t = _h(p[OFF["w2t"]:OFF["b2"]].reshape(HID, HID), fp16)
    b2 = p[OFF["b2"]:OFF["w3"]]
    w3 = _h(p[OFF["w3"]:OFF["b3"]], fp16)
    b3 = p[OFF["b3"]]
    return w1t, b1, w2t, b2, w3, b3


def forward(x, p, fp16=True):
    w1t, b1, w2t, b2, w3, b3 = unpack(p, fp16)
    x = _h(x, fp16)
    z1 = x @ w1t.T + b1
    h1 = _h(np.maximum(z1, 0.0), fp16)
    z2 = h1 @ w2t.T + b2
    h2 = _h(np.maximum(z2, 0.0), fp16)
    y = h2 @ w3 + b3
    return y, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2)


def loss_and_grad(x, p, target, under_weight, fp16=True):
    """(loss, grad [NPARAM]) of the asymmetric squared error."""
    w1t, b1, w2t, b2, w3, b3 = unpack(p, fp16)
    y, c = forward(x, p, fp16)
    m = x.shape[0]
    e = y - target
    w = np.where(e < 0, under_weight, 1.0)
    loss = float(np.sum(w * e * e) / m)
    dy = 2.0 * w * e / m
    g = np.zeros(NPARAM)
    g[OFF["w3"]:OFF["b3"]] = c["h2"].T @ dy
    g[OFF["b3"]] = dy.sum()
    dh2 = np.outer(dy, w3) * (c["z2"] > 0)
    g[OFF["b2"]:OFF["w3"]] = dh2.sum(0)
    dh2q = _h(dh2, fp16)
    g[OFF["w2t"]:OFF["b2"]] = (c["h1"].T @ dh2q).T.reshape(-1)
    dh1 = (dh2q @ w2t) * (c["z1"] > 0)
    g[OFF["b1"]:OFF["w2t"]] = dh1.sum(0)
    dh1q = _h(dh1, fp16)
    g[OFF["w1t"]:OFF["b1"]] = (c["x"].T @ dh1q).T.reshape(-1)
    return loss, g


def adam(step, lr, beta1, beta2, eps, master, grad, m1, m2):
    """One bias-corrected Adam step (FP64); returns new (master, m1, m2)."""
    m1 = beta1 * m1 + (1 - beta1) * grad
    m2 = beta2 * m2 + (1 - beta2) * grad * grad
    mh = m1 / (1 - beta1 ** step)
    vh = m2 / (1 - beta2 ** step)
    return master - lr * mh / (np.sqrt(vh) + eps), m1, m2
