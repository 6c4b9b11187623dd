"""FP64 forward and backward of the learned impulse detector ("gate").

TEST INFRASTRUCTURE ONLY (oracle side).  The network is not in the paper; it
is a learned stand-in for the detection step of switching filters such as the
EVMF (Sec. 3.3, whose entropy switch decides which pixels get filtered):

  x0 = RGB / 255 - 1/2                              (3 x H x W, centred)
  z1 = conv3x3(x0; W1, b1),  a1 = max(z1, 0)        (16 channels)
  z2 = conv3x3(a1; W2, b2),  a2 = max(z2, 0)        (16 channels)
  z3 = conv3x3(a2; W3, b3)                          (1 channel, the logit)
  p  = 1 / (1 + exp(-z3))                            impulse probability

conv3x3 is a cross-correlation with zero padding:
  z[o, y, x] = b[o] + sum_c sum_{u,v in -1..1} W[o, c, u+1, v+1] x[c, y+u, x+v].
Loss: mean binary cross-entropy against a 0/1 target t,
  L = mean(softplus(z3) - t z3)  (= -mean(t log p + (1 - t) log(1 - p))),
so dL/dz3 = (p - t) / (H W B).

Parameters are a flat vector in the order W1, b1, W2, b2, W3, b3 (W as
[out][in][3][3]), the same order the CUDA path uses.
"""
from __future__ import annotations

import numpy as np

SHAPES = [("W1", (16, 3, 3, 3)), ("b1", (16,)), ("W2", (16, 16, 3, 3)), ("b2", (16,)),
          ("W3", (1, 16, 3, 3)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[k:k + n].reshape(shp)
        k += n
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def conv3x3(x, W, b):
    """x: C x H x W, W: O x C x 3 x 3, zero padding."""
    C, H, Wd = x.shape
    xp = np.zeros((C, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((W.shape[0], H, Wd))
    for o in range(W.shape[0]):
        acc = np.full((H, Wd), float(b[o]))
        for c in range(C):
            for u in range(3):
                for v in range(3):
                    acc += W[o, c, u, v] * xp[c, u:u + H, v:v + Wd]
        out[o] = acc
    return out


def conv3x3_grads(x, W, dz):
    """Gradients of sum(dz * conv3x3(x; W, b)) w.r.t. W, b and x."""
    C, H, Wd = x.shape
    O = W.shape[0]
    xp = np.zeros((C, H + 2, Wd + 2))
    xp[:, 1:-1, 1:-1] = x
    dW = np.zeros_like(W)
    for o in range(O):
        for c in range(C):
            for u in range(3):
                for v in range(3):
                    dW[o, c, u, v] = np.sum(dz[o] * xp[c, u:u + H, v:v + Wd])
    db = dz.reshape(O, -1).sum(axis=1)
    # dx[c, y, x] = sum_o sum_{u,v} W[o,c,u,v] dz[o, y-u+1, x-v+1]
    dzp = np.zeros((O, H + 2, Wd + 2))
    dzp[:, 1:-1, 1:-1] = dz
    dx = np.zeros((C, H, Wd))
    for c in range(C):
        for o in range(O):
            for u in range(3):
                for v in range(3):
                    dx[c] += W[o, c, u, v] * dzp[o, 2 - u:2 - u + H, 2 - v:2 - v + Wd]
    return dW, db, dx


def forward(img, theta, act_bf16: bool = False):
    """img: H x W x 3 (or 4) uint8.  Returns the cache of every layer.
    act_bf16 rounds every convolution's input (x0, a1, a2) to bfloat16 first,
    the operand precision of a BF16 tensor-core inference (weights are passed
    in already rounded; accumulation stays exact here)."""
    p = unflatten(theta)
    q = bf16_round if act_bf16 else (lambda v: v)
    x0 = np.transpose(np.asarray(img)[..., :3].astype(np.float64) / 255.0 - 0.5, (2, 0, 1))
    z1 = conv3x3(q(x0), p["W1"], p["b1"])
    a1 = np.maximum(z1, 0.0)
    z2 = conv3x3(q(a1), p["W2"], p["b2"])
    a2 = np.maximum(z2, 0.0)
    z3 = conv3x3(q(a2), p["W3"], p["b3"])[0]
    prob = 1.0 / (1.0 + np.exp(-z3))
    return {"x0": x0, "z1": z1, "a1": a1, "z2": z2, "a2": a2, "z3": z3, "p": prob}


def loss(caches, targets):
    """Mean BCE over all pixels of all images (logit form)."""
    tot, n = 0.0, 0
    for c, t in zip(caches, targets):
        z = c["z3"]
        tot += np.sum(np.logaddexp(0.0, z) - t * z)
        n += z.size
    return tot / n


def backward(caches, targets, theta):
    """Gradient of the mean BCE (over all images) w.r.t. the flat parameters."""
    p = unflatten(theta)
    g = {name: np.zeros(shp) for name, shp in SHAPES}
    n = sum(c["z3"].size for c in caches)
    for c, t in zip(caches, targets):
        dz3 = ((c["p"] - t) / n)[None]
        dW3, db3, da2 = conv3x3_grads(c["a2"], p["W3"], dz3)
        dz2 = da2 * (c["z2"] > 0)
        dW2, db2, da1 = conv3x3_grads(c["a1"], p["W2"], dz2)
        dz1 = da1 * (c["z1"] > 0)
        dW1, db1, _ = conv3x3_grads(c["x0"], p["W1"], dz1)
        for name, v in (("W1", dW1), ("b1", db1), ("W2", dW2), ("b2", db2), ("W3", dW3),
                        ("b3", db3)):
            g[name] += v
    return flatten(g)


def init(seed: int = 0):
    """He-style initial parameters (deterministic)."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, shp in SHAPES:
        if name.startswith("W"):
            fan_in = shp[1] * 9
            out[name] = rng.normal(0.0, np.sqrt(2.0 / fan_in), shp)
        else:
            out[name] = np.zeros(shp)
    return flatten(out)


def target_mask(clean, noisy, threshold: int = 12):
    """1 where some channel of the noisy pixel differs from the clean one by
    more than `threshold` levels (a visible impulse), else 0."""
    d = np.abs(np.asarray(noisy)[..., :3].astype(int) - np.asarray(clean)[..., :3].astype(int))
    return (d.max(axis=-1) > threshold).astype(np.float64)


def bf16_round(x):
    """Round FP64 values to the nearest bfloat16 (ties to even), as FP64."""
    x32 = np.asarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
