"""Seeded synthetic inputs: piecewise-smooth colour images and the impulsive
noise models of Sec. 4 (Eq. eq_noise).

This module only makes inputs.  It holds none of the filters' arithmetic, and
both the CUDA path's tests and benchmark and the CPU oracle's tests draw their
images from it, so the two sides see identical pixels.

Every random number comes from a counter-based generator: splitmix64 (Steele,
Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014;
the finaliser constants as published by S. Vigna) applied to
(seed, stream, index), so an image does not depend on the order it is made in.

The paper's 100 Internet images and the Lenna image are not available; the
images here stand in for them with the same kind of content: K random convex
polygons over a smooth background, each with a linear colour gradient, the
three channels correlated at about 0.9 (a shared luminance plus a small
per-channel offset), and mild smooth texture.
"""
from __future__ import annotations

import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x):
    """splitmix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def rand_u64(seed: int, stream: int, index) -> np.ndarray:
    """Counter-based 64-bit random numbers for (seed, stream, index)."""
    key = splitmix64(np.uint64((int(seed) * 1_000_003 + int(stream)) & 0xFFFFFFFFFFFFFFFF))
    with np.errstate(over="ignore"):
        return splitmix64(key + np.asarray(index, dtype=np.uint64))


def rand_uniform(seed: int, stream: int, index) -> np.ndarray:
    """Uniform doubles in [0, 1) (53-bit)."""
    return (rand_u64(seed, stream, index) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def rand_int(seed: int, stream: int, index, lo: int, hi: int) -> np.ndarray:
    """Uniform integers in [lo, hi] (inclusive)."""
    u = rand_uniform(seed, stream, index)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


# streams
_S_SCENE, _S_POLY, _S_NOISE_SEL, _S_NOISE_VAL, _S_NOISE_PAT, _S_GAUSS, _S_SIZES = range(7)


def _num_polygons(h: int, w: int) -> int:
    return int(min(200, max(20, round(h * w / 3000.0))))


def piecewise_smooth(h: int, w: int, seed: int, *, x0: int = 0, canvas_w: int | None = None,
                     canvas_h: int | None = None) -> np.ndarray:
    """An h x w x 3 uint8 image.  (x0, canvas_w, canvas_h) cut a window out of a
    larger scene, for panning video frames; by default the scene is the image."""
    cw = w if canvas_w is None else canvas_w
    ch = h if canvas_h is None else canvas_h
    K = _num_polygons(ch, cw)
    r = rand_uniform(seed, _S_SCENE, np.arange(64))
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    xx += x0
    # smooth background: luminance gradient plus per-channel offsets
    lum = 60.0 + 120.0 * r[0] + 60.0 * (r[1] - 0.5) * (xx / cw) + 60.0 * (r[2] - 0.5) * (yy / ch)
    img = np.empty((h, w, 3), dtype=np.float64)
    for k in range(3):
        img[..., k] = lum + 60.0 * (r[3 + k] - 0.5)
    scale = math.sqrt(ch * cw / K)
    for p in range(K):
        q = rand_uniform(seed, _S_POLY, np.arange(p * 32, p * 32 + 32))
        cx, cy = q[0] * cw, q[1] * ch
        rad = scale * (0.35 + 0.9 * q[2])
        nv = 3 + int(q[3] * 5)  # 3..7 vertices on a circle: a convex polygon
        ang = np.sort(q[4:4 + nv] * 2.0 * math.pi)
        vx, vy = cx + rad * np.cos(ang), cy + rad * np.sin(ang)
        bx0 = max(int(math.floor(vx.min())) - x0, 0)
        bx1 = min(int(math.ceil(vx.max())) - x0 + 1, w)
        by0 = max(int(math.floor(vy.min())), 0)
        by1 = min(int(math.ceil(vy.max())) + 1, h)
        if bx0 >= bx1 or by0 >= by1:
            continue
        X = xx[by0:by1, bx0:bx1]
        Y = yy[by0:by1, bx0:bx1]
        inside = np.ones(X.shape, dtype=bool)
        for e in range(nv):
            ax, ay = vx[e], vy[e]
            bx, by = vx[(e + 1) % nv], vy[(e + 1) % nv]
            inside &= (bx - ax) * (Y - ay) - (by - ay) * (X - ax) >= 0.0
        if not inside.any():
            continue
        L = 20.0 + 215.0 * q[12]
        gx, gy = (q[13] - 0.5) * 80.0 / rad, (q[14] - 0.5) * 80.0 / rad
        grad = gx * (X - cx) + gy * (Y - cy)
        for k in range(3):
            off = 72.0 * (q[15 + k] - 0.5)  # var(off) ~ var(L) / 9: corr ~ 0.9
            chan = L + off + grad * (1.0 + 0.2 * (q[18 + k] - 0.5))
            sub = img[by0:by1, bx0:bx1, k]
            sub[inside] = chan[inside]
    # mild smooth texture shared by the channels, with a small per-channel part
    tex = np.zeros((h, w))
    for t in range(4):
        f = rand_uniform(seed, _S_SCENE, np.arange(100 + 4 * t, 104 + 4 * t))
        kx, ky = (0.02 + 0.2 * f[0]) * (1 if f[2] > 0.5 else -1), 0.02 + 0.2 * f[1]
        tex += 1.5 * np.sin(kx * xx + ky * yy + 6.283 * f[3])
    for k in range(3):
        img[..., k] += tex * (1.0 + 0.3 * k / 2.0)
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def impulse_uncorrelated(img: np.ndarray, p: float, seed: int) -> np.ndarray:
    """Eq. eq_noise, uncorrelated model: each channel k is replaced by a random
    value r_k (uniform on 0..255) with probability phi_k = p.  One 64-bit draw
    per channel: the top 53 bits decide the replacement, the low 8 bits are
    the value."""
    h, w, _ = img.shape
    u = rand_u64(seed, _S_NOISE_SEL, np.arange(h * w * 3, dtype=np.uint64))
    hit = ((u >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 < p).reshape(h, w, 3)
    val = (u & np.uint64(255)).astype(np.uint8).reshape(h, w, 3)
    out = img[..., :3].copy()
    out[hit] = val[hit]
    return out


def impulse_correlated(img: np.ndarray, p: float, seed: int, phi=(0.25, 0.25, 0.25)) -> np.ndarray:
    """Eq. eq_noise, correlated model: a pixel is corrupted with probability
    phi = p; a corrupted pixel has only channel k replaced with probability
    phi_k, or all three with probability 1 - (phi_1 + phi_2 + phi_3)."""
    h, w, _ = img.shape
    idx = np.arange(h * w, dtype=np.uint64)
    hit = rand_uniform(seed, _S_NOISE_SEL, idx).reshape(h, w) < p
    u = rand_uniform(seed, _S_NOISE_PAT, idx).reshape(h, w)
    c1, c2, c3 = phi[0], phi[0] + phi[1], phi[0] + phi[1] + phi[2]
    pattern = np.where(u < c1, 0, np.where(u < c2, 1, np.where(u < c3, 2, 3)))
    val = rand_int(seed, _S_NOISE_VAL, np.arange(h * w * 3, dtype=np.uint64), 0, 255)
    val = val.reshape(h, w, 3).astype(np.uint8)
    mask = np.zeros((h, w, 3), dtype=bool)
    for k in range(3):
        mask[..., k] = hit & ((pattern == k) | (pattern == 3))
    out = img[..., :3].copy()
    out[mask] = val[mask]
    return out


def gaussian(img: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Additive Gaussian noise (Box-Muller on counter-based uniforms), rounded
    and clamped to 0..255."""
    h, w, _ = img.shape
    n = h * w * 3
    u1 = rand_uniform(seed, _S_GAUSS, np.arange(n, dtype=np.uint64))
    u2 = rand_uniform(seed, _S_GAUSS, np.arange(n, 2 * n, dtype=np.uint64))
    g = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    out = img[..., :3].astype(np.float64) + sigma * g.reshape(h, w, 3)
    return np.clip(np.rint(out), 0, 255).astype(np.uint8)


def mixed(img: np.ndarray, p: float, seed: int, sigma: float = 10.0) -> np.ndarray:
    """Sec. 4, mixed model: Gaussian noise followed by correlated impulsive
    noise.  The paper does not give sigma; 10 (on 0..255) is a reading."""
    return impulse_correlated(gaussian(img, sigma, seed), p, seed + 7919)


def noisy(h: int, w: int, p: float, seed: int, model: str = "uncorrelated"):
    """(clean, noisy) pair of h x w x 3 uint8 images."""
    clean = piecewise_smooth(h, w, seed)
    if model == "uncorrelated":
        return clean, impulse_uncorrelated(clean, p, seed)
    if model == "correlated":
        return clean, impulse_correlated(clean, p, seed)
    if model == "mixed":
        return clean, mixed(clean, p, seed)
    raise ValueError(model)


def impulse_mask(clean: np.ndarray, noisy: np.ndarray, threshold: int = 12) -> np.ndarray:
    """uint8 H x W: 1 where some channel of the noisy pixel differs from the
    clean one by more than `threshold` levels (a visible impulse)."""
    d = np.abs(noisy[..., :3].astype(np.int16) - clean[..., :3].astype(np.int16))
    return (d.max(axis=-1) > threshold).astype(np.uint8)


def to_rgbx(img: np.ndarray) -> np.ndarray:
    """H x W x 3 -> H x W x 4 with the fourth byte 0 (the device layout)."""
    h, w, _ = img.shape
    out = np.zeros((h, w, 4), dtype=np.uint8)
    out[..., :3] = img[..., :3]
    return out


def batch_sizes(count: int, seed: int, lo=(240, 320), hi=(1080, 1920)):
    """`count` (height, width) pairs, each uniform between lo and hi."""
    hs = rand_int(seed, _S_SIZES, np.arange(count), lo[0], hi[0])
    ws = rand_int(seed, _S_SIZES, np.arange(count, 2 * count), lo[1], hi[1])
    return [(int(a), int(b)) for a, b in zip(hs, ws)]


def batch_images(count: int, seed: int, lo=(240, 320), hi=(1080, 1920), p_lo: float = 0.05,
                 p_hi: float = 0.30, scenes: int = 4):
    """`count` (clean, noisy, p) triples of uneven sizes (batch_sizes), each cut
    at a seeded offset out of one of `scenes` hi-sized scenes, with
    uncorrelated impulses at a seeded rate in [p_lo, p_hi]."""
    from concurrent.futures import ThreadPoolExecutor
    import os

    sizes = batch_sizes(count, seed, lo, hi)
    r = rand_uniform(seed, _S_SCENE, np.arange(1000, 1000 + 4 * count)).reshape(count, 4)
    # numpy releases the GIL on large arrays: images are independent, so make
    # them in parallel (the result does not depend on the order)
    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        canvas = list(ex.map(lambda c: piecewise_smooth(hi[0], hi[1], seed * 1000 + c),
                             range(scenes)))

        def one(i):
            h, w = sizes[i]
            k = int(r[i, 0] * scenes)
            y0 = int(r[i, 1] * (hi[0] - h + 1))
            x0 = int(r[i, 2] * (hi[1] - w + 1))
            clean = np.ascontiguousarray(canvas[k][y0:y0 + h, x0:x0 + w])
            p = p_lo + (p_hi - p_lo) * float(r[i, 3])
            return clean, impulse_uncorrelated(clean, p, seed * 100003 + i), p

        return list(ex.map(one, range(count)))


def video_frames(count: int, h: int, w: int, seed: int, pan: int = 4, p_lo: float = 0.05,
                 p_hi: float = 0.30):
    """Iterator over `count` frames (clean, noisy, p) of one slowly panning
    scene (pan pixels per frame, made once), uncorrelated impulses at a rate
    ramping from p_lo to p_hi.  Frames are made ahead on a thread pool."""
    from concurrent.futures import ThreadPoolExecutor
    import os

    scene = piecewise_smooth(h, w + pan * max(count - 1, 0), seed)

    def one(f):
        clean = np.ascontiguousarray(scene[:, pan * f:pan * f + w])
        p = p_lo + (p_hi - p_lo) * (f / max(count - 1, 1))
        return clean, impulse_uncorrelated(clean, p, seed * 1000 + f + 1), p

    with ThreadPoolExecutor(min(8, os.cpu_count() or 1)) as ex:
        pending = [ex.submit(one, f) for f in range(min(count, 8))]
        for f in range(count):
            item = pending[f].result()
            pending[f] = None
            if f + 8 < count:
                pending.append(ex.submit(one, f + 8))
            yield item


def video_frame(h: int, w: int, frame: int, frames: int, seed: int, pan: int = 4,
                p_lo: float = 0.05, p_hi: float = 0.30):
    """Frame `frame` of a slowly panning scene (pan pixels per frame) with
    uncorrelated impulses whose rate ramps from p_lo to p_hi over the frames.
    Returns (clean, noisy, p)."""
    canvas_w = w + pan * max(frames - 1, 0)
    clean = piecewise_smooth(h, w, seed, x0=pan * frame, canvas_w=canvas_w, canvas_h=h)
    p = p_lo + (p_hi - p_lo) * (frame / max(frames - 1, 1))
    return clean, impulse_uncorrelated(clean, p, seed * 1000 + frame + 1), p
