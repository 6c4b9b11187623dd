"""Headless image files: binary PPM (P6, 8-bit RGB) from and to host arrays.

Inputs and outputs of the filters are plain H x W x 3 (or x 4 RGBX, whose
fourth byte is dropped on writing) uint8 arrays; this module is how they are
looked at without any graphics stack.
"""
from __future__ import annotations

import numpy as np


def write_ppm(path: str, img) -> None:
    """Write an H x W x 3 or H x W x 4 uint8 array (a host array or a tensor
    already on the host) as a binary PPM."""
    a = np.asarray(img)
    if a.dtype != np.uint8 or a.ndim != 3 or a.shape[2] not in (3, 4):
        raise ValueError("expected an H x W x 3 or H x W x 4 uint8 array")
    h, w = a.shape[:2]
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (w, h))
        f.write(np.ascontiguousarray(a[..., :3]).tobytes())


def _tokens(data: bytes, count: int):
    """The first `count` whitespace-separated header fields (comments skipped)
    and the offset just past the single whitespace byte that ends the last."""
    out, i, n = [], 0, len(data)
    while len(out) < count:
        while i < n and data[i:i + 1].isspace():
            i += 1
        if i < n and data[i:i + 1] == b"#":
            while i < n and data[i:i + 1] not in (b"\n", b"\r"):
                i += 1
            continue
        j = i
        while j < n and not data[j:j + 1].isspace():
            j += 1
        if j == i:
            raise ValueError("truncated PPM header")
        out.append(data[i:j])
        i = j
    return out, i + 1


def read_ppm(path: str) -> np.ndarray:
    """Read a binary 8-bit PPM (P6, maximum value 255) into an H x W x 3 uint8
    array."""
    with open(path, "rb") as f:
        data = f.read()
    (magic, w, h, maxval), off = _tokens(data, 4)
    if magic != b"P6" or int(maxval) != 255:
        raise ValueError("only binary 8-bit PPM (P6, 255) is read")
    w, h = int(w), int(h)
    body = data[off:off + w * h * 3]
    if len(body) != w * h * 3:
        raise ValueError("truncated PPM data")
    return np.frombuffer(body, dtype=np.uint8).reshape(h, w, 3).copy()
