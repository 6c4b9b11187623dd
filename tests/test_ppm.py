"""Headless image files (binary PPM): round trip, the RGBX fourth byte
dropped, a header with a comment, and the errors."""
import os
import tempfile

import numpy as np
import pytest

from paper_1009_0959_gb300 import ppm, synth


def test_round_trip_and_rgbx():
    clean, noisy = synth.noisy(13, 21, 0.2, 3)
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "a.ppm")
        ppm.write_ppm(p, noisy)
        np.testing.assert_array_equal(ppm.read_ppm(p), noisy)
        with open(p, "rb") as f:
            assert f.read(11) == b"P6\n21 13\n25"  # width first, then height
        ppm.write_ppm(p, synth.to_rgbx(noisy))
        np.testing.assert_array_equal(ppm.read_ppm(p), noisy)


def test_header_comment_and_errors():
    img = np.arange(2 * 3 * 3, dtype=np.uint8).reshape(2, 3, 3)
    with tempfile.TemporaryDirectory() as d:
        p = os.path.join(d, "b.ppm")
        with open(p, "wb") as f:
            f.write(b"P6\n# a comment\n3 2\n255\n" + img.tobytes())
        np.testing.assert_array_equal(ppm.read_ppm(p), img)
        with open(p, "wb") as f:
            f.write(b"P6\n3 2\n255\n" + img.tobytes()[:-1])
        with pytest.raises(ValueError):
            ppm.read_ppm(p)
        with open(p, "wb") as f:
            f.write(b"P5\n3 2\n255\n" + img.tobytes())
        with pytest.raises(ValueError):
            ppm.read_ppm(p)
        with pytest.raises(ValueError):
            ppm.write_ppm(p, img.astype(np.int16))
