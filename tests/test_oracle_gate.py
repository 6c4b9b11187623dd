"""Pins of the FP64 gate oracle: finite differences, closed forms of the
convolution, BCE identities.  CPU only."""
import numpy as np
import pytest

from oracle import gate as G
from paper_1009_0959_gb300 import synth


def test_conv_delta_kernel_is_identity():
    rng = np.random.default_rng(0)
    x = rng.random((3, 7, 9))
    W = np.zeros((3, 3, 3, 3))
    for c in range(3):
        W[c, c, 1, 1] = 1.0
    np.testing.assert_allclose(G.conv3x3(x, W, np.zeros(3)), x)


def test_conv_shift_and_zero_padding():
    """A kernel with its single 1 at (u, v) = (0, 2) reads x[y-1, x+1]; rows
    and columns outside the image read 0."""
    x = np.arange(20, dtype=np.float64).reshape(1, 4, 5)
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, 0, 2] = 1.0
    z = G.conv3x3(x, W, np.array([0.5]))[0]
    ref = np.full((4, 5), 0.5)
    ref[1:, :4] += x[0, :3, 1:]
    np.testing.assert_allclose(z, ref)


def test_forward_closed_form_through_the_relus():
    """A hand-wired network whose logit has a closed form.  Layer 1 splits
    the centred red channel r = R/255 - 1/2 into a1[0] = max(r, 0) and
    a1[1] = max(-r, 0); layer 2 forms a2[0] = max(0.5 a1[1] - 0.1, 0) and
    a2[1] = max(a1[0] + 3 a1[1], 0); layer 3 weighs them 1 and 2, so
    z3 = max(0.5 max(-r, 0) - 0.1, 0) + 2 (max(r, 0) + 3 max(-r, 0)) and
    p = sigmoid(z3).  Without the first ReLU a2[1] would be max(-2r, 0),
    without the second a2[0] could go negative; an uncentred input, a bias
    after the ReLU or layer 2's [out][in] weights read as [in][out]
    (0.5 and 1 swapped) change it too."""
    R = np.array([[0, 12, 60, 76], [127, 128, 200, 255]], np.uint8)
    img = np.zeros(R.shape + (3,), np.uint8)
    img[..., 0] = R
    img[..., 1] = 77  # other channels: weight 0
    p = {name: np.zeros(shp) for name, shp in G.SHAPES}
    p["W1"][0, 0, 1, 1], p["W1"][1, 0, 1, 1] = 1.0, -1.0
    p["W2"][0, 1, 1, 1] = 0.5
    p["W2"][1, 0, 1, 1], p["W2"][1, 1, 1, 1] = 1.0, 3.0
    p["b2"][0] = -0.1
    p["W3"][0, 0, 1, 1], p["W3"][0, 1, 1, 1] = 1.0, 2.0
    c = G.forward(img, G.flatten(p))
    r = R / 255.0 - 0.5
    pos, neg = np.maximum(r, 0.0), np.maximum(-r, 0.0)
    z3 = np.maximum(0.5 * neg - 0.1, 0.0) + 2.0 * (pos + 3.0 * neg)
    np.testing.assert_allclose(c["z3"], z3, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(c["p"], 1.0 / (1.0 + np.exp(-z3)), rtol=1e-13)


def test_target_mask_rule():
    """A pixel is a target when some channel moved by more than the threshold
    (12 levels): 13 in one channel is, 12 is not, and 5 + 5 + 5 in three
    channels is not (the largest channel decides, not the sum)."""
    clean = np.full((1, 5, 3), 100, np.uint8)
    noisy = clean.copy()
    noisy[0, 1] = (113, 100, 100)
    noisy[0, 2] = (100, 88, 100)
    noisy[0, 3] = (105, 95, 105)
    noisy[0, 4] = (100, 100, 87)
    np.testing.assert_array_equal(G.target_mask(clean, noisy), [[0, 1, 0, 0, 1]])


def test_conv_grads_adjoint():
    """<dz, conv(x)> is linear in x and W: its gradients are the adjoints."""
    rng = np.random.default_rng(1)
    x = rng.random((2, 5, 6))
    W = rng.normal(size=(3, 2, 3, 3))
    dz = rng.normal(size=(3, 5, 6))
    dW, db, dx = G.conv3x3_grads(x, W, dz)
    f = lambda xx, WW: np.sum(dz * G.conv3x3(xx, WW, np.zeros(3)))  # noqa: E731
    np.testing.assert_allclose(np.sum(dx * x), f(x, W), rtol=1e-12)
    np.testing.assert_allclose(np.sum(dW * W), f(x, W), rtol=1e-12)
    np.testing.assert_allclose(db, dz.reshape(3, -1).sum(1))


def test_gradient_matches_finite_differences():
    clean, noisy = synth.noisy(6, 7, 0.3, 3)
    t = G.target_mask(clean, noisy)
    theta = G.init(5) * 0.7
    theta[G.NPARAM - 1] = 0.1
    cache = [G.forward(noisy, theta)]
    g = G.backward(cache, [t], theta)
    rng = np.random.default_rng(2)
    idx = np.concatenate([rng.choice(432, 8, replace=False), [432 + 3],
                          448 + rng.choice(2304, 8, replace=False), [2752 + 5],
                          2768 + rng.choice(144, 6, replace=False), [2912]])
    h = 1e-6
    for k in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        num = (G.loss([G.forward(noisy, tp)], [t]) - G.loss([G.forward(noisy, tm)], [t])) / (2 * h)
        assert abs(num - g[k]) <= 1e-6 * max(1.0, abs(num)) + 1e-9, (k, num, g[k])


def test_bce_closed_forms():
    """All-zero weights: p = sigmoid(b3) everywhere; the loss is the BCE of a
    constant; the b3 gradient is mean(p - t)."""
    clean, noisy = synth.noisy(5, 5, 0.4, 4)
    t = G.target_mask(clean, noisy)
    theta = np.zeros(G.NPARAM)
    theta[-1] = 0.3
    c = G.forward(noisy, theta)
    p = 1 / (1 + np.exp(-0.3))
    np.testing.assert_allclose(c["p"], p)
    np.testing.assert_allclose(G.loss([c], [t]), -np.mean(t * np.log(p) + (1 - t) * np.log(1 - p)))
    g = G.backward([c], [t], theta)
    assert g[-1] == pytest.approx(np.mean(p - t))
    assert np.all(g[:-1] == 0.0)


def test_bf16_round():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159, 1e-3])
    r = G.bf16_round(vals)
    np.testing.assert_array_equal(r[:2], [1.0, 1.0])       # tie to even
    assert r[2] == 1.0 + 2 ** -7                              # rounds up
    assert abs(r[3] + 3.14159) <= 2 ** -7 * 4
    assert abs(r[4] - 1e-3) <= 1e-3 * 2 ** -8


def test_bf16_activation_option():
    """act_bf16 only rounds the convolution inputs: exact for inputs already
    on the bfloat16 grid, within 2^-8 relative otherwise."""
    clean, noisy = synth.noisy(6, 6, 0.3, 8)
    theta = G.bf16_round(G.init(4))
    a = G.forward(noisy, theta)
    b = G.forward(noisy, theta, act_bf16=True)
    assert np.max(np.abs(a["z3"] - b["z3"])) < 0.05 * (1 + np.max(np.abs(a["z3"])))
    img = np.zeros((4, 5, 3), np.uint8)  # x0 = -0.5 exactly
    np.testing.assert_array_equal(G.forward(img, theta)["z1"], G.forward(img, theta, True)["z1"])
