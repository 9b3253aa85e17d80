"""Pins for the oracle of the convolutional path proposer: convolution against scipy, gradients against
finite differences, BF16 rounding against torch, and the loss's fixed points."""
import numpy as np
import pytest

from oracle import cnn
from workloads import cnn_init_params


def test_conv3d_matches_scipy_correlate():
    from scipy import ndimage
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 1, 5, 6, 7))
    w = rng.standard_normal((1, 1, 3, 3, 3))
    got = cnn.conv3d(x, w, np.array([0.25]))[0, 0]
    ref = ndimage.correlate(x[0, 0], w[0, 0], mode="constant", cval=0.0) + 0.25
    assert np.abs(got - ref).max() < 1e-12
    # channels mix linearly
    x2 = rng.standard_normal((2, 3, 4, 4, 4))
    w2 = rng.standard_normal((2, 3, 3, 3, 3))
    ref2 = sum(ndimage.correlate(x2[1, c], w2[1, c], mode="constant") for c in range(3))
    assert np.abs(cnn.conv3d(x2, w2, np.zeros(2))[1, 1] - ref2).max() < 1e-12


def test_conv3d_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 4, 3, 5))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    g = rng.standard_normal((2, 2, 4, 3, 5))
    f = lambda x_, w_, b_: float((g * cnn.conv3d(x_, w_, b_)).sum())
    gx, gw, gb = cnn.conv3d_backward(x, w, g)
    h = 1e-6
    for idx in [(0, 0, 0, 0, 0), (1, 2, 3, 2, 4), (0, 1, 2, 1, 2)]:
        e = np.zeros_like(x)
        e[idx] = h
        assert (f(x + e, w, b) - f(x - e, w, b)) / (2 * h) == pytest.approx(gx[idx], rel=1e-7, abs=1e-8)
    for idx in [(0, 0, 0, 0, 0), (1, 2, 1, 2, 0), (0, 1, 2, 2, 2)]:
        e = np.zeros_like(w)
        e[idx] = h
        assert (f(x, w + e, b) - f(x, w - e, b)) / (2 * h) == pytest.approx(gw[idx], rel=1e-7, abs=1e-8)
    e = np.zeros_like(b)
    e[1] = h
    assert (f(x, w, b + e) - f(x, w, b - e)) / (2 * h) == pytest.approx(gb[1], rel=1e-7)


def _unit(a):
    return a / np.sqrt((a * a).sum(axis=1, keepdims=True))


def test_proposer_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    n, shape = 2, (4, 3, 4)
    I, A, B, T = (_unit(rng.standard_normal((n, 3) + shape)) for _ in range(4))
    X = cnn.make_input(I, A, B, [0.3, 0.7])
    params = [(w * 3.0, rng.standard_normal(b.shape) * 0.1) for w, b in cnn_init_params(5)]
    P, loss, cache = cnn.forward(params, X, I, T, round_bf16=False)
    grads = cnn.backward(params, cache, T, round_bf16=False)
    h = 1e-6
    for l, idx in [(0, (3, 7, 1, 2, 0)), (1, (5, 9, 2, 1, 1)), (2, (0, 15, 0, 0, 2)), (3, (2, 4, 1, 1, 1))]:
        w, b = params[l]
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        lp = cnn.forward(params[:l] + [(wp, b)] + params[l + 1:], X, I, T, round_bf16=False)[1]
        lm = cnn.forward(params[:l] + [(wm, b)] + params[l + 1:], X, I, T, round_bf16=False)[1]
        assert (lp - lm) / (2 * h) == pytest.approx(grads[l][0][idx], rel=2e-5, abs=1e-9)
    w, b = params[3]
    bp, bm = b.copy(), b.copy()
    bp[1] += h
    bm[1] -= h
    lp = cnn.forward(params[:3] + [(w, bp)], X, I, T, round_bf16=False)[1]
    lm = cnn.forward(params[:3] + [(w, bm)], X, I, T, round_bf16=False)[1]
    assert (lp - lm) / (2 * h) == pytest.approx(grads[3][1][1], rel=2e-5)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, 65504.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16(x), ref)


def test_loss_vanishes_on_the_target_and_is_bounded():
    rng = np.random.default_rng(4)
    I = _unit(rng.standard_normal((1, 3, 3, 3, 3)))
    params = [(np.zeros_like(w), np.zeros_like(b)) for w, b in cnn_init_params(0)]
    X = cnn.make_input(I, I, I, [0.5])
    P, loss, _ = cnn.forward(params, X, I, I)
    assert np.abs(P - I).max() < 1e-15 and loss == pytest.approx(0.0, abs=1e-15)
    _, loss2, _ = cnn.forward(params, X, I, -I)
    assert loss2 == pytest.approx(2.0)


def test_interpolation_is_constant_speed_on_the_great_circle():
    rng = np.random.default_rng(6)
    A = _unit(rng.standard_normal((1, 3, 5, 4, 3)))[0]
    B = _unit(rng.standard_normal((1, 3, 5, 4, 3)))[0]
    B[:, 0, 0, 0] = -A[:, 0, 0, 0]          # antiparallel site
    B[:, 1, 0, 0] = A[:, 1, 0, 0]           # parallel site
    ang = lambda X, Y: np.arctan2(np.sqrt((np.cross(X, Y, axis=0) ** 2).sum(0)), (X * Y).sum(0))
    th = ang(A, B)
    assert np.abs(cnn.interpolate(A, B, 0.0) - A).max() < 1e-15
    assert np.abs(cnn.interpolate(A, B, 1.0)[:, 1:] - B[:, 1:]).max() < 1e-12
    for s in (0.2, 0.5, 0.85):
        I = cnn.interpolate(A, B, s)
        assert np.abs((I * I).sum(0) - 1).max() < 1e-14
        # angle from A is s * theta, from B (1 - s) * theta: I lies on the shorter arc
        assert np.abs(ang(A, I) - s * th).max() < 1e-9
        assert np.abs(ang(I, B) - (1 - s) * th)[1:].max() < 1e-9
        # in the plane of A and B (generic sites)
        n = np.cross(A, B, axis=0)
        assert np.abs((n * I).sum(0)[1:]).max() < 1e-12
        # antiparallel site: quarter turns through the x-hat direction orthogonal to A
        a = A[:, 0, 0, 0]
        u = np.array([1.0, 0.0, 0.0]) - a[0] * a
        u /= np.linalg.norm(u)
        assert np.abs(I[:, 0, 0, 0] - (np.cos(np.pi * s) * a + np.sin(np.pi * s) * u)).max() < 1e-14


def test_flatten_round_trip_and_size():
    p = cnn_init_params(3)
    f = cnn.flatten(p)
    assert f.size == 19491
    q = cnn.unflatten(f)
    assert all(np.array_equal(a, c) and np.array_equal(b, d) for (a, b), (c, d) in zip(p, q))


def test_adam_constant_gradient_moves_by_lr_times_sign():
    # with bias correction, a constant gradient gives mhat = g and vhat = g^2 at every step, so each update
    # is lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    th, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in (1, 2, 3):
        prev = th
        th, m, v = cnn.adam_step(th, m, v, g, t, lr=0.01)
        assert np.abs((th - prev) - (-0.01 * g / (np.abs(g) + 1e-8))).max() < 1e-15
