"""FP64 oracle of the convolutional path proposer (test infrastructure; only tests/, smoke() and bench.py's
CPU legs may import it).

The proposer maps an image of a minimum-energy-path chain, built by per-site spherical interpolation between
the endpoints (the geodesic interpolation of "Static optimization and minimum-energy paths"), to a better
guess of the converged image:

* input X (10 channels per site): the interpolated image I (3), endpoint A (3), endpoint B (3), the path
  coordinate s in [0, 1] (1);
* four 3x3x3 convolutions with zero padding and bias, 10 -> 16 -> 16 -> 16 -> 3 channels, ReLU after the
  first three;
* proposal P = N[I + Y] per site (Y the last convolution's output);
* loss L = mean over samples and sites of (1 - P . T), T the converged image.

Weights and the activations that feed a convolution are stored in BF16 (round to nearest, ties to even, of
the FP32 value); everything else, and every sum, is FP64 here.  Layout: [sample][channel][z][y][x];
weights [out][in][dz][dy][dx] with dz, dy, dx in {-1, 0, 1} at index 0, 1, 2.
"""
import numpy as np

CHANNELS = (10, 16, 16, 16, 3)


def bf16(x):
    """Round to BF16 (through FP32, round to nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    if nan.any():
        out = np.where(nan, f, out)
    return out.astype(np.float64)


def conv3d(x, w, b, dtype=np.float64):
    """out[n,o,z,y,x] = b[o] + sum_{c,dz,dy,dx} w[o,c,dz,dy,dx] x[n,c,z+dz-1,y+dy-1,x+dx-1], zero outside.

    dtype is the precision of the sums (float64; float32 gives one FP32 summation order, used only to measure
    how far FP32 accumulation in some order may move the result)."""
    n, c, nz, ny, nx = x.shape
    xp = np.zeros((n, c, nz + 2, ny + 2, nx + 2), dtype=dtype)
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((n, w.shape[0], nz, ny, nx), dtype=dtype)
    wd = np.asarray(w, dtype=dtype)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = xp[:, :, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                out += np.einsum("nczyx,oc->nozyx", sl, wd[:, :, dz, dy, dx])
    return (out + np.asarray(b, dtype=dtype)[None, :, None, None, None]).astype(np.float64)


def conv3d_backward(x, w, gout):
    """Gradients of sum(gout * conv3d(x, w, b)) with respect to x, w and b."""
    n, c, nz, ny, nx = x.shape
    xp = np.zeros((n, c, nz + 2, ny + 2, nx + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = xp[:, :, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                gw[:, :, dz, dy, dx] = np.einsum("nozyx,nczyx->oc", gout, sl)
                gxp[:, :, dz:dz + nz, dy:dy + ny, dx:dx + nx] += np.einsum("nozyx,oc->nczyx", gout, w[:, :, dz, dy, dx])
    gb = gout.sum(axis=(0, 2, 3, 4))
    return gxp[:, :, 1:-1, 1:-1, 1:-1], gw, gb


def make_input(I, A, B, s):
    """The 10-channel input of samples with interpolated images I, endpoints A, B (each [n,3,z,y,x]) and
    path coordinates s (n values)."""
    n = I.shape[0]
    sc = np.broadcast_to(np.asarray(s, dtype=np.float64).reshape(n, 1, 1, 1, 1), (n, 1) + I.shape[2:])
    return np.concatenate([I, A, B, sc], axis=1)


def forward(params, X, I, T=None, round_bf16=True, sum_dtype=np.float64):
    """Returns (P, loss or None, cache).  params: list of (w, b) for the four layers; sum_dtype as in conv3d."""
    rb = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    acts = [rb(X)]
    for l, (w, b) in enumerate(params):
        y = conv3d(acts[-1], rb(w), np.asarray(b, dtype=np.float64), dtype=sum_dtype)
        if l < len(params) - 1:
            acts.append(rb(np.maximum(y, 0.0)))
        else:
            Y = y
    Z = I + Y
    nrm = np.sqrt((Z * Z).sum(axis=1, keepdims=True))
    P = Z / nrm
    loss = None
    if T is not None:
        loss = float(np.mean(1.0 - (P * T).sum(axis=1)))
    return P, loss, (acts, Z, nrm, P)


def backward(params, cache, T, round_bf16=True):
    """Gradients [(gw, gb)] of the loss for the cache of forward(); the chain rule through the normalisation,
    the convolutions and the ReLUs (a ReLU passes the gradient where its stored output is positive)."""
    rb = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    acts, Z, nrm, P = cache
    m = T.shape[0] * np.prod(T.shape[2:])
    gP = -T / m
    gZ = (gP - (gP * P).sum(axis=1, keepdims=True) * P) / nrm
    g = gZ
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, b = params[l]
        gx, gw, gb = conv3d_backward(acts[l], rb(w), g)
        grads[l] = (gw, gb)
        if l > 0:
            g = gx * (acts[l] > 0)
    return grads


def interpolate(A, B, s):
    """Geodesic interpolation of one image between the endpoint fields A and B (each [3, ...], unit spins) at path
    coordinate s, site by site: the point at fraction s of the shorter great-circle arc from A_i to B_i,
    (sin((1-s) t) A + sin(s t) B) / sin t with t = atan2(|A x B|, A . B).  Where the two spins are parallel
    (|A x B| < 1e-6 and A . B > 0) the normalised linear blend is used; where they are antiparallel (|A x B| < 1e-6
    and A . B <= 0) every great circle is a geodesic and the one through u is taken, u the unit part of x-hat
    orthogonal to A (of y-hat where |A_x| >= 0.9): cos(pi s) A + sin(pi s) u."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    c = (A * B).sum(axis=0)
    w = np.cross(A, B, axis=0)
    sn = np.sqrt((w * w).sum(axis=0))
    t = np.arctan2(sn, c)
    gen = sn >= 1e-6
    safe = np.where(gen, np.sin(t), 1.0)
    slerp = (np.sin((1.0 - s) * t) * A + np.sin(s * t) * B) / safe
    blend = (1.0 - s) * A + s * B
    with np.errstate(invalid="ignore", divide="ignore"):
        blend = blend / np.sqrt((blend * blend).sum(axis=0))
    e = np.zeros_like(A)
    use_y = np.abs(A[0]) >= 0.9
    e[0] = np.where(use_y, 0.0, 1.0)
    e[1] = np.where(use_y, 1.0, 0.0)
    u = e - (A * e).sum(axis=0) * A
    u = u / np.sqrt((u * u).sum(axis=0))
    anti = np.cos(np.pi * s) * A + np.sin(np.pi * s) * u
    out = np.where(gen, slerp, np.where(c > 0, blend, anti))
    return out


def flatten(params):
    """The flat parameter vector: per layer the weights [out][in][3][3][3] then the biases, layers in order."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unflatten(flat, channels=CHANNELS):
    params, o = [], 0
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        w = np.asarray(flat[o:o + co * ci * 27], dtype=np.float64).reshape(co, ci, 3, 3, 3)
        o += co * ci * 27
        b = np.asarray(flat[o:o + co], dtype=np.float64)
        o += co
        params.append((w, b))
    return params


def adam_step(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, "Adam: a method for stochastic optimization", Algorithm 1) of the flat
    parameters theta with gradient g at step t >= 1; returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
