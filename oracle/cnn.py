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


def conv3d(x, w, b):
    """out[n,o,z,y,x] = b[o] + sum_{c,dz,dy,dx} w[o,c,dz,dy,dx] x[n,c,z+dz-1,y+dy-1,x+dx-1], zero outside."""
    n, c, nz, ny, nx = x.shape
    xp = np.zeros((n, c, nz + 2, ny + 2, nx + 2))
    xp[:, :, 1:-1, 1:-1, 1:-1] = x
    out = np.zeros((n, w.shape[0], nz, ny, nx))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                sl = xp[:, :, dz:dz + nz, dy:dy + ny, dx:dx + nx]
                out += np.einsum("nczyx,oc->nozyx", sl, w[:, :, dz, dy, dx])
    return out + b[None, :, None, None, None]


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


def forward(params, X, I, T=None, round_bf16=True):
    """Returns (P, loss or None, cache).  params: list of (w, b) for the four layers."""
    rb = bf16 if round_bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    acts = [rb(X)]
    for l, (w, b) in enumerate(params):
        y = conv3d(acts[-1], rb(w), np.asarray(b, dtype=np.float64))
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
