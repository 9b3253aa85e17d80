"""Seeded synthetic inputs shaped like the paper's workloads.

This module only describes inputs: lattice cells, sublattice positions, moments,
coupling constants and seeded random spin fields.  It holds none of the
method's arithmetic, so both the CUDA path and the CPU oracle may use it.

Workloads (all synthetic; the paper's benchmark lattices are synthetic too):

* ``sc_nn``      simple cubic, nearest-neighbour exchange J = 1 meV, B = 1 T along z,
                 mu = 1 mu_B, alpha = 0.1, periodic, deterministic Heun, dt = 0.1 fs.
* ``bcc_4shell`` bcc as two sublattices of the conventional cell, exchange on
                 four distance shells J = 20, 10, -1, 0.5 meV, mu = 2.2 mu_B,
                 uniaxial K = 0.005 meV along z, T = 300 K, alpha = 0.05, dt = 0.1 fs.
* ``sc_j123``    simple cubic, J1 = 1, J2 = -0.164, J3 = -0.082 meV on distance
                 shells, periodic in x, y and open in z, mu = 1 mu_B.
* ``sc_j123_dmi`` simple cubic, J1..J3 as above plus interfacial DMI D = 0.1 meV
                 on the first shell, mu = 2.2 mu_B, alpha = 0.1, T = 50 K, periodic.
* ``sc_4shell``  simple cubic, the frustrated four-shell exchange of the hopfion
                 calculation (J1 = 1 meV, J2/J1 = 0.188, J3/J1 = -0.274, J4/J1 = -0.161),
                 open boundaries, mu = 1 mu_B, alpha = 0.1, T = 10 K.

Spins are float64 arrays of shape (3, nsub, nz, ny, nx): three component planes,
sublattice-major, x fastest.  Random spins are uniform on the sphere:
z = 2u - 1, phi = 2 pi v with u, v from numpy's PCG64 seeded generator.
"""
import numpy as np

# lattice constant of the cubic cell in nm (bcc Fe); it only enters the dipolar term
A_NM = 0.287

SC_POS = [[0.0, 0.0, 0.0]]
BCC_POS = [[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]


def cubic_cell(a=A_NM):
    return (np.eye(3) * a).tolist()


WORKLOADS = {
    "sc_nn": dict(pos=SC_POS, mu=[1.0], shells=[1.0], dmi=None, B=[0.0, 0.0, 1.0], K=None,
                  alpha=0.1, T=0.0, dt=0.1, pbc=(1, 1, 1), seed=1),
    "bcc_4shell": dict(pos=BCC_POS, mu=[2.2, 2.2], shells=[20.0, 10.0, -1.0, 0.5], dmi=None, B=[0.0, 0.0, 0.0],
                       K=(0.005, [0.0, 0.0, 1.0]), alpha=0.05, T=300.0, dt=0.1, pbc=(1, 1, 1), seed=2),
    "sc_j123": dict(pos=SC_POS, mu=[1.0], shells=[1.0, -0.164, -0.082], dmi=None, B=[0.0, 0.0, 0.0], K=None,
                    alpha=0.1, T=0.0, dt=0.1, pbc=(1, 1, 0), seed=3),
    "sc_j123_dmi": dict(pos=SC_POS, mu=[2.2], shells=[1.0, -0.164, -0.082], dmi=(1, 0, 0.1), B=[0.0, 0.0, 0.0],
                        K=None, alpha=0.1, T=50.0, dt=0.1, pbc=(1, 1, 1), seed=5),
    "sc_4shell": dict(pos=SC_POS, mu=[1.0], shells=[1.0, 0.188, -0.274, -0.161], dmi=None, B=[0.0, 0.0, 0.0],
                      K=None, alpha=0.1, T=10.0, dt=0.1, pbc=(0, 0, 0), seed=7),
}


def random_spins(nsub, n, seed):
    """Uniform random unit spins, shape (3, nsub, nz, ny, nx), float64."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    m = nsub * nx * ny * nz
    u = rng.random(m)
    v = rng.random(m)
    z = 2.0 * u - 1.0
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = 2.0 * np.pi * v
    S = np.stack([r * np.cos(phi), r * np.sin(phi), z]).reshape(3, nsub, nz, ny, nx)
    return np.ascontiguousarray(S)


def hopf_ansatz(n, radius, center=None):
    """Toroidal Hopf-map texture with Hopf index 1 on a simple-cubic grid, shape (3, 1, nz, ny, nx).

    A degree-1 map of space into the 3-sphere, q = (cos f(r), sin f(r) r/|r|) with
    f = pi (1 - r/radius) inside the ball and 0 outside, composed with the Hopf
    projection Z1 = q0 + i q3, Z2 = q1 + i q2 ->
    S = (2 Re Z1 conj(Z2), 2 Im Z1 conj(Z2), |Z1|^2 - |Z2|^2).  S -> +z far away; the
    preimage of -z is the ring r = radius/2 in the plane through the centre.
    """
    nx, ny, nz = n
    c = np.asarray(center if center is not None else [(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2], dtype=np.float64)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    rx, ry, rz = x - c[0], y - c[1], z - c[2]
    r = np.sqrt(rx * rx + ry * ry + rz * rz)
    f = np.where(r < radius, np.pi * (1.0 - r / radius), 0.0)
    inv = np.where(r > 0, 1.0 / np.where(r > 0, r, 1.0), 0.0)
    q0 = np.cos(f)
    sf = np.sin(f) * inv
    q1, q2, q3 = sf * rx, sf * ry, sf * rz
    z1 = q0 + 1j * q3
    z2 = q1 + 1j * q2
    w = z1 * np.conj(z2)
    S = np.stack([2 * w.real, 2 * w.imag, np.abs(z1) ** 2 - np.abs(z2) ** 2])
    S /= np.sqrt((S * S).sum(0))
    return np.ascontiguousarray(S.reshape(3, 1, nz, ny, nx))


def uniform_spins(nsub, n, direction):
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.sqrt((d * d).sum())
    nx, ny, nz = n
    S = np.empty((3, nsub, nz, ny, nx))
    for c in range(3):
        S[c] = d[c]
    return S


def polar_chain(theta_a, theta_b, nimg, phi_bulge=0.0):
    """A chain of nimg single-spin states S = (sin t cos p, sin t sin p, cos t), shape (nimg, 3, 1, 1, 1, 1):
    t runs linearly from theta_a to theta_b, p = phi_bulge * sin(pi s) for s = n/(nimg-1), so the
    endpoints lie in the x-z plane and the interior bulges towards +y."""
    s = np.linspace(0.0, 1.0, nimg)
    t = theta_a + (theta_b - theta_a) * s
    p = phi_bulge * np.sin(np.pi * s)
    S = np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)], axis=1)
    return np.ascontiguousarray(S.reshape(nimg, 3, 1, 1, 1, 1))


def nlerp_chain(A, B, nimg, jitter=0.0, seed=0):
    """A chain of nimg spin fields between A and B (same shape): image n is the site-wise
    normalised linear blend (1 - s) A + s B, s = n/(nimg-1), plus optional seeded Gaussian
    jitter on the interior images.  Endpoints are A and B unchanged.  Antiparallel site
    pairs are tilted by a fixed small vector before normalising."""
    rng = np.random.default_rng(seed)
    out = np.empty((nimg,) + A.shape)
    tilt = np.zeros_like(A)
    tilt[0] = 1e-3
    for n in range(nimg):
        s = n / (nimg - 1)
        if n == 0:
            out[n] = A
            continue
        if n == nimg - 1:
            out[n] = B
            continue
        X = (1.0 - s) * A + s * B + tilt
        if jitter:
            X = X + jitter * rng.standard_normal(A.shape)
        out[n] = X / np.sqrt((X * X).sum(0))
    return np.ascontiguousarray(out)


def dense_window_bonds(seed=9, radius=3):
    """A 3x3 tensor coupling on every cell offset of the (2 radius + 1)^3 window of one sublattice (the
    genuinely dense kernel the tensor-core backend is for): J(d) = g I / (1 + |d|^2) + 0.02 G, g and G standard
    normal from numpy's PCG64 seeded generator, one unordered bond per offset pair (d, -d)."""
    rng = np.random.default_rng(seed)
    bonds = []
    w = 2 * radius + 1
    for d in np.ndindex(w, w, w):
        d = tuple(int(v) - radius for v in d)
        if d > (0, 0, 0):
            bonds.append((0, 0, d, np.eye(3) * rng.normal() / (1.0 + sum(v * v for v in d))
                          + 0.02 * rng.normal(size=(3, 3))))
    return bonds


def random_spins_torch(nsub, n, seed, device="cuda"):
    """Uniform random unit spins generated on a torch device (for lattices too large to generate in
    numpy in reasonable time), shape (3, nsub, nz, ny, nx), float64: z = 2u - 1, phi = 2 pi v with u, v
    from torch's seeded Philox generator of that device.  Not the same numbers as random_spins."""
    import torch
    nx, ny, nz = n
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    m = nsub * nx * ny * nz
    S = torch.empty((3, m), dtype=torch.float64, device=device)
    u = torch.rand(m, generator=g, device=device, dtype=torch.float64)
    S[2] = 2.0 * u - 1.0
    r = torch.sqrt(torch.clamp(1.0 - S[2] * S[2], min=0.0))
    u = torch.rand(m, generator=g, device=device, dtype=torch.float64)
    u.mul_(2.0 * np.pi)
    torch.cos(u, out=S[0])
    S[0].mul_(r)
    torch.sin(u, out=S[1])
    S[1].mul_(r)
    del u, r
    return S.view(3, nsub, nz, ny, nx)


CNN_CHANNELS = (10, 16, 16, 16, 3)


def cnn_init_params(seed, channels=CNN_CHANNELS):
    """Initial weights of the path proposer's four 3x3x3 convolutions: He-normal (std sqrt(2 / (27 c_in)))
    from numpy's PCG64 seeded generator, the last layer scaled by 0.1 so that the untrained proposer stays
    close to the interpolation; zero biases.  List of (w [out][in][3][3][3], b [out]) in float64."""
    rng = np.random.default_rng(seed)
    params = []
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        w = rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci))
        if l == len(channels) - 2:
            w *= 0.1
        params.append((w, np.zeros(co)))
    return params


def cnn_init_flat(seed, channels=CNN_CHANNELS):
    """cnn_init_params as one float32 vector in the proposer's parameter order (per layer the weights, then the
    biases, layers in order)."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in cnn_init_params(seed, channels)]).astype(
        np.float32)
