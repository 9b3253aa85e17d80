"""GPU parity of the convolutional chain proposer (sx_cnn_*) against the FP64 oracle in oracle/cnn.py.

Tolerances.  Inputs, hidden activations and weights are BF16 on both sides; every convolution sums in FP32 on
the tensor cores and in FP64 in the oracle.  Where a hidden activation's exact value lies within the FP32 sum's
error of a BF16 rounding midpoint, the two sides may store neighbouring BF16 values, both correct roundings of
the definition; elsewhere they store the same value and the proposals differ only by the last layer's FP32 sum
(about 1e-8 here).  How far such flips move the proposals is measured on the oracle itself: the same forward
pass with FP32 sums in the oracle's own order (oracle.cnn.forward(..., sum_dtype=float32)) against FP64 sums.
The GPU must agree with the FP64 oracle at the bulk of the sites (median below 1e-6), may deviate by more than
1e-5 at no more than three times the oracle's own FP32 fraction plus 1%, and nowhere by more than ten times the
oracle's own largest FP32 deviation.  Gradients use split BF16 (hi + lo) operands for the activation gradients
and FP32 sums; they are compared in relative L2 norm per layer."""
import numpy as np
import pytest

from oracle import cnn
from workloads import cnn_init_params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26016_gb300.build import build
    build()


def sx():
    import paper_2605_26016_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def unit(a):
    return a / np.sqrt((a * a).sum(axis=1, keepdims=True))


def sample(n, nb, seed):
    """nb samples on an n = (nx, ny, nz) grid: endpoints A, B, interpolated images I, targets T near I."""
    rng = np.random.default_rng(seed)
    shape = (nb, 3, n[2], n[1], n[0])
    A = unit(rng.standard_normal(shape))
    B = unit(rng.standard_normal(shape))
    s = rng.uniform(0.1, 0.9, nb)
    I = np.stack([cnn.interpolate(A[b], B[b], s[b]) for b in range(nb)])
    T = unit(I + 0.3 * rng.standard_normal(shape))
    return A, B, I, T, s


def strong_params(seed):
    """Seeded weights with a last layer large enough that Y changes P at O(1), and non-zero biases."""
    rng = np.random.default_rng(seed + 100)
    p = cnn_init_params(seed)
    out = []
    for l, (w, b) in enumerate(p):
        out.append((w * (3.0 if l == 3 else 1.0), 0.05 * rng.standard_normal(b.shape)))
    flat32 = cnn.flatten(out).astype(np.float32)
    return flat32, cnn.unflatten(flat32.astype(np.float64))


def check_proposals(got, ref, params, X, I):
    d = np.abs(got - ref).max(axis=1)
    r32, _, _ = cnn.forward(params, X, I, sum_dtype=np.float32)
    d32 = np.abs(r32 - ref).max(axis=1)
    assert np.abs((got * got).sum(1) - 1).max() < 1e-14
    assert np.median(d) < 1e-6
    assert (d > 1e-5).mean() <= 3 * (d32 > 1e-5).mean() + 0.01
    assert d.max() <= 10 * d32.max() + 1e-6, (d.max(), d32.max())


def bf16_bits(x):
    return (np.asarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


SIZES = [((20, 18, 9), 3), ((5, 3, 2), 1), ((32, 16, 8), 2)]


@pytest.mark.parametrize("n,nb", SIZES)
def test_pack_is_bf16_of_the_input_bit_for_bit(n, nb):
    A, B, I, T, s = sample(n, nb, 1)
    P = sx().Proposer(n, nb)
    X = P.new_packed(nb)
    P.pack(dev(I), dev(A), dev(B), dev(s), X)
    got = X.cpu().numpy().view(np.uint16).reshape(nb, n[2], n[1], n[0], 16)
    ref = bf16_bits(cnn.bf16(cnn.make_input(I, A, B, s))).transpose(0, 2, 3, 4, 1)
    assert np.array_equal(got[..., :10], ref)
    assert not got[..., 10:].any()
    # shared endpoints
    X2 = P.new_packed(nb)
    P.pack(dev(I), dev(A[0]), dev(B[0]), dev(s), X2, shared_endpoints=True)
    ref2 = bf16_bits(cnn.bf16(cnn.make_input(I, np.broadcast_to(A[:1], A.shape), np.broadcast_to(B[:1], B.shape),
                                              s))).transpose(0, 2, 3, 4, 1)
    assert np.array_equal(X2.cpu().numpy().view(np.uint16).reshape(got.shape)[..., :10], ref2)
    P.close()


def test_interpolation_matches_oracle():
    n = (7, 5, 4)
    rng = np.random.default_rng(2)
    A = unit(rng.standard_normal((1, 3, 4, 5, 7)))[0]
    B = unit(rng.standard_normal((1, 3, 4, 5, 7)))[0]
    B[:, 0, 0, 0] = -A[:, 0, 0, 0]
    B[:, 1, 2, 3] = A[:, 1, 2, 3]
    A[:, 2, 1, 1] = [0.95, np.sqrt(1 - 0.95 ** 2), 0.0]
    B[:, 2, 1, 1] = -A[:, 2, 1, 1]
    nimg = 6
    chain = np.zeros((nimg, 3, 4, 5, 7))
    chain[0], chain[-1] = A, B
    c = dev(chain)
    P = sx().Proposer(n, nimg - 2)
    P.interpolate(c)
    got = c.cpu().numpy()
    for k in range(nimg):
        ref = A if k == 0 else B if k == nimg - 1 else cnn.interpolate(A, B, k / (nimg - 1))
        assert np.abs(got[k] - ref).max() < 1e-12, k
    P.close()


def _forward_both(n, nb, seed):
    A, B, I, T, s = sample(n, nb, seed)
    flat32, params = strong_params(seed)
    Pr = sx().Proposer(n, nb)
    Pr.set_params(flat32)
    X = Pr.new_packed(nb)
    Pr.pack(dev(I), dev(A), dev(B), dev(s), X)
    out = torch.empty((nb, 3) + (n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
    Pr.forward(X, dev(I), out)
    ref, loss, cache = cnn.forward(params, cnn.make_input(I, A, B, s), I, T)
    return Pr, X, (A, B, I, T, s), params, out.cpu().numpy(), ref, loss, cache


@pytest.mark.parametrize("n,nb", SIZES)
def test_forward_matches_oracle(n, nb):
    Pr, X, data, params, got, ref, _, _ = _forward_both(n, nb, 3)
    A, B, I, T, s = data
    check_proposals(got, ref, params, cnn.make_input(I, A, B, s), I)
    # the proposal really moved away from the interpolation
    assert np.abs(ref - data[2]).max() > 0.1
    Pr.close()


@pytest.mark.parametrize("n,nb", SIZES)
def test_loss_and_gradient_match_oracle(n, nb):
    Pr, X, (A, B, I, T, s), params, got, ref, loss, cache = _forward_both(n, nb, 4)
    grad = torch.empty(Pr.nparams, dtype=torch.float32, device="cuda")
    L = Pr.loss_grad(X, dev(I), dev(T), grad)
    assert L == pytest.approx(loss, rel=1e-4, abs=1e-7)
    g_ref = cnn.backward(params, cache, T)
    g = cnn.unflatten(grad.cpu().numpy().astype(np.float64))
    for l in range(4):
        for k in range(2):
            r, q = g_ref[l][k], g[l][k]
            rel = np.linalg.norm(q - r) / max(np.linalg.norm(r), 1e-30)
            assert rel < 5e-3, (l, k, rel)
    # deterministic: the same call gives the same bits
    grad2 = torch.empty_like(grad)
    assert Pr.loss_grad(X, dev(I), dev(T), grad2) == L
    assert torch.equal(grad, grad2)
    Pr.close()


def test_adam_matches_oracle():
    n = (8, 8, 4)
    rng = np.random.default_rng(5)
    flat32, _ = strong_params(5)
    Pr = sx().Proposer(n, 1)
    Pr.set_params(flat32)
    th, m, v = flat32.astype(np.float64), np.zeros(flat32.size), np.zeros(flat32.size)
    for t in (1, 2, 3):
        g = (rng.standard_normal(flat32.size) * 10.0 ** rng.uniform(-4, 0, flat32.size)).astype(np.float32)
        Pr.adam_step(1e-3, grad=dev(g))
        th, m, v = cnn.adam_step(th, m, v, g.astype(np.float64), t, 1e-3)
    got = Pr.get_params()
    assert np.abs(got - th).max() < 1e-6
    Pr.close()


def test_adam_updates_the_tensor_core_operands():
    # a training step must change what the forward pass computes
    n = (16, 16, 4)
    A, B, I, T, s = sample(n, 2, 6)
    flat32, _ = strong_params(6)
    Pr = sx().Proposer(n, 2)
    Pr.set_params(flat32)
    X = Pr.new_packed(2)
    Pr.pack(dev(I), dev(A), dev(B), dev(s), X)
    L0 = Pr.loss_grad(X, dev(I), dev(T))
    for _ in range(5):
        Pr.loss_grad(X, dev(I), dev(T))
        Pr.adam_step(3e-3)
    L1 = Pr.loss_grad(X, dev(I), dev(T))
    assert L1 < L0
    # the updated operands equal freshly built ones
    out1 = torch.empty((2, 3, 4, 16, 16), dtype=torch.float64, device="cuda")
    Pr.forward(X, dev(I), out1)
    Pr2 = sx().Proposer(n, 2)
    Pr2.set_params(Pr.get_params())
    out2 = torch.empty_like(out1)
    Pr2.forward(X, dev(I), out2)
    assert torch.equal(out1, out2)
    Pr.close()
    Pr2.close()


def test_propose_is_interpolation_then_forward():
    n = (20, 12, 6)
    rng = np.random.default_rng(7)
    A = unit(rng.standard_normal((1, 3, 6, 12, 20)))[0]
    B = unit(rng.standard_normal((1, 3, 6, 12, 20)))[0]
    nimg = 7
    chain = np.zeros((nimg, 3, 6, 12, 20))
    chain[0], chain[-1] = A, B
    flat32, params = strong_params(7)
    Pr = sx().Proposer(n, nimg - 2)
    Pr.set_params(flat32)
    c = dev(chain)
    Pr.propose(c)
    got = c.cpu().numpy()
    assert np.array_equal(got[0], A) and np.array_equal(got[-1], B)
    s = np.arange(1, nimg - 1) / (nimg - 1)
    I = np.stack([cnn.interpolate(A, B, v) for v in s])
    X = cnn.make_input(I, np.broadcast_to(A, I.shape), np.broadcast_to(B, I.shape), s)
    ref, _, _ = cnn.forward(params, X, I)
    check_proposals(got[1:-1], ref, params, X, I)
    Pr.close()


def test_batch_and_argument_errors():
    Pr = sx().Proposer((8, 8, 8), 2)
    X = Pr.new_packed(3)
    I = torch.zeros((3, 3, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(sx().SxError) as e:
        Pr.forward(X, I, I)
    assert e.value.code == sx().SX_ERR_ARG
    with pytest.raises(sx().SxError):
        Pr.adam_step(-1.0)
    Pr.close()


def _crop(n, z, y, x, r=4):
    """Slices of a crop of radius r around (z, y, x) inside a grid n = (nx, ny, nz): four 3x3x3 layers see r = 4
    sites away, so the crop's own zero padding lies only where the lattice has none or beyond the receptive
    field of the centre."""
    z0, y0, x0 = max(0, z - r), max(0, y - r), max(0, x - r)
    sl = (slice(z0, min(n[2], z + r + 1)), slice(y0, min(n[1], y + r + 1)), slice(x0, min(n[0], x + r + 1)))
    return sl, (z - z0, y - y0, x - x0)


def test_full_size_proposals_on_sampled_sites_and_batch_additivity():
    # the proposer at the chain size of the batched-path workload: 64^3 sites, 30 interior images
    n, nb = (64, 64, 64), 30
    rng = np.random.default_rng(11)
    shape = (3, n[2], n[1], n[0])
    A = unit(rng.standard_normal((1,) + shape))[0]
    B = unit(rng.standard_normal((1,) + shape))[0]
    s = (np.arange(nb) + 1) / (nb + 1)
    flat32, params = strong_params(11)
    Pr = sx().Proposer(n, nb)
    Pr.set_params(flat32)
    Ad, Bd = dev(A), dev(B)
    chain = torch.empty((nb + 2, 3, n[0] * n[1] * n[2]), dtype=torch.float64, device="cuda")
    chain[0].copy_(Ad.view(3, -1))
    chain[-1].copy_(Bd.view(3, -1))
    Pr.interpolate(chain)
    I = chain[1:-1].clone()
    X = Pr.new_packed(nb)
    Pr.pack(I, Ad, Bd, dev(s), X, shared_endpoints=True)
    P = torch.empty_like(I)
    Pr.forward(X, I, P)
    Pn = P.cpu().numpy().reshape((nb,) + shape)
    In = I.cpu().numpy().reshape((nb,) + shape)
    # sampled sites: corners, faces, interior, every image
    picks = [(b, int(rng.integers(0, n[2])), int(rng.integers(0, n[1])), int(rng.integers(0, n[0]))) for b in range(nb)]
    picks += [(0, 0, 0, 0), (nb - 1, n[2] - 1, n[1] - 1, n[0] - 1), (5, 0, 31, 63), (7, 63, 0, 17)]
    dev_ = []
    for b, z, y, x in picks:
        sl, c = _crop(n, z, y, x)
        Ac, Bc = A[(slice(None),) + sl], B[(slice(None),) + sl]
        Ic = cnn.interpolate(Ac, Bc, s[b])  # the oracle's own interpolation of the crop
        assert np.abs(In[b][(slice(None),) + sl] - Ic).max() < 1e-12
        ref, _, _ = cnn.forward(params, cnn.make_input(Ic[None], Ac[None], Bc[None], [s[b]]), Ic[None])
        dev_.append(np.abs(Pn[b][:, z, y, x] - ref[0][:, c[0], c[1], c[2]]).max())
    dev_ = np.array(dev_)
    assert np.median(dev_) < 1e-6 and dev_.max() < 2e-3, (np.median(dev_), dev_.max())
    assert np.abs((Pn * Pn).sum(1) - 1).max() < 1e-14
    # the loss gradient of the whole batch is the mean of the gradients of its two halves: the per-CTA
    # partials and their reduction over 7,680 blocks add up
    T = torch.from_numpy(unit(rng.standard_normal((nb,) + shape))).cuda().view(nb, 3, -1)
    g_all = torch.empty(Pr.nparams, dtype=torch.float32, device="cuda")
    g_a, g_b = torch.empty_like(g_all), torch.empty_like(g_all)
    L = Pr.loss_grad(X, I, T, g_all)
    h = nb // 2
    La = Pr.loss_grad(X[:h].contiguous(), I[:h].contiguous(), T[:h].contiguous(), g_a)
    Lb = Pr.loss_grad(X[h:].contiguous(), I[h:].contiguous(), T[h:].contiguous(), g_b)
    assert L == pytest.approx(0.5 * (La + Lb), rel=1e-12)
    ga, gb_, gall = g_a.cpu().numpy(), g_b.cpu().numpy(), g_all.cpu().numpy()
    assert np.linalg.norm(gall - 0.5 * (ga + gb_)) < 1e-5 * np.linalg.norm(gall)
    Pr.close()
