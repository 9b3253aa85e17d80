"""The two STENCIL Heun schemes (fused single launch, two-pass predictor/corrector) give bit-identical
steps; the autotuner picks one of them without touching the input."""
import numpy as np
import pytest

import paper_2605_26016_gb300 as sx
from workloads import random_spins

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_26016_gb300.build import build
    build()


CASES = [
    ("bcc_4shell", (13, 11, 9), (1, 1, 0)),
    ("bcc_4shell", (40, 30, 20), (1, 0, 1)),
    ("sc_j123_dmi", (17, 12, 10), (1, 1, 1)),
    ("sc_j123_dmi", (31, 29, 33), (1, 1, 0)),
    ("sc_j123", (70, 40, 25), (0, 1, 1)),
    ("sc_4shell", (37, 21, 15), (0, 0, 0)),
    ("sc_4shell", (40, 35, 18), (1, 1, 0)),
    ("sc_nn", (33, 5, 7), (1, 1, 1)),
    ("sc_nn", (64, 48, 40), (0, 0, 0)),
    # more tile columns than resident CTAs: the two-pass kernels run on the z-chunked grid
    # instead of the balanced column-plane schedule
    ("sc_j123_dmi", (640, 256, 6), (1, 1, 1)),
    ("bcc_4shell", (512, 256, 5), (1, 1, 1)),
]


@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_fused_and_two_pass_steps_are_bit_identical(case, thermal):
    name, n, pbc = CASES[case]
    s, w = sx.system_from_workload(name, n, pbc=pbc)
    S0 = torch.from_numpy(random_spins(s.nsub, n, 300 + case)).cuda()
    T = 120.0 if thermal else 0.0
    out = {}
    for scheme, launches in (("fused", 1), ("two_pass", 2)):
        sx.sx_set_stencil_scheme(s.ctx, scheme)
        info = s.plan("stencil", "fp32")
        assert info["launches_per_step"] == launches
        S = S0.clone()
        s.heun(S, torch.empty_like(S), dt=w["dt"], alpha=w["alpha"], T=T, seed=9, replica=2, step0=17, nsteps=3)
        torch.cuda.synchronize()
        out[scheme] = S.cpu().numpy()
    assert np.array_equal(out["fused"].view(np.uint64), out["two_pass"].view(np.uint64))


def test_scheme_switch_on_a_planned_context_and_autotune():
    n = (48, 40, 36)
    s, w = sx.system_from_workload("bcc_4shell", n)
    assert s.plan("stencil", "fp32")["launches_per_step"] == 2  # auto: two-pass
    sx.sx_set_stencil_scheme(s.ctx, "fused")
    assert s.info()["launches_per_step"] == 1
    with pytest.raises(sx.SxError):
        sx.sx_set_stencil_scheme(s.ctx, 9)
    assert s.info()["launches_per_step"] == 1
    S = torch.from_numpy(random_spins(2, n, 5)).cuda()
    keep = S.clone()
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=1)
    name, t = sx.sx_autotune(s.ctx, S, torch.empty_like(S), p, s.nsite, steps=3)
    assert name in ("fused", "two_pass")
    assert t["fused"] > 0 and t["two_pass"] > 0
    assert torch.equal(S, keep)
    assert s.info()["launches_per_step"] == (1 if name == "fused" else 2)
    # the gather backend has one scheme
    g, _ = sx.system_from_workload("bcc_4shell", (8, 8, 8))
    g.plan("gather", "fp32")
    S8 = torch.from_numpy(random_spins(2, (8, 8, 8), 5)).cuda()
    assert sx.sx_autotune(g.ctx, S8, torch.empty_like(S8), p, g.nsite)[0] == "fused"


@pytest.mark.parametrize("thermal", [False, True])
@pytest.mark.parametrize("name,n,pbc", [("sc_nn", (32, 32, 32), (1, 1, 1)), ("bcc_4shell", (13, 11, 9), (1, 1, 0)),
                                        ("sc_j123_dmi", (17, 12, 10), (1, 1, 1)), ("bcc_4shell", (40, 30, 20), (1, 0, 1))])
def test_persistent_multi_step_launch_equals_separate_steps(name, n, pbc, thermal):
    # on these few-column lattices sx_llg_heun_step runs all steps in one cooperative launch with a grid
    # barrier between the passes; sx_llg_heun_step_out launches each step's two passes separately
    s, w = sx.system_from_workload(name, n, pbc=pbc)
    sx.sx_set_stencil_scheme(s.ctx, "two_pass")
    s.plan("stencil", "fp32")
    S0 = torch.from_numpy(random_spins(s.nsub, n, 77)).cuda()
    T = 150.0 if thermal else 0.0
    p = sx.llg_params(w["dt"], w["alpha"], T, seed=4, replica=1)
    for nsteps in (2, 5):
        A = S0.clone()
        s.heun(A, torch.empty_like(A), dt=w["dt"], alpha=w["alpha"], T=T, seed=4, replica=1, step0=11, nsteps=nsteps)
        bufs = [S0.clone(), torch.empty_like(S0)]
        for k in range(nsteps):
            sx.sx_llg_heun_step_out(s.ctx, bufs[k & 1], bufs[(k + 1) & 1], p, 11 + k, s.nsite)
        torch.cuda.synchronize()
        sx.sx_device_status(s.ctx)
        assert torch.equal(A, bufs[nsteps & 1])


@pytest.mark.parametrize("scheme", ["fused", "two_pass"])
def test_heun_step_out_is_cuda_graph_capturable(scheme):
    # sx_llg_heun_step_out only enqueues kernels on the given stream (no synchronisation, no allocation
    # after planning), so a loop of steps can be captured once and replayed; the replay equals eager steps
    n = (48, 40, 36)
    s, w = sx.system_from_workload("sc_j123_dmi", n)
    sx.sx_set_stencil_scheme(s.ctx, scheme)
    s.plan("stencil", "fp32")
    S0 = torch.from_numpy(random_spins(1, n, 12)).cuda()
    A, B = S0.clone(), torch.empty_like(S0)
    p = sx.llg_params(w["dt"], w["alpha"], 0.0)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        sx.sx_llg_heun_step_out(s.ctx, A, B, p, 0, s.nsite, stream=stream)  # warm-up outside capture
        sx.sx_llg_heun_step_out(s.ctx, B, A, p, 1, s.nsite, stream=stream)
    stream.synchronize()
    A.copy_(S0)
    with torch.cuda.graph(g, stream=stream):
        sx.sx_llg_heun_step_out(s.ctx, A, B, p, 0, s.nsite, stream=stream)
        sx.sx_llg_heun_step_out(s.ctx, B, A, p, 1, s.nsite, stream=stream)
    A.copy_(S0)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    ref, tmp = S0.clone(), torch.empty_like(S0)
    for _ in range(3):
        sx.sx_llg_heun_step_out(s.ctx, ref, tmp, p, 0, s.nsite)
        sx.sx_llg_heun_step_out(s.ctx, tmp, ref, p, 1, s.nsite)
    torch.cuda.synchronize()
    assert torch.equal(A, ref)


def test_autotune_tile_shapes_keep_the_step_bit_identical():
    # every candidate (scheme x z chunk x launch shape) runs the same per-site arithmetic
    n = (40, 33, 29)
    s, w = sx.system_from_workload("sc_j123_dmi", n)
    s.plan("stencil", "fp32")
    S = torch.from_numpy(random_spins(1, n, 3)).cuda()
    p = sx.llg_params(w["dt"], w["alpha"], w["T"], seed=2)
    ref = torch.empty_like(S)
    sx.sx_llg_heun_step_out(s.ctx, S, ref, p, 4, s.nsite)
    name, t = sx.sx_autotune(s.ctx, S, torch.empty_like(S), p, s.nsite, steps=2)
    tiles = sx.sx_plan_tiles(s.ctx)
    assert tiles["scheme"] == {"fused": 1, "two_pass": 2}[name]
    assert tiles["tile_x"] > 0 and tiles["tile_y"] > 0 and tiles["ctas"] > 0
    assert min(v for v in t.values() if v > 0) > 0
    got = torch.empty_like(S)
    sx.sx_llg_heun_step_out(s.ctx, S, got, p, 4, s.nsite)
    assert torch.equal(got, ref)


@pytest.mark.parametrize("name,n", [("sc_j123_dmi", (40, 33, 29)), ("bcc_4shell", (24, 20, 17))])
def test_every_tile_shape_gives_the_same_step(name, n):
    s, w = sx.system_from_workload(name, n)
    s.plan("stencil", "fp32")
    S = torch.from_numpy(random_spins(s.nsub, n, 3)).cuda()
    p = sx.llg_params(w["dt"], w["alpha"], max(w["T"], 30.0), seed=2)
    ref = torch.empty_like(S)
    sx.sx_llg_heun_step_out(s.ctx, S, ref, p, 4, s.nsite)
    nz = n[2]
    shapes = [("fused", tz, 0, 0) for tz in (nz, 7, 3)]
    shapes += [("two_pass", tz, 0, r) for tz in (nz, 5) for r in (0, 1)]
    shapes += [("two_pass", nz, f, r) for f in (1, 2) for r in (0, 1)]
    for shape in shapes:
        sx.sx_set_tiles(s.ctx, *shape)
        t = sx.sx_plan_tiles(s.ctx)
        assert t["scheme"] == {"fused": 1, "two_pass": 2}[shape[0]] and t["regen_noise"] == shape[3]
        got = torch.empty_like(S)
        sx.sx_llg_heun_step_out(s.ctx, S, got, p, 4, s.nsite)
        assert torch.equal(got, ref), shape
    with pytest.raises(sx.SxError):
        sx.sx_set_tiles(s.ctx, "fused", nz + 1)


# Lattices with interior tiles (load region inside the lattice in x and y), whose planes the pass kernels
# stage with tensor copies: periodic, open z (planes beyond the faces read as zeros by the copy), all open
# with a partial last tile column, and two sublattices with a 2-cell halo.
@pytest.mark.parametrize("name,n,pbc", [("sc_j123_dmi", (96, 80, 24), (1, 1, 1)),
                                         ("sc_j123_dmi", (96, 80, 24), (1, 1, 0)),
                                         ("sc_j123_dmi", (100, 84, 21), (0, 0, 0)),
                                         ("bcc_4shell", (96, 72, 20), (1, 1, 1)),
                                         ("sc_4shell", (104, 50, 16), (1, 0, 1))])
def test_tensor_copied_planes_give_the_same_step_and_field(name, n, pbc):
    s, w = sx.system_from_workload(name, n, pbc=pbc)
    s.plan("stencil", "fp32")
    S = torch.from_numpy(random_spins(s.nsub, n, 5)).cuda()
    p = sx.llg_params(w["dt"], w["alpha"], max(w["T"], 30.0), seed=3)
    nz = n[2]
    assert sx.sx_plan_tiles(s.ctx)["tma_staging"] == 0  # the plan's default: every tile copies site by site
    sx.sx_set_tiles(s.ctx, "two_pass", nz, 0, 0, 0)
    ref = torch.empty_like(S)
    sx.sx_llg_heun_step_out(s.ctx, S, ref, p, 4, s.nsite)
    ref_b64 = s.field(S)
    ref_b32 = s.field(S, dtype=torch.float32)
    for shape, mask in [((nz, 0, 0), 3), ((5, 0, 1), 1), ((nz, 1, 0), 2), ((nz, 2, 1), 3)]:
        sx.sx_set_tiles(s.ctx, "two_pass", *shape, mask)
        assert sx.sx_plan_tiles(s.ctx)["tma_staging"] == mask
        got = torch.empty_like(S)
        sx.sx_llg_heun_step_out(s.ctx, S, got, p, 4, s.nsite)
        assert torch.equal(got, ref), (shape, mask)
        assert torch.equal(s.field(S), ref_b64), (shape, mask)
        assert torch.equal(s.field(S, dtype=torch.float32), ref_b32), (shape, mask)
    sx.sx_device_status(s.ctx)  # no bounded wait gave up


def test_tensor_copied_planes_need_rows_of_16_bytes():
    s, w = sx.system_from_workload("sc_j123_dmi", (90, 40, 12))
    s.plan("stencil", "fp32")
    assert sx.sx_plan_tiles(s.ctx)["tma_staging"] == 0
    with pytest.raises(sx.SxError):
        sx.sx_set_tiles(s.ctx, "two_pass", 12, 0, 0, 1)


# One overlapped launch per step (predictor and corrector units from a dependency-ordered queue) against
# the two pass launches: periodic and open faces, partial edge tiles, the last z chunk shorter than the
# others, 1- and 2-cell halos, stored and regenerated normals, both plane stagings, and three steps in a
# row (the queue and the done flags are reset by every step).
@pytest.mark.parametrize("name,n,pbc,tzs", [("sc_j123_dmi", (96, 80, 40), (1, 1, 1), (10, 7)),
                                             ("sc_j123_dmi", (100, 84, 21), (0, 0, 0), (5, 21)),
                                             ("sc_j123_dmi", (64, 48, 30), (1, 0, 1), (4, 30)),
                                             ("bcc_4shell", (64, 48, 24), (1, 1, 1), (6, 5)),
                                             ("sc_4shell", (96, 50, 26), (1, 1, 0), (7, 8))])
def test_overlapped_launch_gives_the_same_steps(name, n, pbc, tzs):
    s, w = sx.system_from_workload(name, n, pbc=pbc)
    s.plan("stencil", "fp32")
    S = torch.from_numpy(random_spins(s.nsub, n, 7)).cuda()
    p = sx.llg_params(w["dt"], w["alpha"], max(w["T"], 30.0), seed=5)
    nz = n[2]
    sx.sx_set_tiles(s.ctx, "two_pass", nz, 0, 0, 0)
    ref = S.clone()
    sx.sx_llg_heun_step(s.ctx, ref, torch.empty_like(S), p, 11, 3, s.nsite)
    for tz, regen, tma in [(tzs[0], 0, 3), (tzs[1], 1, 0), (tzs[0], 1, 1), (tzs[1], 0, 2)]:
        sx.sx_set_tiles(s.ctx, "two_pass", tz, 5, regen, tma)
        t = sx.sx_plan_tiles(s.ctx)
        assert t["ring_or_schedule"] == 5 and t["tile_z"] == tz and t["ctas"] > 0
        assert sx.sx_plan_info(s.ctx)["launches_per_step"] == 1
        got = S.clone()
        sx.sx_llg_heun_step(s.ctx, got, torch.empty_like(S), p, 11, 3, s.nsite)
        assert torch.equal(got, ref), (tz, regen, tma)
    sx.sx_device_status(s.ctx)  # no bounded wait gave up
    sx.sx_set_tiles(s.ctx, "two_pass", nz, 0, 0, 0)
    assert sx.sx_plan_info(s.ctx)["launches_per_step"] == 2


def test_overlapped_launch_needs_edge_tiles_as_wide_as_the_halo():
    s, w = sx.system_from_workload("sc_4shell", (65, 48, 20))  # halo 2, last tile column 1 cell wide
    s.plan("stencil", "fp32")
    with pytest.raises(sx.SxError):
        sx.sx_set_tiles(s.ctx, "two_pass", 5, 5, 0, 0)
    s2, _ = sx.system_from_workload("sc_4shell", (64, 48, 21))  # last z chunk of 1 plane
    s2.plan("stencil", "fp32")
    with pytest.raises(sx.SxError):
        sx.sx_set_tiles(s2.ctx, "two_pass", 5, 5, 0, 0)


# Host-array steps of the two-pass scheme pipeline chunked uploads and downloads against the passes; the
# results equal device steps bit for bit: periodic and open z, last chunk shorter than the others, 2-cell
# halos, one and several steps, a pageable host array, and the fused scheme (whole copies).
@pytest.mark.parametrize("name,n,pbc", [("sc_j123_dmi", (40, 36, 64), (1, 1, 1)),
                                         ("sc_j123_dmi", (33, 20, 30), (1, 1, 0)),
                                         ("sc_4shell", (40, 24, 37), (1, 1, 1)),
                                         ("bcc_4shell", (20, 18, 24), (1, 0, 1))])
@pytest.mark.parametrize("nsteps", [1, 3])
def test_pipelined_host_steps_equal_device_steps(name, n, pbc, nsteps):
    s, w = sx.system_from_workload(name, n, pbc=pbc)
    s.plan("stencil", "fp32")
    S = torch.from_numpy(random_spins(s.nsub, n, 12)).cuda()
    kw = dict(dt=w["dt"], alpha=w["alpha"], T=max(w["T"], 30.0), seed=4, step0=7, nsteps=nsteps)
    for scheme, pinned in [("two_pass", True), ("two_pass", False), ("fused", True)]:
        sx.sx_set_stencil_scheme(s.ctx, scheme)
        Sd = S.clone()
        s.heun(Sd, torch.empty_like(Sd), **kw)
        Sh = S.cpu()
        if pinned:
            Sh = Sh.pin_memory()
        s.heun_host(Sh, **kw)
        torch.cuda.synchronize()
        assert torch.equal(Sd.cpu(), Sh), (scheme, pinned)
