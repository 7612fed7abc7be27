"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

import oracle as O
from paper_1807_02137_gb300 import synth
from tests.gpu_common import gpu_solver, need_gpu, oracle_params, relmax, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def segmg():
    return need_gpu()


def both(segmg, image, markers, **kw):
    s, p = gpu_solver(segmg, image, markers, **kw)
    o = O.Solver(np.asarray(image, dtype=np.float64), markers, oracle_params(*image.shape, p))
    return s, o, p


@pytest.mark.parametrize("shape", [(128, 128), (100, 77), (37, 53)])
def test_setup_fields_fp64(segmg, shape):
    n, m = shape
    img, mk, _ = synth.disc_square(max(n, m), 0.05, 0)
    img = img[:n, :m].copy()
    mk = mk[(mk[:, 0] <= m - 1) & (mk[:, 1] <= n - 1)]
    s, o, p = both(segmg, img, mk, precision=segmg.MG_F64, levels=3)
    for l in range(3):
        for f in ("w", "z", "d"):
            assert relmax(s.level(l, f).cpu().numpy(), o.level(l, f)) < 1e-13, (l, f)
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-13
    st, so = s.stats(), o.scalars()
    assert abs(st["c1"] - so["c1"]) < 1e-12 and abs(st["c2"] - so["c2"]) < 1e-12
    assert abs(st["A1"] - so["A1"]) < 1e-9


@pytest.mark.parametrize("smoother", [0, 1])
def test_vcycles_fp64_match_oracle(segmg, smoother):
    W = synth.workload("disc128")
    s, o, p = both(segmg, W.image, W.markers, precision=segmg.MG_F64, levels=W.levels,
                   smoother=smoother)
    r0g, r0o = s.begin_step(), o.begin_step()
    assert abs(r0g - r0o) <= 1e-12 * r0o
    for l in range(W.levels):   # fitting field minus phi^n / tau on every grid
        Fg = s.level(l, "F").cpu().numpy() - s.level(l, "phi").cpu().numpy() / p.tau
        assert relmax(Fg, o.level(l, "Fn")) < 1e-12, l
    for c in range(3):
        rg, ro = s.vcycle(), o.vcycle()
        assert abs(rg - ro) <= 1e-8 * ro, (c, rg, ro)
        assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-10, c


def test_fp64_first_step_to_1e8_matches_oracle(segmg):
    W = synth.workload("disc128")
    s, o, p = both(segmg, W.image, W.markers, precision=segmg.MG_F64, levels=W.levels)
    cyc, rho = s.solve_step(W.tol, 60)
    o.set_tau(s.stats()["tau"])      # the tau the step control accepted (the step from phi^n)
    hist = o.solve_step(W.tol, 60)
    o.end_step()
    assert rho <= W.tol and hist[-1] <= W.tol
    if s.stats()["attempts_rejected"] == 0:
        assert abs(cyc - len(hist)) <= 1
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-9
    st, so = s.stats(), o.scalars()
    assert abs(st["c1"] - so["c1"]) < 1e-10 and abs(st["c2"] - so["c2"]) < 1e-10


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_fused_and_phased_smoothers_are_bitwise_equal(segmg, precision):
    prec = segmg.MG_F64 if precision == "f64" else segmg.MG_F32
    img, mk, _ = synth.ellipses(200, 170, 6, (20, 80), 6, 0.05, 7)
    outs = []
    for sm in (0, 1, 2):   # TMA-staged fused sweep (FP32) / per-phase kernels / vector-load fused sweep
        s, _ = gpu_solver(segmg, img, mk, precision=prec, levels=4, smoother=sm)
        s.begin_step()
        for _ in range(2):
            s.vcycle()
        outs.append(s.phi().cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_fp32_solution_matches_oracle_small(segmg):
    img, mk, _ = synth.ellipses(256, 256, 12, (10, 60), 8, 0.05, 11)
    s, o, p = both(segmg, img.astype(np.float32), mk, precision=segmg.MG_F32, levels=7)
    cyc, rho = s.solve_step(1e-6, 60)
    o.set_tau(s.stats()["tau"])
    hist = o.solve_step(1e-9, 80)
    assert rho <= 1e-6 and hist[-1] <= 1e-9
    pg, po = s.phi().cpu().numpy(), o.phi
    assert relmax(pg, po) < 1e-5
    assert np.mean((pg > 0) != (po > 0)) <= 1e-4


def test_rada_chen_fp64_matches_oracle(segmg):
    img, mk, _ = synth.disc_square(96, 0.05, 2)
    s, o, p = both(segmg, img, mk, precision=segmg.MG_F64, levels=4, model=segmg.MG_MODEL_RC)
    s.begin_step(); o.begin_step()
    for c in range(3):
        rg, ro = s.vcycle(), o.vcycle()
        assert abs(rg - ro) <= 1e-8 * ro
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-10


def test_multi_step_fp64_with_region_update(segmg):
    W = synth.workload("disc128")
    s, o, p = both(segmg, W.image, W.markers, precision=segmg.MG_F64, levels=W.levels)
    for step in range(3):
        s.begin_step(); o.begin_step()
        for _ in range(4):
            s.vcycle(); o.vcycle()
        eg, eo = s.end_step(), o.end_step()
        assert abs(eg - eo) <= 1e-9 * eo
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-9
    m = s.mask().cpu().numpy()
    assert np.array_equal(m.astype(bool), o.phi > 0)


@pytest.mark.parametrize("shape,levels", [((1, 1), 1), ((2, 3), 1), ((5, 4), 2), ((33, 65), 4)])
def test_tiny_and_ragged_grids(segmg, shape, levels):
    n, m = shape
    rng = np.random.default_rng(n * 100 + m)
    img = rng.uniform(0, 1, (n, m))
    mk = np.array([[m // 2, n // 2]], dtype=float)
    s, o, p = both(segmg, img, mk, precision=segmg.MG_F64, levels=levels)
    s.begin_step(); o.begin_step()
    for _ in range(2):
        rg, ro = s.vcycle(), o.vcycle()
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-10


def test_degenerate_markers(segmg):
    img, _, _ = synth.disc_square(64, 0.05, 3)
    for mk in ([[20, 30]], [[10, 10], [20, 20], [30, 30]]):
        s, o, p = both(segmg, img, np.array(mk, float), precision=segmg.MG_F64, levels=4)
        assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-13
        assert abs(s.stats()["A1"] - o.scalars()["A1"]) < 1e-9


def test_repeated_runs_are_bitwise_identical(segmg):
    img, mk, _ = synth.ellipses(192, 192, 8, (20, 80), 6, 0.05, 5)
    outs = []
    for _ in range(2):
        s, _ = gpu_solver(segmg, img, mk, levels=6)
        s.solve_step(1e-6, 40)
        outs.append(s.phi().cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_graph_and_eager_launches_agree(segmg):
    img, mk, _ = synth.ellipses(160, 160, 8, (20, 60), 6, 0.05, 9)
    outs = []
    for g in (0, 1):
        s, _ = gpu_solver(segmg, img, mk, levels=6, use_graph=g)
        s.begin_step()
        for _ in range(3):
            s.vcycle()
        outs.append(s.phi().cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_device_step_loop_equals_host_driven_step(segmg):
    # a whole pseudo-time step run as one graph launch (the device step loop, whose V-cycle norm
    # is computed by the next V-cycle's first snapshot) and the same step run V-cycle by V-cycle
    # from the host with eager launches (the separate norm kernel): same V-cycles, same rho,
    # same phi, bitwise; FP32 and mixed storage
    img, mk, _ = synth.ellipses(192, 176, 8, (16, 70), 6, 0.05, 19)
    for prec in (segmg.MG_F32, segmg.MG_MIXED):
        res = []
        for g in (1, 0):
            s, _ = gpu_solver(segmg, img, mk, precision=prec, levels=6, use_graph=g)
            cyc, rho = s.solve_step(1e-6, 50)
            res.append((cyc, rho, s.phi().cpu().numpy(), s.stats()["tau"]))
            s.close()
        assert res[0][0] == res[1][0] and res[0][1] == res[1][1] and res[0][3] == res[1][3]
        assert np.array_equal(res[0][2], res[1][2])
        assert res[0][1] <= 1e-6


def test_host_pipeline_matches_device_pipeline(segmg):
    img, mk, _ = synth.ellipses(256, 256, 10, (20, 80), 8, 0.05, 4)
    p = segmg.default_params(256, 256)
    mask_h, phi_h, st = segmg.segment_host(img, mk, p, 1e-6, 50, 0.0, 1, want_phi=True)
    s, _ = gpu_solver(segmg, img, mk)
    s.solve_step(1e-6, 50)
    assert np.array_equal(phi_h, s.phi().cpu().numpy())
    assert np.array_equal(mask_h, s.mask().cpu().numpy())
    assert st["steps"] == 1 and st["rho"] <= 1e-6


def test_host_pipeline_kept_context_equals_a_fresh_one(segmg):
    # mg_segment_host keeps its handle between calls of one size: a second image through the kept
    # context, a size change, and a marker-count change give bitwise what a fresh context gives
    imgs = [synth.ellipses(192, 160, 8, (16, 60), 6, 0.05, s)[:2] for s in (21, 22)]
    other = synth.ellipses(96, 128, 6, (10, 40), 5, 0.05, 23)[:2]
    p = segmg.default_params(192, 160)
    p2 = segmg.default_params(96, 128)

    def run(img, mk, params, fresh):
        if fresh:
            segmg.segment_host_release()
        mask_out = np.empty(img.shape, dtype=np.uint8)
        mask, phi, st = segmg.segment_host(img, mk, params, 1e-6, 50, 0.0, 1, want_phi=True, mask_out=mask_out)
        assert mask is mask_out
        return mask.copy(), phi, st

    fresh = [run(i, m, p, True) for i, m in imgs] + [run(other[0], other[1], p2, True)]
    segmg.segment_host_release()
    kept = [run(i, m, p, False) for i, m in imgs] + [run(other[0], other[1], p2, False)]
    # more markers than the kept context was set up for: a new context
    mk_many = np.array([[20 + 7 * q, 30 + 5 * q] for q in range(20)], dtype=float)
    many_kept = run(imgs[0][0], mk_many, p, False)
    many_fresh = run(imgs[0][0], mk_many, p, True)
    for a, b in zip(kept + [many_kept], fresh + [many_fresh]):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert a[2]["cycles_total"] == b[2]["cycles_total"] and a[2]["rho"] == b[2]["rho"]
    segmg.segment_host_release()


def test_errors_are_reported_not_raised_on_the_gpu(segmg):
    img, mk, _ = synth.disc_square(64, 0.05, 0)
    bad = img.copy()
    bad[3, 4] = np.nan
    with pytest.raises(segmg.SegmgError) as e:
        gpu_solver(segmg, bad, mk, precision=segmg.MG_F64)
    assert e.value.code == -2
    with pytest.raises(segmg.SegmgError) as e:
        gpu_solver(segmg, img, np.array([[70.0, 3.0]]), precision=segmg.MG_F64)
    assert e.value.code == -1
    with pytest.raises(segmg.SegmgError) as e:
        gpu_solver(segmg, img, mk, precision=segmg.MG_F64, levels=4, Sigma=0.5)
    assert e.value.code == -1
    with pytest.raises(segmg.SegmgError) as e:      # coarsest grid too large for the direct solve
        gpu_solver(segmg, np.zeros((256, 256)), mk, precision=segmg.MG_F64, levels=2)
    assert e.value.code == -1
    s, _ = gpu_solver(segmg, img, mk, precision=segmg.MG_F64, levels=4)
    with pytest.raises(segmg.SegmgError) as e:
        s.vcycle()
    assert e.value.code == -8
    s.begin_step()
    s.vcycle()          # the handle is still usable after a rejected call


def test_mixed_precision_error_vs_oracle(segmg):
    # w held in BF16, everything else as the FP32 path: the error against the FP64 oracle is
    # stated, not hidden (measured ~1e-6 on 2048^2 crops of the 25000^2 workload); the bound
    # asserted here is 1e-4 relative on phi and 1e-4 of the pixels on the mask.
    img, mk, _ = synth.ellipses(256, 256, 12, (10, 60), 8, 0.05, 11)
    s, o, p = both(segmg, img.astype(np.float32), mk, precision=segmg.MG_MIXED, levels=7)
    cyc, rho = s.solve_step(1e-6, 60)
    o.set_tau(s.stats()["tau"])
    hist = o.solve_step(1e-9, 80)
    pg, po = s.phi().cpu().numpy(), o.phi
    assert rho <= 1e-6
    assert relmax(pg, po) < 1e-4
    assert np.mean((pg > 0) != (po > 0)) <= 1e-4


def test_large_tiles_cover_boundary_and_interior(segmg):
    # a grid with interior 64 x 64 tiles and ragged edge tiles in both directions: the fused
    # sweep (interior fast path and boundary path) equals the per-phase path bitwise
    img, mk, _ = synth.ellipses(301, 333, 10, (20, 120), 8, 0.05, 12)
    outs = []
    for sm in (0, 1):
        s, _ = gpu_solver(segmg, img, mk, precision=segmg.MG_F32, levels=5, smoother=sm)
        s.begin_step()
        for _ in range(2):
            s.vcycle()
        outs.append(s.phi().cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_every_tile_shape_gives_the_same_result(segmg, precision):
    prec = segmg.MG_F64 if precision == "f64" else segmg.MG_F32
    img, mk, _ = synth.ellipses(233, 301, 10, (20, 120), 8, 0.05, 13)
    outs = []
    for sh in range(6):
        s, p = gpu_solver(segmg, img, mk, precision=prec, levels=5)
        s.set_tile_shapes([sh] * (p.levels - 1))
        s.begin_step()
        for _ in range(2):
            s.vcycle()
        outs.append(s.phi().cpu().numpy())
    for x in outs[1:]:
        assert np.array_equal(outs[0], x)


def test_autotune_keeps_the_state_and_the_results(segmg):
    img, mk, _ = synth.ellipses(320, 320, 10, (20, 120), 8, 0.05, 14)
    s1, _ = gpu_solver(segmg, img, mk)
    s1.solve_step(1e-6, 50)
    s2, p = gpu_solver(segmg, img, mk)
    s2.begin_step()
    shapes = s2.autotune(reps=1)
    assert len(shapes) == p.levels - 1 and all(0 <= x <= 5 for x in shapes)
    lb, lc = s2.stats()["bottom_level"], s2.stats()["cluster_level"]
    assert (0 <= lb <= p.levels - 2) != (0 <= lc <= p.levels - 2)
    s2.end_step()          # the autotuner restored phi: this step changed nothing
    s2.solve_step(1e-6, 50)
    assert np.array_equal(s1.phi().cpu().numpy(), s2.phi().cpu().numpy())


def test_batch_equals_individual_solves(segmg):
    shapes = [(64, 64), (96, 80), (128, 128), (40, 200), (160, 160)]
    imgs, mks, params = [], [], []
    for q, (n, m) in enumerate(shapes):
        img, mk, _ = synth.ellipses(n, m, 6, (10, min(n, m) / 2), 4 + q, 0.05, 30 + q)
        imgs.append(img.astype(np.float32))
        mks.append(mk)
        params.append(segmg.default_params(n, m))
    b = segmg.Batch([torch.as_tensor(x, device="cuda") for x in imgs], mks, params)
    cyc, rho = b.solve_step(1e-6, 60)
    for q in range(len(shapes)):
        s, _ = gpu_solver(segmg, imgs[q], mks[q])
        c, r = s.solve_step(1e-6, 60)
        assert cyc[q] == c and rho[q] == r
        v = b.solver(q)
        assert np.array_equal(v.phi().cpu().numpy(), s.phi().cpu().numpy())
        assert np.array_equal(v.mask().cpu().numpy(), s.mask().cpu().numpy())
        assert v.stats()["steps"] == 1
    b.close()


@pytest.mark.parametrize("shape,levels,nu", [((256, 256), 7, (2, 2)), ((200, 170), 6, (1, 3)),
                                             ((61, 47), 4, (2, 2)), ((130, 97), 6, (3, 0))])
@pytest.mark.parametrize("precision", ["f32", "mixed"])
def test_bottom_kernel_equals_per_grid_kernels(segmg, shape, levels, nu, precision):
    # the one-block bottom of the V-cycle performs the per-grid kernels' operations cell by cell
    prec = segmg.MG_MIXED if precision == "mixed" else segmg.MG_F32
    n, m = shape
    img, mk, _ = synth.ellipses(n, m, 8, (8, min(n, m) / 2), 6, 0.05, 40 + n)
    outs, firsts, stats = [], [], []
    for on in (1, 0):
        s, p = gpu_solver(segmg, img, mk, precision=prec, levels=levels, nu1=nu[0], nu2=nu[1])
        firsts.append(s.set_bottom_kernel(bool(on)))
        s.begin_step()
        rhos = [s.vcycle() for _ in range(3)]
        outs.append((s.phi().cpu().numpy(), rhos))
        stats.append(s.stats())
    assert firsts[0] >= 0 and firsts[1] == -1
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1]
    assert stats[0]["picard_last"] == stats[1]["picard_last"]


def largest_fitting_bottom(s, levels):
    """The largest grid the one-block bottom kernel can start at (the first level accepted)."""
    for lb in range(levels - 1):
        try:
            s.set_bottom_level(lb)
            return lb
        except Exception:
            continue
    return -1


@pytest.mark.parametrize("precision", ["f32", "mixed"])
def test_every_bottom_level_gives_the_same_result(segmg, precision):
    # where the one-block bottom kernel starts changes only which kernels run the small grids
    prec = segmg.MG_MIXED if precision == "mixed" else segmg.MG_F32
    img, mk, _ = synth.ellipses(256, 256, 8, (8, 128), 6, 0.05, 77)
    outs = []
    s, p = gpu_solver(segmg, img, mk, precision=prec, levels=7)
    default = s.set_bottom_kernel(True)
    first = largest_fitting_bottom(s, p.levels)
    assert 0 <= first <= default
    s.close()
    for lb in [first, first + 1, first + 2, -1]:
        s, p = gpu_solver(segmg, img, mk, precision=prec, levels=7)
        s.set_bottom_level(lb)
        assert s.stats()["bottom_level"] == lb
        s.begin_step()
        rhos = [s.vcycle() for _ in range(3)]
        outs.append((s.phi().cpu().numpy(), rhos))
        s.close()
    for x in outs[1:]:
        assert np.array_equal(outs[0][0], x[0]) and outs[0][1] == x[1]
    s, p = gpu_solver(segmg, img, mk, precision=prec, levels=7)
    for bad in (first - 1, p.levels - 1):
        with pytest.raises(segmg.SegmgError):
            s.set_bottom_level(bad)
    s.close()


@pytest.mark.parametrize("shape,levels", [((256, 256), 7), ((200, 170), 6)])
@pytest.mark.parametrize("precision", ["f32", "mixed"])
def test_cluster_bottom_equals_one_block_and_per_grid(segmg, shape, levels, precision):
    # the bottom of the V-cycle spread over a thread-block cluster (one CTA per 32 x 32 tile,
    # ragged tiles included) performs the same operations cell by cell
    prec = segmg.MG_MIXED if precision == "mixed" else segmg.MG_F32
    n, m = shape
    img, mk, _ = synth.ellipses(n, m, 14, (6, min(n, m) / 2), 6, 0.1, 91 + n)
    s, p = gpu_solver(segmg, img, mk, precision=prec, levels=levels)
    # the default at set-up: the cluster from the largest grid the one-block kernel can start at
    default_cluster = s.stats()["cluster_level"]
    first = largest_fitting_bottom(s, p.levels)
    assert first >= 0 and default_cluster == first
    s.close()
    # the largest grid the one-block kernel can start at always fits a cluster here; the grid above it may
    # not (its cluster needs one SM per tile within one GPC), and is then refused
    runs = [("one-block", None), ("none", None), ("cluster", first), ("cluster", first - 1)]
    outs = []
    for kind, lc in runs:
        s, p = gpu_solver(segmg, img, mk, precision=prec, levels=levels)
        if kind == "one-block":
            s.set_bottom_kernel(True)   # (the default at set-up may be the cluster)
            assert s.stats()["cluster_level"] == -1
        elif kind == "none":
            s.set_bottom_kernel(False)
        elif kind == "cluster":
            try:
                s.set_cluster_level(lc)
            except segmg.SegmgError:
                assert lc == first - 1
                s.close()
                continue
            assert s.stats()["cluster_level"] == lc
        s.begin_step()
        rhos = [s.vcycle() for _ in range(3)]
        outs.append((s.phi().cpu().numpy(), rhos, s.stats()["picard_last"]))
        s.close()
    for x in outs[1:]:
        assert np.array_equal(outs[0][0], x[0]) and outs[0][1] == x[1] and outs[0][2] == x[2]
    s, p = gpu_solver(segmg, img, mk, precision=prec, levels=levels)
    for bad in (first - 2, p.levels - 1):
        with pytest.raises(segmg.SegmgError):
            s.set_cluster_level(bad)
    s.close()


def test_bottom_kernel_applies_only_where_it_is_exact(segmg):
    img, mk, _ = synth.ellipses(128, 128, 6, (10, 60), 4, 0.05, 3)
    for kw, expect in (({}, True), ({"precision": segmg.MG_F64}, False),
                       ({"model": segmg.MG_MODEL_RC}, False), ({"smoother": 1}, False)):
        s, p = gpu_solver(segmg, img, mk, levels=6, **kw)
        lb = s.set_bottom_kernel(True)
        assert (lb >= 0) == expect
        if expect:
            assert 0 <= lb <= p.levels - 2


def test_fused_sweep_is_scheduling_independent_on_multi_wave_grids(segmg):
    # 2048^2 needs several waves of 32 x 64 tiles: a tile must never see a neighbour's updated
    # cells, so the fused sweep equals the per-phase path bitwise and runs repeat bitwise
    img, mk, _ = synth.ellipses(2048, 2048, 24, (40, 400), 8, 0.05, 21)
    outs = []
    for sm in (0, 0, 1, 2):
        s, _ = gpu_solver(segmg, img, mk, precision=segmg.MG_F32, levels=10, smoother=sm)
        s.begin_step()
        for _ in range(2):
            s.vcycle()
        outs.append(s.phi().cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[0], outs[3])


@pytest.mark.parametrize("model", [0, 1])
def test_energy_matches_oracle(segmg, model):
    # the energy of the level set (Table 7's diagnostic) after set-up, after V-cycles and after
    # the end-of-step c1/c2 update, FP64 and FP32
    img, mk, _ = synth.ellipses(150, 131, 6, (20, 70), 5, 0.05, 17)
    for prec, tol in ((segmg.MG_F64, 1e-10), (segmg.MG_F32, 2e-5)):
        s, o, p = both(segmg, img.astype(np.float32) if prec == segmg.MG_F32 else img, mk,
                       precision=prec, levels=4, model=model)
        assert abs(s.energy() - o.energy()) <= tol * abs(o.energy())
        s.begin_step(); o.begin_step()
        for _ in range(3):
            s.vcycle(); o.vcycle()
        assert abs(s.energy() - o.energy()) <= tol * abs(o.energy())
        s.end_step(); o.end_step()
        assert abs(s.energy() - o.energy()) <= tol * abs(o.energy())
        s.close()


@pytest.mark.parametrize("smoother", [3, 4])
def test_gsline_and_hybrid_smoother_1_match_oracle(segmg, smoother):
    # Algorithm 1 (GSLINE-I, zebra columns) and Algorithm 2 (Hybrid Smoother 1, parallel
    # ordering) against the oracle's same orderings: FP64 per V-cycle, FP32 to the solution
    img, mk, _ = synth.ellipses(140, 117, 6, (20, 70), 5, 0.05, 23)
    s, o, p = both(segmg, img, mk, precision=segmg.MG_F64, levels=4, smoother=smoother)
    s.begin_step(); o.begin_step()
    for _ in range(3):
        rg, ro = s.vcycle(), o.vcycle()
        assert abs(rg - ro) <= 1e-8 * ro
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-10
    s.close(); o.close()
    s32, o2, _ = both(segmg, img.astype(np.float32), mk, precision=segmg.MG_F32, levels=4, smoother=smoother)
    cyc, rho = s32.solve_step(1e-6, 80)
    o2.set_tau(s32.stats()["tau"])
    hist = o2.solve_step(1e-9, 120)
    assert rho <= 1e-6 and hist[-1] <= 1e-9
    pg, po = s32.phi().cpu().numpy(), o2.phi
    assert relmax(pg, po) < 1e-5
    assert np.mean((pg > 0) != (po > 0)) <= 1e-4


def test_aos_coarsest_solver_matches_oracle(segmg):
    # V-cycles whose coarsest solve is 100 AOS iterations (Sec. 5), FP64 against the oracle
    img, mk, _ = synth.ellipses(160, 144, 6, (20, 70), 5, 0.05, 27)
    s, o, p = both(segmg, img, mk, precision=segmg.MG_F64, levels=5, coarse_solver=segmg.MG_COARSE_AOS,
                   aos_dt=10.0)
    s.begin_step(); o.begin_step()
    for _ in range(3):
        rg, ro = s.vcycle(), o.vcycle()
        assert abs(rg - ro) <= 1e-8 * ro
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-10
    # FP32: the one-block bottom kernel runs the same AOS coarsest solve (bitwise)
    outs = []
    for on in (1, 0):
        s32, _ = gpu_solver(segmg, img, mk, precision=segmg.MG_F32, levels=5,
                            coarse_solver=segmg.MG_COARSE_AOS, aos_dt=10.0)
        s32.set_bottom_kernel(bool(on))
        c, r = s32.solve_step(1e-6, 60)
        assert r <= 1e-6
        outs.append(s32.phi().cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("model", [0, 1])
def test_finest_grid_aos_matches_oracle(segmg, model):
    # the AOS method of Table 6 on the finest grid, FP64 and FP32
    img, mk, _ = synth.ellipses(120, 136, 5, (20, 60), 5, 0.05, 29)
    for prec, tol in ((segmg.MG_F64, 1e-10), (segmg.MG_F32, 1e-5)):
        s, o, p = both(segmg, img.astype(np.float32) if prec == segmg.MG_F32 else img, mk,
                       precision=prec, levels=4, model=model)
        s.begin_step(); o.begin_step()
        ig, rg = s.aos(0.5, 12, 0.0)
        io, ro = o.aos(0.5, 12, 0.0)
        assert ig == io == 12
        assert abs(rg - ro) <= 100 * tol * ro
        assert relmax(s.phi().cpu().numpy(), o.phi) < tol
        # the relative-change stop ends both at the same iteration
        s.begin_step(); o.begin_step()
        ig, _ = s.aos(0.5, 200, 1e-4)
        io, _ = o.aos(0.5, 200, 1e-4)
        assert abs(ig - io) <= (0 if prec == segmg.MG_F64 else 1)
        s.close()


def test_bench_workload_full_size_matches_oracle(segmg):
    # the bench's 1024^2 FP32 workload in the bench's launch configuration (TMA sweeps, bottom
    # kernel, graphs, autotuned tiles) against the FP64 oracle's converged solution
    W = synth.workload("ellipse1024")
    s, p = gpu_solver(segmg, W.image.astype(np.float32), W.markers, levels=W.levels)
    s.begin_step()
    s.autotune(reps=1)
    s.end_step()
    s.reset(torch.as_tensor(W.image.astype(np.float32), device="cuda"), W.markers)
    cyc, rho = s.solve_step(1e-6, 60)
    assert rho <= 1e-6
    o = O.Solver(W.image.astype(np.float32).astype(np.float64), W.markers, oracle_params(1024, 1024, p))
    o.set_tau(s.stats()["tau"])
    hist = o.solve_step(1e-9, 80)
    assert hist[-1] <= 1e-9
    pg, po = s.phi().cpu().numpy(), o.phi
    assert relmax(pg, po) < 1e-5
    assert np.mean((pg > 0) != (po > 0)) <= 1e-4
    o.close()


def test_mixed_precision_large_grid_properties_and_crop(segmg):
    # 8192^2 mixed precision (w in BF16): properties that hold at any size (monotone residual,
    # rho <= 1e-6, a mask with both regions), and a 512^2 crop solved standalone against the oracle
    dev = torch.device("cuda", 0)
    img, mk = synth.ellipses_device(8192, 8192, 200, (100 * 8192 / 25000, 3000 * 8192 / 25000), 20, 0.05, 2, dev)
    p = segmg.default_params(8192, 8192, precision=segmg.MG_MIXED)
    s = segmg.Solver(img, mk, p)
    s.begin_step()
    hist = []
    for _ in range(40):
        hist.append(s.vcycle())
        if hist[-1] <= 1e-6:
            break
    assert hist[-1] <= 1e-6
    assert all(b < a for a, b in zip(hist, hist[1:]))
    frac = float(s.mask().float().mean())
    assert 0.0 < frac < 0.5            # the selected object: present, a small part of the image
    s.close()
    crop = img[3000:3512, 1000:1512].float().cpu().numpy()
    cm = np.array([[256.0 + 20 * np.cos(t), 256.0 + 20 * np.sin(t)] for t in np.linspace(0, 6, 6)])
    s2, o2, p2 = both(segmg, crop, cm, precision=segmg.MG_MIXED, levels=7)
    c2, r2 = s2.solve_step(1e-6, 60)
    o2.set_tau(s2.stats()["tau"])
    h2 = o2.solve_step(1e-9, 80)
    assert r2 <= 1e-6 and h2[-1] <= 1e-9
    pg, po = s2.phi().cpu().numpy(), o2.phi
    assert relmax(pg, po) < 1e-4
    assert np.mean((pg > 0) != (po > 0)) <= 1e-4


def test_successive_steps_each_reach_the_tolerance_and_match_the_oracle(segmg):
    # three pseudo-time steps of a 512^2 image under the step control (the later steps stall at
    # rho ~ 1e-3 when tau stays 1): every step reaches rho <= 1e-6, and each matches the oracle's
    # solution of the same step (same phi^n, c1, c2 and the tau the control accepted)
    img, mk, _ = synth.ellipses(512, 512, 12, (10, 100), 13, 0.05, 3)
    img = img.astype(np.float32)
    s, p = gpu_solver(segmg, img, mk, precision=segmg.MG_F32)
    o = O.Solver(img.astype(np.float64), mk, oracle_params(512, 512, p))
    taus = []
    for step in range(3):
        phin, st0 = s.phi().cpu().numpy().astype(np.float64), s.stats()
        cyc, rho = s.solve_step(1e-6, 40)
        st = s.stats()
        assert rho <= 1e-6, (step, rho)
        taus.append(st["tau"])
        o.phi = phin
        o.set_c(st0["c1"], st0["c2"])
        o.set_tau(st["tau"])
        hist = o.solve_step(1e-9, 80)
        assert hist[-1] <= 1e-7, (step, hist[-1])
        pg, po = s.phi().cpu().numpy(), o.phi
        assert relmax(pg, po) < 1e-5, step
        assert np.mean((pg > 0) != (po > 0)) <= 1e-4, step
        # eta of the step, read by stats() after the step end only enqueued its sums: this
        # step's, not the previous one's (phi agrees to 1e-5 of max |phi|, so eta to ~1e-5)
        eo = o.end_step()
        assert abs(st["eta"] - eo) <= 1e-4 * max(1.0, eo), (step, st["eta"], eo)
        so = o.scalars()
        assert abs(st["c1"] - so["c1"]) <= 1e-5 and abs(st["c2"] - so["c2"]) <= 1e-5
    assert all(b <= a for a, b in zip(taus, taus[1:]))
    s.close()


def test_batch_members_match_the_oracle(segmg):
    # members of a batch against the FP64 oracle (not only against one-by-one GPU solves)
    shapes = [(96, 96), (160, 128), (200, 200)]
    imgs, mks, params = [], [], []
    for q, (n, m) in enumerate(shapes):
        img, mk, _ = synth.ellipses(n, m, 8, (10, min(n, m) / 2), 5 + q, 0.05, 60 + q)
        imgs.append(img.astype(np.float32))
        mks.append(mk)
        params.append(segmg.default_params(n, m))
    b = segmg.Batch([torch.as_tensor(x, device="cuda") for x in imgs], mks, params)
    cyc, rho = b.solve_step(1e-6, 40)
    assert max(rho) <= 1e-6
    for q, (n, m) in enumerate(shapes):
        v = b.solver(q)
        o = O.Solver(imgs[q].astype(np.float64), mks[q], oracle_params(n, m, params[q]))
        o.set_tau(v.stats()["tau"])
        hist = o.solve_step(1e-9, 80)
        assert hist[-1] <= 1e-7
        pg, po = v.phi().cpu().numpy(), o.phi
        assert relmax(pg, po) < 1e-5, q
        assert np.mean((pg > 0) != (po > 0)) <= 1e-4, q
        o.close()
    b.close()


def test_divergence_is_reported_and_the_step_control_restarts_from_phi_n(segmg):
    # a diverged V-cycle, injected on the host (the third V-cycle of the step reports a residual
    # ratio of 1e9): without the step control mg_vcycle returns MG_ERR_DIVERGED; with it the
    # attempt is rejected, phi^n restored and the step solved with tau / 2, which gives bitwise
    # the solution of that step solved directly with tau / 2
    img, mk, _ = synth.ellipses(192, 192, 8, (10, 80), 6, 0.05, 19)
    img = img.astype(np.float32)
    s, p = gpu_solver(segmg, img, mk, stall_ratio=0.0)
    s.begin_step()
    s.inject_divergence(3)
    s.vcycle(); s.vcycle()
    with pytest.raises(segmg.SegmgError) as e:
        s.vcycle()
    assert e.value.code == -4
    s.close()
    s, p = gpu_solver(segmg, img, mk)
    s.inject_divergence(3)
    c, rho = s.solve_step(1e-6, 40)
    st = s.stats()
    assert rho <= 1e-6 and st["attempts_rejected"] == 1 and st["tau"] == 0.5 * p.tau
    ref, _ = gpu_solver(segmg, img, mk, tau=0.5 * p.tau)
    c2, rho2 = ref.solve_step(1e-6, 40)
    assert c == c2 + 3 and rho == rho2
    assert np.array_equal(s.phi().cpu().numpy(), ref.phi().cpu().numpy())
    s.close(); ref.close()


def test_sweep_wait_limit_time_out_is_reported_and_the_handle_recovers(segmg):
    # every TMA wait of the fused sweep gives up at once (limit 0): each block records the
    # time-out, waits (bounded) for its copies in flight and ends; the V-cycle returns
    # MG_ERR_TIMEOUT.  With the default limit restored the handle gives the normal results.
    img, mk, _ = synth.ellipses(256, 256, 8, (10, 80), 6, 0.05, 8)
    s, p = gpu_solver(segmg, img.astype(np.float32), mk)
    phi0 = s.phi()
    s.set_wait_limit(0)
    s.begin_step()
    with pytest.raises(segmg.SegmgError) as e:
        s.vcycle()
    assert e.value.code == -5 and "wait limit" in str(e.value)
    s.set_wait_limit(1 << 22)
    s.set_phi(phi0)
    s.begin_step()
    got = [s.vcycle() for _ in range(2)]
    ref, _ = gpu_solver(segmg, img.astype(np.float32), mk)
    ref.begin_step()
    want = [ref.vcycle() for _ in range(2)]
    assert got == want
    assert np.array_equal(s.phi().cpu().numpy(), ref.phi().cpu().numpy())
    s.close(); ref.close()


def test_checkpoint_and_resume_at_a_step_boundary_is_bitwise(segmg):
    # state at a step boundary = phi, c1, c2 and the step control's tau; a new handle resumed from
    # it continues exactly as the uninterrupted run
    img, mk, _ = synth.ellipses(256, 256, 12, (10, 90), 9, 0.05, 6)
    img = img.astype(np.float32)
    a, p = gpu_solver(segmg, img, mk)
    for _ in range(3):
        a.solve_step(1e-6, 40)
    b, _ = gpu_solver(segmg, img, mk)
    for _ in range(2):
        b.solve_step(1e-6, 40)
    ck = dict(phi=b.phi().cpu().numpy(), **{k: b.stats()[k] for k in ("c1", "c2", "tau")})
    b.close()
    c, _ = gpu_solver(segmg, img, mk, tau=ck["tau"])
    c.set_phi(torch.as_tensor(ck["phi"], device="cuda"))
    c.set_regions(ck["c1"], ck["c2"])
    c.solve_step(1e-6, 40)
    assert np.array_equal(c.phi().cpu().numpy(), a.phi().cpu().numpy())
    sa, sc = a.stats(), c.stats()
    assert (sa["c1"], sa["c2"], sa["tau"]) == (sc["c1"], sc["c2"], sc["tau"])
    a.close(); c.close()


@pytest.mark.parametrize("k", [33, 150])
def test_setup_fields_with_many_markers_on_a_circle(segmg, k):
    # markers on a circle: every marker is a hull vertex, so the set-up handles more markers than
    # one shared-memory chunk of the distance kernel (32) and, for k = 150, more hull edges than
    # one chunk of the initial-level-set kernel (64); FP64 against the oracle
    n, m = 150, 131
    img, _, _ = synth.disc_square(150, 0.05, 3)
    img = img[:n, :m].copy()
    t = 2 * np.pi * np.arange(k) / k
    mk = np.stack([65.0 + 40.0 * np.cos(t), 75.0 + 45.0 * np.sin(t)], axis=1)
    s, o, p = both(segmg, img, mk, precision=segmg.MG_F64, levels=3)
    for l in range(3):
        for f in ("w", "z", "d"):
            assert relmax(s.level(l, f).cpu().numpy(), o.level(l, f)) < 1e-13, (l, f)
    assert relmax(s.phi().cpu().numpy(), o.phi) < 1e-13
    st, so = s.stats(), o.scalars()
    assert abs(st["c1"] - so["c1"]) < 1e-12 and abs(st["c2"] - so["c2"]) < 1e-12
    assert abs(st["A1"] - so["A1"]) < 1e-9
    # FP32 storage: the same fields to FP32 rounding
    s32, _ = gpu_solver(segmg, img.astype(np.float32), mk, precision=segmg.MG_F32, levels=3)
    for f in ("w", "d"):   # d: a product of k factors, each rounded in FP32
        assert relmax(s32.level(0, f).cpu().numpy(), o.level(0, f)) < 3e-5, f
    assert relmax(s32.phi().cpu().numpy(), o.phi) < 1e-6


def test_reset_after_a_non_finite_image_recovers(segmg):
    # the image check runs while the image is copied in and is read at the end of the set-up:
    # a NaN image is refused with MG_ERR_NAN, and a following reset with a good image gives
    # what a fresh handle gives, bitwise
    img, mk, _ = synth.ellipses(96, 80, 6, (10, 50), 5, 0.05, 8)
    s, p = gpu_solver(segmg, img, mk, levels=4)
    bad = img.copy()
    bad[50, 7] = np.inf
    with pytest.raises(segmg.SegmgError) as e:
        s.reset(torch.as_tensor(bad, device="cuda"), mk)
    assert e.value.code == -2
    s.reset(torch.as_tensor(img, device="cuda"), mk)
    s.solve_step(1e-6, 40)
    ref, _ = gpu_solver(segmg, img, mk, levels=4)
    ref.solve_step(1e-6, 40)
    assert np.array_equal(s.phi().cpu().numpy(), ref.phi().cpu().numpy())


def test_time_residuals_reports_the_v_cycle_residual_kernels(segmg):
    img, mk, _ = synth.ellipses(256, 200, 6, (20, 80), 5, 0.05, 4)
    s, p = gpu_solver(segmg, img, mk, levels=5)
    with pytest.raises(segmg.SegmgError) as e:
        s.time_residuals(0, 1)
    assert e.value.code == -8          # outside a step
    s.begin_step()
    for l in range(p.levels):
        norm_ms, rr_ms = s.time_residuals(l, 2)
        assert norm_ms > 0
        assert (rr_ms > 0) if l + 1 < p.levels else rr_ms == -1.0
    with pytest.raises(segmg.SegmgError):
        s.time_residuals(p.levels, 1)
    s.end_step()
    # the timing runs leave the step's state usable: a fresh step still converges
    cyc, rho = s.solve_step(1e-6, 60)
    assert rho <= 1e-6


def test_time_sweeps_graph_times_the_replayed_sweeps(segmg):
    img, mk, _ = synth.ellipses(256, 200, 6, (20, 80), 5, 0.05, 4)
    s, p = gpu_solver(segmg, img, mk, levels=5)
    with pytest.raises(segmg.SegmgError) as e:
        s.time_sweeps_graph(0, 2)
    assert e.value.code == -8          # outside a step
    s.begin_step()
    for l in range(p.levels):
        assert s.time_sweeps_graph(l, 2) > 0
    for level, reps in ((0, 0), (0, 257), (p.levels, 1)):
        with pytest.raises(segmg.SegmgError):
            s.time_sweeps_graph(level, reps)
    s.end_step()
    # the timing runs leave the handle usable: a fresh step still converges
    cyc, rho = s.solve_step(1e-6, 60)
    assert rho <= 1e-6


def test_rada_chen_fp32_step_matches_oracle(segmg):
    # the Rada-Chen model in FP32 storage: the area term on every grid, the FAS right-hand side
    # completed by the coarse grids' first snapshots (the interpolation keeps its own launch for
    # this model); one whole step against the FP64 oracle's converged solution of the same step
    img, mk, _ = synth.ellipses(200, 170, 8, (15, 70), 6, 0.05, 31)
    s, o, p = both(segmg, img.astype(np.float32), mk, precision=segmg.MG_F32, levels=5,
                   model=segmg.MG_MODEL_RC)
    cyc, rho = s.solve_step(1e-6, 60)
    o.set_tau(s.stats()["tau"])
    hist = o.solve_step(1e-9, 80)
    assert rho <= 1e-6 and hist[-1] <= 1e-9
    pg, po = s.phi().cpu().numpy(), o.phi
    assert relmax(pg, po) < 1e-5
    assert np.mean((pg > 0) != (po > 0)) <= 1e-4
