"""Small cases that reach every kernel family of the library, run in a child process by
tests/test_gpu_debug.py: once with the default library and once with the bounds-checked build
(SEGMG_DEBUG=1 selects it).  Writes every result array and the device error words to an .npz.

    python tests/debug_cases.py OUT.npz
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def run(out_path):
    import torch
    from paper_1807_02137_gb300 import segmg, synth

    res = {}
    dev = "cuda"

    def solver(img, mk, **kw):
        n, m = img.shape
        p = segmg.default_params(n, m, **kw)
        dt = torch.float64 if p.precision == segmg.MG_F64 else torch.float32
        return segmg.Solver(torch.as_tensor(np.ascontiguousarray(img), dtype=dt, device=dev), mk, p)

    def keep(name, s, extra=()):
        res[name + "/phi"] = s.phi().cpu().numpy()
        res[name + "/mask"] = s.mask().cpu().numpy()
        for k, v in extra:
            res[name + "/" + k] = np.asarray(v)
        s.close()

    # tiny and ragged grids, FP64, per-grid kernels down to a coarsest grid of one cell
    for (n, m), levels in [((1, 1), 1), ((2, 3), 1), ((5, 4), 2), ((33, 65), 4)]:
        rng = np.random.default_rng(n * 100 + m)
        s = solver(rng.uniform(0, 1, (n, m)), np.array([[m // 2, n // 2]], float),
                   precision=segmg.MG_F64, levels=levels)
        s.begin_step()
        rhos = [s.vcycle() for _ in range(2)]
        keep(f"tiny{n}x{m}", s, [("rho", rhos)])
    # degenerate markers (one point, collinear points)
    img, _, _ = synth.disc_square(64, 0.05, 3)
    for q, mk in enumerate(([[20, 30]], [[10, 10], [20, 20], [30, 30]])):
        s = solver(img, np.array(mk, float), precision=segmg.MG_F64, levels=4)
        s.begin_step()
        keep(f"degenerate{q}", s, [("rho", [s.vcycle()])])
    # FP32 fused sweeps (TMA), one-block bottom kernel, a ragged grid, a whole step
    img, mk, _ = synth.ellipses(100, 77, 6, (8, 40), 5, 0.05, 7)
    s = solver(img, mk, precision=segmg.MG_F32, levels=5)
    cyc, rho = s.solve_step(1e-5, 40)
    keep("f32_step", s, [("rho", [rho]), ("cycles", [cyc])])
    # FP32 with the cluster bottom and the per-grid kernels on grids above it
    img, mk, _ = synth.ellipses(256, 256, 8, (8, 100), 6, 0.05, 41)
    s = solver(img, mk, precision=segmg.MG_F32, levels=7)
    for lvl in range(7):
        try:
            s.set_cluster_level(lvl)
            break
        except segmg.SegmgError:
            continue
    s.begin_step()
    keep("cluster", s, [("rho", [s.vcycle() for _ in range(2)])])
    # mixed precision (BF16 weights, FP64 coarsest solve), per-grid kernels only
    img, mk, _ = synth.ellipses(130, 97, 8, (8, 48), 6, 0.05, 170)
    s = solver(img, mk, precision=segmg.MG_MIXED, levels=6)
    s.set_bottom_kernel(False)
    s.begin_step()
    keep("mixed", s, [("rho", [s.vcycle() for _ in range(2)])])
    # the phased smoother, GSLINE-I, Hybrid Smoother 1 (FP64 and FP32)
    img, mk, _ = synth.ellipses(61, 47, 5, (6, 20), 4, 0.05, 12)
    for name, sm in (("phased", segmg.MG_SMOOTH_PHASED), ("gsline", segmg.MG_SMOOTH_GSLINE),
                     ("hs1", segmg.MG_SMOOTH_HS1)):
        for prec in (segmg.MG_F64, segmg.MG_F32):
            s = solver(img, mk, precision=prec, levels=4, smoother=sm)
            s.begin_step()
            keep(f"{name}{prec}", s, [("rho", [s.vcycle() for _ in range(2)])])
    # AOS: the coarsest solve by AOS iterations, and AOS time marching on the finest grid
    img, mk, _ = synth.ellipses(80, 72, 6, (10, 35), 5, 0.05, 27)
    s = solver(img, mk, precision=segmg.MG_F64, levels=4, coarse_solver=segmg.MG_COARSE_AOS, aos_dt=10.0)
    s.begin_step()
    keep("aos_coarse", s, [("rho", [s.vcycle() for _ in range(2)])])
    s = solver(img, mk, precision=segmg.MG_F32, levels=4)
    s.begin_step()
    it, r = s.aos(5.0, 4, 0.0)
    keep("aos_fine", s, [("rho", [r]), ("energy", [0.0])])
    # energy and the allocation-free residual norm
    s = solver(img, mk, precision=segmg.MG_F64, levels=4)
    e = s.energy()
    p = segmg.default_params(80, 72, precision=segmg.MG_F64)
    t = torch.as_tensor(img, dtype=torch.float64, device=dev)
    nrm = segmg.residual_norm_noalloc(t, torch.ones_like(t), t * 0.5, p)
    keep("energy", s, [("energy", [e]), ("noalloc", [nrm])])
    # learned weights: inference (tensor cores) inside V-cycles, crop recording and training
    img, mk, _ = synth.ellipses(128, 96, 8, (10, 40), 6, 0.05, 11)
    s = solver(img.astype(np.float32), mk, precision=segmg.MG_F32, levels=5)
    tr = segmg.Trainer(capacity=16, batch_max=8, seed=3)
    th = tr.theta().copy()
    th[3056:3200] = np.random.default_rng(5).normal(0, 0.05, 144)   # a non-constant output layer
    s.set_learned(th, mode=2, refresh=1)
    s.begin_step()
    rhos = [s.vcycle() for _ in range(2)]
    res["learned/omega"] = s.level(0, 7).cpu().numpy()
    tr.record(s, 8)
    loss = tr.train(2, 4, 1e-3)
    res["learned/theta"] = tr.theta()
    tr.close()
    keep("learned", s, [("rho", rhos), ("loss", [loss])])
    # a batch of three images, one graph launch per V-cycle
    imgs, mks, params = [], [], []
    for q, (n, m) in enumerate([(64, 64), (96, 80), (72, 72)]):
        im, mk, _ = synth.ellipses(n, m, 6, (8, min(n, m) / 2), 4 + q, 0.05, 60 + q)
        imgs.append(torch.as_tensor(im.astype(np.float32), device=dev))
        mks.append(mk)
        params.append(segmg.default_params(n, m, levels=4))
    b = segmg.Batch(imgs, mks, params)
    cyc, rho = b.solve_step(1e-5, 30)
    for q in range(3):
        res[f"batch{q}/phi"] = b.solver(q).phi().cpu().numpy()
    b.close()
    torch.cuda.synchronize()
    d = segmg.debug_status(clear=False)
    res["debug/status"] = np.array([d["enabled"], d["first_site"], d["first_index"], d["sites"], d["count"]],
                                   dtype=np.int64)
    # the reporting path itself: one recorded index with no memory access behind it
    segmg.debug_selftest()
    d = segmg.debug_status(clear=True)
    res["debug/selftest"] = np.array([d["enabled"], d["first_site"], d["first_index"], d["sites"], d["count"]],
                                     dtype=np.int64)
    d = segmg.debug_status()
    res["debug/cleared"] = np.array([d["count"], d["sites"]], dtype=np.int64)
    res["library"] = np.array(segmg.library_path())
    np.savez(out_path, **res)


if __name__ == "__main__":
    run(sys.argv[1])
