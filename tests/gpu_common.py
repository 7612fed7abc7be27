"""Shared helpers of the GPU tests: build the library once, run the same case on both sides."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1807_02137_gb300 import buildlib
    buildlib.build()
    from paper_1807_02137_gb300 import segmg
    return segmg


# the oracle's smoother with the GPU smoother's ordering: Hybrid Smoother 2 parallel (all three
# kernel variants), GSLINE-I zebra, Hybrid Smoother 1 parallel
ORACLE_SMOOTHER = {0: 0, 1: 0, 2: 0, 3: 3, 4: 5}


def oracle_params(n, m, gp):
    """Oracle parameters equal to the GPU parameters `gp` (a segmg.Params)."""
    import oracle as O
    return O.params(n, m, model=gp.model, mu=gp.mu, lambda1=gp.lambda1, lambda2=gp.lambda2,
                    theta=gp.theta, nu=gp.nu, eps=gp.eps, beta=gp.beta, beta_edge=gp.beta_edge,
                    sigma_blur=gp.sigma_blur, sigma_d=gp.sigma_d, Sigma=gp.Sigma,
                    inv_tau=(1.0 / gp.tau if gp.tau > 0 else 0.0), nu1=gp.nu1, nu2=gp.nu2,
                    levels=gp.levels, smoother=ORACLE_SMOOTHER[gp.smoother], coarse_maxit=gp.coarse_maxit,
                    coarse_tol=gp.coarse_tol, coarse_solver=gp.coarse_solver, aos_dt=gp.aos_dt)


def gpu_solver(segmg, image, markers, **kw):
    n, m = image.shape
    p = segmg.default_params(n, m, **kw)
    dt = torch.float64 if p.precision == segmg.MG_F64 else torch.float32
    img = torch.as_tensor(np.ascontiguousarray(image), dtype=dt, device="cuda")
    return segmg.Solver(img, markers, p), p


def relmax(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
