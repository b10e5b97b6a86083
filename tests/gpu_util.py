"""Helpers shared by the GPU tests: paired oracle / library problems on the
same seeded inputs."""
import numpy as np
import pytest

from paper_1307_2036_gb300 import inputs


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    # on a GPU machine the library must be present: importing fails loudly otherwise
    from paper_1307_2036_gb300 import ellsolve  # noqa: F401
    return torch


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def sensitivity(fn, *arrays, trials=2, seed=0, ulps=4, eps=None, norm="l2"):
    """Relative change of fn's output when each input is perturbed by random
    relative amounts of up to `ulps` units of `eps` (default the FP64 machine
    epsilon): how far two correct evaluations of the same map at that
    precision can drift apart from rounding alone.  norm "l2": relative L2
    change; "max": largest element change over the output's largest element."""
    eps = np.finfo(np.float64).eps if eps is None else eps
    base = fn(*arrays)
    rng = np.random.default_rng(seed)
    worst = 0.0
    for _ in range(trials):
        pert = [a * (1.0 + ulps * eps * rng.uniform(-1.0, 1.0, np.shape(a))) for a in arrays]
        out = fn(*pert)
        if norm == "max":
            d = np.max(np.abs(out - base)) / max(np.max(np.abs(base)), 1e-300)
        else:
            d = rel_l2(out, base)
        worst = max(worst, d)
    return worst


def fp64_tol(fn, *arrays, floor=1e-13):
    """Tolerance of an FP64 parity check: 16x the oracle's own rounding
    sensitivity, at least `floor`."""
    return max(floor, 16.0 * sensitivity(fn, *arrays))


EPS32 = float(np.finfo(np.float32).eps)


class Pair:
    """An oracle grid and a library solver for the same problem."""

    def __init__(self, oracle_mod, kind, n, nz, omega2=0.01, lambda2=1.0, graded=False, mapping=0,
                 precision=0, solver=0, coarsest_min=4, **opts):
        import torch
        from paper_1307_2036_gb300 import ellsolve
        self.torch = torch
        self.r = inputs.radial_levels(nz, graded=graded)
        self.og = oracle_mod.Grid(kind, n, nz, self.r, omega2, lambda2, mapping=mapping,
                                  coarsest_min=coarsest_min, max_levels=opts.get("max_levels", 0),
                                  smoother=opts.get("smoother", 0), precond=opts.get("precond", 0),
                                  fmg=bool(opts.get("fmg", 0)))
        self.sv = ellsolve.Solver(kind, n, nz, self.r, omega2, lambda2, mapping=mapping,
                                  precision=precision, solver=solver, coarsest_min=coarsest_min,
                                  **opts)
        assert self.sv.nlevels == self.og.nlevels

    def dev(self, a, fp32=False):
        t = self.torch.tensor(np.ascontiguousarray(a), dtype=self.torch.float64, device="cuda")
        return t.float().contiguous() if fp32 else t

    def host(self, t):
        self.torch.cuda.synchronize()
        return t.double().cpu().numpy()

    def empty(self, level=0, fp32=False):
        dt = self.torch.float32 if fp32 else self.torch.float64
        return self.torch.zeros(self.og.shape(level), dtype=dt, device="cuda")
