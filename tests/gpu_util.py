"""Helpers for the GPU parity tests: build the library once, run the method
through the C ABI, and compare with the oracle."""
import numpy as np
import pytest

import paper_1304_6514_gb300 as nvp
from paper_1304_6514_gb300 import _build

_built = False


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    global _built
    if not _built:
        _build.build()
        _built = True
    nvp.load_library()
    return torch


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def run_method(torch, rhs, t0, T, S, smp, st, y0, maps=None):
    """Build + compose through the ABI.  Returns (maps, table (numpy), yT, lambdas)."""
    maps = nvp.build_propagators(rhs, t0, T, S, smp, st, maps=maps)
    y0_t = torch.tensor(np.atleast_1d(y0), dtype=torch.float64, device="cuda")
    yT = torch.empty_like(y0_t)
    lam = torch.empty((S + 1, y0_t.numel()), dtype=torch.float64, device="cuda")
    nvp.compose(maps, y0_t, yT, lam)
    oob = nvp.maps_check(maps)
    tab = nvp.maps_data(maps).cpu().numpy()
    return maps, tab, yT.cpu().numpy(), lam.cpu().numpy(), oob
