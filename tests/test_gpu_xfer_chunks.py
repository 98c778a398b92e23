"""pdg_set_w / pdg_get_w with host buffers on states of at least 8 x 2^19 points: the copies
move in 8 chunks of points on a private stream, each overlapping the equilibrium (or moment)
kernel of its neighbour chunk on the context stream.  The kernels compute point by point, so
the chunked host path must give bitwise the state and moments of the one-piece device path
(a device buffer is never chunked), for every model family's equilibrium and moment kernels,
both precisions, pageable and pinned host memory, and point counts that 8 does not divide."""
import dataclasses

import numpy as np
import pytest

from paper_1702_00169_gb300 import workloads as W

pytestmark = pytest.mark.gpu
THRESHOLD = 8 << 19


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1702_00169_gb300 import pdg  # noqa: F401


CASES = {
    # 2079 x 2025 points (odd): shallow water and D2Q9 at degree 2
    "shallow_water": dataclasses.replace(W.SW_D2Q4, n_macro=(99, 75), n_sub=(7, 9), order=2),
    "d2q9": dataclasses.replace(W.D2Q9_ISO, n_macro=(99, 75), n_sub=(7, 9), order=2),
    # 168 x 162 x 156 points: Euler, D3Q19 and D3Q27
    "euler": dataclasses.replace(W.EULER_D3Q6, n_macro=(28, 27, 26), n_sub=(2, 2, 2), order=2),
    "d3q19": dataclasses.replace(W.D3Q19_ISO, n_macro=(28, 27, 26), n_sub=(2, 2, 2), order=2),
    "d3q27": dataclasses.replace(W.D3Q27_ISO, n_macro=(28, 27, 26), n_sub=(2, 2, 2), order=2),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [0, 1])
def test_chunked_host_copies_equal_the_device_path(name, precision):
    import torch
    from paper_1702_00169_gb300 import pdg
    cfg = CASES[name]
    s = pdg.solver_for(cfg, precision=precision)
    info = s.info()
    assert info.npoints >= THRESHOLD
    w0 = np.ascontiguousarray(W.initial_w(cfg, [s.points(a) for a in range(cfg.dim)]).reshape(-1))
    s.set_w(w0)                                          # pageable host: chunked
    f_host = s.get_f()
    s.set_w(torch.from_numpy(w0).cuda())                 # device: one copy, one kernel
    f_dev = s.get_f()
    np.testing.assert_array_equal(f_host, f_dev)
    s.set_w(torch.from_numpy(w0).pin_memory())           # pinned host: chunked
    np.testing.assert_array_equal(s.get_f(), f_dev)
    s.step(cfg.dt, 2)
    w_host = s.get_w()                                   # pageable host: chunked
    w_pin = torch.empty(info.w_len, dtype=torch.float64).pin_memory()
    s.get_w(w_pin)                                       # pinned host: chunked
    w_dev = torch.empty(info.w_len, dtype=torch.float64, device="cuda")
    s.get_w(w_dev)                                       # device: one kernel
    s.synchronize()
    np.testing.assert_array_equal(w_host, w_dev.cpu().numpy())
    np.testing.assert_array_equal(w_pin.numpy(), w_host)
    assert np.isfinite(w_host).all()
    s.close()
