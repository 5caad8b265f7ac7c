"""chhs_energy_noalloc: the allocation-free way to get mass and energies.

Callers that cannot call cudaMalloc (a framework whose memory pool owns the
device, or a loop that cannot take an allocation's device-wide sync) use this
entry point instead of a handle.  It must report exactly what chhs_mass and
chhs_energy report for the same fields, call after call, although every call
reuses the library's one fixed scratch array.  This file is collected last on
purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1611_02967_gb300 import chhs, inputs

pytestmark = pytest.mark.gpu

REL = 1e-12  # the tolerance of the mass/energy parity test


def _close(a, b):
    return abs(a - b) <= REL * max(1.0, abs(b))


@pytest.mark.parametrize("shape,h,eps,gamma,dt", [
    ((64, 64), 0.05, 0.05, 1.0, 0.01),
    ((24, 40), 0.1, 0.08, 2.0, 0.01),
    ((16, 8, 12), 0.1, 0.08, 4.0, 0.005),
])
def test_noalloc_matches_handle_two_calls(shape, h, eps, gamma, dt):
    import torch
    with chhs.Run(shape, h, eps, gamma, dt) as run:
        run.set_phi(inputs.spinodal(shape, 77, mean=0.0, amplitude=0.5))
        run.step(3)
        phim, phimm1, _, _ = run.get_state()
        m_ref = run.mass()
        E_ref, F_ref = run.energy()
    dphi = torch.from_numpy(phim).cuda()
    dpsi = torch.from_numpy(phimm1).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    for _ in range(2):
        m, E, F = chhs.energy_noalloc(dphi, dpsi, h, eps, stream=stream)
        assert _close(m, m_ref) and _close(E, E_ref) and _close(F, F_ref), (m, m_ref, E, E_ref, F, F_ref)


def test_noalloc_rejects_oversize_grid():
    import torch
    small = torch.zeros(16, dtype=torch.float64, device="cuda")
    n = (ctypes.c_int * 3)(4096, 2048, 1)  # 8.4M cells > CHHS_NOALLOC_MAX_CELLS
    out = ctypes.c_double(0.0)
    s = chhs.lib().chhs_energy_noalloc(2, n, 0.1, 0.1, ctypes.c_void_p(small.data_ptr()), None, None,
                                       ctypes.byref(out), None, None)
    assert s == chhs.CHHS_ERR_INVALID_ARG
