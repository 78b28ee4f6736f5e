"""The pressure solve for callers that cannot allocate device memory.

Callers such as a host framework that owns all device memory through its own pool, a
process under a hard device-memory cap, or latency-sensitive code that must avoid the
device-wide synchronisation of cudaMalloc/cudaFree use ccm_solve_pressure_noalloc: the
same FP64 Jacobi-PCG as ccm_solve_pressure, with its scratch in one fixed device array of
the library.  This test calls it through the C ABI on device buffers of its own and checks
it against ccm_solve_pressure on the same case, twice in a row (the second call must not
see the first call's leftovers).  It sits in its own file, collected last."""
import ctypes

import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative L2: both entry points run the same FP64 kernel on the same inputs


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("which", ["cylinder", "closed_box"])
def test_noalloc_matches_allocating_solve(which):
    torch = pytest.importorskip("torch")
    if which == "cylinder":
        case = I.small_cylinder(nx=96, ny=48, box=(-2.0, 4.0, -1.5, 1.5), r=0.5, cx=0.0, cy=0.0)
    else:
        case = I.small_cylinder(nx=64, ny=40, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, cx=0.07, cy=-0.05,
                                bc=I.closed_box_bc())
    case.tol_p = 1e-12
    g = ccm.Case(case)
    rng = np.random.default_rng(123)
    rhs = rng.standard_normal(case.shape)
    if which == "closed_box":
        rhs -= rhs[1:-2, 1:-2].mean()

    # the allocating entry point, from a zero warm start
    g.set_field(ccm.CCM_F_PHI, np.zeros(case.shape))
    ref_stats = g.solve_pressure(rhs)
    phi_ref = g.get_field(ccm.CCM_F_PHI)

    # device buffers of the caller, in the case's pitched layout
    _, pitch = g.device_ptr(ccm.CCM_F_PHI)
    rows, cols = case.shape
    assert rows * pitch <= 131072
    rhs_d = torch.zeros((rows, pitch), dtype=torch.float64, device="cuda")
    rhs_d[:, :cols] = torch.from_numpy(rhs).cuda()
    for call in range(2):
        phi_d = torch.zeros((rows, pitch), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st = ccm.ccm_solve_stats()
        status = ccm.lib().ccm_solve_pressure_noalloc(g.h, ctypes.c_void_p(rhs_d.data_ptr()),
                                                      ctypes.c_void_p(phi_d.data_ptr()), ctypes.byref(st))
        assert status == ccm.CCM_OK, ccm.lib().ccm_last_error()
        got = phi_d[:, :cols].cpu().numpy()
        assert _rel(got, phi_ref) < TOL, (call, _rel(got, phi_ref))
        # same method; the sums run over another block layout, so the count may differ by rounding
        assert st.converged and abs(st.iters - ref_stats["iters"]) <= 2
    g.close()


def test_noalloc_rejects_grids_beyond_its_maximum():
    case = I.small_cylinder(nx=512, ny=256, box=(-2.0, 4.0, -1.5, 1.5), r=0.5, cx=0.0, cy=0.0)
    g = ccm.Case(case)
    dummy = ctypes.c_void_p(1)
    status = ccm.lib().ccm_solve_pressure_noalloc(g.h, dummy, dummy, None)
    assert status == ccm.CCM_E_INVALID
    assert b"too large" in ccm.lib().ccm_last_error()
    g.close()
