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


def _cylinder(**kw):
    return I.small_cylinder(nx=96, ny=48, box=(-2.0, 4.0, -1.5, 1.5), r=0.5, cx=0.0, cy=0.0, **kw)


@pytest.mark.parametrize("which", ["cylinder", "closed_box", "cylinder_chebyshev", "cylinder_mixed"])
def test_noalloc_matches_allocating_solve(which):
    """The no-allocation solve equals ccm_solve_pressure.  For a case configured for Chebyshev
    or mixed precision it still runs FP64 Jacobi-PCG, so it is compared with the allocating
    solve of the same system on an FP64 Jacobi case; both then stop at a residual of 1e-13,
    and their solutions agree to the system's conditioning times that."""
    torch = pytest.importorskip("torch")
    tol, iters_slack = TOL, 2
    if which == "closed_box":
        case = I.small_cylinder(nx=64, ny=40, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, cx=0.07, cy=-0.05,
                                bc=I.closed_box_bc())
    elif which == "cylinder_chebyshev":
        case = _cylinder(precond="chebyshev", cheb_degree=4)
    elif which == "cylinder_mixed":
        case = _cylinder(precision="mixed")
    else:
        case = _cylinder()
    case.tol_p = 1e-12
    rng = np.random.default_rng(123)
    rhs = rng.standard_normal(case.shape)
    if which == "closed_box":
        rhs -= rhs[1:-2, 1:-2].mean()

    # the allocating entry point, from a zero warm start, on an FP64 Jacobi case of the system
    ref_case = case
    if which in ("cylinder_chebyshev", "cylinder_mixed"):
        case.tol_p = 1e-13
        ref_case = _cylinder()
        ref_case.tol_p = 1e-13
        tol, iters_slack = 1e-9, None
    gr = ccm.Case(ref_case)
    gr.set_field(ccm.CCM_F_PHI, np.zeros(case.shape))
    ref_stats = gr.solve_pressure(rhs)
    phi_ref = gr.get_field(ccm.CCM_F_PHI)
    if ref_case is case:
        g = gr
    else:
        gr.close()
        g = ccm.Case(case)

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
        assert _rel(got, phi_ref) < tol, (call, _rel(got, phi_ref))
        assert st.converged and st.rel_res <= case.tol_p
        if iters_slack is not None:
            # same method; the sums run over another block layout, so the count may differ by rounding
            assert abs(st.iters - ref_stats["iters"]) <= iters_slack
    g.close()


def test_noalloc_rejects_grids_beyond_its_maximum():
    case = I.small_cylinder(nx=512, ny=256, box=(-2.0, 4.0, -1.5, 1.5), r=0.5, cx=0.0, cy=0.0)
    g = ccm.Case(case)
    dummy = ctypes.c_void_p(1)
    status = ccm.lib().ccm_solve_pressure_noalloc(g.h, dummy, dummy, None)
    assert status == ccm.CCM_E_INVALID
    assert b"too large" in ccm.lib().ccm_last_error()
    g.close()
