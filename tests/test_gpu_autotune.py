"""Launch-shape autotuner of the single-case Poisson solve: the chosen tile plan (FP64), or
block count or one-barrier tile plan (mixed), is a valid shape, the solve with it gives the fields of the built-in
shape within the solver tolerances, and the choice is cached per grid size."""
import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _case(nx, ny, precision, autotune, precond="jacobi"):
    c = I.small_cylinder(nx=nx, ny=ny, box=(-2.0, 6.0, -2.0, 2.0), r=0.5, cx=0.0, cy=0.0)
    c.precision, c.precond, c.autotune = precision, precond, autotune
    c.tol_p = 1e-12
    c.tol_h = 1e-13
    return c


@pytest.mark.parametrize("nx,ny", [(128, 64), (61, 20), (300, 36)])
def test_fp64_tile_plan(nx, ny):
    tuned = ccm.Case(_case(nx, ny, "fp64", 1))
    plain = ccm.Case(_case(nx, ny, "fp64", 0))
    tx, ty, nbx, ntiles, mb, cl, res = tuned.launch_plan()
    assert mb == 0
    if cl:
        assert cl in (2, 4, 8, 16) and cl <= ny and (tx, ty, nbx, ntiles, res) == (0, 0, 0, 0, 0)
    else:
        assert tx in (32, 64, 128, 256, 512) and ty >= 1
        assert nbx == -(-nx // tx) and ntiles == nbx * -(-ny // ty)
    assert plain.launch_plan() == (0,) * 7
    # the same size again: the cached plan
    assert ccm.Case(_case(nx, ny, "fp64", 1)).launch_plan() == (tx, ty, nbx, ntiles, mb, cl, res)
    st_t = tuned.step(3)
    st_p = plain.step(3)
    assert st_t["converged"] and st_p["converged"]
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
        assert _rel(tuned.get_field(f), plain.get_field(f)) < 1e-9, f


@pytest.mark.parametrize("precond", ["jacobi", "chebyshev"])
def test_mixed_block_count(precond):
    tuned = ccm.Case(_case(160, 64, "mixed", 1, precond))
    plain = ccm.Case(_case(160, 64, "mixed", 0, precond))
    plan = tuned.launch_plan()
    if plan[0]:
        # the one-barrier mixed solve's tiles (pcg_mixed1.cu), vectors resident or not, which
        # exclude a block count and a cluster
        tx, ty, nbx, ntiles = plan[:4]
        assert tx in (32, 64, 128, 256, 512) and ty >= 1
        assert nbx == -(-160 // tx) and ntiles == nbx * -(-64 // ty)
        assert plan[4:6] == (0, 0) and plan[6] in (0, 1)
    else:
        assert plan[:4] == (0, 0, 0, 0) and plan[5:] == (0, 0) and plan[4] >= 1
    assert ccm.Case(_case(160, 64, "mixed", 1, precond)).launch_plan() == plan
    st_t = tuned.step(3)
    st_p = plain.step(3)
    assert st_t["converged"] and st_p["converged"]
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
        assert _rel(tuned.get_field(f), plain.get_field(f)) < 1e-8, f


def test_singular_and_fp64_chebyshev_keep_builtin_shape():
    closed = I.small_cylinder(nx=37, ny=23, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, cx=0.07, cy=-0.05,
                              bc=I.closed_box_bc(lid=1.0), re=50.0)
    closed.autotune = 1
    assert ccm.Case(closed).launch_plan() == (0,) * 7
    assert ccm.Case(_case(64, 32, "fp64", 1, "chebyshev")).launch_plan() == (0,) * 7


@pytest.mark.parametrize("nx,ny,ctas", [(128, 64, 16), (128, 64, 2), (61, 20, 16), (96, 40, 8), (300, 36, 4)])
def test_cluster_solve_matches_tiled_solve(nx, ny, ctas):
    """The FP64 solve held in one thread-block cluster (bands of rows, neighbour rows through
    distributed shared memory) gives the fields of the tiled one-barrier solve."""
    clus = ccm.Case(_case(nx, ny, "fp64", 0))
    clus.set_launch_plan((0, 0, 0, 0, 0, ctas))
    assert clus.launch_plan()[5] == ctas
    tiled = ccm.Case(_case(nx, ny, "fp64", 0))
    st_c = clus.step(3)
    st_t = tiled.step(3)
    assert st_c["converged"] and st_t["converged"]
    assert abs(st_c["iters_p"] - st_t["iters_p"]) <= 3
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
        assert _rel(clus.get_field(f), tiled.get_field(f)) < 1e-9, f


def test_launch_plan_validation():
    c = ccm.Case(_case(128, 64, "fp64", 0))
    for bad in [(48, 8, 3, 24, 0, 0), (64, 8, 2, 15, 0, 0), (0, 0, 0, 0, 0, 3), (0, 0, 0, 0, 0, 128),
                (64, 8, 2, 16, 0, 8)]:
        with pytest.raises(ccm.CcmError):
            c.set_launch_plan(bad)
    big = ccm.Case(_case(1024, 512, "fp64", 0))
    with pytest.raises(ccm.CcmError):
        big.set_launch_plan((0, 0, 0, 0, 0, 16))  # a band of 32 rows does not fit shared memory
    c.set_launch_plan((64, 8, 2, 16, 0, 0))
    assert c.launch_plan() == (64, 8, 2, 16, 0, 0, 0)
    with pytest.raises(ccm.CcmError):
        c.set_launch_plan((0, 0, 0, 0, 0, 0, 1))  # resident tiles need a tile plan
    with pytest.raises(ccm.CcmError):
        big.set_launch_plan((512, 512, 2, 2, 0, 0, 1))  # a tile of 262144 cells cannot stay resident


@pytest.mark.parametrize("nx,ny,plan", [(1024, 512, (64, 27, 16, 304)), (128, 64, (128, 1, 1, 64)),
                                        (300, 36, (32, 4, 10, 90)), (61, 20, (32, 3, 2, 14)),
                                        (96, 40, (64, 5, 2, 16))])
def test_resident_tiles_match_global_tiles(nx, ny, plan):
    """The one-barrier FP64 solve with each tile's vectors kept in shared memory (only the
    perimeter published per iteration) gives the fields of the same tiles in global memory."""
    res = ccm.Case(_case(nx, ny, "fp64", 0))
    res.set_launch_plan(plan + (0, 0, 1))
    glob = ccm.Case(_case(nx, ny, "fp64", 0))
    glob.set_launch_plan(plan + (0, 0, 0))
    st_r = res.step(3)
    st_g = glob.step(3)
    assert st_r["converged"] and st_g["converged"]
    assert st_r["iters_p"] == st_g["iters_p"]
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
        assert _rel(res.get_field(f), glob.get_field(f)) < 1e-12, f
