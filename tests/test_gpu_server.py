"""Request loop: requests of different sizes, geometries, step counts and precision settings,
admitted against an HBM budget and advanced in chunks through the batches, end with the same
fields as each case stepped alone; admission is first-come first-served, the budget is never
exceeded, and requests submitted while others run join between rounds."""
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


def _specs():
    cs = [
        I.small_cylinder(nx=48, ny=24, box=(-2.0, 4.0, -1.5, 1.5), r=0.5, cx=0.0, cy=0.0),
        I.make_case("naca", 96, 48, (-0.5, 1.5, -0.5, 0.5),
                    I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=7.0), re=200.0, cfl=0.5, lref=1.0),
        I.small_cylinder(nx=96, ny=40, box=(-2.0, 4.0, -1.25, 1.25), r=0.43, cx=0.1, cy=-0.05),
        I.small_cylinder(nx=37, ny=23, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, cx=0.07, cy=-0.05,
                         bc=I.closed_box_bc(lid=1.0), re=50.0),
        I.small_cylinder(nx=64, ny=32, box=(-2.0, 4.0, -1.5, 1.5), r=0.45, cx=0.2, cy=0.1),
    ]
    for k, c in enumerate(cs):
        c.precision = "mixed" if k in (1, 4) else "fp64"
        c.tol_p = 1e-12 if c.precision == "mixed" else 1e-13
        c.tol_h = 1e-13
    return cs


FIELDS = (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P)


def _alone(spec, n):
    c = ccm.Case(spec)
    c.step(n)
    out = [c.get_field(f) for f in FIELDS]
    c.close()
    return out


def test_server_matches_alone_within_budget():
    specs = _specs()
    nsteps = [3, 5, 2, 4, 6]
    sizes = [ccm.case_bytes(c) for c in specs]
    budget = sizes[2] + max(sizes) + 1  # never room for all five at once
    srv = ccm.Server(budget, max_batch=4, chunk_steps=2)
    ids = [srv.submit(c, nsteps=n) for c, n in zip(specs, nsteps)]
    for _ in range(100):
        active = srv.run(1)
        assert srv.bytes_in_use() <= budget
        if active == 0:
            break
    assert active == 0
    polls = [srv.poll(i) for i in ids]
    admits = [p["t_admit"] for p in polls]
    assert admits == sorted(admits)  # first come, first served
    assert max(admits) > min(p["t_done"] for p in polls)  # some waited for memory
    for spec, n, rid, p in zip(specs, nsteps, ids, polls):
        assert p["state"] == "done" and p["steps"] == n and p["converged"]
        ref = _alone(spec, n)
        tol = 1e-8 if spec.precision == "mixed" else 1e-9
        for f, r in zip(FIELDS, ref):
            assert _rel(srv.get_field(rid, f, spec.shape), r) < tol, (spec.name, f)
    assert srv.bytes_in_use() == 0  # finished requests hold no device memory
    for rid in ids:
        srv.release(rid)
    srv.close()


def test_requests_join_between_rounds():
    specs = _specs()
    srv = ccm.Server(1 << 34, max_batch=8, chunk_steps=1)
    early = srv.submit(specs[0], nsteps=4)
    srv.run(2)
    late = srv.submit(specs[2], nsteps=2)
    assert srv.poll(late)["state"] == "queued"
    srv.run(1)
    assert srv.poll(late)["state"] == "running" and srv.poll(early)["state"] == "running"
    while srv.run(1):
        pass
    pe, pl = srv.poll(early), srv.poll(late)
    assert pe["state"] == pl["state"] == "done"
    assert pl["t_admit"] < pe["t_done"]
    for rid, spec, n in ((early, specs[0], 4), (late, specs[2], 2)):
        ref = _alone(spec, n)
        for f, r in zip(FIELDS, ref):
            assert _rel(srv.get_field(rid, f, spec.shape), r) < 1e-9
    srv.close()


def test_server_errors():
    specs = _specs()
    small = ccm.case_bytes(specs[0])
    srv = ccm.Server(small + 1, max_batch=2, chunk_steps=1)
    with pytest.raises(ccm.CcmError):
        srv.submit(specs[2], nsteps=1)  # can never fit the budget
    rid = srv.submit(specs[0], nsteps=3)
    srv.run(1)
    with pytest.raises(ccm.CcmError):
        srv.release(rid)  # still running
    with pytest.raises(ccm.CcmError):
        srv.poll(rid + 100)
    while srv.run(1):
        pass
    assert srv.bytes_in_use() == 0
    srv.release(rid)
    with pytest.raises(ccm.CcmError):
        srv.get_field(rid, ccm.CCM_F_U, specs[0].shape)  # released
    srv.close()
