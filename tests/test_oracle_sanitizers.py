"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: a build of ccm_oracle.c with
both (every report fatal) runs capacities, operators, solves and steps of several kinds of case
in a child process without a report.  CPU only."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r})
    import numpy as np
    import oracle
    oracle._LIB = {lib!r}
    from paper_2211_10698_gb300 import inputs as I

    cases = [
        I.small_cylinder(nx=24, ny=12),
        I.make_case("naca", 32, 16, (-0.5, 1.5, -0.5, 0.5),
                    I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=6.0), re=200.0, cfl=0.5, lref=1.0),
        I.small_cylinder(nx=24, ny=12, bc=I.closed_box_bc()),
        I.small_cylinder(nx=24, ny=12, box=(-2.0, 2.0, -1.0, 1.0), r=0.35, cx=0.1, bc=I.periodic_bc(True, False)),
        I.stretched_cylinder(nx=48, ny=40, fine=(16, 16)),
    ]
    for case in cases:
        case.precond = "jacobi"
        o = oracle.Oracle(case)
        st = o.init_state()
        o.step(st, 2)
        u, v = st["u"], st["v"]
        o.cont(u, v)
        o.pres(st["p"])
        sxx, syy, sxy = o.strain(u, v)
        o.visc(sxx, syy, sxy)
        o.conv(u, v)
        o.body_force(u, v, st["p"])
        o.kinetic(u, v)
    case = I.small_cylinder(nx=24, ny=12, precond="chebyshev", cheb_degree=3)
    o = oracle.Oracle(case)
    rng = np.random.default_rng(0)
    o.solve_poisson(rng.standard_normal(o.shape) * (o.cap("p", "V") > 0))
    st = o.init_state()
    st["Dx"], st["Dy"] = rng.standard_normal(o.shape) * 0.1, rng.standard_normal(o.shape) * 0.1
    st["motion"] = (0.5, 0.5, 3.0, 0.0)
    st["gx"], st["gy"] = np.full(o.shape, 0.1), np.zeros(o.shape)
    o.step(st, 2)
    print("sanitized oracle ok")
""")


def test_oracle_runs_clean_under_asan_and_ubsan(tmp_path):
    asan = subprocess.run(["gcc", "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("gcc has no AddressSanitizer runtime here")
    lib = str(tmp_path / "liboracle_san.so")
    src = os.path.join(ROOT, "oracle", "ccm_oracle.c")
    subprocess.check_call(["gcc", "-std=c11", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                           "-fno-sanitize-recover=all", "-ffp-contract=off", "-fPIC", "-shared", "-o", lib, src, "-lm"])
    script = tmp_path / "run.py"
    script.write_text(SCRIPT.format(root=ROOT, lib=lib))
    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1")
    r = subprocess.run([sys.executable, str(script)], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "sanitized oracle ok" in r.stdout
