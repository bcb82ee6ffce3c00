"""The FP64 helpers of the localisation finish on the device
(paper_2212_02988_gb300/csrc/linalg64.cuh), compiled with nvcc into a
temporary program:

* rcp64 (a third-order reciprocal iteration from a single-precision seed) is within
  one unit in the last place of CUDA's correctly rounded 1.0 / d over
  mantissas and exponents across its whole range;
* warp_ldlt6_solve (square-root-free Cholesky of a 6x6 SPD system on one
  warp) agrees with numpy's FP64 solve to the accuracy the condition number
  allows, and reports indefinite systems as not positive definite."""
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2212_02988_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    from paper_2212_02988_gb300 import build as B
    exe = str(tmp_path_factory.mktemp("linalg64") / "linalg64_check")
    subprocess.check_call([B.nvcc(), *B.ARCH, "-O3", "-std=c++17", "-fmad=false", "-I" + CSRC,
                           os.path.join(ROOT, "tests", "cuda", "linalg64_check.cu"), "-o", exe])
    return exe


def run(exe, ds, systems):
    lines = [str(len(ds))] + [f"{int(u):016x}" for u in np.asarray(ds, np.float64).view(np.uint64)]
    lines.append(str(len(systems)))
    for A, b in systems:
        tri = [A[i, j] for i in range(6) for j in range(i + 1)]
        lines += [f"{int(u):016x}" for u in np.asarray(tri + list(b), np.float64).view(np.uint64)]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    rcp, sol = [], []
    for ln in out.splitlines():
        f = ln.split()
        if f[0] == "rcp":
            rcp.append((int(f[1], 16), int(f[2], 16)))
        elif f[0] == "x":
            sol.append((np.array([int(v, 16) for v in f[1:7]], np.uint64).view(np.float64), int(f[7])))
    return rcp, sol


def test_rcp64_within_one_ulp_of_division(checker):
    rng = np.random.default_rng(3)
    e = rng.uniform(-1000, 1000, 20000)
    m = rng.uniform(1.0, 2.0, 20000)
    special = [1.0, 1.5, 2.0 - 2.0 ** -52, 1.0 + 2.0 ** -52, 3.0, 0.1, 7.0, 2.0 ** -1021, 2.0 ** 1021 * 1.999]
    ds = np.concatenate([m * 2.0 ** np.round(e), special])
    rcp, _ = run(checker, ds, [])
    got = np.array([a for a, _ in rcp], np.int64)
    ref = np.array([b for _, b in rcp], np.int64)
    assert np.all(np.abs(got - ref) <= 1), np.abs(got - ref).max()   # bit patterns of positive doubles
    assert np.mean(got == ref) > 0.9


def test_ldlt_solve_matches_numpy(checker):
    rng = np.random.default_rng(4)
    systems, conds = [], []
    for k in range(300):
        Q, _ = np.linalg.qr(rng.normal(size=(6, 6)))
        cond = 10.0 ** rng.uniform(0, 8)
        ev = np.exp(rng.uniform(0, np.log(cond), 6))
        ev[0], ev[-1] = 1.0, cond
        scale = 10.0 ** rng.uniform(-3, 7)
        A = scale * (Q * ev) @ Q.T
        A = 0.5 * (A + A.T)
        b = rng.normal(size=6) * scale
        systems.append((A, b))
        conds.append(cond)
    # indefinite and zero-pivot systems
    bad = np.diag([1.0, 2.0, -1.0, 3.0, 1.0, 1.0])
    systems += [(bad, np.ones(6)), (np.zeros((6, 6)), np.ones(6))]
    _, sol = run(checker, [], systems)
    for (A, b), cond, (x, pd) in zip(systems, conds, sol):
        assert pd == 1
        ref = np.linalg.solve(A, b)
        err = np.linalg.norm(x - ref) / np.linalg.norm(ref)
        assert err < 1e-15 * cond * 50 + 1e-14, (cond, err)
    assert sol[-2][1] == 0 and sol[-1][1] == 0
