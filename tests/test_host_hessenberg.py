"""Host linear algebra of the Arnoldi coarse construction (csrc/coarse_host.cpp, plain
C++, no GPU): the Hessenberg eigen-solver and inverse iteration against LAPACK (numpy)
on random upper Hessenberg matrices with real and complex eigenvalues, and on Arnoldi
Hessenbergs of M_BD A from the oracle.  Compiled here with g++."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1408_3048_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <vector>
#include "coarse_host.h"
int main() {
    int n;
    if (std::scanf("%d", &n) != 1) return 2;
    std::vector<double> H((size_t)n * n);
    for (auto& v : H) if (std::scanf("%lf", &v) != 1) return 2;
    std::vector<std::complex<double>> lam;
    if (!mm::hessenberg_eigenvalues(H, n, lam)) return 3;
    for (int i = 0; i < n; ++i) {
        std::printf("%.17g %.17g\n", lam[i].real(), lam[i].imag());
        auto v = mm::hessenberg_eigenvector(H, n, lam[i]);
        for (int q = 0; q < n; ++q) std::printf("%.17g %.17g\n", v[q].real(), v[q].imag());
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("hess")
    (d / "main.cpp").write_text(DRIVER)
    exe = d / "hess"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", SRC, str(d / "main.cpp"), os.path.join(SRC, "coarse_host.cpp"),
                    "-o", str(exe)], check=True)
    return str(exe)


def run(exe, H):
    n = H.shape[0]
    txt = f"{n}\n" + " ".join(repr(float(v)) for v in H.ravel())
    out = subprocess.run([exe], input=txt, capture_output=True, text=True, check=True).stdout.split()
    vals = np.array(out, dtype=np.float64).reshape(-1, 2)
    lam, vecs = [], []
    for i in range(n):
        blk = vals[i * (n + 1):(i + 1) * (n + 1)]
        lam.append(complex(*blk[0]))
        vecs.append(blk[1:, 0] + 1j * blk[1:, 1])
    return np.array(lam), vecs


def check(exe, H):
    lam, vecs = run(exe, H)
    ref = np.linalg.eigvals(H)
    # eigenvalues as multisets (match greedily)
    scale = np.abs(ref).max()
    left = list(ref)
    for l in lam:
        i = int(np.argmin([abs(l - r) for r in left]))
        assert abs(l - left[i]) <= 1e-9 * scale
        left.pop(i)
    for l, v in zip(lam, vecs):
        assert np.linalg.norm(H @ v - l * v) <= 1e-9 * scale * np.linalg.norm(v)
        assert np.linalg.norm(v) == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 40])
def test_random_hessenberg(driver, n):
    rng = np.random.default_rng(n)
    H = np.triu(rng.standard_normal((n, n)), -1)   # general: complex pairs appear
    check(driver, H)


def test_rotation_block_and_defective_like(driver):
    # exact complex pair (rotation) and a nearly repeated real eigenvalue
    H = np.array([[0.0, -1.0, 0.3], [1.0, 0.0, 0.2], [0.0, 1e-9, 2.0]])
    check(driver, H)
    H2 = np.array([[1.0, 1.0, 0.0], [1e-6, 1.0, 1.0], [0.0, 1e-6, 1.0]])
    check(driver, H2)


def test_arnoldi_hessenberg_of_map_making(driver):
    # the matrices the coarse construction meets: Arnoldi on M_BD A (oracle)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from problems import oracle_problem, tiny_scan
    from oracle import precond
    prob = oracle_problem(tiny_scan(ncomp=3, psds=((1.0, 3.0, 1.8), (1.2, 1.5, 1.2)), lam=10))
    bd = precond.BlockJacobi(prob)
    b = prob.rhs(np.random.default_rng(2).standard_normal(prob.nt))
    W, H, _, _ = precond.arnoldi(lambda x: bd.apply(prob.A(x)), bd.apply(b), 30)
    j = H.shape[1]
    check(driver, H[:j, :j])
