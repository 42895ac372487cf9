"""Host dense algebra of the coarse space (csrc/coarse_host.cpp, plain C++, no GPU) on the
CPU: the k smallest eigenpairs of a symmetric tridiagonal (the Lanczos T_m of Sec. 3.3.2)
against LAPACK, and the Cholesky factor, the SPD inverse and the pivoted Gauss-Jordan
inverse of the coarse operator E = Z^T A Z (Eq. 12, App. C) against numpy.  Compiled
here with g++.  (The orthonormalisation with column dropping runs on the device; its
GPU test is in test_gpu_parity.py.)"""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg

from oracle import precond

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1408_3048_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <cstring>
#include <vector>
#include "coarse_host.h"
static std::vector<double> read_vec(size_t n) {
    std::vector<double> v(n);
    for (auto& x : v) if (std::scanf("%lf", &x) != 1) std::exit(2);
    return v;
}
static void put(const std::vector<double>& v) { for (double x : v) std::printf("%.17g\n", x); }
int main() {
    char cmd[16];
    int k;
    if (std::scanf("%15s %d", cmd, &k) != 2) return 2;
    if (!std::strcmp(cmd, "tri")) {
        int m;
        if (std::scanf("%d", &m) != 1) return 2;
        const std::vector<double> d = read_vec((size_t)m), e = read_vec((size_t)(m - 1));
        std::vector<double> theta, S;
        mm::tridiag_smallest(d, e, k, theta, S);
        put(theta);
        put(S);
    } else if (!std::strcmp(cmd, "chol")) {
        std::vector<double> L;
        const bool ok = mm::cholesky_lower(read_vec((size_t)k * k), k, L);
        std::printf("%d\n", ok ? 1 : 0);
        if (ok) put(mm::spd_inverse_from_cholesky(L, k));
        put(L);
    } else if (!std::strcmp(cmd, "lu")) {
        std::vector<double> inv;
        double ratio = -1.0;
        const bool ok = mm::lu_inverse(read_vec((size_t)k * k), k, inv, &ratio);
        std::printf("%d\n%.17g\n", ok ? 1 : 0, ratio);
        put(inv);
    } else {
        return 2;
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("coarse_host")
    (d / "main.cpp").write_text(DRIVER)
    exe = d / "coarse_host"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", SRC, str(d / "main.cpp"),
                    os.path.join(SRC, "coarse_host.cpp"), "-o", str(exe)], check=True)

    def call(head, *arrays):
        txt = head + " " + " ".join(" ".join(repr(float(v)) for v in np.ravel(a)) for a in arrays)
        out = subprocess.run([str(exe)], input=txt, capture_output=True, text=True, check=True).stdout
        return np.array(out.split(), dtype=np.float64)
    return call


@pytest.mark.parametrize("m,k", [(1, 1), (5, 3), (40, 8), (120, 32)])
def test_tridiagonal_smallest_eigenpairs(host, m, k):
    rng = np.random.default_rng(m)
    d = rng.uniform(0.5, 3.0, m)
    e = rng.uniform(0.05, 1.0, m - 1)
    out = host(f"tri {k} {m}", d, e)
    theta, S = out[:k], out[k:].reshape(m, k)
    ref = scipy.linalg.eigh_tridiagonal(d, e, eigvals_only=True)[:k]
    np.testing.assert_allclose(theta, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.abs(T @ S - S * theta).max() <= 1e-10 * np.abs(d).max()
    np.testing.assert_allclose(S.T @ S, np.eye(k), atol=1e-10)


def test_tridiagonal_of_a_lanczos_run(host):
    """T_m from the CG scalars of an oracle solve (Sec. 3.3.2): the library's smallest
    Ritz values equal LAPACK's on the same matrix."""
    rng = np.random.default_rng(1)
    n = 80
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.geomspace(1e-3, 1.0, n)) @ Q.T
    from oracle.pcg import pcg
    res = pcg(lambda x: A @ x, lambda r: r, rng.standard_normal(n), 1e-8, 60)
    T = precond.lanczos_tridiagonal(res.alphas, res.betas[: len(res.alphas) - 1])
    m = T.shape[0]
    k = min(10, m)
    out = host(f"tri {k} {m}", np.diag(T), np.diag(T, 1))
    ref = np.linalg.eigvalsh(T)[:k]
    np.testing.assert_allclose(out[:k], ref, rtol=0, atol=1e-13 * np.abs(np.diag(T)).max())


@pytest.mark.parametrize("k", [1, 4, 32, 64])
def test_cholesky_and_spd_inverse(host, k):
    rng = np.random.default_rng(k)
    B = rng.standard_normal((k, k))
    E = B @ B.T + k * np.eye(k)
    out = host(f"chol {k}", E)
    assert int(out[0]) == 1
    inv, L = out[1:1 + k * k].reshape(k, k), out[1 + k * k:].reshape(k, k)
    np.testing.assert_allclose(L, np.linalg.cholesky(E), rtol=1e-12, atol=1e-12)
    assert np.array_equal(inv, inv.T)
    np.testing.assert_allclose(inv, np.linalg.inv(E), rtol=0, atol=1e-12 * np.abs(np.linalg.inv(E)).max())


def test_cholesky_rejects_an_indefinite_matrix(host):
    E = np.array([[1.0, 2.0], [2.0, 1.0]])
    assert int(host("chol 2", E)[0]) == 0


@pytest.mark.parametrize("k", [1, 3, 16, 64])
def test_pivoted_inverse(host, k):
    rng = np.random.default_rng(100 + k)
    E = rng.standard_normal((k, k))
    out = host(f"lu {k}", E)
    ok, ratio, inv = int(out[0]), out[1], out[2:].reshape(k, k)
    assert ok == 1
    ref = np.linalg.inv(E)
    np.testing.assert_allclose(inv, ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    # partial pivoting takes LU's pivots: the smallest |U_ii| over the largest |E_ij|
    _, _, U = scipy.linalg.lu(E)
    assert ratio == pytest.approx(np.abs(np.diag(U)).min() / np.abs(E).max(), rel=1e-10)


def test_pivoted_inverse_of_a_singular_matrix(host):
    E = np.array([[1.0, 2.0], [2.0, 4.0]])
    out = host("lu 2", E)
    assert int(out[0]) == 0 or out[1] <= 1e-15
