"""Host numerics of the plan (csrc/plan_host.cpp, plain C++ run at plan time, no GPU)
against the oracle on the CPU: the Toeplitz rows of N^-1 from the PSD (Eq. 19, App. D,
Eq. 28), their derivatives in (sigma, f_knee, alpha), the positive-definiteness check of
the band, the overlap-save kernel spectrum, the 3x3 conditioning test of the I/Q/U
pixel blocks and the radix-2 FFT beneath them.  Compiled here with g++ against the CUDA
headers (nothing of the CUDA runtime is linked or called)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import adjoint as oadj
from oracle import noise as onoise
from oracle import pointing as opoint

try:
    from hypothesis import event, given, settings
    from hypothesis import strategies as st
except ImportError:   # the deterministic cases below still run
    given = None

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1408_3048_gb300", "csrc")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")

# commands on standard input, one per line; results on standard output, one per line
DRIVER = r"""
#include <cstdio>
#include <cstring>
#include <vector>
#include "mm_internal.h"
static std::vector<double> read_vec(int n) {
    std::vector<double> v((size_t)n);
    for (auto& x : v) if (std::scanf("%lf", &x) != 1) std::exit(2);
    return v;
}
static void put(const std::vector<double>& v) { for (double x : v) std::printf("%.17g\n", x); }
int main() {
    char cmd[16];
    while (std::scanf("%15s", cmd) == 1) {
        if (!std::strcmp(cmd, "row") || !std::strcmp(cmd, "deriv")) {
            double sigma, fknee, alpha, fsamp;
            long long L;
            int lam, window;
            if (std::scanf("%lf %lf %lf %lld %lf %d %d", &sigma, &fknee, &alpha, &L, &fsamp, &lam, &window) != 7)
                return 2;
            if (cmd[0] == 'r') put(mm::toeplitz_row(sigma, fknee, alpha, L, fsamp, lam, window));
            else for (const auto& d : mm::toeplitz_row_derivatives(sigma, fknee, alpha, L, fsamp, lam, window)) put(d);
        } else if (!std::strcmp(cmd, "sympos")) {
            int n;
            if (std::scanf("%d", &n) != 1) return 2;
            std::printf("%d\n", mm::symbol_positive(read_vec(n)) ? 1 : 0);
        } else if (!std::strcmp(cmd, "oss")) {
            long long N;
            int n;
            if (std::scanf("%lld %d", &N, &n) != 2) return 2;
            put(mm::overlap_save_spectrum(read_vec(n), N));
        } else if (!std::strcmp(cmd, "rcond")) {
            const std::vector<double> b = read_vec(6);
            std::printf("%.17g\n", mm::rcond_sym3(b.data()));
        } else if (!std::strcmp(cmd, "fft")) {
            int n, inverse;
            if (std::scanf("%d %d", &n, &inverse) != 2) return 2;
            std::vector<double> re = read_vec(n), im = read_vec(n);
            mm::host_fft(re, im, inverse != 0);
            put(re);
            put(im);
        } else {
            return 2;
        }
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    if not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("CUDA headers not available")
    d = tmp_path_factory.mktemp("plan_host")
    (d / "main.cpp").write_text(DRIVER)
    exe = d / "plan_host"
    subprocess.run(["g++", "-O2", "-std=c++17", "-I", SRC, "-I", CUDA_INC, str(d / "main.cpp"),
                    os.path.join(SRC, "plan_host.cpp"), "-o", str(exe)], check=True)

    def call(line):
        out = subprocess.run([str(exe)], input=line, capture_output=True, text=True, check=True).stdout
        return np.array(out.split(), dtype=np.float64)
    return call


def _nums(v):
    return " ".join(repr(float(x)) for x in np.ravel(v))


# (sigma, f_knee, alpha, L, lambda): 1/f spectra of the workloads, white noise, steep and
# shallow slopes, lambda from 0 to a quarter of the grid
ROWS = [(1.0, 1.0, 1.0, 2 ** 10, 6), (1.3, 0.5, 1.7, 2 ** 12, 64), (1.0, 0.1, 2.0, 2 ** 15, 1024),
        (0.7, 2.0, 1.2, 2 ** 17, 4096), (2.0, 0.0, 1.0, 2 ** 11, 100), (1.0, 1.5, 1.0, 2 ** 16, 16384),
        (1.0, 1.0, 1.0, 2 ** 8, 0)]


@pytest.mark.parametrize("sigma,fknee,alpha,L,lam", ROWS)
@pytest.mark.parametrize("window", [onoise.WINDOW_GAUSS, onoise.WINDOW_RECT])
def test_rows_match_the_oracle(host, sigma, fknee, alpha, L, lam, window):
    t = host(f"row {sigma} {fknee} {alpha} {L} 100.0 {lam} {window}")
    ref = onoise.toeplitz_row(sigma, fknee, alpha, L, 100.0, lam, window)
    assert t.shape == ref.shape
    assert np.abs(t - ref).max() <= 1e-13 * np.abs(ref).max()


if given is not None:
    @settings(max_examples=60, deadline=None, derandomize=True)
    @given(st.floats(0.3, 3.0), st.floats(0.0, 3.0), st.floats(0.5, 3.0), st.integers(3, 16), st.data())
    def test_random_rows_match_the_oracle(host, sigma, fknee, alpha, logL, data):
        L = 2 ** logL
        lam = data.draw(st.integers(0, min(L - 1, 2000)))   # past L/2 too: rows that wrap
        window = data.draw(st.sampled_from([onoise.WINDOW_GAUSS, onoise.WINDOW_RECT]))
        t = host(f"row {sigma!r} {fknee!r} {alpha!r} {L} 100.0 {lam} {window}")
        ref = onoise.toeplitz_row(sigma, fknee, alpha, L, 100.0, lam, window)
        assert np.abs(t - ref).max() <= 1e-13 * np.abs(ref).max()
        pos = bool(host(f"sympos {len(t)} {_nums(t)}")[0])
        event(f"positive definite: {pos}")
        assert pos == onoise.is_positive_definite(ref)


@pytest.mark.parametrize("sigma,fknee,alpha,L,lam", [r for r in ROWS if r[1] > 0])
def test_row_derivatives_match_the_oracle(host, sigma, fknee, alpha, L, lam):
    dt = host(f"deriv {sigma} {fknee} {alpha} {L} 100.0 {lam} {onoise.WINDOW_GAUSS}").reshape(3, lam + 1)
    ref = oadj.row_derivatives(sigma, fknee, alpha, L, 100.0, lam)
    for c in range(3):
        assert np.abs(dt[c] - ref[c]).max() <= 1e-12 * np.abs(ref[c]).max(), c


def test_symbol_check_matches_the_oracle(host):
    cases = [onoise.toeplitz_row(*r[:3], r[3], 100.0, r[4]) for r in ROWS]
    # a hard-truncated steep spectrum has a negative symbol (rejected by both)
    cases.append(onoise.toeplitz_row(1.0, 1.0, 4.0, 8192, 100.0, 64, onoise.WINDOW_RECT))
    # t_0 + 2 t_1 cos w: positive iff |t_1| < t_0 / 2
    cases += [np.array([1.0, -0.49]), np.array([1.0, -0.51]), np.array([1.0, 0.5]), np.array([1.0])]
    got = [bool(host(f"sympos {len(t)} {_nums(t)}")[0]) for t in cases]
    want = [onoise.is_positive_definite(t) for t in cases]
    assert got == want
    assert want[-5:] == [False, True, False, False, True]


@pytest.mark.parametrize("N,lam", [(8, 3), (512, 100), (16384, 4096)])
def test_overlap_save_spectrum(host, N, lam):
    """h_k = symbol(2 pi k / 2N) / N, k = 0..N: the even row laid out on 2N points."""
    t = onoise.toeplitz_row(1.0, 1.0, 1.5, 2 ** 15, 100.0, lam)
    h = host(f"oss {N} {len(t)} {_nums(t)}")
    ref = onoise.symbol_fft(t, 2 * N)[: N + 1] / N
    assert h.shape == (N + 1,)
    assert np.abs(h - ref).max() <= 1e-13 * np.abs(ref).max()


def test_rcond_sym3(host):
    rng = np.random.default_rng(7)
    blocks = []
    for _ in range(20):
        a = rng.standard_normal((3, 3))
        blocks.append(a @ a.T)
    blocks.append(np.diag([4.0, 1.0, 0.25]))               # diagonal: 1/16
    u = rng.standard_normal((3, 2))
    blocks.append(u @ u.T)                                  # rank 2: 0
    blocks.append(np.ones((3, 3)))                          # rank 1: 0
    blocks.append(np.diag([1.0, 1.0, 1.0]))
    B = np.array(blocks)
    got = np.array([host("rcond " + _nums(b[np.triu_indices(3)]))[0] for b in B])
    ref = opoint.rcond2(B)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    assert got[-4] == pytest.approx(1 / 16, abs=1e-15) and got[-1] == 1.0


@pytest.mark.parametrize("n", [1, 2, 8, 1024])
@pytest.mark.parametrize("inverse", [0, 1])
def test_host_fft(host, n, inverse):
    rng = np.random.default_rng(n)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    out = host(f"fft {n} {inverse} {_nums(z.real)} {_nums(z.imag)}")
    got = out[:n] + 1j * out[n:]
    ref = n * np.fft.ifft(z) if inverse else np.fft.fft(z)
    assert np.abs(got - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1.0)
