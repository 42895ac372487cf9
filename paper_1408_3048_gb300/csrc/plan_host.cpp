// Host-side FP64 numerics of the plan: the Toeplitz rows of N^-1 from the noise PSD
// (Eq. 19; App. D and Eq. 28), their positive-definiteness check, the overlap-save
// spectra, and the conditioning test of a 3x3 polarisation block.
//
// The FFT here is a plain iterative radix-2 Cooley-Tukey transform written for this
// library (plan time only; the solver's FFTs run on the GPU).
#include <cmath>
#include <stdexcept>

#include "mm_internal.h"

namespace mm {

static const double kPi = 3.14159265358979323846264338327950288;

// In-place complex FFT of length 2^m (re, im), forward sign exp(-2 pi i jk/n).
// inverse = true uses exp(+2 pi i jk/n) and no 1/n scaling.
void host_fft(std::vector<double>& re, std::vector<double>& im, bool inverse) {
    const size_t n = re.size();
    if (n == 0 || (n & (n - 1)) != 0 || im.size() != n) throw Error{MM_ERR_ARG, "host_fft: size"};
    // bit reversal
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    const double sgn = inverse ? 1.0 : -1.0;
    for (size_t len = 2; len <= n; len <<= 1) {
        const size_t half = len >> 1;
        // twiddles of this stage evaluated directly (no recurrence drift)
        std::vector<double> wc(half), ws(half);
        for (size_t k = 0; k < half; ++k) {
            const double a = 2.0 * kPi * (double)k / (double)len;
            wc[k] = std::cos(a);
            ws[k] = sgn * std::sin(a);
        }
        for (size_t i = 0; i < n; i += len) {
            for (size_t k = 0; k < half; ++k) {
                const size_t a = i + k, b = i + k + half;
                const double xr = re[b] * wc[k] - im[b] * ws[k];
                const double xi = re[b] * ws[k] + im[b] * wc[k];
                re[b] = re[a] - xr;
                im[b] = im[a] - xi;
                re[a] += xr;
                im[a] += xi;
            }
        }
    }
}

// t_k = w_k r_k, k = 0..lam, with
//   r_k = (1/L) sum_{j=0}^{L-1} S_{min(j, L-j)}^-1 cos(2 pi j k / L),
//   S_j = sigma^2 (1 + (fknee / f_j)^alpha), f_j = j fsamp / L, S_0^-1 = lim_{f->0},
//   w_k = exp(-2 (k / lam)^2) (GAUSS) or 1 (RECT).
std::vector<double> toeplitz_row(double sigma, double fknee, double alpha, int64_t L,
                                 double fsamp, int lam, int window) {
    std::vector<double> re((size_t)L), im((size_t)L, 0.0);
    const double s2 = sigma * sigma;
    for (int64_t j = 0; j < L; ++j) {
        const int64_t jj = j <= L - j ? j : L - j;
        double inv;
        if (jj == 0) {
            inv = fknee > 0.0 ? 0.0 : 1.0 / s2;
        } else {
            const double f = (double)jj * fsamp / (double)L;
            inv = 1.0 / (s2 * (1.0 + std::pow(fknee / f, alpha)));
        }
        re[(size_t)j] = inv;
    }
    host_fft(re, im, true);
    std::vector<double> t((size_t)lam + 1);
    for (int k = 0; k <= lam; ++k) {
        double w = 1.0;
        if (window == MM_WINDOW_GAUSS && lam > 0) {
            const double u = (double)k / (double)lam;
            w = std::exp(-2.0 * u * u);
        }
        t[(size_t)k] = w * re[(size_t)k] / (double)L;
    }
    return t;
}

// dt_k / d(sigma, fknee, alpha), k = 0..lam: the row transform above applied to the
// analytic derivatives of 1/S_j (zero at j = 0; needs fknee > 0):
//   d(1/S)/dsigma = -(2/sigma)/S,  d(1/S)/dfknee = -(1/S) alpha x / (fknee (1+x)),
//   d(1/S)/dalpha = -(1/S) x ln(fknee/f) / (1+x),  x = (fknee/f)^alpha.
std::vector<std::vector<double>> toeplitz_row_derivatives(double sigma, double fknee, double alpha, int64_t L,
                                                          double fsamp, int lam, int window) {
    std::vector<std::vector<double>> out(3, std::vector<double>((size_t)lam + 1));
    for (int c = 0; c < 3; ++c) {
        std::vector<double> re((size_t)L), im((size_t)L, 0.0);
        for (int64_t j = 0; j < L; ++j) {
            const int64_t jj = j <= L - j ? j : L - j;
            double v = 0.0;
            if (jj > 0) {
                const double f = (double)jj * fsamp / (double)L;
                const double x = std::pow(fknee / f, alpha);
                const double invS = 1.0 / (sigma * sigma * (1.0 + x));
                if (c == 0) v = -2.0 / sigma * invS;
                else if (c == 1) v = -invS * alpha * x / (fknee * (1.0 + x));
                else v = -invS * x * std::log(fknee / f) / (1.0 + x);
            }
            re[(size_t)j] = v;
        }
        host_fft(re, im, true);
        for (int k = 0; k <= lam; ++k) {
            double w = 1.0;
            if (window == MM_WINDOW_GAUSS && lam > 0) {
                const double u = (double)k / (double)lam;
                w = std::exp(-2.0 * u * u);
            }
            out[(size_t)c][(size_t)k] = w * re[(size_t)k] / (double)L;
        }
    }
    return out;
}

// Spectrum of the even kernel (t_|k| for |k| <= lam, 0 beyond) laid out circularly over
// M points: sigma(2 pi m / M) = t_0 + 2 sum_k t_k cos(2 pi m k / M), m = 0..M-1.
static std::vector<double> kernel_spectrum(const std::vector<double>& t, int64_t M) {
    std::vector<double> re((size_t)M, 0.0), im((size_t)M, 0.0);
    const int64_t lam = (int64_t)t.size() - 1;
    re[0] = t[0];
    for (int64_t k = 1; k <= lam; ++k) {
        re[(size_t)k] = t[(size_t)k];
        re[(size_t)(M - k)] = t[(size_t)k];
    }
    host_fft(re, im, false);
    return re;
}

// Reading R4: positive on M = 2^ceil(log2(max(8 lam, 8))) frequencies.
bool symbol_positive(const std::vector<double>& t) {
    const int64_t lam = (int64_t)t.size() - 1;
    int64_t M = 1;
    while (M < (8 * lam > 8 ? 8 * lam : 8)) M *= 2;
    const std::vector<double> s = kernel_spectrum(t, M);
    for (double v : s)
        if (!(v > 0.0)) return false;
    return true;
}

// Overlap-save spectrum for a real block of B = 2N samples, k = 0..N, divided by N.
std::vector<double> overlap_save_spectrum(const std::vector<double>& t, int64_t N) {
    const std::vector<double> s = kernel_spectrum(t, 2 * N);
    std::vector<double> h((size_t)N + 1);
    for (int64_t k = 0; k <= N; ++k) h[(size_t)k] = s[(size_t)k] / (double)N;
    return h;
}

// Twiddles of the in-shared-memory Stockham FFT (toeplitz.cuh): for every pass after the
// first, radix R = 16 (8 for N < 512) or the remainder, Ns = product of the earlier
// radices, entry [(r - 1) Ns + k] = (cos, sin) of 2 pi r k / (Ns R).  Same pass schedule
// as fft_all on the device.
std::vector<double> pass_twiddle_table(int logn) {
    const int maxr = ((1 << logn) / 16 >= 32) ? 4 : 3;
    std::vector<double> out;
    int l = 0;
    while (l < logn) {
        const int rem = logn - l;
        const int lr = rem >= maxr ? maxr : rem;
        const int64_t Ns = int64_t(1) << l, R = int64_t(1) << lr;
        // (the first pass, Ns = 1, reads no twiddles but keeps its R - 1 slots so the
        // offsets match ptw_offset on the device)
        for (int64_t r = 1; r < R; ++r)
            for (int64_t k = 0; k < Ns; ++k) {
                const double ang = 2.0 * kPi * (double)((r * k) % (Ns * R)) / (double)(Ns * R);
                out.push_back(std::cos(ang));
                out.push_back(std::sin(ang));
            }
        l += lr;
    }
    return out;
}

// lambda_min / lambda_max of a symmetric 3x3 block given packed (a00 a01 a02 a11 a12 a22),
// by cyclic Jacobi rotations (converges to working precision in a few sweeps).
double rcond_sym3(const double Bp[6]) {
    double a[3][3] = {{Bp[0], Bp[1], Bp[2]}, {Bp[1], Bp[3], Bp[4]}, {Bp[2], Bp[4], Bp[5]}};
    for (int sweep = 0; sweep < 50; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-36 * dia || off == 0.0) break;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double tt = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(tt * tt + 1.0), s = tt * c;
                for (int k = 0; k < 3; ++k) {   // A <- A J
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {   // A <- J^T A
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
            }
        }
    }
    double lo = a[0][0], hi = a[0][0];
    for (int i = 1; i < 3; ++i) {
        lo = a[i][i] < lo ? a[i][i] : lo;
        hi = a[i][i] > hi ? a[i][i] : hi;
    }
    if (!(hi > 0.0)) return 0.0;
    const double r = lo / hi;
    return r > 0.0 ? r : 0.0;
}

}  // namespace mm
