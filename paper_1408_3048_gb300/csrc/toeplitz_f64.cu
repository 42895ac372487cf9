// double instantiations of the overlap-save Toeplitz kernel (see toeplitz.cuh).
#include "toeplitz.cuh"

namespace mm {

template <>
size_t toeplitz_smem_bytes<double>(int logn) { return toeplitz_smem_bytes_impl<double>(logn); }

template <>
int toeplitz_max_logn<double>() { return 13; }

// Load mode from the inputs: y (mode 0), yd without x (2, FP32 only), yd with x (4 / 5,
// FP64 only), else the gather of x (1 / 3).
template <>
void launch_toeplitz_any<double>(const Plan& P, const ToeplitzDev& tz, const double* y, const double* yd, const double* x,
                             int R, int64_t in_stride, double* z, int64_t out_stride, const int* done, cudaStream_t s) {
    if (tz.logn == 0) throw Error{MM_ERR_ARG, "no FP64 Toeplitz block fits this lambda"};
    if (tz.ntiles == 0) return;
    TzArgs<double> A;
    A.tiles = tz.tiles;
    A.twiddle = static_cast<const double*>(tz.twiddle);
    A.ptw = static_cast<const typename Cx<double>::type*>(tz.ptw);
    A.H = static_cast<const double*>(tz.H);
    A.y = y;
    A.yd = yd;
    A.x = x;
    A.pixc = P.pixc;
    A.w = P.w64;
    A.z = z;
    A.done = done;
    A.lambda = P.lambda;
    A.R = R;
    A.in_stride = in_stride;
    A.out_stride = out_stride;
    A.pf_ahead = P.num_sms;
    const int mode = y != nullptr ? 0 : (yd != nullptr ? (x == nullptr ? 2 : (P.ncomp == 1 ? 4 : 5)) : (P.ncomp == 1 ? 1 : 3));
    if (tz.cluster == 2 && tz.logn == 14) {
        launch_mode_cl<double, 13, 2>(A, tz.ntiles, mode, s);
        return;
    }
    if (tz.cluster == 4 && tz.logn == 15) {
        launch_mode_cl<double, 13, 4>(A, tz.ntiles, mode, s);
        return;
    }
    if (tz.cluster != 1) throw Error{MM_ERR_ARG, "unsupported cluster FFT length"};
    switch (tz.logn) {
        case 8: launch_mode<double, 8>(A, tz.ntiles, mode, s); break;
        case 9: launch_mode<double, 9>(A, tz.ntiles, mode, s); break;
        case 10: launch_mode<double, 10>(A, tz.ntiles, mode, s); break;
        case 11: launch_mode<double, 11>(A, tz.ntiles, mode, s); break;
        case 12: launch_mode<double, 12>(A, tz.ntiles, mode, s); break;
        case 13: launch_mode<double, 13>(A, tz.ntiles, mode, s); break;
        default: throw Error{MM_ERR_ARG, "unsupported FFT length"};
    }
}

template <>
void launch_toeplitz<double>(const Plan& P, const ToeplitzDev& tz, const double* y, const double* x, double* z,
                         const int* done, cudaStream_t s) {
    launch_toeplitz_any<double>(P, tz, y, nullptr, x, 1, 0, z, 0, done, s);
}

template <>
void launch_toeplitz_rhs<double>(const Plan& P, const ToeplitzDev& tz, const double* y, const double* x, int R,
                             int64_t in_stride, double* z, int64_t out_stride, const int* done, cudaStream_t s) {
    launch_toeplitz_any<double>(P, tz, y, nullptr, x, R, in_stride, z, out_stride, done, s);
}

}  // namespace mm
