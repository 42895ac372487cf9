// Double-float instantiations of the overlap-save Toeplitz kernel (see toeplitz.cuh and
// dfloat.cuh): N^-1 of Eq. 4 on FP64 data with the FFT in double-float arithmetic on the
// FP32 pipe, for the refinement residual P^T N^-1 (d - P x) of the mixed solver (Eq. 5,
// 7).  Same blocks, tiles and thread counts as the FP64 kernel.
#include "toeplitz.cuh"

namespace mm {

// Launchers of the instantiations, spread over three translation units so that they
// compile in parallel (toeplitz_df.cu: blocks 2^9 .. 2^11 reals; toeplitz_df_large.cu:
// 2^12 .. 2^14; toeplitz_df_cluster.cu: the 2- and 4-CTA cluster blocks).  Only the
// residual loads (modes 4 and 5, d - P x) are built.
void df_launch_large(const TzArgs<dfl>& A, int logn, int ntiles, int mode, cudaStream_t s);
void df_launch_cluster(const TzArgs<dfl>& A, int cluster, int ntiles, int mode, cudaStream_t s);

template <int LOGN>
static void df_single(const TzArgs<dfl>& A, int ntiles, int mode, cudaStream_t s) {
    if (mode == 4) return launch_one<dfl, LOGN, 4>(A, ntiles, s);
    if (mode == 5) return launch_one<dfl, LOGN, 5>(A, ntiles, s);
    throw Error{MM_ERR_ARG, "unsupported double-float Toeplitz load mode"};
}

void launch_toeplitz_df(const Plan& P, const double* y, const double* d, const double* x, int R, int64_t in_stride,
                        double* z, int64_t out_stride, cudaStream_t s) {
    const ToeplitzDev& tz = P.tzdf;
    if (tz.logn == 0) throw Error{MM_ERR_ARG, "no double-float Toeplitz block for this plan"};
    if (tz.ntiles == 0) return;
    TzArgs<dfl> A;
    A.tiles = tz.tiles;
    A.twiddle = static_cast<const dfl*>(tz.twiddle);
    A.ptw = static_cast<const dfl2*>(tz.ptw);
    A.H = static_cast<const dfl*>(tz.H);
    A.y = y;
    A.yd = d;
    A.x = x;
    A.pixc = P.pixc;
    A.w = P.w64;
    A.z = z;
    A.done = nullptr;
    A.lambda = P.lambda;
    A.R = R;
    A.in_stride = in_stride;
    A.out_stride = out_stride;
    A.pf_ahead = P.num_sms;
    if (y != nullptr || d == nullptr || x == nullptr)
        throw Error{MM_ERR_ARG, "double-float Toeplitz: only the residual data d - P x is supported"};
    const int mode = P.ncomp == 1 ? 4 : 5;
    if (tz.cluster != 1) return df_launch_cluster(A, tz.cluster, tz.ntiles, mode, s);
    switch (tz.logn) {
        case 8: return df_single<8>(A, tz.ntiles, mode, s);
        case 9: return df_single<9>(A, tz.ntiles, mode, s);
        case 10: return df_single<10>(A, tz.ntiles, mode, s);
        default: return df_launch_large(A, tz.logn, tz.ntiles, mode, s);
    }
    throw Error{MM_ERR_ARG, "unsupported FFT length"};
}

}  // namespace mm
