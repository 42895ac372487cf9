// Double-float Toeplitz kernels for single-CTA blocks of 2^12 .. 2^14 reals (see
// toeplitz_df.cu).
#include "toeplitz.cuh"

namespace mm {

template <int LOGN>
static void df_single_l(const TzArgs<dfl>& A, int ntiles, int mode, cudaStream_t s) {
    if (mode == 4) return launch_one<dfl, LOGN, 4>(A, ntiles, s);
    if (mode == 5) return launch_one<dfl, LOGN, 5>(A, ntiles, s);
    throw Error{MM_ERR_ARG, "unsupported double-float Toeplitz load mode"};
}

void df_launch_large(const TzArgs<dfl>& A, int logn, int ntiles, int mode, cudaStream_t s) {
    switch (logn) {
        case 11: return df_single_l<11>(A, ntiles, mode, s);
        case 12: return df_single_l<12>(A, ntiles, mode, s);
        case 13: return df_single_l<13>(A, ntiles, mode, s);
        default: break;
    }
    throw Error{MM_ERR_ARG, "unsupported FFT length"};
}

}  // namespace mm
