// Double-float Toeplitz kernels for the 2- and 4-CTA cluster blocks (see toeplitz_df.cu).
#include "toeplitz.cuh"

namespace mm {

template <int CL>
static void df_cl(const TzArgs<dfl>& A, int ntiles, int mode, cudaStream_t s) {
    if (mode == 4) return launch_cl<dfl, 13, 4, CL>(A, ntiles, s);
    if (mode == 5) return launch_cl<dfl, 13, 5, CL>(A, ntiles, s);
    throw Error{MM_ERR_ARG, "unsupported double-float Toeplitz load mode"};
}

void df_launch_cluster(const TzArgs<dfl>& A, int cluster, int ntiles, int mode, cudaStream_t s) {
    if (cluster == 2) return df_cl<2>(A, ntiles, mode, s);
    if (cluster == 4) return df_cl<4>(A, ntiles, mode, s);
    throw Error{MM_ERR_ARG, "unsupported cluster FFT length"};
}

}  // namespace mm
