// Time-domain helpers of the adjoint / noise-PSD gradient:
//   sub_time       out = a - b over the samples (residual d - P m)
//   interval_dot   part[i] = sum_{t in interval i} u_t w_t, one block per interval,
//                  fixed-order block reduction (the host adds the intervals of each PSD
//                  id in interval order, so the gradient is reproducible)
#include "mm_internal.h"

namespace mm {

__global__ void sub_time_kernel(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                                int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

void launch_sub_time(const double* a, const double* b, double* out, int64_t n, cudaStream_t s) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    sub_time_kernel<<<(int)g, 256, 0, s>>>(a, b, out, n);
    check_cuda(cudaGetLastError(), "sub_time launch");
    note_launch();
}

__global__ void interval_dot_kernel(const double* __restrict__ u, const double* __restrict__ w,
                                    const int64_t* __restrict__ ioff, double* __restrict__ part) {
    __shared__ double sh[32];
    const int64_t a = ioff[blockIdx.x], b = ioff[blockIdx.x + 1];
    double s = 0.0;
    for (int64_t t = a + threadIdx.x; t < b; t += blockDim.x) s += u[t] * w[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
        part[blockIdx.x] = t;
    }
}

void launch_interval_dot(const double* u, const double* w, const int64_t* ioff, int K, double* part,
                         cudaStream_t s) {
    interval_dot_kernel<<<K, 256, 0, s>>>(u, w, ioff, part);
    check_cuda(cudaGetLastError(), "interval_dot launch");
    note_launch();
}

}  // namespace mm
