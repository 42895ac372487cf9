// float instantiations of the overlap-save Toeplitz kernel (see toeplitz.cuh).
#include "toeplitz.cuh"

namespace mm {

template <>
size_t toeplitz_smem_bytes<float>(int logn) { return toeplitz_smem_bytes_impl<float>(logn); }

template <>
int toeplitz_max_logn<float>() { return 14; }

// Launch of the instance for the plan's FP32 block (single CTA or 2- / 4-CTA cluster).
static void dispatch_f32(const TzArgs<float>& A, const ToeplitzDev& tz, int mode, cudaStream_t s) {
    if (tz.cluster == 2 && tz.logn == 15) {
        launch_mode_cl<float, 14, 2>(A, tz.ntiles, mode, s);
        return;
    }
    if (tz.cluster == 4 && tz.logn == 16) {
        launch_mode_cl<float, 14, 4>(A, tz.ntiles, mode, s);
        return;
    }
    if (tz.cluster != 1) throw Error{MM_ERR_ARG, "unsupported cluster FFT length"};
    switch (tz.logn) {
        case 8: launch_mode<float, 8>(A, tz.ntiles, mode, s); break;
        case 9: launch_mode<float, 9>(A, tz.ntiles, mode, s); break;
        case 10: launch_mode<float, 10>(A, tz.ntiles, mode, s); break;
        case 11: launch_mode<float, 11>(A, tz.ntiles, mode, s); break;
        case 12: launch_mode<float, 12>(A, tz.ntiles, mode, s); break;
        case 13: launch_mode<float, 13>(A, tz.ntiles, mode, s); break;
        case 14: launch_mode<float, 14>(A, tz.ntiles, mode, s); break;
        default: throw Error{MM_ERR_ARG, "unsupported FFT length"};
    }
}

// Load mode from the inputs: y (mode 0), yd without x (2, FP32 only), yd with x (4 / 5,
// FP64 only), else the gather of x (1 / 3).
template <>
void launch_toeplitz_any<float>(const Plan& P, const ToeplitzDev& tz, const float* y, const double* yd, const float* x,
                             int R, int64_t in_stride, float* z, int64_t out_stride, const int* done, cudaStream_t s) {
    if (tz.logn == 0) throw Error{MM_ERR_ARG, "no FP32 Toeplitz block fits this lambda"};
    if (tz.ntiles == 0) return;
    TzArgs<float> A;
    A.tiles = tz.tiles;
    A.twiddle = static_cast<const float*>(tz.twiddle);
    A.ptw = static_cast<const typename Cx<float>::type*>(tz.ptw);
    A.H = static_cast<const float*>(tz.H);
    A.y = y;
    A.yd = yd;
    A.x = x;
    A.pixc = P.pixc;
    A.w = P.w32;
    A.z = z;
    A.done = done;
    A.lambda = P.lambda;
    A.R = R;
    A.in_stride = in_stride;
    A.out_stride = out_stride;
    A.pf_ahead = P.num_sms;
    const int mode = y != nullptr ? 0 : (yd != nullptr ? (x == nullptr ? 2 : (P.ncomp == 1 ? 4 : 5)) : (P.ncomp == 1 ? 1 : 3));
    dispatch_f32(A, tz, mode, s);
}

template <>
void launch_toeplitz<float>(const Plan& P, const ToeplitzDev& tz, const float* y, const float* x, float* z,
                         const int* done, cudaStream_t s) {
    launch_toeplitz_any<float>(P, tz, y, nullptr, x, 1, 0, z, 0, done, s);
}

template <>
void launch_toeplitz_rhs<float>(const Plan& P, const ToeplitzDev& tz, const float* y, const float* x, int R,
                             int64_t in_stride, float* z, int64_t out_stride, const int* done, cudaStream_t s) {
    launch_toeplitz_any<float>(P, tz, y, nullptr, x, R, in_stride, z, out_stride, done, s);
}

// x (I/Q/U interleaved, npix entries of three) -> map4 (one float4 per pixel)
__global__ void pack_map4_kernel(const float* __restrict__ x, float4* __restrict__ map4, int npix, const int* done) {
    if (done != nullptr && *(volatile const int*)done) return;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npix; q += gridDim.x * blockDim.x)
        map4[q] = make_float4(x[3 * (int64_t)q], x[3 * (int64_t)q + 1], x[3 * (int64_t)q + 2], 0.f);
}

void launch_toeplitz_f32_packed(const Plan& P, const float* x, bool pack, float* z, const int* done, cudaStream_t s) {
    if (P.map4 == nullptr || P.ncomp != 3) throw Error{MM_ERR_ARG, "packed gather: no packed map in this plan"};
    const ToeplitzDev& tz = P.tz32;
    if (tz.logn == 0) throw Error{MM_ERR_ARG, "no FP32 Toeplitz block fits this lambda"};
    if (tz.ntiles == 0) return;
    if (pack && P.npix_obs > 0) {
        const int threads = 256;
        const int blocks = std::max(1, std::min((P.npix_obs + threads - 1) / threads, P.num_sms * 8));
        pack_map4_kernel<<<blocks, threads, 0, s>>>(x, P.map4, P.npix_obs, done);
        check_cuda(cudaGetLastError(), "pack_map4 launch");
        note_launch();
    }
    TzArgs<float> A;
    A.tiles = tz.tiles;
    A.twiddle = static_cast<const float*>(tz.twiddle);
    A.ptw = static_cast<const typename Cx<float>::type*>(tz.ptw);
    A.H = static_cast<const float*>(tz.H);
    A.y = nullptr;
    A.yd = nullptr;
    A.x = x;
    A.pixc = P.pixc;
    A.w = P.w32;
    A.z = z;
    A.done = done;
    A.lambda = P.lambda;
    A.R = 1;
    A.in_stride = 0;
    A.out_stride = 0;
    A.pf_ahead = P.num_sms;
    A.x4 = P.map4;
    dispatch_f32(A, tz, 3, s);
}

}  // namespace mm
