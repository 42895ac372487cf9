// Device kernels of the coarse-space construction (Sec. 3.3.2, App. A and C):
//   lincomb  out[c][i] = sum_j V[j][i] C[j][c]   (Ritz vectors from the stored z_j;
//                                                  Y W re-orthonormalisation)
//   gram     per-block partials of A^T B         (Y^T Y, and E = Z^T (A Z))
// FP64 accumulation; partial sums are reduced on the host in block order, so the
// results are reproducible.
#include "coarse.cuh"

namespace mm {

template <typename TIN>
__global__ void lincomb_kernel(const TIN* __restrict__ V, int m, int64_t n, const double* __restrict__ C,
                               int kk, double* __restrict__ out) {
    constexpr int CH = 8;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int c0 = 0; c0 < kk; c0 += CH) {
            double acc[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) acc[c] = 0.0;
            for (int j = 0; j < m; ++j) {
                const double v = (double)V[(size_t)j * n + i];
                const double* cj = C + (size_t)j * kk + c0;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    if (c0 + c < kk) acc[c] += v * cj[c];
            }
#pragma unroll
            for (int c = 0; c < CH; ++c)
                if (c0 + c < kk) out[(size_t)(c0 + c) * n + i] = acc[c];
        }
    }
}

template <typename TIN>
void launch_lincomb(const TIN* V, int m, int64_t n, const double* C, int kk, double* out, cudaStream_t s) {
    const int th = 256;
    int64_t g = (n + th - 1) / th;
    if (g > 4096) g = 4096;
    lincomb_kernel<TIN><<<(int)g, th, 0, s>>>(V, m, n, C, kk, out);
    check_cuda(cudaGetLastError(), "lincomb launch");
    note_launch();
}
template void launch_lincomb<double>(const double*, int, int64_t, const double*, int, double*, cudaStream_t);
template void launch_lincomb<float>(const float*, int, int64_t, const double*, int, double*, cudaStream_t);

// Each block reduces rows [b*chunk, (b+1)*chunk) through 32-row shared-memory tiles.
__global__ void gram_kernel(const double* __restrict__ A, int ka, const double* __restrict__ B, int kb,
                            int64_t n, int64_t chunk, double* __restrict__ part) {
    __shared__ double sa[GRAM_KMAX][33];
    __shared__ double sb[GRAM_KMAX][33];
    const int npairs = ka * kb;
    const int64_t r0 = blockIdx.x * chunk;
    const int64_t r1 = r0 + chunk < n ? r0 + chunk : n;
    double acc[GRAM_KMAX * GRAM_KMAX / 256];
#pragma unroll
    for (int u = 0; u < GRAM_KMAX * GRAM_KMAX / 256; ++u) acc[u] = 0.0;
    for (int64_t t0 = r0; t0 < r1; t0 += 32) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < ka * 32; idx += blockDim.x) {
            const int a = idx / 32, l = idx % 32;
            const int64_t i = t0 + l;
            sa[a][l] = i < r1 ? A[(size_t)a * n + i] : 0.0;
        }
        for (int idx = threadIdx.x; idx < kb * 32; idx += blockDim.x) {
            const int b = idx / 32, l = idx % 32;
            const int64_t i = t0 + l;
            sb[b][l] = i < r1 ? B[(size_t)b * n + i] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < GRAM_KMAX * GRAM_KMAX / 256; ++u) {
            const int pidx = threadIdx.x + u * 256;
            if (pidx < npairs) {
                const int a = pidx / kb, b = pidx % kb;
                double s = 0.0;
#pragma unroll 8
                for (int l = 0; l < 32; ++l) s += sa[a][l] * sb[b][l];
                acc[u] += s;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < GRAM_KMAX * GRAM_KMAX / 256; ++u) {
        const int pidx = threadIdx.x + u * 256;
        if (pidx < npairs) part[(size_t)blockIdx.x * npairs + pidx] = acc[u];
    }
}

int launch_gram(const double* A, int ka, const double* B, int kb, int64_t n, double* part, cudaStream_t s) {
    const int nblk = GRAM_BLOCKS;
    int64_t chunk = (n + nblk - 1) / nblk;
    chunk = (chunk + 31) / 32 * 32;
    gram_kernel<<<nblk, 256, 0, s>>>(A, ka, B, kb, n, chunk, part);
    check_cuda(cudaGetLastError(), "gram launch");
    note_launch();
    return nblk;
}

}  // namespace mm
