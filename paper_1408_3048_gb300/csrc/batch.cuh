// Batched (many right-hand sides) kernels and their arguments (see batch.cu).
#pragma once

#include <cuda_fp16.h>

#include "mm_internal.h"

namespace mm {

constexpr int BATCH_RMAX = 64;                 // right-hand sides per batched launch
constexpr int BATCH_THREADS = 512;
constexpr int BATCH_PSTRIDE = 3 * BATCH_RMAX;  // per-block partial slots
constexpr int BATCH_MAX_LOGB_CTA = 14;         // largest complex block in one CTA
constexpr int BATCH_MAX_LOGB = 16;             // 2- and 4-CTA clusters above it

struct BatchTzArgs {
    const SpanTile* tiles;
    const float* H;            // [npsd][B/2 + 1], divided by B
    const float2* ptw;         // per-pass FFT twiddles of the per-CTA transform
    const float* twiddle;      // cos(2 pi k / B), k = 0..B/4 (cluster variants)
    const float* X;            // [R][n]
    const int32_t* pixc;
    const float2* w;
    float* Z;                  // [R][nt]
    const int* done;
    int64_t n;
    int64_t nt;
    int R;
    int lambda;
};

struct BatchPcgArgs {
    int64_t n;
    int npix;
    int R;
    int maxit;
    float* x;
    float* r;
    float* p;
    const float* q;
    float* z;
    const float* bd;
    double* partial;           // [grid][BATCH_PSTRIDE]
    double* rho;               // [R]
    double* bb;
    double* rr;
    const double* tol2;        // [R] squared relative tolerance
    int* iters;                // [R]
    unsigned char* state;      // [R] 0 running, 1 converged, 2 maxit, 3 breakdown
    int* flags;
    unsigned* bar;
    unsigned bar_absent;           // 0 (see grid_sync)
    unsigned long long wait_ns;    // limit of each barrier wait
};

// Tensor-core form (batch_tc.cu): banded product as FP16 split-operand MMAs, four
// 128-row tiles of one interval and up to 64 columns per CTA (groups: out0 = first
// output, [ibeg, iend) = its interval, nout <= 512 outputs).
struct BatchTcArgs {
    const SpanTile* groups;
    const __half* atab;        // [npsd][nchunk][hi, lo][128 x 64] band chunks, canonical layout
    const float* inv_cscale;   // [npsd] 1 / (power-of-two scale of the band row)
    const float* Y;            // [R][nt] P X
    float* Z;                  // [R][nt] N^-1 P X
    const float* scale;        // [R] power-of-two column scales and their inverses
    const float* inv_scale;
    const int* done;
    int* flags;                // F_STATUS / F_DONE on a wait that runs out
    int64_t nt;
    int R;
    int RB;                    // columns per tile: R rounded up to 16
    int lambda;
    int nchunk;                // K chunks of 64: (128 + 2 lambda) / 64 rounded up
};
size_t batch_tc_smem();
void launch_batch_tc(const BatchTcArgs& A, int ngroups, cudaStream_t s);
void launch_batch_gather(const Plan& P, const float* X, int R, float* Y, cudaStream_t s);
void launch_batch_colscale(const float* X, int64_t n, int R, float* scale, float* inv_scale, cudaStream_t s);

size_t batch_toeplitz_smem(int logb);
void launch_batch_toeplitz(const BatchTzArgs& A, int logb, int ntiles, int ncomp, cudaStream_t s);
void launch_batch_scatter(const Plan& P, const float* Z, float* W, int R, const int* done, cudaStream_t s);
void launch_batch_pcg(int which, int ncomp, const BatchPcgArgs& a, int nblocks, cudaStream_t s);
int batch_pcg_max_blocks(int num_sms);

}  // namespace mm

namespace mm {
void launch_scale_f32(const double* a, double s, float* out, int64_t n, cudaStream_t st);
void launch_axpy_host(double* x, const float* d, double s, int64_t n, cudaStream_t st);
}  // namespace mm
