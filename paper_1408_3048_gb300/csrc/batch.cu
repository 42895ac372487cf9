// Many right-hand sides through one plan (Monte-Carlo noise realisations sharing the
// pointing, the noise model and the preconditioner):
//
//   batch_toeplitz   Z_r = N^-1 P X_r for R maps at once, FP32.  Because the spectrum of
//                    the even Toeplitz kernel is real, two real inputs packed as one
//                    complex sequence y_a + i y_b convolve independently in the real and
//                    imaginary parts: one complex B-point FFT per RHS pair and tile, no
//                    real-FFT split.  The RHS pair is the fastest grid index, so the
//                    pointing of a tile is read from HBM once and from L2 by the other
//                    pairs.  Same shared-memory Stockham FFT as toeplitz.cuh.
//   batch_scatter    W_r = P^T Z_r, one warp per pixel looping over the RHS (the pixel's
//                    sorted sample indices and weights stay in L1 across RHS).
//   batch_pcg        per-RHS PCG steps (alpha_r, beta_r, own convergence) for all RHS in
//                    one cooperative kernel per iteration, M = M_BD; FP64 dot products.
// Layouts: maps [R][n], time-domain [R][nt], both FP32.
#include "batch.cuh"
#include "pcg.cuh"
#include "toeplitz.cuh"

#include <cooperative_groups.h>

namespace mm {

// ------------------------------------------------------------------ batched Toeplitz
// Gathers points [s0, s0 + count) of the packed complex block (column pair x0 + i x1)
// into a[0 .. count).
template <int NT, int NC>
__device__ __forceinline__ void batch_load(const BatchTzArgs& A, const SpanTile& tile, int64_t ws, const float* x0,
                                           const float* x1, bool has1, float2* a, int s0, int count) {
    const int tid = threadIdx.x;
    const int PER = count / NT;
    constexpr int UNR = 4;
#pragma unroll 1
    for (int base = 0; base < PER; base += UNR) {
        int q[UNR];
        float2 w[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            const int64_t t = ws + s0 + (int64_t)((base + u) * NT + tid);
            const bool ok = base + u < PER && t >= tile.ibeg && t < tile.iend;
            q[u] = ok ? __ldg(A.pixc + t) : -1;
            if constexpr (NC == 3) {
                if (ok) w[u] = A.w[t];
            }
        }
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            float2 c = make_float2(0.f, 0.f);
            if (q[u] >= 0) {
                if constexpr (NC == 1) {
                    c.x = __ldg(x0 + q[u]);
                    c.y = __ldg(x1 + q[u]);
                } else {
                    const int64_t e = 3 * (int64_t)q[u];
                    c.x = __ldg(x0 + e) + w[u].x * __ldg(x0 + e + 1) + w[u].y * __ldg(x0 + e + 2);
                    c.y = __ldg(x1 + e) + w[u].x * __ldg(x1 + e + 1) + w[u].y * __ldg(x1 + e + 2);
                }
                if (!has1) c.y = 0.f;
            }
            if (base + u < PER) a[pad<float>((base + u) * NT + tid)] = c;
        }
    }
}

template <int LOGB, int NT, int NC>
__global__ void __launch_bounds__(NT) batch_toeplitz_kernel(BatchTzArgs A) {
    constexpr int Bn = 1 << LOGB;            // complex points (= real block length)
    if (A.done != nullptr && *(volatile const int*)A.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* a = reinterpret_cast<float2*>(smem_raw);
    const int npairs = (A.R + 1) / 2;
    const int pair = blockIdx.x % npairs;
    const SpanTile tile = A.tiles[blockIdx.x / npairs];
    const int r0 = 2 * pair;
    const bool has1 = r0 + 1 < A.R;
    const float* x0 = A.X + (size_t)r0 * A.n;
    const float* x1 = A.X + (size_t)(has1 ? r0 + 1 : r0) * A.n;
    const int tid = threadIdx.x;
    const int64_t ws = tile.out0 - A.lambda;
    batch_load<NT, NC>(A, tile, ws, x0, x1, has1, a, 0, Bn);
    __syncthreads();
    fft_all<float, LOGB, NT, 0>(a, A.ptw);
    // spectrum product (real, even kernel; H holds k = 0..Bn/2, already divided by Bn),
    // conjugated for the inverse by the forward transform
    const float* H = A.H + (int64_t)tile.psd * (Bn / 2 + 1);
    for (int k = tid; k < Bn; k += NT) {
        const float h = H[k <= Bn / 2 ? k : Bn - k];
        float2 v = a[pad<float>(k)];
        v.x *= h;
        v.y *= -h;
        a[pad<float>(k)] = v;
    }
    __syncthreads();
    fft_all<float, LOGB, NT, 0>(a, A.ptw);
    float* z0 = A.Z + (size_t)r0 * A.nt + tile.out0;
    float* z1 = A.Z + (size_t)(r0 + 1) * A.nt + tile.out0;
    for (int n = tid; n < tile.nout; n += NT) {
        const float2 v = a[pad<float>(n + A.lambda)];
        z0[n] = v.x;
        if (has1) z1[n] = -v.y;
    }
}

// Cluster variant (CL = 2 or 4 CTAs) for blocks above the single-CTA maximum: CTA c holds
// the complex points c M .. c M + M - 1.  Forward: cross-CTA radix-CL step with twiddles
// W_Bn^(n1 c) (distributed shared memory), local M-point FFT -> bins CL k1 + c; pointwise
// product; local FFT; cross-CTA radix-CL recombination written straight to global memory
// (decimation in frequency, then in time, as in the single-RHS cluster kernel).
template <int LOGM, int NT, int NC, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT) batch_toeplitz_cl_kernel(BatchTzArgs A) {
    constexpr int M = 1 << LOGM;
    constexpr int Bn = CL * M;
    constexpr int LOGQ = LOGM + (CL == 2 ? 1 : 2) - 2;   // Bn / 4 = 2^LOGQ
    constexpr int PER = M / NT;
    static_assert(PER >= 1 && M % NT == 0, "points per thread");
    if (A.done != nullptr && *(volatile const int*)A.done) return;   // uniform over the cluster
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* a = reinterpret_cast<float2*>(smem_raw);
    float2* part[CL];
#pragma unroll
    for (int c = 0; c < CL; ++c) part[c] = cl.map_shared_rank(a, c);
    const int npairs = (A.R + 1) / 2;
    const int cid = blockIdx.x / CL;
    const int pair = cid % npairs;
    const SpanTile tile = A.tiles[cid / npairs];
    const int r0 = 2 * pair;
    const bool has1 = r0 + 1 < A.R;
    const float* x0 = A.X + (size_t)r0 * A.n;
    const float* x1 = A.X + (size_t)(has1 ? r0 + 1 : r0) * A.n;
    const int tid = threadIdx.x;
    const int64_t ws = tile.out0 - A.lambda;
    batch_load<NT, NC>(A, tile, ws, x0, x1, has1, a, rank * M, M);
    cl.sync();
    float2 y[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int n1 = u * NT + tid;
        float2 acc = part[0][pad<float>(n1)];
#pragma unroll
        for (int n2 = 1; n2 < CL; ++n2) {
            const float2 v = rot_c<float, CL>(part[n2][pad<float>(n1)], n2 * rank);
            acc.x += v.x;
            acc.y += v.y;
        }
        if (rank != 0) {
            float c, s;
            twiddle<float, LOGQ>(A.twiddle, n1 * rank, c, s);
            acc = cmul<float>(acc, c, s);
        }
        y[u] = acc;
    }
    cl.sync();
#pragma unroll
    for (int u = 0; u < PER; ++u) a[pad<float>(u * NT + tid)] = y[u];
    __syncthreads();
    fft_all<float, LOGM, NT, 0>(a, A.ptw);
    const float* H = A.H + (int64_t)tile.psd * (Bn / 2 + 1);
    for (int k1 = tid; k1 < M; k1 += NT) {
        const int k = CL * k1 + rank;
        const float h = H[k <= Bn / 2 ? k : Bn - k];
        float2 v = a[pad<float>(k1)];
        v.x *= h;
        v.y *= -h;
        a[pad<float>(k1)] = v;
    }
    __syncthreads();
    fft_all<float, LOGM, NT, 0>(a, A.ptw);
    cl.sync();
    float* z0 = A.Z + (size_t)r0 * A.nt + tile.out0;
    float* z1 = A.Z + (size_t)(r0 + 1) * A.nt + tile.out0;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int n1 = u * NT + tid;
        float2 f = part[0][pad<float>(n1)];
#pragma unroll
        for (int m2 = 1; m2 < CL; ++m2) {
            float c, s;
            twiddle<float, LOGQ>(A.twiddle, n1 * m2, c, s);   // W_Bn^(m2 n1)
            const float2 v = rot_c<float, CL>(cmul<float>(part[m2][pad<float>(n1)], c, s), m2 * rank);
            f.x += v.x;
            f.y += v.y;
        }
        const int n = rank * M + n1 - A.lambda;
        if (n >= 0 && n < tile.nout) {
            z0[n] = f.x;
            if (has1) z1[n] = -f.y;
        }
    }
    cl.sync();   // the other CTAs may still read this CTA's shared memory
}

size_t batch_toeplitz_smem(int logb) {
    const int lm = logb > BATCH_MAX_LOGB_CTA ? BATCH_MAX_LOGB_CTA : logb;   // per CTA
    const size_t B = size_t(1) << lm;
    return sizeof(float2) * (B + (B >> PadLog<float>::v));
}

template <int LOGB, int NC>
static void launch_bt(const BatchTzArgs& A, int ntiles, cudaStream_t s) {
    constexpr int NT = tz_threads<float, LOGB>();
    const size_t smem = batch_toeplitz_smem(LOGB);
    auto kern = batch_toeplitz_kernel<LOGB, NT, NC>;
    ensure_smem_attr((const void*)kern, (int)smem, "cudaFuncSetAttribute(batch toeplitz)");
    const int64_t grid = (int64_t)ntiles * ((A.R + 1) / 2);
    kern<<<(unsigned)grid, NT, smem, s>>>(A);
    check_cuda(cudaGetLastError(), "batch toeplitz launch");
    note_launch();
}

template <int LOGM, int NC, int CL>
static void launch_bt_cl(const BatchTzArgs& A, int ntiles, cudaStream_t s) {
    constexpr int NT = tz_threads<float, LOGM>();
    const size_t smem = batch_toeplitz_smem(LOGM);
    auto kern = batch_toeplitz_cl_kernel<LOGM, NT, NC, CL>;
    ensure_smem_attr((const void*)kern, (int)smem, "cudaFuncSetAttribute(batch toeplitz cluster)");
    const int64_t grid = (int64_t)CL * ntiles * ((A.R + 1) / 2);
    kern<<<(unsigned)grid, NT, smem, s>>>(A);
    check_cuda(cudaGetLastError(), "batch toeplitz cluster launch");
    note_launch();
}

void launch_batch_toeplitz(const BatchTzArgs& A, int logb, int ntiles, int ncomp, cudaStream_t s) {
    static_assert(BATCH_MAX_LOGB_CTA == 14, "cluster instantiations below");
    if (logb == 15) {
        if (ncomp == 1) launch_bt_cl<14, 1, 2>(A, ntiles, s);
        else launch_bt_cl<14, 3, 2>(A, ntiles, s);
        return;
    }
    if (logb == 16) {
        if (ncomp == 1) launch_bt_cl<14, 1, 4>(A, ntiles, s);
        else launch_bt_cl<14, 3, 4>(A, ntiles, s);
        return;
    }
#define MM_BT(L)                                                     \
    case L:                                                          \
        if (ncomp == 1) launch_bt<L, 1>(A, ntiles, s);               \
        else launch_bt<L, 3>(A, ntiles, s);                          \
        return;
    switch (logb) {
        MM_BT(9)
        MM_BT(10)
        MM_BT(11)
        MM_BT(12)
        MM_BT(13)
        MM_BT(14)
        default: throw Error{MM_ERR_ARG, "unsupported batched FFT length"};
    }
#undef MM_BT
}

// ------------------------------------------------------------------- batched scatter
template <int NC>
__global__ void batch_scatter_kernel(const int32_t* __restrict__ off, const int32_t* __restrict__ tsort,
                                     const float2* __restrict__ ws, const float* __restrict__ Z, float* __restrict__ W,
                                     int npix, int64_t nt, int64_t n, int R, const int* done) {
    if (done != nullptr && *(volatile const int*)done) return;
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int q = blockIdx.x * warps + (threadIdx.x >> 5); q < npix; q += gridDim.x * warps) {
        const int b = off[q];
        const int e = off[q + 1];
        for (int r = 0; r < R; ++r) {
            const float* z = Z + (size_t)r * nt;
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
            for (int j = b + lane; j < e; j += 32) {
                const float v = z[tsort[j]];
                a0 += v;
                if constexpr (NC == 3) {
                    const float2 ww = ws[j];
                    a1 += ww.x * v;
                    a2 += ww.y * v;
                }
            }
            // exact FP32-pair warp trees (FP64 shuffles per pixel and RHS would make
            // this kernel FP64-bound on GB300)
            float h0 = a0, l0 = 0.f, h1 = a1, l1 = 0.f, h2 = a2, l2 = 0.f;
            warp_pair_reduce(h0, l0);
            if constexpr (NC == 3) {
                warp_pair_reduce(h1, l1);
                warp_pair_reduce(h2, l2);
            }
            if (lane == 0) {
                float* w = W + (size_t)r * n + (int64_t)q * NC;
                w[0] = h0 + l0;
                if constexpr (NC == 3) {
                    w[1] = h1 + l1;
                    w[2] = h2 + l2;
                }
            }
        }
    }
}

void launch_batch_scatter(const Plan& P, const float* Z, float* W, int R, const int* done, cudaStream_t s) {
    if (P.npix_obs == 0) return;
    const int th = 256;
    int g = (P.npix_obs + 7) / 8;
    if (g > P.num_sms * 32) g = P.num_sms * 32;
    if (P.ncomp == 1)
        batch_scatter_kernel<1><<<g, th, 0, s>>>(P.csr_off, P.tsort, nullptr, Z, W, P.npix_obs, P.nt, P.n, R, done);
    else
        batch_scatter_kernel<3><<<g, th, 0, s>>>(P.csr_off, P.tsort, P.wsort32, Z, W, P.npix_obs, P.nt, P.n, R,
                                                  done);
    check_cuda(cudaGetLastError(), "batch scatter launch");
    note_launch();
}

// --------------------------------------------------------------------- batched PCG

// Totals over blocks of slot j for j < count (slots hold FP32 pairs), one warp per slot,
// lanes over blocks in a fixed order; result (FP64) in sh[j].
__device__ void batch_totals(const double* part, int stride, int slot0, int count, double* sh) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = w; j < count; j += nw) {
        float hi = 0.f, lo = 0.f;
        for (unsigned b = l; b < gridDim.x; b += 32) {
            const float2 p = __ldcg(reinterpret_cast<const float2*>(part + (size_t)b * stride + slot0 + j));
            pair_add(hi, lo, p.x, p.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            pair_add(hi, lo, h2, l2);
        }
        if (l == 0) sh[j] = (double)hi + (double)lo;
    }
    __syncthreads();
}

// Block partial of sum_i a_r[i] b_r[i] for every RHS r, i over this block's elements:
// exact products accumulated as FP32 pairs, stored as a pair in the slot.  Warp w owns
// the RHS w, w + nw, ...; each lane issues a group of 8 loads before accumulating them in
// element order (the same order as one at a time).
__device__ void batch_dots(const float* A_, const float* B_, int64_t n, int64_t e0, int64_t e1, int R,
                           double* part_row, const unsigned char* active) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int r = w; r < R; r += nw) {
        DotAcc<float> acc;
        if (active[r]) {
            const float* a = A_ + (size_t)r * n;
            const float* b = B_ + (size_t)r * n;
            for (int64_t base = e0 + l; base < e1; base += 32 * 8) {
                float va[8], vb[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int64_t i = base + 32 * t;
                    va[t] = i < e1 ? a[i] : 0.f;
                    vb[t] = i < e1 ? b[i] : 0.f;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (base + 32 * t < e1) acc.add(va[t], vb[t]);
            }
        }
        float hi = acc.hi, lo = acc.lo;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            pair_add(hi, lo, h2, l2);
        }
        if (l == 0) *reinterpret_cast<float2*>(part_row + r) = make_float2(hi, lo);
    }
}

// z_r = M_BD r_r for every running RHS on this block's pixels; (RHS, pixel) pairs are
// spread over the threads so that all loads of a block are in flight together.
template <int NC>
__device__ void batch_bd_all(const BatchPcgArgs& a, int p0, int p1, int R, const unsigned char* active) {
    const int np = p1 - p0;
    for (int idx = threadIdx.x; idx < R * np; idx += blockDim.x) {
        const int r = idx / np;
        if (!active[r]) continue;
        const int q = p0 + (idx - r * np);
        const float* rv = a.r + (size_t)r * a.n;
        float* zv = a.z + (size_t)r * a.n;
        if constexpr (NC == 1) {
            zv[q] = a.bd[q] * rv[q];
        } else {
            const float* m = a.bd + 6 * (int64_t)q;
            const int64_t e = 3 * (int64_t)q;
            const float r0 = rv[e], r1 = rv[e + 1], r2 = rv[e + 2];
            zv[e] = m[0] * r0 + m[1] * r1 + m[2] * r2;
            zv[e + 1] = m[1] * r0 + m[3] * r1 + m[4] * r2;
            zv[e + 2] = m[2] * r0 + m[4] * r1 + m[5] * r2;
        }
    }
}

__device__ __forceinline__ void block_range(int npix, int& lo, int& hi) {
    const int chunk = (npix + gridDim.x - 1) / gridDim.x;
    lo = blockIdx.x * chunk;
    hi = min(npix, lo + chunk);
    if (lo > hi) lo = hi;
}

// which = 0: init (x = 0, z = M r, p = z, rho, bb); 1: one iteration after q = A p.
template <int NC>
__global__ void __launch_bounds__(BATCH_THREADS) batch_pcg_kernel(BatchPcgArgs a, int which) {
    __shared__ double sh[BATCH_RMAX];
    __shared__ double sh2[BATCH_RMAX];
    __shared__ unsigned char act[BATCH_RMAX];
    __shared__ float coef[BATCH_RMAX];
    if (*(volatile int*)&a.flags[F_DONE]) return;
    int p0, p1;
    block_range(a.npix, p0, p1);
    const int64_t e0 = (int64_t)p0 * NC, e1 = (int64_t)p1 * NC;
    const int R = a.R;
    double* prow = a.partial + (size_t)blockIdx.x * BATCH_PSTRIDE;
    for (int r = threadIdx.x; r < R; r += blockDim.x) act[r] = a.state[r] == 0;
    __syncthreads();
    if (which == 0) {
        // (every RHS is running here: the host resets the states before this launch)
        const int len = (int)(e1 - e0);   // one block's elements: far below 2^31 / R
        for (int idx = threadIdx.x; idx < R * len; idx += blockDim.x) {
            const int r = idx / len;
            a.x[(size_t)r * a.n + e0 + (idx - r * len)] = 0.f;
        }
        batch_bd_all<NC>(a, p0, p1, R, act);
        __syncthreads();
        for (int idx = threadIdx.x; idx < R * len; idx += blockDim.x) {
            const int r = idx / len;
            const size_t o = (size_t)r * a.n + e0 + (idx - r * len);
            a.p[o] = a.z[o];
        }
        batch_dots(a.r, a.r, a.n, e0, e1, R, prow, act);
        batch_dots(a.r, a.z, a.n, e0, e1, R, prow + BATCH_RMAX, act);
        if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
        batch_totals(a.partial, BATCH_PSTRIDE, 0, R, sh);
        batch_totals(a.partial, BATCH_PSTRIDE, BATCH_RMAX, R, sh2);
        if (blockIdx.x == 0) {
            for (int r = threadIdx.x; r < R; r += blockDim.x) {
                a.bb[r] = sh[r];
                a.rr[r] = sh[r];
                a.rho[r] = sh2[r];
                a.iters[r] = 0;
                a.state[r] = (sh[r] > 0.0) ? 0 : 1;   // zero right-hand side: done at x = 0
            }
            if (threadIdx.x == 0) a.flags[F_ITER] = 0;
        }
        return;
    }
    // phase A: alpha_r = rho_r / p_r^T q_r
    batch_dots(a.p, a.q, a.n, e0, e1, R, prow, act);
    if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
    batch_totals(a.partial, BATCH_PSTRIDE, 0, R, sh);
    // phase B: x += alpha p, r -= alpha q (active RHS only; (RHS, element) pairs spread
    // over the threads); r^T r
    for (int r = threadIdx.x; r < R; r += blockDim.x) coef[r] = act[r] ? (float)(a.rho[r] / sh[r]) : 0.f;
    __syncthreads();
    {
        const int len = (int)(e1 - e0);
        for (int idx = threadIdx.x; idx < R * len; idx += blockDim.x) {
            const int r = idx / len;
            if (!act[r]) continue;
            const size_t o = (size_t)r * a.n + e0 + (idx - r * len);
            const float al = coef[r];
            a.x[o] += al * a.p[o];
            a.r[o] -= al * a.q[o];
        }
    }
    __syncthreads();
    batch_dots(a.r, a.r, a.n, e0, e1, R, prow + BATCH_RMAX, act);
    if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
    batch_totals(a.partial, BATCH_PSTRIDE, BATCH_RMAX, R, sh2);
    const int it = a.flags[F_ITER] + 1;
    // convergence per RHS (every block decides the same)
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        if (!act[r]) continue;
        const double pq = sh[r], rr = sh2[r];
        unsigned char st = 0;
        if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rr)) st = 3;            // breakdown
        else if (rr <= a.tol2[r] * a.bb[r]) st = 1;                            // converged
        else if (it >= a.maxit) st = 2;                                         // maxit
        if (st != 0) act[r] = 0;
        if (blockIdx.x == 0) {
            if (st != 0) {
                a.state[r] = st;
                a.iters[r] = it;
                a.rr[r] = rr;
            }
        }
    }
    __syncthreads();
    // phase C: z = M_BD r, r^T z for the RHS still running
    batch_bd_all<NC>(a, p0, p1, R, act);
    __syncthreads();
    batch_dots(a.r, a.z, a.n, e0, e1, R, prow + 2 * BATCH_RMAX, act);
    if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
    batch_totals(a.partial, BATCH_PSTRIDE, 2 * BATCH_RMAX, R, sh);
    bool any = false;
    for (int r = 0; r < R; ++r) any = any || act[r];
    for (int r = threadIdx.x; r < R; r += blockDim.x) coef[r] = act[r] ? (float)(sh[r] / a.rho[r]) : 0.f;
    __syncthreads();
    {
        const int len = (int)(e1 - e0);
        for (int idx = threadIdx.x; idx < R * len; idx += blockDim.x) {
            const int r = idx / len;
            if (!act[r]) continue;
            const size_t o = (size_t)r * a.n + e0 + (idx - r * len);
            a.p[o] = a.z[o] + coef[r] * a.p[o];
        }
    }
    // every block has read rho and F_ITER above; block 0 publishes the new values after a
    // final barrier so no block can see them early
    if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
    if (blockIdx.x == 0) {
        for (int r = threadIdx.x; r < R; r += blockDim.x) {
            if (act[r]) {
                a.rho[r] = sh[r];
                a.rr[r] = sh2[r];
                a.iters[r] = it;
            }
        }
        if (threadIdx.x == 0) {
            a.flags[F_ITER] = it;
            if (!any) a.flags[F_DONE] = 1;
        }
    }
}

void launch_batch_pcg(int which, int ncomp, const BatchPcgArgs& a, int nblocks, cudaStream_t s) {
    void* args[] = {(void*)&a, (void*)&which};
    const void* k = ncomp == 1 ? (const void*)batch_pcg_kernel<1> : (const void*)batch_pcg_kernel<3>;
    check_cuda(cudaLaunchCooperativeKernel(k, dim3(nblocks), dim3(BATCH_THREADS), args, 0, s),
               "cooperative batch PCG launch");
    note_launch();
}

int batch_pcg_max_blocks(int num_sms) {
    int per_sm = 0;
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_pcg_kernel<3>, BATCH_THREADS, 0),
               "occupancy");
    if (per_sm < 1) throw Error{MM_ERR_CUDA, "batch PCG kernel does not fit on an SM"};
    return num_sms;
}

}  // namespace mm

namespace mm {

__global__ void scale_f32_kernel(const double* __restrict__ a, double s, float* __restrict__ out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)(a[i] * s);
}

void launch_scale_f32(const double* a, double s, float* out, int64_t n, cudaStream_t st) {
    int64_t g = (n + 255) / 256;
    if (g > 2048) g = 2048;
    scale_f32_kernel<<<(int)g, 256, 0, st>>>(a, s, out, n);
    check_cuda(cudaGetLastError(), "scale_f32 launch");
    note_launch();
}

__global__ void axpy_host_kernel(double* __restrict__ x, const float* __restrict__ d, double s, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += s * (double)d[i];
}

void launch_axpy_host(double* x, const float* d, double s, int64_t n, cudaStream_t st) {
    int64_t g = (n + 255) / 256;
    if (g > 2048) g = 2048;
    axpy_host_kernel<<<(int)g, 256, 0, st>>>(x, d, s, n);
    check_cuda(cudaGetLastError(), "axpy launch");
    note_launch();
}

}  // namespace mm
