// Pointing operators and the block-Jacobi preconditioner.
//
//   gather   y = P x        (Eq. 2: y_t = x_I + cos 2phi_t x_Q + sin 2phi_t x_U)
//   scatter  w = P^T z      segmented, warp-reduced sum over the pixel-sorted samples of
//                           each observed pixel (CSR built at plan time); no atomics, so
//                           the result is bit-reproducible
//   M_BD     Eq. 10: B_p = sum_{t in p} t^(i(t))_0 w_t w_t^T, stored inverted
//                           (symmetric, packed a00 a01 a02 a11 a12 a22)
#include <algorithm>

#include "mm_internal.h"
#include "pcg.cuh"

namespace mm {

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

// ----------------------------------------------------------------------------- gather
template <typename T, int NC>
__global__ void gather_kernel(const int32_t* __restrict__ pixc,
                              const typename V2<T>::type* __restrict__ w,
                              const T* __restrict__ x, T* __restrict__ y, int64_t nt) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int q = pixc[t];
        T v = (T)0;
        if (q >= 0) {
            if constexpr (NC == 1) {
                v = __ldg(x + q);
            } else {
                const typename V2<T>::type ww = w[t];
                const T* xq = x + 3 * (int64_t)q;
                v = __ldg(xq) + ww.x * __ldg(xq + 1) + ww.y * __ldg(xq + 2);
            }
        }
        y[t] = v;
    }
}

template <typename T>
static const typename V2<T>::type* weights_time(const Plan& P);
template <>
const double2* weights_time<double>(const Plan& P) { return P.w64; }
template <>
const float2* weights_time<float>(const Plan& P) { return P.w32; }

template <typename T>
static const typename V2<T>::type* weights_sorted(const Plan& P);
template <>
const double2* weights_sorted<double>(const Plan& P) { return P.wsort64; }
template <>
const float2* weights_sorted<float>(const Plan& P) { return P.wsort32; }

static int grid_for(int64_t n, int threads, int num_sms) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms * 16;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

template <typename T>
void launch_gather(const Plan& P, const T* x, T* y, cudaStream_t s) {
    const int th = 256;
    const int g = grid_for(P.nt, th, P.num_sms);
    if (P.ncomp == 1)
        gather_kernel<T, 1><<<g, th, 0, s>>>(P.pixc, nullptr, x, y, P.nt);
    else
        gather_kernel<T, 3><<<g, th, 0, s>>>(P.pixc, weights_time<T>(P), x, y, P.nt);
    check_cuda(cudaGetLastError(), "gather launch");
    note_launch();
}
template void launch_gather<double>(const Plan&, const double*, double*, cudaStream_t);
template void launch_gather<float>(const Plan&, const float*, float*, cudaStream_t);

// ---------------------------------------------------------------------------- scatter
// LPP lanes per observed pixel (the pixel tile: 32, 16 or 8, so a warp holds 1, 2 or 4
// pixels; plan.scatter_lpp, chosen by timing in an autotuned plan).  The lanes of a pixel
// stride over its sorted samples and keep per-lane partial sums in T.  The tree over the
// LPP lanes (xor shuffles, fixed order) runs in double for T = double and on exact FP32
// (hi, lo) pairs for T = float -- GB300 issues a warp's FP64 instruction at 1/64 of the
// FP32 rate, and a double tree per pixel would cost more SM time than the pixel's memory
// traffic.  The sample loop issues SCATTER_U (index, weight) loads per lane before their
// dependent TOD loads, so each lane keeps several random TOD reads in flight; every lane
// still adds its samples j, j + LPP, j + 2 LPP, ... in ascending order (the result does
// not depend on the unrolling, only on LPP).
constexpr int SCATTER_U = 8;
constexpr int SCATTER_THREADS = 256;

// Optional fused dot product with the output (DOT): *pq = sum_q p_q . w_q.
struct ScatterDot {
    const void* p;      // T[n]
    double* part;       // [gridDim.x]
    unsigned* count;
    double* pq;
};

// Sum over the LPP lanes of a pixel group (every lane gets it); call with all 32 lanes.
template <typename T, int LPP>
__device__ __forceinline__ T group_total(T v) {
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int o = LPP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    } else {
        float hi = v, lo = 0.f;
#pragma unroll
        for (int o = LPP / 2; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            pair_add(hi, lo, h2, l2);
        }
        return hi + lo;
    }
}

// Weight pair of sorted sample j: read, or (ANG, FP32) formed from the stored angle a_j
// (cos pi a_j, sin pi a_j) -- 4 bytes per sample instead of 8 for unit-norm weights -- by
// the hardware's fast sine and cosine (absolute error below 4e-7 on [-pi, pi]; a_j lies in
// [-1, 1]).  (A table-driven form, a 513-entry table plus the angle-addition formula, was
// no faster than sincospif; this one is.)
template <typename T, bool ANG>
__device__ __forceinline__ typename V2<T>::type sorted_weight(const typename V2<T>::type* ws, const float* ang,
                                                              int64_t j) {
    if constexpr (ANG) {
        float sv, cv;
        __sincosf(3.14159265358979f * __ldg(ang + j), &sv, &cv);
        return make_float2(cv, sv);
    } else {
        return __ldg(ws + j);
    }
}

template <typename T, int NC, bool DOT, int LPP, bool ANG = false>
__global__ void __launch_bounds__(SCATTER_THREADS) scatter_kernel(const int32_t* __restrict__ off,
                                                                  const int32_t* __restrict__ tsort,
                                                                  const typename V2<T>::type* __restrict__ ws,
                                                                  const float* __restrict__ ang,
                                                                  const T* __restrict__ z, T* __restrict__ w,
                                                                  int npix, const int* done, ScatterDot sd) {
    using W2 = typename V2<T>::type;
    constexpr int PPW = 32 / LPP;                 // pixels per warp
    griddep_wait();   // launched as a dependent launch: the previous kernel's outputs
    if (done != nullptr && *(volatile const int*)done) return;
    const int lane = threadIdx.x & 31;
    const int sl = lane % LPP, seg = lane / LPP;
    const int warps = blockDim.x >> 5;
    DotAcc<T> dacc;   // DOT: this lane group's pixels, ascending (lane sl == 0)
    const int stride = gridDim.x * warps * PPW;
    for (int qb = (blockIdx.x * warps + (threadIdx.x >> 5)) * PPW; qb < npix; qb += stride) {
        const int q = qb + seg;
        const bool valid = q < npix;
        const int b = valid ? off[q] : 0;
        const int e = valid ? off[q + 1] : 0;
        T a0 = 0, a1 = 0, a2 = 0;
        int j = b + sl;
        for (; j + LPP * (SCATTER_U - 1) < e; j += LPP * SCATTER_U) {
            int t[SCATTER_U];
            W2 ww[SCATTER_U];
            T v[SCATTER_U];
#pragma unroll
            for (int u = 0; u < SCATTER_U; ++u) t[u] = __ldg(tsort + j + LPP * u);
            if constexpr (NC == 3) {
#pragma unroll
                for (int u = 0; u < SCATTER_U; ++u) ww[u] = sorted_weight<T, ANG>(ws, ang, j + LPP * u);
            }
#pragma unroll
            for (int u = 0; u < SCATTER_U; ++u) v[u] = z[t[u]];
#pragma unroll
            for (int u = 0; u < SCATTER_U; ++u) {
                a0 += v[u];
                if constexpr (NC == 3) {
                    a1 += ww[u].x * v[u];
                    a2 += ww[u].y * v[u];
                }
            }
        }
        for (; j < e; j += LPP) {
            const T v = z[__ldg(tsort + j)];
            a0 += v;
            if constexpr (NC == 3) {
                const W2 ww = sorted_weight<T, ANG>(ws, ang, j);
                a1 += ww.x * v;
                a2 += ww.y * v;
            }
        }
        const T s0 = group_total<T, LPP>(a0);
        T s1 = 0, s2 = 0;
        if constexpr (NC == 3) {
            s1 = group_total<T, LPP>(a1);
            s2 = group_total<T, LPP>(a2);
        }
        if (sl == 0 && valid) {
            if constexpr (NC == 1) {
                w[q] = s0;
                if constexpr (DOT) dacc.add(static_cast<const T*>(sd.p)[q], s0);
            } else {
                w[3 * (int64_t)q] = s0;
                w[3 * (int64_t)q + 1] = s1;
                w[3 * (int64_t)q + 2] = s2;
                if constexpr (DOT) {
                    const T* pp = static_cast<const T*>(sd.p) + 3 * (int64_t)q;
                    dacc.add(pp[0], s0);
                    dacc.add(pp[1], s1);
                    dacc.add(pp[2], s2);
                }
            }
        }
    }
    if constexpr (DOT) {
        __shared__ DotAcc<T> wacc[SCATTER_THREADS];
        __shared__ double wsum[SCATTER_THREADS / 32];
        __shared__ bool last;
        if (sl == 0) wacc[(threadIdx.x >> 5) * PPW + seg] = dacc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = 0.0;
            for (int i = 0; i < warps * PPW; ++i) b += wacc[i].total();
            sd.part[blockIdx.x] = b;
            __threadfence();
            last = atomicAdd(sd.count, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (last) {
            // fixed partition of the block partials over the warps, then warps in order
            __threadfence();
            const int per = (gridDim.x + warps - 1) / warps;
            const int w0 = (threadIdx.x >> 5) * per;
            const int w1 = min((int)gridDim.x, w0 + per);
            double t = 0.0;
            for (int i = w0 + lane; i < w1; i += 32) t += __ldcg(sd.part + i);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) wsum[threadIdx.x >> 5] = t;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int i = 0; i < warps; ++i) tot += wsum[i];
                *sd.pq = tot;
                *sd.count = 0;
            }
        }
    }
}

// Grid: LPP lanes per pixel up to 8 resident blocks of 256 threads per SM (full
// occupancy), lane groups loop over pixels beyond that.
int scatter_blocks(const Plan& P) {
    const int ppb = (SCATTER_THREADS / 32) * (32 / P.scatter_lpp);
    int g = (int)(((int64_t)P.npix_obs + ppb - 1) / ppb);
    return std::max(1, std::min(g, P.num_sms * 8));
}

template <typename T, bool DOT, int LPP>
static void scatter_launch_lpp(const Plan& P, const T* z, T* w, const int* done, ScatterDot sd, cudaStream_t s) {
    const int g = scatter_blocks(P);
    using W2 = typename V2<T>::type;
    const int32_t* off = P.csr_off;
    const int32_t* ts = P.tsort;
    const W2* nw = nullptr;
    const float* na = nullptr;
    if (P.ncomp == 1) {
        launch_pdl(scatter_kernel<T, 1, DOT, LPP>, g, SCATTER_THREADS, 0, s, off, ts, nw, na, z, w, P.npix_obs, done,
                   sd);
        return;
    }
    if constexpr (sizeof(T) == 4) {
        if (P.asort32 != nullptr) {
            const float* ang = P.asort32;
            launch_pdl(scatter_kernel<T, 3, DOT, LPP, true>, g, SCATTER_THREADS, 0, s, off, ts, nw, ang, z, w,
                       P.npix_obs, done, sd);
            return;
        }
    }
    const W2* ws = weights_sorted<T>(P);
    launch_pdl(scatter_kernel<T, 3, DOT, LPP>, g, SCATTER_THREADS, 0, s, off, ts, ws, na, z, w, P.npix_obs, done, sd);
}

template <typename T, bool DOT>
static void scatter_launch(const Plan& P, const T* z, T* w, const int* done, ScatterDot sd, cudaStream_t s) {
    switch (P.scatter_lpp) {
        case 8: scatter_launch_lpp<T, DOT, 8>(P, z, w, done, sd, s); break;
        case 16: scatter_launch_lpp<T, DOT, 16>(P, z, w, done, sd, s); break;
        default: scatter_launch_lpp<T, DOT, 32>(P, z, w, done, sd, s); break;
    }
    check_cuda(cudaGetLastError(), "scatter launch");
    note_launch();
}

template <typename T>
void launch_scatter(const Plan& P, const T* z, T* w, const int* done, cudaStream_t s) {
    if (P.npix_obs == 0) return;
    scatter_launch<T, false>(P, z, w, done, ScatterDot{nullptr, nullptr, nullptr, nullptr}, s);
}
template void launch_scatter<double>(const Plan&, const double*, double*, const int*, cudaStream_t);
template void launch_scatter<float>(const Plan&, const float*, float*, const int*, cudaStream_t);

template <typename T>
void launch_scatter_dot(const Plan& P, const T* z, T* w, const T* p, double* part, unsigned* count, double* pq,
                        const int* done, cudaStream_t s) {
    if (P.npix_obs == 0) throw Error{MM_ERR_ARG, "no observed pixels"};
    scatter_launch<T, true>(P, z, w, done, ScatterDot{p, part, count, pq}, s);
}
template void launch_scatter_dot<double>(const Plan&, const double*, double*, const double*, double*, unsigned*,
                                         double*, const int*, cudaStream_t);
template void launch_scatter_dot<float>(const Plan&, const float*, float*, const float*, double*, unsigned*,
                                        double*, const int*, cudaStream_t);

// ------------------------------------------------------------------------ M_BD build
__device__ __forceinline__ int interval_of(const int64_t* ioff, int K, int64_t t) {
    int lo = 0, hi = K;   // ioff[lo] <= t < ioff[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ioff[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

template <int NC>
__global__ void bd_build_kernel(const int32_t* __restrict__ off, const int32_t* __restrict__ tsort,
                                const double2* __restrict__ ws, const int64_t* __restrict__ ioff,
                                const int32_t* __restrict__ ipsd, const double* __restrict__ t0,
                                int K, int npix, double* __restrict__ bd64, float* __restrict__ bd32) {
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int q = blockIdx.x * warps + (threadIdx.x >> 5); q < npix; q += gridDim.x * warps) {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int j = off[q] + lane; j < off[q + 1]; j += 32) {
            const int t = tsort[j];
            const double d = t0[ipsd[interval_of(ioff, K, t)]];
            s[0] += d;
            if constexpr (NC == 3) {
                const double2 w = ws[j];
                s[1] += d * w.x;
                s[2] += d * w.y;
                s[3] += d * w.x * w.x;
                s[4] += d * w.x * w.y;
                s[5] += d * w.y * w.y;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < (NC == 3 ? 6 : 1); ++c) s[c] += __shfl_xor_sync(0xffffffffu, s[c], o);
        if (lane == 0) {
            if constexpr (NC == 1) {
                const double inv = 1.0 / s[0];
                bd64[q] = inv;
                bd32[q] = (float)inv;
            } else {
                // B = [[s0 s1 s2][s1 s3 s4][s2 s4 s5]]; inverse by cofactors (B is SPD and
                // well conditioned for every observed pixel)
                const double a = s[0], b = s[1], c = s[2], d = s[3], e = s[4], f = s[5];
                const double c00 = d * f - e * e;
                const double c01 = c * e - b * f;
                const double c02 = b * e - c * d;
                const double c11 = a * f - c * c;
                const double c12 = b * c - a * e;
                const double c22 = a * d - b * b;
                const double det = a * c00 + b * c01 + c * c02;
                const double id = 1.0 / det;
                const double v[6] = {c00 * id, c01 * id, c02 * id, c11 * id, c12 * id, c22 * id};
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    bd64[6 * (int64_t)q + i] = v[i];
                    bd32[6 * (int64_t)q + i] = (float)v[i];
                }
            }
        }
    }
}

void launch_bd_build(const Plan& P, double* bd64, float* bd32, cudaStream_t s) {
    if (P.npix_obs == 0) return;
    const int th = 256;
    int g = (P.npix_obs + 7) / 8;
    if (g > P.num_sms * 32) g = P.num_sms * 32;
    if (P.ncomp == 1)
        bd_build_kernel<1><<<g, th, 0, s>>>(P.csr_off, P.tsort, nullptr, P.ioff, P.ipsd, P.t0, P.K,
                                             P.npix_obs, bd64, bd32);
    else
        bd_build_kernel<3><<<g, th, 0, s>>>(P.csr_off, P.tsort, P.wsort64, P.ioff, P.ipsd, P.t0, P.K,
                                             P.npix_obs, bd64, bd32);
    check_cuda(cudaGetLastError(), "bd build launch");
    note_launch();
}

// --------------------------------------------------- a priori coarse space (Sec. 3.3.1)
// Z[g][p * NC] = (kept samples of pixel p in intervals of group g) / (all kept samples of
// p), interval i in group (i r) / K; Q/U rows stay 0 (Z is zeroed by the caller).  One
// warp per pixel; lanes count into per-warp shared counters (integer, order-free).
constexpr int APRIORI_THREADS = 256;
constexpr int APRIORI_RMAX = 64;

template <int NC>
__global__ void __launch_bounds__(APRIORI_THREADS) apriori_kernel(const int32_t* __restrict__ off,
                                                                  const int32_t* __restrict__ tsort,
                                                                  const int64_t* __restrict__ ioff, int K, int r,
                                                                  int npix, int64_t n, double* __restrict__ Z) {
    __shared__ int cnt[APRIORI_THREADS / 32][APRIORI_RMAX];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    for (int q = blockIdx.x * warps + wib; q < npix; q += gridDim.x * warps) {
        for (int g = lane; g < r; g += 32) cnt[wib][g] = 0;
        __syncwarp();
        const int b = off[q], e = off[q + 1];
        for (int j = b + lane; j < e; j += 32) {
            const int i = interval_of(ioff, K, tsort[j]);
            atomicAdd(&cnt[wib][(int)(((int64_t)i * r) / K)], 1);
        }
        __syncwarp();
        const double hits = (double)(e - b);
        for (int g = lane; g < r; g += 32) Z[(size_t)g * n + (int64_t)q * NC] = (double)cnt[wib][g] / hits;
        __syncwarp();
    }
}

void launch_apriori(const Plan& P, int r, double* Z, cudaStream_t s) {
    if (r < 1 || r > APRIORI_RMAX) throw Error{MM_ERR_ARG, "r must be in [1, 64]"};
    check_cuda(cudaMemsetAsync(Z, 0, (size_t)r * P.n * 8, s), "memset Z");
    if (P.npix_obs == 0) return;
    const int g = std::max(1, std::min((P.npix_obs + 7) / 8, P.num_sms * 8));
    if (P.ncomp == 1)
        apriori_kernel<1><<<g, APRIORI_THREADS, 0, s>>>(P.csr_off, P.tsort, P.ioff, P.K, r, P.npix_obs, P.n, Z);
    else
        apriori_kernel<3><<<g, APRIORI_THREADS, 0, s>>>(P.csr_off, P.tsort, P.ioff, P.K, r, P.npix_obs, P.n, Z);
    check_cuda(cudaGetLastError(), "a priori coarse launch");
    note_launch();
}

// ------------------------------------------------------------------------ M_BD apply
template <typename T, int NC>
__global__ void bd_apply_kernel(const T* __restrict__ bd, const T* __restrict__ r, T* __restrict__ z,
                                int npix) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npix; q += gridDim.x * blockDim.x) {
        if constexpr (NC == 1) {
            z[q] = bd[q] * r[q];
        } else {
            const T* m = bd + 6 * (int64_t)q;
            const T r0 = r[3 * (int64_t)q], r1 = r[3 * (int64_t)q + 1], r2 = r[3 * (int64_t)q + 2];
            z[3 * (int64_t)q] = m[0] * r0 + m[1] * r1 + m[2] * r2;
            z[3 * (int64_t)q + 1] = m[1] * r0 + m[3] * r1 + m[4] * r2;
            z[3 * (int64_t)q + 2] = m[2] * r0 + m[4] * r1 + m[5] * r2;
        }
    }
}

template <typename T>
static const T* bd_of(const Plan& P);
template <>
const double* bd_of<double>(const Plan& P) { return P.bd64; }
template <>
const float* bd_of<float>(const Plan& P) { return P.bd32; }

template <typename T>
void launch_bd_apply(const Plan& P, const T* r, T* z, cudaStream_t s) {
    if (P.npix_obs == 0) return;
    const int th = 256;
    const int g = grid_for(P.npix_obs, th, P.num_sms);
    if (P.ncomp == 1)
        bd_apply_kernel<T, 1><<<g, th, 0, s>>>(bd_of<T>(P), r, z, P.npix_obs);
    else
        bd_apply_kernel<T, 3><<<g, th, 0, s>>>(bd_of<T>(P), r, z, P.npix_obs);
    check_cuda(cudaGetLastError(), "bd apply launch");
    note_launch();
}
template void launch_bd_apply<double>(const Plan&, const double*, double*, cudaStream_t);
template void launch_bd_apply<float>(const Plan&, const float*, float*, cudaStream_t);

// -------------------------------------------------------------------------- helpers
__global__ void convert_kernel(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

void launch_convert_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    convert_kernel<<<grid_for(n, 256, 160), 256, 0, s>>>(a, b, n);
    check_cuda(cudaGetLastError(), "convert launch");
    note_launch();
}

// ang[j] = atan2(w2, w1) / pi rounded to FP32 for the sorted weight pairs; *bad counts the
// pairs whose squared norm is more than 1e-12 from 1 (the angle form is then not used)
__global__ void angle_kernel(const double2* __restrict__ w, float* __restrict__ ang, int64_t n, unsigned* bad) {
    unsigned nb = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = w[i];
        ang[i] = (float)(atan2(v.y, v.x) * 0.31830988618379067154);   // 1 / pi
        nb += fabs(v.x * v.x + v.y * v.y - 1.0) > 1e-12;
    }
    if (nb) atomicAdd(bad, nb);
}

void launch_angles(const double2* w, float* ang, int64_t n, unsigned* bad, cudaStream_t s) {
    if (n == 0) return;
    angle_kernel<<<grid_for(n, 256, 160), 256, 0, s>>>(w, ang, n, bad);
    check_cuda(cudaGetLastError(), "angle launch");
    note_launch();
}

__global__ void widen_kernel(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

void launch_convert_f32_to_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
    if (n == 0) return;
    widen_kernel<<<grid_for(n, 256, 160), 256, 0, s>>>(a, b, n);
    check_cuda(cudaGetLastError(), "widen launch");
    note_launch();
}

}  // namespace mm
