// Preconditioned CG (Sec. 3.1) -- everything except the product q = A p runs in one
// persistent cooperative kernel per iteration:
//
//   alpha = rho / p^T q;  x += alpha p;  r -= alpha q;  stop if ||r|| <= tol ||b||
//   z = M r  (M_BD of Eq. 10; M_2lvl of Eq. 12 applied as in App. C:
//             v = E^-1 Z^T r with the FP64 E^-1, z = M_BD (r - AZ v) + Z v; or the
//             A-DEF2 form of App. B: y = M_BD r, v = E^-1 (Z^T r - (AZ)^T y),
//             z = y + Z v, started from x_0 = Z E^-1 Z^T b)
//   rho' = r^T z;  beta = rho' / rho;  p = z + beta p
//
// Dot products are accumulated in FP64 per block (fixed thread order), written as block
// partials and summed by every block in block order after a grid barrier, so every block
// sees the same scalars and the result is bit-reproducible.  The grid barrier is a
// counter whose top bit flips once all blocks arrived; each wait is bounded in time
// (a kernel argument, 2 s on the global timer in every solve), after which the kernel
// records MM_ERR_TIMEOUT and returns.
// The iteration count, stopping decision and scalar history live in device memory; the
// host only polls a done flag every few iterations.
#include "pcg.cuh"

namespace mm {

// Reductions.  GB300 runs FP64 at 1/64 of the FP32 rate, so the wide part of every
// reduction (within warps) works on exact FP32 pairs and only warp 0 does a few FP64
// additions.  All trees are fixed (xor shuffles, lanes over blocks in order), so every
// block obtains bit-identical scalars.

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block total of per-thread accumulators; valid in every thread.  Call with all threads.
__device__ double block_total(DotAcc<float> acc, double* sh) {
    __shared__ float2 wp[32];
    float hi = acc.hi, lo = acc.lo;
    warp_pair_reduce(hi, lo);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (l == 0) wp[w] = make_float2(hi, lo);
    __syncthreads();
    if (w == 0) {
        const double v = warp_sum64(l < nw ? (double)wp[l].x + (double)wp[l].y : 0.0);
        if (l == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

__device__ double block_total(DotAcc<double> acc, double* sh) {
    const double v = warp_sum64(acc.s);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[1 + w] = v;
    __syncthreads();
    if (w == 0) {
        const double t = warp_sum64(l < nw ? sh[1 + l] : 0.0);
        if (l == 0) sh[0] = t;
    }
    __syncthreads();
    return sh[0];
}

// Sum of slot `slot` over all block partials (warp 0: lanes over blocks in order, then a
// shuffle tree), valid in every thread.  Call with all threads.
__device__ double grid_total(const double* part, int slot, double* sh) {
    if (threadIdx.x < 32) {
        // each lane issues its (up to 8) loads before adding them in block order
        double s = 0.0;
        for (unsigned base = 0; base < gridDim.x; base += 256) {
            double v[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const unsigned b = base + threadIdx.x + 32u * t;
                v[t] = b < gridDim.x ? __ldcg(part + (size_t)b * PSTRIDE + slot) : 0.0;
            }
#pragma unroll
            for (int t = 0; t < 8; ++t) s += v[t];
        }
        s = warp_sum64(s);
        if (threadIdx.x == 0) sh[0] = s;
    }
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Pixel range of this block.
__device__ __forceinline__ void block_pixels(int npix, int& lo, int& hi) {
    const int chunk = (npix + gridDim.x - 1) / gridDim.x;
    lo = blockIdx.x * chunk;
    hi = min(npix, lo + chunk);
    if (lo > hi) lo = hi;
}

// Z^T r (CM 1) or Z^T r - (AZ)^T y with y = M_BD r already in a.z (CM 2) over this
// block's elements -> part[blk][S_COARSE + j] (a preconditioner input, not a CG dot
// product: lanes accumulate in T, the reductions above them in FP64)
template <typename T, int CM = 1>
__device__ void coarse_partials(const PcgArgs<T>& a, const T* r, int64_t e0, int64_t e1) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = w; j < a.k; j += nw) {
        const T* zj = a.Z + (size_t)j * a.n;
        const T* azj = a.AZ + (size_t)j * a.n;
        // per-lane partial in T (a few dozen terms: for T = float this keeps the FP64 pipe,
        // which GB300 runs at 1/64 of the FP32 rate, for the cross-lane / block sums)
        T sl = (T)0;
#pragma unroll 8
        for (int64_t i = e0 + l; i < e1; i += 32) {
            sl += __ldg(zj + i) * r[i];
            if constexpr (CM == 2) sl -= __ldg(azj + i) * a.z[i];
        }
        double* slot = a.partial + (size_t)blockIdx.x * PSTRIDE + S_COARSE + j;
        if constexpr (sizeof(T) == 4) {
            float hi = sl, lo = 0.f;
            warp_pair_reduce(hi, lo);
            if (l == 0) *reinterpret_cast<float2*>(slot) = make_float2(hi, lo);
        } else {
            const double s = warp_sum64(sl);
            if (l == 0) *slot = s;
        }
    }
}

// v = E^-1 u, u = Z^T r from the block partials (warps reduce the k coarse slots, lanes
// over blocks in a fixed order), then the k x k matvec with the stored E^-1: warp w owns
// rows w, w + nw, ...; lanes split the row, FP64 throughout.
template <typename T>
__device__ void coarse_solve(const PcgArgs<T>& a, double* v_sh) {
    __shared__ double u_sh[KMAX];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = w; j < a.k; j += nw) {
        const double* col = a.partial + S_COARSE + j;
        // each lane issues its (up to 8) loads before adding them in block order
        if constexpr (sizeof(T) == 4) {
            float hi = 0.f, lo = 0.f;
            for (unsigned base = 0; base < gridDim.x; base += 256) {
                float2 v[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const unsigned b = base + l + 32u * t;
                    v[t] = b < gridDim.x ? __ldcg(reinterpret_cast<const float2*>(col + (size_t)b * PSTRIDE))
                                         : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) pair_add(hi, lo, v[t].x, v[t].y);
            }
            warp_pair_reduce(hi, lo);
            if (l == 0) u_sh[j] = (double)hi + (double)lo;
        } else {
            double s = 0.0;
            for (unsigned base = 0; base < gridDim.x; base += 256) {
                double v[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const unsigned b = base + l + 32u * t;
                    v[t] = b < gridDim.x ? __ldcg(col + (size_t)b * PSTRIDE) : 0.0;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) s += v[t];
            }
            s = warp_sum64(s);
            if (l == 0) u_sh[j] = s;
        }
    }
    __syncthreads();
    // one thread per row of E^-1 (k <= 64 threads; a short FP64 FMA chain each rather
    // than warp trees, whose FP64 shuffles and adds occupy GB300's narrow FP64 pipe).
    // E^-1 is symmetric: thread i reads column i, so a warp's loads for one j coalesce.
    if (threadIdx.x < a.k) {
        double s = 0.0;
#pragma unroll 8
        for (int j = 0; j < a.k; ++j) s = fma(__ldg(a.Einv + (size_t)j * a.k + threadIdx.x), u_sh[j], s);
        v_sh[threadIdx.x] = s;
    }
    __syncthreads();
}

// The iteration kernel's form of coarse_solve: E^-1 already in shared memory (einv, loaded
// at the start of the step) and the r^T r total reduced in the same round of loads as the
// first coarse slot (warp 0), so that the step waits on one round trip to the block
// partials after its first grid barrier instead of three.  Sums in the same order as
// grid_total and coarse_solve.  Returns r^T r; v_sh as coarse_solve.
template <typename T>
__device__ double coarse_solve_rr(const PcgArgs<T>& a, double* v_sh, const double* einv, double* sh) {
    __shared__ double u_sh[KMAX];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = w; j < a.k; j += nw) {
        const bool rr_too = j == 0;
        const double* col = a.partial + S_COARSE + j;
        double srr = 0.0;
        if constexpr (sizeof(T) == 4) {
            float hi = 0.f, lo = 0.f;
            for (unsigned base = 0; base < gridDim.x; base += 256) {
                float2 v[8];
                double vr[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const unsigned b = base + l + 32u * t;
                    v[t] = b < gridDim.x ? __ldcg(reinterpret_cast<const float2*>(col + (size_t)b * PSTRIDE))
                                         : make_float2(0.f, 0.f);
                    vr[t] = rr_too && b < gridDim.x ? __ldcg(a.partial + (size_t)b * PSTRIDE + S_RR) : 0.0;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) pair_add(hi, lo, v[t].x, v[t].y);
#pragma unroll
                for (int t = 0; t < 8; ++t) srr += vr[t];
            }
            warp_pair_reduce(hi, lo);
            if (l == 0) u_sh[j] = (double)hi + (double)lo;
        } else {
            double s = 0.0;
            for (unsigned base = 0; base < gridDim.x; base += 256) {
                double v[8], vr[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const unsigned b = base + l + 32u * t;
                    v[t] = b < gridDim.x ? __ldcg(col + (size_t)b * PSTRIDE) : 0.0;
                    vr[t] = rr_too && b < gridDim.x ? __ldcg(a.partial + (size_t)b * PSTRIDE + S_RR) : 0.0;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) s += v[t];
#pragma unroll
                for (int t = 0; t < 8; ++t) srr += vr[t];
            }
            s = warp_sum64(s);
            if (l == 0) u_sh[j] = s;
        }
        if (rr_too) {
            srr = warp_sum64(srr);
            if (l == 0) sh[0] = srr;
        }
    }
    __syncthreads();
    if (threadIdx.x < a.k) {
        double s = 0.0;
#pragma unroll 8
        for (int j = 0; j < a.k; ++j) s = fma(einv[(size_t)j * a.k + threadIdx.x], u_sh[j], s);
        v_sh[threadIdx.x] = s;
    }
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

// z = M_BD r (CM 0), M_BD (r - AZ v) + Z v (CM 1) or y + Z v with y = M_BD r in a.z
// (CM 2) on this block's pixels; returns partial r^T z.  With a coarse space, G = 2 or 4
// consecutive lanes share a pixel when the block has that many threads per pixel: lane
// g of the group sums the coarse columns j = g, g + G, ... and the group combines its
// partial sums by a fixed xor-shuffle tree (G fixed by the plan's sizes, so results are
// reproducible); the group's first lane finishes the pixel.
template <typename T, int NC, int CM>
__device__ DotAcc<T> apply_precond(const PcgArgs<T>& a, const double* v_sh, int p0, int p1) {
    __shared__ T vt[KMAX];
    DotAcc<T> rz;
    if constexpr (CM == 0) {
        for (int q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
            const int64_t e = (int64_t)q * NC;
            T t[NC], out[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) t[c] = a.r[e + c];
            if constexpr (NC == 1) {
                out[0] = a.bd[q] * t[0];
            } else {
                const T* m = a.bd + 6 * (int64_t)q;
                out[0] = m[0] * t[0] + m[1] * t[1] + m[2] * t[2];
                out[1] = m[1] * t[0] + m[3] * t[1] + m[4] * t[2];
                out[2] = m[2] * t[0] + m[4] * t[1] + m[5] * t[2];
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                a.z[e + c] = out[c];
                rz.add(t[c], out[c]);
            }
        }
        return rz;
    } else {
        if (threadIdx.x < a.k) vt[threadIdx.x] = (T)v_sh[threadIdx.x];
        __syncthreads();
        const int np = p1 - p0;
        const int nt = (int)blockDim.x;
        const int G = np * 4 <= nt ? 4 : (np * 2 <= nt ? 2 : 1);   // the same in every lane
        const int lg = threadIdx.x % G;
        const int per = nt / G;   // pixels per round
        for (int base = 0; base < np; base += per) {
            const int qi = base + (int)threadIdx.x / G;
            const bool valid = qi < np;
            const int q = p0 + (valid ? qi : 0);
            const int64_t e = (int64_t)q * NC;
            T t[NC], zc[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                t[c] = (T)0;
                zc[c] = (T)0;
            }
            if (valid) {
                if constexpr (CM == 2) {
#pragma unroll 4
                    for (int j = lg; j < a.k; j += G) {
                        const T vj = vt[j];
                        const T* zz = a.Z + (size_t)j * a.n + e;
#pragma unroll
                        for (int c = 0; c < NC; ++c) zc[c] += __ldg(zz + c) * vj;
                    }
                } else {
#pragma unroll 4
                    for (int j = lg; j < a.k; j += G) {
                        const T vj = vt[j];
                        const T* az = a.AZ + (size_t)j * a.n + e;
                        const T* zz = a.Z + (size_t)j * a.n + e;
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            t[c] -= __ldg(az + c) * vj;
                            zc[c] += __ldg(zz + c) * vj;
                        }
                    }
                }
            }
            for (int o = 1; o < G; o <<= 1) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    t[c] += __shfl_xor_sync(0xffffffffu, t[c], o);
                    zc[c] += __shfl_xor_sync(0xffffffffu, zc[c], o);
                }
            }
            if (!valid || lg != 0) continue;
            T r0[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) r0[c] = a.r[e + c];
            if constexpr (CM == 2) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    const T out = a.z[e + c] + zc[c];
                    a.z[e + c] = out;
                    rz.add(r0[c], out);
                }
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) t[c] += r0[c];
                T out[NC];
                if constexpr (NC == 1) {
                    out[0] = a.bd[q] * t[0] + zc[0];
                } else {
                    const T* m = a.bd + 6 * (int64_t)q;
                    out[0] = m[0] * t[0] + m[1] * t[1] + m[2] * t[2] + zc[0];
                    out[1] = m[1] * t[0] + m[3] * t[1] + m[4] * t[2] + zc[1];
                    out[2] = m[2] * t[0] + m[4] * t[1] + m[5] * t[2] + zc[2];
                }
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    a.z[e + c] = out[c];
                    rz.add(r0[c], out[c]);
                }
            }
        }
        return rz;
    }
}

// y = M_BD r into a.z on this block's pixels (the first step of the A-DEF2 form).
// p = z (first step) or p = z + be p over the block's pixels [p0, p1); zs (optional)
// records z.  FP32 I/Q/U plans also keep p packed per pixel (a.p4) for the Toeplitz gather.
template <typename T, int NC>
__device__ __forceinline__ void update_p(const PcgArgs<T>& a, int p0, int p1, bool first, T be, T* zs) {
    if constexpr (NC == 3 && sizeof(T) == 4) {
        if (a.p4 != nullptr) {
            for (int q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
                const int64_t i = 3 * (int64_t)q;
                T v[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const T zi = a.z[i + c];
                    v[c] = first ? zi : zi + be * a.p[i + c];
                    a.p[i + c] = v[c];
                    if (zs != nullptr) zs[i + c] = zi;
                }
                a.p4[q] = make_float4(v[0], v[1], v[2], 0.f);
            }
            return;
        }
    }
    for (int64_t i = (int64_t)p0 * NC + threadIdx.x; i < (int64_t)p1 * NC; i += blockDim.x) {
        const T zi = a.z[i];
        a.p[i] = first ? zi : zi + be * a.p[i];
        if (zs != nullptr) zs[i] = zi;
    }
}

template <typename T, int NC>
__device__ void bd_into_z(const PcgArgs<T>& a, int p0, int p1) {
    for (int q = p0 + threadIdx.x; q < p1; q += blockDim.x) {
        const int64_t e = (int64_t)q * NC;
        if constexpr (NC == 1) {
            a.z[e] = a.bd[q] * a.r[e];
        } else {
            const T* m = a.bd + 6 * (int64_t)q;
            const T r0 = a.r[e], r1 = a.r[e + 1], r2 = a.r[e + 2];
            a.z[e] = m[0] * r0 + m[1] * r1 + m[2] * r2;
            a.z[e + 1] = m[1] * r0 + m[3] * r1 + m[4] * r2;
            a.z[e + 2] = m[2] * r0 + m[4] * r1 + m[5] * r2;
        }
    }
}

// ------------------------------------------------------------------------ init kernel
// r = b is already in a.r.  x = 0 (CM 2: x = Z E^-1 Z^T b, r = b - AZ E^-1 Z^T b),
// z = M r, p = z, rho = r^T z, bb = b^T b.
template <typename T, int NC, int CM>
__global__ void __launch_bounds__(PCG_THREADS) pcg_init_kernel(PcgArgs<T> a) {
    __shared__ double sh[40];   // [0] total, [1 + w] per-warp sums (up to 32 warps)
    __shared__ double v_sh[KMAX];
    int p0, p1;
    block_pixels(a.npix, p0, p1);
    const int64_t e0 = (int64_t)p0 * NC, e1 = (int64_t)p1 * NC;
    DotAcc<T> bacc;
    for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
        a.x[i] = (T)0;
        bacc.add(a.r[i], a.r[i]);
    }
    const double bb = block_total(bacc, sh);
    if (threadIdx.x == 0) a.partial[(size_t)blockIdx.x * PSTRIDE + S_RR] = bb;
    if constexpr (CM != 0) coarse_partials<T, 1>(a, a.r, e0, e1);
    if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
    const double bbt = grid_total(a.partial, S_RR, sh);
    if constexpr (CM != 0) coarse_solve(a, v_sh);
    if constexpr (CM == 2) {
        // x0 = Z v, r0 = b - AZ v with v = E^-1 Z^T b (every block holds the same v)
        for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
            T xi = (T)0, ri = a.r[i];
            for (int j = 0; j < a.k; ++j) {
                const T vj = (T)v_sh[j];
                xi += __ldg(a.Z + (size_t)j * a.n + i) * vj;
                ri -= __ldg(a.AZ + (size_t)j * a.n + i) * vj;
            }
            a.x[i] = xi;
            a.r[i] = ri;
        }
        __syncthreads();   // bd_into_z reads whole pixels of r written element-wise above
        bd_into_z<T, NC>(a, p0, p1);
        // every block has read the first coarse partials before they are overwritten
        if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
        coarse_partials<T, 2>(a, a.r, e0, e1);
        if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
        coarse_solve(a, v_sh);
    }
    const DotAcc<T> rzacc = apply_precond<T, NC, CM>(a, v_sh, p0, p1);
    __syncthreads();
    update_p<T, NC>(a, p0, p1, true, (T)0, a.zstore);
    const double rz = block_total(rzacc, sh);
    if (threadIdx.x == 0) a.partial[(size_t)blockIdx.x * PSTRIDE + S_RZ] = rz;
    if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
    const double rho = grid_total(a.partial, S_RZ, sh);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.scal[SC_RHO] = rho;
        a.scal[SC_BB] = bbt;
        a.scal[SC_RR] = bbt;
        a.flags[F_ITER] = 0;
        if (a.hist_rz != nullptr) a.hist_rz[0] = rho;
        if (a.hist_rr != nullptr) a.hist_rr[0] = bbt;
        if (!(bbt > 0.0)) {
            a.flags[F_DONE] = 1;
            a.flags[F_STATUS] = isfinite(bbt) ? (int)MM_OK : (int)MM_ERR_NUMERIC;
        } else if (!isfinite(rho) || !(rho > 0.0)) {
            a.flags[F_DONE] = 1;
            a.flags[F_STATUS] = isfinite(rho) ? (int)MM_ERR_NOT_SPD : (int)MM_ERR_NUMERIC;
        } else {
            a.flags[F_DONE] = 0;
            a.flags[F_STATUS] = (int)MM_OK;
        }
    }
}

// ------------------------------------------------------------------- iteration kernel
template <typename T, int NC, int CM>
__global__ void __launch_bounds__(PCG_THREADS) pcg_iter_kernel(PcgArgs<T> a) {
    __shared__ double sh[40];   // [0] total, [1 + w] per-warp sums (up to 32 warps)
    __shared__ double v_sh[KMAX];
    __shared__ double einv_sh[CM != 0 ? KMAX * KMAX : 1];
    if (*(volatile int*)&a.flags[F_DONE]) return;
    int p0, p1;
    block_pixels(a.npix, p0, p1);
    const int64_t e0 = (int64_t)p0 * NC, e1 = (int64_t)p1 * NC;
    // E^-1 into shared memory now; it is read after the first grid barrier
    if constexpr (CM != 0)
        for (int i = threadIdx.x; i < a.k * a.k; i += blockDim.x) einv_sh[i] = __ldg(a.Einv + i);
    // p^T q comes from the scatter that formed q = A p (its last block summed it)
    const double pqt = __ldcg(a.scal + SC_PQ);
    const double rho = a.scal[SC_RHO];
    if (!(pqt > 0.0) || !isfinite(pqt)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.flags[F_STATUS] = isfinite(pqt) ? (int)MM_ERR_NOT_SPD : (int)MM_ERR_NUMERIC;
            a.flags[F_DONE] = 1;
        }
        return;
    }
    const double alpha = rho / pqt;
    // phase B: x += alpha p, r -= alpha q, r^T r, Z^T r
    const T al = (T)alpha;
    DotAcc<T> racc;
    for (int64_t i = e0 + threadIdx.x; i < e1; i += blockDim.x) {
        a.x[i] += al * a.p[i];
        const T ri = a.r[i] - al * a.q[i];
        a.r[i] = ri;
        racc.add(ri, ri);
    }
    const double rr = block_total(racc, sh);
    if (threadIdx.x == 0) a.partial[(size_t)blockIdx.x * PSTRIDE + S_RR] = rr;
    if constexpr (CM == 1) {
        __syncthreads();
        coarse_partials<T, 1>(a, a.r, e0, e1);
    }
    if constexpr (CM == 2) {
        __syncthreads();
        bd_into_z<T, NC>(a, p0, p1);
        __syncthreads();
        coarse_partials<T, 2>(a, a.r, e0, e1);
    }
    if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
    // r^T r and (two-level) v = E^-1 Z^T r in one round of loads
    double rrt;
    if constexpr (CM != 0) {
        if (a.k > 0) rrt = coarse_solve_rr(a, v_sh, einv_sh, sh);
        else rrt = grid_total(a.partial, S_RR, sh);
    } else {
        rrt = grid_total(a.partial, S_RR, sh);
    }
    const int it = a.flags[F_ITER] + 1;     // every block reads the same value here
    bool stop = false;
    int status = MM_OK;
    if (!isfinite(rrt)) {
        stop = true;
        status = MM_ERR_NUMERIC;
    } else if (rrt <= a.scal[SC_TOL2] * a.scal[SC_BB]) {
        stop = true;
    } else if (it >= a.maxit) {
        stop = true;
        status = MM_ERR_NOT_CONVERGED;
    }
    if (stop) {
        // every block has read F_ITER above; wait for all before block 0 updates it
        if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.flags[F_ITER] = it;
            a.scal[SC_RR] = rrt;
            if (a.hist_alpha != nullptr && it - 1 < a.maxhist) a.hist_alpha[it - 1] = alpha;
            if (a.hist_rr != nullptr && it < a.maxhist) a.hist_rr[it] = rrt;
            a.flags[F_STATUS] = status;
            a.flags[F_DONE] = 1;
        }
        return;
    }
    // phase C: z = M r, r^T z (v_sh holds v for the two-level forms)
    const DotAcc<T> rzacc = apply_precond<T, NC, CM>(a, v_sh, p0, p1);
    const double rz = block_total(rzacc, sh);
    if (threadIdx.x == 0) a.partial[(size_t)blockIdx.x * PSTRIDE + S_RZ] = rz;
    if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
    const double rzt = grid_total(a.partial, S_RZ, sh);
    const double beta = rzt / rho;
    const T be = (T)beta;
    T* zs = (a.zstore != nullptr && it < a.maxstore) ? a.zstore + (size_t)it * a.n : nullptr;
    update_p<T, NC>(a, p0, p1, false, be, zs);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.flags[F_ITER] = it;
        a.scal[SC_RHO] = rzt;
        a.scal[SC_RR] = rrt;
        if (a.hist_alpha != nullptr && it - 1 < a.maxhist) a.hist_alpha[it - 1] = alpha;
        if (a.hist_beta != nullptr && it - 1 < a.maxhist) a.hist_beta[it - 1] = beta;
        if (a.hist_rz != nullptr && it < a.maxhist) a.hist_rz[it] = rzt;
        if (a.hist_rr != nullptr && it < a.maxhist) a.hist_rr[it] = rrt;
        if (!isfinite(rzt) || !(rzt > 0.0)) {
            a.flags[F_STATUS] = isfinite(rzt) ? (int)MM_ERR_NOT_SPD : (int)MM_ERR_NUMERIC;
            a.flags[F_DONE] = 1;
        }
    }
}

// --------------------------------------------------------------- stand-alone M_2lvl
// Used by mm_precond: the same device functions as in PCG, launched cooperatively.
template <typename T, int NC, int CM>
__global__ void __launch_bounds__(PCG_THREADS) precond_kernel(PcgArgs<T> a) {
    __shared__ double v_sh[KMAX];
    int p0, p1;
    block_pixels(a.npix, p0, p1);
    const int64_t e0 = (int64_t)p0 * NC, e1 = (int64_t)p1 * NC;
    if constexpr (CM == 2) {
        bd_into_z<T, NC>(a, p0, p1);
        __syncthreads();
    }
    if constexpr (CM != 0) {
        coarse_partials<T, CM>(a, a.r, e0, e1);
        if (!grid_sync(a.bar, a.flags, a.bar_absent, a.wait_ns)) return;
        coarse_solve(a, v_sh);
    }
    (void)apply_precond<T, NC, CM>(a, v_sh, p0, p1);
}

// ----------------------------------------------------------------------- launchers
template <typename T>
static void coop(void (*kern)(PcgArgs<T>), const PcgArgs<T>& a, int nblocks, cudaStream_t s) {
    void* args[] = {(void*)&a};
    check_cuda(cudaLaunchCooperativeKernel((const void*)kern, dim3(nblocks), dim3(PCG_THREADS), args,
                                           0, s),
               "cooperative PCG launch");
    note_launch();
}

template <typename T>
void launch_pcg(int which, int ncomp, int cm, const PcgArgs<T>& a, int nblocks, cudaStream_t s) {
#define MM_PCG_CASE(NC, CM)                                                 \
    if (ncomp == NC && cm == CM) {                                          \
        if (which == 0) coop<T>(pcg_init_kernel<T, NC, CM>, a, nblocks, s); \
        else if (which == 1) coop<T>(pcg_iter_kernel<T, NC, CM>, a, nblocks, s); \
        else coop<T>(precond_kernel<T, NC, CM>, a, nblocks, s);              \
        return;                                                             \
    }
    MM_PCG_CASE(1, 0)
    MM_PCG_CASE(1, 1)
    MM_PCG_CASE(1, 2)
    MM_PCG_CASE(3, 0)
    MM_PCG_CASE(3, 1)
    MM_PCG_CASE(3, 2)
#undef MM_PCG_CASE
    throw Error{MM_ERR_ARG, "launch_pcg: bad ncomp or coarse mode"};
}
template void launch_pcg<double>(int, int, int, const PcgArgs<double>&, int, cudaStream_t);
template void launch_pcg<float>(int, int, int, const PcgArgs<float>&, int, cudaStream_t);

// One block per SM: enough threads for the map-sized vectors, and few block partials
// for the reductions.
int pcg_max_blocks(int num_sms) {
    int per_sm = 0;
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_iter_kernel<double, 3, 2>,
                                                             PCG_THREADS, 0),
               "occupancy");
    if (per_sm < 1) throw Error{MM_ERR_CUDA, "PCG kernel does not fit on an SM"};
    return num_sms;
}

// ------------------------------------------------------------------ vector helpers
// Deterministic FP64 dot: per-block partials then one block sums them in order.
template <typename TA, typename TB>
__global__ void dot_partial_kernel(const TA* a, const TB* b, int64_t n, double* part) {
    __shared__ double sh[40];   // [0] total, [1 + w] per-warp sums (up to 32 warps)
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)b[i];
    s = block_total(DotAcc<double>{s}, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void sum_kernel(const double* part, int m, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += part[i];
        *out = s;
    }
}

void launch_dot64(const double* a, const double* b, int64_t n, double* part, double* out, cudaStream_t s) {
    const int g = DOT_BLOCKS;
    dot_partial_kernel<double, double><<<g, 256, 0, s>>>(a, b, n, part);
    sum_kernel<<<1, 32, 0, s>>>(part, g, out);
    check_cuda(cudaGetLastError(), "dot launch");
    note_launch(2);
}

__global__ void scale_to_f32_kernel(const double* a, const double* scale, float* b, int64_t n) {
    const double sc = 1.0 / sqrt(*scale);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)(a[i] * sc);
}

// b = (float)(a / sqrt(*sq))
void launch_scale_to_f32(const double* a, const double* sq, float* b, int64_t n, cudaStream_t s) {
    scale_to_f32_kernel<<<DOT_BLOCKS, 256, 0, s>>>(a, sq, b, n);
    check_cuda(cudaGetLastError(), "scale launch");
    note_launch();
}

__global__ void axpy_f32_kernel(double* x, const float* d, const double* sq, int64_t n) {
    const double sc = sqrt(*sq);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += sc * (double)d[i];
}

// x += sqrt(*sq) * d
void launch_axpy_f32(double* x, const float* d, const double* sq, int64_t n, cudaStream_t s) {
    axpy_f32_kernel<<<DOT_BLOCKS, 256, 0, s>>>(x, d, sq, n);
    check_cuda(cudaGetLastError(), "axpy launch");
    note_launch();
}

__global__ void sub_kernel(const double* b, const double* ax, double* r, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = b[i] - ax[i];
}

void launch_sub(const double* b, const double* ax, double* r, int64_t n, cudaStream_t s) {
    sub_kernel<<<DOT_BLOCKS, 256, 0, s>>>(b, ax, r, n);
    check_cuda(cudaGetLastError(), "sub launch");
    note_launch();
}

}  // namespace mm
