// Banded Toeplitz N^-1 for many right-hand sides on the tensor cores (tcgen05), the
// third form of the batched operator (Sec. 2.1 / Eq. 4 applied to R columns at once).
//
// For output rows t0 .. t0 + 127 of one stationary interval the band product is a dense
// contraction over the window w = t0 - lambda .. t0 + 127 + lambda:
//     Z[t0 + m][r] = sum_k A[m][k] Y[w + k][r],   A[m][k] = c[k - m],
//     c[j] = t_|j - lambda| for 0 <= j <= 2 lambda (0 elsewhere),
// with Y zero outside the interval.  A depends on (k - m) only, so its K-chunks are the
// same for every tile of a PSD: they are prepared once per plan.  One CTA computes four
// consecutive 128-row tiles of an interval for up to 64 columns, N = 4 x (columns rounded
// up to 16) <= 256, with the FP32 accumulators in tensor memory.
//
// Accuracy: the products run in FP16 on split operands.  A column is scaled by a power of
// two so that its largest value is below 2^14 and split as hi + 2^-11 lo (hi = the FP16
// rounding of the value, lo = the FP16 rounding of 2^11 times the rest); the band rows
// likewise.  D = A_hi Y_hi + 2^-11 (A_hi Y_lo + A_lo Y_hi) leaves out only the 2^-22
// term and FP16 rounding of lo, about FP32 accuracy relative to the operands' norms.
//
// Pipeline: K-chunks of 64; two shared-memory stages of (A_hi, A_lo, B_hi, B_lo) in the
// no-swizzle K-major canonical layout (8 x 16-byte core matrices; 128 bytes between core
// matrices along K, 1024 bytes between them along M or N).  All warps stage chunk i
// while the tensor core works on chunk i - 1; one thread issues the twelve MMAs of a
// chunk (4 K-steps x 3 products) and commits them to the stage's mbarrier.  Every
// mbarrier wait is bounded; a wait that runs out records MM_ERR_TIMEOUT in the batched
// solver's flags and the CTA stops issuing, waits (bounded) for what it issued, frees
// its tensor memory and returns.
#include <cuda_fp16.h>

#include "batch.cuh"
#include "pcg.cuh"

namespace mm {

namespace {

constexpr int TC_M = 128;         // rows (times) per tile
constexpr int TC_TILES = 4;       // tiles per CTA
constexpr int TC_KC = 64;         // K per chunk (4 MMA K-steps of 16)
constexpr int TC_THREADS = 256;
constexpr int TC_A_BYTES = TC_M * TC_KC * 2;         // one FP16 A chunk (16 KB)
constexpr int TC_B_MAX = 256 * TC_KC * 2;            // one FP16 B chunk at N = 256 (32 KB)
constexpr int TC_STAGE = 2 * TC_A_BYTES + 2 * TC_B_MAX;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_now() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor: no swizzle, K-major; LBO = bytes between core matrices
// along K, SBO = bytes between core matrices along M / N.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Bounded wait for the given phase parity of an mbarrier; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = tc_now();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (tc_now() - t0 > TC_WAIT_NS) return false;
    }
}

// FP16 split of a scaled value: v = hi + 2^-11 lo.
__device__ __forceinline__ void split16(float v, __half& hi, __half& lo) {
    hi = __float2half_rn(v);
    lo = __float2half_rn((v - __half2float(hi)) * 2048.f);
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS, 1) batch_tc_kernel(BatchTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    if (a.done != nullptr && *(volatile const int*)a.done) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const SpanTile grp = a.groups[blockIdx.x];
    const int RB = a.RB;                       // columns per tile (multiple of 16)
    const int N = TC_TILES * RB;
    const int lam = a.lambda;
    const int nchunk = a.nchunk;
    const __half* atab = a.atab + (size_t)grp.psd * nchunk * (2 * TC_M * TC_KC);
    unsigned char* stage0 = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tm = tmem_base;
    const uint32_t d_hh = tm, d_x = tm + 256;   // accumulator columns
    // instruction descriptor: D FP32, A and B FP16, both K-major, N, M = 128
    const uint32_t idesc = (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    int issued = 0;   // chunks whose MMAs were issued (thread 0)
    for (int c = 0; c < nchunk; ++c) {
        const int s = c & 1;
        unsigned char* st = stage0 + s * TC_STAGE;
        __half* sAh = reinterpret_cast<__half*>(st);
        __half* sAl = reinterpret_cast<__half*>(st + TC_A_BYTES);
        __half* sBh = reinterpret_cast<__half*>(st + 2 * TC_A_BYTES);
        __half* sBl = reinterpret_cast<__half*>(st + 2 * TC_A_BYTES + TC_B_MAX);
        if (c >= 2) {
            // the MMAs of chunk c - 2 read this stage: wait for their commit
            if (!mbar_wait(&mbar[s], (uint32_t)(((c - 2) >> 1) & 1))) s_abort = 1;
        }
        __syncthreads();
        if (s_abort) break;
        // A chunk: prepared hi and lo halves, contiguous in the table (32 KB)
        {
            const uint4* src = reinterpret_cast<const uint4*>(atab + (size_t)c * (2 * TC_M * TC_KC));
            uint4* dst = reinterpret_cast<uint4*>(sAh);
            for (int i = tid; i < 2 * TC_A_BYTES / 16; i += TC_THREADS) dst[i] = __ldg(src + i);
        }
        // B chunk: for column col = g RB + r and k = c KC + kk, Y[r][w_g + k] scaled and
        // split; lane (row 0..7 of a core matrix, pair of k) writes 4 bytes of hi and lo
        {
            const int rr = lane >> 2, kp = (lane & 3) * 2;
            const int ncore = (N / 8) * (TC_KC / 8);
            for (int cm = warp; cm < ncore; cm += TC_THREADS / 32) {
                const int ni = cm >> 3, ki = cm & 7;
                const int col = ni * 8 + rr;
                const int g = col / RB, r = col - g * RB;
                const int kk = ki * 8 + kp;
                float v0 = 0.f, v1 = 0.f;
                if (r < a.R) {
                    const int64_t t = grp.out0 + (int64_t)g * TC_M - lam + (int64_t)c * TC_KC + kk;
                    const float* yr = a.Y + (size_t)r * a.nt;
                    const float sc = a.scale[r];
                    if (t >= grp.ibeg && t < grp.iend) v0 = __ldg(yr + t) * sc;
                    if (t + 1 >= grp.ibeg && t + 1 < grp.iend) v1 = __ldg(yr + t + 1) * sc;
                }
                __half h0, l0, h1, l1;
                split16(v0, h0, l0);
                split16(v1, h1, l1);
                const int off = (ni * 1024 + ki * 128 + rr * 16 + kp * 2) / 2;
                *reinterpret_cast<__half2*>(sBh + off) = __halves2half2(h0, h1);
                *reinterpret_cast<__half2*>(sBl + off) = __halves2half2(l0, l1);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
#pragma unroll
            for (int ks = 0; ks < TC_KC / 16; ++ks) {
                const uint32_t o = ks * 256;   // two core matrices along K per step
                const int first = c == 0 && ks == 0;
                mma_f16(d_hh, sdesc(ah + o, 128, 1024), sdesc(bh + o, 128, 1024), idesc, !first);
                mma_f16(d_x, sdesc(ah + o, 128, 1024), sdesc(bl + o, 128, 1024), idesc, !first);
                mma_f16(d_x, sdesc(al + o, 128, 1024), sdesc(bh + o, 128, 1024), idesc, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[s])));
        }
        issued = c + 1;
    }
    // wait for the last issued chunk (its commit covers every earlier MMA); the outcome
    // is made uniform over the CTA before the warp-collective tensor-memory loads
    bool ok = s_abort == 0;
    if (issued > 0) {
        const int c = issued - 1;
        if (!mbar_wait(&mbar[c & 1], (uint32_t)((c >> 1) & 1))) ok = false;
    }
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) {
        if (tid == 0) {
            atomicExch(&a.flags[F_STATUS], (int)MM_ERR_TIMEOUT);
            atomicExch(&a.flags[F_DONE], 1);
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. (rows m), columns of half w / 4
        const int q = warp & 3, h = warp >> 2;
        const int m = q * 32 + lane;
        const float inv_c = a.inv_cscale[grp.psd];
        for (int c0 = h * (N / 2); c0 < (h + 1) * (N / 2); c0 += 16) {
            uint32_t vh[16], vx[16];
            const uint32_t lane_off = (uint32_t)(q * 32) << 16;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(vh[0]), "=r"(vh[1]), "=r"(vh[2]), "=r"(vh[3]), "=r"(vh[4]), "=r"(vh[5]), "=r"(vh[6]),
                  "=r"(vh[7]), "=r"(vh[8]), "=r"(vh[9]), "=r"(vh[10]), "=r"(vh[11]), "=r"(vh[12]), "=r"(vh[13]),
                  "=r"(vh[14]), "=r"(vh[15])
                : "r"(d_hh + lane_off + c0));
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(vx[0]), "=r"(vx[1]), "=r"(vx[2]), "=r"(vx[3]), "=r"(vx[4]), "=r"(vx[5]), "=r"(vx[6]),
                  "=r"(vx[7]), "=r"(vx[8]), "=r"(vx[9]), "=r"(vx[10]), "=r"(vx[11]), "=r"(vx[12]), "=r"(vx[13]),
                  "=r"(vx[14]), "=r"(vx[15])
                : "r"(d_x + lane_off + c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int col = c0 + j;
                const int g = col / RB, r = col - g * RB;
                const int64_t n = (int64_t)g * TC_M + m;   // output index within the group
                if (r < a.R && n < grp.nout) {
                    const float v = __uint_as_float(vh[j]) + __uint_as_float(vx[j]) * (1.f / 2048.f);
                    a.Z[(size_t)r * a.nt + grp.out0 + n] = v * inv_c * a.inv_scale[r];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tm));
}

size_t batch_tc_smem() { return 2 * (size_t)TC_STAGE + 1024; }

void launch_batch_tc(const BatchTcArgs& A, int ngroups, cudaStream_t s) {
    const size_t smem = batch_tc_smem();
    ensure_smem_attr((const void*)batch_tc_kernel, (int)smem, "cudaFuncSetAttribute(batch tensor)");
    batch_tc_kernel<<<(unsigned)ngroups, TC_THREADS, smem, s>>>(A);
    check_cuda(cudaGetLastError(), "batch tensor launch");
    note_launch();
}

// Y_r = P X_r for r < R (time-domain [R][nt]) and the power-of-two column scales: scale_r
// = 2^(13 - e), 2^e >= 3 max |X_r| (a bound of max |Y_r|), inv_scale_r = 1 / scale_r.
template <int NC>
__global__ void batch_gather_kernel(const int32_t* __restrict__ pixc, const float2* __restrict__ w,
                                    const float* __restrict__ X, int64_t n, int64_t nt, int R, float* __restrict__ Y) {
    const int r = blockIdx.y;
    const float* x = X + (size_t)r * n;
    float* y = Y + (size_t)r * nt;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nt; t += (int64_t)gridDim.x * blockDim.x) {
        const int q = __ldg(pixc + t);
        float v = 0.f;
        if (q >= 0) {
            if constexpr (NC == 1) {
                v = __ldg(x + q);
            } else {
                const float2 c = w[t];
                const float* xq = x + 3 * (int64_t)q;
                v = __ldg(xq) + c.x * __ldg(xq + 1) + c.y * __ldg(xq + 2);
            }
        }
        y[t] = v;
    }
}

__global__ void batch_colscale_kernel(const float* __restrict__ X, int64_t n, float* scale, float* inv_scale) {
    __shared__ float wm[32];
    const int r = blockIdx.x;
    const float* x = X + (size_t)r * n;
    float mx = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx = fmaxf(mx, fabsf(x[i]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, wm[i]);
        const float bound = 3.f * m;
        int e = 0;
        if (bound > 0.f && isfinite(bound)) frexpf(bound, &e);   // bound < 2^e
        scale[r] = ldexpf(1.f, 13 - e);
        inv_scale[r] = ldexpf(1.f, e - 13);
    }
}

void launch_batch_gather(const Plan& P, const float* X, int R, float* Y, cudaStream_t s) {
    const int th = 256;
    int64_t g = (P.nt + th - 1) / th;
    if (g > 2048) g = 2048;
    const dim3 grid((unsigned)g, (unsigned)R);
    if (P.ncomp == 1)
        batch_gather_kernel<1><<<grid, th, 0, s>>>(P.pixc, P.w32, X, P.n, P.nt, R, Y);
    else
        batch_gather_kernel<3><<<grid, th, 0, s>>>(P.pixc, P.w32, X, P.n, P.nt, R, Y);
    check_cuda(cudaGetLastError(), "batch gather launch");
    note_launch();
}

void launch_batch_colscale(const float* X, int64_t n, int R, float* scale, float* inv_scale, cudaStream_t s) {
    batch_colscale_kernel<<<R, 512, 0, s>>>(X, n, scale, inv_scale);
    check_cuda(cudaGetLastError(), "batch column scale launch");
    note_launch();
}

}  // namespace mm
