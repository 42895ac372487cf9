// PCG kernel arguments and launchers (see pcg.cu).
#pragma once

#include "mm_internal.h"

namespace mm {

constexpr int PCG_THREADS = 1024;
constexpr int KMAX = 64;          // largest coarse dimension
constexpr int DOT_BLOCKS = 304;   // blocks of the stand-alone dot / vector kernels

// partial-sum slots per block
constexpr int S_PQ = 0, S_RR = 1, S_RZ = 2, S_COARSE = 3;
constexpr int PSTRIDE = S_COARSE + KMAX;

// device scalars (SC_PQ: p^T q, written by the scatter that forms q = A p)
constexpr int SC_RHO = 0, SC_BB = 1, SC_RR = 2, SC_TOL2 = 3, SC_PQ = 4;
// device flags
constexpr int F_DONE = 0, F_STATUS = 1, F_ITER = 2;

template <typename T>
struct PcgArgs {
    int64_t n;
    int npix;
    int maxit;
    T* x;
    T* r;
    T* p;
    float4* p4;          // FP32 I/Q/U: p packed per pixel for the Toeplitz gather, or nullptr
    const T* q;
    T* z;
    const T* bd;         // M_BD inverse blocks
    int k;               // coarse dimension (TWOLEVEL)
    const T* Z;          // [k][n]
    const T* AZ;         // [k][n]
    const double* Einv;  // E^-1 from the Cholesky factor of E, row-major [k][k]
    double* partial;     // [grid][PSTRIDE]
    double* scal;
    int* flags;
    unsigned* bar;
    unsigned bar_absent;           // 0 (diagnostic launches: blocks the barrier waits for in vain)
    unsigned long long wait_ns;    // limit of each barrier wait
    double* hist_alpha;  // optional, [maxhist]
    double* hist_beta;
    double* hist_rz;
    double* hist_rr;
    int maxhist;
    T* zstore;           // optional [maxstore][n]: z_j of every step (Ritz construction)
    int maxstore;
};

// Grid-wide barrier of a cooperative launch: a counter whose top bit flips once every
// block arrived (block 0 adds 2^31 - (blocks + absent - 1), the others 1; `absent` is 0
// in every solve, a diagnostic launch sets it to make the barrier wait for blocks that
// were never launched).  Each wait is bounded by wait_ns on the global timer (2 s in
// every solve); on timeout the block records MM_ERR_TIMEOUT, raises the done flag and the
// caller returns.  A timed-out barrier keeps partial arrivals in its counter: the host
// zeroes the counter before every launch sequence.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false when this block gave up waiting (timeout recorded in flags).
__device__ __forceinline__ bool grid_sync(unsigned* bar, int* flags, unsigned absent, unsigned long long wait_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        const unsigned nb = gridDim.x + absent;
        const unsigned inc = blockIdx.x == 0 ? (0x80000000u - (nb - 1u)) : 1u;
        __threadfence();
        const unsigned old = atomicAdd(bar, inc);
        const unsigned long long t0 = global_ns();
        while (((old ^ ld_acquire_u32(bar)) & 0x80000000u) == 0u) {
            if (global_ns() - t0 > wait_ns) {
                atomicExch(&flags[F_STATUS], (int)MM_ERR_TIMEOUT);
                atomicExch(&flags[F_DONE], 1);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

constexpr unsigned long long BARRIER_WAIT_NS = 2000000000ull;   // per wait, every solve

// Dot-product accumulator of one thread.  FP64 vectors: plain FP64 FMAs.  FP32 vectors:
// each product a b is formed exactly as p + e (p = fl(a b), e = fma(a, b, -p)) and
// accumulated as an unevaluated FP32 pair (hi, lo) with a two-sum, so the per-thread
// partial carries ~48 bits; it is converted to FP64 once for the block and grid sums.
// (Per-element FP32 -> FP64 conversions would run on the FP64 pipe, 1/64 of FP32 rate.)
// (hi, lo) += (h2, l2) with a two-sum of the high parts; symmetric in its operands.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float h2, float l2) {
    const float s = hi + h2;
    const float bv = s - hi;
    const float e = (hi - (s - bv)) + (h2 - bv);
    hi = s;
    lo = lo + l2 + e;
}

// Fixed xor-shuffle tree over the warp on (hi, lo) pairs; every lane gets the total.
__device__ __forceinline__ void warp_pair_reduce(float& hi, float& lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        pair_add(hi, lo, h2, l2);
    }
}

template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double total() const { return s; }
};
template <> struct DotAcc<float> {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);
        const float s = hi + p;
        const float bv = s - hi;
        const float err = (hi - (s - bv)) + (p - bv);
        hi = s;
        lo += err + e;
    }
    __device__ __forceinline__ double total() const { return (double)hi + (double)lo; }
};

template <typename T>
void launch_pcg(int which, int ncomp, int cm, const PcgArgs<T>& a, int nblocks, cudaStream_t s);  // cm: 0 M_BD, 1 M_2lvl, 2 A-DEF2
int pcg_max_blocks(int num_sms);

void launch_dot64(const double* a, const double* b, int64_t n, double* part, double* out, cudaStream_t s);
void launch_scale_to_f32(const double* a, const double* sq, float* b, int64_t n, cudaStream_t s);
void launch_axpy_f32(double* x, const float* d, const double* sq, int64_t n, cudaStream_t s);
void launch_sub(const double* b, const double* ax, double* r, int64_t n, cudaStream_t s);

}  // namespace mm
