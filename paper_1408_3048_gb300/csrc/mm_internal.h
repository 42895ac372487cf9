// Internal declarations shared by the translation units of libmm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/mm.h"

namespace mm {

// ---------------------------------------------------------------------------------
// Overlap-save tile of the single-right-hand-side Toeplitz kernels: a block of B real
// positions holding up to TILE_SEGS segments of samples.  Segment g covers block positions
// [pb[g], pe[g]) and position p in it holds the sample of time p + d[g]; every other
// position is 0.  The segments of one tile come from consecutive stationary intervals of
// one PSD, separated in the block by at least lambda zeros, so the band product of one
// interval never reaches another (Eq. 4: no coupling between intervals).  The valid
// outputs are block positions [lambda, lambda + nout); those inside a segment are stored
// at their time.  Unused segments have pb = pe = TILE_NONE.
constexpr int TILE_SEGS = 3;
constexpr int32_t TILE_NONE = 0x7fffffff;
struct Tile {
    int64_t d[TILE_SEGS];
    int32_t pb[TILE_SEGS];
    int32_t pe[TILE_SEGS];
    int32_t nout;
    int32_t psd;
};

// Tile of the batched kernels: block of B real samples [in0, in0 + B) of one interval
// producing the valid outputs [out0, out0 + nout) (out0 = in0 + lambda); samples outside
// [ibeg, iend) read as 0.
struct SpanTile {
    int64_t out0;
    int64_t ibeg;
    int64_t iend;
    int32_t nout;
    int32_t psd;
};

// Device tables of one arithmetic precision (T = double or float).
struct ToeplitzDev {
    int logn = 0;            // complex FFT length N = 2^logn, real block B = 2N
    int cluster = 1;         // CTAs per tile (2 or 4: split across a thread-block cluster)
    int ntiles = 0;
    Tile* tiles = nullptr;   // [ntiles]
    void* twiddle = nullptr; // T[B/4 + 1]: cos(2 pi k / B)
    void* ptw = nullptr;     // T2[...]: per-pass twiddles of the N-point FFT
    void* H = nullptr;       // T[npsd][N + 1]: kernel spectrum / N (real, even kernel)
};

struct CoarseDev {
    int k = 0;                   // kept dimension
    double* Z64 = nullptr;       // [k][n]
    double* AZ64 = nullptr;      // [k][n]
    float* Z32 = nullptr;        // [k][n]
    float* AZ32 = nullptr;       // [k][n]
    double* Einv = nullptr;      // [k][k] E^-1 = L^-T L^-1 from the Cholesky factor (row-major)
    std::vector<double> ritz;    // k smallest Ritz values
};

// Scratch and state of the PCG driver.
struct PcgDev {
    int64_t n = 0;
    int nblocks = 0;             // cooperative grid size
    double* partial = nullptr;   // [nblocks][2 + KMAX] block partial sums
    double* scal = nullptr;      // [16] device scalars (see pcg.cu)
    int* flags = nullptr;        // [8] done / status / iteration / barrier words
    unsigned* barrier = nullptr; // grid barrier word
    void* x = nullptr;           // vectors, sized for double
    void* r = nullptr;
    void* p = nullptr;
    void* q = nullptr;
    void* z = nullptr;
    double* hist_alpha = nullptr;  // [maxhist]
    double* hist_beta = nullptr;   // [maxhist]
    double* hist_rz = nullptr;     // [maxhist]
    double* hist_rr = nullptr;     // [maxhist]
    int maxhist = 0;
    double* sc_part = nullptr;     // [scatter blocks] p^T q partials of the fused scatter
    unsigned* sc_count = nullptr;  // arrival counter of that scatter's last-block sum
};

// Per-stage CUDA-event timers (enabled by mm_profile).
enum { ST_TZ64 = 0, ST_TZ32 = 1, ST_SC64 = 2, ST_SC32 = 3, ST_PCG64 = 4, ST_PCG32 = 5, ST_TZDF = 6, ST_COUNT = 8 };
struct Prof {
    bool on = false;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[ST_COUNT] = {0, 0, 0, 0, 0, 0, 0, 0};
    int64_t launches[ST_COUNT] = {0, 0, 0, 0, 0, 0, 0, 0};
};

struct Plan {
    // problem
    int64_t nt = 0;
    int32_t npix_sky = 0;
    int32_t ncomp = 1;
    int32_t K = 0;
    int32_t npsd = 0;
    int32_t lambda = 0;
    int32_t window = MM_WINDOW_GAUSS;
    double fsamp = 100.0;
    double rcond_min = 1e-6;
    cudaStream_t stream = 0;
    int device = 0;                // device current when the plan was made
    int num_sms = 0;
    int scatter_lpp = 32;          // scatter lanes per pixel (32, 16 or 8; the pixel tile)
    int64_t L_grid = 0;

    // observed pixels
    int32_t npix_obs = 0;
    int64_t n = 0;
    int64_t nkept = 0;
    std::vector<int32_t> h_obs2sky, h_hits;
    std::vector<std::vector<double>> rows;   // [npsd][lambda+1]
    std::vector<int64_t> h_ioff;
    std::vector<int32_t> h_ipsd;

    // device pointing (time order) and pixel-sorted CSR
    int32_t* pixc = nullptr;       // [nt] observed index or -1
    double2* w64 = nullptr;        // [nt] (cos, sin), pol only
    float2* w32 = nullptr;         // [nt]
    int32_t* csr_off = nullptr;    // [npix_obs + 1]
    int32_t* tsort = nullptr;      // [nkept] sample index, pixel-major, ascending t
    double2* wsort64 = nullptr;    // [nkept] weights in sorted order (pol)
    float2* wsort32 = nullptr;     // [nkept]
    float* asort32 = nullptr;      // [nkept] angle / pi of the sorted weights when every weight
                                   // pair has unit norm (the FP32 scatter reads 4 bytes, not 8)
    int64_t* ioff = nullptr;       // [K+1]
    int32_t* ipsd = nullptr;       // [K]
    double* t0 = nullptr;          // [npsd] diagonal of each row

    ToeplitzDev tz64, tz32;
    ToeplitzDev tzdf;              // double-float tables on tz64's blocks (refinement residual)

    // block-Jacobi: inverse blocks, symmetric packed (a00 a01 a02 a11 a12 a22) or 1
    double* bd64 = nullptr;        // [npix_obs][ncomp == 3 ? 6 : 1]
    float* bd32 = nullptr;

    // time-domain scratch
    double* tod64 = nullptr;       // [nt]
    float* tod32 = nullptr;        // [nt]
    float4* map4 = nullptr;        // [npix_obs] FP32 I/Q/U map packed per pixel (ncomp 3): the
                                   // layout the Toeplitz gather reads in one 16-byte load
    double* dbuf = nullptr;        // [nt] staging for host data
    double* b64 = nullptr;         // [n] last right-hand side
    bool have_b = false;

    CoarseDev coarse;
    PcgDev pcg;
    Prof prof;

    std::string err;
};

// profiling helpers (api.cu): begin returns a slot (or -1 when off), end closes it
int prof_begin(Plan& P, int stage);
void prof_end(Plan& P, int slot);
void prof_flush(Plan& P);   // after a stream synchronisation

// error helpers ----------------------------------------------------------------------
struct Error {
    mm_status st;
    std::string msg;
};

void check_cuda(cudaError_t e, const char* what);   // throws Error{MM_ERR_CUDA}
// cudaFuncSetAttribute(kern, MaxDynamicSharedMemorySize, bytes) once per kernel and
// device (thread-safe; the attribute is per device, so a second GPU gets its own call)
void ensure_smem_attr(const void* kern, int bytes, const char* what);
// Runs f and turns what it throws into a status: sets P->err (P may be null) and the
// calling thread's last-error message (mm_last_error(NULL)).  Nothing leaves it.
mm_status run_guarded(Plan* P, void (*f)(void*), void* ctx);
// No-allocation scratch of mm_apply_A_static (apply_static.cu): looks up the device
// address of the library's static array on the current device (called by mm_plan with
// the plan's device current) and returns it / its size.
void static_scratch_setup(int device);
void* static_scratch_ptr(int device);
size_t static_scratch_bytes();
void note_launch(int kernels = 1);                   // process-wide kernel launch counter

// Launch with programmatic dependent launch: the kernel may be scheduled before the
// previous kernel in the stream has finished, and must execute griddep_wait() before it
// reads anything that kernel wrote (the wait returns once that kernel has completed and
// its writes are visible).  Only kernels that wait first are launched this way.
template <typename... KA, typename... A>
void launch_pdl(void (*kern)(KA...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    check_cuda(cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...), "kernel launch (dependent)");
}

#ifdef __CUDACC__
// Wait for the kernel before this one in the stream (programmatic dependent launch);
// returns at once for a kernel launched the ordinary way.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif
void* dmalloc(size_t bytes);                         // throws Error{MM_ERR_OOM}
void dfree(void* p);

// host numerics (plan.cpp) -------------------------------------------------------------
void host_fft(std::vector<double>& re, std::vector<double>& im, bool inverse);
std::vector<double> toeplitz_row(double sigma, double fknee, double alpha, int64_t L,
                                 double fsamp, int lam, int window);
bool symbol_positive(const std::vector<double>& t);
std::vector<std::vector<double>> toeplitz_row_derivatives(double sigma, double fknee, double alpha, int64_t L,
                                                          double fsamp, int lam, int window);
std::vector<double> overlap_save_spectrum(const std::vector<double>& t, int64_t N);
// per-pass Stockham twiddles of an N = 2^logn point FFT as interleaved (cos, sin)
std::vector<double> pass_twiddle_table(int logn);
double rcond_sym3(const double B[6]);

// kernels (launchers) --------------------------------------------------------------------
// Toeplitz overlap-save (toeplitz_f64.cu / toeplitz_f32.cu)
template <typename T>
void launch_toeplitz(const Plan& P, const ToeplitzDev& tz, const T* y_tod, const T* x_map,
                     T* z, const int* done, cudaStream_t s);
// R right-hand sides in one launch: RHS r reads y_tod + r in_stride (or x_map + r in_stride)
// and writes z + r out_stride
template <typename T>
void launch_toeplitz_rhs(const Plan& P, const ToeplitzDev& tz, const T* y_tod, const T* x_map, int R,
                         int64_t in_stride, T* z, int64_t out_stride, const int* done, cudaStream_t s);
// General form: d_tod (FP64 time domain) alone is rounded to T (FP32 only); with x_map the
// input is d - P x (FP64 only: the residual data of b - A x).
template <typename T>
void launch_toeplitz_any(const Plan& P, const ToeplitzDev& tz, const T* y_tod, const double* d_tod, const T* x_map,
                         int R, int64_t in_stride, T* z, int64_t out_stride, const int* done, cudaStream_t s);
// Double-float N^-1 on FP64 data (toeplitz_df.cu): y (time domain) given, or else the
// residual data d - P x; output z FP64 [nt] (R right-hand sides as for launch_toeplitz_rhs)
void launch_toeplitz_df(const Plan& P, const double* y, const double* d, const double* x, int R, int64_t in_stride,
                        double* z, int64_t out_stride, cudaStream_t s);
// FP32 I/Q/U N^-1 P x with the gather reading x from P.map4; pack: first write x into
// P.map4 (one small kernel), else P.map4 already holds x (the FP32 PCG kernels keep it)
void launch_toeplitz_f32_packed(const Plan& P, const float* x, bool pack, float* z, const int* done,
                                cudaStream_t s);
template <typename T>
size_t toeplitz_smem_bytes(int logn);
template <typename T>
int toeplitz_max_logn();          // largest single-CTA FFT (the cluster kernels add one or two)

// pointing (pointing.cu)
template <typename T>
void launch_gather(const Plan& P, const T* x, T* y, cudaStream_t s);
template <typename T>
void launch_scatter(const Plan& P, const T* z, T* w, const int* done, cudaStream_t s);
// w = P^T z and, fused, *pq = p^T w (FP64, fixed summation order: warp partials over their
// pixels, block partials in part[], summed in block order by the last block to finish,
// which also resets *count to 0).  part holds scatter_blocks(P) doubles.
template <typename T>
void launch_scatter_dot(const Plan& P, const T* z, T* w, const T* p, double* part, unsigned* count, double* pq,
                        const int* done, cudaStream_t s);
int scatter_blocks(const Plan& P);
void launch_bd_build(const Plan& P, double* bd64, float* bd32, cudaStream_t s);
// merged a priori coarse space Z_S (Sec. 3.3.1), r groups of consecutive intervals, into
// Z [r][n] FP64 (zeroed here)
void launch_apriori(const Plan& P, int r, double* Z, cudaStream_t s);
template <typename T>
void launch_bd_apply(const Plan& P, const T* r, T* z, cudaStream_t s);
void launch_angles(const double2* w, float* ang, int64_t n, unsigned* bad, cudaStream_t s);
void launch_convert_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
void launch_convert_f32_to_f64(const float* a, double* b, int64_t n, cudaStream_t s);
// gradient helpers (grad.cu)
void launch_sub_time(const double* a, const double* b, double* out, int64_t n, cudaStream_t s);
void launch_interval_dot(const double* u, const double* w, const int64_t* ioff, int K, double* part,
                         cudaStream_t s);

}  // namespace mm
