// C-ABI entry points of libmm (declared in include/mm.h) and the host drivers behind
// them: plan construction (Sec. 2 observed pixels, Eq. 4 / App. D Toeplitz rows,
// overlap-save tiling and its block choice, Eq. 10 M_BD), operator applications
// (Eq. 5-8), the PCG driver (Sec. 3.1) with FP64 or mixed arithmetic plus iterative
// refinement and its residual history (Sec. 5.1), the coarse spaces (a posteriori from
// CG-Lanczos or Arnoldi, Sec. 3.3.2 and App. A; a priori, Sec. 3.3.1; imported), the
// A-DEF2 start (App. B), the adjoint and PSD gradients, and the batched solver.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <set>
#include <utility>

#include "coarse.cuh"
#include "coarse_host.h"
#include "dfloat.cuh"
#include "mm_internal.h"
#include "pcg.cuh"
#include "batch.cuh"

namespace mm {

static thread_local std::string g_last_error = "no error";
static std::atomic<int64_t> g_launches{0};

void note_launch(int kernels) { g_launches.fetch_add(kernels, std::memory_order_relaxed); }

void check_cuda(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        throw Error{MM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e)};
    }
}

void ensure_smem_attr(const void* kern, int bytes, const char* what) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;   // (kernel, device)
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kern, dev})) return;
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes), what);
    done.insert({kern, dev});
}

void* dmalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error{e == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
    }
    return p;
}

void dfree(void* p) {
    if (p != nullptr) (void)cudaFree(p);
}

template <typename T>
static T* dalloc(size_t count) { return static_cast<T*>(dmalloc(count * sizeof(T))); }

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static void h2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes) check_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s), "memcpy H2D");
}
static void d2h(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (bytes) check_cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s), "memcpy D2H");
}
static void sync(cudaStream_t s) { check_cuda(cudaStreamSynchronize(s), "stream synchronize"); }
static void sync(Plan& P) {
    sync(P.stream);
    if (P.prof.on) prof_flush(P);
}

// ------------------------------------------------------------------------ profiling
int prof_begin(Plan& P, int stage) {
    if (!P.prof.on) return -1;
    cudaEvent_t ev[2];
    for (int i = 0; i < 2; ++i) {
        if (!P.prof.pool.empty()) {
            ev[i] = P.prof.pool.back();
            P.prof.pool.pop_back();
        } else {
            check_cuda(cudaEventCreate(&ev[i]), "event");
        }
    }
    check_cuda(cudaEventRecord(ev[0], P.stream), "event record");
    P.prof.pending.push_back({stage, ev[0], ev[1]});
    return (int)P.prof.pending.size() - 1;
}

void prof_end(Plan& P, int slot) {
    if (slot < 0) return;
    check_cuda(cudaEventRecord(P.prof.pending[(size_t)slot].b, P.stream), "event record");
}

void prof_flush(Plan& P) {
    for (auto& e : P.prof.pending) {
        float ms = 0.f;
        check_cuda(cudaEventElapsedTime(&ms, e.a, e.b), "event elapsed");
        P.prof.ms[e.stage] += ms;
        P.prof.launches[e.stage] += 1;
        P.prof.pool.push_back(e.a);
        P.prof.pool.push_back(e.b);
    }
    P.prof.pending.clear();
}

// ----------------------------------------------------------------------------- plan
// Buffers of the batched (many right-hand sides) solver, allocated on first use.
enum { BATCH_PAIR = 0, BATCH_REAL = 1, BATCH_TENSOR = 2 };

struct BatchState {
    int kind = -1;                // BATCH_PAIR / BATCH_REAL / BATCH_TENSOR, -1 before the first call
    float tuned_ms[3] = {};       // timed forms (autotuning), 0 when not timed
    int logb = 0;                 // complex FFT length of the pair kernel
    int ntiles = 0;
    SpanTile* tiles = nullptr;
    float* H = nullptr;           // [npsd][B/2 + 1] / B
    float* ptw = nullptr;         // per-pass FFT twiddles of the per-CTA transform
    float* twiddle = nullptr;     // cos(2 pi k / B), k = 0..B/4 (cluster blocks)
    int cap = 0;                  // right-hand sides the vectors below hold
    float *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *tod = nullptr;
    double *x64 = nullptr, *b64 = nullptr, *r64 = nullptr;
    double *partial = nullptr, *rho = nullptr, *bb = nullptr, *rr = nullptr, *tol2 = nullptr;
    int* iters = nullptr;
    unsigned char* state = nullptr;
    int* flags = nullptr;
    unsigned* bar = nullptr;
    int nblocks = 0;
    // tensor-core form (batch_tc.cu)
    SpanTile* tc_groups = nullptr;
    int tc_ngroups = 0;
    int tc_nchunk = 0;
    __half* tc_atab = nullptr;    // [npsd][nchunk][hi, lo][128 x 64] band chunks
    float* tc_invc = nullptr;     // [npsd]
    float* tc_y = nullptr;        // [cap][nt] P X
    float* tc_scale = nullptr;    // [2][BATCH_RMAX] column scales, inverses
    int tc_cap = 0;
    cudaGraphExec_t graph = nullptr;   // `graph_iters` batched iterations, or null
    int graph_R = -1;             // R and maxit the graph was captured with
    int graph_maxit = -1;
    bool graph_failed = false;
};

struct PlanHolder : Plan {
    BatchState batch;
    // grid-barrier settings of the PCG kernels: every solve waits for the launched blocks
    // with a 2 s limit per wait; mm_pcg_barrier_check changes them for one run
    unsigned bar_absent = 0;
    unsigned long long bar_wait_ns = BARRIER_WAIT_NS;
    std::vector<mm_psd> h_psd;
    double* grad_H = nullptr;   // [3][npsd][N+1] derivative spectra (FP64 block)
    double* grad_u = nullptr;   // [nt] P mu
    double* grad_part = nullptr;  // [K]
    int* h_flags = nullptr;     // pinned
    double* h_scal = nullptr;   // pinned
    double* d_dot = nullptr;    // [DOT_BLOCKS + 2]
    double* x64 = nullptr;      // [n] refinement iterate
    double* r64 = nullptr;      // [n] refinement residual
    double* ax64 = nullptr;     // [n]
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
    bool autotune = false;      // measured block / batched-kernel choice (mm_opts.autotune)
    float tuned_ms64[16] = {};  // timed candidates by logn - 8 (0: not tried)
    float tuned_ms32[16] = {};
    float tuned_scatter_ms[3] = {};   // FP32 scatter timed with 32, 16, 8 lanes per pixel
    // Residual history of the last solve: PCG run j wrote r^T r of its steps to
    // pcg.hist_rr[off ..]; relative residual = sqrt(rr / bb) * scale (mm_solve_history).
    // A run with bb = 0 took no step: its entry 0 is `scale` itself (the relative
    // residual of x_0 = 0: 0 for b = 0, else 1).
    struct HistRun {
        int off, iters;
        double bb, scale;
    };
    std::vector<HistRun> hist_runs;
};

static void free_tz(ToeplitzDev& t) {
    dfree(t.tiles);
    dfree(t.twiddle);
    dfree(t.ptw);
    dfree(t.H);
    t = ToeplitzDev{};
}

static void free_coarse(CoarseDev& c) {
    dfree(c.Z64);
    dfree(c.AZ64);
    dfree(c.Z32);
    dfree(c.AZ32);
    dfree(c.Einv);
    c = CoarseDev{};
}

static void destroy_plan(PlanHolder* P) {
    if (P == nullptr) return;
    for (void* p : {(void*)P->pixc, (void*)P->w64, (void*)P->w32, (void*)P->csr_off, (void*)P->tsort,
                    (void*)P->wsort64, (void*)P->wsort32, (void*)P->asort32, (void*)P->ioff, (void*)P->ipsd, (void*)P->t0,
                    (void*)P->bd64, (void*)P->bd32, (void*)P->tod64, (void*)P->tod32, (void*)P->map4, (void*)P->dbuf,
                    (void*)P->b64, (void*)P->d_dot, (void*)P->x64, (void*)P->r64, (void*)P->ax64,
                    (void*)P->grad_H, (void*)P->grad_u, (void*)P->grad_part})
        dfree(p);
    free_tz(P->tz64);
    free_tz(P->tz32);
    free_tz(P->tzdf);
    free_coarse(P->coarse);
    PcgDev& g = P->pcg;
    for (void* p : {(void*)g.partial, (void*)g.sc_part, (void*)g.sc_count, (void*)g.scal, (void*)g.flags,
                    (void*)g.barrier, g.x, g.r, g.p, g.q, g.z,
                    (void*)g.hist_alpha, (void*)g.hist_beta, (void*)g.hist_rz, (void*)g.hist_rr})
        dfree(p);
    if (P->h_flags) (void)cudaFreeHost(P->h_flags);
    if (P->h_scal) (void)cudaFreeHost(P->h_scal);
    if (P->ev0) (void)cudaEventDestroy(P->ev0);
    if (P->ev1) (void)cudaEventDestroy(P->ev1);
    if (P->ev2) (void)cudaEventDestroy(P->ev2);
    for (auto& e : P->prof.pending) {
        (void)cudaEventDestroy(e.a);
        (void)cudaEventDestroy(e.b);
    }
    for (auto e : P->prof.pool) (void)cudaEventDestroy(e);
    BatchState& bt = P->batch;
    if (bt.graph) (void)cudaGraphExecDestroy(bt.graph);
    for (void* p : {(void*)bt.tiles, (void*)bt.H, (void*)bt.ptw, (void*)bt.twiddle, (void*)bt.x, (void*)bt.r,
                    (void*)bt.p, (void*)bt.q, (void*)bt.z,
                    (void*)bt.tod, (void*)bt.x64, (void*)bt.b64, (void*)bt.r64, (void*)bt.partial, (void*)bt.rho,
                    (void*)bt.bb, (void*)bt.rr, (void*)bt.tol2, (void*)bt.iters, (void*)bt.state, (void*)bt.flags,
                    (void*)bt.bar, (void*)bt.tc_groups, (void*)bt.tc_atab, (void*)bt.tc_invc, (void*)bt.tc_y,
                    (void*)bt.tc_scale})
        dfree(p);
    delete P;
}

// Cost of a block relative to its FFT operation count, from launch timings of every
// admissible block on polarised scans of 2^24-2^25 samples with lambda = 1024, 4096,
// 8192 and 16384.  FP64 kernels are bound by the FP64 pipe, so the cross-CTA steps of a
// 2-CTA cluster cost little; the largest single-CTA FP64 block (2^14 reals) runs one
// 512-thread CTA per SM.  FP32 kernels are bound by shared-memory and L1 latency, where
// the cluster steps (distributed shared memory) cost more.  The batched complex-pair
// blocks are FP32 and take the FP32 weights by cluster size.
static double fp32_cluster_weight(int cluster) { return cluster == 4 ? 3.3 : (cluster == 2 ? 1.6 : 1.0); }
template <typename T>
static double block_weight(int logn);
template <>
double block_weight<double>(int logn) { return logn >= 15 ? 2.0 : (logn == 14 ? 1.2 : (logn == 13 ? 1.12 : 1.0)); }
// FP32 single-CTA blocks below 2^15 reals run several CTAs per SM (1024 threads in all),
// which hides part of their gathers: measured on the 2^24-sample I/Q/U scan at lambda =
// 512 .. 8192, their time per unit of the model falls with the block.
template <>
double block_weight<float>(int logn) {
    if (logn >= 15) return fp32_cluster_weight(logn >= 16 ? 4 : 2);
    return logn == 14 ? 1.0 : (logn == 13 ? 0.87 : (logn == 12 ? 0.83 : (logn == 11 ? 0.72 : 0.67)));
}

// Overlap-save tiles of blocks of B real positions (B - 2 lambda valid outputs each) for
// the single-right-hand-side kernels.  Consecutive stationary intervals with the same PSD
// form a run; a run is laid out as its intervals one after another with lambda zeros
// between them (so no band product reaches across an interval edge, Eq. 4) and tiled as
// one sequence, which saves the partly filled last tile of every interval but one.  A run
// is packed only when that gives fewer tiles and no tile needs more than TILE_SEGS
// segments; otherwise each interval is tiled on its own (one segment per tile).
static std::vector<Tile> make_tiles(const Plan& P, int64_t B) {
    const int64_t lam = P.lambda;
    const int64_t Lv = B - 2 * lam;
    std::vector<Tile> out;
    auto tile_run = [&](int i0, int i1, std::vector<Tile>& dst) -> bool {
        // virtual start of each interval of the run [i0, i1)
        std::vector<int64_t> V((size_t)(i1 - i0));
        int64_t vlen = 0;
        for (int i = i0; i < i1; ++i) {
            if (i > i0) vlen += lam;
            V[(size_t)(i - i0)] = vlen;
            vlen += P.h_ioff[i + 1] - P.h_ioff[i];
        }
        int first = 0;   // first interval that can still meet the current window
        for (int64_t k = 0; k * Lv < vlen; ++k) {
            const int64_t w0 = k * Lv - lam;   // virtual position of block position 0
            Tile t;
            for (int g = 0; g < TILE_SEGS; ++g) {
                t.d[g] = 0;
                t.pb[g] = t.pe[g] = TILE_NONE;
            }
            int ns = 0;
            while (first < i1 - i0 && V[(size_t)first] + (P.h_ioff[i0 + first + 1] - P.h_ioff[i0 + first]) <= w0) ++first;
            for (int j = first; j < i1 - i0; ++j) {
                const int64_t L = P.h_ioff[i0 + j + 1] - P.h_ioff[i0 + j];
                const int64_t a = std::max(V[(size_t)j], w0), b = std::min(V[(size_t)j] + L, w0 + B);
                if (V[(size_t)j] >= w0 + B) break;
                if (a >= b) continue;
                if (ns == TILE_SEGS) return false;
                t.pb[ns] = (int32_t)(a - w0);
                t.pe[ns] = (int32_t)(b - w0);
                t.d[ns] = P.h_ioff[i0 + j] + w0 - V[(size_t)j];   // time of block position p: p + d
                ++ns;
            }
            t.nout = (int32_t)std::min<int64_t>(Lv, vlen - k * Lv);
            t.psd = P.h_ipsd[i0];
            dst.push_back(t);
        }
        return true;
    };
    for (int i0 = 0; i0 < P.K;) {
        int i1 = i0 + 1;
        while (i1 < P.K && P.h_ipsd[i1] == P.h_ipsd[i0]) ++i1;
        std::vector<Tile> single, packed;
        for (int i = i0; i < i1; ++i) tile_run(i, i + 1, single);
        if (i1 - i0 > 1 && tile_run(i0, i1, packed) && packed.size() < single.size())
            out.insert(out.end(), packed.begin(), packed.end());
        else
            out.insert(out.end(), single.begin(), single.end());
        i0 = i1;
    }
    return out;
}

static int64_t overlap_tiles(const Plan& P, int64_t Lv) {
    return (int64_t)make_tiles(P, Lv + 2 * (int64_t)P.lambda).size();
}

// Tiles of the batched kernels: every interval on its own.
static int64_t interval_tiles(const Plan& P, int64_t Lv) {
    int64_t tiles = 0;
    for (int i = 0; i < P.K; ++i) tiles += (P.h_ioff[i + 1] - P.h_ioff[i] + Lv - 1) / Lv;
    return tiles;
}

// Admissible overlap-save blocks (B = 2^(logn+1) reals > 2 lambda) ordered by the cost
// model tiles x (N (logn + 1) + 2048) x block weight; the two blocks above the
// single-CTA maximum run on 2- and 4-CTA clusters.
template <typename T>
static std::vector<std::pair<double, int>> block_candidates(const Plan& P) {
    const int maxl = toeplitz_max_logn<T>();
    std::vector<std::pair<double, int>> c;
    for (int logn = 8; logn <= maxl + 2; ++logn) {
        const int64_t N = int64_t(1) << logn;
        const int64_t Lv = 2 * N - 2 * (int64_t)P.lambda;
        if (Lv < 1) continue;
        c.push_back({(double)overlap_tiles(P, Lv) * ((double)N * (logn + 1) + 2048.0) * block_weight<T>(logn), logn});
    }
    std::stable_sort(c.begin(), c.end());
    return c;
}

// Block choice: forced (log2 of the real block), else the cheapest candidate.  Returns
// logn; sets *cluster to 1, 2 or 4.
template <typename T>
static int choose_logn(const Plan& P, int forced_log2B, int* cluster) {
    const int maxl = toeplitz_max_logn<T>();
    int logn;
    if (forced_log2B > 0) {
        logn = forced_log2B - 1;
        if (logn < 8 || logn > maxl + 2) throw Error{MM_ERR_ARG, "fft block size out of range"};
        if ((int64_t(2) << logn) - 2 * (int64_t)P.lambda < 1) throw Error{MM_ERR_ARG, "fft block too short for lambda"};
    } else {
        const auto c = block_candidates<T>(P);
        if (c.empty()) throw Error{MM_ERR_ARG, "lambda too large for the largest FFT block"};
        logn = c[0].second;
    }
    *cluster = logn > maxl ? 1 << (logn - maxl) : 1;
    return logn;
}

template <typename T>
static void build_toeplitz(Plan& P, ToeplitzDev& tz, int forced_log2B) {
    tz.logn = choose_logn<T>(P, forced_log2B, &tz.cluster);
    const int64_t N = int64_t(1) << tz.logn;
    const int64_t B = 2 * N;
    const std::vector<Tile> tiles = make_tiles(P, B);
    tz.ntiles = (int)tiles.size();
    tz.tiles = dalloc<Tile>(tiles.size());
    h2d(tz.tiles, tiles.data(), tiles.size() * sizeof(Tile), P.stream);
    std::vector<T> tw((size_t)(B / 4 + 1));
    for (int64_t k = 0; k <= B / 4; ++k) tw[(size_t)k] = (T)std::cos(2.0 * 3.14159265358979323846 * (double)k / (double)B);
    tz.twiddle = dalloc<T>(tw.size());
    h2d(tz.twiddle, tw.data(), tw.size() * sizeof(T), P.stream);
    {
        // the cluster kernel runs local FFTs of half the length
        const int lc = tz.cluster == 4 ? 2 : (tz.cluster == 2 ? 1 : 0);
        const std::vector<double> pt = pass_twiddle_table(tz.logn - lc);
        std::vector<T> ptT(pt.begin(), pt.end());
        tz.ptw = dalloc<T>(ptT.size());
        h2d(tz.ptw, ptT.data(), ptT.size() * sizeof(T), P.stream);
        sync(P.stream);
    }
    std::vector<T> H((size_t)P.npsd * (N + 1));
    for (int p = 0; p < P.npsd; ++p) {
        const std::vector<double> h = overlap_save_spectrum(P.rows[(size_t)p], N);
        for (int64_t k = 0; k <= N; ++k) H[(size_t)p * (N + 1) + k] = (T)h[(size_t)k];
    }
    tz.H = dalloc<T>(H.size());
    h2d(tz.H, H.data(), H.size() * sizeof(T), P.stream);
    sync(P.stream);   // host vectors go out of scope
}

// Double-float tables on the blocks of the FP64 kernel (tz64, which must be final):
// its tiles copied, the cosine and per-pass twiddles and the kernel spectra rounded to
// double-float pairs (hi = FP32 rounding, lo = FP32 rounding of the rest).
static void build_toeplitz_df(Plan& P) {
    const ToeplitzDev& src = P.tz64;
    ToeplitzDev& tz = P.tzdf;
    free_tz(tz);
    tz = ToeplitzDev{};
    if (src.logn == 0) return;
    tz.logn = src.logn;
    tz.cluster = src.cluster;
    tz.ntiles = src.ntiles;
    const int64_t N = int64_t(1) << tz.logn;
    const int64_t B = 2 * N;
    try {
        tz.tiles = dalloc<Tile>((size_t)tz.ntiles);
        check_cuda(cudaMemcpyAsync(tz.tiles, src.tiles, (size_t)tz.ntiles * sizeof(Tile), cudaMemcpyDeviceToDevice,
                                   P.stream), "copy tiles");
        std::vector<dfl> tw((size_t)(B / 4 + 1));
        for (int64_t k = 0; k <= B / 4; ++k) tw[(size_t)k] = dfl(std::cos(2.0 * 3.14159265358979323846 * (double)k / (double)B));
        tz.twiddle = dalloc<dfl>(tw.size());
        h2d(tz.twiddle, tw.data(), tw.size() * sizeof(dfl), P.stream);
        const int lc = tz.cluster == 4 ? 2 : (tz.cluster == 2 ? 1 : 0);
        const std::vector<double> pt = pass_twiddle_table(tz.logn - lc);
        std::vector<dfl> ptd(pt.size());
        for (size_t i = 0; i < pt.size(); ++i) ptd[i] = dfl(pt[i]);
        tz.ptw = dalloc<dfl>(ptd.size());
        h2d(tz.ptw, ptd.data(), ptd.size() * sizeof(dfl), P.stream);
        std::vector<dfl> H((size_t)P.npsd * (N + 1));
        for (int p = 0; p < P.npsd; ++p) {
            const std::vector<double> h = overlap_save_spectrum(P.rows[(size_t)p], N);
            for (int64_t k = 0; k <= N; ++k) H[(size_t)p * (N + 1) + k] = dfl(h[(size_t)k]);
        }
        tz.H = dalloc<dfl>(H.size());
        h2d(tz.H, H.data(), H.size() * sizeof(dfl), P.stream);
        sync(P.stream);   // host vectors go out of scope
    } catch (...) {
        free_tz(tz);
        tz = ToeplitzDev{};
        throw;
    }
}

// Average milliseconds of `reps` launches of f on the plan's stream (one untimed first).
template <typename F>
static float time_launches(PlanHolder& P, F&& f, int reps) {
    f();
    check_cuda(cudaEventRecord(P.ev0, P.stream), "event");
    for (int i = 0; i < reps; ++i) f();
    check_cuda(cudaEventRecord(P.ev1, P.stream), "event");
    check_cuda(cudaEventSynchronize(P.ev1), "event sync");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, P.ev0, P.ev1), "event time");
    return ms / (float)reps;
}

// Measured block choice: the (up to) three cheapest candidates of the cost model are built
// and their de-pointing launch (the one inside A x) is timed on a zero map; the fastest
// stays in tz.  Timings go to tuned_ms (0 for candidates not tried).
template <typename T>
static void autotune_toeplitz(PlanHolder& P, ToeplitzDev& tz, T* tod, const T* zmap, float* tuned_ms) {
    const auto c = block_candidates<T>(P);
    if (c.size() < 2) return;
    float best_ms = 0.f;
    for (size_t i = 0; i < c.size() && i < 3; ++i) {
        ToeplitzDev cand;
        const bool fresh = c[i].second != tz.logn;
        float ms = 0.f;
        try {
            if (fresh) build_toeplitz<T>(P, cand, c[i].second + 1);
            else cand = tz;
            ms = time_launches(P, [&] { launch_toeplitz<T>(P, cand, nullptr, zmap, tod, nullptr, P.stream); }, 3);
        } catch (...) {
            if (fresh) free_tz(cand);   // a candidate built here and not kept
            throw;
        }
        tuned_ms[c[i].second - 8] = ms;
        if (cand.logn == tz.logn) {
            if (best_ms == 0.f || ms < best_ms) best_ms = ms;
            continue;
        }
        if (ms < best_ms || best_ms == 0.f) {
            free_tz(tz);
            tz = cand;
            best_ms = ms;
        } else {
            free_tz(cand);
        }
    }
}

static void build_plan(PlanHolder& P, const int32_t* pix, int64_t nt, int32_t npix_sky, const double* weights,
                       const int64_t* ioff, int32_t K, const int32_t* ipsd, const mm_psd* psd, int32_t npsd,
                       const mm_opts* o) {
    if (o == nullptr || pix == nullptr || ioff == nullptr || ipsd == nullptr || psd == nullptr)
        throw Error{MM_ERR_ARG, "null argument"};
    if (o->ncomp != 1 && o->ncomp != 3) throw Error{MM_ERR_ARG, "ncomp must be 1 or 3"};
    if ((o->ncomp == 3) != (weights != nullptr)) throw Error{MM_ERR_ARG, "weights required iff ncomp == 3"};
    if (nt < 1 || nt >= (int64_t(1) << 31)) throw Error{MM_ERR_ARG, "nt out of range"};
    if (npix_sky < 1 || K < 1 || npsd < 1) throw Error{MM_ERR_ARG, "npix_sky, K and npsd must be >= 1"};
    if (!(o->fsamp > 0.0)) throw Error{MM_ERR_ARG, "fsamp must be > 0"};
    if (o->window != MM_WINDOW_GAUSS && o->window != MM_WINDOW_RECT) throw Error{MM_ERR_ARG, "bad window"};
    if (o->lambda < 0) throw Error{MM_ERR_ARG, "lambda must be >= 0"};
    P.nt = nt;
    P.npix_sky = npix_sky;
    P.ncomp = o->ncomp;
    P.K = K;
    P.npsd = npsd;
    P.lambda = o->lambda;
    P.window = o->window;
    P.fsamp = o->fsamp;
    P.rcond_min = o->rcond_min > 0.0 ? o->rcond_min : 1e-6;
    P.stream = static_cast<cudaStream_t>(o->stream);
    P.h_ioff.assign(ioff, ioff + K + 1);
    P.h_psd.assign(psd, psd + npsd);
    P.h_ipsd.assign(ipsd, ipsd + K);
    if (P.h_ioff[0] != 0 || P.h_ioff[(size_t)K] != nt) throw Error{MM_ERR_ARG, "interval offsets must span [0, nt)"};
    int64_t minlen = nt, maxlen = 0;
    for (int i = 0; i < K; ++i) {
        const int64_t len = P.h_ioff[i + 1] - P.h_ioff[i];
        if (len <= 0) throw Error{MM_ERR_ARG, "interval offsets must increase strictly"};
        minlen = std::min(minlen, len);
        maxlen = std::max(maxlen, len);
        if (P.h_ipsd[i] < 0 || P.h_ipsd[i] >= npsd) throw Error{MM_ERR_ARG, "interval psd id out of range"};
    }
    if ((int64_t)P.lambda >= minlen) throw Error{MM_ERR_ARG, "lambda must be < the shortest interval"};
    for (int p = 0; p < npsd; ++p) {
        if (!(psd[p].sigma > 0.0) || !(psd[p].fknee >= 0.0) || !(psd[p].alpha > 0.0) || !std::isfinite(psd[p].sigma) ||
            !std::isfinite(psd[p].fknee) || !std::isfinite(psd[p].alpha))
            throw Error{MM_ERR_ARG, "psd parameters must be sigma > 0, fknee >= 0, alpha > 0"};
    }
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    P.device = dev;
    check_cuda(cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    // the no-allocation A x (mm_apply_A_static) finds its scratch address set up here
    static_scratch_setup(dev);

    // --- host copies of the pointing
    std::vector<int32_t> hpix((size_t)nt);
    std::vector<double> hw;
    if (is_device_ptr(pix)) {
        check_cuda(cudaMemcpy(hpix.data(), pix, (size_t)nt * 4, cudaMemcpyDeviceToHost), "copy pix");
    } else {
        std::memcpy(hpix.data(), pix, (size_t)nt * 4);
    }
    if (P.ncomp == 3) {
        hw.resize((size_t)nt * 2);
        if (is_device_ptr(weights))
            check_cuda(cudaMemcpy(hw.data(), weights, (size_t)nt * 16, cudaMemcpyDeviceToHost), "copy weights");
        else
            std::memcpy(hw.data(), weights, (size_t)nt * 16);
    }
    // --- observed pixels (reading: hits >= 1, or hits >= 3 and well-conditioned I/Q/U block)
    std::vector<int32_t> hits_sky((size_t)npix_sky, 0);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t p = hpix[(size_t)t];
        if (p < 0 || p >= npix_sky) throw Error{MM_ERR_ARG, "pixel index out of range"};
        ++hits_sky[(size_t)p];
    }
    std::vector<char> obs((size_t)npix_sky, 0);
    if (P.ncomp == 1) {
        for (int32_t p = 0; p < npix_sky; ++p) obs[(size_t)p] = hits_sky[(size_t)p] >= 1;
    } else {
        std::vector<double> Bs((size_t)npix_sky * 6, 0.0);
        for (int64_t t = 0; t < nt; ++t) {
            double* b = &Bs[(size_t)hpix[(size_t)t] * 6];
            const double c = hw[(size_t)t * 2], s = hw[(size_t)t * 2 + 1];
            b[0] += 1.0;
            b[1] += c;
            b[2] += s;
            b[3] += c * c;
            b[4] += c * s;
            b[5] += s * s;
        }
        for (int32_t p = 0; p < npix_sky; ++p)
            obs[(size_t)p] = hits_sky[(size_t)p] >= 3 && rcond_sym3(&Bs[(size_t)p * 6]) >= P.rcond_min;
    }
    std::vector<int32_t> sky2obs((size_t)npix_sky, -1);
    for (int32_t p = 0; p < npix_sky; ++p) {
        if (obs[(size_t)p]) {
            sky2obs[(size_t)p] = (int32_t)P.h_obs2sky.size();
            P.h_obs2sky.push_back(p);
            P.h_hits.push_back(hits_sky[(size_t)p]);
        }
    }
    P.npix_obs = (int32_t)P.h_obs2sky.size();
    P.n = (int64_t)P.npix_obs * P.ncomp;
    std::vector<int32_t> pixc((size_t)nt);
    for (int64_t t = 0; t < nt; ++t) pixc[(size_t)t] = sky2obs[(size_t)hpix[(size_t)t]];
    // --- pixel-sorted CSR (stable: ascending sample index inside each pixel)
    std::vector<int32_t> off((size_t)P.npix_obs + 1, 0);
    for (int32_t q = 0; q < P.npix_obs; ++q) off[(size_t)q + 1] = off[(size_t)q] + P.h_hits[(size_t)q];
    P.nkept = off[(size_t)P.npix_obs];
    std::vector<int32_t> tsort((size_t)P.nkept);
    std::vector<double> wsort(P.ncomp == 3 ? (size_t)P.nkept * 2 : 0);
    {
        std::vector<int32_t> pos(off.begin(), off.end() - 1);
        for (int64_t t = 0; t < nt; ++t) {
            const int32_t q = pixc[(size_t)t];
            if (q < 0) continue;
            const int32_t j = pos[(size_t)q]++;
            tsort[(size_t)j] = (int32_t)t;
            if (P.ncomp == 3) {
                wsort[(size_t)j * 2] = hw[(size_t)t * 2];
                wsort[(size_t)j * 2 + 1] = hw[(size_t)t * 2 + 1];
            }
        }
    }
    // --- Toeplitz rows (reading R1-R4)
    int64_t L = 1;
    while (L < maxlen) L *= 2;
    if (L < 2) L = 2;
    P.L_grid = L;
    P.rows.resize((size_t)npsd);
    std::vector<double> t0((size_t)npsd);
    for (int p = 0; p < npsd; ++p) {
        P.rows[(size_t)p] = toeplitz_row(psd[p].sigma, psd[p].fknee, psd[p].alpha, L, P.fsamp, P.lambda, P.window);
        if (!symbol_positive(P.rows[(size_t)p])) throw Error{MM_ERR_NOT_SPD, "Toeplitz row " + std::to_string(p) + " is not positive definite"};
        t0[(size_t)p] = P.rows[(size_t)p][0];
    }
    // --- device buffers
    cudaStream_t s = P.stream;
    P.pixc = dalloc<int32_t>((size_t)nt);
    h2d(P.pixc, pixc.data(), (size_t)nt * 4, s);
    P.csr_off = dalloc<int32_t>(off.size());
    h2d(P.csr_off, off.data(), off.size() * 4, s);
    P.tsort = dalloc<int32_t>((size_t)P.nkept);
    h2d(P.tsort, tsort.data(), (size_t)P.nkept * 4, s);
    if (P.ncomp == 3) {
        P.w64 = dalloc<double2>((size_t)nt);
        h2d(P.w64, hw.data(), (size_t)nt * 16, s);
        P.w32 = dalloc<float2>((size_t)nt);
        launch_convert_f64_to_f32(reinterpret_cast<const double*>(P.w64), reinterpret_cast<float*>(P.w32), nt * 2, s);
        P.wsort64 = dalloc<double2>((size_t)P.nkept);
        h2d(P.wsort64, wsort.data(), (size_t)P.nkept * 16, s);
        P.wsort32 = dalloc<float2>((size_t)P.nkept);
        launch_convert_f64_to_f32(reinterpret_cast<const double*>(P.wsort64), reinterpret_cast<float*>(P.wsort32),
                                  P.nkept * 2, s);
        // unit-norm weights (cos 2 psi, sin 2 psi): the FP32 scatter forms them from the
        // angle, (cos pi a, sin pi a) with a = atan2(w2, w1) / pi rounded to FP32, which
        // halves its weight bytes (the weight is then within ~2e-7 of the FP64 pair)
        if (P.nkept > 0) {
            P.asort32 = dalloc<float>((size_t)P.nkept);
            std::unique_ptr<unsigned, void (*)(unsigned*)> bad(dalloc<unsigned>(1), [](unsigned* q) { dfree(q); });
            check_cuda(cudaMemsetAsync(bad.get(), 0, 4, s), "memset");
            launch_angles(P.wsort64, P.asort32, P.nkept, bad.get(), s);
            unsigned hbad = 1;
            check_cuda(cudaMemcpyAsync(&hbad, bad.get(), 4, cudaMemcpyDeviceToHost, s), "angle check");
            check_cuda(cudaStreamSynchronize(s), "angle check");
            if (hbad != 0) {
                dfree(P.asort32);
                P.asort32 = nullptr;
            }
        }
    }
    P.ioff = dalloc<int64_t>((size_t)K + 1);
    h2d(P.ioff, P.h_ioff.data(), ((size_t)K + 1) * 8, s);
    P.ipsd = dalloc<int32_t>((size_t)K);
    h2d(P.ipsd, P.h_ipsd.data(), (size_t)K * 4, s);
    P.t0 = dalloc<double>((size_t)npsd);
    h2d(P.t0, t0.data(), (size_t)npsd * 8, s);
    // A precision whose largest block cannot hold the band is left unbuilt (logn = 0):
    // its operators then fail with MM_ERR_ARG; at least one precision must exist.
    for (int prec = 0; prec < 2; ++prec) {
        try {
            if (prec == 0) build_toeplitz<double>(P, P.tz64, o->fft_log2_f64);
            else build_toeplitz<float>(P, P.tz32, o->fft_log2_f32);
        } catch (const Error& e) {
            const bool forced = prec == 0 ? o->fft_log2_f64 > 0 : o->fft_log2_f32 > 0;
            if (e.st != MM_ERR_ARG || forced) throw;
            (prec == 0 ? P.tz64 : P.tz32) = ToeplitzDev{};
        }
    }
    if (P.tz64.logn == 0 && P.tz32.logn == 0) throw Error{MM_ERR_ARG, "lambda too large for every FFT block"};
    // M_BD (Eq. 10)
    const size_t bdn = (size_t)P.npix_obs * (P.ncomp == 3 ? 6 : 1);
    P.bd64 = dalloc<double>(bdn);
    P.bd32 = dalloc<float>(bdn);
    launch_bd_build(P, P.bd64, P.bd32, s);
    // scratch
    P.tod64 = dalloc<double>((size_t)nt);
    P.tod32 = dalloc<float>((size_t)nt);
    if (P.ncomp == 3) P.map4 = dalloc<float4>((size_t)std::max(P.npix_obs, 1));
    P.dbuf = dalloc<double>((size_t)nt);
    P.b64 = dalloc<double>((size_t)P.n);
    P.x64 = dalloc<double>((size_t)P.n);
    P.r64 = dalloc<double>((size_t)P.n);
    P.ax64 = dalloc<double>((size_t)P.n);
    P.d_dot = dalloc<double>(DOT_BLOCKS + 4);
    // PCG state
    PcgDev& g = P.pcg;
    g.n = P.n;
    g.nblocks = std::max(1, std::min(pcg_max_blocks(P.num_sms), (P.npix_obs + 31) / 32));
    g.partial = dalloc<double>((size_t)g.nblocks * PSTRIDE);
    g.sc_part = dalloc<double>((size_t)scatter_blocks(P));   // 32 lanes per pixel: the most blocks
    g.sc_count = dalloc<unsigned>(1);
    check_cuda(cudaMemsetAsync(g.sc_count, 0, 4, s), "memset");
    g.scal = dalloc<double>(16);
    g.flags = dalloc<int>(8);
    g.barrier = dalloc<unsigned>(4);
    check_cuda(cudaMemsetAsync(g.barrier, 0, 16, s), "memset");
    check_cuda(cudaMemsetAsync(g.flags, 0, 32, s), "memset");
    for (void** v : {&g.x, &g.r, &g.p, &g.q, &g.z}) *v = dmalloc((size_t)P.n * 8);
    check_cuda(cudaMallocHost(&P.h_flags, 64), "cudaMallocHost");
    check_cuda(cudaMallocHost(&P.h_scal, 16 * 8), "cudaMallocHost");
    check_cuda(cudaEventCreate(&P.ev0), "event");
    check_cuda(cudaEventCreate(&P.ev1), "event");
    check_cuda(cudaEventCreate(&P.ev2), "event");
    P.autotune = o->autotune != 0;
    if (o->scatter_lanes != 0) {
        if (o->scatter_lanes != 32 && o->scatter_lanes != 16 && o->scatter_lanes != 8)
            throw Error{MM_ERR_ARG, "scatter_lanes must be 0, 32, 16 or 8"};
        P.scatter_lpp = o->scatter_lanes;
    }
    if (P.autotune) {
        // zero maps for the timed launches (x64 / the first half of r64 as FP32)
        check_cuda(cudaMemsetAsync(P.x64, 0, (size_t)P.n * 8, s), "memset");
        if (P.tz64.logn != 0 && o->fft_log2_f64 <= 0) autotune_toeplitz<double>(P, P.tz64, P.tod64, P.x64, P.tuned_ms64);
        if (P.tz32.logn != 0 && o->fft_log2_f32 <= 0)
            autotune_toeplitz<float>(P, P.tz32, P.tod32, reinterpret_cast<const float*>(P.x64), P.tuned_ms32);
        // the pixel tile of the scatter: lanes per observed pixel, timed on the FP32
        // scatter of a zero time-domain array (its cost does not depend on the values)
        if (P.npix_obs > 0 && o->scatter_lanes == 0) {
            check_cuda(cudaMemsetAsync(P.tod32, 0, (size_t)P.nt * 4, s), "memset");
            const int lpp[3] = {32, 16, 8};
            int best = 0;
            for (int i = 0; i < 3; ++i) {
                P.scatter_lpp = lpp[i];
                P.tuned_scatter_ms[i] = time_launches(
                    P, [&] { launch_scatter<float>(P, P.tod32, reinterpret_cast<float*>(P.r64), nullptr, s); }, 5);
                if (P.tuned_scatter_ms[i] < P.tuned_scatter_ms[best]) best = i;
            }
            P.scatter_lpp = lpp[best];
        }
    }
    build_toeplitz_df(P);
    sync(s);
}

// -------------------------------------------------------------------- operators
template <typename T> static const ToeplitzDev& tz_of(const Plan& P);
template <> const ToeplitzDev& tz_of<double>(const Plan& P) { return P.tz64; }
template <> const ToeplitzDev& tz_of<float>(const Plan& P) { return P.tz32; }
template <typename T> static T* tod_of(Plan& P);
template <> double* tod_of<double>(Plan& P) { return P.tod64; }
template <> float* tod_of<float>(Plan& P) { return P.tod32; }
template <typename T> static const T* bd_ptr(const Plan& P);
template <> const double* bd_ptr<double>(const Plan& P) { return P.bd64; }
template <> const float* bd_ptr<float>(const Plan& P) { return P.bd32; }

// y = A x = P^T N^-1 P x, de-pointing fused into the Toeplitz tile load (Eq. 8).
template <typename T>
static void apply_A(Plan& P, const T* x, T* y, const int* done) {
    const bool f64 = sizeof(T) == 8;
    int s0 = prof_begin(P, f64 ? ST_TZ64 : ST_TZ32);
    if constexpr (sizeof(T) == 4) {
        if (P.map4 != nullptr) launch_toeplitz_f32_packed(P, x, true, tod_of<T>(P), done, P.stream);
        else launch_toeplitz<T>(P, tz_of<T>(P), nullptr, x, tod_of<T>(P), done, P.stream);
    } else {
        launch_toeplitz<T>(P, tz_of<T>(P), nullptr, x, tod_of<T>(P), done, P.stream);
    }
    prof_end(P, s0);
    s0 = prof_begin(P, f64 ? ST_SC64 : ST_SC32);
    launch_scatter<T>(P, tod_of<T>(P), y, done, P.stream);
    prof_end(P, s0);
}

// ---------------------------------------------------------------------------- PCG
struct PcgOutcome {
    int iters = 0;
    int status = MM_OK;
    double rr = 0.0, bb = 0.0;
};

// Coarse mode of the PCG kernels for a preconditioner kind: 0 M_BD, 1 M_2lvl, 2 A-DEF2.
static int coarse_mode(int kind) { return kind == MM_PREC_BD ? 0 : (kind == MM_PREC_TWOLEVEL ? 1 : 2); }

template <typename T>
static PcgArgs<T> pcg_args(PlanHolder& P, bool two, int maxit) {
    PcgArgs<T> a{};
    PcgDev& g = P.pcg;
    a.n = P.n;
    a.npix = P.npix_obs;
    a.maxit = maxit;
    a.x = static_cast<T*>(g.x);
    a.r = static_cast<T*>(g.r);
    a.p = static_cast<T*>(g.p);
    if constexpr (sizeof(T) == 4) a.p4 = P.map4;   // p also kept packed for the gather
    a.q = static_cast<T*>(g.q);
    a.z = static_cast<T*>(g.z);
    a.bd = bd_ptr<T>(P);
    if (two) {
        a.k = P.coarse.k;
        if constexpr (sizeof(T) == 8) {
            a.Z = reinterpret_cast<const T*>(P.coarse.Z64);
            a.AZ = reinterpret_cast<const T*>(P.coarse.AZ64);
        } else {
            a.Z = reinterpret_cast<const T*>(P.coarse.Z32);
            a.AZ = reinterpret_cast<const T*>(P.coarse.AZ32);
        }
        a.Einv = P.coarse.Einv;
    }
    a.partial = g.partial;
    a.scal = g.scal;
    a.flags = g.flags;
    a.bar = g.barrier;
    a.bar_absent = P.bar_absent;
    a.wait_ns = P.bar_wait_ns;
    a.hist_alpha = g.hist_alpha;
    a.hist_beta = g.hist_beta;
    a.hist_rz = g.hist_rz;
    a.hist_rr = g.hist_rr;
    a.maxhist = g.maxhist;
    return a;
}

// Runs PCG on the right-hand side already stored in pcg.r (as T); solution in pcg.x.
// The scalar history of this run goes to the history arrays from entry hist_off on.
template <typename T>
static PcgOutcome run_pcg(PlanHolder& P, int cm, double tol, int maxit, T* zstore, int maxstore,
                          int hist_off = 0) {
    cudaStream_t s = P.stream;
    PcgArgs<T> a = pcg_args<T>(P, cm != 0, maxit);
    a.zstore = zstore;
    a.maxstore = maxstore;
    if (a.hist_rr != nullptr) {
        if (hist_off >= a.maxhist) {
            a.hist_alpha = a.hist_beta = a.hist_rz = a.hist_rr = nullptr;
            a.maxhist = 0;
        } else {
            a.hist_alpha += hist_off;
            a.hist_beta += hist_off;
            a.hist_rz += hist_off;
            a.hist_rr += hist_off;
            a.maxhist -= hist_off;
        }
    }
    P.h_scal[0] = tol * tol;
    h2d(P.pcg.scal + SC_TOL2, P.h_scal, 8, s);
    const int nb = P.pcg.nblocks;
    // a barrier that timed out keeps partial arrivals: start every run from zero
    check_cuda(cudaMemsetAsync(P.pcg.barrier, 0, sizeof(unsigned), s), "memset barrier");
    launch_pcg<T>(0, P.ncomp, cm, a, nb, s);
    int launched = 0;
    PcgOutcome out;
    while (true) {
        // poll the done flag, the step count and the residual; launch as many steps as the
        // residual's average decay so far predicts are left (one more for margin, 2..16;
        // 4 before any step): a step launched after convergence exits at once, a poll
        // costs a host round trip
        d2h(P.h_flags, P.pcg.flags, 16, s);
        d2h(P.h_scal + 4, P.pcg.scal, 4 * 8, s);
        sync(P);
        if (P.h_flags[F_DONE]) break;
        if (launched >= maxit) break;   // defensive: device counter stops at maxit
        int chunk = 4;
        const int done_steps = P.h_flags[F_ITER];
        const double rr = P.h_scal[4 + SC_RR], bb0 = P.h_scal[4 + SC_BB], tol2 = P.h_scal[4 + SC_TOL2];
        if (done_steps >= 2 && rr > 0.0 && bb0 > 0.0 && rr < bb0 && tol2 > 0.0) {
            const double rate = std::log(rr / bb0) / done_steps;   // < 0
            const double left = std::log(tol2 * bb0 / rr) / rate;
            chunk = left <= 0.0 ? 2 : (int)std::min(16.0, std::max(2.0, std::ceil(left) + 1.0));
        }
        const int c = std::min(chunk, maxit - launched + 1);
        for (int i = 0; i < c; ++i) {
            // q = A p with p^T q fused into the scatter (scal[SC_PQ])
            const bool f64 = sizeof(T) == 8;
            int sl = prof_begin(P, f64 ? ST_TZ64 : ST_TZ32);
            if (sizeof(T) == 4 && a.p4 != nullptr)
                launch_toeplitz_f32_packed(P, reinterpret_cast<const float*>(a.p), false,
                                           reinterpret_cast<float*>(tod_of<T>(P)), P.pcg.flags + F_DONE, s);
            else
                launch_toeplitz<T>(P, tz_of<T>(P), nullptr, a.p, tod_of<T>(P), P.pcg.flags + F_DONE, s);
            prof_end(P, sl);
            sl = prof_begin(P, f64 ? ST_SC64 : ST_SC32);
            launch_scatter_dot<T>(P, tod_of<T>(P), static_cast<T*>(P.pcg.q), a.p, P.pcg.sc_part, P.pcg.sc_count,
                                  P.pcg.scal + SC_PQ, P.pcg.flags + F_DONE, s);
            prof_end(P, sl);
            sl = prof_begin(P, f64 ? ST_PCG64 : ST_PCG32);
            launch_pcg<T>(1, P.ncomp, cm, a, nb, s);
            prof_end(P, sl);
        }
        launched += c;
    }
    d2h(P.h_scal + 4, P.pcg.scal, 4 * 8, s);
    sync(P);
    out.iters = P.h_flags[F_ITER];
    out.status = P.h_flags[F_STATUS];
    out.rr = P.h_scal[4 + SC_RR];
    out.bb = P.h_scal[4 + SC_BB];
    if (out.status == MM_ERR_TIMEOUT) throw Error{MM_ERR_TIMEOUT, "grid barrier wait ran out"};
    return out;
}

static double dot64(PlanHolder& P, const double* a, const double* b) {
    launch_dot64(a, b, P.n, P.d_dot, P.d_dot + DOT_BLOCKS, P.stream);
    d2h(P.h_scal + 8, P.d_dot + DOT_BLOCKS, 8, P.stream);
    sync(P.stream);
    return P.h_scal[8];
}

// ------------------------------------------------------------------- coarse space
constexpr int MAX_HISTORY = 1 << 20;   // residual-history entries kept for a solve

static void ensure_history(PlanHolder& P, int m) {
    PcgDev& g = P.pcg;
    if (g.maxhist >= m + 1) return;
    dfree(g.hist_alpha);
    dfree(g.hist_beta);
    dfree(g.hist_rz);
    dfree(g.hist_rr);
    g.hist_alpha = g.hist_beta = g.hist_rz = g.hist_rr = nullptr;
    g.maxhist = 0;
    g.hist_alpha = dalloc<double>((size_t)m + 1);
    g.hist_beta = dalloc<double>((size_t)m + 1);
    g.hist_rz = dalloc<double>((size_t)m + 1);
    g.hist_rr = dalloc<double>((size_t)m + 1);
    g.maxhist = m + 1;
}

static std::vector<double> gram_host(PlanHolder& P, const double* A, int ka, const double* B, int kb) {
    double* part = dalloc<double>((size_t)GRAM_BLOCKS * ka * kb);
    std::vector<double> hp((size_t)GRAM_BLOCKS * ka * kb);
    try {
        const int nb = launch_gram(A, ka, B, kb, P.n, part, P.stream);
        d2h(hp.data(), part, hp.size() * 8, P.stream);
        sync(P.stream);
        dfree(part);
        std::vector<double> G((size_t)ka * kb, 0.0);
        for (int b = 0; b < nb; ++b)
            for (int i = 0; i < ka * kb; ++i) G[(size_t)i] += hp[(size_t)b * ka * kb + i];
        return G;
    } catch (...) {
        dfree(part);
        throw;
    }
}

// Takes Z (FP64 [k][n], device, ownership passes here), forms AZ = A Z (FP64),
// E = Z^T A Z (symmetrised), its Cholesky factor and E^-1 = L^-T L^-1 (FP64: inside PCG
// the coarse solve is then one k x k matvec spread over the block instead of two
// sequential triangular solves in one warp), and the FP32 copies of Z and AZ (App. C,
// "Constructing").  P.coarse is replaced only when every step succeeded.
static void install_coarse(PlanHolder& P, double* Z, int k, std::vector<double> ritz) {
    cudaStream_t s = P.stream;
    CoarseDev cd;
    cd.k = k;
    cd.ritz = std::move(ritz);
    cd.Z64 = Z;
    try {
        cd.AZ64 = dalloc<double>((size_t)k * P.n);
        for (int j = 0; j < k; ++j) apply_A<double>(P, cd.Z64 + (size_t)j * P.n, cd.AZ64 + (size_t)j * P.n, nullptr);
        std::vector<double> E = gram_host(P, cd.Z64, k, cd.AZ64, k);
        for (double v : E)
            if (!std::isfinite(v)) throw Error{MM_ERR_NUMERIC, "coarse vectors hold NaN or Inf"};
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < i; ++j) {
                const double v = 0.5 * (E[(size_t)i * k + j] + E[(size_t)j * k + i]);
                E[(size_t)i * k + j] = E[(size_t)j * k + i] = v;
            }
        std::vector<double> Lf, Einv;
        if (cholesky_lower(E, k, Lf)) {
            Einv = spd_inverse_from_cholesky(Lf, k);
        } else {
            // E is SPD in exact arithmetic but can be numerically indefinite when Z holds
            // near-null vectors of A (the a priori Z_S contains the temperature ones
            // vector, Eq. 15): invert by LU with partial pivoting as App. C does
            double ratio = 0.0;
            if (!lu_inverse(E, k, Einv, &ratio) || !(ratio > 1e-15))
                throw Error{MM_ERR_NOT_SPD, "coarse operator E is singular"};
            // symmetric like E (the PCG kernels read E^-1 by columns)
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < i; ++j) {
                    const double v = 0.5 * (Einv[(size_t)i * k + j] + Einv[(size_t)j * k + i]);
                    Einv[(size_t)i * k + j] = Einv[(size_t)j * k + i] = v;
                }
        }
        cd.Einv = dalloc<double>(Einv.size());
        h2d(cd.Einv, Einv.data(), Einv.size() * 8, s);
        cd.Z32 = dalloc<float>((size_t)k * P.n);
        cd.AZ32 = dalloc<float>((size_t)k * P.n);
        launch_convert_f64_to_f32(cd.Z64, cd.Z32, (int64_t)k * P.n, s);
        launch_convert_f64_to_f32(cd.AZ64, cd.AZ32, (int64_t)k * P.n, s);
        sync(s);
    } catch (...) {
        free_coarse(cd);
        throw;
    }
    free_coarse(P.coarse);
    P.coarse = cd;
}

// Orthonormalises the kc columns of Y (FP64 [kc][n], device) in order by classical
// Gram-Schmidt with a second projection (CGS2) in FP64 on the device.  Reading R16 (the
// paper is silent on dependent coarse columns, and E = Z^T A Z of Eq. 12 must be
// invertible): column j is dropped when its part orthogonal to the columns kept before
// it has norm below COARSE_DROP_RTOL times the largest column norm of Y.  Two
// projections resolve that part to a few eps of the column's norm, so an exact
// duplicate (~1e-16) is dropped and a near-duplicate 1e-9 away is kept.  Y is replaced
// by the orthonormal columns (kept order), kc updated, *kept_out = the input columns
// kept.  Non-finite columns: MM_ERR_NUMERIC.  Uses P.r64 and P.x64 as scratch.
static constexpr double COARSE_DROP_RTOL = 1e-10;
static void orthonormalise_drop(PlanHolder& P, double*& Y, int& kc, std::vector<int>* kept_out = nullptr) {
    cudaStream_t s = P.stream;
    const int64_t n = P.n;
    double scale = 0.0;
    for (int j = 0; j < kc; ++j) {
        const double nj = std::sqrt(dot64(P, Y + (size_t)j * n, Y + (size_t)j * n));
        if (!std::isfinite(nj)) throw Error{MM_ERR_NUMERIC, "coarse vectors hold NaN or Inf"};
        scale = std::max(scale, nj);
    }
    if (!(scale > 0.0)) throw Error{MM_ERR_NUMERIC, "coarse vectors are all zero"};
    double* Q = nullptr;
    double* hv = nullptr;
    try {
        Q = dalloc<double>((size_t)kc * n);
        hv = dalloc<double>((size_t)kc);
        double* v = P.r64;
        double* t = P.x64;
        std::vector<int> kept;
        for (int j = 0; j < kc; ++j) {
            check_cuda(cudaMemcpyAsync(v, Y + (size_t)j * n, (size_t)n * 8, cudaMemcpyDeviceToDevice, s), "copy column");
            const int q = (int)kept.size();
            for (int pass = 0; q > 0 && pass < 2; ++pass) {
                const std::vector<double> h = gram_host(P, Q, q, v, 1);
                h2d(hv, h.data(), h.size() * 8, s);
                launch_lincomb<double>(Q, q, n, hv, 1, t, s);
                launch_sub(v, t, v, n, s);
            }
            const double piv = std::sqrt(dot64(P, v, v));
            if (!std::isfinite(piv)) throw Error{MM_ERR_NUMERIC, "coarse orthonormalisation produced NaN or Inf"};
            if (!(piv > 0.0) || piv < COARSE_DROP_RTOL * scale) continue;
            const double inv = 1.0 / piv;
            h2d(hv, &inv, 8, s);
            launch_lincomb<double>(v, 1, n, hv, 1, Q + (size_t)q * n, s);
            sync(s);   // hv is rewritten by the next column
            kept.push_back(j);
        }
        sync(s);
        dfree(hv);
        hv = nullptr;
        if (kept.empty()) throw Error{MM_ERR_NUMERIC, "coarse orthonormalisation kept no column"};
        dfree(Y);
        Y = Q;
        kc = (int)kept.size();
        if (kept_out != nullptr) *kept_out = kept;
    } catch (...) {
        dfree(Q);
        dfree(hv);
        throw;
    }
}

// The a posteriori coarse space from the paper's own Ritz source (App. A, Algorithm 1):
// the basic Arnoldi process on B = M_BD A from w_1 = r_0 / ||r_0||, r_0 = M_BD b'
// (x_0 = 0), in FP64 on the device (classical Gram-Schmidt as in Algorithm 1 with one
// re-orthogonalisation pass), until the GMRES residual min ||beta e_1 - Hbar y|| (Givens
// updates on the host) is <= tol beta, maxit steps, or breakdown.  The Ritz pairs of H_m
// (Eq. A.4) with |Re lambda| < eps_tol (Sec. 5), at most kmax, smallest Re first, give
// y = W_m v (a complex pair: the real and imaginary parts of one member), then the
// orthonormalisation with dropping (orthonormalise_drop) and the coarse operators.
static void build_coarse_arnoldi(PlanHolder& P, int kmax, double eps_tol, const double* bprime, double tol,
                                 int maxit) {
    cudaStream_t s = P.stream;
    if (kmax < 1 || kmax > KMAX) throw Error{MM_ERR_ARG, "kmax must be in [1, 64]"};
    if (maxit < 1 || !(eps_tol > 0.0)) throw Error{MM_ERR_ARG, "need maxit >= 1 and eps_tol > 0"};
    if (P.tz64.logn == 0) throw Error{MM_ERR_ARG, "the Arnoldi construction needs the FP64 Toeplitz block"};
    const double* bsrc = bprime;
    if (bsrc == nullptr) {
        if (!P.have_b) throw Error{MM_ERR_STATE, "no right-hand side: pass bprime or call mm_solve first"};
        bsrc = P.b64;
    }
    const int64_t n = P.n;
    const int mcap = (int)std::min<int64_t>(maxit, n);
    double* W = nullptr;
    double* hv = nullptr;
    double* Y = nullptr;
    int wcap = std::min(mcap, 63) + 1;   // basis columns allocated; doubled on demand
    try {
        W = dalloc<double>((size_t)wcap * n);
        hv = dalloc<double>((size_t)mcap + 1);
        double* v = P.r64;       // scratch [n]
        double* t = P.x64;       // scratch [n]
        // w_1 = M_BD b' / ||M_BD b'||
        launch_bd_apply<double>(P, bsrc, v, s);
        const double beta = std::sqrt(dot64(P, v, v));
        if (!(beta > 0.0)) throw Error{MM_ERR_ARG, "M_BD b' is zero"};
        std::vector<double> sc = {1.0 / beta};
        h2d(hv, sc.data(), 8, s);
        launch_lincomb<double>(v, 1, n, hv, 1, W, s);
        std::vector<double> H((size_t)(mcap + 1) * mcap, 0.0);   // Hbar, row-major (mcap + 1) x mcap
        std::vector<double> gc, gs, g = {beta};                  // Givens of the GMRES update
        int j = 0;
        while (j < mcap) {
            if (j + 2 > wcap) {
                const int ncap = std::min(2 * wcap, mcap + 1);
                double* W2 = dalloc<double>((size_t)ncap * n);
                try {
                    check_cuda(cudaMemcpyAsync(W2, W, (size_t)wcap * n * 8, cudaMemcpyDeviceToDevice, s), "grow W");
                    sync(s);
                } catch (...) {
                    dfree(W2);
                    throw;
                }
                dfree(W);
                W = W2;
                wcap = ncap;
            }
            double* wj = W + (size_t)j * n;
            apply_A<double>(P, wj, P.ax64, nullptr);
            launch_bd_apply<double>(P, P.ax64, v, s);
            std::vector<double> h((size_t)j + 1, 0.0);
            for (int pass = 0; pass < 2; ++pass) {
                const std::vector<double> hp = gram_host(P, W, j + 1, v, 1);
                h2d(hv, hp.data(), hp.size() * 8, s);
                launch_lincomb<double>(W, j + 1, n, hv, 1, t, s);
                launch_sub(v, t, v, n, s);
                for (int i = 0; i <= j; ++i) h[(size_t)i] += hp[(size_t)i];
            }
            const double hn = std::sqrt(dot64(P, v, v));
            for (int i = 0; i <= j; ++i) H[(size_t)i * mcap + j] = h[(size_t)i];
            H[(size_t)(j + 1) * mcap + j] = hn;
            // GMRES residual: previous rotations on the new column, then a new one
            std::vector<double> col(h);
            col.push_back(hn);
            for (int i = 0; i < j; ++i) {
                const double a = col[(size_t)i], b = col[(size_t)i + 1];
                col[(size_t)i] = gc[(size_t)i] * a + gs[(size_t)i] * b;
                col[(size_t)i + 1] = -gs[(size_t)i] * a + gc[(size_t)i] * b;
            }
            const double rr = std::hypot(col[(size_t)j], col[(size_t)j + 1]);
            const double cj = rr > 0.0 ? col[(size_t)j] / rr : 1.0, sj = rr > 0.0 ? col[(size_t)j + 1] / rr : 0.0;
            gc.push_back(cj);
            gs.push_back(sj);
            g.push_back(-sj * g[(size_t)j]);
            g[(size_t)j] = cj * g[(size_t)j];
            ++j;
            const bool stop = hn == 0.0 || std::fabs(g[(size_t)j]) <= tol * beta;
            if (hn > 0.0) {
                sc[0] = 1.0 / hn;
                h2d(hv, sc.data(), 8, s);
                launch_lincomb<double>(v, 1, n, hv, 1, W + (size_t)j * n, s);
            }
            if (stop) break;
        }
        sync(s);
        // Ritz pairs of the square H_j
        std::vector<double> Hj((size_t)j * j);
        for (int r = 0; r < j; ++r)
            for (int c = 0; c < j; ++c) Hj[(size_t)r * j + c] = H[(size_t)r * mcap + c];
        std::vector<std::complex<double>> lam;
        if (!hessenberg_eigenvalues(Hj, j, lam)) throw Error{MM_ERR_NUMERIC, "Hessenberg QR did not converge"};
        std::vector<int> order((size_t)j);
        for (int i = 0; i < j; ++i) order[(size_t)i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lam[(size_t)a].real() < lam[(size_t)b].real(); });
        std::vector<char> taken((size_t)j, 0);
        std::vector<std::vector<double>> cols;   // coefficient columns over W_j
        std::vector<double> vals;
        for (int i : order) {
            if (taken[(size_t)i] || !(std::fabs(lam[(size_t)i].real()) < eps_tol) || (int)vals.size() >= kmax) continue;
            taken[(size_t)i] = 1;
            std::vector<std::complex<double>> ev = hessenberg_eigenvector(Hj, j, lam[(size_t)i]);
            const bool real = std::fabs(lam[(size_t)i].imag()) <= 1e-12 * std::abs(lam[(size_t)i]);
            if (real) {
                // rotate the largest component onto the real axis, keep the real part
                size_t im = 0;
                for (size_t q = 1; q < ev.size(); ++q)
                    if (std::abs(ev[q]) > std::abs(ev[im])) im = q;
                const std::complex<double> ph = std::abs(ev[im]) / ev[im];
                std::vector<double> c((size_t)j);
                for (int q = 0; q < j; ++q) c[(size_t)q] = (ev[(size_t)q] * ph).real();
                cols.push_back(c);
                vals.push_back(lam[(size_t)i].real());
            } else {
                std::vector<double> cr((size_t)j), ci((size_t)j);
                for (int q = 0; q < j; ++q) {
                    cr[(size_t)q] = ev[(size_t)q].real();
                    ci[(size_t)q] = ev[(size_t)q].imag();
                }
                cols.push_back(cr);
                cols.push_back(ci);
                vals.push_back(lam[(size_t)i].real());
                vals.push_back(lam[(size_t)i].real());
                int pair = -1;
                double best = 0.0;
                for (int q = 0; q < j; ++q) {
                    if (taken[(size_t)q]) continue;
                    const double dd = std::abs(lam[(size_t)q] - std::conj(lam[(size_t)i]));
                    if (pair < 0 || dd < best) {
                        pair = q;
                        best = dd;
                    }
                }
                if (pair >= 0) taken[(size_t)pair] = 1;
            }
        }
        if (cols.empty()) throw Error{MM_ERR_STATE, "no Ritz value below eps_tol"};
        if ((int)cols.size() > KMAX) cols.resize(KMAX), vals.resize(KMAX);
        const int kk = (int)cols.size();
        std::vector<double> C((size_t)j * kk);
        for (int q = 0; q < j; ++q)
            for (int c = 0; c < kk; ++c) C[(size_t)q * kk + c] = cols[(size_t)c][(size_t)q];
        Y = dalloc<double>((size_t)kk * n);   // freed by the handler below on failure
        double* Cd = dalloc<double>(C.size());
        try {
            h2d(Cd, C.data(), C.size() * 8, s);
            launch_lincomb<double>(W, j, n, Cd, kk, Y, s);
            sync(s);
        } catch (...) {
            dfree(Cd);
            throw;
        }
        dfree(Cd);
        dfree(W);
        W = nullptr;
        dfree(hv);
        hv = nullptr;
        int kc = kk;
        std::vector<int> kept;
        orthonormalise_drop(P, Y, kc, &kept);
        double* Zk = Y;
        Y = nullptr;
        std::vector<double> kept_vals;   // the values of the kept columns
        for (int c : kept) kept_vals.push_back(vals[(size_t)c]);
        install_coarse(P, Zk, kc, kept_vals);
    } catch (...) {
        dfree(W);
        dfree(hv);
        dfree(Y);
        throw;
    }
}

// The a priori coarse space Z_S of Sec. 3.3.1 (Eq. 16-17) with its K interval columns
// merged into r groups of consecutive intervals (interval i -> group floor(i r / K); a
// merged column is the sum of its members, so observed temperature rows still sum to 1,
// Q/U rows are 0), then replaced by an orthonormal basis of its range (orthonormalise_drop:
// intervals that see the same hit fractions give equal columns, which are dropped).
// M_2lvl depends on Z only through
// its range, and raw hit-fraction columns of a scan that covers the patch evenly are
// nearly parallel, which leaves E = Z^T A Z numerically singular; the orthonormal basis
// keeps E as well conditioned as A is on that range.
static void build_coarse_apriori(PlanHolder& P, int r) {
    if (r < 1 || r > KMAX || r > P.K) throw Error{MM_ERR_ARG, "r must be in [1, min(64, K)]"};
    double* Z = dalloc<double>((size_t)r * P.n);
    try {
        launch_apriori(P, r, Z, P.stream);
        int kc = r;
        orthonormalise_drop(P, Z, kc);
        double* Zt = Z;
        Z = nullptr;
        install_coarse(P, Zt, kc, {});
    } catch (...) {
        dfree(Z);
        throw;
    }
}

template <typename T>
static void build_coarse(PlanHolder& P, int k, const double* bprime, double tol, int maxit, double eps_tol = 0.0) {
    cudaStream_t s = P.stream;
    if (k < 1 || k > KMAX) throw Error{MM_ERR_ARG, "k must be in [1, 64]"};
    if (maxit < 1) throw Error{MM_ERR_ARG, "maxit must be >= 1"};
    const double* bsrc = bprime;
    if (bsrc == nullptr) {
        if (!P.have_b) throw Error{MM_ERR_STATE, "no right-hand side: pass bprime or call mm_solve first"};
        bsrc = P.b64;
    }
    // first solve with M_BD, keeping z_j and the step scalars (Sec. 3.3.2 step 1)
    if constexpr (sizeof(T) == 8) {
        check_cuda(cudaMemcpyAsync(P.pcg.r, bsrc, (size_t)P.n * 8, cudaMemcpyDeviceToDevice, s), "copy b'");
    } else {
        launch_convert_f64_to_f32(bsrc, static_cast<float*>(P.pcg.r), P.n, s);
    }
    ensure_history(P, maxit);
    P.hist_runs.clear();
    T* zstore = static_cast<T*>(dmalloc((size_t)(maxit + 1) * P.n * sizeof(T)));
    double* Y = nullptr;
    double* C = nullptr;
    try {
        const PcgOutcome o = run_pcg<T>(P, 0, tol, maxit, zstore, maxit + 1);
        P.hist_runs.assign(1, PlanHolder::HistRun{0, o.iters, o.bb, o.bb == 0.0 ? 0.0 : 1.0});   // the last PCG run
        if (o.status != MM_OK && o.status != MM_ERR_NOT_CONVERGED)
            throw Error{(mm_status)o.status, "first solve of the coarse construction failed"};
        const int m = o.iters;   // alphas 0..m-1, betas 0..m-2, z_0..z_{m-1}
        if (m < 1) throw Error{MM_ERR_STATE, "first solve took no step"};
        std::vector<double> al((size_t)m), be((size_t)std::max(m - 1, 1)), rz((size_t)m);
        d2h(al.data(), P.pcg.hist_alpha, (size_t)m * 8, s);
        if (m > 1) d2h(be.data(), P.pcg.hist_beta, (size_t)(m - 1) * 8, s);
        d2h(rz.data(), P.pcg.hist_rz, (size_t)m * 8, s);
        sync(s);
        // Lanczos tridiagonal of M_BD A (App. A, CG form)
        std::vector<double> d((size_t)m), e((size_t)std::max(m - 1, 0));
        for (int j = 0; j < m; ++j) d[(size_t)j] = 1.0 / al[(size_t)j] + (j > 0 ? be[(size_t)j - 1] / al[(size_t)j - 1] : 0.0);
        for (int j = 0; j + 1 < m; ++j) e[(size_t)j] = std::sqrt(be[(size_t)j]) / al[(size_t)j];
        std::vector<double> theta, S;
        int kk = std::min(k, m);
        tridiag_smallest(d, e, kk, theta, S);
        if (eps_tol > 0.0) {
            // keep the Ritz pairs with |theta| < eps_tol (Sec. 5), smallest first
            int c = 0;
            while (c < kk && std::fabs(theta[(size_t)c]) < eps_tol) ++c;
            if (c == 0) throw Error{MM_ERR_STATE, "no Ritz value below eps_tol"};
            if (c < kk) {
                std::vector<double> S2((size_t)m * c);
                for (int j = 0; j < m; ++j)
                    for (int q = 0; q < c; ++q) S2[(size_t)j * c + q] = S[(size_t)j * kk + q];
                S.swap(S2);
                theta.resize((size_t)c);
                kk = c;
            }
        }
        // Ritz vectors Y = sum_j (-1)^j z_j / sqrt(r_j^T z_j) S_j  (step 2-4)
        std::vector<double> Cs((size_t)m * kk);
        for (int j = 0; j < m; ++j) {
            const double f = ((j & 1) ? -1.0 : 1.0) / std::sqrt(rz[(size_t)j]);
            for (int c = 0; c < kk; ++c) Cs[(size_t)j * kk + c] = f * S[(size_t)j * kk + c];
        }
        C = dalloc<double>(Cs.size());
        h2d(C, Cs.data(), Cs.size() * 8, s);
        Y = dalloc<double>((size_t)kk * P.n);
        launch_lincomb<T>(zstore, m, P.n, C, kk, Y, s);
        sync(s);
        dfree(zstore);
        zstore = nullptr;
        dfree(C);
        C = nullptr;
        // Euclidean orthonormalisation with dependent columns dropped (reading R16)
        int kcur = kk;
        std::vector<int> kept;
        orthonormalise_drop(P, Y, kcur, &kept);
        if (kcur < kk) {   // the reported Ritz values follow the kept columns
            std::vector<double> th2;
            for (int c : kept) th2.push_back(theta[(size_t)c]);
            theta.swap(th2);
        }
        double* Zk = Y;
        Y = nullptr;
        install_coarse(P, Zk, kcur, theta);
    } catch (...) {
        dfree(zstore);
        dfree(Y);
        dfree(C);
        throw;
    }
}

// -------------------------------------------------------------------------- solve
static void check_solve_opts(const PlanHolder& P, const mm_solve_opts& so) {
    if (!(so.tol >= 0.0) || so.maxit < 1) throw Error{MM_ERR_ARG, "tol must be >= 0 and maxit >= 1"};
    if (so.residual != MM_RESID_DF32 && so.residual != MM_RESID_FP64) throw Error{MM_ERR_ARG, "bad residual arithmetic"};
    if (so.kind != MM_PREC_BD && so.kind != MM_PREC_TWOLEVEL && so.kind != MM_PREC_ADEF2)
        throw Error{MM_ERR_ARG, "bad preconditioner kind"};
    if (so.solver != MM_SOLVE_FP64 && so.solver != MM_SOLVE_MIXED) throw Error{MM_ERR_ARG, "bad solver"};
    if (so.kind != MM_PREC_BD && P.coarse.k == 0)
        throw Error{MM_ERR_STATE, "two-level preconditioner needs mm_build_coarse"};
}

// FP64 residual r = b - A x: with the data d (device, FP64) as P^T N^-1 (d - P x) -- one
// Toeplitz pass on the residual data, free of the cancellation between b and A x --
// else as b - A x from P.b64.  df: that Toeplitz pass in double-float arithmetic (FP64
// data, ~48-bit FFT on the FP32 pipe) when the plan has the tables for it.
static void residual64(PlanHolder& P, const double* d, const double* x, double* r, bool df = false) {
    cudaStream_t s = P.stream;
    if (d != nullptr) {
        const bool use_df = df && P.tzdf.logn != 0;
        int sl = prof_begin(P, use_df ? ST_TZDF : ST_TZ64);
        if (use_df)
            launch_toeplitz_df(P, nullptr, d, x, 1, 0, P.tod64, 0, s);
        else
            launch_toeplitz_any<double>(P, P.tz64, nullptr, d, x, 1, 0, P.tod64, 0, nullptr, s);
        prof_end(P, sl);
        sl = prof_begin(P, ST_SC64);
        launch_scatter<double>(P, P.tod64, r, nullptr, s);
        prof_end(P, sl);
    } else {
        apply_A<double>(P, x, P.ax64, nullptr);
        launch_sub(P.b64, P.ax64, r, P.n, s);
    }
}

// Solve A x = b for the b in P.b64 into xout (device); fills the iteration part of stats
// and returns the status.  d: the data b came from (device, FP64) or null; with it the
// FP64 residuals take the one-pass form of residual64.
static int solve_from_b(PlanHolder& P, const mm_solve_opts& so, double* xout, mm_stats& stats,
                        const double* d = nullptr) {
    cudaStream_t s = P.stream;
    const double tol = so.tol;
    const int maxit = so.maxit;
    const int cm = coarse_mode(so.kind);
    const int max_outer = so.max_outer > 0 ? so.max_outer : 20;
    const double inner_min = so.inner_tol_min > 0.0 ? so.inner_tol_min : 3e-7;
    int status = MM_OK;
    const double bb = dot64(P, P.b64, P.b64);
    const double bn = std::sqrt(bb);
    // residual history: each PCG run of this solve writes from its own offset, one spare
    // entry after the previous run's last (at most maxit steps and max_outer runs in all)
    ensure_history(P, (int)std::min<int64_t>((int64_t)maxit + max_outer + 1, MAX_HISTORY));
    P.hist_runs.clear();
    if (so.solver == MM_SOLVE_FP64) {
        check_cuda(cudaMemcpyAsync(P.pcg.r, P.b64, (size_t)P.n * 8, cudaMemcpyDeviceToDevice, s), "copy b");
        const PcgOutcome o = run_pcg<double>(P, cm, tol, maxit, nullptr, 0, 0);
        P.hist_runs.push_back({0, o.iters, o.bb, o.bb == 0.0 ? 0.0 : 1.0});
        if (o.status != MM_OK) status = o.status;
        check_cuda(cudaMemcpyAsync(xout, P.pcg.x, (size_t)P.n * 8, cudaMemcpyDeviceToDevice, s), "copy x");
        stats.iters = o.iters;
        stats.outer = 1;
        stats.rel_resid_rec = bb > 0 ? std::sqrt(o.rr / o.bb) : 0.0;
        // true residual of the returned map
        residual64(P, d, xout, P.r64);
        const double rr = dot64(P, P.r64, P.r64);
        stats.rel_resid = bn > 0 ? std::sqrt(rr) / bn : 0.0;
        stats.fp64_products = 1;
        stats.converged = status == MM_OK;
        return status;
    }
    // iterative refinement: FP64 residual, FP32 inner PCG on the scaled residual
    check_cuda(cudaMemsetAsync(xout, 0, (size_t)P.n * 8, s), "memset x");
    check_cuda(cudaMemcpyAsync(P.r64, P.b64, (size_t)P.n * 8, cudaMemcpyDeviceToDevice, s), "copy b");
    double rr = bb;
    int total = 0;
    int outer = 0;
    int fp64 = 0;
    double last_rec = 1.0;
    status = MM_ERR_NOT_CONVERGED;
    while (true) {
        if (std::sqrt(rr) <= tol * bn || bb == 0.0) {
            status = MM_OK;
            break;
        }
        if (total >= maxit || outer >= max_outer) break;
        // r32 = r / ||r||  (the norm^2 stays in device memory for the update)
        launch_dot64(P.r64, P.r64, P.n, P.d_dot, P.d_dot + DOT_BLOCKS, s);
        launch_scale_to_f32(P.r64, P.d_dot + DOT_BLOCKS, static_cast<float*>(P.pcg.r), P.n, s);
        double tol_in = 0.5 * tol * bn / std::sqrt(rr);
        tol_in = std::min(0.5, std::max(tol_in, inner_min));
        if (outer == 0 && so.first_inner_tol > 0.0) tol_in = so.first_inner_tol;
        const PcgOutcome o = run_pcg<float>(P, cm, tol_in, maxit - total, nullptr, 0, total + outer);
        // the inner right-hand side is r / ||r||: its residuals scale by ||r|| / ||b||
        P.hist_runs.push_back({total + outer, o.iters, o.bb, std::sqrt(rr) / bn});
        if (o.status != MM_OK && o.status != MM_ERR_NOT_CONVERGED) {
            status = o.status;
            break;
        }
        total += o.iters;
        last_rec = o.bb > 0 ? std::sqrt(o.rr / o.bb) : 0.0;
        launch_axpy_f32(xout, static_cast<const float*>(P.pcg.x), P.d_dot + DOT_BLOCKS, P.n, s);
        residual64(P, d, xout, P.r64, so.residual != MM_RESID_FP64);
        ++fp64;
        rr = dot64(P, P.r64, P.r64);
        ++outer;
        if (!std::isfinite(rr)) {
            status = MM_ERR_NUMERIC;
            break;
        }
    }
    // no inner solve ran (b = 0, or tol >= 1): the history is the start alone
    if (P.hist_runs.empty()) P.hist_runs.push_back({0, 0, 0.0, bb > 0.0 ? 1.0 : 0.0});
    stats.iters = total;
    stats.outer = outer;
    stats.fp64_products = fp64;
    stats.rel_resid = bn > 0 ? std::sqrt(rr) / bn : 0.0;
    stats.rel_resid_rec = last_rec;
    stats.converged = status == MM_OK;
    return status;
}

static const char* status_text(int status) {
    return status == MM_ERR_NOT_CONVERGED ? "maxit reached before tol" : "solve failed";
}

static void solve(PlanHolder& P, const double* d, const mm_solve_opts& so, double* m, mm_stats* st) {
    cudaStream_t s = P.stream;
    check_solve_opts(P, so);
    mm_stats stats{};
    check_cuda(cudaEventRecord(P.ev0, s), "event");
    const double* dd = d;
    if (!is_device_ptr(d)) {
        h2d(P.dbuf, d, (size_t)P.nt * 8, s);
        dd = P.dbuf;
    }
    // b = P^T N^-1 d (Eq. 7): in FP64 for the FP64 solver; in FP32 for the mixed solver,
    // whose FP64 residuals come from the data (residual64), so b only seeds the first
    // inner solve and scales the residual norm
    if (so.solver == MM_SOLVE_MIXED && P.tz32.logn != 0) {
        int sl = prof_begin(P, ST_TZ32);
        launch_toeplitz_any<float>(P, P.tz32, nullptr, dd, nullptr, 1, 0, P.tod32, 0, nullptr, s);
        prof_end(P, sl);
        sl = prof_begin(P, ST_SC32);
        float* b32 = static_cast<float*>(P.pcg.z);   // scratch until the first PCG start
        launch_scatter<float>(P, P.tod32, b32, nullptr, s);
        prof_end(P, sl);
        launch_convert_f32_to_f64(b32, P.b64, P.n, s);
    } else {
        int sl = prof_begin(P, ST_TZ64);
        launch_toeplitz<double>(P, P.tz64, dd, nullptr, P.tod64, nullptr, s);
        prof_end(P, sl);
        sl = prof_begin(P, ST_SC64);
        launch_scatter<double>(P, P.tod64, P.b64, nullptr, s);
        prof_end(P, sl);
    }
    P.have_b = true;
    check_cuda(cudaEventRecord(P.ev1, s), "event");
    const bool m_dev = is_device_ptr(m);
    double* xout = m_dev ? m : P.x64;
    const int status = solve_from_b(P, so, xout, stats, P.tz64.logn != 0 ? dd : nullptr);
    if (!m_dev) d2h(m, xout, (size_t)P.n * 8, s);
    check_cuda(cudaEventRecord(P.ev2, s), "event");
    sync(P);
    float ms = 0.f, ms_rhs = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, P.ev0, P.ev2), "event time");
    check_cuda(cudaEventElapsedTime(&ms_rhs, P.ev0, P.ev1), "event time");
    stats.ms_total = ms;
    stats.ms_rhs = ms_rhs;
    if (st != nullptr) *st = stats;
    if (status != MM_OK) throw Error{(mm_status)status, status_text(status)};
}

// ----------------------------------------------------------------------- gradient
// Derivative spectra of the Toeplitz rows, built on the first gradient call.
static void ensure_grad(PlanHolder& P) {
    if (P.grad_H != nullptr) return;
    if (P.tz64.logn == 0) throw Error{MM_ERR_ARG, "the PSD gradient needs an FP64 Toeplitz block for this lambda"};
    const int64_t N = int64_t(1) << P.tz64.logn;
    std::vector<double> H((size_t)3 * P.npsd * (N + 1));
    for (int p = 0; p < P.npsd; ++p) {
        if (!(P.h_psd[(size_t)p].fknee > 0.0)) throw Error{MM_ERR_ARG, "the PSD gradient needs fknee > 0"};
        const auto D = toeplitz_row_derivatives(P.h_psd[(size_t)p].sigma, P.h_psd[(size_t)p].fknee,
                                                P.h_psd[(size_t)p].alpha, P.L_grid, P.fsamp, P.lambda, P.window);
        for (int c = 0; c < 3; ++c) {
            const std::vector<double> h = overlap_save_spectrum(D[(size_t)c], N);
            std::copy(h.begin(), h.end(), H.begin() + ((size_t)c * P.npsd + p) * (N + 1));
        }
    }
    P.grad_H = dalloc<double>(H.size());
    h2d(P.grad_H, H.data(), H.size() * 8, P.stream);
    P.grad_u = dalloc<double>((size_t)P.nt);
    P.grad_part = dalloc<double>((size_t)P.K);
    sync(P.stream);
}

// dL/dd = N^-1 P mu and dL/dtheta[p][c] = u^T (dN^-1/dtheta_pc) (d - P m), mu = A^-1 g.
static void grad(PlanHolder& P, const double* d, const double* m, const double* g, double* dLdd, double* dLdpsd,
                 const mm_solve_opts& so, mm_stats* st) {
    cudaStream_t s = P.stream;
    check_solve_opts(P, so);
    if (dLdpsd != nullptr) ensure_grad(P);
    else if (P.grad_u == nullptr) P.grad_u = dalloc<double>((size_t)P.nt);
    mm_stats stats{};
    check_cuda(cudaEventRecord(P.ev0, s), "event");
    // adjoint solve A mu = g (A is symmetric)
    if (is_device_ptr(g))
        check_cuda(cudaMemcpyAsync(P.b64, g, (size_t)P.n * 8, cudaMemcpyDeviceToDevice, s), "copy g");
    else
        h2d(P.b64, g, (size_t)P.n * 8, s);
    P.have_b = false;
    double* mu = P.x64;
    const int status = solve_from_b(P, so, mu, stats);
    if (status != MM_OK) {
        if (st) *st = stats;
        throw Error{(mm_status)status, std::string("adjoint solve: ") + status_text(status)};
    }
    // u = P mu
    launch_gather<double>(P, mu, P.grad_u, s);
    if (dLdd != nullptr) {
        const bool dev = is_device_ptr(dLdd);
        double* out = dev ? dLdd : P.tod64;
        launch_toeplitz<double>(P, P.tz64, P.grad_u, nullptr, out, nullptr, s);
        if (!dev) d2h(dLdd, out, (size_t)P.nt * 8, s);
    }
    if (dLdpsd != nullptr) {
        // v = d - P m in dbuf (staging the inputs when they are host memory)
        const double* mm_ = m;
        if (!is_device_ptr(m)) {
            h2d(P.r64, m, (size_t)P.n * 8, s);
            mm_ = P.r64;
        }
        launch_gather<double>(P, mm_, P.tod64, s);
        const double* dd = d;
        if (!is_device_ptr(d)) {
            h2d(P.dbuf, d, (size_t)P.nt * 8, s);
            dd = P.dbuf;
        }
        launch_sub_time(dd, P.tod64, P.dbuf, P.nt, s);
        const int64_t N = int64_t(1) << P.tz64.logn;
        std::vector<double> part((size_t)P.K);
        for (int c = 0; c < 3; ++c) {
            ToeplitzDev tzc = P.tz64;
            tzc.H = P.grad_H + (size_t)c * P.npsd * (N + 1);
            launch_toeplitz<double>(P, tzc, P.dbuf, nullptr, P.tod64, nullptr, s);
            launch_interval_dot(P.grad_u, P.tod64, P.ioff, P.K, P.grad_part, s);
            d2h(part.data(), P.grad_part, (size_t)P.K * 8, s);
            sync(P.stream);
            for (int p = 0; p < P.npsd; ++p) dLdpsd[(size_t)p * 3 + c] = 0.0;
            for (int i = 0; i < P.K; ++i) dLdpsd[(size_t)P.h_ipsd[(size_t)i] * 3 + c] += part[(size_t)i];
        }
    }
    check_cuda(cudaEventRecord(P.ev2, s), "event");
    sync(P);
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, P.ev0, P.ev2), "event time");
    stats.ms_total = ms;
    if (st != nullptr) *st = stats;
}


// ------------------------------------------------------------------ batched solver
// Complex-pair kernel tables for a 2^logb-point block.
static void build_batch_pair(PlanHolder& P, int logb) {
    BatchState& bt = P.batch;
    bt.logb = logb;
    const int64_t B = int64_t(1) << logb;
    const int64_t Lv = B - 2 * (int64_t)P.lambda;
    std::vector<SpanTile> tiles;
    for (int i = 0; i < P.K; ++i) {
        const int64_t a = P.h_ioff[i], b = P.h_ioff[i + 1];
        for (int64_t s0 = a; s0 < b; s0 += Lv) {
            SpanTile t;
            t.out0 = s0;
            t.ibeg = a;
            t.iend = b;
            t.nout = (int32_t)std::min<int64_t>(Lv, b - s0);
            t.psd = P.h_ipsd[i];
            tiles.push_back(t);
        }
    }
    bt.ntiles = (int)tiles.size();
    bt.tiles = dalloc<SpanTile>(tiles.size());
    h2d(bt.tiles, tiles.data(), tiles.size() * sizeof(SpanTile), P.stream);
    std::vector<float> H((size_t)P.npsd * (B / 2 + 1));
    for (int p = 0; p < P.npsd; ++p) {
        // overlap_save_spectrum(t, N) returns sigma_k / N for k <= N on a 2N grid
        const std::vector<double> h = overlap_save_spectrum(P.rows[(size_t)p], B / 2);
        for (int64_t k = 0; k <= B / 2; ++k) H[(size_t)p * (B / 2 + 1) + k] = (float)(h[(size_t)k] * 0.5);
    }
    bt.H = dalloc<float>(H.size());
    h2d(bt.H, H.data(), H.size() * 4, P.stream);
    const std::vector<double> pt = pass_twiddle_table(std::min(logb, BATCH_MAX_LOGB_CTA));
    std::vector<float> ptf(pt.begin(), pt.end());
    bt.ptw = dalloc<float>(ptf.size());
    h2d(bt.ptw, ptf.data(), ptf.size() * 4, P.stream);
    std::vector<float> tw((size_t)(B / 4 + 1));
    for (int64_t k = 0; k <= B / 4; ++k) tw[(size_t)k] = (float)std::cos(2.0 * 3.14159265358979323846 * (double)k / (double)B);
    bt.twiddle = dalloc<float>(tw.size());
    h2d(bt.twiddle, tw.data(), tw.size() * 4, P.stream);
    sync(P.stream);
}

// Tables of the tensor-core form: groups of four 128-row tiles per interval, and per PSD
// the K-chunks (64 wide) of the band matrix A[m][k] = c[k - m], c[j] = t_|j - lambda|
// (0 <= j <= 2 lambda), scaled by a power of two (largest |c| below 2^14) and split into
// FP16 hi + 2^-11 lo, each chunk in the no-swizzle K-major core-matrix layout (element
// (m, kk) at byte (m / 8) 1024 + (kk / 8) 128 + (m % 8) 16 + (kk % 8) 2).
static void build_batch_tc(PlanHolder& P) {
    BatchState& bt = P.batch;
    if (bt.tc_atab != nullptr) return;
    constexpr int M = 128, KC = 64, G = 4;
    const int64_t lam = P.lambda;
    const int nchunk = (int)((M + 2 * lam + KC - 1) / KC);
    std::vector<SpanTile> groups;
    for (int i = 0; i < P.K; ++i) {
        const int64_t a = P.h_ioff[i], b = P.h_ioff[i + 1];
        for (int64_t s0 = a; s0 < b; s0 += M * G)
            groups.push_back(SpanTile{s0, a, b, (int32_t)std::min<int64_t>(M * G, b - s0), P.h_ipsd[i]});
    }
    const size_t per_chunk = 2 * (size_t)M * KC;   // halves
    std::vector<__half> tab((size_t)P.npsd * nchunk * per_chunk);
    std::vector<float> invc((size_t)P.npsd);
    for (int p = 0; p < P.npsd; ++p) {
        const std::vector<double>& row = P.rows[(size_t)p];
        double mx = 0.0;
        for (double v : row) mx = std::max(mx, std::fabs(v));
        int e = 0;
        if (mx > 0.0) std::frexp(mx, &e);   // mx < 2^e
        const double sc = std::ldexp(1.0, 14 - e);
        invc[(size_t)p] = (float)std::ldexp(1.0, e - 14);
        for (int c = 0; c < nchunk; ++c) {
            __half* hi = tab.data() + ((size_t)p * nchunk + c) * per_chunk;
            __half* lo = hi + (size_t)M * KC;
            for (int m = 0; m < M; ++m)
                for (int kk = 0; kk < KC; ++kk) {
                    const int64_t j = (int64_t)c * KC + kk - m;
                    const double v = (j >= 0 && j <= 2 * lam) ? row[(size_t)std::llabs(j - lam)] * sc : 0.0;
                    const float vf = (float)v;
                    const __half h = __float2half_rn(vf);
                    const __half l = __float2half_rn((float)((v - (double)__half2float(h)) * 2048.0));
                    const size_t off = (size_t)((m / 8) * 1024 + (kk / 8) * 128 + (m % 8) * 16 + (kk % 8) * 2) / 2;
                    hi[off] = h;
                    lo[off] = l;
                }
        }
    }
    try {
        bt.tc_groups = dalloc<SpanTile>(groups.size());
        h2d(bt.tc_groups, groups.data(), groups.size() * sizeof(SpanTile), P.stream);
        bt.tc_atab = dalloc<__half>(tab.size());
        h2d(bt.tc_atab, tab.data(), tab.size() * sizeof(__half), P.stream);
        bt.tc_invc = dalloc<float>(invc.size());
        h2d(bt.tc_invc, invc.data(), invc.size() * 4, P.stream);
        bt.tc_scale = dalloc<float>(2 * BATCH_RMAX);
        sync(P.stream);
    } catch (...) {
        for (void* q : {(void*)bt.tc_groups, (void*)bt.tc_atab, (void*)bt.tc_invc, (void*)bt.tc_scale}) dfree(q);
        bt.tc_groups = nullptr;
        bt.tc_atab = nullptr;
        bt.tc_invc = nullptr;
        bt.tc_scale = nullptr;
        throw;
    }
    bt.tc_ngroups = (int)groups.size();
    bt.tc_nchunk = nchunk;
}

static void ensure_batch_tc_buffer(PlanHolder& P, int R) {
    BatchState& bt = P.batch;
    if (bt.tc_cap >= R) return;
    dfree(bt.tc_y);
    bt.tc_y = nullptr;
    bt.tc_cap = 0;
    bt.tc_y = dalloc<float>((size_t)P.nt * R);
    bt.tc_cap = R;
}

static void launch_batch_tz(PlanHolder& P, int R, const float* X, float* Z, const int* done);
static void launch_batch_tz(PlanHolder& P, int R, const float* X, float* Z, const int* done);

// Batched Toeplitz form, chosen once per plan (before any graph capture), after the
// R-column buffers exist:
//   BATCH_PAIR  two RHS per complex FFT (y_a + i y_b, one complex block of 2^logb points,
//               block > 2 lambda complex points);
//   BATCH_REAL  the single-RHS real-FFT kernel with an RHS grid dimension (its FP32
//               block, B > 2 lambda reals, so half the FFT length of the pair form).
// Cost model per RHS: tiles x (points x log2 + 2048) x cluster weight, halved for the
// pair form; ties go to the pair form.  With autotuning both are timed at this R.
static void ensure_batch_tables(PlanHolder& P, int R, int want = -1) {
    BatchState& bt = P.batch;
    if (bt.kind >= 0) {
        if (want >= 0 && want != bt.kind) throw Error{MM_ERR_ARG, "the batched form is already fixed"};
        if (bt.kind == BATCH_TENSOR) ensure_batch_tc_buffer(P, R);
        return;
    }
    if (want == BATCH_TENSOR) {
        build_batch_tc(P);
        ensure_batch_tc_buffer(P, R);
        bt.kind = BATCH_TENSOR;
        return;
    }
    int best = -1;
    double best_cost = 0.0;
    for (int logb = 9; logb <= BATCH_MAX_LOGB; ++logb) {
        const int64_t B = int64_t(1) << logb;
        const int64_t Lv = B - 2 * (int64_t)P.lambda;
        if (Lv < 1) continue;
        const int cl = logb > BATCH_MAX_LOGB_CTA ? 1 << (logb - BATCH_MAX_LOGB_CTA) : 1;
        const double cost = 0.5 * (double)interval_tiles(P, Lv) * ((double)B * logb + 2048.0) * fp32_cluster_weight(cl);
        if (best < 0 || cost < best_cost) {
            best = logb;
            best_cost = cost;
        }
    }
    double real_cost = -1.0;
    if (P.tz32.logn != 0) {
        const int64_t N = int64_t(1) << P.tz32.logn;
        real_cost = (double)P.tz32.ntiles * ((double)N * (P.tz32.logn + 1) + 2048.0) * block_weight<float>(P.tz32.logn);
    }
    if (best < 0 && real_cost < 0.0) throw Error{MM_ERR_ARG, "lambda too large for the batched FFT blocks"};
    if ((want == BATCH_PAIR && best < 0) || (want == BATCH_REAL && real_cost < 0.0))
        throw Error{MM_ERR_ARG, "no FFT block supports this batched form for lambda"};
    if (best >= 0) build_batch_pair(P, best);
    if (want >= 0) {
        bt.kind = want;
    } else if (best < 0) {
        bt.kind = BATCH_REAL;
    } else if (real_cost < 0.0) {
        bt.kind = BATCH_PAIR;
    } else if (P.autotune) {
        // every form timed on the same R columns (random maps: the tensor form scales
        // its columns by their largest value); the fastest is kept
        {
            std::vector<float> hx((size_t)R * P.n);
            uint64_t st = 0x2545F4914F6CDD1Dull;
            for (auto& v : hx) {
                st ^= st << 13; st ^= st >> 7; st ^= st << 17;
                v = (float)((double)(st >> 11) / 9007199254740992.0 - 0.5);
            }
            h2d(bt.x, hx.data(), hx.size() * 4, P.stream);
            sync(P.stream);
        }
        bt.kind = BATCH_PAIR;
        bt.tuned_ms[0] = time_launches(P, [&] { launch_batch_tz(P, R, bt.x, bt.tod, nullptr); }, 3);
        bt.kind = BATCH_REAL;
        bt.tuned_ms[1] = time_launches(P, [&] { launch_batch_tz(P, R, bt.x, bt.tod, nullptr); }, 3);
        build_batch_tc(P);
        ensure_batch_tc_buffer(P, R);
        bt.kind = BATCH_TENSOR;
        bt.tuned_ms[2] = time_launches(P, [&] { launch_batch_tz(P, R, bt.x, bt.tod, nullptr); }, 3);
        int k = bt.tuned_ms[0] <= bt.tuned_ms[1] ? BATCH_PAIR : BATCH_REAL;
        if (bt.tuned_ms[2] < bt.tuned_ms[k]) k = BATCH_TENSOR;
        bt.kind = k;
    } else {
        bt.kind = best_cost <= real_cost ? BATCH_PAIR : BATCH_REAL;
    }
}

static void ensure_batch_buffers(PlanHolder& P, int R) {
    BatchState& bt = P.batch;
    if (bt.cap >= R) return;
    for (void* p : {(void*)bt.x, (void*)bt.r, (void*)bt.p, (void*)bt.q, (void*)bt.z, (void*)bt.tod, (void*)bt.x64,
                    (void*)bt.b64, (void*)bt.r64})
        dfree(p);
    bt.x = bt.r = bt.p = bt.q = bt.z = bt.tod = nullptr;
    bt.x64 = bt.b64 = bt.r64 = nullptr;
    bt.cap = 0;
    if (bt.graph) {
        (void)cudaGraphExecDestroy(bt.graph);
        bt.graph = nullptr;
    }
    const size_t n = (size_t)P.n, nt = (size_t)P.nt;
    for (float** v : {&bt.x, &bt.r, &bt.p, &bt.q, &bt.z}) *v = dalloc<float>(n * R);
    bt.tod = dalloc<float>(nt * R);
    for (double** v : {&bt.x64, &bt.b64, &bt.r64}) *v = dalloc<double>(n * R);
    if (bt.partial == nullptr) {
        bt.nblocks = std::max(1, std::min(batch_pcg_max_blocks(P.num_sms), (P.npix_obs + 31) / 32));
        bt.partial = dalloc<double>((size_t)bt.nblocks * BATCH_PSTRIDE);
        for (double** v : {&bt.rho, &bt.bb, &bt.rr, &bt.tol2}) *v = dalloc<double>(BATCH_RMAX);
        bt.iters = dalloc<int>(BATCH_RMAX);
        bt.state = dalloc<unsigned char>(BATCH_RMAX);
        bt.flags = dalloc<int>(8);
        bt.bar = dalloc<unsigned>(4);
        check_cuda(cudaMemsetAsync(bt.bar, 0, 16, P.stream), "memset");
    }
    bt.cap = R;
}

static BatchTzArgs batch_tz_args(PlanHolder& P, int R, const float* X, float* Z, const int* done) {
    BatchTzArgs A{};
    A.tiles = P.batch.tiles;
    A.H = P.batch.H;
    A.ptw = reinterpret_cast<const float2*>(P.batch.ptw);
    A.twiddle = P.batch.twiddle;
    A.X = X;
    A.pixc = P.pixc;
    A.w = P.w32;
    A.Z = Z;
    A.done = done;
    A.n = P.n;
    A.nt = P.nt;
    A.R = R;
    A.lambda = P.lambda;
    return A;
}

// Z_r = N^-1 P X_r (FP32) in the plan's batched form
static void launch_batch_tz(PlanHolder& P, int R, const float* X, float* Z, const int* done) {
    BatchState& bt = P.batch;
    if (bt.kind == BATCH_REAL) {
        launch_toeplitz_rhs<float>(P, P.tz32, nullptr, X, R, P.n, Z, P.nt, done, P.stream);
    } else if (bt.kind == BATCH_TENSOR) {
        // column scales from the maps, Y = P X, then the band product on the tensor cores
        launch_batch_colscale(X, P.n, R, bt.tc_scale, bt.tc_scale + BATCH_RMAX, P.stream);
        launch_batch_gather(P, X, R, bt.tc_y, P.stream);
        BatchTcArgs A{};
        A.groups = bt.tc_groups;
        A.atab = bt.tc_atab;
        A.inv_cscale = bt.tc_invc;
        A.Y = bt.tc_y;
        A.Z = Z;
        A.scale = bt.tc_scale;
        A.inv_scale = bt.tc_scale + BATCH_RMAX;
        A.done = done;
        A.flags = bt.flags;
        A.nt = P.nt;
        A.R = R;
        A.RB = (R + 15) / 16 * 16;
        A.lambda = P.lambda;
        A.nchunk = bt.tc_nchunk;
        launch_batch_tc(A, bt.tc_ngroups, P.stream);
    } else {
        launch_batch_toeplitz(batch_tz_args(P, R, X, Z, done), bt.logb, bt.ntiles, P.ncomp, P.stream);
    }
}

// Y_r = A X_r (FP32), r < R <= BATCH_RMAX
static void apply_A_batch(PlanHolder& P, int R, const float* X, float* Y, const int* done) {
    launch_batch_tz(P, R, X, P.batch.tod, done);
    launch_batch_scatter(P, P.batch.tod, Y, R, done, P.stream);
}

static BatchPcgArgs batch_pcg_args(PlanHolder& P, int R, int maxit) {
    BatchState& bt = P.batch;
    BatchPcgArgs a{};
    a.n = P.n;
    a.npix = P.npix_obs;
    a.R = R;
    a.maxit = maxit;
    a.x = bt.x;
    a.r = bt.r;
    a.p = bt.p;
    a.q = bt.q;
    a.z = bt.z;
    a.bd = P.bd32;
    a.partial = bt.partial;
    a.rho = bt.rho;
    a.bb = bt.bb;
    a.rr = bt.rr;
    a.tol2 = bt.tol2;
    a.iters = bt.iters;
    a.state = bt.state;
    a.flags = bt.flags;
    a.bar = bt.bar;
    a.bar_absent = P.bar_absent;
    a.wait_ns = P.bar_wait_ns;
    return a;
}

// One batched PCG run on the right-hand sides in batch.r (FP32); iterations are replayed
// from a captured CUDA graph of `chunk` iterations when capture works on this stream.
static void run_batch_pcg(PlanHolder& P, int R, int maxit) {
    BatchState& bt = P.batch;
    cudaStream_t s = P.stream;
    const BatchPcgArgs a = batch_pcg_args(P, R, maxit);
    check_cuda(cudaMemsetAsync(bt.flags, 0, 32, s), "memset flags");
    check_cuda(cudaMemsetAsync(bt.state, 0, BATCH_RMAX, s), "memset state");
    check_cuda(cudaMemsetAsync(bt.bar, 0, sizeof(unsigned), s), "memset barrier");
    launch_batch_pcg(0, P.ncomp, a, bt.nblocks, s);
    constexpr int kChunk = 4;
    auto body = [&]() {
        for (int i = 0; i < kChunk; ++i) {
            apply_A_batch(P, R, bt.p, bt.q, bt.flags + F_DONE);
            launch_batch_pcg(1, P.ncomp, a, bt.nblocks, s);
        }
    };
    // the graph is keyed on R and maxit (kernel arguments are captured by value)
    if (bt.graph != nullptr && (bt.graph_R != R || bt.graph_maxit != maxit)) {
        (void)cudaGraphExecDestroy(bt.graph);
        bt.graph = nullptr;
    }
    if (bt.graph == nullptr && !bt.graph_failed && s != nullptr) {
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            bool ok = true;
            try {
                body();
            } catch (const Error&) {
                ok = false;
            }
            const cudaError_t e = cudaStreamEndCapture(s, &g);
            ok = ok && e == cudaSuccess && g != nullptr;
            if (ok && cudaGraphInstantiate(&bt.graph, g, 0) != cudaSuccess) {
                bt.graph = nullptr;
                ok = false;
            }
            if (g) (void)cudaGraphDestroy(g);
            if (!ok) bt.graph_failed = true;
        } else {
            bt.graph_failed = true;
        }
        (void)cudaGetLastError();
        bt.graph_R = R;
        bt.graph_maxit = maxit;
    }
    int launched = 0;
    int h_flags[4];
    while (true) {
        d2h(h_flags, bt.flags, 16, s);
        sync(s);
        if (h_flags[F_DONE] || launched > maxit) break;
        if (bt.graph != nullptr) {
            check_cuda(cudaGraphLaunch(bt.graph, s), "graph launch");
            note_launch(3 * kChunk);
        } else {
            body();
        }
        launched += kChunk;
    }
}

static void solve_batch(PlanHolder& P, const double* D, int R, const mm_solve_opts& so, double* M, mm_stats* st) {
    cudaStream_t s = P.stream;
    if (R < 1) throw Error{MM_ERR_ARG, "R must be >= 1"};
    check_solve_opts(P, so);
    if (so.solver != MM_SOLVE_MIXED || so.kind != MM_PREC_BD)
        throw Error{MM_ERR_ARG, "the batched solver runs MM_SOLVE_MIXED with MM_PREC_BD"};
    const int RB = std::min(R, BATCH_RMAX);
    ensure_batch_buffers(P, RB);
    ensure_batch_tables(P, RB);
    BatchState& bt = P.batch;
    const bool d_dev = is_device_ptr(D), m_dev = is_device_ptr(M);
    const size_t n = (size_t)P.n, nt = (size_t)P.nt;
    const int max_outer = so.max_outer > 0 ? so.max_outer : 20;
    const double inner_min = so.inner_tol_min > 0.0 ? so.inner_tol_min : 3e-7;
    int overall = MM_OK;
    for (int c0 = 0; c0 < R; c0 += RB) {
        const int Rc = std::min(RB, R - c0);
        check_cuda(cudaEventRecord(P.ev0, s), "event");
        std::vector<double> bb(Rc), rr(Rc);
        std::vector<int> iters(Rc, 0), outer(Rc, 0), fp64(Rc, 0);
        // the group's data on the device (host data copied once; the FP64 residuals read it
        // again every refinement step)
        const double* Dg = D + (size_t)c0 * nt;
        double* Dtmp = nullptr;
        if (!d_dev) {
            Dtmp = dalloc<double>((size_t)Rc * nt);
            h2d(Dtmp, Dg, (size_t)Rc * nt * 8, s);
            Dg = Dtmp;
        }
        std::unique_ptr<double, void (*)(double*)> dguard(Dtmp, [](double* q) { dfree(q); });
        // b_r = P^T N^-1 d_r in FP32 for all columns in one batched Toeplitz launch (it seeds
        // the first inner solve and scales the residual; the FP64 residuals come from the
        // data, residual64)
        launch_toeplitz_any<float>(P, P.tz32, nullptr, Dg, nullptr, Rc, (int64_t)nt, bt.tod, (int64_t)nt, nullptr, s);
        launch_batch_scatter(P, bt.tod, bt.z, Rc, nullptr, s);
        launch_convert_f32_to_f64(bt.z, bt.b64, (int64_t)Rc * n, s);
        for (int r = 0; r < Rc; ++r) {
            bb[(size_t)r] = dot64(P, bt.b64 + (size_t)r * n, bt.b64 + (size_t)r * n);
            rr[(size_t)r] = bb[(size_t)r];
        }
        check_cuda(cudaMemsetAsync(bt.x64, 0, n * Rc * 8, s), "memset x");
        check_cuda(cudaMemcpyAsync(bt.r64, bt.b64, n * Rc * 8, cudaMemcpyDeviceToDevice, s), "copy b");
        int total = 0;
        for (int o = 0; o < max_outer; ++o) {
            std::vector<double> tol2(BATCH_RMAX, 0.0), nrm(Rc, 0.0);
            bool any = false;
            for (int r = 0; r < Rc; ++r) {
                const bool act = bb[(size_t)r] > 0.0 && std::sqrt(rr[(size_t)r]) > so.tol * std::sqrt(bb[(size_t)r]);
                float* r32 = bt.r + (size_t)r * n;
                if (act) {
                    any = true;
                    nrm[(size_t)r] = std::sqrt(rr[(size_t)r]);
                    launch_scale_f32(bt.r64 + (size_t)r * n, 1.0 / nrm[(size_t)r], r32, (int64_t)n, s);
                    double ti = 0.5 * so.tol * std::sqrt(bb[(size_t)r]) / nrm[(size_t)r];
                    ti = std::min(0.5, std::max(ti, inner_min));
                    if (o == 0 && so.first_inner_tol > 0.0) ti = so.first_inner_tol;
                    tol2[(size_t)r] = ti * ti;
                } else {
                    check_cuda(cudaMemsetAsync(r32, 0, n * 4, s), "memset r");
                }
            }
            if (!any || total >= so.maxit) break;
            h2d(bt.tol2, tol2.data(), BATCH_RMAX * 8, s);
            run_batch_pcg(P, Rc, so.maxit - total);
            std::vector<int> it(BATCH_RMAX);
            std::vector<unsigned char> stt(BATCH_RMAX);
            d2h(it.data(), bt.iters, BATCH_RMAX * 4, s);
            d2h(stt.data(), bt.state, BATCH_RMAX, s);
            sync(s);
            int mx = 0;
            for (int r = 0; r < Rc; ++r) {
                if (nrm[(size_t)r] == 0.0) continue;
                if (stt[(size_t)r] == 3) throw Error{MM_ERR_NOT_SPD, "batched PCG breakdown"};
                iters[(size_t)r] += it[(size_t)r];
                mx = std::max(mx, it[(size_t)r]);
                outer[(size_t)r] += 1;
                fp64[(size_t)r] += 1;
                double* x64 = bt.x64 + (size_t)r * n;
                launch_axpy_host(x64, bt.x + (size_t)r * n, nrm[(size_t)r], (int64_t)n, s);
                residual64(P, Dg + (size_t)r * nt, x64, bt.r64 + (size_t)r * n, so.residual != MM_RESID_FP64);
                rr[(size_t)r] = dot64(P, bt.r64 + (size_t)r * n, bt.r64 + (size_t)r * n);
            }
            total += mx;
        }
        for (int r = 0; r < Rc; ++r) {
            double* mr = M + (size_t)(c0 + r) * n;
            if (m_dev) check_cuda(cudaMemcpyAsync(mr, bt.x64 + (size_t)r * n, n * 8, cudaMemcpyDeviceToDevice, s), "copy m");
            else d2h(mr, bt.x64 + (size_t)r * n, n * 8, s);
        }
        check_cuda(cudaEventRecord(P.ev2, s), "event");
        sync(P);
        float ms = 0.f;
        check_cuda(cudaEventElapsedTime(&ms, P.ev0, P.ev2), "event time");
        for (int r = 0; r < Rc; ++r) {
            mm_stats x{};
            x.iters = iters[(size_t)r];
            x.outer = outer[(size_t)r];
            x.fp64_products = fp64[(size_t)r];
            // NaN or Inf in a column's data reaches its b (and it then never runs) or its
            // residual: reported, never taken for a converged zero map
            const bool finite = std::isfinite(bb[(size_t)r]) && std::isfinite(rr[(size_t)r]);
            x.rel_resid = !finite ? std::nan("")
                                  : (bb[(size_t)r] > 0 ? std::sqrt(rr[(size_t)r] / bb[(size_t)r]) : 0.0);
            x.converged = finite && x.rel_resid <= so.tol;
            x.ms_total = ms / Rc;
            if (!finite) overall = MM_ERR_NUMERIC;
            else if (!x.converged && overall == MM_OK) overall = MM_ERR_NOT_CONVERGED;
            if (st) st[c0 + r] = x;
        }
    }
    if (overall == MM_ERR_NUMERIC) throw Error{MM_ERR_NUMERIC, "NaN or Inf in a right-hand side or residual"};
    if (overall != MM_OK) throw Error{(mm_status)overall, "some right-hand sides did not reach tol"};
}

}  // namespace mm

// ================================================================== C entry points
using namespace mm;

namespace {
template <typename F>
mm_status guarded(mm_plan_t plan, F&& f) {
    PlanHolder* P = reinterpret_cast<PlanHolder*>(plan);
    try {
        f();
        return MM_OK;
    } catch (const Error& e) {
        if (P) P->err = e.msg;
        g_last_error = e.msg;
        return e.st;
    } catch (const std::bad_alloc&) {
        if (P) P->err = "host allocation failed";
        g_last_error = "host allocation failed";
        return MM_ERR_OOM;
    } catch (const std::exception& e) {
        if (P) P->err = e.what();
        g_last_error = e.what();
        return MM_ERR_ARG;
    }
}

}  // namespace

mm_status mm::run_guarded(Plan* P, void (*f)(void*), void* ctx) {
    return guarded(reinterpret_cast<mm_plan_t>(static_cast<PlanHolder*>(P)), [&] { f(ctx); });
}

namespace {
PlanHolder* get(mm_plan_t p) {
    if (p == nullptr) throw Error{MM_ERR_ARG, "null plan"};
    return reinterpret_cast<PlanHolder*>(p);
}

int prec_ok(int precision) {
    if (precision != MM_FP64 && precision != MM_FP32) throw Error{MM_ERR_ARG, "precision must be MM_FP64 or MM_FP32"};
    return precision;
}
}  // namespace

extern "C" {

mm_status mm_plan(mm_plan_t* out, const int32_t* pix, int64_t nt, int32_t npix_sky, const double* weights,
                  const int64_t* interval_off, int32_t K, const int32_t* interval_psd, const mm_psd* psd,
                  int32_t npsd, const mm_opts* opts) {
    if (out == nullptr) return MM_ERR_ARG;
    *out = nullptr;
    PlanHolder* P = nullptr;
    try {
        P = new PlanHolder();
        build_plan(*P, pix, nt, npix_sky, weights, interval_off, K, interval_psd, psd, npsd, opts);
        *out = reinterpret_cast<mm_plan_t>(P);
        return MM_OK;
    } catch (const Error& e) {
        g_last_error = e.msg;
        destroy_plan(P);
        return e.st;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        destroy_plan(P);
        return MM_ERR_OOM;
    } catch (const std::exception& e) {   // nothing may leave an extern "C" function
        g_last_error = e.what();
        destroy_plan(P);
        return MM_ERR_ARG;
    }
}

mm_status mm_plan_info(mm_plan_t plan, int32_t* npix_obs, int64_t* n, int64_t* nkept, int32_t* fft_block_f64,
                       int32_t* fft_block_f32) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (npix_obs) *npix_obs = P->npix_obs;
        if (n) *n = P->n;
        if (nkept) *nkept = P->nkept;
        if (fft_block_f64) *fft_block_f64 = P->tz64.logn ? 2 << P->tz64.logn : 0;
        if (fft_block_f32) *fft_block_f32 = P->tz32.logn ? 2 << P->tz32.logn : 0;
    });
}

mm_status mm_plan_pixels(mm_plan_t plan, int32_t* obs2sky, int32_t* hits) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        const size_t bytes = (size_t)P->npix_obs * 4;
        for (auto pr : {std::make_pair(obs2sky, &P->h_obs2sky), std::make_pair(hits, &P->h_hits)}) {
            if (pr.first == nullptr) continue;
            if (is_device_ptr(pr.first))
                check_cuda(cudaMemcpy(pr.first, pr.second->data(), bytes, cudaMemcpyHostToDevice), "copy");
            else
                std::memcpy(pr.first, pr.second->data(), bytes);
        }
    });
}

mm_status mm_plan_row(mm_plan_t plan, int32_t psd_id, double* row) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (row == nullptr || psd_id < 0 || psd_id >= P->npsd) throw Error{MM_ERR_ARG, "bad psd id or null row"};
        std::memcpy(row, P->rows[(size_t)psd_id].data(), ((size_t)P->lambda + 1) * 8);
    });
}

mm_status mm_gather(mm_plan_t plan, int precision, const void* x, void* y) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!x || !y) throw Error{MM_ERR_ARG, "null vector"};
        if (prec_ok(precision) == MM_FP64)
            launch_gather<double>(*P, static_cast<const double*>(x), static_cast<double*>(y), P->stream);
        else
            launch_gather<float>(*P, static_cast<const float*>(x), static_cast<float*>(y), P->stream);
        sync(P->stream);
    });
}

mm_status mm_apply_ninv(mm_plan_t plan, int precision, const void* y, void* z) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!y || !z) throw Error{MM_ERR_ARG, "null vector"};
        if (prec_ok(precision) == MM_FP64)
            launch_toeplitz<double>(*P, P->tz64, static_cast<const double*>(y), nullptr, static_cast<double*>(z), nullptr,
                                    P->stream);
        else
            launch_toeplitz<float>(*P, P->tz32, static_cast<const float*>(y), nullptr, static_cast<float*>(z), nullptr,
                                   P->stream);
        sync(P->stream);
    });
}

mm_status mm_scatter(mm_plan_t plan, int precision, const void* z, void* w) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!z || !w) throw Error{MM_ERR_ARG, "null vector"};
        if (prec_ok(precision) == MM_FP64)
            launch_scatter<double>(*P, static_cast<const double*>(z), static_cast<double*>(w), nullptr, P->stream);
        else
            launch_scatter<float>(*P, static_cast<const float*>(z), static_cast<float*>(w), nullptr, P->stream);
        sync(P->stream);
    });
}

mm_status mm_apply_A(mm_plan_t plan, int precision, const void* x, void* y) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!x || !y) throw Error{MM_ERR_ARG, "null vector"};
        if (prec_ok(precision) == MM_FP64)
            apply_A<double>(*P, static_cast<const double*>(x), static_cast<double*>(y), nullptr);
        else
            apply_A<float>(*P, static_cast<const float*>(x), static_cast<float*>(y), nullptr);
        sync(*P);
    });
}

mm_status mm_profile(mm_plan_t plan, int enable) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        sync(*P);
        P->prof.on = enable != 0;
        for (int i = 0; i < ST_COUNT; ++i) {
            P->prof.ms[i] = 0.0;
            P->prof.launches[i] = 0;
        }
    });
}

mm_status mm_profile_read(mm_plan_t plan, double* ms, int64_t* launches) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        sync(*P);
        for (int i = 0; i < ST_COUNT; ++i) {
            if (ms) ms[i] = P->prof.ms[i];
            if (launches) launches[i] = P->prof.launches[i];
        }
    });
}

mm_status mm_rhs(mm_plan_t plan, const double* d, double* b) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!d || !b) throw Error{MM_ERR_ARG, "null vector"};
        launch_toeplitz<double>(*P, P->tz64, d, nullptr, P->tod64, nullptr, P->stream);
        launch_scatter<double>(*P, P->tod64, b, nullptr, P->stream);
        sync(P->stream);
    });
}

mm_status mm_precond(mm_plan_t plan, int kind, int precision, const void* r, void* z) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!r || !z) throw Error{MM_ERR_ARG, "null vector"};
        if (kind != MM_PREC_BD && kind != MM_PREC_TWOLEVEL && kind != MM_PREC_ADEF2)
            throw Error{MM_ERR_ARG, "bad preconditioner kind"};
        const int cm = coarse_mode(kind);
        const bool two = cm != 0;
        if (two && P->coarse.k == 0) throw Error{MM_ERR_STATE, "two-level preconditioner needs mm_build_coarse"};
        check_cuda(cudaMemsetAsync(P->pcg.barrier, 0, sizeof(unsigned), P->stream), "memset barrier");
        if (prec_ok(precision) == MM_FP64) {
            PcgArgs<double> a = pcg_args<double>(*P, two, 0);
            a.r = const_cast<double*>(static_cast<const double*>(r));
            a.z = static_cast<double*>(z);
            launch_pcg<double>(2, P->ncomp, cm, a, P->pcg.nblocks, P->stream);
        } else {
            PcgArgs<float> a = pcg_args<float>(*P, two, 0);
            a.r = const_cast<float*>(static_cast<const float*>(r));
            a.z = static_cast<float*>(z);
            launch_pcg<float>(2, P->ncomp, cm, a, P->pcg.nblocks, P->stream);
        }
        sync(P->stream);
    });
}

mm_status mm_build_coarse(mm_plan_t plan, int k, int precision, const double* bprime, double tol, int maxit) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (prec_ok(precision) == MM_FP64)
            build_coarse<double>(*P, k, bprime, tol, maxit);
        else
            build_coarse<float>(*P, k, bprime, tol, maxit);
    });
}

mm_status mm_build_coarse_eps(mm_plan_t plan, int kmax, double eps_tol, int precision, const double* bprime,
                              double tol, int maxit) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!(eps_tol > 0.0)) throw Error{MM_ERR_ARG, "eps_tol must be > 0"};
        if (prec_ok(precision) == MM_FP64)
            build_coarse<double>(*P, kmax, bprime, tol, maxit, eps_tol);
        else
            build_coarse<float>(*P, kmax, bprime, tol, maxit, eps_tol);
    });
}

mm_status mm_coarse_import(mm_plan_t plan, const double* Z, int k) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (Z == nullptr || k < 1 || k > KMAX) throw Error{MM_ERR_ARG, "need non-null Z and 1 <= k <= 64"};
        double* Zd = dalloc<double>((size_t)k * P->n);
        int kc = k;
        try {
            check_cuda(cudaMemcpyAsync(Zd, Z, (size_t)k * P->n * 8, cudaMemcpyDefault, P->stream), "copy Z");
            orthonormalise_drop(*P, Zd, kc);
        } catch (...) {
            dfree(Zd);
            throw;
        }
        install_coarse(*P, Zd, kc, {});
    });
}

mm_status mm_build_coarse_arnoldi(mm_plan_t plan, int kmax, double eps_tol, const double* bprime, double tol,
                                  int maxit) {
    return guarded(plan, [&] { build_coarse_arnoldi(*get(plan), kmax, eps_tol, bprime, tol, maxit); });
}

mm_status mm_build_coarse_apriori(mm_plan_t plan, int r) {
    return guarded(plan, [&] { build_coarse_apriori(*get(plan), r); });
}

mm_status mm_coarse_info(mm_plan_t plan, int32_t* k_kept, double* ritz_values) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (k_kept) *k_kept = P->coarse.k;
        if (ritz_values) {
            const size_t m = std::min(P->coarse.ritz.size(), (size_t)P->coarse.k);
            std::copy(P->coarse.ritz.begin(), P->coarse.ritz.begin() + (std::ptrdiff_t)m, ritz_values);
        }
    });
}

mm_status mm_coarse_vectors(mm_plan_t plan, double* Z) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (P->coarse.k == 0) throw Error{MM_ERR_STATE, "no coarse space"};
        if (Z == nullptr) throw Error{MM_ERR_ARG, "null output"};
        check_cuda(cudaMemcpy(Z, P->coarse.Z64, (size_t)P->coarse.k * P->n * 8, cudaMemcpyDefault), "copy Z");
    });
}

mm_status mm_residual(mm_plan_t plan, int arith, const double* d, const double* x, double* r) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!d || !x || !r) throw Error{MM_ERR_ARG, "null vector"};
        if (arith != MM_RESID_DF32 && arith != MM_RESID_FP64) throw Error{MM_ERR_ARG, "bad residual arithmetic"};
        if (P->tz64.logn == 0) throw Error{MM_ERR_ARG, "no FP64 Toeplitz block fits this lambda"};
        residual64(*P, d, x, r, arith == MM_RESID_DF32);
        sync(*P);
    });
}

mm_status mm_pcg_barrier_check(mm_plan_t plan, int32_t absent_blocks, double wait_s) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (absent_blocks < 0 || absent_blocks > 1024 || !(wait_s > 0.0) || !(wait_s <= 10.0))
            throw Error{MM_ERR_ARG, "need 0 <= absent_blocks <= 1024 and 0 < wait_s <= 10"};
        P->bar_absent = (unsigned)absent_blocks;
        P->bar_wait_ns = (unsigned long long)(wait_s * 1e9);
        try {
            check_cuda(cudaMemsetAsync(P->pcg.r, 0, (size_t)P->n * 8, P->stream), "memset r");
            (void)run_pcg<double>(*P, 0, 0.0, 1, nullptr, 0, 0);
        } catch (...) {
            P->bar_absent = 0;
            P->bar_wait_ns = BARRIER_WAIT_NS;
            throw;
        }
        P->bar_absent = 0;
        P->bar_wait_ns = BARRIER_WAIT_NS;
    });
}

mm_status mm_solve_history(mm_plan_t plan, int32_t max, double* rel_resid, int32_t* count) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (max < 0) throw Error{MM_ERR_ARG, "max must be >= 0"};
        std::vector<double> out;
        if (!P->hist_runs.empty() && P->pcg.hist_rr != nullptr) {
            const PlanHolder::HistRun& last = P->hist_runs.back();
            const int len = std::min(last.off + last.iters + 1, P->pcg.maxhist);
            std::vector<double> h((size_t)std::max(len, 0));
            d2h(h.data(), P->pcg.hist_rr, h.size() * 8, P->stream);
            sync(P->stream);
            // entry 0 of the first run, then steps 1..iters of every run
            for (size_t r = 0; r < P->hist_runs.size(); ++r) {
                const PlanHolder::HistRun& run = P->hist_runs[r];
                for (int j = r == 0 ? 0 : 1; j <= run.iters && run.off + j < len; ++j)
                    out.push_back(run.bb == 0.0 ? run.scale : std::sqrt(h[(size_t)(run.off + j)] / run.bb) * run.scale);
            }
        }
        if (count) *count = (int32_t)out.size();
        if (rel_resid) std::copy(out.begin(), out.begin() + (std::ptrdiff_t)std::min<size_t>((size_t)max, out.size()),
                                 rel_resid);
    });
}

mm_status mm_solve(mm_plan_t plan, const double* d, double tol, int maxit, int kind, int solver, double* m,
                   mm_stats* st) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!d || !m) throw Error{MM_ERR_ARG, "null vector"};
        mm_solve_opts o{};
        o.tol = tol;
        o.maxit = maxit;
        o.kind = kind;
        o.solver = solver;
        solve(*P, d, o, m, st);
    });
}

mm_status mm_solve_ex(mm_plan_t plan, const double* d, const mm_solve_opts* opts, double* m, mm_stats* st) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!d || !m || !opts) throw Error{MM_ERR_ARG, "null argument"};
        solve(*P, d, *opts, m, st);
    });
}

mm_status mm_grad(mm_plan_t plan, const double* d, const double* m, const double* g, double* dL_dd,
                  double* dL_dpsd, const mm_solve_opts* opts, mm_stats* st) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!d || !m || !g || !opts) throw Error{MM_ERR_ARG, "null argument"};
        grad(*P, d, m, g, dL_dd, dL_dpsd, *opts, st);
    });
}

mm_status mm_autotune_read(mm_plan_t plan, float* ms_f64, float* ms_f32) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (ms_f64) std::memcpy(ms_f64, P->tuned_ms64, sizeof(P->tuned_ms64));
        if (ms_f32) std::memcpy(ms_f32, P->tuned_ms32, sizeof(P->tuned_ms32));
    });
}

mm_status mm_scatter_config(mm_plan_t plan, int32_t* lanes_per_pixel, float* ms) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (lanes_per_pixel) *lanes_per_pixel = P->scatter_lpp;
        if (ms) std::memcpy(ms, P->tuned_scatter_ms, sizeof(P->tuned_scatter_ms));
    });
}

mm_status mm_batch_config(mm_plan_t plan, int32_t R, int32_t* kind, int32_t* log2_block, float* ms) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (R < 1 || R > BATCH_RMAX) throw Error{MM_ERR_ARG, "need 1 <= R <= 64"};
        if (kind == nullptr || *kind < -1 || *kind > 2) throw Error{MM_ERR_ARG, "kind must point to -1, 0, 1 or 2"};
        ensure_batch_buffers(*P, R);
        ensure_batch_tables(*P, R, *kind);
        sync(*P);
        const BatchState& bt = P->batch;
        *kind = bt.kind;
        if (log2_block) *log2_block = bt.kind == BATCH_REAL ? P->tz32.logn + 1 : (bt.kind == BATCH_TENSOR ? 7 : bt.logb);
        if (ms) {
            ms[0] = bt.tuned_ms[0];
            ms[1] = bt.tuned_ms[1];
            ms[2] = bt.tuned_ms[2];
        }
    });
}

mm_status mm_apply_A_batch(mm_plan_t plan, int R, const float* X, float* Y) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!X || !Y || R < 1 || R > BATCH_RMAX) throw Error{MM_ERR_ARG, "need 1 <= R <= 64 and non-null X, Y"};
        ensure_batch_buffers(*P, R);
        ensure_batch_tables(*P, R);
        apply_A_batch(*P, R, X, Y, nullptr);
        sync(*P);
    });
}

mm_status mm_solve_batch(mm_plan_t plan, const double* D, int R, const mm_solve_opts* opts, double* M,
                         mm_stats* st) {
    return guarded(plan, [&] {
        PlanHolder* P = get(plan);
        if (!D || !M || !opts) throw Error{MM_ERR_ARG, "null argument"};
        solve_batch(*P, D, R, *opts, M, st);
    });
}

const char* mm_last_error(mm_plan_t plan) {
    if (plan != nullptr) {
        const PlanHolder* P = reinterpret_cast<const PlanHolder*>(plan);
        if (!P->err.empty()) return P->err.c_str();
    }
    return g_last_error.c_str();
}

void mm_destroy(mm_plan_t plan) { destroy_plan(reinterpret_cast<PlanHolder*>(plan)); }

const char* mm_version(void) { return "libmm 0.1 (sm_103a)"; }

int64_t mm_launch_count(void) { return g_launches.load(); }

}  // extern "C"
