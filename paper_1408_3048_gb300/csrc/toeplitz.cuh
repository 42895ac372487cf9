// Banded block-Toeplitz N^-1 by overlap-save FFT in shared memory (Eq. 4; band of
// Sec. 4.1.4; FFT product of Sec. 2.1).  Included by toeplitz_f64.cu / toeplitz_f32.cu.
//
// One CTA per overlap-save tile.  A tile holds B = 2N real positions filled from up to
// three segments of consecutive stationary intervals of one PSD (zeros between and
// around them, at least lambda between two intervals: see Tile),
// packs them as N complex values u_m = y_2m + i y_2m+1, runs an N-point complex FFT,
// turns that into the spectrum of the real block (real-FFT post-processing), multiplies
// by the real spectrum H of the even kernel (t_|k| for |k| <= lambda, laid out
// circularly over B), converts back to the packed N-point form and inverts with the
// same forward FFT (conjugation trick).  Outputs [lambda, lambda + nout) of the block
// equal the truncated band product exactly (no wrap-around reaches them when
// nout <= B - 2 lambda).
//
// FFT: Stockham autosort, radix-16 passes (radix 8 for blocks below 2^10 reals) and one
// shorter pass where the length asks for it, data in shared
// memory with one padding slot after every 16 complex values so that the strided stores
// of a pass are free of bank conflicts, butterflies of a pass held in registers (in
// place, with barriers).  Twiddles: FP32 computes them in registers (sincospif and a few
// products); FP64 and double-float read the per-pass tables and a quarter-wave cosine
// table cos(2 pi k / B), k = 0..B/4 (host-computed in FP64), the latter staged in
// shared memory.
//
// The tile load can evaluate y = P x on the fly from the map (fused de-pointing); the
// FP32 I/Q/U form reads the map packed per pixel (one 16-byte load per sample).
#pragma once

#include <atomic>
#include <type_traits>
#include <cooperative_groups.h>

#include "dfloat.cuh"
#include "mm_internal.h"

namespace mm {

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<dfl> { using type = dfl2; };

// Type of the arrays a kernel of arithmetic T reads and writes: the double-float kernel
// works on FP64 data.
template <typename T> struct InT { using type = T; };
template <> struct InT<dfl> { using type = double; };
template <typename T> using In = typename InT<T>::type;

// Read-only load of a complex table entry.
// Input-precision value -> arithmetic type and back (bit-level for double-float).
template <typename T>
__device__ __forceinline__ T from_in(In<T> v) {
    if constexpr (sizeof(T) == 8 && !std::is_same<T, double>::value) return dfl_from_double(v);
    else return (T)v;
}
template <typename T>
__device__ __forceinline__ In<T> to_in(T v) {
    if constexpr (sizeof(T) == 8 && !std::is_same<T, double>::value) return dfl_to_double(v);
    else return (In<T>)v;
}

__device__ __forceinline__ float2 ldc(const float2* p) { return __ldg(p); }
__device__ __forceinline__ double2 ldc(const double2* p) { return __ldg(p); }
__device__ __forceinline__ dfl2 ldc(const dfl2* p) {
    const float4 f = __ldg(reinterpret_cast<const float4*>(p));
    return dfl2{dfl(f.x, f.y), dfl(f.z, f.w)};
}

template <typename T>
struct TzArgs {
    const Tile* tiles;
    const T* twiddle;      // [N/2 + 1]: cos(2 pi k / B), real-FFT split
    const typename Cx<T>::type* ptw;  // per-pass FFT twiddles (ptw_offset)
    const T* H;            // [npsd][N + 1]
    const In<T>* y;        // time-domain input (mode 0)
    const double* yd;      // FP64 time-domain input (modes 2, 4, 5)
    const In<T>* x;        // map (gather modes)
    const int32_t* pixc;   // [nt]
    const typename Cx<In<T>>::type* w;  // [nt] (cos, sin) for ncomp = 3
    In<T>* z;              // [nt] output
    const int* done;       // early-exit flag (PCG) or nullptr
    int lambda;
    int R;                 // right-hand sides (grid: tile-major, RHS fastest)
    int64_t in_stride;     // elements between RHS in y (mode 0) or x (gather modes)
    int64_t out_stride;    // elements between RHS in z
    int pf_ahead = 0;      // CTAs resident at once: L2 prefetch distance (0: no prefetch)
    const float4* x4 = nullptr;   // FP32 I/Q/U map packed per pixel (mode 3), else nullptr
};

// (tile, RHS) of a CTA (or cluster) index: RHS fastest, so the R CTAs of one tile read
// its pointing from L2 after the first.
struct TileRhs {
    int tile;
    int rhs;
};
__device__ __forceinline__ TileRhs tile_rhs(int cid, int R) {
    if (R == 1) return {cid, 0};
    return {cid / R, cid % R};
}

template <typename T>
__device__ __forceinline__ typename Cx<T>::type cmul(typename Cx<T>::type a, T c, T s) {
    // a * (c - i s)
    typename Cx<T>::type r;
    r.x = a.x * c + a.y * s;
    r.y = a.y * c - a.x * s;
    return r;
}

// cos / sin of 2 pi m / B from the quarter table (Q = B/4 entries + 1).
template <typename T, int LOGQ>
__device__ __forceinline__ void twiddle(const T* tab, int m, T& c, T& s) {
    constexpr int Q = 1 << LOGQ;
    const int q = (m >> LOGQ) & 3;
    const int r = m & (Q - 1);
    const T cr = tab[r];
    const T sr = tab[Q - r];
    switch (q) {
        case 0: c = cr; s = sr; break;
        case 1: c = -sr; s = cr; break;
        case 2: c = -cr; s = -sr; break;
        default: c = sr; s = -cr; break;
    }
}

template <typename T>
__device__ __forceinline__ void bfly2(typename Cx<T>::type& a, typename Cx<T>::type& b) {
    typename Cx<T>::type t = a;
    a.x = t.x + b.x; a.y = t.y + b.y;
    b.x = t.x - b.x; b.y = t.y - b.y;
}


template <typename T>
__device__ __forceinline__ void dft4(typename Cx<T>::type& a0, typename Cx<T>::type& a1,
                                     typename Cx<T>::type& a2, typename Cx<T>::type& a3) {
    // forward 4-point DFT, outputs in natural order in (a0, a1, a2, a3)
    typename Cx<T>::type t0, t1, t2, t3;
    t0.x = a0.x + a2.x; t0.y = a0.y + a2.y;
    t1.x = a0.x - a2.x; t1.y = a0.y - a2.y;
    t2.x = a1.x + a3.x; t2.y = a1.y + a3.y;
    // (a1 - a3) * (-i)
    t3.x = a1.y - a3.y; t3.y = a3.x - a1.x;
    a0.x = t0.x + t2.x; a0.y = t0.y + t2.y;
    a2.x = t0.x - t2.x; a2.y = t0.y - t2.y;
    a1.x = t1.x + t3.x; a1.y = t1.y + t3.y;
    a3.x = t1.x - t3.x; a3.y = t1.y - t3.y;
}


template <typename T>
__device__ __forceinline__ void dft8(typename Cx<T>::type* v) {
    using C2 = typename Cx<T>::type;
    const T h = (T)0.70710678118654752440084436210484903928;  // sqrt(1/2)
    C2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<T>(e0, e1, e2, e3);
    dft4<T>(o0, o1, o2, o3);
    // o_k *= W8^k, W8 = exp(-2 pi i / 8)
    C2 t;
    t.x = h * (o1.x + o1.y); t.y = h * (o1.y - o1.x); o1 = t;        // (1 - i)/sqrt2
    t.x = o2.y; t.y = -o2.x; o2 = t;                                   // -i
    t.x = h * (o3.y - o3.x); t.y = -h * (o3.x + o3.y); o3 = t;        // (-1 - i)/sqrt2
    v[0].x = e0.x + o0.x; v[0].y = e0.y + o0.y;
    v[4].x = e0.x - o0.x; v[4].y = e0.y - o0.y;
    v[1].x = e1.x + o1.x; v[1].y = e1.y + o1.y;
    v[5].x = e1.x - o1.x; v[5].y = e1.y - o1.y;
    v[2].x = e2.x + o2.x; v[2].y = e2.y + o2.y;
    v[6].x = e2.x - o2.x; v[6].y = e2.y - o2.y;
    v[3].x = e3.x + o3.x; v[3].y = e3.y + o3.y;
    v[7].x = e3.x - o3.x; v[7].y = e3.y - o3.y;
}


// 16-point DFT as 4 x 4: DFT4 over n1 of x[4 n1 + n2], twiddle W16^(n2 k1), DFT4 over
// n2; outputs in natural order.  (c, s) below are cos and sin of 2 pi m / 16.
template <typename T>
__device__ __forceinline__ void dft16(typename Cx<T>::type* v) {
    using C2 = typename Cx<T>::type;
    const T C1 = (T)0.92387953251128675613, S1 = (T)0.38268343236508977173, H = (T)0.70710678118654752440;
    C2 y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        C2 a0 = v[n2], a1 = v[4 + n2], a2 = v[8 + n2], a3 = v[12 + n2];
        dft4<T>(a0, a1, a2, a3);
        y[n2][0] = a0;
        y[n2][1] = a1;
        y[n2][2] = a2;
        y[n2][3] = a3;
    }
    // W16^(n2 k1): (1,1):m1 (1,2):m2 (1,3):m3 (2,1):m2 (2,2):m4 (2,3):m6 (3,1):m3 (3,2):m6 (3,3):m9
    y[1][1] = cmul<T>(y[1][1], C1, S1);
    y[1][2] = cmul<T>(y[1][2], H, H);
    y[1][3] = cmul<T>(y[1][3], S1, C1);
    y[2][1] = cmul<T>(y[2][1], H, H);
    {
        const C2 t = y[2][2];   // * (-i)
        y[2][2].x = t.y;
        y[2][2].y = -t.x;
    }
    y[2][3] = cmul<T>(y[2][3], -H, H);
    y[3][1] = cmul<T>(y[3][1], S1, C1);
    y[3][2] = cmul<T>(y[3][2], -H, H);
    y[3][3] = cmul<T>(y[3][3], -C1, -S1);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C2 b0 = y[0][k1], b1 = y[1][k1], b2 = y[2][k1], b3 = y[3][k1];
        dft4<T>(b0, b1, b2, b3);
        v[k1] = b0;
        v[k1 + 4] = b1;
        v[k1 + 8] = b2;
        v[k1 + 12] = b3;
    }
}

// R-point forward DFT of v in place (natural order out).
template <typename T, int R>
__device__ __forceinline__ void dft(typename Cx<T>::type* v) {
    if constexpr (R == 2) bfly2<T>(v[0], v[1]);
    else if constexpr (R == 4) dft4<T>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<T>(v);
    else dft16<T>(v);
}

// Padding: one slot after every 16 elements, so the stride-16 stores of a first radix-16
// pass (thread j writes 16 j + r) hit distinct banks within every 128-byte wavefront for
// both 8-byte (float2) and 16-byte (double2) elements; the other passes are contiguous.
template <typename T> struct PadLog;
template <> struct PadLog<double> { static constexpr int v = 4; };
template <> struct PadLog<float> { static constexpr int v = 4; };
template <> struct PadLog<dfl> { static constexpr int v = 4; };

template <typename T>
__device__ __forceinline__ int pad(int i) { return i + (i >> PadLog<T>::v); }

// Largest radix of the passes: 16 when N/16 >= 32 threads can hold one butterfly each.
template <int LOGN>
__host__ __device__ constexpr int fft_max_logr() { return (1 << LOGN) / 16 >= 32 ? 4 : 3; }

// Per-pass twiddle table: pass p (Ns_p = 2^LOGNS, radix R_p) stores W_{Ns R}^{r k} as
// (cos, sin) of 2 pi r k / (Ns R) at [(r - 1) Ns + k], r = 1..R-1, k < Ns (consecutive
// threads read consecutive entries); the passes follow each other.  Offset of the pass
// that starts at LOGNS:
template <int LOGN>
__host__ __device__ constexpr int ptw_offset(int logns) {
    int off = 0, l = 0;
    while (l < logns) {
        const int rem = LOGN - l;
        const int lr = rem >= fft_max_logr<LOGN>() ? fft_max_logr<LOGN>() : rem;
        off += (1 << l) * ((1 << lr) - 1);
        l += lr;
    }
    return off;
}

// (c, s) pairs stand for c - i s = exp(-i theta); their product is another such pair.
__device__ __forceinline__ float2 tw_mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// FP32 pass twiddles computed in registers instead of read from a table: v[r] *= W^(r k)
// with W = exp(-2 pi i / (Ns R)) for r = 1..R-1, from sincospif at x = 2k / (Ns R) and
// 4x (exact scalings of an exact float): W^r = W^(4a) W^b, r = 4a + b, with W^2, W^3,
// W^8, W^12 formed by one or two products, so every twiddle is at most four roundings
// from the correctly rounded value.  (A table in global memory put an L2 load after
// every barrier of the FFT on the critical path.)
template <int R>
__device__ __forceinline__ void apply_twiddles_f32(float2* v, float x) {
    float s1, c1;
    sincospif(x, &s1, &c1);
    float2 w[4];
    w[0] = make_float2(1.f, 0.f);
    w[1] = make_float2(c1, s1);
    w[2] = tw_mul(w[1], w[1]);
    w[3] = tw_mul(w[1], w[2]);
#pragma unroll
    for (int b = 1; b < (R < 4 ? R : 4); ++b) v[b] = cmul<float>(v[b], w[b].x, w[b].y);
    if constexpr (R > 4) {
        float s4, c4;
        sincospif(4.f * x, &s4, &c4);
        float2 W[4];
        W[0] = make_float2(1.f, 0.f);
        W[1] = make_float2(c4, s4);
        W[2] = tw_mul(W[1], W[1]);
        W[3] = tw_mul(W[1], W[2]);
#pragma unroll
        for (int a = 1; a < R / 4; ++a) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float2 t = b == 0 ? W[a] : tw_mul(W[a], w[b]);
                v[4 * a + b] = cmul<float>(v[4 * a + b], t.x, t.y);
            }
        }
    }
}

// One in-place Stockham pass of radix R on N = 2^LOGN points (Ns = 2^LOGNS).
template <typename T, int LOGN, int NT, int LOGR, int LOGNS>
__device__ __forceinline__ void fft_pass(typename Cx<T>::type* a, const typename Cx<T>::type* ptw) {
    using C2 = typename Cx<T>::type;
    constexpr int N = 1 << LOGN;
    constexpr int R = 1 << LOGR;
    constexpr int NB = N >> LOGR;
    constexpr int BPT = NB / NT;
    constexpr int Ns = 1 << LOGNS;
    static_assert(BPT >= 1 && NB % NT == 0, "butterflies per thread");
    // pad(i + r S) = pad(i) + r (S + S/16) when S is a multiple of 16 (and, for S = 1,
    // when i is and r < 16): one base address per butterfly and constant offsets
    constexpr int PADL = 1 << PadLog<T>::v;
    constexpr bool LD_CONST = NB % PADL == 0;
    constexpr bool ST_CONST = Ns % PADL == 0 || (Ns == 1 && R <= PADL);
    constexpr int LD_STEP = NB + (NB >> PadLog<T>::v);
    constexpr int ST_STEP = Ns % PADL == 0 ? Ns + (Ns >> PadLog<T>::v) : 1;
    C2 v[BPT][R];
    const int tid = threadIdx.x;
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = tid + b * NT;
        if constexpr (LD_CONST) {
            const C2* src = a + pad<T>(j);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = src[r * LD_STEP];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) v[b][r] = a[pad<T>(j + r * NB)];
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < BPT; ++b) {
        const int j = tid + b * NT;
        const int k = j & (Ns - 1);
        if constexpr (LOGNS > 0) {
            if constexpr (sizeof(T) == 4) {
                apply_twiddles_f32<R>(v[b], (float)(2 * k) * (1.f / (float)(Ns * R)));
            } else {
                const C2* tw = ptw + ptw_offset<LOGN>(LOGNS) + k;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    const C2 w = ldc(tw + (r - 1) * Ns);
                    v[b][r] = cmul<T>(v[b][r], w.x, w.y);
                }
            }
        }
        dft<T, R>(v[b]);
        const int idx = ((j - k) << LOGR) + k;
        if constexpr (ST_CONST) {
            C2* dst = a + pad<T>(idx);
#pragma unroll
            for (int r = 0; r < R; ++r) dst[r * ST_STEP] = v[b][r];
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) a[pad<T>(idx + r * Ns)] = v[b][r];
        }
    }
    __syncthreads();
}

template <typename T, int LOGN, int NT, int LOGNS>
__device__ __forceinline__ void fft_all(typename Cx<T>::type* a, const typename Cx<T>::type* ptw) {
    if constexpr (LOGNS < LOGN) {
        constexpr int REM = LOGN - LOGNS;
        constexpr int MAXR = fft_max_logr<LOGN>();
        constexpr int LOGR = REM >= MAXR ? MAXR : REM;
        fft_pass<T, LOGN, NT, LOGR, LOGNS>(a, ptw);
        fft_all<T, LOGN, NT, LOGNS + LOGR>(a, ptw);
    }
}

// Segment of block position p in a tile (the segments ascend): g with pb[g] <= p, and
// whether p lies inside it (else it is a zero between or around the segments).
__device__ __forceinline__ int tile_seg(const Tile& tl, int p, bool& inside) {
    // selects, not indexing: a dynamically indexed Tile would be placed in local memory
    const int g = (p >= tl.pb[1]) + (p >= tl.pb[2]);
    const int b = g == 0 ? tl.pb[0] : (g == 1 ? tl.pb[1] : tl.pb[2]);
    const int e = g == 0 ? tl.pe[0] : (g == 1 ? tl.pe[1] : tl.pe[2]);
    inside = p >= b && p < e;
    return g;
}

__device__ __forceinline__ int64_t seg_d(const Tile& tl, int g) {
    return g == 0 ? tl.d[0] : (g == 1 ? tl.d[1] : tl.d[2]);
}

// MODE 0: y from a time-domain array; 1: gather T map; 3: gather I/Q/U map;
// 2: y from an FP64 time-domain array (rounded to T); 4 / 5: FP64 data minus the T /
// I/Q/U gather, d - P x (the residual b - A x = P^T N^-1 (d - P x) of Eq. 5 and 7).
// Load block positions [s0, s0 + count) into ar[0..count) (one position per lane,
// coalesced within a segment; ar is the packed complex array viewed as reals, so local
// position s lands in component s & 1 of complex slot s / 2).  A position outside the
// tile's segments reads as 0.  The common tile of one segment covering the whole range
// takes a branch-free path.
template <typename T, int NT, int MODE>
__device__ __forceinline__ void load_block(const TzArgs<T>& A, const Tile& tile, T* ar, int s0, int count,
                                           int64_t roff) {
    using I = In<T>;
    const I* __restrict__ y = A.y + roff;
    const I* __restrict__ x = A.x + roff;
    const double* __restrict__ yd = A.yd + roff;
    const int tid = threadIdx.x;
    const int PER = count / NT;
    constexpr bool IQU = MODE == 3 || MODE == 5;
    constexpr int UMAX = IQU ? 4 : 8;
    const bool whole = tile.pb[0] <= s0 && s0 + count <= tile.pe[0];
    const int64_t d0 = tile.d[0];
    const int sbase = 2 * pad<T>(tid >> 1) + (tid & 1);   // real slot of local position tid
    if constexpr (sizeof(T) == 4 && MODE == 3 && NT % (2 << PadLog<T>::v) == 0) {
        // FP32 I/Q/U from the packed map on a tile of one segment: indices and weights from
        // base pointers with 32-bit offsets, eight samples a round (the map's one 16-byte
        // load per sample leaves the registers for it)
        if (whole && A.x4 != nullptr && PER % 8 == 0) {
            const int32_t* pq = A.pixc + d0 + s0 + tid;
            const float2* pw = A.w + d0 + s0 + tid;
            constexpr int RSTEP = 2 * (NT / 2 + (NT >> (PadLog<T>::v + 1)));
#pragma unroll 1
            for (int base = 0; base < PER; base += 8) {
                int q[8];
                float2 w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) q[u] = __ldg(pq + (base + u) * NT);
#pragma unroll
                for (int u = 0; u < 8; ++u) w[u] = pw[(base + u) * NT];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float r = 0.f;
                    if (q[u] >= 0) {
                        const float4 m = __ldg(A.x4 + q[u]);
                        r = m.x + w[u].x * m.y + w[u].y * m.z;
                    }
                    ar[sbase + (base + u) * RSTEP] = r;
                }
            }
            return;
        }
        // the same over a tile of several segments: per sample the segment's base pointers
        // are selected (unused segments have pb = pe = TILE_NONE and are never selected)
        if (A.x4 != nullptr && PER % 8 == 0) {
            const int pb1 = tile.pb[1], pb2 = tile.pb[2];
            const int32_t* q0 = A.pixc + tile.d[0];
            const int32_t* q1 = A.pixc + (tile.pb[1] < tile.pe[1] ? tile.d[1] : 0);
            const int32_t* q2 = A.pixc + (tile.pb[2] < tile.pe[2] ? tile.d[2] : 0);
            const float2* w0 = A.w + tile.d[0];
            const float2* w1 = A.w + (tile.pb[1] < tile.pe[1] ? tile.d[1] : 0);
            const float2* w2 = A.w + (tile.pb[2] < tile.pe[2] ? tile.d[2] : 0);
            constexpr int RSTEP = 2 * (NT / 2 + (NT >> (PadLog<T>::v + 1)));
#pragma unroll 1
            for (int base = 0; base < PER; base += 8) {
                int q[8];
                float2 w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int p = s0 + (base + u) * NT + tid;
                    const int g = (p >= pb1) + (p >= pb2);
                    const int lo = g == 0 ? tile.pb[0] : (g == 1 ? pb1 : pb2);
                    const int hi = g == 0 ? tile.pe[0] : (g == 1 ? tile.pe[1] : tile.pe[2]);
                    const bool in = p >= lo && p < hi;
                    const int32_t* qb = g == 0 ? q0 : (g == 1 ? q1 : q2);
                    const float2* wb = g == 0 ? w0 : (g == 1 ? w1 : w2);
                    q[u] = in ? __ldg(qb + p) : -1;
                    w[u] = in ? wb[p] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    float r = 0.f;
                    if (q[u] >= 0) {
                        const float4 m = __ldg(A.x4 + q[u]);
                        r = m.x + w[u].x * m.y + w[u].y * m.z;
                    }
                    ar[sbase + (base + u) * RSTEP] = r;
                }
            }
            return;
        }
    }
#pragma unroll 1
    for (int base = 0; base < PER; base += UMAX) {
        T v[UMAX];
        int64_t tt[UMAX];
        bool okv[UMAX];
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
            const int p = s0 + (base + u) * NT + tid;
            if (whole) {
                tt[u] = p + d0;
                okv[u] = base + u < PER;
            } else {
                bool in;
                const int g = tile_seg(tile, p, in);
                tt[u] = p + seg_d(tile, g);
                okv[u] = base + u < PER && in;
            }
        }
        if constexpr (MODE == 0 || MODE == 2) {
#pragma unroll
            for (int u = 0; u < UMAX; ++u) {
                if constexpr (MODE == 0) v[u] = okv[u] ? from_in<T>(y[tt[u]]) : (T)0;
                else v[u] = okv[u] ? (T)yd[tt[u]] : (T)0;
            }
        } else {
            // the gather (and d - P x) is formed in the precision of the data, I
            int q[UMAX];
            typename Cx<I>::type w[UMAX];
            I dv[UMAX];
#pragma unroll
            for (int u = 0; u < UMAX; ++u) {
                q[u] = okv[u] ? __ldg(A.pixc + tt[u]) : -1;
                if constexpr (IQU) {
                    if (okv[u]) w[u] = A.w[tt[u]];
                }
                if constexpr (MODE >= 4) dv[u] = okv[u] ? (I)yd[tt[u]] : (I)0;
            }
#pragma unroll
            for (int u = 0; u < UMAX; ++u) {
                I r = (I)0;
                if (q[u] >= 0) {
                    if constexpr (!IQU) {
                        r = __ldg(x + q[u]);
                    } else {
                        bool packed = false;
                        if constexpr (sizeof(I) == 4 && MODE == 3) {
                            // one 16-byte load per sample instead of three: a warp's gather
                            // touches a cache line per pixel it visits (eight on a column
                            // scan) once rather than three times
                            if (A.x4 != nullptr) {
                                const float4 m = __ldg(A.x4 + q[u]);
                                r = m.x + w[u].x * m.y + w[u].y * m.z;
                                packed = true;
                            }
                        }
                        if (!packed) {
                            const I* xq = x + 3 * (int64_t)q[u];
                            r = __ldg(xq) + w[u].x * __ldg(xq + 1) + w[u].y * __ldg(xq + 2);
                        }
                    }
                }
                if constexpr (MODE >= 4) v[u] = from_in<T>(dv[u] - r);
                else v[u] = (T)r;
            }
        }
#pragma unroll
        for (int u = 0; u < UMAX; ++u) {
            if (base + u < PER) {
                if constexpr (NT % (2 << PadLog<T>::v) == 0) {
                    // sidx = (base + u) NT + tid with NT a multiple of 2 * 16: the padded
                    // slot is a per-thread base plus a per-round constant
                    constexpr int RSTEP = 2 * (NT / 2 + (NT >> (PadLog<T>::v + 1)));
                    ar[sbase + (base + u) * RSTEP] = v[u];
                } else {
                    const int sidx = (base + u) * NT + tid;
                    ar[2 * pad<T>(sidx >> 1) + (sidx & 1)] = v[u];
                }
            }
        }
    }
}

// Bulk L2 prefetch of the bytes [p, p + nbytes), shrunk inwards to 16-byte boundaries
// (the alignment cp.async.bulk.prefetch.L2 wants), in pieces of at most 32 KB.
__device__ __forceinline__ void l2_prefetch(const void* p, int64_t nbytes) {
    uint64_t a = (uint64_t)__cvta_generic_to_global(p);
    const uint64_t e = (a + (uint64_t)nbytes) & ~(uint64_t)15;
    a = (a + 15) & ~(uint64_t)15;
    for (; a < e; a += 32768) {
        const uint32_t n = (uint32_t)(e - a < 32768 ? e - a : 32768);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
    }
}

// L2 prefetch of the streamed inputs of CTA cid: the pointing and weights of its tile
// (gather modes; once per tile, by its first right-hand side) or its time-domain input,
// over the tile's segments, one lane per segment.  Issued for the CTA that will run one
// wave later, once this CTA's own gather is done, the copy overlaps this CTA's FFTs and
// more of that CTA's gathers wait on L2 instead of HBM.  (Measured on the 2^24-sample
// bench: two waves ahead, or issued at the start of the CTA, was slower.)  prefetch_seg reads the segment (lane g < TILE_SEGS) early,
// prefetch_issue starts the copies once the descriptor load has long arrived.
struct PfSeg {
    int64_t t0;
    int n;     // samples (0: nothing to prefetch)
    int rhs;
};

template <typename T>
__device__ __forceinline__ PfSeg prefetch_seg(const TzArgs<T>& A, int cid) {
    PfSeg sg{0, 0, 0};
    const int g = threadIdx.x;
    if (g >= TILE_SEGS) return sg;
    const TileRhs tr = tile_rhs(cid, A.R);
    const Tile& tl = A.tiles[tr.tile];
    const int pb = g == 0 ? tl.pb[0] : (g == 1 ? tl.pb[1] : tl.pb[2]);
    const int pe = g == 0 ? tl.pe[0] : (g == 1 ? tl.pe[1] : tl.pe[2]);
    if (pb < pe) {
        sg.t0 = pb + seg_d(tl, g);
        sg.n = pe - pb;
        sg.rhs = tr.rhs;
    }
    return sg;
}

template <typename T, int MODE>
__device__ __forceinline__ void prefetch_issue(const TzArgs<T>& A, const PfSeg& sg) {
    if (sg.n == 0) return;
    const int64_t roff = sg.rhs * A.in_stride, t0 = sg.t0, n = sg.n;
    if constexpr (MODE == 0) l2_prefetch(A.y + roff + t0, n * (int64_t)sizeof(In<T>));
    if constexpr (MODE == 2 || MODE >= 4) l2_prefetch(A.yd + roff + t0, n * 8);
    if constexpr (MODE != 0 && MODE != 2) {
        if (sg.rhs == 0) {
            l2_prefetch(A.pixc + t0, n * 4);
            if constexpr (MODE == 3 || MODE == 5) l2_prefetch(A.w + t0, n * (int64_t)sizeof(A.w[0]));
        }
    }
}

// Store output n (block position lambda + n) at its time, unless it falls between segments.
template <typename T>
__device__ __forceinline__ void store_out(const Tile& tile, In<T>* z, int lambda, int n, T v) {
    bool in;
    const int p = n + lambda;
    const int g = tile_seg(tile, p, in);
    if (in) z[p + seg_d(tile, g)] = to_in<T>(v);
}

// Real-FFT split of the packed spectrum at the bin pair (k, N - k), product with the real
// kernel spectrum (h1 = H[k], h2 = H[N - k]) and the merge back to packed form, returned
// conjugated for the inverse-by-forward transform.  (cw, sw) = (cos, sin) of 2 pi k / B.
template <typename T>
__device__ __forceinline__ void split_product(typename Cx<T>::type u1, typename Cx<T>::type u2, T cw, T sw, T h1,
                                              T h2, typename Cx<T>::type& V1, typename Cx<T>::type& V2) {
    using C2 = typename Cx<T>::type;
    // E = (u1 + conj u2)/2, O = -i (u1 - conj u2)/2
    C2 E, O;
    E.x = (T)0.5 * (u1.x + u2.x); E.y = (T)0.5 * (u1.y - u2.y);
    O.x = (T)0.5 * (u1.y + u2.y); O.y = (T)-0.5 * (u1.x - u2.x);
    const C2 WO = cmul<T>(O, cw, sw);
    C2 X1, X2;                         // X_k = E + W O, X_{N-k} = conj(E - W O)
    X1.x = E.x + WO.x; X1.y = E.y + WO.y;
    X2.x = E.x - WO.x; X2.y = -(E.y - WO.y);
    C2 Z1, Z2;
    Z1.x = h1 * X1.x; Z1.y = h1 * X1.y;
    Z2.x = h2 * X2.x; Z2.y = h2 * X2.y;
    // V1 = (Z1 + conj Z2)/2 + i conj(W) (Z1 - conj Z2)/2
    // V2 = (Z2 + conj Z1)/2 - i W (Z2 - conj Z1)/2
    C2 S1, D1, S2, D2;
    S1.x = (T)0.5 * (Z1.x + Z2.x); S1.y = (T)0.5 * (Z1.y - Z2.y);
    D1.x = (T)0.5 * (Z1.x - Z2.x); D1.y = (T)0.5 * (Z1.y + Z2.y);
    S2.x = S1.x; S2.y = -S1.y;
    D2.x = -D1.x; D2.y = D1.y;
    {
        const T px = cw * D1.x - sw * D1.y;   // conj(W) * D1
        const T py = cw * D1.y + sw * D1.x;
        V1.x = S1.x - py; V1.y = S1.y + px;   // + i (px + i py)
    }
    {
        const T px = cw * D2.x + sw * D2.y;   // W * D2
        const T py = cw * D2.y - sw * D2.x;
        V2.x = S2.x + py; V2.y = S2.y - px;   // - i (px + i py)
    }
    // conjugates: the forward FFT of conj(V) is conj of N * IFFT(V)
    V1.y = -V1.y;
    V2.y = -V2.y;
}

template <typename T, int LOGN, int NT, int MODE>
__device__ __forceinline__ void toeplitz_os_tile(const TzArgs<T>& A) {
    griddep_wait();   // launched as a dependent launch: the previous kernel's outputs
    using C2 = typename Cx<T>::type;
    constexpr int N = 1 << LOGN;
    constexpr int Q = N / 2;             // B/4
    if (A.done != nullptr && *(volatile const int*)A.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* a = reinterpret_cast<C2*>(smem_raw);
    T* tab = reinterpret_cast<T*>(smem_raw + sizeof(C2) * (N + (N >> PadLog<T>::v)));
    const TileRhs tr = tile_rhs(blockIdx.x, A.R);
    const Tile tile = A.tiles[tr.tile];
    const int tid = threadIdx.x;
    // every CTA prefetches the inputs of the CTA one wave on (the first wave's own inputs
    // are not: a prefetch racing the CTA's own loads measured slower than none)
    PfSeg next{0, 0, 0};
    if (A.pf_ahead > 0 && (int64_t)blockIdx.x + A.pf_ahead < (int64_t)gridDim.x)
        next = prefetch_seg(A, blockIdx.x + A.pf_ahead);
    // FP32: the split twiddles are computed (sincospif), which leaves the table's 32 KB of
    // shared memory to the L1 cache that serves the de-pointing gathers
    if constexpr (sizeof(T) != 4)
        for (int i = tid; i <= Q; i += NT) tab[i] = A.twiddle[i];
    load_block<T, NT, MODE>(A, tile, reinterpret_cast<T*>(a), 0, 2 * N, tr.rhs * A.in_stride);
    __syncthreads();
    prefetch_issue<T, MODE>(A, next);
    fft_all<T, LOGN, NT, 0>(a, A.ptw);
    // real-FFT post-processing, spectrum product, pre-processing for the inverse.
    const T* H = A.H + (int64_t)tile.psd * (N + 1);
    for (int k = tid; k <= N / 2; k += NT) {
        const int k2 = (N - k) & (N - 1);
        T cw, sw;                         // W = cw - i sw = exp(-2 pi i k / B)
        if constexpr (sizeof(T) == 4) {
            float sv, cv;
            sincospif((float)k * (1.f / (float)N), &sv, &cv);   // 2 pi k / B = pi k / N
            cw = cv;
            sw = sv;
        } else {
            twiddle<T, LOGN - 1>(tab, k, cw, sw);
        }
        C2 V1, V2;
        split_product<T>(a[pad<T>(k)], a[pad<T>(k2)], cw, sw, H[k], H[N - k], V1, V2);
        a[pad<T>(k)] = V1;
        if (k2 != k) a[pad<T>(k2)] = V2;
    }
    __syncthreads();
    fft_all<T, LOGN, NT, 0>(a, A.ptw);
    // outputs: real block positions lambda .. lambda + nout - 1, stored at their times
    In<T>* zo = A.z + tr.rhs * A.out_stride;
    if (tile.pb[0] <= A.lambda && A.lambda + tile.nout <= tile.pe[0]) {
        // every output inside the first segment: time = position + d[0]
        // (four shared-memory reads in flight per thread before their stores)
        In<T>* z0 = zo + tile.d[0];
        const int nout = tile.nout;
#pragma unroll 1
        for (int n0 = tid; n0 < nout; n0 += 4 * NT) {
            C2 c[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (n0 + u * NT < nout) c[u] = a[pad<T>((n0 + u * NT + A.lambda) >> 1)];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = n0 + u * NT + A.lambda;
                if (n0 + u * NT < nout) z0[i] = to_in<T>((i & 1) ? -c[u].y : c[u].x);
            }
        }
    } else {
        for (int n = tid; n < tile.nout; n += NT) {
            const int i = n + A.lambda;
            const C2 v = a[pad<T>(i >> 1)];
            store_out<T>(tile, zo, A.lambda, n, (i & 1) ? -v.y : v.x);
        }
    }
}

// Resident CTAs per SM: FP32 blocks below 2^15 reals run 1024 / NT CTAs of NT threads per
// SM (at most 64 registers a thread), so that one CTA's gather overlaps another's FFT;
// the 1024-thread FP32 block and FP64 / double-float keep their own register use (one
// CTA per SM), and so do 32-thread CTAs, which the 64-register cap would make spill.
template <typename T, int NT>
__host__ __device__ constexpr int tz_min_blocks() {
    return sizeof(T) == 4 && NT < 1024 && NT >= 64 ? 1024 / NT : 1;
}

template <typename T, int LOGN, int NT, int MODE>
__global__ void __launch_bounds__(NT) toeplitz_os_kernel(TzArgs<T> A) {
    toeplitz_os_tile<T, LOGN, NT, MODE>(A);
}

template <typename T, int LOGN, int NT, int MODE>
__global__ void __launch_bounds__(NT, (tz_min_blocks<T, NT>())) toeplitz_os_kernel_mb(TzArgs<T> A) {
    toeplitz_os_tile<T, LOGN, NT, MODE>(A);
}

// v * W_C^m for C in {2, 4} (m taken mod C): multiplications by +-1, +-i only.
template <typename T, int C>
__device__ __forceinline__ typename Cx<T>::type rot_c(typename Cx<T>::type v, int m) {
    typename Cx<T>::type r;
    const int q = (C == 2 ? 2 * m : m) & 3;   // power of W_4 = -i
    switch (q) {
        case 0: r = v; break;
        case 1: r.x = v.y; r.y = -v.x; break;    // * (-i)
        case 2: r.x = -v.x; r.y = -v.y; break;
        default: r.x = -v.y; r.y = v.x; break;   // * (+i)
    }
    return r;
}

// Cluster variant (C = 2 or 4 CTAs): the packed block of N = C M complex points (B = 2N
// reals) is split in C chunks, CTA c holding u[c M + n1].  Forward transform (decimation
// in frequency): y_c[n1] = W_N^(n1 c) sum_n2 u_n2[n1] W_C^(n2 c) across the cluster
// (distributed shared memory, same local index in every CTA), then a local M-point FFT
// leaves X[C k1 + c] in CTA c.  The real-FFT partner N - k of bin k lies in CTA (C - c)
// mod C: the same CTA for c = 0 (and c = C/2), the opposite one of the pair (1, 3) when
// C = 4, read there across the cluster.  Inverse (decimation in time): local M-point FFT,
// then out_c[n1] = sum_m2 W_C^(m2 c) W_N^(m2 n1) Z_m2[n1] across the cluster, written
// straight to global memory.
template <typename T, int LOGM, int NT, int MODE, int CL>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(NT) toeplitz_oscl_kernel(TzArgs<T> A) {
    using C2 = typename Cx<T>::type;
    constexpr int M = 1 << LOGM;
    constexpr int N = CL * M;
    constexpr int LOGQ = LOGM + (CL == 2 ? 0 : 1);   // B/4 = N/2 = 2^LOGQ
    constexpr int PER = M / NT;
    static_assert(PER >= 1 && M % NT == 0, "points per thread");
    if (A.done != nullptr && *(volatile const int*)A.done) return;   // uniform over the cluster
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2* a = reinterpret_cast<C2*>(smem_raw);
    C2* part[CL];
#pragma unroll
    for (int c = 0; c < CL; ++c) part[c] = cl.map_shared_rank(a, c);
    const TileRhs tr = tile_rhs(blockIdx.x / CL, A.R);
    const Tile tile = A.tiles[tr.tile];
    const int tid = threadIdx.x;
    load_block<T, NT, MODE>(A, tile, reinterpret_cast<T*>(a), rank * 2 * M, 2 * M, tr.rhs * A.in_stride);
    cl.sync();
    C2 y[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int n1 = u * NT + tid;
        C2 acc = part[0][pad<T>(n1)];
#pragma unroll
        for (int n2 = 1; n2 < CL; ++n2) {
            const C2 v = rot_c<T, CL>(part[n2][pad<T>(n1)], n2 * rank);
            acc.x += v.x;
            acc.y += v.y;
        }
        if (rank != 0) {
            T c, s;
            twiddle<T, LOGQ>(A.twiddle, 2 * n1 * rank, c, s);   // W_N^(n1 rank) = W_B^(2 n1 rank)
            acc = cmul<T>(acc, c, s);
        }
        y[u] = acc;
    }
    cl.sync();
#pragma unroll
    for (int u = 0; u < PER; ++u) a[pad<T>(u * NT + tid)] = y[u];
    __syncthreads();
    fft_all<T, LOGM, NT, 0>(a, A.ptw);
    const T* H = A.H + (int64_t)tile.psd * (N + 1);
    const int prank = (CL - rank) % CL;
    if (prank == rank) {
        // partner bins inside this CTA: process each pair once
        const int npairs = rank == 0 ? M / 2 + 1 : M / 2;
        for (int k1 = tid; k1 < npairs; k1 += NT) {
            const int k = CL * k1 + rank;
            const int p = rank == 0 ? ((M - k1) & (M - 1)) : (M - 1 - k1);
            T cw, sw;
            twiddle<T, LOGQ>(A.twiddle, k, cw, sw);
            C2 V1, V2;
            split_product<T>(a[pad<T>(k1)], a[pad<T>(p)], cw, sw, H[k], H[N - k], V1, V2);
            a[pad<T>(k1)] = V1;
            if (p != k1) a[pad<T>(p)] = V2;
        }
        cl.sync();
        cl.sync();
    } else {
        // partner bins in CTA prank (C = 4, ranks 1 and 3): compute this CTA's bins only
        C2 vo[PER];
        cl.sync();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int k1 = u * NT + tid;
            const int k = CL * k1 + rank;
            T cw, sw;
            twiddle<T, LOGQ>(A.twiddle, k, cw, sw);
            C2 V2;
            split_product<T>(a[pad<T>(k1)], part[prank][pad<T>(M - 1 - k1)], cw, sw, H[k], H[N - k], vo[u], V2);
        }
        cl.sync();
#pragma unroll
        for (int u = 0; u < PER; ++u) a[pad<T>(u * NT + tid)] = vo[u];
    }
    __syncthreads();
    fft_all<T, LOGM, NT, 0>(a, A.ptw);
    cl.sync();
    In<T>* zo = A.z + tr.rhs * A.out_stride;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int n1 = u * NT + tid;
        C2 f = part[0][pad<T>(n1)];
#pragma unroll
        for (int m2 = 1; m2 < CL; ++m2) {
            T c, s;
            twiddle<T, LOGQ>(A.twiddle, 2 * n1 * m2, c, s);   // W_N^(m2 n1)
            const C2 v = rot_c<T, CL>(cmul<T>(part[m2][pad<T>(n1)], c, s), m2 * rank);
            f.x += v.x;
            f.y += v.y;
        }
        // packed index m = rank M + n1 -> real samples 2m (f.x) and 2m + 1 (-f.y)
        const int i0 = 2 * (rank * M + n1) - A.lambda;
        if (i0 >= 0 && i0 < tile.nout) store_out<T>(tile, zo, A.lambda, i0, f.x);
        if (i0 + 1 >= 0 && i0 + 1 < tile.nout) store_out<T>(tile, zo, A.lambda, i0 + 1, -f.y);
    }
    cl.sync();   // the other CTAs may still read this CTA's shared memory
}

// Threads per CTA: one largest-radix butterfly per thread and pass (N/16, or N/8 for
// small N), capped at 1024 for FP32 (16 complex values per thread fit the 64-register
// budget of a 1024-thread CTA) and 512 for FP64, at least 32.
template <typename T, int LOGN>
__host__ __device__ constexpr int tz_threads() {
    constexpr int cap = sizeof(T) == 4 ? 1024 : 512;
    constexpr int want = (1 << LOGN) >> fft_max_logr<LOGN>();
    return want >= cap ? cap : (want < 32 ? 32 : want);
}

template <typename T>
size_t toeplitz2_smem_bytes_impl(int logm) {
    const size_t M = size_t(1) << logm;
    return sizeof(typename Cx<T>::type) * (M + (M >> PadLog<T>::v));
}

template <typename T, int LOGM, int MODE, int CL>
void launch_cl(const TzArgs<T>& A, int ntiles, cudaStream_t s) {
    constexpr int NT = tz_threads<T, LOGM>();
    const size_t smem = toeplitz2_smem_bytes_impl<T>(LOGM);
    auto kern = toeplitz_oscl_kernel<T, LOGM, NT, MODE, CL>;
    ensure_smem_attr((const void*)kern, (int)smem, "cudaFuncSetAttribute(toeplitz cluster)");
    kern<<<(unsigned)((int64_t)CL * ntiles * A.R), NT, smem, s>>>(A);
    check_cuda(cudaGetLastError(), "toeplitz cluster kernel launch");
    note_launch();
}

template <typename T, int LOGM, int CL>
void launch_mode_cl(const TzArgs<T>& A, int ntiles, int mode, cudaStream_t s) {
    switch (mode) {
        case 0: launch_cl<T, LOGM, 0, CL>(A, ntiles, s); return;
        case 1: launch_cl<T, LOGM, 1, CL>(A, ntiles, s); return;
        case 3: launch_cl<T, LOGM, 3, CL>(A, ntiles, s); return;
        default: break;
    }
    if constexpr (sizeof(T) == 4) {
        if (mode == 2) return launch_cl<T, LOGM, 2, CL>(A, ntiles, s);
    } else {
        if (mode == 4) return launch_cl<T, LOGM, 4, CL>(A, ntiles, s);
        if (mode == 5) return launch_cl<T, LOGM, 5, CL>(A, ntiles, s);
    }
    throw Error{MM_ERR_ARG, "unsupported Toeplitz load mode"};
}

template <typename T>
size_t toeplitz_smem_bytes_impl(int logn) {
    const size_t N = size_t(1) << logn;
    // the FP32 kernel computes its split twiddles and holds no cosine table
    const size_t table = sizeof(T) == 4 ? 0 : sizeof(T) * (N / 2 + 1);
    return sizeof(typename Cx<T>::type) * (N + (N >> PadLog<T>::v)) + table;
}

template <typename T, int LOGN, int MODE>
void launch_one(const TzArgs<T>& A, int ntiles, cudaStream_t s) {
    constexpr int NT = tz_threads<T, LOGN>();
    const size_t smem = toeplitz_smem_bytes_impl<T>(LOGN);
    void (*kern)(TzArgs<T>) = nullptr;
    if constexpr (tz_min_blocks<T, NT>() > 1) kern = toeplitz_os_kernel_mb<T, LOGN, NT, MODE>;
    else kern = toeplitz_os_kernel<T, LOGN, NT, MODE>;
    ensure_smem_attr((const void*)kern, (int)smem, "cudaFuncSetAttribute(toeplitz)");
    TzArgs<T> B = A;
    if (B.pf_ahead > 0) {
        // resident CTAs = SMs (pf_ahead on entry) x CTAs per SM, measured once per kernel
        static std::atomic<int> per_sm{0};
        int occ = per_sm.load();
        if (occ == 0) {
            check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem), "toeplitz occupancy");
            per_sm.store(occ = occ > 0 ? occ : 1);
        }
        B.pf_ahead *= occ;
    }
    launch_pdl(kern, (unsigned)((int64_t)ntiles * A.R), NT, smem, s, B);
    note_launch();
}

// Load modes 0, 1, 3 for both precisions; 2 (FP64 data rounded) for FP32 only; 4 and 5
// (FP64 residual data) for FP64 only.
template <typename T, int LOGN>
void launch_mode(const TzArgs<T>& A, int ntiles, int mode, cudaStream_t s) {
    switch (mode) {
        case 0: launch_one<T, LOGN, 0>(A, ntiles, s); return;
        case 1: launch_one<T, LOGN, 1>(A, ntiles, s); return;
        case 3: launch_one<T, LOGN, 3>(A, ntiles, s); return;
        default: break;
    }
    if constexpr (sizeof(T) == 4) {
        if (mode == 2) return launch_one<T, LOGN, 2>(A, ntiles, s);
    } else {
        if (mode == 4) return launch_one<T, LOGN, 4>(A, ntiles, s);
        if (mode == 5) return launch_one<T, LOGN, 5>(A, ntiles, s);
    }
    throw Error{MM_ERR_ARG, "unsupported Toeplitz load mode"};
}

}  // namespace mm
