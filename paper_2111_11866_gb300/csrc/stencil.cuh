// stencil.cuh -- device building blocks shared by the single-grid kernels
// (solve_kernels.cu) and the batched-window kernels (batch.cu): FP64 block
// reductions, the red-black neighbour sum of the sweep, and the reduced
// diamond-cell face gradients of the coefficient kernel.  Layout:
// seg4d_internal.cuh.
#pragma once

#include <cfloat>
#include <cmath>

#include <cuda_bf16.h>

#include "seg4d_internal.cuh"

namespace seg4d_impl {

// ------------------------------------------------------------------ helpers

struct Acc3 {
    double sum, mn, mx;
};

__device__ inline Acc3 acc3_merge(Acc3 a, Acc3 b)
{
    return {a.sum + b.sum, fmin(a.mn, b.mn), fmax(a.mx, b.mx)};
}

__device__ inline Acc3 warp_reduce3(Acc3 a)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Acc3 b;
        b.sum = __shfl_down_sync(0xffffffffu, a.sum, o);
        b.mn = __shfl_down_sync(0xffffffffu, a.mn, o);
        b.mx = __shfl_down_sync(0xffffffffu, a.mx, o);
        a = acc3_merge(a, b);
    }
    return a;
}

// Block-wide reduction; thread 0 writes the record (sum, min, max).
__device__ inline void block_write3(Acc3 a, double *rec)
{
    __shared__ Acc3 sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    a = warp_reduce3(a);
    if (lane == 0) sh[wid] = a;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        Acc3 b = lane < nw ? sh[lane] : Acc3{0.0, DBL_MAX, -DBL_MAX};
        b = warp_reduce3(b);
        if (lane == 0) {
            rec[0] = b.sum;
            rec[1] = b.mn;
            rec[2] = b.mx;
        }
    }
}

// Block-wide maximum of a non-negative float; thread 0 writes it as a double.
// Must follow the block's other reductions (it reuses no shared memory of
// theirs, but every thread of the block must call it).
__device__ inline void block_write_max(float v, double *out)
{
    __shared__ float shm[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0) shm[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        float b = lane < nw ? shm[lane] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b = fmaxf(b, __shfl_down_sync(0xffffffffu, b, o));
        if (lane == 0) *out = (double)b;
    }
}

struct RowPos {
    int j, k, l, p;
};

// Division of n < 2^31 by a runtime constant d >= 1 with a multiply-high and a
// shift (round-up method): s = ceil(log2 d), m = ceil(2^(32+s) / d) - 2^32,
// then n / d = (umulhi(n, m) + n) >> s; the sum stays below 2^32.
struct FastDiv {
    unsigned m, s, d, pad;
};

inline FastDiv make_fastdiv(unsigned d)
{
    unsigned s = 0;
    while ((1ull << s) < d) ++s;
    const unsigned long long m = ((1ull << (32 + s)) + d - 1) / d - (1ull << 32);
    return FastDiv{(unsigned)m, s, d, 0};
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv &f)
{
    return (__umulhi(n, f.m) + n) >> f.s;
}

// Work items t = 2 * tile + colour of the tile loops: tile = (chunk, y-block
// of 8 rows, plane), chunk fastest, with nch chunks per row and the planes in
// the tiled traversal order (Layout::kt); the number of items is below 2^31
// (checked when the handle is created).
struct ItemDecode {
    FastDiv fch, fjb, fkt, fn4;
    unsigned nch;
};

inline ItemDecode make_item_decode(const Layout &L, int nch)
{
    return ItemDecode{make_fastdiv((unsigned)nch), make_fastdiv((unsigned)L.njb),
                      make_fastdiv((unsigned)L.kt), make_fastdiv((unsigned)L.n4), (unsigned)nch};
}

inline long long item_count(const Layout &L, int nch)
{
    return 2LL * nch * L.njb * ((long long)L.ntile * L.kt) * L.n4;
}

// item t -> colour, chunk and the row position of warp `warp` (rp.p set); a
// hole of the last z-tile, like a row past n2, comes back as rp.j >= n2
__device__ __forceinline__ void decode_item(const ItemDecode &D, const Layout &L, unsigned t,
                                            int warp, int &C, int &chunk, RowPos &rp)
{
    C = (int)(t & 1u);
    const unsigned r = t >> 1;
    const unsigned a = fdiv(r, D.fch);
    chunk = (int)(r - a * D.nch);
    const unsigned b = fdiv(a, D.fjb);
    const int jb = (int)(a - b * (unsigned)L.njb);
    const unsigned c = fdiv(b, D.fkt);
    const unsigned tile = fdiv(c, D.fn4);
    rp.k = (int)(tile * (unsigned)L.kt + (b - c * (unsigned)L.kt));
    rp.l = (int)(c - tile * (unsigned)L.n4);
    rp.j = rp.k < L.n3 ? jb * 8 + warp : L.n2;
    rp.p = (rp.j + rp.k + rp.l) & 1;
}

// The 8 face edge coefficients of the voxel in slot s of colour C in row
// `row` (layout: gb_offsets).  A red voxel reads its own slot of the 8
// planes; a black voxel reads each interior face across the face (the
// opposite face of the red neighbour: x-neighbours in red slots s - p and
// s + 1 - p, y/z/t neighbours in the same slot of rows -+1, -+n2, -+n2 n3)
// and each face to the ring from the side table.  Zeros when !act.
template <int C>
__device__ __forceinline__ void load_G8(const Layout &L, const float *__restrict__ G, bool act,
                                        int row, int s, const RowPos &rp, float (&g)[8])
{
    const long long S = L.S;
    const long long q = (long long)row * L.P + s;
    if (C == 0) {
#pragma unroll
        for (int f = 0; f < 8; ++f) g[f] = act ? G[(long long)f * S + q] : 0.0f;
        return;
    }
    const int i = 2 * s + 1 - rp.p;
    const long long dy = L.P, dz = (long long)L.n2 * L.P, dt = (long long)L.n2 * L.n3 * L.P;
    const long long rb = (long long)row * L.P;
    const long long idx[8] = {1 * S + rb + s - rp.p, 0 * S + rb + s + 1 - rp.p,
                              3 * S + q - dy,         2 * S + q + dy,
                              5 * S + q - dz,         4 * S + q + dz,
                              7 * S + q - dt,         6 * S + q + dt};
    const bool in[8] = {i >= 1, i + 1 < L.n1, rp.j > 0, rp.j + 1 < L.n2,
                        rp.k > 0, rp.k + 1 < L.n3, rp.l > 0, rp.l + 1 < L.n4};
    const GbOff o = gb_offsets(L);
#pragma unroll
    for (int f = 0; f < 8; ++f)
        g[f] = !act ? 0.0f
                    : (in[f] ? G[idx[f]]
                             : G[8 * S + gb_index(L, o, f, row, s, rp.j, rp.k, rp.l)]);
}

// face weight load: FP32, or BF16 widened to FP32
__device__ __forceinline__ float ldw(const float *p) { return *p; }
__device__ __forceinline__ float ldw(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// Relaxation arithmetic with every rounding explicit (no contraction left to
// the compiler), so that all sweep kernels -- per colour or fused, single
// grid or batched -- produce the same bits:
//   acc = sum over faces of w_f x_f (products rounded, fixed addition tree),
//   x  <- x + omega (B + G acc - x).
__device__ __forceinline__ float sum8(float t0, float t1, float t2, float t3, float t4, float t5,
                                      float t6, float t7)
{
    return __fadd_rn(__fadd_rn(__fadd_rn(t0, t1), __fadd_rn(t2, t3)),
                     __fadd_rn(__fadd_rn(t4, t5), __fadd_rn(t6, t7)));
}

__device__ __forceinline__ float relax(float x, float B, float G, float acc, float omega)
{
    return __fmaf_rn(omega, __fsub_rn(__fmaf_rn(G, acc, B), x), x);
}

// ------------------------------------------------ N voxels per thread

// Voxels per thread of the sweep kernels (2: float2 loads of x and the
// coefficients, 8- or 4-byte loads of the weights; 4 costs occupancy), and
// the resident 256-thread blocks per SM they are compiled for.
#ifndef SEG4D_VEC_F32
#define SEG4D_VEC_F32 2
#endif
#ifndef SEG4D_VEC_BF16
#define SEG4D_VEC_BF16 2
#endif
constexpr int kVecF32 = SEG4D_VEC_F32;
constexpr int kVecBF16 = SEG4D_VEC_BF16;
static_assert((kVecF32 == 2 || kVecF32 == 4) && (kVecBF16 == 2 || kVecBF16 == 4),
              "2 or 4 voxels per thread (P is a multiple of 4)");
// voxels per thread of the single-grid defect pass (1, 2 or 4) and its resident
// blocks per SM (3: measured faster than 2 and than one voxel per thread)
#ifndef SEG4D_DEFECT_N
#define SEG4D_DEFECT_N 2
#endif
#ifndef SEG4D_DEFECT_MINB
#define SEG4D_DEFECT_MINB 3
#endif
constexpr int kDefectN = SEG4D_DEFECT_N;
#ifndef SEG4D_VEC2_MINB
#define SEG4D_VEC2_MINB 4
#endif
#ifndef SEG4D_VEC4_MINB
#define SEG4D_VEC4_MINB 2
#endif
template <int N>
constexpr int vec_min_blocks() { return N == 1 ? 8 : (N == 2 ? SEG4D_VEC2_MINB : SEG4D_VEC4_MINB); }

// N-wide vector loads (N = 2 or 4 consecutive slots, N-aligned) into float
// arrays; a load whose condition is false yields zeros.
template <int N>
__device__ __forceinline__ void ldv(float (&v)[N], bool c, const float *p)
{
    if constexpr (N == 1) {
        v[0] = c ? *p : 0.0f;
    } else if constexpr (N == 2) {
        const float2 t = c ? *reinterpret_cast<const float2 *>(p) : make_float2(0.0f, 0.0f);
        v[0] = t.x;
        v[1] = t.y;
    } else {
        const float4 t =
            c ? *reinterpret_cast<const float4 *>(p) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
}

template <int N>
__device__ __forceinline__ void ldv(float (&v)[N], bool c, const __nv_bfloat16 *p)
{
    if constexpr (N == 1) {
        v[0] = c ? __bfloat162float(*p) : 0.0f;
    } else if constexpr (N == 2) {
        const unsigned t = c ? *reinterpret_cast<const unsigned *>(p) : 0u;
        v[0] = __uint_as_float(t << 16);
        v[1] = __uint_as_float(t & 0xFFFF0000u);
    } else {
        const uint2 t = c ? *reinterpret_cast<const uint2 *>(p) : make_uint2(0u, 0u);
        v[0] = __uint_as_float(t.x << 16);
        v[1] = __uint_as_float(t.x & 0xFFFF0000u);
        v[2] = __uint_as_float(t.y << 16);
        v[3] = __uint_as_float(t.y & 0xFFFF0000u);
    }
}

template <int N>
__device__ __forceinline__ void stv(float *p, const float (&v)[N])
{
    if constexpr (N == 1)
        *p = v[0];
    else if constexpr (N == 2)
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    else
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// Loads and lane shuffles shared by the group kernels: for the N voxels in
// slots s0 .. s0+N-1 (s0 a multiple of N) of colour C in row `row`, calls
// fn(m, xm, xp, wm, wp, inm, inp, a, y, in) per voxel m with its -x / +x
// neighbour values and weights (inm / inp: that neighbour slot exists) and
// the y, z, t faces f = 0..5 (a[f][m] weight, y[f][m] neighbour value, in[f]
// face inside the grid).  x is the [2][S] iterate, W the [8][S] face weights
// by red end (FP32, or BF16 widened exactly).  Every load is an N-wide vector
// load, all issued before any is used; a caller that needs more per-voxel
// data issues those loads before calling, so that they are in flight
// together.  The x-neighbour just past either end of the group (and, for
// black voxels, its face weight) comes from the adjacent lane by shuffle when
// that lane holds the adjacent group of the same row, and is loaded
// otherwise.  kAllW (red only): also load the weights of faces outside the
// grid (a red voxel owns them).  kOwnW (black only): W is a copy of the
// weights stored by their black end ([8][S] at the black voxel's own slot,
// faces to the ring 0), read as the red voxels read theirs.  All 32 lanes of
// the warp must call this; lanes without a group pass act = false (fn is not
// called).
template <int C, typename WT, int N, bool kAllW, typename Fn, bool kOwnW = false>
__device__ __forceinline__ void gather_core(const Layout &L, const float *__restrict__ x,
                                            const WT *__restrict__ W, bool act, int row, int s0,
                                            const RowPos &rp, Fn fn)
{
    const long long S = L.S;
    const long long q = (long long)row * L.P + s0;
    const float *xo = x + (C ? 0 : S);
    const int e = C ^ rp.p;   // i = 2 s + e
    const long long dy = L.P, dz = (long long)L.n2 * L.P, dt = (long long)L.n2 * L.n3 * L.P;
    // y, z, t faces f = 2..7: neighbour offset and presence
    const long long off[6] = {-dy, dy, -dz, dz, -dt, dt};
    const bool in[6] = {act && rp.j > 0, act && rp.j + 1 < L.n2, act && rp.k > 0,
                        act && rp.k + 1 < L.n3, act && rp.l > 0, act && rp.l + 1 < L.n4};
    float X[N], W0[N], W1[N], a[6][N], y[6][N];
    ldv<N>(X, act, xo + q);
    // x-direction weights: red owns faces 0 (-x) and 1 (+x); black reads
    // face 1 of the red voxel on its left and face 0 of the one on its right
    // (or, with kOwnW, its own faces 0 and 1)
    constexpr bool kOwn = C == 0 || kOwnW;
    ldv<N>(W0, act, W + 0 * S + q);
    ldv<N>(W1, act, W + 1 * S + q);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        // red (or kOwnW): own face f+2; black: the opposite face of the red
        // neighbour
        const long long wi = kOwn ? (long long)(f + 2) * S + q
                                  : (long long)((f + 2) ^ 1) * S + q + off[f];
        ldv<N>(a[f], (kAllW && C == 0) ? act : in[f], W + wi);
        ldv<N>(y[f], in[f], xo + q + off[f]);
    }
    const bool hasL = s0 > 0, hasR = s0 + N < L.P;
    const unsigned key = act ? (unsigned)q : 0xFFFFFFFFu;   // q is even; the sentinel odd
    const unsigned keyL = __shfl_up_sync(0xFFFFFFFFu, key, 1);
    const unsigned keyR = __shfl_down_sync(0xFFFFFFFFu, key, 1);
    const float xLs = __shfl_up_sync(0xFFFFFFFFu, X[N - 1], 1);
    const float xRs = __shfl_down_sync(0xFFFFFFFFu, X[0], 1);
    const float wLs = __shfl_up_sync(0xFFFFFFFFu, W1[N - 1], 1);
    const float wRs = __shfl_down_sync(0xFFFFFFFFu, W0[0], 1);
    if (!act) return;
    const bool shL = hasL && keyL == (unsigned)(q - N);
    const bool shR = hasR && keyR == (unsigned)(q + N);
    float xl = 0.0f, xr = 0.0f, wl = 0.0f, wr = 0.0f;
    if (e == 0) {
        xl = shL ? xLs : (hasL ? xo[q - 1] : 0.0f);
        if (!kOwn) wl = shL ? wLs : (hasL ? ldw(W + 1 * S + q - 1) : 0.0f);
    } else {
        xr = shR ? xRs : (hasR ? xo[q + N] : 0.0f);
        if (!kOwn) wr = shR ? wRs : (hasR ? ldw(W + 0 * S + q + N) : 0.0f);
    }
#pragma unroll
    for (int m = 0; m < N; ++m) {
        // e = 0: x-neighbours of slot s are slots s-1 and s; e = 1: s and s+1
        const float xm = e == 0 ? (m == 0 ? xl : X[m - 1]) : X[m];
        const float xp = e == 0 ? X[m] : (m == N - 1 ? xr : X[m + 1]);
        float wm, wp;
        if (kOwn) {
            wm = W0[m];
            wp = W1[m];
        } else {
            wm = e == 0 ? (m == 0 ? wl : W1[m - 1]) : W1[m];
            wp = e == 0 ? W0[m] : (m == N - 1 ? wr : W0[m + 1]);
        }
        const bool inm = e == 1 || m > 0 || hasL;
        const bool inp = e == 0 || m < N - 1 || hasR;
        fn(m, xm, xp, wm, wp, inm, inp, a, y, in);
    }
}

// Neighbour sums acc[m] = sum_f w_f x_nb(f) of a group (see gather_core):
// products rounded, the fixed addition tree of sum8, a face outside the grid
// contributes exactly 0.
template <int C, typename WT, int N, bool kOwnW = false>
__device__ __forceinline__ void gather_vec(const Layout &L, const float *__restrict__ x,
                                           const WT *__restrict__ W, bool act, int row, int s0,
                                           const RowPos &rp, float (&acc)[N])
{
    auto fn = [&](int m, float xm, float xp, float wm, float wp, bool inm, bool inp,
                  const float (&a)[6][N], const float (&y)[6][N], const bool (&in)[6]) {
        acc[m] = sum8(inm ? __fmul_rn(wm, xm) : 0.0f, inp ? __fmul_rn(wp, xp) : 0.0f,
                      in[0] ? __fmul_rn(a[0][m], y[0][m]) : 0.0f,
                      in[1] ? __fmul_rn(a[1][m], y[1][m]) : 0.0f,
                      in[2] ? __fmul_rn(a[2][m], y[2][m]) : 0.0f,
                      in[3] ? __fmul_rn(a[3][m], y[3][m]) : 0.0f,
                      in[4] ? __fmul_rn(a[4][m], y[4][m]) : 0.0f,
                      in[5] ? __fmul_rn(a[5][m], y[5][m]) : 0.0f);
    };
    gather_core<C, WT, N, false, decltype(fn), kOwnW>(L, x, W, act, row, s0, rp, fn);
}

// Exact residual of the step system in flux form for the N voxels of a
// group (see gather_core), FP32 weights:
//   r = (b - u) - c (sum_f w_f (u - u_nb) + u * w_bnd),   c = gamma * D,
// the same A u as D u - c sum_f w_f u_nb, but the differences u - u_nb are
// small and exact, so r carries far less rounding noise than D (ubar - u).
// Faces to an existing slot enter the flux (a padding slot holds 0, so a
// face to it contributes w u, as a boundary face does); w_bnd collects the
// rest.  A red voxel owns all its weights; a black voxel's boundary weights
// are stored nowhere, so for a black voxel on the grid boundary w_bnd =
// (D - 1)/c - (sum of the weights in the flux), and 0 elsewhere.  xs, b,
// gm, dg: the group's u, b, gamma, D, loaded by the caller before the call.
template <int C, int N>
__device__ __forceinline__ void flux_residual_vec(const Layout &L, const float *__restrict__ x,
                                                  const float *__restrict__ W, bool act, int row,
                                                  int s0, const RowPos &rp,
                                                  const float (&xs)[N], const float (&b)[N],
                                                  const float (&gm)[N], const float (&dg)[N],
                                                  float (&r)[N])
{
    const int e = C ^ rp.p;
    gather_core<C, float, N, true>(
        L, x, W, act, row, s0, rp,
        [&](int m, float xm, float xp, float wm, float wp, bool inm, bool inp,
            const float (&a)[6][N], const float (&y)[6][N], const bool (&in)[6]) {
            const float u = xs[m];
            const float flux = sum8(inm ? __fmul_rn(wm, __fsub_rn(u, xm)) : 0.0f,
                                    inp ? __fmul_rn(wp, __fsub_rn(u, xp)) : 0.0f,
                                    in[0] ? __fmul_rn(a[0][m], __fsub_rn(u, y[0][m])) : 0.0f,
                                    in[1] ? __fmul_rn(a[1][m], __fsub_rn(u, y[1][m])) : 0.0f,
                                    in[2] ? __fmul_rn(a[2][m], __fsub_rn(u, y[2][m])) : 0.0f,
                                    in[3] ? __fmul_rn(a[3][m], __fsub_rn(u, y[3][m])) : 0.0f,
                                    in[4] ? __fmul_rn(a[4][m], __fsub_rn(u, y[4][m])) : 0.0f,
                                    in[5] ? __fmul_rn(a[5][m], __fsub_rn(u, y[5][m])) : 0.0f);
            const float c = __fmul_rn(gm[m], dg[m]);
            float wb;
            if (C == 0) {
                wb = sum8(inm ? 0.0f : wm, inp ? 0.0f : wp, in[0] ? 0.0f : a[0][m],
                          in[1] ? 0.0f : a[1][m], in[2] ? 0.0f : a[2][m], in[3] ? 0.0f : a[3][m],
                          in[4] ? 0.0f : a[4][m], in[5] ? 0.0f : a[5][m]);
            } else {
                const int i = 2 * (s0 + m) + e;
                const bool bnd = i == 0 || i + 1 == L.n1 || !(in[0] && in[1] && in[2] && in[3] &&
                                                              in[4] && in[5]);
                const float wint = sum8(inm ? wm : 0.0f, inp ? wp : 0.0f, in[0] ? a[0][m] : 0.0f,
                                        in[1] ? a[1][m] : 0.0f, in[2] ? a[2][m] : 0.0f,
                                        in[3] ? a[3][m] : 0.0f, in[4] ? a[4][m] : 0.0f,
                                        in[5] ? a[5][m] : 0.0f);
                wb = bnd ? __fsub_rn(__fdiv_rn(__fsub_rn(dg[m], 1.0f), c), wint) : 0.0f;
            }
            r[m] = __fsub_rn(__fsub_rn(b[m], u), __fmul_rn(c, __fmaf_rn(u, wb, flux)));
        });
}

// One colour-C relaxation of the N voxels of a group (see gather_vec):
// x <- x + omega (B + G acc - x) with B and G the [2][S] per-voxel
// coefficients, the arithmetic of gather_vec + relax.  kUnit: G = 1 (the
// symmetrically scaled system, where no G is stored or read).  kOwnW (black
// only): W is the copy of the weights by black end (gather_core).  Slots past
// the row end (i >= n1) are padding and keep their value (zero).
template <int C, typename WT, int N, bool kUnit = false, bool kOwnW = false>
__device__ __forceinline__ void relax_vec(const Layout &L, float *__restrict__ x,
                                          const float *__restrict__ B,
                                          const float *__restrict__ Gm,
                                          const WT *__restrict__ W, float omega, bool act,
                                          int row, int s0, const RowPos &rp)
{
    const long long S = L.S;
    const long long q = (long long)row * L.P + s0;
    float *xs = x + (C ? S : 0);
    float Xs[N], Bp[N], Gp[N], acc[N];
    ldv<N>(Xs, act, xs + q);
    ldv<N>(Bp, act, B + C * S + q);
    if (kUnit) {
#pragma unroll
        for (int m = 0; m < N; ++m) Gp[m] = 1.0f;
    } else {
        ldv<N>(Gp, act, Gm + C * S + q);
    }
    gather_vec<C, WT, N, kOwnW>(L, x, W, act, row, s0, rp, acc);
    if (!act) return;
    const int e = C ^ rp.p;
    float out[N];
#pragma unroll
    for (int m = 0; m < N; ++m)
        out[m] = 2 * (s0 + m) + e < L.n1 ? relax(Xs[m], Bp[m], Gp[m], acc[m], omega) : Xs[m];
    stv<N>(xs + q, out);
}

// Per-thread record (sum of squares, min, max) in FP32, the sum compensated
// (TwoSum, error term carried separately), so that a thread's share is
// accurate to FP32 rounding of its final value; converted to the FP64 Acc3
// for the block and grid reductions.  Keeps FP64 arithmetic (a slow pipe on
// this part) out of the per-voxel loop.
struct Rec3f {
    float s, c, mn, mx;
};

__device__ __forceinline__ Rec3f rec3f_init() { return {0.0f, 0.0f, FLT_MAX, -FLT_MAX}; }

__device__ __forceinline__ void rec3f_add(Rec3f &a, float v2, float u)
{
    const float t = __fadd_rn(a.s, v2);
    const float bp = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(v2, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, err);
    a.mn = fminf(a.mn, u);
    a.mx = fmaxf(a.mx, u);
}

__device__ __forceinline__ Acc3 rec3f_acc(const Rec3f &a)
{
    return {(double)a.s + (double)a.c, (double)a.mn, (double)a.mx};
}

// ------------------------------------------------------- step coefficients

struct StepConst {
    float inv_h[4];    // 1/h_d
    float inv_h2[4];   // 1/h_d^2
    float tau, eps2;
};

// Reduced diamond-cell |grad^f u|^2 (times nothing: already divided by h) on
// the 8 faces of voxel c = (i,j,k,l), zero Dirichlet ghosts (Section 3.2).
// The normal component of face (d, +-) is (u(+-e_d) - u)/h_d.  Its tangential
// component along t is the difference of the two diamond-point values,
//   (1/4) [ (u(+e_t) - u(-e_t)) + (u(+-e_d+e_t) - u(+-e_d-e_t)) ] / h_t.
// Each unordered axis pair (d, t) has 4 edge neighbours u(+-e_d +-e_t), which
// serve the t-component of both d-faces and the d-component of both t-faces.
//
// |grad^f u|^2 of the 8 faces from gathered values: u0 = u(x), sm[d] / sp[d]
// = u(x -+ e_d), ed[pi][a][b] = u(x + (a ? 1 : -1) e_d + (b ? 1 : -1) e_t)
// for the axis pairs pi = (d, t), d < t, in the order (0,1) (0,2) (0,3)
// (1,2) (1,3) (2,3).
__device__ __forceinline__ void face_grad_sq8_from(float u0, const float (&sm)[4],
                                                   const float (&sp)[4],
                                                   const float (&ed)[6][2][2],
                                                   const float *inv_h, float g2[8])
{
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const float nm = (sm[d] - u0) * inv_h[d];
        const float np = (sp[d] - u0) * inv_h[d];
        g2[2 * d] = nm * nm;
        g2[2 * d + 1] = np * np;
    }
    int pi = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
#pragma unroll
        for (int t = d + 1; t < 4; ++t, ++pi) {
            const float(&e)[2][2] = ed[pi];
            const float dt0 = sp[t] - sm[t];   // u(+e_t) - u(-e_t)
            const float dd0 = sp[d] - sm[d];   // u(+e_d) - u(-e_d)
            // faces (d, -) and (d, +): component along t
            const float cdm = 0.25f * (dt0 + (e[0][1] - e[0][0])) * inv_h[t];
            const float cdp = 0.25f * (dt0 + (e[1][1] - e[1][0])) * inv_h[t];
            // faces (t, -) and (t, +): component along d
            const float ctm = 0.25f * (dd0 + (e[1][0] - e[0][0])) * inv_h[d];
            const float ctp = 0.25f * (dd0 + (e[1][1] - e[0][1])) * inv_h[d];
            g2[2 * d] += cdm * cdm;
            g2[2 * d + 1] += cdp * cdp;
            g2[2 * t] += ctm * ctm;
            g2[2 * t + 1] += ctp * ctp;
        }
    }
}

// The 33 values face_grad_sq8_from needs for the voxel in slot s of colour C
// in row `row` (one voxel per lane, lanes on consecutive slots): the centre,
// its 8 face neighbours (other colour) and its 24 edge neighbours (same
// colour: two steps in parity), zero outside the grid.  With i = 2s + e, the
// x-neighbours i -+ 1 of any colour-C or other-colour row are the slots
// (s-1, s) for e = 0 and (s, s+1) for e = 1 of that row, so each row array
// is loaded once per lane and the slot beside it comes from the adjacent
// lane by shuffle (or a load at a warp's end).  All 32 lanes call this;
// lanes without a voxel pass act = false.
template <int C>
__device__ __forceinline__ void coef_gather(const Layout &L, const float *__restrict__ u, bool act,
                                            int row, int s, const RowPos &rp, float &u0,
                                            float (&sm)[4], float (&sp)[4], float (&ed)[6][2][2])
{
    const long long S = L.S;
    const long long q = (long long)row * L.P + s;
    const float *uc = u + (C ? S : 0);   // same colour
    const float *uo = u + (C ? 0 : S);   // other colour
    const int e = C ^ rp.p;
    const long long dy = L.P, dz = (long long)L.n2 * L.P, dt = (long long)L.n2 * L.n3 * L.P;
    const long long off[6] = {-dy, dy, -dz, dz, -dt, dt};
    const bool in[6] = {act && rp.j > 0, act && rp.j + 1 < L.n2, act && rp.k > 0,
                        act && rp.k + 1 < L.n3, act && rp.l > 0, act && rp.l + 1 < L.n4};
    u0 = act ? uc[q] : 0.0f;
    const float X = act ? uo[q] : 0.0f;
    float nb[6], V[6], dg[3][2][2];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        nb[f] = in[f] ? uo[q + off[f]] : 0.0f;   // face neighbours along y, z, t
        V[f] = in[f] ? uc[q + off[f]] : 0.0f;    // same-colour rows of the x-edges
    }
    // edge neighbours in the (y,z), (y,t), (z,t) planes: same slot
#pragma unroll
    for (int pp = 0; pp < 3; ++pp) {
        const int da = pp < 2 ? 0 : 1, tb = pp == 0 ? 1 : 2;   // axes among (y, z, t)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const bool ok = in[2 * da + a] && in[2 * tb + b];
                dg[pp][a][b] = ok ? uc[q + off[2 * da + a] + off[2 * tb + b]] : 0.0f;
            }
    }
    const unsigned key = act ? (unsigned)q : 0xFFFFFFFFu;
    const unsigned keyL = __shfl_up_sync(0xFFFFFFFFu, key, 1);
    const unsigned keyR = __shfl_down_sync(0xFFFFFFFFu, key, 1);
    float XL, XR, VL[6], VR[6];
    XL = __shfl_up_sync(0xFFFFFFFFu, X, 1);
    XR = __shfl_down_sync(0xFFFFFFFFu, X, 1);
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        VL[f] = __shfl_up_sync(0xFFFFFFFFu, V[f], 1);
        VR[f] = __shfl_down_sync(0xFFFFFFFFu, V[f], 1);
    }
    if (!act) return;
    const bool hasL = s > 0, hasR = s + 1 < L.P;
    const bool shL = hasL && keyL == (unsigned)(q - 1);
    const bool shR = hasR && keyR == (unsigned)(q + 1);
    if (e == 0) {   // x -+ 1 are slots s-1, s
        sm[0] = shL ? XL : (hasL ? uo[q - 1] : 0.0f);
        sp[0] = X;
    } else {        // slots s, s+1
        sm[0] = X;
        sp[0] = shR ? XR : (hasR ? uo[q + 1] : 0.0f);
    }
#pragma unroll
    for (int d = 1; d < 4; ++d) {
        sm[d] = nb[2 * d - 2];
        sp[d] = nb[2 * d - 1];
    }
    // (x, t) edges, t = y, z, t: pairs 0, 1, 2; a = x side, b = t side
#pragma unroll
    for (int t = 0; t < 3; ++t)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int f = 2 * t + b;
            if (e == 0) {
                ed[t][0][b] = shL ? VL[f] : (hasL && in[f] ? uc[q + off[f] - 1] : 0.0f);
                ed[t][1][b] = V[f];
            } else {
                ed[t][0][b] = V[f];
                ed[t][1][b] = shR ? VR[f] : (hasR && in[f] ? uc[q + off[f] + 1] : 0.0f);
            }
        }
#pragma unroll
    for (int pp = 0; pp < 3; ++pp)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) ed[3 + pp][a][b] = dg[pp][a][b];
}

__device__ __forceinline__ float ghost_at(const Ghost &G, const float *g, const Layout &L, int c0,
                                          int c1, int c2, int c3)
{
    const int c[4] = {c0, c1, c2, c3};
    const int n[4] = {L.n1, L.n2, L.n3, L.n4};
    int d = 0;
    while (d < 3 && c[d] >= 0 && c[d] < n[d]) ++d;
    long long idx = G.off[d] + (c[d] < 0 ? 0 : G.size[d]), stride = 1;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (e == d) continue;
        idx += (long long)(c[e] + 1) * stride;
        stride *= G.np[e];
    }
    return g[idx];
}

// The gathered values of voxel (i, j, k, l) with the neighbours that lie on
// the ghost ring taken from G.prev instead of zero.
__device__ __forceinline__ void apply_ghosts(const Ghost &G, const Layout &L, int i, int j, int k,
                                             int l, float (&sm)[4], float (&sp)[4],
                                             float (&ed)[6][2][2])
{
    const int c[4] = {i, j, k, l};
    const int n[4] = {L.n1, L.n2, L.n3, L.n4};
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        int a[4] = {c[0], c[1], c[2], c[3]};
        a[d] = c[d] - 1;
        if (a[d] < 0) sm[d] = ghost_at(G, G.prev, L, a[0], a[1], a[2], a[3]);
        a[d] = c[d] + 1;
        if (a[d] >= n[d]) sp[d] = ghost_at(G, G.prev, L, a[0], a[1], a[2], a[3]);
    }
    int pi = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int t = d + 1; t < 4; ++t, ++pi)
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    int q[4] = {c[0], c[1], c[2], c[3]};
                    q[d] += a ? 1 : -1;
                    q[t] += b ? 1 : -1;
                    if (q[d] < 0 || q[d] >= n[d] || q[t] < 0 || q[t] >= n[t])
                        ed[pi][a][b] = ghost_at(G, G.prev, L, q[0], q[1], q[2], q[3]);
                }
}

// Step coefficients of one voxel (Eq. new1) from its gathered values and
// its 8 face edge coefficients g: A_f = sqrt(eps^2 + |grad^f u|^2),
// Abar = sqrt(eps^2 + (1/8) sum_f |grad^f u|^2), w_f = G_f / (A_f h_d^2),
// c = tau Abar, D = 1 + c sum_f w_f, beta = b / D, gamma = c / D (b = u0).
// 1/A_f is a correctly rounded reciprocal square root and both quotients by
// D use one correctly rounded reciprocal (IEEE operations, no approximate
// intrinsics): the coefficients are defined to FP32 accuracy, not to the bit,
// and the solve meets its tolerance on whatever system they form.
__device__ __forceinline__ void coef_finish(const StepConst &K, const float (&g)[8], float u0,
                                            const float (&sm)[4], const float (&sp)[4],
                                            const float (&ed)[6][2][2], float (&w)[8],
                                            float &D, float &bt, float &gm, float &cc)
{
    float g2[8];
    face_grad_sq8_from(u0, sm, sp, ed, K.inv_h, g2);
    float sum = 0.0f;
#pragma unroll
    for (int f = 0; f < 8; ++f) sum += g2[f];
    const float Abar = sqrtf(K.eps2 + 0.125f * sum);
    cc = K.tau * Abar;
    float wsum = 0.0f;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
        w[f] = g[f] * __frsqrt_rn(K.eps2 + g2[f]) * K.inv_h2[f >> 1];
        wsum += w[f];
    }
    D = 1.0f + cc * wsum;
    const float iD = __frcp_rn(D);
    bt = u0 * iD;
    gm = cc * iD;
}

// Sum over the interior faces of (w_f - bf16(w_f)) for the voxel in slot s
// (red voxels own their weights, black voxels read them across the face).
template <int C>
__device__ __forceinline__ float rounding_excess(const Layout &L, const float *__restrict__ W,
                                                 int row, int s, const RowPos &rp)
{
    const long long S = L.S;
    const long long rb = (long long)row * L.P;
    const long long q = rb + s;
    const long long dy = L.P, dz = (long long)L.n2 * L.P, dt = (long long)L.n2 * L.n3 * L.P;
    long long idx[8];
    bool in[8];
    if (C == 0) {
        in[0] = s - 1 + rp.p >= 0 && 2 * s + rp.p >= 1;
        in[1] = 2 * s + rp.p + 1 < L.n1;
        for (int f = 0; f < 8; ++f) idx[f] = (long long)f * S + q;
    } else {
        const int i = 2 * s + 1 - rp.p;
        in[0] = i >= 1;
        in[1] = i + 1 < L.n1;
        idx[0] = 1 * S + rb + s - rp.p;
        idx[1] = 0 * S + rb + s + 1 - rp.p;
        idx[2] = 3 * S + q - dy;
        idx[3] = 2 * S + q + dy;
        idx[4] = 5 * S + q - dz;
        idx[5] = 4 * S + q + dz;
        idx[6] = 7 * S + q - dt;
        idx[7] = 6 * S + q + dt;
    }
    in[2] = rp.j > 0;
    in[3] = rp.j + 1 < L.n2;
    in[4] = rp.k > 0;
    in[5] = rp.k + 1 < L.n3;
    in[6] = rp.l > 0;
    in[7] = rp.l + 1 < L.n4;
    float ex = 0.0f;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
        if (!in[f]) continue;
        const float w = W[idx[f]];
        ex += w - __bfloat162float(__float2bfloat16_rn(w));
    }
    return ex;
}

}  // namespace seg4d_impl
