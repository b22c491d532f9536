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

struct RowPos {
    int j, k, l, p;
};

// Sum over the 8 faces of  w_f * x_nb(f)  for the voxel in slot s of row `row`
// (colour C, row parity p); neighbours outside the grid are Dirichlet zeros.
// Red voxels own their 8 face weights; a black voxel reads each weight from
// the red voxel across the face (opposite face index).
// u loads: plain, or at L2 only (ld.global.cg) where other CTAs of the same
// launch write u, so that no stale L1 line can be read.
template <bool kCG>
__device__ __forceinline__ float ldu(const float *p)
{
    return kCG ? __ldcg(p) : *p;
}

// face weight load: FP32, or BF16 widened to FP32
__device__ __forceinline__ float ldw(const float *p) { return *p; }
__device__ __forceinline__ float ldw(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

template <int C, bool kCG = false, typename WT = float>
__device__ __forceinline__ float neighbour_sum(const Layout &L, const float *__restrict__ xo,
                                               const WT *__restrict__ W, int row, int s,
                                               const RowPos &rp)
{
    const long long S = L.S;
    const long long rb = (long long)row * L.P;
    const long long q = rb + s;
    const long long dy = L.P;
    const long long dz = (long long)L.n2 * L.P;
    const long long dt = (long long)L.n2 * L.n3 * L.P;
    float t0, t1, t2, t3, t4, t5, t6, t7;
    if (C == 0) {
        const int sxm = s - 1 + rp.p, sxp = s + rp.p;
        t0 = sxm >= 0 ? ldw(W + 0 * S + q) * ldu<kCG>(xo + rb + sxm) : 0.0f;
        t1 = sxp < L.P ? ldw(W + 1 * S + q) * ldu<kCG>(xo + rb + sxp) : 0.0f;
        t2 = rp.j > 0 ? ldw(W + 2 * S + q) * ldu<kCG>(xo + q - dy) : 0.0f;
        t3 = rp.j + 1 < L.n2 ? ldw(W + 3 * S + q) * ldu<kCG>(xo + q + dy) : 0.0f;
        t4 = rp.k > 0 ? ldw(W + 4 * S + q) * ldu<kCG>(xo + q - dz) : 0.0f;
        t5 = rp.k + 1 < L.n3 ? ldw(W + 5 * S + q) * ldu<kCG>(xo + q + dz) : 0.0f;
        t6 = rp.l > 0 ? ldw(W + 6 * S + q) * ldu<kCG>(xo + q - dt) : 0.0f;
        t7 = rp.l + 1 < L.n4 ? ldw(W + 7 * S + q) * ldu<kCG>(xo + q + dt) : 0.0f;
    } else {
        const int sxm = s - rp.p, sxp = s + 1 - rp.p;
        t0 = sxm >= 0 ? ldw(W + 1 * S + rb + sxm) * ldu<kCG>(xo + rb + sxm) : 0.0f;
        t1 = sxp < L.P ? ldw(W + 0 * S + rb + sxp) * ldu<kCG>(xo + rb + sxp) : 0.0f;
        t2 = rp.j > 0 ? ldw(W + 3 * S + q - dy) * ldu<kCG>(xo + q - dy) : 0.0f;
        t3 = rp.j + 1 < L.n2 ? ldw(W + 2 * S + q + dy) * ldu<kCG>(xo + q + dy) : 0.0f;
        t4 = rp.k > 0 ? ldw(W + 5 * S + q - dz) * ldu<kCG>(xo + q - dz) : 0.0f;
        t5 = rp.k + 1 < L.n3 ? ldw(W + 4 * S + q + dz) * ldu<kCG>(xo + q + dz) : 0.0f;
        t6 = rp.l > 0 ? ldw(W + 7 * S + q - dt) * ldu<kCG>(xo + q - dt) : 0.0f;
        t7 = rp.l + 1 < L.n4 ? ldw(W + 6 * S + q + dt) * ldu<kCG>(xo + q + dt) : 0.0f;
    }
    return ((t0 + t1) + (t2 + t3)) + ((t4 + t5) + (t6 + t7));
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
// The centre and its 8 face neighbours are loaded once; each unordered axis
// pair (d, t) then loads its 4 edge neighbours u(+-e_d +-e_t), which serve the
// t-component of both d-faces and the d-component of both t-faces.
__device__ inline void face_grad_sq8(const Layout &L, const float *__restrict__ u, int i, int j,
                                     int k, int l, const float *inv_h, float g2[8])
{
    const int c[4] = {i, j, k, l};
    const float u0 = ld_dirichlet(L, u, i, j, k, l);
    float sm[4], sp[4];   // u(-e_d), u(+e_d)
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        int a[4] = {c[0], c[1], c[2], c[3]};
        a[d] -= 1;
        sm[d] = ld_dirichlet(L, u, a[0], a[1], a[2], a[3]);
        a[d] += 2;
        sp[d] = ld_dirichlet(L, u, a[0], a[1], a[2], a[3]);
        const float nm = (sm[d] - u0) * inv_h[d];
        const float np = (sp[d] - u0) * inv_h[d];
        g2[2 * d] = nm * nm;
        g2[2 * d + 1] = np * np;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d) {
#pragma unroll
        for (int t = d + 1; t < 4; ++t) {
            float e[2][2];   // e[sd][st] = u(x + sd' e_d + st' e_t), index 0 = -1, 1 = +1
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    int q[4] = {c[0], c[1], c[2], c[3]};
                    q[d] += a ? 1 : -1;
                    q[t] += b ? 1 : -1;
                    e[a][b] = ld_dirichlet(L, u, q[0], q[1], q[2], q[3]);
                }
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
