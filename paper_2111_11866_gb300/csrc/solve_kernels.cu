// solve_kernels.cu -- per-step coefficients (Eqs. 111th, new1), the red-black
// SOR half sweep (Eqs. 5.33, gsee with the red-black ordering of Section 3.2),
// the residual of the step system and the FP64 reductions of the stopping
// test.  Layout: seg4d_internal.cuh.
#include <cfloat>
#include <cmath>

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

__device__ inline RowPos row_pos(const Layout &L, int row)
{
    RowPos r;
    r.j = row % L.n2;
    const int t = row / L.n2;
    r.k = t % L.n3;
    r.l = t / L.n3;
    r.p = (r.j + r.k + r.l) & 1;
    return r;
}

// Sum over the 8 faces of  w_f * x_nb(f)  for the voxel in slot s of row `row`
// (colour C, row parity p); neighbours outside the grid are Dirichlet zeros.
// Red voxels own their 8 face weights; a black voxel reads each weight from
// the red voxel across the face (opposite face index).
template <int C>
__device__ __forceinline__ float neighbour_sum(const Layout &L, const float *__restrict__ xo,
                                               const float *__restrict__ W, int row, int s,
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
        t0 = sxm >= 0 ? W[0 * S + q] * xo[rb + sxm] : 0.0f;
        t1 = sxp < L.P ? W[1 * S + q] * xo[rb + sxp] : 0.0f;
        t2 = rp.j > 0 ? W[2 * S + q] * xo[q - dy] : 0.0f;
        t3 = rp.j + 1 < L.n2 ? W[3 * S + q] * xo[q + dy] : 0.0f;
        t4 = rp.k > 0 ? W[4 * S + q] * xo[q - dz] : 0.0f;
        t5 = rp.k + 1 < L.n3 ? W[5 * S + q] * xo[q + dz] : 0.0f;
        t6 = rp.l > 0 ? W[6 * S + q] * xo[q - dt] : 0.0f;
        t7 = rp.l + 1 < L.n4 ? W[7 * S + q] * xo[q + dt] : 0.0f;
    } else {
        const int sxm = s - rp.p, sxp = s + 1 - rp.p;
        t0 = sxm >= 0 ? W[1 * S + rb + sxm] * xo[rb + sxm] : 0.0f;
        t1 = sxp < L.P ? W[0 * S + rb + sxp] * xo[rb + sxp] : 0.0f;
        t2 = rp.j > 0 ? W[3 * S + q - dy] * xo[q - dy] : 0.0f;
        t3 = rp.j + 1 < L.n2 ? W[2 * S + q + dy] * xo[q + dy] : 0.0f;
        t4 = rp.k > 0 ? W[5 * S + q - dz] * xo[q - dz] : 0.0f;
        t5 = rp.k + 1 < L.n3 ? W[4 * S + q + dz] * xo[q + dz] : 0.0f;
        t6 = rp.l > 0 ? W[7 * S + q - dt] * xo[q - dt] : 0.0f;
        t7 = rp.l + 1 < L.n4 ? W[6 * S + q + dt] * xo[q + dt] : 0.0f;
    }
    return ((t0 + t1) + (t2 + t3)) + ((t4 + t5) + (t6 + t7));
}

// ------------------------------------------------------------ red-black sweep

// One half sweep of colour C: every voxel of that colour gets
//   ubar = (b + c sum_f w_f u_nb) / D   (the Gauss-Seidel value of Eq. gsee,
//   here = beta + gamma * sum_f w_f u_nb with beta = b/D, gamma = c/D), then
//   u <- u + omega (ubar - u)           (Eq. 5.33).
// Grid: x = 32-slot chunk + nchunk * (8-row block along y), y = k, z = l;
// block (32, 8).  A warp covers 32 consecutive slots of one row.
template <int C>
__global__ void __launch_bounds__(256) k_sweep(Layout L, float *__restrict__ x,
                                               const float *__restrict__ beta,
                                               const float *__restrict__ gamma,
                                               const float *__restrict__ W, float omega)
{
    const int chunk = blockIdx.x % L.nchunk;
    const int jb = blockIdx.x / L.nchunk;
    const int s = chunk * 32 + threadIdx.x;
    RowPos rp;
    rp.j = jb * 8 + threadIdx.y;
    rp.k = blockIdx.y;
    rp.l = blockIdx.z;
    if (rp.j >= L.n2 || s >= L.P) return;
    rp.p = (rp.j + rp.k + rp.l) & 1;
    if (2 * s + (C ^ rp.p) >= L.n1) return;
    const int row = rp.j + L.n2 * (rp.k + L.n3 * rp.l);
    const long long q = (long long)row * L.P + s;
    const float *xo = x + (C ? 0 : L.S);
    float *xs = x + (C ? L.S : 0);
    const float acc = neighbour_sum<C>(L, xo, W, row, s, rp);
    const float ubar = beta[C * L.S + q] + gamma[C * L.S + q] * acc;
    const float u0 = xs[q];
    xs[q] = u0 + omega * (ubar - u0);
}

void launch_sweep(const Layout &L, int colour, float *x, const float *beta, const float *gamma,
                  const float *W, float omega, cudaStream_t st)
{
    dim3 block(32, 8);
    dim3 grid((unsigned)(L.nchunk * L.njb), (unsigned)L.n3, (unsigned)L.n4);
    if (colour == 0)
        k_sweep<0><<<grid, block, 0, st>>>(L, x, beta, gamma, W, omega);
    else
        k_sweep<1><<<grid, block, 0, st>>>(L, x, beta, gamma, W, omega);
}

// --------------------------------------------------------------- residual

// r_v = b_v - (A u)_v = D_v (ubar_v - u_v) for every voxel; per-block records
// of (sum r^2, min u, max u) in FP64.  One warp per (colour, row) unit.
__global__ void __launch_bounds__(kPartThreads) k_residual(Layout L, const float *__restrict__ x,
                                                           const float *__restrict__ beta,
                                                           const float *__restrict__ gamma,
                                                           const float *__restrict__ diag,
                                                           const float *__restrict__ W,
                                                           double *__restrict__ partials)
{
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    Acc3 a{0.0, DBL_MAX, -DBL_MAX};
    for (long long unit = warp0; unit < 2LL * L.R; unit += nwarps) {
        const int C = unit >= L.R ? 1 : 0;
        const int row = (int)(unit - (long long)C * L.R);
        const RowPos rp = row_pos(L, row);
        for (int s = lane; s < L.P; s += 32) {
            if (2 * s + (C ^ rp.p) >= L.n1) continue;
            const long long q = (long long)row * L.P + s;
            const float acc = C ? neighbour_sum<1>(L, x, W, row, s, rp)
                                : neighbour_sum<0>(L, x + L.S, W, row, s, rp);
            const float u = x[C * L.S + q];
            const float ubar = beta[C * L.S + q] + gamma[C * L.S + q] * acc;
            const double r = (double)diag[C * L.S + q] * ((double)ubar - (double)u);
            a.sum += r * r;
            a.mn = fmin(a.mn, (double)u);
            a.mx = fmax(a.mx, (double)u);
        }
    }
    block_write3(a, partials + 3 * blockIdx.x);
}

void launch_residual(const Layout &L, const float *x, const float *beta, const float *gamma,
                     const float *diag, const float *W, double *partials, int nparts,
                     cudaStream_t st)
{
    k_residual<<<nparts, kPartThreads, 0, st>>>(L, x, beta, gamma, diag, W, partials);
}

// Deterministic final reduction of the per-block records (one block).
__global__ void __launch_bounds__(1024) k_reduce(const double *__restrict__ partials, int n,
                                                 double *__restrict__ out)
{
    Acc3 a{0.0, DBL_MAX, -DBL_MAX};
    for (int b = threadIdx.x; b < n; b += blockDim.x)
        a = acc3_merge(a, Acc3{partials[3 * b], partials[3 * b + 1], partials[3 * b + 2]});
    block_write3(a, out);
}

void launch_reduce_partials(const double *partials, int nparts, double *out, cudaStream_t st)
{
    k_reduce<<<1, 1024, 0, st>>>(partials, nparts, out);
}

// ------------------------------------------------------- step coefficients

struct StepConst {
    float inv_h[4];    // 1/h_d
    float inv_h2[4];   // 1/h_d^2
    float tau, eps2;
};

// Reduced diamond-cell |grad^f u|^2 on the 8 faces of voxel (i,j,k,l) from a
// u-like field with zero Dirichlet ghosts (Section 3.2):  the normal
// component is (u_nb - u)/h_d; the tangential one along t is the difference of
// the two diamond-point values, i.e. (1/4)(u(+t) + u_nb(+t) - u(-t) - u_nb(-t))/h_t.
__device__ inline void face_grad_sq8(const Layout &L, const float *__restrict__ u, int i, int j,
                                     int k, int l, const float *inv_h, float g2[8])
{
    const int c[4] = {i, j, k, l};
    const float u0 = ld_dirichlet(L, u, i, j, k, l);
#pragma unroll
    for (int f = 0; f < 8; ++f) {
        const int d = f >> 1;
        const int sg = (f & 1) ? 1 : -1;
        int nb[4] = {c[0], c[1], c[2], c[3]};
        nb[d] += sg;
        const float un = ld_dirichlet(L, u, nb[0], nb[1], nb[2], nb[3]);
        const float nrm = (un - u0) * inv_h[d];
        float sum = nrm * nrm;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (t == d) continue;
            int a[4] = {c[0], c[1], c[2], c[3]};
            int b[4] = {nb[0], nb[1], nb[2], nb[3]};
            a[t] += 1;
            b[t] += 1;
            const float up = ld_dirichlet(L, u, a[0], a[1], a[2], a[3]) +
                             ld_dirichlet(L, u, b[0], b[1], b[2], b[3]);
            a[t] -= 2;
            b[t] -= 2;
            const float dn = ld_dirichlet(L, u, a[0], a[1], a[2], a[3]) +
                             ld_dirichlet(L, u, b[0], b[1], b[2], b[3]);
            const float comp = 0.25f * (up - dn) * inv_h[t];
            sum += comp * comp;
        }
        g2[f] = sum;
    }
}

// Coefficients of the step system from u = u^{resc,n-1} (also b):
//   A_f = sqrt(eps^2 + |grad^f u|^2), Abar = sqrt(eps^2 + (1/8) sum_f |grad^f u|^2)
//   w_f = G_f / (A_f h_d^2), c = tau * Abar, D = 1 + c sum_f w_f      (Eq. new1)
//   beta = b / D, gamma = c / D.
// Red voxels store their 8 w_f.  Records: (sum b^2, min b, max b).
__global__ void __launch_bounds__(kPartThreads) k_step_coef(Layout L, const float *__restrict__ u,
                                                            const float *__restrict__ G,
                                                            StepConst K, float *__restrict__ beta,
                                                            float *__restrict__ gamma,
                                                            float *__restrict__ diag,
                                                            float *__restrict__ W,
                                                            double *__restrict__ partials)
{
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    Acc3 a{0.0, DBL_MAX, -DBL_MAX};
    for (long long unit = warp0; unit < 2LL * L.R; unit += nwarps) {
        const int C = unit >= L.R ? 1 : 0;
        const int row = (int)(unit - (long long)C * L.R);
        const RowPos rp = row_pos(L, row);
        for (int s = lane; s < L.P; s += 32) {
            const int i = 2 * s + (C ^ rp.p);
            if (i >= L.n1) continue;
            const long long q = (long long)row * L.P + s;
            float g2[8];
            face_grad_sq8(L, u, i, rp.j, rp.k, rp.l, K.inv_h, g2);
            float sum = 0.0f;
#pragma unroll
            for (int f = 0; f < 8; ++f) sum += g2[f];
            const float Abar = sqrtf(K.eps2 + 0.125f * sum);
            const float cc = K.tau * Abar;
            float wsum = 0.0f;
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                const float Af = sqrtf(K.eps2 + g2[f]);
                const float w = G[((long long)C * 8 + f) * L.S + q] / Af * K.inv_h2[f >> 1];
                wsum += w;
                if (C == 0) W[(long long)f * L.S + q] = w;
            }
            const float D = 1.0f + cc * wsum;
            const float b = u[C * L.S + q];
            diag[C * L.S + q] = D;
            beta[C * L.S + q] = b / D;
            gamma[C * L.S + q] = cc / D;
            a.sum += (double)b * (double)b;
            a.mn = fmin(a.mn, (double)b);
            a.mx = fmax(a.mx, (double)b);
        }
    }
    block_write3(a, partials + 3 * blockIdx.x);
}

void launch_step_coef(const Layout &L, const float *u, const float *G, const double *h,
                      double tau, double eps, float *beta, float *gamma, float *diag, float *W,
                      double *partials, int nparts, cudaStream_t st)
{
    StepConst K;
    for (int d = 0; d < 4; ++d) {
        K.inv_h[d] = (float)(1.0 / h[d]);
        K.inv_h2[d] = (float)(1.0 / (h[d] * h[d]));
    }
    K.tau = (float)tau;
    K.eps2 = (float)(eps * eps);
    k_step_coef<<<nparts, kPartThreads, 0, st>>>(L, u, G, K, beta, gamma, diag, W, partials);
}

}  // namespace seg4d_impl
