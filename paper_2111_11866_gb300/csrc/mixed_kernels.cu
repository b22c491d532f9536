// mixed_kernels.cu -- the mixed-precision solve (params.precision = 1).
//
// The sweeps stream BF16 face weights wb_f = bf16(w_f) instead of FP32 ones
// (8 instead of 16 bytes per voxel per colour pass).  The BF16 system A_b
// keeps the structure of Eq. new1: its diagonal D_b = 1 + c (sum over interior
// faces of wb_f + sum over boundary faces of w_f) is built from the same
// rounded weights, so A_b is again a strictly diagonally dominant M-matrix.
// Accuracy is won back by defect correction against the exact FP32 system A:
//   r = b - A u             (exact FP32 weights, FP64 norms: the stopping test)
//   solve A_b delta = r     (red-black SOR on delta from 0, BF16 weights)
//   u <- u + delta
// The fixed point is A u = b, the same as the plain FP32 path's.
#include <cuda_bf16.h>

#include "stencil.cuh"

namespace seg4d_impl {

// Grid-stride over the sweep's 32 x 8 tiles (as in solve_kernels.cu).
#define MX_FOR_TILES(L, s, rp, row, BODY)                                                  \
    {                                                                                      \
        const long long ntile_ = (long long)(L).nchunk * (L).njb * (L).n3 * (L).n4;       \
        for (long long t_ = blockIdx.x; t_ < ntile_; t_ += gridDim.x) {                    \
            const int chunk_ = (int)(t_ % (L).nchunk);                                     \
            long long r_ = t_ / (L).nchunk;                                                \
            const int jb_ = (int)(r_ % (L).njb);                                           \
            r_ /= (L).njb;                                                                 \
            RowPos rp;                                                                     \
            rp.k = (int)(r_ % (L).n3);                                                     \
            rp.l = (int)(r_ / (L).n3);                                                     \
            rp.j = jb_ * 8 + (int)(threadIdx.x >> 5);                                      \
            const int s = chunk_ * 32 + (int)(threadIdx.x & 31);                           \
            if (rp.j < (L).n2 && s < (L).P) {                                              \
                rp.p = (rp.j + rp.k + rp.l) & 1;                                           \
                const int row = rp.j + (L).n2 * (rp.k + (L).n3 * rp.l);                   \
                BODY                                                                       \
            }                                                                              \
        }                                                                                  \
    }

// After the FP32 coefficients: Wb = bf16(W) (red ends); per voxel
// gamma_b = c / D_b, invD_b = 1 / D_b with D_b = D - c * excess, c = gamma*D.
__global__ void __launch_bounds__(256) k_mixed_prepare(Layout L, const float *__restrict__ W,
                                                       const float *__restrict__ gamma,
                                                       const float *__restrict__ diag,
                                                       __nv_bfloat16 *__restrict__ Wb,
                                                       float *__restrict__ gb,
                                                       float *__restrict__ ib)
{
    MX_FOR_TILES(L, s, rp, row, {
        const long long q = (long long)row * L.P + s;
        for (int C = 0; C < 2; ++C) {
            if (2 * s + (C ^ rp.p) >= L.n1) continue;
            const float D = diag[C * L.S + q];
            const float c = gamma[C * L.S + q] * D;
            const float ex = C ? rounding_excess<1>(L, W, row, s, rp)
                               : rounding_excess<0>(L, W, row, s, rp);
            const float Db = D - c * ex;
            gb[C * L.S + q] = c / Db;
            ib[C * L.S + q] = 1.0f / Db;
            if (C == 0)
                for (int f = 0; f < 8; ++f)
                    Wb[(long long)f * L.S + q] = __float2bfloat16_rn(W[(long long)f * L.S + q]);
        }
    })
}

// Defect pass: the exact residual r of every voxel in flux form
// (flux_residual_vec); rho = r / D_b, delta = 0; records (sum r^2, min u,
// max u) in `partials` and max |r| of each block in amax[block].  b is the
// prepared beta array.  Work items and grid as the residual kernel: item
// t = 2 * tile + colour over the sweep's tiles.
template <int N>
__global__ void __launch_bounds__(256, SEG4D_DEFECT_MINB) k_defect(Layout L, const float *__restrict__ u,
                                                   const float *__restrict__ b,
                                                   const float *__restrict__ gamma,
                                                   const float *__restrict__ diag,
                                                   const float *__restrict__ W,
                                                   const float *__restrict__ ib,
                                                   float *__restrict__ rho,
                                                   float *__restrict__ delta,
                                                   double *__restrict__ partials,
                                                   double *__restrict__ amax,
                                                   ItemDecode dec, unsigned items)
{
    Rec3f a = rec3f_init();
    float ra = 0.0f;   // max |r| of the thread's voxels
    for (unsigned t = blockIdx.x; t < items; t += gridDim.x) {
        int C, chunk;
        RowPos rp;
        decode_item(dec, L, t, (int)(threadIdx.x >> 5), C, chunk, rp);
        const int s0 = chunk * 32 * N + N * (int)(threadIdx.x & 31);
        if (rp.j >= L.n2) continue;   // the whole warp
        const bool act = s0 < L.P && 2 * s0 + (C ^ rp.p) < L.n1;
        const int row = rp.j + L.n2 * (rp.k + L.n3 * rp.l);
        const long long q = (long long)row * L.P + s0 + (C ? L.S : 0);
        float xs[N], bv[N], gm[N], dg[N], iv[N], res[N];
        ldv<N>(xs, act, u + q);
        ldv<N>(bv, act, b + q);
        ldv<N>(gm, act, gamma + q);
        ldv<N>(dg, act, diag + q);
        ldv<N>(iv, act, ib + q);
        if (C)
            flux_residual_vec<1, N>(L, u, W, act, row, s0, rp, xs, bv, gm, dg, res);
        else
            flux_residual_vec<0, N>(L, u, W, act, row, s0, rp, xs, bv, gm, dg, res);
        if (!act) continue;
        const int e = C ^ rp.p;
        float rh[N], zero[N];
#pragma unroll
        for (int m = 0; m < N; ++m) {
            zero[m] = 0.0f;
            rh[m] = 0.0f;
            if (2 * (s0 + m) + e < L.n1) {
                rh[m] = __fmul_rn(res[m], iv[m]);
                rec3f_add(a, __fmul_rn(res[m], res[m]), xs[m]);
                ra = fmaxf(ra, fabsf(res[m]));
            }
        }
        stv<N>(rho + q, rh);
        stv<N>(delta + q, zero);
    }
    block_write3(rec3f_acc(a), partials + 3 * blockIdx.x);
    block_write_max(ra, amax + blockIdx.x);
}

// Before an FP32 solve (the correction sweeps run on the scaled system, see
// k_scaled_weights): per voxel r = sqrt(gamma) and ib = 1 / (D r), so that
// the defect pass writes the scaled right-hand side rho = r_res / (D r).
// Without rs (a lean handle sweeps the unscaled correction system) ib = 1/D.
// Padding slots (gamma = 0) get r = ib = 0.
__global__ void __launch_bounds__(256) k_plain_prepare(long long n4,
                                                       const float4 *__restrict__ gamma,
                                                       const float4 *__restrict__ diag,
                                                       float4 *__restrict__ rs,
                                                       float4 *__restrict__ ib)
{
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n4;
         e += (long long)gridDim.x * blockDim.x) {
        const float4 g = gamma[e], d = diag[e];
        const float *gp = &g.x, *dp = &d.x;
        float4 r, iv;
        float *rp = &r.x, *ip = &iv.x;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            rp[m] = gp[m] > 0.0f ? sqrtf(gp[m]) : 0.0f;
            // unscaled correction system (no rs): rho = r_res / D
            ip[m] = gp[m] > 0.0f ? 1.0f / (rs ? dp[m] * rp[m] : dp[m]) : 0.0f;
        }
        if (rs) rs[e] = r;
        ib[e] = iv;
    }
}

// u <- u + r delta (the FP32 solve's correction is in scaled units)
__global__ void __launch_bounds__(256) k_apply_scaled(float4 *__restrict__ u,
                                                      const float4 *__restrict__ delta,
                                                      const float4 *__restrict__ rs, long long n4)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        float4 a = u[i];
        const float4 b = delta[i], r = rs[i];
        a.x = __fmaf_rn(r.x, b.x, a.x);
        a.y = __fmaf_rn(r.y, b.y, a.y);
        a.z = __fmaf_rn(r.z, b.z, a.z);
        a.w = __fmaf_rn(r.w, b.w, a.w);
        u[i] = a;
    }
}

// u <- u + delta over both colour halves (padding holds 0 in both)
__global__ void __launch_bounds__(256) k_apply(float4 *__restrict__ u,
                                               const float4 *__restrict__ delta, long long n4)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        float4 a = u[i];
        const float4 b = delta[i];
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
        u[i] = a;
    }
}

void launch_mixed_prepare(const Layout &L, const float *W, const float *gamma, const float *diag,
                          void *Wb, float *gb, float *ib, cudaStream_t st)
{
    k_mixed_prepare<<<kPartBlocks, 256, 0, st>>>(L, W, gamma, diag, (__nv_bfloat16 *)Wb, gb, ib);
}

int launch_defect(const Layout &L, const float *u, const float *b, const float *gamma,
                  const float *diag, const float *W, const float *ib, float *rho, float *delta,
                  double *partials, double *amax, cudaStream_t st)
{
    const int nch = (L.P + 32 * kDefectN - 1) / (32 * kDefectN);
    const long long items = item_count(L, nch);
    const int blocks = (int)(items < kResBlocks ? items : kResBlocks);
    k_defect<kDefectN><<<blocks, 256, 0, st>>>(L, u, b, gamma, diag, W, ib, rho, delta, partials,
                                               amax, make_item_decode(L, nch), (unsigned)items);
    return blocks;
}

static int vec4_blocks(long long n4)
{
    long long blocks = (n4 + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    return (int)(blocks < 1 ? 1 : blocks);
}

void launch_plain_prepare(const Layout &L, const float *gamma, const float *diag, float *rs,
                          float *ib, cudaStream_t st)
{
    const long long n4 = 2 * L.S / 4;   // P is a multiple of 4
    k_plain_prepare<<<vec4_blocks(n4), 256, 0, st>>>(n4, (const float4 *)gamma,
                                                     (const float4 *)diag, (float4 *)rs,
                                                     (float4 *)ib);
}

void launch_apply_scaled(const Layout &L, float *u, const float *delta, const float *rs,
                         cudaStream_t st)
{
    const long long n4 = 2 * L.S / 4;
    k_apply_scaled<<<vec4_blocks(n4), 256, 0, st>>>((float4 *)u, (const float4 *)delta,
                                                    (const float4 *)rs, n4);
}

void launch_apply(const Layout &L, float *u, const float *delta, cudaStream_t st)
{
    // 2S floats; P is a multiple of 4, so 2S is too and the halves are 16-byte aligned
    const long long n4 = 2 * L.S / 4;
    long long blocks = (n4 + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    k_apply<<<(int)(blocks < 1 ? 1 : blocks), 256, 0, st>>>((float4 *)u, (const float4 *)delta,
                                                            n4);
}

}  // namespace seg4d_impl
