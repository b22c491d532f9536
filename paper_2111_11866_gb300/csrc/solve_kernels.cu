// solve_kernels.cu -- per-step coefficients (Eqs. 111th, new1), the red-black
// SOR half sweep (Eqs. 5.33, gsee with the red-black ordering of Section 3.7),
// the residual of the step system and the FP64 reductions of the stopping
// test.  Layout: seg4d_internal.cuh.
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "stencil.cuh"

namespace seg4d_impl {

// ------------------------------------------------------------ red-black sweep

// One half sweep of colour C: every voxel of that colour gets
//   ubar = (b + c sum_f w_f u_nb) / D   (the Gauss-Seidel value of Eq. gsee,
//   here = beta + gamma * sum_f w_f u_nb with beta = b/D, gamma = c/D), then
//   u <- u + omega (ubar - u)           (Eq. 5.33).
// N voxels per thread (relax_vec): a warp covers 32 N consecutive slots of
// one row, a block (32, 8) 8 rows; grid (row chunks x y-blocks, kt,
// ntile n4): the (k, l) planes in the tiled traversal order of Layout::kt.
// The black pass walks that order backwards, so it starts on the data the
// red pass touched last, which is still in L2.  The same kernel with BF16 weights
// sweeps the correction system of the mixed-precision solve.  kOwnW: the black
// pass reads a copy of the weights stored by black end at its own slots, as
// the red pass reads its own (the same values and bits).
template <int C, typename WT, int N, bool kUnit, bool kOwnW = false>
__global__ void __launch_bounds__(256, vec_min_blocks<N>()) k_sweep_vec(
    Layout L, FastDiv fn4, float *__restrict__ x, const float *__restrict__ B,
    const float *__restrict__ Gm, const WT *__restrict__ W, float omega)
{
    const int nch = (L.P + 32 * N - 1) / (32 * N);
    const int bx = C ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int chunk = bx % nch;
    const int jb = bx / nch;
    RowPos rp;
    rp.j = jb * 8 + threadIdx.y;
    const unsigned kin = C ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
    const unsigned c = C ? gridDim.z - 1 - blockIdx.z : blockIdx.z;   // tile n4 + l
    const unsigned tile = fdiv(c, fn4);
    rp.k = (int)(tile * (unsigned)L.kt + kin);
    rp.l = (int)(c - tile * (unsigned)L.n4);
    if (rp.j >= L.n2 || rp.k >= L.n3) return;   // the whole warp
    rp.p = (rp.j + rp.k + rp.l) & 1;
    const int s0 = chunk * 32 * N + N * threadIdx.x;
    const bool act = s0 < L.P && 2 * s0 + (C ^ rp.p) < L.n1;
    const int row = rp.j + L.n2 * (rp.k + L.n3 * rp.l);
    relax_vec<C, WT, N, kUnit, kOwnW>(L, x, B, Gm, W, omega, act, row, s0, rp);
}

template <typename WT, int N, bool kUnit>
void launch_vec(const Layout &L, int colour, float *x, const float *B, const float *Gm,
                const WT *W, float omega, cudaStream_t st, const WT *Wblack = nullptr)
{
    dim3 block(32, 8);
    dim3 grid((unsigned)(((L.P + 32 * N - 1) / (32 * N)) * L.njb), (unsigned)L.kt,
              (unsigned)(L.ntile * L.n4));
    const FastDiv fn4 = make_fastdiv((unsigned)L.n4);
    if (colour == 0)
        k_sweep_vec<0, WT, N, kUnit><<<grid, block, 0, st>>>(L, fn4, x, B, Gm, W, omega);
    else if (Wblack)
        k_sweep_vec<1, WT, N, kUnit, true><<<grid, block, 0, st>>>(L, fn4, x, B, Gm, Wblack,
                                                                   omega);
    else
        k_sweep_vec<1, WT, N, kUnit><<<grid, block, 0, st>>>(L, fn4, x, B, Gm, W, omega);
}

void launch_sweep(const Layout &L, int colour, float *x, const float *beta, const float *gamma,
                  const float *W, float omega, cudaStream_t st, const float *Wblack)
{
    if (gamma)
        launch_vec<float, kVecF32, false>(L, colour, x, beta, gamma, W, omega, st, Wblack);
    else
        launch_vec<float, kVecF32, true>(L, colour, x, beta, nullptr, W, omega, st, Wblack);
}

void launch_sweep_mixed(const Layout &L, int colour, float *delta, const float *rho,
                        const float *gb, const void *Wb, float omega, cudaStream_t st)
{
    launch_vec<__nv_bfloat16, kVecBF16, false>(L, colour, delta, rho, gb,
                                               (const __nv_bfloat16 *)Wb, omega, st);
}

// ---------------------------------------------------- symmetric scaling

// The system D u - c sum_f w_f u_nb = b, divided by c row by row, is
// M u = b / c with the symmetric M = diag(D/c) - W.  With r = sqrt(c/D) =
// sqrt(gamma) and u = r v it becomes (I - Ws) v = b / (c / r) with unit
// diagonal and Ws_f = w_f r_i r_nb(f); its Gauss-Seidel / SOR iterates are
// the original ones mapped by u = r v (row and variable scaling by positive
// diagonals).  The FP32 solve sweeps its correction system in this form, so a
// sweep reads no per-voxel c/D.
//
// Ws <- W r_i r_nb on the interior faces of every red voxel (0 on faces to the
// boundary), r = sqrt(gamma) of both ends; with Wsb, the same values also by
// black end: face f of red slot q is face f ^ 1 of its black neighbour
// (Wsb's faces to the ring stay 0 from its allocation).
__global__ void __launch_bounds__(256) k_scaled_weights(Layout L, const float *__restrict__ W,
                                                        float *__restrict__ Ws,
                                                        float *__restrict__ Wsb,
                                                        const float *__restrict__ gamma,
                                                        ItemDecode dec, unsigned items)
{
    for (unsigned t = blockIdx.x; t < items; t += gridDim.x) {
        int C, chunk;
        RowPos rp;
        decode_item(dec, L, 2u * t, (int)(threadIdx.x >> 5), C, chunk, rp);   // red tiles
        if (rp.j >= L.n2) continue;
        const int s = chunk * 32 + (int)(threadIdx.x & 31);
        if (s >= L.P || 2 * s + rp.p >= L.n1) continue;
        const int row = rp.j + L.n2 * (rp.k + L.n3 * rp.l);
        const long long q = (long long)row * L.P + s;
        const long long dy = L.P, dz = (long long)L.n2 * L.P, dt = (long long)L.n2 * L.n3 * L.P;
        const float *gb = gamma + L.S;   // black neighbours
        const int i = 2 * s + rp.p;
        const long long nb[8] = {q - 1 + rp.p, q + rp.p, q - dy, q + dy, q - dz, q + dz,
                                 q - dt, q + dt};
        const bool in[8] = {i >= 1, i + 1 < L.n1, rp.j > 0, rp.j + 1 < L.n2,
                            rp.k > 0, rp.k + 1 < L.n3, rp.l > 0, rp.l + 1 < L.n4};
        const float rs = sqrtf(gamma[q]);
#pragma unroll
        for (int f = 0; f < 8; ++f) {
            const long long o = (long long)f * L.S + q;
            const float v = in[f] ? W[o] * rs * sqrtf(gb[nb[f]]) : 0.0f;
            Ws[o] = v;
            if (Wsb && in[f]) Wsb[(long long)(f ^ 1) * L.S + nb[f]] = v;
        }
    }
}

void launch_scaled_weights(const Layout &L, const float *W, float *Ws, float *Wsb,
                           const float *gamma, cudaStream_t st)
{
    const long long red_items = item_count(L, L.nchunk) / 2;
    const int blocks = (int)(red_items < kResBlocks ? red_items : kResBlocks);
    k_scaled_weights<<<blocks, 256, 0, st>>>(L, W, Ws, Wsb, gamma,
                                             make_item_decode(L, L.nchunk), (unsigned)red_items);
}

// Deterministic final reduction of the per-block records (one block); with
// amax, also the maximum of amax[0..n) into out[3].
__global__ void __launch_bounds__(1024) k_reduce(const double *__restrict__ partials, int n,
                                                 const double *__restrict__ amax,
                                                 double *__restrict__ out)
{
    Acc3 a{0.0, DBL_MAX, -DBL_MAX};
    float m = 0.0f;
#pragma unroll 4
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
        a = acc3_merge(a, Acc3{partials[3 * b], partials[3 * b + 1], partials[3 * b + 2]});
        if (amax) m = fmaxf(m, (float)amax[b]);   // amax holds FP32 values
    }
    block_write3(a, out);
    if (amax) block_write_max(m, out + 3);
}

void launch_reduce_partials(const double *partials, int nparts, double *out, cudaStream_t st,
                            const double *amax)
{
    k_reduce<<<1, 1024, 0, st>>>(partials, nparts, amax, out);
}

// Coefficients of the step system (coef_finish, Eq. new1) from
// u = u^{resc,n-1}: w (red voxels store their 8), D, gamma = c/D, and b
// itself in beta (u, plus the Dirichlet column of ghost data when given).  Records: (sum b^2, min b, max b).  Work
// item t = 2 * tile + colour, tile = 32 slots x 8 rows at one (k, l), one
// voxel per lane (coef_gather); blocks stride over the items.
// Coefficients of the step system (coef_finish, Eq. new1) from
// u = u^{resc,n-1}: w (red voxels store their 8), D, gamma = c/D, and b
// itself in beta (u, plus the Dirichlet column of ghost data when given).
// Records: (sum b^2, min b, max b).  Work item t = 2 * tile + colour, tile =
// 32 slots x 8 rows at one (k, l), one voxel per lane (coef_gather); blocks
// stride over the items, so a tile's red and black voxels are handled one
// after the other and the black ones find the shared rows in cache.
template <bool kGhost>
__global__ void __launch_bounds__(256, 2) k_step_coef(Layout L, const float *__restrict__ u,
                                                      const float *__restrict__ G, StepConst K,
                                                      float *__restrict__ beta,
                                                      float *__restrict__ gamma,
                                                      float *__restrict__ diag,
                                                      float *__restrict__ W,
                                                      double *__restrict__ partials,
                                                      ItemDecode dec, unsigned items, Ghost gh)
{
    Rec3f a = rec3f_init();
    for (unsigned t = blockIdx.x; t < items; t += gridDim.x) {
        int C, chunk;
        RowPos rp;
        decode_item(dec, L, t, (int)(threadIdx.x >> 5), C, chunk, rp);
        if (rp.j >= L.n2) continue;   // the whole warp
        const int s = chunk * 32 + (int)(threadIdx.x & 31);
        const bool act = s < L.P && 2 * s + (C ^ rp.p) < L.n1;
        const int row = rp.j + L.n2 * (rp.k + L.n3 * rp.l);
        const long long q = (long long)row * L.P + s;
        float g[8];
        if (C)
            load_G8<1>(L, G, act, row, s, rp, g);
        else
            load_G8<0>(L, G, act, row, s, rp, g);
        float u0, sm[4], sp[4], ed[6][2][2];
        if (C)
            coef_gather<1>(L, u, act, row, s, rp, u0, sm, sp, ed);
        else
            coef_gather<0>(L, u, act, row, s, rp, u0, sm, sp, ed);
        if (!act) continue;
        const int i = 2 * s + (C ^ rp.p);
        if (kGhost) apply_ghosts(gh, L, i, rp.j, rp.k, rp.l, sm, sp, ed);
        float w[8], D, bt, gm, cc;
        coef_finish(K, g, u0, sm, sp, ed, w, D, bt, gm, cc);
        // b = u^{n-1}; with Dirichlet data, + c w_f g_f for every face to the
        // ghost ring (the ghost value's column moved to the right-hand side)
        float b = u0;
        if (kGhost) {
            const int c[4] = {i, rp.j, rp.k, rp.l};
            const int nn[4] = {L.n1, L.n2, L.n3, L.n4};
            float fold = 0.0f;
#pragma unroll
            for (int f = 0; f < 8; ++f) {
                int e[4] = {c[0], c[1], c[2], c[3]};
                e[f >> 1] += (f & 1) ? 1 : -1;
                if (e[f >> 1] < 0 || e[f >> 1] >= nn[f >> 1])
                    fold = __fmaf_rn(w[f], ghost_at(gh, gh.now, L, e[0], e[1], e[2], e[3]), fold);
            }
            b = __fmaf_rn(cc, fold, u0);
        }
        const long long qc = (long long)C * L.S + q;
        if (C == 0)
#pragma unroll
            for (int f = 0; f < 8; ++f) W[(long long)f * L.S + q] = w[f];
        diag[qc] = D;
        beta[qc] = b;
        gamma[qc] = gm;
        rec3f_add(a, __fmul_rn(b, b), b);
    }
    block_write3(rec3f_acc(a), partials + 3 * blockIdx.x);
}

int launch_step_coef(const Layout &L, const float *u, const float *G, const double *h,
                     double tau, double eps, float *beta, float *gamma, float *diag, float *W,
                     double *partials, const Ghost *ghost, cudaStream_t st)
{
    StepConst K;
    for (int d = 0; d < 4; ++d) {
        K.inv_h[d] = (float)(1.0 / h[d]);
        K.inv_h2[d] = (float)(1.0 / (h[d] * h[d]));
    }
    K.tau = (float)tau;
    K.eps2 = (float)(eps * eps);
    const long long items = item_count(L, L.nchunk);
    const int blocks = (int)(items < kResBlocks ? items : kResBlocks);
    if (ghost)
        k_step_coef<true><<<blocks, 256, 0, st>>>(L, u, G, K, beta, gamma, diag, W, partials,
                                                  make_item_decode(L, L.nchunk), (unsigned)items,
                                                  *ghost);
    else
        k_step_coef<false><<<blocks, 256, 0, st>>>(L, u, G, K, beta, gamma, diag, W, partials,
                                                   make_item_decode(L, L.nchunk),
                                                   (unsigned)items, Ghost{});
    return blocks;
}

}  // namespace seg4d_impl
