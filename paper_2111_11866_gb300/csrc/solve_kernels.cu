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

template <int C, bool kCG = false>
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
        t0 = sxm >= 0 ? W[0 * S + q] * ldu<kCG>(xo + rb + sxm) : 0.0f;
        t1 = sxp < L.P ? W[1 * S + q] * ldu<kCG>(xo + rb + sxp) : 0.0f;
        t2 = rp.j > 0 ? W[2 * S + q] * ldu<kCG>(xo + q - dy) : 0.0f;
        t3 = rp.j + 1 < L.n2 ? W[3 * S + q] * ldu<kCG>(xo + q + dy) : 0.0f;
        t4 = rp.k > 0 ? W[4 * S + q] * ldu<kCG>(xo + q - dz) : 0.0f;
        t5 = rp.k + 1 < L.n3 ? W[5 * S + q] * ldu<kCG>(xo + q + dz) : 0.0f;
        t6 = rp.l > 0 ? W[6 * S + q] * ldu<kCG>(xo + q - dt) : 0.0f;
        t7 = rp.l + 1 < L.n4 ? W[7 * S + q] * ldu<kCG>(xo + q + dt) : 0.0f;
    } else {
        const int sxm = s - rp.p, sxp = s + 1 - rp.p;
        t0 = sxm >= 0 ? W[1 * S + rb + sxm] * ldu<kCG>(xo + rb + sxm) : 0.0f;
        t1 = sxp < L.P ? W[0 * S + rb + sxp] * ldu<kCG>(xo + rb + sxp) : 0.0f;
        t2 = rp.j > 0 ? W[3 * S + q - dy] * ldu<kCG>(xo + q - dy) : 0.0f;
        t3 = rp.j + 1 < L.n2 ? W[2 * S + q + dy] * ldu<kCG>(xo + q + dy) : 0.0f;
        t4 = rp.k > 0 ? W[5 * S + q - dz] * ldu<kCG>(xo + q - dz) : 0.0f;
        t5 = rp.k + 1 < L.n3 ? W[4 * S + q + dz] * ldu<kCG>(xo + q + dz) : 0.0f;
        t6 = rp.l > 0 ? W[7 * S + q - dt] * ldu<kCG>(xo + q - dt) : 0.0f;
        t7 = rp.l + 1 < L.n4 ? W[6 * S + q + dt] * ldu<kCG>(xo + q + dt) : 0.0f;
    }
    return ((t0 + t1) + (t2 + t3)) + ((t4 + t5) + (t6 + t7));
}

// Grid-stride loop over the sweep's tiles (32 slots x 8 rows along y at one
// (k, l)); a block of 256 threads takes one tile per iteration, lane -> slot,
// warp -> row, so each iteration issues the same coalesced loads as a sweep.
#define FOR_TILES(L, s, rp, row, BODY)                                                     \
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

// ------------------------------------------ fused red-black wavefront sweep

// One launch performs `nsweeps` complete red-black sweeps in a single pass
// over memory per sweep.  The frame axis l is swept as a wavefront: work item
// (g, t), g = sweep*(n4+1) + s, updates the RED voxels of frame s and then the
// BLACK voxels of frame s-1 on tile t (kWaveTJ x kWaveTK rows at every x).
// Red of frame s reads black of frames s-1, s, s+1 before any of them is
// updated in this sweep; black of frame s-1 reads red of frames s-2, s-1, s
// after their update.  So the result is exactly that of all-red-then-all-black
// sweeps (bit for bit: the arithmetic per voxel is the same), while the data
// of a frame is read from DRAM once per sweep: the black pass of frame s-1
// re-reads what the red pass of frame s-1 touched one wavefront step earlier,
// which is still in L2.
//
// Scheduling: CTAs take items in ticket order (g-major).  Item (g, t) starts
// when its own tile and its 4 in-plane neighbour tiles have completed item
// g-1 (done[t'] >= g); that covers every read-after-write and write-after-read
// dependence above, including those between consecutive sweeps.  Waits only
// ever point at smaller tickets, which were taken by running CTAs, so the
// schedule cannot deadlock.  Every wait is bounded (kWaveTimeoutNs on the
// global timer): on expiry the CTA raises ctrl[2] (error) and ctrl[1] (abort)
// and all CTAs leave; the host reports SEG4D_ERR_TIMEOUT.
//
// ctrl layout (u32, zeroed before every launch): [0] ticket, [1] abort,
// [2] error, [3] reserved, [4 ..] done[T] per tile.
constexpr int kWaveTJ = 8;
constexpr int kWaveTK = 4;
constexpr unsigned long long kWaveTimeoutNs = 2000000000ull;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned *p)
{
    return *(const volatile unsigned *)p;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// one colour of one tile of one frame; warp -> rows, lane -> slots
template <int C>
__device__ __forceinline__ void wave_half(const Layout &L, float *__restrict__ x,
                                          const float *__restrict__ beta,
                                          const float *__restrict__ gamma,
                                          const float *__restrict__ W, float omega, int l, int j0,
                                          int k0)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float *xo = x + (C ? 0 : L.S);
    float *xs = x + (C ? L.S : 0);
    for (int r = warp; r < kWaveTJ * kWaveTK; r += (int)(blockDim.x >> 5)) {
        RowPos rp;
        rp.j = j0 + r % kWaveTJ;
        rp.k = k0 + r / kWaveTJ;
        rp.l = l;
        if (rp.j >= L.n2 || rp.k >= L.n3) continue;
        rp.p = (rp.j + rp.k + l) & 1;
        const int row = rp.j + L.n2 * (rp.k + L.n3 * l);
        const long long rb = (long long)row * L.P;
        for (int s = lane; s < L.P; s += 32) {
            if (2 * s + (C ^ rp.p) >= L.n1) continue;
            const long long q = rb + s;
            const float acc = neighbour_sum<C, true>(L, xo, W, row, s, rp);
            const float ubar = beta[C * L.S + q] + gamma[C * L.S + q] * acc;
            const float u0 = __ldcg(xs + q);
            xs[q] = u0 + omega * (ubar - u0);
        }
    }
}

__global__ void __launch_bounds__(256) k_sweep_wave(Layout L, float *__restrict__ x,
                                                    const float *__restrict__ beta,
                                                    const float *__restrict__ gamma,
                                                    const float *__restrict__ W, float omega,
                                                    int nsweeps, unsigned *__restrict__ ctrl,
                                                    int test_wait)
{
    __shared__ unsigned sh_ticket, sh_stop;
    unsigned *done = ctrl + 4;
    const int ntj = (L.n2 + kWaveTJ - 1) / kWaveTJ;
    const int ntk = (L.n3 + kWaveTK - 1) / kWaveTK;
    const unsigned T = (unsigned)(ntj * ntk);
    const unsigned steps = (unsigned)(L.n4 + 1);
    const unsigned total = (unsigned)nsweeps * steps * T;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned tk = atomicAdd(&ctrl[0], 1u);
            unsigned stop = (tk >= total) || ld_volatile_u32(&ctrl[1]) != 0u;
            if (!stop) {
                const unsigned g = tk / T, t = tk % T;
                const int tj = (int)(t % ntj), tkk = (int)(t / ntj);
                unsigned deps[5];
                int nd = 0;
                deps[nd++] = t;
                if (tj > 0) deps[nd++] = t - 1;
                if (tj + 1 < ntj) deps[nd++] = t + 1;
                if (tkk > 0) deps[nd++] = t - ntj;
                if (tkk + 1 < ntk) deps[nd++] = t + ntj;
                const unsigned long long t0 = global_ns();
                // test hook: the first item also waits for ctrl[3], which
                // nothing sets, so the bounded wait below must expire
                if (test_wait && tk == 0u) {
                    while (ld_acquire_u32(&ctrl[3]) == 0u) {
                        if (global_ns() - t0 > kWaveTimeoutNs) {
                            atomicExch(&ctrl[2], 1u);
                            atomicExch(&ctrl[1], 1u);
                            stop = 1;
                            break;
                        }
                        __nanosleep(1000);
                    }
                }
                for (int d = 0; d < nd && !stop; ++d) {
                    while (ld_acquire_u32(&done[deps[d]]) < g) {
                        if (ld_volatile_u32(&ctrl[1]) != 0u) {
                            stop = 1;
                            break;
                        }
                        if (global_ns() - t0 > kWaveTimeoutNs) {
                            atomicExch(&ctrl[2], 1u);
                            atomicExch(&ctrl[1], 1u);
                            stop = 1;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
            }
            sh_ticket = tk;
            sh_stop = stop;
        }
        __syncthreads();
        const unsigned tk = sh_ticket;
        if (sh_stop) break;
        const unsigned g = tk / T, t = tk % T;
        const int s = (int)(g % steps);
        const int j0 = (int)(t % ntj) * kWaveTJ, k0 = (int)(t / ntj) * kWaveTK;
        if (s < L.n4) wave_half<0>(L, x, beta, gamma, W, omega, s, j0, k0);
        __syncthreads();
        if (s >= 1) wave_half<1>(L, x, beta, gamma, W, omega, s - 1, j0, k0);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u32(&done[t], g + 1u);
        }
    }
}

int wave_tiles(const Layout &L)
{
    return ((L.n2 + kWaveTJ - 1) / kWaveTJ) * ((L.n3 + kWaveTK - 1) / kWaveTK);
}

int wave_max_ctas_per_sm()
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep_wave, 256, 0) != cudaSuccess)
        return 1;
    return nb < 1 ? 1 : nb;
}

void launch_sweep_wave(const Layout &L, int nsweeps, float *x, const float *beta,
                       const float *gamma, const float *W, float omega, unsigned *ctrl, int ctas,
                       int test_wait, cudaStream_t st)
{
    k_sweep_wave<<<ctas, 256, 0, st>>>(L, x, beta, gamma, W, omega, nsweeps, ctrl, test_wait);
}

// --------------------------------------------------------------- residual

// r_v = b_v - (A u)_v = D_v (ubar_v - u_v) for every voxel; per-block records
// of (sum r^2, min u, max u) in FP64.
__global__ void __launch_bounds__(kPartThreads) k_residual(Layout L, const float *__restrict__ x,
                                                           const float *__restrict__ beta,
                                                           const float *__restrict__ gamma,
                                                           const float *__restrict__ diag,
                                                           const float *__restrict__ W,
                                                           double *__restrict__ partials)
{
    Acc3 a{0.0, DBL_MAX, -DBL_MAX};
    FOR_TILES(L, s, rp, row, {
        const long long q = (long long)row * L.P + s;
#pragma unroll
        for (int C = 0; C < 2; ++C) {
            if (2 * s + (C ^ rp.p) < L.n1) {
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
    })
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
    Acc3 a{0.0, DBL_MAX, -DBL_MAX};
    FOR_TILES(L, s, rp, row, {
        const long long q = (long long)row * L.P + s;
#pragma unroll 1
        for (int C = 0; C < 2; ++C) {
            const int i = 2 * s + (C ^ rp.p);
            if (i < L.n1) {
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
    })
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
