// batch.cu -- many independent segmentation windows advanced together.
//
// A batch owns one device arena.  Each admitted window (its own 4D grid,
// image and seeds, e.g. a window around one nucleus) gets a contiguous block
// of the arena for its step arrays and a second block for its images, which
// is released once the set-up is done.  Admission fails with SEG4D_ERR_OOM
// when the arena has no room: the byte budget is the admission control.
//
// One call of seg4d_batch_advance runs the set-up of every newly admitted
// window and then one time step (coefficients, red-black SOR solve, local
// rescale -- the same scheme as the single-grid path) for every active window.
// The hot kernels are batched: one launch covers all windows.  A block finds
// its window by binary search in a short table of tile offsets, then runs
// the same per-voxel code as the single-grid kernels (stencil.cuh).
//
// Every window keeps its own stopping test (the single-grid rule: the
// residual's 2-norm and its largest entry, FP64 sums reduced per window in a
// fixed order), decided on the device, on its own schedule predicted from
// its own residuals and rounded to a fixed grid of sweeps.  A window's
// iterates therefore depend on nothing but the window itself: its result is
// the same, bit for bit, alone or in any mix of other windows.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/seg4d.h"
#include "stencil.cuh"

namespace seg4d_impl {

constexpr int kChunkTiles = 16;   // tiles per block of the reduction kernels
#ifndef SEG4D_CHECK_GRID
#define SEG4D_CHECK_GRID 4
#endif
constexpr int kCheckGrid = SEG4D_CHECK_GRID;   // batch checks fall on multiples of this

struct BWin {
    Layout L;
    FastDiv fP, fn2, fn3;          // division by P, n2, n3
    float *x;                      // array the current solve iterates on
    float *u, *beta, *gamma, *diag, *W, *G;
    int *owner;
    SeedDev *seeds;
    SeedStat *stat;
    int nseeds;
    // defect-correction solve: rho = r * ib (right-hand side of the correction
    // system), dlt (the correction), ib = 1/D (FP32) or 1/D_b (mixed), [2][S]
    float *ib, *rho, *dlt;
    int mixed;                     // precision 1: Wb and gb exist
    __nv_bfloat16 *Wb;             // bf16 [8][S] face weights by red end
    float *gb;                     // c / D_b, [2][S]
};

// A window's (row, slot) pairs of one colour are enumerated linearly,
// e = row * P + slot, and cut into tiles of 256 consecutive pairs, one tile
// per block: no lane idles on short rows (small windows have P = 12..32).
__host__ __device__ inline long long win_tiles(const Layout &L) { return (L.S + 255) / 256; }

// largest w with starts[w] <= b (starts ascending, starts[0] = 0)
__device__ inline int find_win(const long long *__restrict__ starts, int n, long long b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// tile t of window wd -> thread's (row position, slot); false past the end
__device__ inline bool tile_pos(const BWin &wd, long long t, RowPos &rp, int &s, int &row)
{
    const long long e = t * 256 + threadIdx.x;
    if (e >= wd.L.S) return false;
    const unsigned ue = (unsigned)e;
    const unsigned r = fdiv(ue, wd.fP);
    s = (int)(ue - r * (unsigned)wd.L.P);
    const unsigned a = fdiv(r, wd.fn2);
    rp.j = (int)(r - a * (unsigned)wd.L.n2);
    const unsigned c = fdiv(a, wd.fn3);
    rp.k = (int)(a - c * (unsigned)wd.L.n3);
    rp.l = (int)c;
    rp.p = (rp.j + rp.k + rp.l) & 1;
    row = (int)r;
    return true;
}

// Sweeps take N slots per thread (N = kVecF32, or kVecBF16 in mixed
// precision): the groups (row, s0), s0 a multiple of N, of one colour are
// enumerated as e = (row * P + s0) / N and cut into tiles of 256.
__host__ __device__ inline long long win_gtiles(const Layout &L, int N)
{
    return (L.S / N + 255) / 256;
}

// group tile t of window wd -> thread's (row position, s0); false past the end
template <int N>
__device__ inline bool group_pos(const BWin &wd, long long t, RowPos &rp, int &s0, int &row)
{
    const long long e = t * 256 + threadIdx.x;
    if (N * e >= wd.L.S) return false;
    const unsigned ue = (unsigned)(N * e);
    const unsigned r = fdiv(ue, wd.fP);
    s0 = (int)(ue - r * (unsigned)wd.L.P);
    const unsigned a = fdiv(r, wd.fn2);
    rp.j = (int)(r - a * (unsigned)wd.L.n2);
    const unsigned c = fdiv(a, wd.fn3);
    rp.k = (int)(a - c * (unsigned)wd.L.n3);
    rp.l = (int)c;
    rp.p = (rp.j + rp.k + rp.l) & 1;
    row = (int)r;
    return true;
}

// --------------------------------------------------------------- kernels

// per-window fixed-order reduction of the chunk records (one block per
// window) into out[4 w .. 4 w + 2]; with amax (the defect pass's per-chunk
// max |r|), also its maximum into out[4 w + 3]
__global__ void __launch_bounds__(256) k_breduce(const long long *__restrict__ cstarts,
                                                 const double *__restrict__ parts,
                                                 const double *__restrict__ amax,
                                                 double *__restrict__ out)
{
    const int w = blockIdx.x;
    Acc3 a{0.0, DBL_MAX, -DBL_MAX};
    float m = 0.0f;
    for (long long c = cstarts[w] + threadIdx.x; c < cstarts[w + 1]; c += blockDim.x) {
        a = acc3_merge(a, Acc3{parts[3 * c], parts[3 * c + 1], parts[3 * c + 2]});
        if (amax) m = fmaxf(m, (float)amax[c]);
    }
    block_write3(a, out + 4 * w);
    if (amax) block_write_max(m, out + 4 * w + 3);
}

// step coefficients (coef_finish, Eq. new1) for every window, one voxel per
// lane on the window's linear 256-slot tiles (coef_gather): w, D, gamma = c/D,
// b itself in beta, ib = 1/D; records (sum b^2, min, max)
__global__ void __launch_bounds__(256, 2) k_bcoef(const BWin *__restrict__ wins,
                                                  const long long *__restrict__ cstarts, int nwin,
                                                  StepConst K, double *__restrict__ parts)
{
    const long long b = blockIdx.x;
    const int w = find_win(cstarts, nwin, b);
    const Layout L = wins[w].L;
    const float *u = wins[w].u, *G = wins[w].G;
    float *beta = wins[w].beta, *gamma = wins[w].gamma, *diag = wins[w].diag, *W = wins[w].W;
    float *ib = wins[w].ib;
    const long long nt = win_tiles(L);
    const long long t0 = (b - cstarts[w]) * kChunkTiles;
    Rec3f a = rec3f_init();
    for (long long t = t0; t < t0 + kChunkTiles && t < nt; ++t) {
        RowPos rp{0, 0, 0, 0};
        int s = 0, row = 0;
        const bool in_win = tile_pos(wins[w], t, rp, s, row);
        const long long q = (long long)row * L.P + s;
        for (int C = 0; C < 2; ++C) {
            const bool act = in_win && 2 * s + (C ^ rp.p) < L.n1;
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
            float wf[8], D, bt, gm, cc;
            coef_finish(K, g, u0, sm, sp, ed, wf, D, bt, gm, cc);
            if (C == 0)
#pragma unroll
                for (int f = 0; f < 8; ++f) W[(long long)f * L.S + q] = wf[f];
            diag[C * L.S + q] = D;
            beta[C * L.S + q] = u0;
            gamma[C * L.S + q] = gm;
            ib[C * L.S + q] = __frcp_rn(D);
            rec3f_add(a, __fmul_rn(u0, u0), u0);
        }
    }
    block_write3(rec3f_acc(a), parts + 3 * b);
}

// presmoothing coefficients for every window's x (one implicit heat step,
// zero-Neumann): w_f = 1/h_d^2 inside the grid, 0 on boundary faces
__global__ void __launch_bounds__(256) k_bsmooth_coef(const BWin *__restrict__ wins,
                                                      const long long *__restrict__ cstarts,
                                                      int nwin, float4 inv_h2, float sigma_t,
                                                      double *__restrict__ parts)
{
    const long long b = blockIdx.x;
    const int w = find_win(cstarts, nwin, b);
    const Layout L = wins[w].L;
    const float *I = wins[w].x;
    float *beta = wins[w].beta, *gamma = wins[w].gamma, *diag = wins[w].diag, *W = wins[w].W;
    float *ib = wins[w].ib;
    const float ih2[4] = {inv_h2.x, inv_h2.y, inv_h2.z, inv_h2.w};
    const int nn[4] = {L.n1, L.n2, L.n3, L.n4};
    const long long nt = win_tiles(L);
    const long long t0 = (b - cstarts[w]) * kChunkTiles;
    Rec3f a = rec3f_init();
    for (long long t = t0; t < t0 + kChunkTiles && t < nt; ++t) {
        RowPos rp;
        int s, row;
        if (!tile_pos(wins[w], t, rp, s, row)) continue;
        const long long q = (long long)row * L.P + s;
        for (int C = 0; C < 2; ++C) {
            const int i = 2 * s + (C ^ rp.p);
            if (i >= L.n1) continue;
            const int c[4] = {i, rp.j, rp.k, rp.l};
            float wsum = 0.0f;
            for (int f = 0; f < 8; ++f) {
                const int d = f >> 1;
                const int nb = c[d] + ((f & 1) ? 1 : -1);
                const float wf = (nb >= 0 && nb < nn[d]) ? ih2[d] : 0.0f;
                wsum += wf;
                if (C == 0) W[(long long)f * L.S + q] = wf;
            }
            const float D = 1.0f + sigma_t * wsum;
            const float bv = I[C * L.S + q];
            diag[C * L.S + q] = D;
            beta[C * L.S + q] = bv;
            gamma[C * L.S + q] = sigma_t / D;
            ib[C * L.S + q] = __frcp_rn(D);
            rec3f_add(a, __fmul_rn(bv, bv), bv);
        }
    }
    block_write3(rec3f_acc(a), parts + 3 * b);
}

// ---- mixed precision (see mixed_kernels.cu for the scheme)

__global__ void __launch_bounds__(256) k_bmixed_prepare(const BWin *__restrict__ wins,
                                                        const long long *__restrict__ cstarts,
                                                        int nwin)
{
    const long long b = blockIdx.x;
    const int w = find_win(cstarts, nwin, b);
    if (!wins[w].mixed) return;
    const Layout L = wins[w].L;
    const float *W = wins[w].W, *gamma = wins[w].gamma, *diag = wins[w].diag;
    __nv_bfloat16 *Wb = wins[w].Wb;
    float *gb = wins[w].gb, *ib = wins[w].ib;
    const long long nt = win_tiles(L);
    const long long t0 = (b - cstarts[w]) * kChunkTiles;
    for (long long t = t0; t < t0 + kChunkTiles && t < nt; ++t) {
        RowPos rp;
        int s, row;
        if (!tile_pos(wins[w], t, rp, s, row)) continue;
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
    }
}

// Exact residual in flux form (flux_residual_vec) of the voxels of chunk c
// of window wd (kChunkTiles / N tiles of 256 N-slot groups), with rho =
// r * ib and delta = 0 (beta holds b itself): adds to the chunk's record a
// (sum r^2, min u, max u) and max |r| ra.
__device__ __forceinline__ void bdefect_chunk(const BWin &wd, long long c, Rec3f &a, float &ra)
{
    constexpr int N = kVecF32;
    const Layout L = wd.L;
    const float *x = wd.x, *beta = wd.beta, *gamma = wd.gamma;
    const float *diag = wd.diag, *W = wd.W, *ib = wd.ib;
    float *rho = wd.rho, *dlt = wd.dlt;
    const long long nt = win_gtiles(L, N);
    const long long t0 = c * (kChunkTiles / N);
    for (long long t = t0; t < t0 + kChunkTiles / N && t < nt; ++t) {
        RowPos rp{0, 0, 0, 0};
        int s0 = 0, row = 0;
        const bool in_win = group_pos<N>(wd, t, rp, s0, row);
        for (int C = 0; C < 2; ++C) {
            const bool act = in_win && 2 * s0 + (C ^ rp.p) < L.n1;
            const long long q = (long long)row * L.P + s0 + (C ? L.S : 0);
            float xs[N], bv[N], gm[N], dg[N], iv[N], res[N];
            ldv<N>(xs, act, x + q);
            ldv<N>(bv, act, beta + q);
            ldv<N>(gm, act, gamma + q);
            ldv<N>(dg, act, diag + q);
            ldv<N>(iv, act, ib + q);
            if (C)
                flux_residual_vec<1, N>(L, x, W, act, row, s0, rp, xs, bv, gm, dg, res);
            else
                flux_residual_vec<0, N>(L, x, W, act, row, s0, rp, xs, bv, gm, dg, res);
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
            stv<N>(dlt + q, zero);
        }
    }
}


__device__ inline double bseed_d2(const SeedDev &sd, int i, int j, int k)
{
    const double dx = __dsub_rn((double)i, sd.x);
    const double dy = __dsub_rn((double)j, sd.y);
    const double dz = __dsub_rn((double)k, sd.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// ----------------------------------------- solves with device-side checks
//
// A solve of many windows runs in rounds of kCheckGrid sweeps.  Every
// window's tests fall on multiples of kCheckGrid sweeps, so in a round each
// window still solving sweeps kCheckGrid times, and the windows whose test
// is due at the round's end are tested: u += delta, the exact defect pass,
// the per-window reduction and the decision (check_decision, the same rule
// as the single-grid solve) -- all on the device.  The decision kernel also
// builds the tables of the next round: the windows still solving (for the
// sweeps) and those due at its end (for the tests), by position in the
// solve's window array, with prefix offsets of their work units.  The host
// only enqueues rounds and reads the count of windows still solving a few
// rounds late, so a round costs no host synchronisation.  Each window's
// arithmetic and schedule depend on nothing but its own residuals.

enum { kSolveRun = 0, kSolveOk = 1, kSolveFail = 2 };

struct BSolve {
    double bnorm, bmax;   // ||b||_2 and max |b| of the window's system
    double last_rel;      // ||r||_2 / ||b||_2 at its last test
    double omega;         // its SOR relaxation (raised by sor_omega_update when adaptive)
    CheckState cs;        // residual history of its tests
    int next_check;       // sweep count of its next test (a multiple of kCheckGrid)
    int state;            // kSolveRun, kSolveOk, kSolveFail
    int iters;            // sweeps when it stopped
    int fail;             // 1: max_iters reached, 2: residual not finite
};

// Work tables of a round (device): a list of window positions and, per
// listed window, prefix offsets of its units (sweep groups, 256-slot tiles,
// reduction chunks); n = listed windows.
struct DevTabs {
    int *act_idx;          // windows still solving
    long long *act_pt;     // their sweep tiles (256 groups of N slots), prefix
    int *act_n;
    int *due_idx;          // windows due for a test at the round's end
    long long *due_t;      // their 256-slot tiles, prefix
    long long *due_c;      // their reduction chunks, prefix
    int *due_n;
    int *n_solving;        // windows still solving after the last decision
};

// Sweep of colour C over the windows still solving, grid-stride over their
// sweep tiles (the black pass walks them backwards, starting on what the red
// pass left in L2); the per-voxel work is k_bsweep's.
template <int C, bool kMixed, int N = kMixed ? kVecBF16 : kVecF32>
__global__ void __launch_bounds__(256, vec_min_blocks<N>()) k_bsweep_dev(
    const BWin *__restrict__ wins, DevTabs T, const BSolve *__restrict__ sw)
{
    const int nw = *T.act_n;
    const long long total = nw > 0 ? T.act_pt[nw] : 0;
    for (long long g = blockIdx.x; g < total; g += gridDim.x) {
        const long long b = C ? total - 1 - g : g;
        const int i = find_win(T.act_pt, nw, b);
        const BWin &wd = wins[T.act_idx[i]];
        const float omega = (float)sw[T.act_idx[i]].omega;
        const Layout L = wd.L;
        RowPos rp{0, 0, 0, 0};
        int s0 = 0, row = 0;
        bool act = group_pos<N>(wd, b - T.act_pt[i], rp, s0, row);
        act = act && 2 * s0 + (C ^ rp.p) < L.n1;
        if (kMixed)
            relax_vec<C, __nv_bfloat16, N>(L, wd.dlt, wd.rho, wd.gb, wd.Wb, omega, act, row, s0,
                                           rp);
        else
            relax_vec<C, float, N>(L, wd.dlt, wd.rho, wd.gamma, wd.W, omega, act, row, s0, rp);
    }
}

// x <- x + delta over the windows due for a test
__global__ void __launch_bounds__(256) k_bapply_dev(const BWin *__restrict__ wins, DevTabs T)
{
    const int nw = *T.due_n;
    const long long total = nw > 0 ? T.due_t[nw] : 0;
    for (long long b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = find_win(T.due_t, nw, b);
        const BWin &wd = wins[T.due_idx[i]];
        const long long e = (b - T.due_t[i]) * 256 + threadIdx.x;
        const long long S = wd.L.S;
        if (e >= S) continue;
        float *x = wd.x;
        const float *d = wd.dlt;
        x[e] += d[e];
        x[S + e] += d[S + e];
    }
}

// exact defect pass over the windows due for a test, grid-stride over their
// reduction chunks: one record (sum r^2, min u, max u) and one max |r| per
// chunk, numbered in the due table's chunk order
__global__ void __launch_bounds__(256, 2) k_bdefect_dev(const BWin *__restrict__ wins, DevTabs T,
                                                        double *__restrict__ parts,
                                                        double *__restrict__ amax)
{
    const int nw = *T.due_n;
    const long long total = nw > 0 ? T.due_c[nw] : 0;
    for (long long b = blockIdx.x; b < total; b += gridDim.x) {
        const int i = find_win(T.due_c, nw, b);
        Rec3f a = rec3f_init();
        float ra = 0.0f;
        bdefect_chunk(wins[T.due_idx[i]], b - T.due_c[i], a, ra);
        block_write3(rec3f_acc(a), parts + 3 * b);
        block_write_max(ra, amax + b);
        __syncthreads();   // the record helpers' shared memory is reused next
    }
}

// per due window (block i): fixed-order reduction of its chunk records into
// out[4 i .. 4 i + 3] = (sum r^2, min u, max u, max |r|)
__global__ void __launch_bounds__(256) k_breduce_dev(DevTabs T, const double *__restrict__ parts,
                                                     const double *__restrict__ amax,
                                                     double *__restrict__ out)
{
    const int i = blockIdx.x;
    if (i >= *T.due_n) return;
    Acc3 a{0.0, DBL_MAX, -DBL_MAX};
    float m = 0.0f;
    for (long long c = T.due_c[i] + threadIdx.x; c < T.due_c[i + 1]; c += blockDim.x) {
        a = acc3_merge(a, Acc3{parts[3 * c], parts[3 * c + 1], parts[3 * c + 2]});
        m = fmaxf(m, (float)amax[c]);
    }
    block_write3(a, out + 4 * i);
    block_write_max(m, out + 4 * i + 3);
}

struct DecideConst {
    double tol, tol_inf;
    int check_every, max_iters, mixed, K, adapt;
};

// Block-wide exclusive prefix sum (1024 threads at most); *total gets the
// block's sum.  Every thread calls it.
__device__ inline long long block_scan_excl(long long v, long long *total)
{
    __shared__ long long ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long s = lane < nw ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) ws[lane] = s;   // inclusive sums of the warps
    }
    __syncthreads();
    const long long before = (wid > 0 ? ws[wid - 1] : 0) + x - v;
    *total = ws[nw - 1];
    __syncthreads();
    return before;
}

// One block: the decisions of the windows due at sweep count `it`, then the
// tables of the next round (windows still solving; those of them whose test
// falls at it + K).  cnt: per window of the solve, its sweep tiles, 256-slot
// tiles and reduction chunks ([3][nsolve]).
__global__ void __launch_bounds__(1024) k_bdecide(BSolve *__restrict__ sw, int nsolve,
                                                  const double *__restrict__ out, int it,
                                                  DecideConst P,
                                                  const long long *__restrict__ cnt, DevTabs T)
{
    const int nd = *T.due_n;
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        BSolve &s = sw[T.due_idx[i]];
        const double rn = sqrt(out[4 * i]);
        const double rinf = out[4 * i + 3];
        s.last_rel = s.bnorm > 0.0 ? rn / s.bnorm : rn;
        if (!isfinite(rn)) {
            s.state = kSolveFail;
            s.fail = 2;
            s.iters = it;
            continue;
        }
        int n = P.check_every;
        const double prev_rn = s.cs.prev_rn;
        const int prev_it = s.cs.prev_it;
        const int dec = check_decision(s.cs, rn, s.bnorm, rinf, s.bmax, it, P.tol, P.tol_inf,
                                       P.check_every, P.mixed != 0, n);
        if (dec != kGoOn) {
            s.state = kSolveOk;
            s.iters = it;
        } else if (it >= P.max_iters) {
            s.state = kSolveFail;
            s.fail = 1;
            s.iters = it;
        } else {
            s.next_check = (it + n + P.K - 1) / P.K * P.K;
            if (P.adapt && prev_rn > 0.0 && rn < prev_rn && it - prev_it >= 4)
                s.omega = sor_omega_update(s.omega, pow(rn / prev_rn, 1.0 / (it - prev_it)));
        }
    }
    __syncthreads();
    __shared__ long long run[5];   // running (solving, due, sweep tiles, tiles, chunks)
    if (threadIdx.x < 5) run[threadIdx.x] = 0;
    __syncthreads();
    for (int base = 0; base < nsolve; base += blockDim.x) {
        const int w = base + (int)threadIdx.x;
        const bool act = w < nsolve && sw[w].state == kSolveRun;
        const bool due = act && sw[w].next_check == it + P.K;
        long long tot[5];
        const long long oa = block_scan_excl(act ? 1 : 0, &tot[0]);
        const long long od = block_scan_excl(due ? 1 : 0, &tot[1]);
        const long long op = block_scan_excl(act ? cnt[w] : 0, &tot[2]);
        const long long ot = block_scan_excl(due ? cnt[nsolve + w] : 0, &tot[3]);
        const long long oc = block_scan_excl(due ? cnt[2 * nsolve + w] : 0, &tot[4]);
        if (act) {
            T.act_idx[run[0] + oa] = w;
            T.act_pt[run[0] + oa] = run[2] + op;
        }
        if (due) {
            T.due_idx[run[1] + od] = w;
            T.due_t[run[1] + od] = run[3] + ot;
            T.due_c[run[1] + od] = run[4] + oc;
        }
        __syncthreads();
        if (threadIdx.x < 5) run[threadIdx.x] += tot[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        T.act_pt[run[0]] = run[2];
        T.due_t[run[1]] = run[3];
        T.due_c[run[1]] = run[4];
        *T.act_n = (int)run[0];
        *T.due_n = (int)run[1];
        *T.n_solving = (int)run[0];
    }
}

// per (window, seed) block: min/max of u over the ball (Eq. 841), then the
// affine map of the owned voxels (two kernels: all min/max first)
__global__ void __launch_bounds__(256) k_bball_minmax(const BWin *__restrict__ wins,
                                                      const long long *__restrict__ sstarts,
                                                      int nwin, double r2)
{
    const long long b = blockIdx.x;
    const int w = find_win(sstarts, nwin, b);
    const int m = (int)(b - sstarts[w]);
    const Layout L = wins[w].L;
    const SeedDev sd = wins[w].seeds[m];
    const float *u = wins[w].u;
    float mn = FLT_MAX, mx = -FLT_MAX;
    int cnt = 0;
    const int nx = sd.bx1 - sd.bx0 + 1, ny = sd.by1 - sd.by0 + 1, nz = sd.bz1 - sd.bz0 + 1;
    const long long nb = (nx > 0 && ny > 0 && nz > 0 && sd.frame >= 0 && sd.frame < L.n4)
                             ? (long long)nx * ny * nz
                             : 0;
    for (long long e = threadIdx.x; e < nb; e += blockDim.x) {
        const int i = sd.bx0 + (int)(e % nx);
        const int j = sd.by0 + (int)((e / nx) % ny);
        const int k = sd.bz0 + (int)(e / ((long long)nx * ny));
        if (bseed_d2(sd, i, j, k) <= r2) {
            int c;
            const long long sl = slot_of(L, i, j, k, sd.frame, c);
            const float v = u[c * L.S + sl];
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
            ++cnt;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    __shared__ float smn[8], smx[8];
    __shared__ int scnt[8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        smn[wid] = mn;
        smx[wid] = mx;
        scnt[wid] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            mn = fminf(mn, smn[q]);
            mx = fmaxf(mx, smx[q]);
            cnt += scnt[q];
        }
        wins[w].stat[m] = SeedStat{mn, mx, cnt, 0};
    }
}

__global__ void __launch_bounds__(256) k_brescale_apply(const BWin *__restrict__ wins,
                                                        const long long *__restrict__ sstarts,
                                                        int nwin, double r2)
{
    const long long b = blockIdx.x;
    const int w = find_win(sstarts, nwin, b);
    const int m = (int)(b - sstarts[w]);
    const Layout L = wins[w].L;
    const SeedDev sd = wins[w].seeds[m];
    const SeedStat ss = wins[w].stat[m];
    if (ss.count == 0) return;
    const double mu = ss.mn, span = (double)ss.mx - (double)ss.mn;
    if (!(span > 1e-30)) return;
    float *u = wins[w].u;
    const int *owner = wins[w].owner;
    const int nx = sd.bx1 - sd.bx0 + 1, ny = sd.by1 - sd.by0 + 1, nz = sd.bz1 - sd.bz0 + 1;
    const long long nb = (nx > 0 && ny > 0 && nz > 0 && sd.frame >= 0 && sd.frame < L.n4)
                             ? (long long)nx * ny * nz
                             : 0;
    for (long long e = threadIdx.x; e < nb; e += blockDim.x) {
        const int i = sd.bx0 + (int)(e % nx);
        const int j = sd.by0 + (int)((e / nx) % ny);
        const int k = sd.bz0 + (int)(e / ((long long)nx * ny));
        if (bseed_d2(sd, i, j, k) <= r2) {
            int c;
            const long long sl = slot_of(L, i, j, k, sd.frame, c);
            if (owner[c * L.S + sl] == m)
                u[c * L.S + sl] = (float)(((double)u[c * L.S + sl] - mu) / span);
        }
    }
}

}  // namespace seg4d_impl

// ==================================================================== host

using namespace seg4d_impl;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// first-fit allocator over the arena (offsets), with coalescing
struct Arena {
    char *base = nullptr;
    size_t bytes = 0;
    std::map<size_t, size_t> free_;   // offset -> size
    size_t used = 0;

    void init(char *b, size_t n)
    {
        base = b;
        bytes = n;
        free_.clear();
        free_[0] = n;
        used = 0;
    }
    bool alloc(size_t n, size_t &off)
    {
        n = align_up(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                off = it->first;
                const size_t rest = it->second - n;
                free_.erase(it);
                if (rest) free_[off + n] = rest;
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t n)
    {
        n = align_up(n);
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

enum WinState { kPending = 0, kActive = 1, kDone = 2, kFailed = 3 };

struct Window {
    int id = 0;
    seg4d_dims dims{};
    Layout L{};
    size_t off_main = 0, bytes_main = 0, off_img = 0, bytes_img = 0;
    bool has_img = false;
    BWin d{};
    float *I0 = nullptr, *ITH = nullptr, *Is0 = nullptr, *IsTH = nullptr;
    std::vector<seg4d_seed> seeds;
    int nsteps = 0, steps_done = 0;
    int state = kPending;
    long long sweeps = 0;
    int last_iters = 0;
    double last_res_rel = 0.0;
    std::string err;
};

}  // namespace

struct seg4d_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    seg4d_params p{};
    char *arena_mem = nullptr;
    Arena arena;
    int max_windows = 0;
    std::map<int, Window> wins;
    int next_id = 1;
    // device tables (capacity max_windows) and their pinned host mirrors
    // window table of the current launch set and its offset arrays; the
    // pinned host copies are not rewritten before their last upload has run
    BWin *d_wins = nullptr, *h_wins = nullptr;
    long long *d_chunk = nullptr, *h_chunk = nullptr;   // reduction chunks
    long long *d_seed = nullptr, *h_seed = nullptr;     // seed blocks
    cudaEvent_t ev_table = nullptr;
    bool table_pending = false;
    std::vector<std::pair<int, float *>> table_key;     // (window id, x) uploaded
    long long n_chunk = 0, n_seed = 0;
    double *d_out = nullptr, *h_out = nullptr;
    double *d_parts = nullptr;
    size_t parts_cap = 0;    // chunk records
    long long launches = 0;
    double sweep_ms = 0.0;
    // solves with device-side checks (batch_solve): per-window state, unit
    // counts, the round tables and their staging, the count of windows still
    // solving read back a few rounds late
    int num_sms = 0;
    BSolve *d_sw = nullptr, *h_sw = nullptr;
    long long *d_cnt = nullptr, *h_cnt = nullptr;        // [3][max_windows]
    int *d_tab_int = nullptr, *h_tab_int = nullptr;      // act_idx, due_idx, act_n, due_n, n
    long long *d_tab_ll = nullptr, *h_tab_ll = nullptr;  // act_pt, due_t, due_c
    int *h_nsolv = nullptr;
    cudaEvent_t ev_round[3] = {}, ev_s0[3] = {}, ev_s1[3] = {};
    std::string err;
};

namespace {

seg4d_status bfail(seg4d_batch *b, seg4d_status st, const std::string &m)
{
    if (b) b->err = m;
    return st;
}

#define BCK(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return bfail(b, SEG4D_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

Layout layout_of(const seg4d_dims &d)
{
    Layout L;
    L.n1 = d.n1;
    L.n2 = d.n2;
    L.n3 = d.n3;
    L.n4 = d.n4;
    L.P = ((d.n1 + 1) / 2 + 3) / 4 * 4;
    L.nchunk = (L.P + 31) / 32;
    L.njb = (d.n2 + 7) / 8;
    L.R = d.n2 * d.n3 * d.n4;
    L.S = (long long)L.R * L.P;
    L.kt = L.n3;
    L.ntile = 1;
    return L;
}

// main block: u, beta, gamma, diag (2S each), W (8S), G (16S) floats, owner
// (2S ints), seeds, seed stats, ib, rho, dlt (2S each) [+ Wb (8S bf16), gb
// (2S) in mixed precision]; image block: I0, ITH, Is0, IsTH (2S each)
size_t main_bytes(const Layout &L, int nseeds, bool mixed)
{
    const size_t S = (size_t)L.S;
    return align_up((16 * S + (size_t)g_floats(L)) * 4) + align_up(2 * S * 4) +
           align_up(sizeof(SeedDev) * std::max(nseeds, 1)) +
           align_up(sizeof(SeedStat) * std::max(nseeds, 1)) + 3 * align_up(2 * S * 4) +
           (mixed ? align_up(8 * S * 2) + align_up(2 * S * 4) : 0);
}

size_t img_bytes(const Layout &L) { return align_up(8 * (size_t)L.S * 4); }

void carve(seg4d_batch *b, Window &w)
{
    const size_t S = (size_t)w.L.S;
    char *m = b->arena.base + w.off_main;
    float *f = (float *)m;
    w.d.L = w.L;
    w.d.fP = make_fastdiv((unsigned)w.L.P);
    w.d.fn2 = make_fastdiv((unsigned)w.L.n2);
    w.d.fn3 = make_fastdiv((unsigned)w.L.n3);
    w.d.u = f;
    w.d.beta = f + 2 * S;
    w.d.gamma = f + 4 * S;
    w.d.diag = f + 6 * S;
    w.d.W = f + 8 * S;
    w.d.G = f + 16 * S;   // g_floats(L): 8 planes by red end + side table
    char *p = m + align_up((16 * S + (size_t)g_floats(w.L)) * 4);
    w.d.owner = (int *)p;
    p += align_up(2 * S * 4);
    w.d.seeds = (SeedDev *)p;
    p += align_up(sizeof(SeedDev) * std::max((int)w.seeds.size(), 1));
    w.d.stat = (SeedStat *)p;
    p += align_up(sizeof(SeedStat) * std::max((int)w.seeds.size(), 1));
    w.d.nseeds = (int)w.seeds.size();
    w.d.ib = (float *)p;
    p += align_up(2 * S * 4);
    w.d.rho = (float *)p;
    p += align_up(2 * S * 4);
    w.d.dlt = (float *)p;
    p += align_up(2 * S * 4);
    w.d.mixed = b->p.precision == 1;
    w.d.Wb = nullptr;
    w.d.gb = nullptr;
    if (w.d.mixed) {
        w.d.Wb = (__nv_bfloat16 *)p;
        p += align_up(8 * S * 2);
        w.d.gb = (float *)p;
    }
    w.d.x = w.d.u;
    float *g = (float *)(b->arena.base + w.off_img);
    w.I0 = g;
    w.ITH = g + 2 * S;
    w.Is0 = g + 4 * S;
    w.IsTH = g + 6 * S;
}

long long chunks_of(const Window &w);

// Make `ws` (in this order) the window table of the following launches:
// descriptors plus chunk, tile and seed offsets.  Nothing is copied when the
// same windows with the same solution arrays are already in place.
seg4d_status set_table(seg4d_batch *b, const std::vector<Window *> &ws)
{
    std::vector<std::pair<int, float *>> key;
    key.reserve(ws.size());
    for (Window *w : ws) key.emplace_back(w->id, w->d.x);
    if (key == b->table_key) return SEG4D_OK;
    if (b->table_pending) {
        BCK(cudaEventSynchronize(b->ev_table));
        b->table_pending = false;
    }
    long long c = 0, sd = 0;
    for (size_t i = 0; i < ws.size(); ++i) {
        b->h_wins[i] = ws[i]->d;
        b->h_chunk[i] = c;
        b->h_seed[i] = sd;
        c += chunks_of(*ws[i]);
        sd += ws[i]->d.nseeds;
    }
    const size_t n = ws.size();
    b->h_chunk[n] = c;
    b->h_seed[n] = sd;
    b->n_chunk = c;
    b->n_seed = sd;
    BCK(cudaMemcpyAsync(b->d_wins, b->h_wins, sizeof(BWin) * n, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemcpyAsync(b->d_chunk, b->h_chunk, sizeof(long long) * (n + 1), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaMemcpyAsync(b->d_seed, b->h_seed, sizeof(long long) * (n + 1), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaEventRecord(b->ev_table, b->stream));
    b->table_pending = true;
    b->table_key.swap(key);
    return SEG4D_OK;
}

long long chunks_of(const Window &w) { return (win_tiles(w.L) + kChunkTiles - 1) / kChunkTiles; }

seg4d_status ensure_parts(seg4d_batch *b, long long nchunks)
{
    if ((size_t)nchunks <= b->parts_cap) return SEG4D_OK;
    BCK(cudaStreamSynchronize(b->stream));
    cudaFree(b->d_parts);
    b->d_parts = nullptr;
    const size_t cap = (size_t)nchunks + nchunks / 4 + 1024;
    // records (3 doubles per chunk), then the defect pass's max |r| per chunk
    if (cudaMalloc(&b->d_parts, 4 * sizeof(double) * cap) != cudaSuccess) {
        cudaGetLastError();
        b->parts_cap = 0;
        return bfail(b, SEG4D_ERR_OOM, "batch: reduction records: allocation failed");
    }
    b->parts_cap = cap;
    return SEG4D_OK;
}

// Records of a chunked kernel -> per-window (sum, min, max[, max |r|]) in
// h_out[4 w ..]; with_max after the defect pass.
seg4d_status reduce_windows(seg4d_batch *b, size_t nw, bool with_max = false)
{
    k_breduce<<<(unsigned)nw, 256, 0, b->stream>>>(
        b->d_chunk, b->d_parts, with_max ? b->d_parts + 3 * b->parts_cap : nullptr, b->d_out);
    b->launches += 1;
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(b->h_out, b->d_out, 4 * sizeof(double) * nw, cudaMemcpyDeviceToHost,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return SEG4D_OK;
}

struct SolveItem {
    Window *w;
    double bnorm;
    double bmax;        // max |b|
    int iters;
    bool done;
    bool ok;
};

// Batched red-black SOR over every window of `items` (each window's d.x,
// beta = b, gamma, diag, W, ib already set up), as defect correction (see
// solve_system in api.cu), in rounds of kCheckGrid sweeps with the tests
// decided on the device (k_bdecide).  A window stops on its own residuals:
// ||b - A x|| <= tol ||b|| and, with tol_inf > 0, max |b - A x| <= tol_inf
// max |b| (or max |r| at its FP32 floor), exactly as the single-grid solve
// decides; its tests fall on multiples of kCheckGrid sweeps (max_iters is
// honoured to that grid).  Nothing a window computes depends on the other
// windows, so its result is the same alone or in any mix.
seg4d_status batch_solve(seg4d_batch *b, std::vector<SolveItem> &items, double omega, double tol,
                         int max_iters, int check_every, long long &sweeps_total,
                         bool mixed = false, double tol_inf = 0.0, bool adapt = false)
{
    const int ns = (int)items.size();
    if (ns == 0) return SEG4D_OK;
    seg4d_status st;
    std::vector<Window *> ws;
    for (auto &it : items) ws.push_back(it.w);
    if ((st = set_table(b, ws))) return st;   // d_wins holds the solve's windows
    const int N = mixed ? kVecBF16 : kVecF32;
    // per-window unit counts, initial state, and the first test table (every
    // window is tested before its first sweep)
    long long *cnt = b->h_cnt;
    for (int i = 0; i < ns; ++i) {
        cnt[i] = win_gtiles(ws[i]->L, N);
        cnt[ns + i] = win_tiles(ws[i]->L);
        cnt[2 * ns + i] = chunks_of(*ws[i]);
        b->h_sw[i] = BSolve{items[i].bnorm, items[i].bmax, 0.0, omega, CheckState{}, 0,
                            kSolveRun, 0, 0};
        b->h_tab_int[i] = i;   // due_idx
    }
    b->h_tab_int[ns] = ns;    // due_n
    long long *ht = b->h_tab_ll;   // due_t then due_c
    ht[0] = 0;
    ht[ns + 1] = 0;
    for (int i = 0; i < ns; ++i) {
        ht[i + 1] = ht[i] + cnt[ns + i];
        ht[ns + 2 + i] = ht[ns + 1 + i] + cnt[2 * ns + i];
    }
    const long long all_chunks = ht[2 * ns + 1];
    if ((st = ensure_parts(b, all_chunks))) return st;
    const int cap = b->max_windows;
    DevTabs T;
    T.act_idx = b->d_tab_int;
    T.due_idx = b->d_tab_int + cap;
    T.act_n = b->d_tab_int + 2 * cap;
    T.due_n = b->d_tab_int + 2 * cap + 1;
    T.n_solving = b->d_tab_int + 2 * cap + 2;
    T.act_pt = b->d_tab_ll;
    T.due_t = b->d_tab_ll + (cap + 1);
    T.due_c = b->d_tab_ll + 2 * (cap + 1);
    BCK(cudaMemcpyAsync(b->d_cnt, cnt, 3 * ns * sizeof(long long), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaMemcpyAsync(b->d_sw, b->h_sw, ns * sizeof(BSolve), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemcpyAsync(T.due_idx, b->h_tab_int, ns * sizeof(int), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaMemcpyAsync(T.due_n, b->h_tab_int + ns, sizeof(int), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaMemcpyAsync(T.due_t, ht, (ns + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                        b->stream));
    BCK(cudaMemcpyAsync(T.due_c, ht + ns + 1, (ns + 1) * sizeof(long long),
                        cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemsetAsync(T.act_n, 0, sizeof(int), b->stream));
    const DecideConst P{tol, tol_inf, check_every, max_iters, mixed ? 1 : 0, kCheckGrid,
                        adapt ? 1 : 0};
    double *amax = b->d_parts + 3 * b->parts_cap;
    const int sms = b->num_sms;
    const unsigned g_sweep = (unsigned)(sms * (N == 2 ? SEG4D_VEC2_MINB : SEG4D_VEC4_MINB));
    const unsigned g_apply = (unsigned)(sms * 8), g_defect = (unsigned)(sms * 2);
    // the host runs at most kLag rounds ahead of the last count it has read
    constexpr int kLag = 3;
    for (int r = 0;; ++r) {
        const int slot = r % kLag;
        if (r > 0) {
            BCK(cudaEventRecord(b->ev_s0[slot], b->stream));
            for (int s = 0; s < kCheckGrid; ++s) {
                if (mixed) {
                    k_bsweep_dev<0, true><<<g_sweep, 256, 0, b->stream>>>(b->d_wins, T, b->d_sw);
                    k_bsweep_dev<1, true><<<g_sweep, 256, 0, b->stream>>>(b->d_wins, T, b->d_sw);
                } else {
                    k_bsweep_dev<0, false><<<g_sweep, 256, 0, b->stream>>>(b->d_wins, T, b->d_sw);
                    k_bsweep_dev<1, false><<<g_sweep, 256, 0, b->stream>>>(b->d_wins, T, b->d_sw);
                }
            }
            BCK(cudaEventRecord(b->ev_s1[slot], b->stream));
            k_bapply_dev<<<g_apply, 256, 0, b->stream>>>(b->d_wins, T);
            b->launches += 2LL * kCheckGrid + 1;
        }
        k_bdefect_dev<<<g_defect, 256, 0, b->stream>>>(b->d_wins, T, b->d_parts, amax);
        k_breduce_dev<<<(unsigned)ns, 256, 0, b->stream>>>(T, b->d_parts, amax, b->d_out);
        k_bdecide<<<1, 1024, 0, b->stream>>>(b->d_sw, ns, b->d_out, r * kCheckGrid, P, b->d_cnt,
                                             T);
        b->launches += 3;
        BCK(cudaGetLastError());
        BCK(cudaMemcpyAsync(b->h_nsolv + slot, T.n_solving, sizeof(int), cudaMemcpyDeviceToHost,
                            b->stream));
        BCK(cudaEventRecord(b->ev_round[slot], b->stream));
        const int q = r - (kLag - 1);   // the oldest round in flight
        if (q >= 0) {
            const int qs = q % kLag;
            BCK(cudaEventSynchronize(b->ev_round[qs]));
            if (q > 0) {
                float ms = 0.0f;
                if (cudaEventElapsedTime(&ms, b->ev_s0[qs], b->ev_s1[qs]) == cudaSuccess)
                    b->sweep_ms += ms;
            }
            if (b->h_nsolv[qs] == 0) break;
        }
    }
    BCK(cudaMemcpyAsync(b->h_sw, b->d_sw, ns * sizeof(BSolve), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < ns; ++i) {
        const BSolve &s = b->h_sw[i];
        SolveItem &a = items[i];
        a.done = true;
        a.ok = s.state == kSolveOk;
        a.iters = s.iters;
        a.w->last_res_rel = s.last_rel;
        if (s.state == kSolveFail)
            a.w->err = s.fail == 2 ? "residual is not finite" : "solve reached max_iters";
        sweeps_total += s.iters;
    }
    return SEG4D_OK;
}

seg4d_status batch_rescale(seg4d_batch *b, const std::vector<Window *> &ws)
{
    if (ws.empty()) return SEG4D_OK;
    seg4d_status st;
    if ((st = set_table(b, ws))) return st;
    const long long nsd = b->n_seed;
    if (nsd == 0) return SEG4D_OK;
    const double r2 = b->p.r_ball * b->p.r_ball;
    // windows without seeds own no block: find_win takes the last equal offset
    k_bball_minmax<<<(unsigned)nsd, 256, 0, b->stream>>>(b->d_wins, b->d_seed, (int)ws.size(), r2);
    k_brescale_apply<<<(unsigned)nsd, 256, 0, b->stream>>>(b->d_wins, b->d_seed, (int)ws.size(),
                                                           r2);
    b->launches += 2;
    BCK(cudaGetLastError());
    return SEG4D_OK;
}

seg4d_status upload_seed_table(seg4d_batch *b, Window &w)
{
    const int n = (int)w.seeds.size();
    if (n == 0) return SEG4D_OK;
    std::vector<SeedDev> sd(n);
    const double rad = std::max(b->p.r_ball, b->p.R_init) + 1.0;
    for (int m = 0; m < n; ++m) {
        const seg4d_seed &s = w.seeds[m];
        SeedDev &d = sd[m];
        d.x = s.x;
        d.y = s.y;
        d.z = s.z;
        d.frame = s.frame;
        auto lo = [&](double c, int nmax) {
            double v = std::ceil(c - rad);
            return (int)std::max(0.0, std::min(v, (double)nmax));
        };
        auto hi = [&](double c, int nmax) {
            double v = std::floor(c + rad);
            return (int)std::min((double)(nmax - 1), std::max(v, -1.0));
        };
        d.bx0 = lo(s.x, w.dims.n1);
        d.bx1 = hi(s.x, w.dims.n1);
        d.by0 = lo(s.y, w.dims.n2);
        d.by1 = hi(s.y, w.dims.n2);
        d.bz0 = lo(s.z, w.dims.n3);
        d.bz1 = hi(s.z, w.dims.n3);
    }
    BCK(cudaMemcpyAsync(w.d.seeds, sd.data(), sizeof(SeedDev) * n, cudaMemcpyHostToDevice,
                        b->stream));
    // the host copy `sd` must outlive the copy
    BCK(cudaStreamSynchronize(b->stream));
    return SEG4D_OK;
}

// set-up of the pending windows: owners, thresholding, presmoothing (batched
// solves), face G, u0 and its rescale.  Image blocks are released at the end.
seg4d_status batch_setup(seg4d_batch *b, std::vector<Window *> &pend, long long &sweeps)
{
    seg4d_status st;
    const seg4d_params &p = b->p;
    for (Window *w : pend) {
        const Layout &L = w->L;
        const size_t S2 = 2 * (size_t)L.S;
        if ((st = upload_seed_table(b, *w))) return st;
        BCK(cudaMemsetAsync(w->d.owner, 0x7F, S2 * sizeof(int), b->stream));
        if (w->d.nseeds > 0) {
            // owner distance keys live in the (not yet used) presmoothing arrays
            unsigned long long *dkey = (unsigned long long *)w->Is0;
            BCK(cudaMemsetAsync(dkey, 0xFF, S2 * sizeof(unsigned long long), b->stream));
            launch_owner(L, w->d.seeds, w->d.nseeds, p.r_ball, dkey, w->d.owner, b->stream);
        }
        BCK(cudaMemcpyAsync(w->ITH, w->I0, S2 * sizeof(float), cudaMemcpyDeviceToDevice, b->stream));
        if (w->d.nseeds > 0) {
            launch_ball_minmax(L, w->d.seeds, w->d.nseeds, p.r_ball, w->I0, w->d.stat, b->stream);
            launch_threshold_apply(L, w->d.seeds, w->d.nseeds, p.r_ball, p.lambda_th, w->d.stat,
                                   w->d.owner, w->I0, w->ITH, b->stream);
            b->launches += 4;
        }
        BCK(cudaGetLastError());
    }
    // two batched presmoothing solves: I0 -> Is0, ITH -> IsTH
    const float4 ih2 = make_float4((float)(1.0 / (p.h[0] * p.h[0])), (float)(1.0 / (p.h[1] * p.h[1])),
                                   (float)(1.0 / (p.h[2] * p.h[2])), (float)(1.0 / (p.h[3] * p.h[3])));
    for (int img = 0; img < 2; ++img) {
        std::vector<Window *> ws;
        for (Window *w : pend) {
            float *src = img == 0 ? w->I0 : w->ITH;
            float *dst = img == 0 ? w->Is0 : w->IsTH;
            BCK(cudaMemcpyAsync(dst, src, 2 * (size_t)w->L.S * sizeof(float),
                                cudaMemcpyDeviceToDevice, b->stream));
            w->d.x = dst;
            ws.push_back(w);
        }
        if ((st = set_table(b, ws))) return st;
        const long long nch = b->n_chunk;
        if ((st = ensure_parts(b, nch))) return st;
        k_bsmooth_coef<<<(unsigned)nch, 256, 0, b->stream>>>(b->d_wins, b->d_chunk, (int)ws.size(),
                                                             ih2, (float)p.sigma_t, b->d_parts);
        b->launches += 1;
        BCK(cudaGetLastError());
        if ((st = reduce_windows(b, ws.size()))) return st;
        std::vector<SolveItem> items;
        for (size_t i = 0; i < ws.size(); ++i)
            items.push_back(SolveItem{ws[i], std::sqrt(b->h_out[4 * i]), 0.0, 0, false, false});
        if ((st = batch_solve(b, items, p.omega_smooth, p.tol_smooth, p.max_iters, p.check_every,
                              sweeps)))
            return st;
        for (auto &itm : items)
            if (!itm.ok) itm.w->state = kFailed;
    }
    for (Window *w : pend) {
        w->d.x = w->d.u;
        if (w->state == kFailed) continue;
        launch_face_G(w->L, w->Is0, w->IsTH, p.h, p.K, p.delta, p.vartheta, w->d.G, b->stream);
        BCK(cudaMemsetAsync(w->d.u, 0, 2 * (size_t)w->L.S * sizeof(float), b->stream));
        launch_init_u(w->L, w->d.seeds, w->d.nseeds, p.R_init, p.v_init, w->d.u, b->stream);
        b->launches += 2;
        BCK(cudaGetLastError());
    }
    std::vector<Window *> ok;
    for (Window *w : pend)
        if (w->state != kFailed) ok.push_back(w);
    if ((st = batch_rescale(b, ok))) return st;
    BCK(cudaStreamSynchronize(b->stream));
    for (Window *w : pend) {
        if (w->has_img) {
            b->arena.release(w->off_img, w->bytes_img);
            w->has_img = false;
        }
        if (w->state != kFailed) w->state = kActive;
    }
    return SEG4D_OK;
}

seg4d_status batch_step(seg4d_batch *b, std::vector<Window *> &act, long long &sweeps)
{
    const seg4d_params &p = b->p;
    seg4d_status st;
    for (Window *w : act) w->d.x = w->d.u;
    if ((st = set_table(b, act))) return st;
    const long long nch = b->n_chunk;
    if ((st = ensure_parts(b, nch))) return st;
    StepConst K;
    for (int d = 0; d < 4; ++d) {
        K.inv_h[d] = (float)(1.0 / p.h[d]);
        K.inv_h2[d] = (float)(1.0 / (p.h[d] * p.h[d]));
    }
    K.tau = (float)p.tau;
    K.eps2 = (float)(p.eps * p.eps);
    k_bcoef<<<(unsigned)nch, 256, 0, b->stream>>>(b->d_wins, b->d_chunk, (int)act.size(), K,
                                                  b->d_parts);
    b->launches += 1;
    BCK(cudaGetLastError());
    const bool mixed = p.precision == 1;
    if (mixed) {
        k_bmixed_prepare<<<(unsigned)nch, 256, 0, b->stream>>>(b->d_wins, b->d_chunk,
                                                               (int)act.size());
        b->launches += 1;
        BCK(cudaGetLastError());
    }
    if ((st = reduce_windows(b, act.size()))) return st;
    std::vector<SolveItem> items;
    for (size_t i = 0; i < act.size(); ++i)
        items.push_back(SolveItem{act[i], std::sqrt(b->h_out[4 * i]),
                                  std::max(std::fabs(b->h_out[4 * i + 1]),
                                           std::fabs(b->h_out[4 * i + 2])),
                                  0, false, false});
    if ((st = batch_solve(b, items, p.omega, p.tol, p.max_iters, p.check_every, sweeps, mixed,
                          p.tol_inf, p.omega_adapt != 0)))
        return st;
    std::vector<Window *> ok;
    for (auto &itm : items) {
        itm.w->last_iters = itm.iters;
        itm.w->sweeps += itm.iters;
        if (itm.ok)
            ok.push_back(itm.w);
        else
            itm.w->state = kFailed;
    }
    if ((st = batch_rescale(b, ok))) return st;
    for (Window *w : ok) {
        w->steps_done += 1;
        if (w->steps_done >= w->nsteps) w->state = kDone;
    }
    return SEG4D_OK;
}

void batch_free(seg4d_batch *b)
{
    cudaFree(b->arena_mem);
    cudaFree(b->d_wins);
    cudaFree(b->d_chunk);
    cudaFree(b->d_seed);
    cudaFree(b->d_out);
    cudaFree(b->d_parts);
    if (b->h_wins) cudaFreeHost(b->h_wins);
    if (b->h_chunk) cudaFreeHost(b->h_chunk);
    if (b->h_seed) cudaFreeHost(b->h_seed);
    if (b->ev_table) cudaEventDestroy(b->ev_table);
    if (b->h_out) cudaFreeHost(b->h_out);
    cudaFree(b->d_sw);
    cudaFree(b->d_cnt);
    cudaFree(b->d_tab_int);
    cudaFree(b->d_tab_ll);
    if (b->h_sw) cudaFreeHost(b->h_sw);
    if (b->h_cnt) cudaFreeHost(b->h_cnt);
    if (b->h_tab_int) cudaFreeHost(b->h_tab_int);
    if (b->h_tab_ll) cudaFreeHost(b->h_tab_ll);
    if (b->h_nsolv) cudaFreeHost(b->h_nsolv);
    for (int k = 0; k < 3; ++k) {
        if (b->ev_round[k]) cudaEventDestroy(b->ev_round[k]);
        if (b->ev_s0[k]) cudaEventDestroy(b->ev_s0[k]);
        if (b->ev_s1[k]) cudaEventDestroy(b->ev_s1[k]);
    }
}

}  // namespace

// ===================================================================== ABI

extern "C" {

seg4d_status seg4d_batch_create(size_t arena_bytes, int max_windows, void *cuda_stream,
                                seg4d_batch **out)
{
    handle_free_error().clear();
    if (!out || max_windows < 1 || arena_bytes < (1u << 20)) {
        handle_free_error() = "batch_create: out != NULL, max_windows >= 1, arena >= 1 MiB";
        return SEG4D_ERR_INVALID;
    }
    *out = nullptr;
    seg4d_batch *b = new (std::nothrow) seg4d_batch();
    if (!b) return SEG4D_ERR_OOM;
    cudaGetDevice(&b->device);
    b->stream = (cudaStream_t)cuda_stream;
    seg4d_default_params(&b->p);
    b->max_windows = max_windows;
    const size_t arena = align_up(arena_bytes);
    bool ok = cudaMalloc(&b->arena_mem, arena) == cudaSuccess &&
              cudaMalloc(&b->d_wins, sizeof(BWin) * max_windows) == cudaSuccess &&
              cudaMalloc(&b->d_chunk, sizeof(long long) * (max_windows + 1)) == cudaSuccess &&
              cudaMalloc(&b->d_seed, sizeof(long long) * (max_windows + 1)) == cudaSuccess &&
              cudaMalloc(&b->d_out, 4 * sizeof(double) * max_windows) == cudaSuccess &&
              cudaMallocHost(&b->h_wins, sizeof(BWin) * max_windows) == cudaSuccess &&
              cudaMallocHost(&b->h_chunk, sizeof(long long) * (max_windows + 1)) == cudaSuccess &&
              cudaMallocHost(&b->h_seed, sizeof(long long) * (max_windows + 1)) == cudaSuccess &&
              cudaEventCreate(&b->ev_table) == cudaSuccess &&
              cudaMallocHost(&b->h_out, 4 * sizeof(double) * max_windows) == cudaSuccess;
    const size_t mw = (size_t)max_windows;
    ok = ok && cudaMalloc(&b->d_sw, sizeof(BSolve) * mw) == cudaSuccess &&
         cudaMallocHost(&b->h_sw, sizeof(BSolve) * mw) == cudaSuccess &&
         cudaMalloc(&b->d_cnt, sizeof(long long) * 3 * mw) == cudaSuccess &&
         cudaMallocHost(&b->h_cnt, sizeof(long long) * 3 * mw) == cudaSuccess &&
         cudaMalloc(&b->d_tab_int, sizeof(int) * (2 * mw + 3)) == cudaSuccess &&
         cudaMallocHost(&b->h_tab_int, sizeof(int) * (mw + 1)) == cudaSuccess &&
         cudaMalloc(&b->d_tab_ll, sizeof(long long) * 3 * (mw + 1)) == cudaSuccess &&
         cudaMallocHost(&b->h_tab_ll, sizeof(long long) * 2 * (mw + 1)) == cudaSuccess &&
         cudaMallocHost(&b->h_nsolv, sizeof(int) * 3) == cudaSuccess &&
         cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) ==
             cudaSuccess;
    for (int k = 0; ok && k < 3; ++k)
        ok = cudaEventCreate(&b->ev_round[k]) == cudaSuccess &&
             cudaEventCreate(&b->ev_s0[k]) == cudaSuccess &&
             cudaEventCreate(&b->ev_s1[k]) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        delete b;
        handle_free_error() = "batch_create: device allocation failed";
        return SEG4D_ERR_OOM;
    }
    b->arena.init(b->arena_mem, arena);
    *out = b;
    return SEG4D_OK;
}

seg4d_status seg4d_batch_destroy(seg4d_batch *b)
{
    if (!b) return SEG4D_OK;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
    return SEG4D_OK;
}

seg4d_status seg4d_batch_set_params(seg4d_batch *b, const seg4d_params *p)
{
    if (!b || !p) return SEG4D_ERR_INVALID;
    // the same validation as the single-grid handle
    if ((p->precision != 0 && p->precision != 1) || !(p->omega > 0 && p->omega < 2) ||
        !(p->omega_smooth > 0 && p->omega_smooth < 2) || !(p->tol > 0) || !(p->tol_smooth > 0) ||
        p->max_iters < 1 || p->check_every < 1 || !(p->tau > 0) || !(p->eps > 0) ||
        !(p->sigma_t > 0) || !(p->r_ball > 0) || !(p->R_init > 0) || !(p->v_init > 0) ||
        !(p->tol_inf >= 0) || !std::isfinite(p->tol_inf) ||
        (p->omega_adapt != 0 && p->omega_adapt != 1))
        return bfail(b, SEG4D_ERR_INVALID, "batch_set_params: invalid parameters");
    for (int d = 0; d < 4; ++d)
        if (!(p->h[d] > 0) || !std::isfinite(p->h[d]))
            return bfail(b, SEG4D_ERR_INVALID, "batch_set_params: h must be > 0");
    if (!b->wins.empty() && p->precision != b->p.precision)
        return bfail(b, SEG4D_ERR_INVALID,
                     "batch_set_params: precision cannot change while windows are resident");
    b->p = *p;
    return SEG4D_OK;
}

seg4d_status seg4d_batch_add(seg4d_batch *b, const seg4d_dims *dims, const float *image,
                             int on_device, const seg4d_seed *seeds, int nseeds, int nsteps,
                             int *id_out)
{
    if (!b) return SEG4D_ERR_INVALID;
    if (!dims || dims->n1 < 1 || dims->n2 < 1 || dims->n3 < 1 || dims->n4 < 1 ||
        dims->n3 > 65535 || dims->n4 > 65535 || !image || nseeds < 0 || (nseeds && !seeds) ||
        nsteps < 0 || !id_out)
        return bfail(b, SEG4D_ERR_INVALID, "batch_add: invalid arguments");
    if ((int)b->wins.size() >= b->max_windows)
        return bfail(b, SEG4D_ERR_OOM, "batch_add: window table full");
    for (int m = 0; m < nseeds; ++m)
        if (!std::isfinite(seeds[m].x) || !std::isfinite(seeds[m].y) || !std::isfinite(seeds[m].z))
            return bfail(b, SEG4D_ERR_INVALID, "batch_add: seed coordinates must be finite");
    Window w;
    w.id = b->next_id;
    w.dims = *dims;
    w.L = layout_of(*dims);
    w.seeds.assign(seeds, seeds + nseeds);
    w.nsteps = nsteps;
    w.bytes_main = main_bytes(w.L, nseeds, b->p.precision == 1);
    w.bytes_img = img_bytes(w.L);
    if (!b->arena.alloc(w.bytes_main, w.off_main))
        return bfail(b, SEG4D_ERR_OOM, "batch_add: no room in the arena (admission refused)");
    if (!b->arena.alloc(w.bytes_img, w.off_img)) {
        b->arena.release(w.off_main, w.bytes_main);
        return bfail(b, SEG4D_ERR_OOM, "batch_add: no room in the arena (admission refused)");
    }
    // both blocks go back to the arena on every error path below, until the
    // window is in the table
    struct BlockGuard {
        Arena &a;
        size_t o1, n1, o2, n2;
        bool armed = true;
        ~BlockGuard()
        {
            if (armed) {
                a.release(o1, n1);
                a.release(o2, n2);
            }
        }
    } guard{b->arena, w.off_main, w.bytes_main, w.off_img, w.bytes_img};
    w.has_img = true;
    carve(b, w);
    // zero the main block (padding slots must read as zero)
    BCK(cudaMemsetAsync(b->arena.base + w.off_main, 0, w.bytes_main, b->stream));
    BCK(cudaMemsetAsync(b->arena.base + w.off_img, 0, w.bytes_img, b->stream));
    const size_t n = (size_t)dims->n1 * dims->n2 * dims->n3 * dims->n4;
    const float *nat = image;
    if (!on_device) {
        // stage the natural-layout image in the (still unused) ITH..IsTH area
        BCK(cudaMemcpyAsync(w.Is0, image, n * sizeof(float), cudaMemcpyHostToDevice, b->stream));
        nat = w.Is0;
    }
    launch_split_from_natural(w.L, nat, w.I0, nullptr, b->stream);
    b->launches += 1;
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(b->stream));
    b->next_id += 1;
    *id_out = w.id;
    b->wins[w.id] = w;
    guard.armed = false;
    return SEG4D_OK;
}

seg4d_status seg4d_batch_advance(seg4d_batch *b, seg4d_batch_info *info)
{
    if (!b) return SEG4D_ERR_INVALID;
    if (info) std::memset(info, 0, sizeof(*info));
    b->launches = 0;
    b->sweep_ms = 0.0;
    long long sweeps = 0;
    seg4d_status st;
    cudaEvent_t c0, c1;
    cudaEventCreate(&c0);
    cudaEventCreate(&c1);
    cudaEventRecord(c0, b->stream);
    std::vector<Window *> pend, act;
    for (auto &kv : b->wins) {
        if (kv.second.state == kPending) pend.push_back(&kv.second);
    }
    if (!pend.empty() && (st = batch_setup(b, pend, sweeps))) goto out;
    for (auto &kv : b->wins)
        if (kv.second.state == kActive && kv.second.steps_done < kv.second.nsteps)
            act.push_back(&kv.second);
    for (auto &kv : b->wins)
        if (kv.second.state == kActive && kv.second.steps_done >= kv.second.nsteps)
            kv.second.state = kDone;
    if (!act.empty() && (st = batch_step(b, act, sweeps))) goto out;
    st = SEG4D_OK;
out:
    cudaEventRecord(c1, b->stream);
    float ms = 0.0f;
    if (cudaEventSynchronize(c1) == cudaSuccess) cudaEventElapsedTime(&ms, c0, c1);
    cudaEventDestroy(c0);
    cudaEventDestroy(c1);
    if (info) {
        info->setup_windows = (int)pend.size();
        info->stepped_windows = (int)act.size();
        info->window_sweeps = sweeps;
        info->ms = ms;
        info->sweep_ms = b->sweep_ms;
        info->launches = b->launches;
        int a = 0, d = 0, f = 0;
        for (auto &kv : b->wins) {
            a += kv.second.state == kActive || kv.second.state == kPending;
            d += kv.second.state == kDone;
            f += kv.second.state == kFailed;
        }
        info->active_windows = a;
        info->done_windows = d;
        info->failed_windows = f;
        info->arena_used = b->arena.used;
        info->status = st;
    }
    return st;
}

seg4d_status seg4d_batch_poll(seg4d_batch *b, int id, seg4d_window_info *wi)
{
    if (!b || !wi) return SEG4D_ERR_INVALID;
    auto it = b->wins.find(id);
    if (it == b->wins.end()) return bfail(b, SEG4D_ERR_INVALID, "batch_poll: unknown window");
    const Window &w = it->second;
    std::memset(wi, 0, sizeof(*wi));
    wi->state = w.state;
    wi->steps_done = w.steps_done;
    wi->nsteps = w.nsteps;
    wi->sweeps = w.sweeps;
    wi->last_iters = w.last_iters;
    wi->last_res_rel = w.last_res_rel;
    wi->device_bytes = (long long)(w.bytes_main + (w.has_img ? w.bytes_img : 0));
    return SEG4D_OK;
}

seg4d_status seg4d_batch_read_u(seg4d_batch *b, int id, float *dst, size_t n, int on_device)
{
    if (!b || !dst) return SEG4D_ERR_INVALID;
    auto it = b->wins.find(id);
    if (it == b->wins.end()) return bfail(b, SEG4D_ERR_INVALID, "batch_read_u: unknown window");
    Window &w = it->second;
    const size_t nv = (size_t)w.dims.n1 * w.dims.n2 * w.dims.n3 * w.dims.n4;
    if (n != nv) return bfail(b, SEG4D_ERR_INVALID, "batch_read_u: size mismatch");
    if (w.state == kPending) return bfail(b, SEG4D_ERR_STATE, "batch_read_u: set-up not run yet");
    if (on_device) {
        launch_natural_from_split(w.L, w.d.u, dst, b->stream);
        BCK(cudaGetLastError());
        BCK(cudaStreamSynchronize(b->stream));
        return SEG4D_OK;
    }
    // stage through the diag array (free between steps)
    launch_natural_from_split(w.L, w.d.u, w.d.diag, b->stream);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(dst, w.d.diag, n * sizeof(float), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return SEG4D_OK;
}

seg4d_status seg4d_batch_remove(seg4d_batch *b, int id)
{
    if (!b) return SEG4D_ERR_INVALID;
    auto it = b->wins.find(id);
    if (it == b->wins.end()) return bfail(b, SEG4D_ERR_INVALID, "batch_remove: unknown window");
    BCK(cudaStreamSynchronize(b->stream));
    Window &w = it->second;
    b->arena.release(w.off_main, w.bytes_main);
    if (w.has_img) b->arena.release(w.off_img, w.bytes_img);
    b->wins.erase(it);
    return SEG4D_OK;
}

size_t seg4d_batch_window_bytes(const seg4d_dims *dims, int nseeds, int precision)
{
    if (!dims || dims->n1 < 1 || dims->n2 < 1 || dims->n3 < 1 || dims->n4 < 1) return 0;
    const Layout L = layout_of(*dims);
    return main_bytes(L, nseeds, precision == 1) + img_bytes(L);
}

const char *seg4d_batch_last_error(const seg4d_batch *b)
{
    if (!b) return handle_free_error().c_str();
    return b->err.c_str();
}

}  // extern "C"
