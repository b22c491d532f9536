// api.cu -- host side of the C ABI declared in include/seg4d.h.
//
// The handle owns every device buffer (colour-split layout, see
// seg4d_internal.cuh).  All work goes to the handle's stream; the host waits
// on that stream only where it needs a device value (the stopping test of
// each solve, and the end of every call).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/seg4d.h"
#include "seg4d_internal.cuh"

using namespace seg4d_impl;

namespace seg4d_impl {
// message of the last failed handle-free call of this thread (seg4d_create,
// seg4d_residual_norms_noalloc), reported by seg4d_last_error(NULL)
std::string &handle_free_error()
{
    thread_local std::string s;
    return s;
}
}  // namespace seg4d_impl

#define g_create_error handle_free_error()

struct seg4d {
    seg4d_dims dims{};
    Layout L{};
    int device = 0;
    cudaStream_t stream = nullptr;
    seg4d_params p{};
    // colour-split device arrays ([2][S] unless noted)
    float *u = nullptr, *beta = nullptr, *gamma = nullptr, *diag = nullptr;
    float *W = nullptr;            // [8][S] face weights by red end
    float *G = nullptr;            // face edge coefficients: [8][S] by red end + side table
    float *I0 = nullptr, *ITH = nullptr, *Is0 = nullptr, *IsTH = nullptr;
    int *owner = nullptr;
    float *stage = nullptr;        // natural-layout staging, n1*n2*n3*n4 floats
    double *partials = nullptr;    // 3 * kPartCap doubles (scratch)
    double *scal = nullptr;        // 8 doubles: reduced records
    double *host_scal = nullptr;   // pinned mirror of scal
    unsigned *host_flag = nullptr; // pinned: non-finite flag of the last checked input
    unsigned *d_check = nullptr;   // device flag: a checked input held a non-finite value
    // defect-correction solve (allocated at the first solve that needs them)
    void *Wb = nullptr;            // mixed: bf16 [8][S] face weights by red end
    float *gb = nullptr;           // mixed: c / D_b, [2][S]
    float *ib = nullptr;           // 1 / D_b (mixed) or 1 / (D r) (FP32), [2][S]
    float *rho = nullptr, *dlt = nullptr; // right-hand side and correction of the correction system
    // FP32 solves (allocated at the first one): scaled weights, r = sqrt(gamma)
    float *Ws = nullptr;           // [8][S] by red end
    float *Wsb = nullptr;          // [8][S] the same by black end (sweep_variant 1)
    float *rs = nullptr;           // [2][S]
    // Dirichlet data on the ghost ring (seg4d_set_dirichlet); zero when unset
    float *gh_prev = nullptr, *gh_now = nullptr;
    bool has_ghost = false;
    Ghost ghost{};
    int num_sms = 0;
    SeedDev *seeds_d = nullptr;
    SeedStat *stat_d = nullptr;
    int nseeds = 0;
    int seeds_cap = 0;
    std::vector<seg4d_seed> seeds;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;    // whole call
    cudaEvent_t evs0 = nullptr, evs1 = nullptr;  // one batch of sweeps
    long long launches = 0;                      // kernels launched by the current call
    long long sweep_launches = 0;                // of which sweep kernels
    double sweep_ms = 0.0;                       // sweep time of the current call
    bool has_image = false;
    bool setup_dirty = true;
    bool need_u0 = false;
    bool has_u = false;
    bool has_coef = false;
    bool lean = false;      // SEG4D_CREATE_LEAN: 80 B/voxel, images not kept
    bool img_live = false;  // lean: the image planes inside G still hold the image
    std::string err;
};

namespace {

seg4d_status fail(seg4d *h, seg4d_status st, const std::string &msg)
{
    if (h) h->err = msg;
    return st;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, SEG4D_ERR_CUDA, std::string(#call " failed: ") +               \
                                               cudaGetErrorString(e_));                   \
    } while (0)

#define CK_LAUNCH(what)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            return fail(h, SEG4D_ERR_CUDA, std::string(what " launch failed: ") +         \
                                               cudaGetErrorString(e_));                   \
    } while (0)

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }
bool in01(double v) { return std::isfinite(v) && v >= 0.0 && v <= 1.0; }

Layout make_layout(const seg4d_dims &d)
{
    Layout L;
    L.n1 = d.n1;
    L.n2 = d.n2;
    L.n3 = d.n3;
    L.n4 = d.n4;
    const int half = (d.n1 + 1) / 2;
    L.P = (half + 3) / 4 * 4;
    L.nchunk = (L.P + 31) / 32;
    L.njb = (d.n2 + 7) / 8;
    L.R = d.n2 * d.n3 * d.n4;
    L.S = (long long)L.R * L.P;
    L.kt = plane_tile(d.n2, d.n3, d.n4, L.P);
    L.ntile = (d.n3 + L.kt - 1) / L.kt;
    return L;
}

bool dims_ok(const seg4d_dims *d)
{
    if (!d || d->n1 < 1 || d->n2 < 1 || d->n3 < 1 || d->n4 < 1) return false;
    if (d->n3 > 65535 || d->n4 > 65535) return false;   // grid.y / grid.z of the sweep
    const long long rows = (long long)d->n2 * d->n3 * d->n4;
    if (rows >= (1LL << 31)) return false;
    // work items of the tile loops (2 colours x 32-slot chunks x 8-row blocks
    // x the planes of the traversal order, holes of the last z-tile included)
    const int P = ((d->n1 + 1) / 2 + 3) / 4 * 4;
    const long long chunks = P / 32 + 1;
    const int kt = plane_tile(d->n2, d->n3, d->n4, P);
    const long long planes = (long long)((d->n3 + kt - 1) / kt) * kt * d->n4;
    if ((d->n3 + kt - 1) / kt * (long long)d->n4 > 65535) return false;
    if (2 * chunks * ((d->n2 + 7) / 8) * planes >= (1LL << 31)) return false;
    const long long nv = rows * d->n1;
    return nv < (1LL << 33);
}

size_t bytes_for(const Layout &L, long long nv, bool lean = false)
{
    if (lean) {
        // u, beta, gamma, diag, W, G, owner, ib, rho, dlt (see seg4d_create_ex)
        const size_t S = (size_t)L.S;
        return 2 * S * 4 * 4 + 8 * S * 4 + (size_t)g_floats(L) * 4 + 2 * S * 4 + 3 * 2 * S * 4 +
               4 * kPartCap * sizeof(double) + 8 * sizeof(double);
    }
    const size_t S = (size_t)L.S;
    size_t b = 0;
    b += 2 * S * sizeof(float) * 4;        // u, beta, gamma, diag
    b += 8 * S * sizeof(float);            // W
    b += (size_t)g_floats(L) * sizeof(float);   // G, once per face
    b += 2 * S * sizeof(float) * 4;        // I0, ITH, Is0, IsTH
    b += 2 * S * sizeof(int);              // owner
    b += (size_t)nv * sizeof(float);       // staging
    b += 4 * kPartCap * sizeof(double) + 8 * sizeof(double);
    // FP32 solve: Ws and its copy by black end, rs, ib, rho, dlt
    b += 2 * 8 * S * sizeof(float) + 2 * S * sizeof(float) * 4;
    return b;
}

long long nvox(const seg4d *h)
{
    return (long long)h->dims.n1 * h->dims.n2 * h->dims.n3 * h->dims.n4;
}

void free_all(seg4d *h)
{
    cudaFree(h->u);
    cudaFree(h->beta);
    cudaFree(h->gamma);
    cudaFree(h->diag);
    cudaFree(h->W);
    cudaFree(h->G);
    if (!h->lean) {
        cudaFree(h->I0);
        cudaFree(h->ITH);
        cudaFree(h->Is0);
        cudaFree(h->IsTH);
    }
    cudaFree(h->owner);
    if (!h->lean) cudaFree(h->stage);
    cudaFree(h->partials);
    cudaFree(h->scal);
    cudaFree(h->d_check);
    if (h->host_flag) cudaFreeHost(h->host_flag);
    cudaFree(h->Wb);
    cudaFree(h->gb);
    cudaFree(h->ib);
    cudaFree(h->rho);
    cudaFree(h->dlt);
    cudaFree(h->Ws);
    cudaFree(h->Wsb);
    cudaFree(h->rs);
    cudaFree(h->gh_prev);
    cudaFree(h->gh_now);
    cudaFree(h->seeds_d);
    cudaFree(h->stat_d);
    if (h->host_scal) cudaFreeHost(h->host_scal);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->evs0) cudaEventDestroy(h->evs0);
    if (h->evs1) cudaEventDestroy(h->evs1);
}

seg4d_status use_device(seg4d *h)
{
    int cur = -1;
    CK(cudaGetDevice(&cur));
    if (cur != h->device) CK(cudaSetDevice(h->device));
    return SEG4D_OK;
}

// reduce the per-block records into scal[slot..slot+2]; with_max: also the
// defect pass's per-block max |r| into scal[slot+3]
seg4d_status reduce_into(seg4d *h, int slot, int nrec = kPartBlocks, bool with_max = false)
{
    launch_reduce_partials(h->partials, nrec, h->scal + slot, h->stream,
                           with_max ? h->partials + 3 * kPartCap : nullptr);
    h->launches += 1;
    CK_LAUNCH("reduce");
    return SEG4D_OK;
}

seg4d_status fetch_scal(seg4d *h)
{
    CK(cudaMemcpyAsync(h->host_scal, h->scal, 8 * sizeof(double), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SEG4D_OK;
}

struct SolveOut {
    int iters = 0;
    double res = 0, bnorm = 0, umin = 0, umax = 0;
    double res_inf = 0, bmax = 0;   // max |r| and max |b|
    bool converged = false;
};

// Arrays of the defect-correction solve: rho (scaled right-hand side of the
// correction system), dlt (the correction), ib; then Ws and rs (FP32: scaled
// weights, r = sqrt(gamma)) or Wb and gb (mixed: BF16 weights, c / D_b).
// Allocated at the first solve that needs them; the correction's padding
// slots must read as zero.
seg4d_status ensure_solve_arrays(seg4d *h, bool mixed)
{
    const size_t S2 = 2 * (size_t)h->L.S;
    auto alloc = [&](void **p, size_t bytes) {
        if (*p) return true;
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        return cudaMemsetAsync(*p, 0, bytes, h->stream) == cudaSuccess;
    };
    bool ok = alloc((void **)&h->rho, S2 * sizeof(float)) &&
              alloc((void **)&h->dlt, S2 * sizeof(float)) &&
              alloc((void **)&h->ib, S2 * sizeof(float));
    if (ok && mixed)
        ok = alloc(&h->Wb, 4 * S2 * sizeof(unsigned short)) &&
             alloc((void **)&h->gb, S2 * sizeof(float));
    if (ok && !mixed && !h->lean)
        ok = alloc((void **)&h->Ws, 4 * S2 * sizeof(float)) &&
             alloc((void **)&h->rs, S2 * sizeof(float)) &&
             (h->p.sweep_variant != 1 || alloc((void **)&h->Wsb, 4 * S2 * sizeof(float)));
    if (!ok) return fail(h, SEG4D_ERR_OOM, "solve arrays: device allocation failed");
    return SEG4D_OK;
}

// Red-black SOR for the system in beta (= b) / gamma / diag / W, as
// defect correction: every check is an exact residual pass in flux form
// (k_defect: r = b - A u from differences of the stored u, accurate far below
// the FP32 noise of D (ubar - u)), the sweeps solve the correction system for
// delta from 0, and u += delta follows each batch.  FP32 (precision 0): the
// correction system is A itself, swept in its symmetrically scaled form
// (Ws, r; see k_scaled_weights), u += r delta.  Mixed (precision 1): BF16
// weights with the consistent diagonal D_b, u += delta.  The brec per-block
// records of ||b||^2 must be in `partials` (written by the coefficient
// kernel).  Stopping rule: ||b - A u||_2 <= tol ||b||_2 and, with tol_inf >
// 0, also max |b - A u| <= tol_inf max |b| -- a per-voxel bound, since the
// M-matrix of the Theorem in Section 3.3 has ||A^-1||_inf <= 1, so each
// voxel of the solve is within max |r| of the exact solution.  Tested before
// the first sweep and then at the spacing check_decision picks (which also
// ends a solve whose max |r| has reached its FP32 floor).
seg4d_status solve_system(seg4d *h, float *x, int brec, double omega, double tol, int max_iters,
                          int check_every, SolveOut &out, bool mixed = false,
                          double tol_inf = 0.0, double *omega_adapt = nullptr)
{
    if (omega_adapt) omega = *omega_adapt;
    const Layout &L = h->L;
    seg4d_status st = reduce_into(h, 0, brec);   // scal[0..2] = sum b^2, min b, max b
    if (st) return st;
    if ((st = ensure_solve_arrays(h, mixed))) return st;
    if (mixed) {
        launch_mixed_prepare(L, h->W, h->gamma, h->diag, h->Wb, h->gb, h->ib, h->stream);
        h->launches += 1;
    } else if (h->lean) {   // unscaled correction sweeps: ib = 1/D, no Ws / r
        launch_plain_prepare(L, h->gamma, h->diag, nullptr, h->ib, h->stream);
        h->launches += 1;
    } else {
        launch_plain_prepare(L, h->gamma, h->diag, h->rs, h->ib, h->stream);
        launch_scaled_weights(L, h->W, h->Ws, h->p.sweep_variant == 1 ? h->Wsb : nullptr,
                              h->gamma, h->stream);
        h->launches += 2;
    }
    CK_LAUNCH("solve_prepare");
    int it = 0;
    bool timed_batch = false;
    int batch = check_every;
    CheckState cs;
    for (;;) {
        const int nrec = launch_defect(L, x, h->beta, h->gamma, h->diag, h->W, h->ib, h->rho,
                                       h->dlt, h->partials, h->partials + 3 * kPartCap,
                                       h->stream);
        h->launches += 1;
        CK_LAUNCH("defect");
        // scal[3..6] = sum r^2, min u, max u, max |r|
        if ((st = reduce_into(h, 3, nrec, true))) return st;
        if ((st = fetch_scal(h))) return st;
        if (timed_batch) {   // the batch before this check has completed
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, h->evs0, h->evs1) == cudaSuccess) h->sweep_ms += ms;
            timed_batch = false;
        }
        const double bn = std::sqrt(h->host_scal[0]);
        const double rn = std::sqrt(h->host_scal[3]);
        out.iters = it;
        out.res = rn;
        out.bnorm = bn;
        out.umin = h->host_scal[4];
        out.umax = h->host_scal[5];
        out.res_inf = h->host_scal[6];
        out.bmax = std::max(std::fabs(h->host_scal[1]), std::fabs(h->host_scal[2]));
        if (!std::isfinite(rn))
            return fail(h, SEG4D_ERR_NOT_CONVERGED, "residual is not finite");
        const double prev_rn = cs.prev_rn;
        const int prev_it = cs.prev_it;
        if (check_decision(cs, rn, bn, out.res_inf, out.bmax, it, tol, tol_inf, check_every,
                           mixed, batch) != kGoOn) {
            if (omega_adapt) *omega_adapt = omega;
            out.converged = true;
            return SEG4D_OK;
        }
        if (it >= max_iters) {   // not converged; caller reports it
            if (omega_adapt) *omega_adapt = omega;
            return SEG4D_OK;
        }
        // relaxation from the contraction of the last batch (sor_omega_update)
        if (omega_adapt && prev_rn > 0.0 && rn < prev_rn && it - prev_it >= 4)
            omega = sor_omega_update(omega, std::pow(rn / prev_rn, 1.0 / (it - prev_it)));
        const int n = std::min(batch, max_iters - it);
        CK(cudaEventRecord(h->evs0, h->stream));
        if (mixed) {
            for (int s = 0; s < n; ++s) {
                launch_sweep_mixed(L, 0, h->dlt, h->rho, h->gb, h->Wb, (float)omega, h->stream);
                launch_sweep_mixed(L, 1, h->dlt, h->rho, h->gb, h->Wb, (float)omega, h->stream);
            }
            h->launches += 2LL * n;
            h->sweep_launches += 2LL * n;
        } else {
            const float *gam = h->lean ? h->gamma : nullptr;
            const float *wts = h->lean ? h->W : h->Ws;
            // the black pass reads the copy by black end at its own slots
            const float *wblk = !h->lean && h->p.sweep_variant == 1 ? h->Wsb : nullptr;
            for (int s = 0; s < n; ++s) {
                launch_sweep(L, 0, h->dlt, h->rho, gam, wts, (float)omega, h->stream);
                launch_sweep(L, 1, h->dlt, h->rho, gam, wts, (float)omega, h->stream, wblk);
            }
            h->launches += 2LL * n;
            h->sweep_launches += 2LL * n;
        }
        CK_LAUNCH("sweep");
        CK(cudaEventRecord(h->evs1, h->stream));
        if (mixed || h->lean)
            launch_apply(L, x, h->dlt, h->stream);
        else
            launch_apply_scaled(L, x, h->dlt, h->rs, h->stream);
        h->launches += 1;
        CK_LAUNCH("apply");
        timed_batch = true;
        it += n;
    }
}

seg4d_status upload_seeds(seg4d *h)
{
    const int n = (int)h->seeds.size();
    if (n > h->seeds_cap) {
        cudaFree(h->seeds_d);
        cudaFree(h->stat_d);
        h->seeds_d = nullptr;
        h->stat_d = nullptr;
        h->seeds_cap = 0;
        if (cudaMalloc(&h->seeds_d, sizeof(SeedDev) * n) != cudaSuccess ||
            cudaMalloc(&h->stat_d, sizeof(SeedStat) * n) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, SEG4D_ERR_OOM, "seed arrays: device allocation failed");
        }
        h->seeds_cap = n;
    }
    std::vector<SeedDev> sd(n);
    const double rad = std::max(h->p.r_ball, h->p.R_init) + 1.0;
    for (int m = 0; m < n; ++m) {
        const seg4d_seed &s = h->seeds[m];
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
        d.bx0 = lo(s.x, h->dims.n1);
        d.bx1 = hi(s.x, h->dims.n1);
        d.by0 = lo(s.y, h->dims.n2);
        d.by1 = hi(s.y, h->dims.n2);
        d.bz0 = lo(s.z, h->dims.n3);
        d.bz1 = hi(s.z, h->dims.n3);
    }
    h->nseeds = n;
    if (n > 0) {
        CK(cudaMemcpyAsync(h->seeds_d, sd.data(), sizeof(SeedDev) * n, cudaMemcpyHostToDevice,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));
    }
    return SEG4D_OK;
}

// presmoothing of `src` into `dst` (one implicit heat step, Section 3.1)
seg4d_status presmooth(seg4d *h, const float *src, float *dst, long long &sweeps)
{
    const Layout &L = h->L;
    launch_smooth_coef(L, src, h->p.h, h->p.sigma_t, h->beta, h->gamma, h->diag, h->W,
                       h->partials, kPartBlocks, h->stream);
    h->launches += 1;
    CK_LAUNCH("smooth_coef");
    CK(cudaMemcpyAsync(dst, src, 2 * L.S * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    SolveOut so;
    seg4d_status st = solve_system(h, dst, kPartBlocks, h->p.omega_smooth, h->p.tol_smooth,
                                   h->p.max_iters, h->p.check_every, so);
    if (st) return st;
    sweeps += so.iters;
    if (!so.converged)
        return fail(h, SEG4D_ERR_NOT_CONVERGED, "presmoothing solve reached max_iters");
    return SEG4D_OK;
}

seg4d_status rescale(seg4d *h)
{
    if (h->nseeds == 0) return SEG4D_OK;
    launch_ball_minmax(h->L, h->seeds_d, h->nseeds, h->p.r_ball, h->u, h->stat_d, h->stream);
    launch_rescale_apply(h->L, h->seeds_d, h->nseeds, h->p.r_ball, h->stat_d, h->owner, h->u,
                         h->stream);
    h->launches += 2;
    CK_LAUNCH("rescale");
    return SEG4D_OK;
}

seg4d_status run_setup(seg4d *h, long long &sweeps)
{
    if (!h->has_image) return fail(h, SEG4D_ERR_STATE, "no image set");
    const Layout &L = h->L;
    seg4d_status st;
    if (h->setup_dirty) {
        if (h->lean && !h->img_live)
            return fail(h, SEG4D_ERR_STATE,
                        "a lean handle keeps no image after its set-up: call set_image again");
        if ((st = upload_seeds(h))) return st;
        // Where the image fields live.  A lean handle keeps them inside G (not
        // computed yet; at least 4 planes of 2S floats): I0 in plane 0, I^TH in plane 2,
        // I_sigma^TH in plane 3, I_sigma^0 in u (set from the seeds at the
        // end); the owner keys borrow W.
        const size_t plane = 2 * (size_t)L.S;
        float *I0 = h->I0;
        float *ITH = h->lean ? h->G + 2 * plane : h->ITH;
        float *Is0 = h->lean ? h->u : h->Is0;
        float *IsTH = h->lean ? h->G + 3 * plane : h->IsTH;
        // owners of the thresholding / rescaling balls
        CK(cudaMemsetAsync(h->owner, 0x7F, 2 * L.S * sizeof(int), h->stream));
        if (h->nseeds > 0) {
            unsigned long long *dkey = nullptr;
            if (h->lean) {
                dkey = (unsigned long long *)h->W;   // 8S floats hold 2S keys
            } else if (cudaMallocAsync((void **)&dkey, 2 * L.S * sizeof(unsigned long long),
                                       h->stream) != cudaSuccess) {
                cudaGetLastError();
                return fail(h, SEG4D_ERR_OOM, "owner distance buffer: allocation failed");
            }
            CK(cudaMemsetAsync(dkey, 0xFF, 2 * L.S * sizeof(unsigned long long), h->stream));
            launch_owner(L, h->seeds_d, h->nseeds, h->p.r_ball, dkey, h->owner, h->stream);
            h->launches += 2;
            CK_LAUNCH("owner");
            if (h->lean)   // W's padding slots must read as zero again
                CK(cudaMemsetAsync(h->W, 0, 8 * L.S * sizeof(float), h->stream));
            else
                CK(cudaFreeAsync(dkey, h->stream));
        }
        // local thresholding
        CK(cudaMemcpyAsync(ITH, I0, 2 * L.S * sizeof(float), cudaMemcpyDeviceToDevice,
                           h->stream));
        if (h->nseeds > 0) {
            launch_ball_minmax(L, h->seeds_d, h->nseeds, h->p.r_ball, I0, h->stat_d, h->stream);
            launch_threshold_apply(L, h->seeds_d, h->nseeds, h->p.r_ball, h->p.lambda_th,
                                   h->stat_d, h->owner, I0, ITH, h->stream);
            h->launches += 2;
            CK_LAUNCH("threshold");
        }
        // presmoothing of both images, then the face coefficients
        if ((st = presmooth(h, I0, Is0, sweeps))) return st;
        if ((st = presmooth(h, ITH, IsTH, sweeps))) return st;
        if (h->lean) {   // G overwrites plane 3: I_sigma^TH moves to the scratch first
            CK(cudaMemcpyAsync(h->rho, IsTH, plane * sizeof(float), cudaMemcpyDeviceToDevice,
                               h->stream));
            IsTH = h->rho;
            h->img_live = false;
            h->need_u0 = true;   // u held I_sigma^0
        }
        launch_face_G(L, Is0, IsTH, h->p.h, h->p.K, h->p.delta, h->p.vartheta, h->G, h->stream);
        h->launches += 1;
        CK_LAUNCH("face_G");
        h->setup_dirty = false;
        h->has_coef = false;
    }
    if (h->need_u0) {
        CK(cudaMemsetAsync(h->u, 0, 2 * L.S * sizeof(float), h->stream));
        launch_init_u(L, h->seeds_d, h->nseeds, h->p.R_init, h->p.v_init, h->u, h->stream);
        h->launches += h->nseeds > 0 ? 1 : 0;
        CK_LAUNCH("init_u");
        if ((st = rescale(h))) return st;
        h->need_u0 = false;
        h->has_u = true;
    }
    if (!h->has_u) return fail(h, SEG4D_ERR_STATE, "u is not set: call set_seed or set_u");
    return SEG4D_OK;
}

// coefficients + solve on u; fills info fields of the solve
seg4d_status one_solve(seg4d *h, seg4d_info *info, long long &sweeps)
{
    const int brec = launch_step_coef(h->L, h->u, h->G, h->p.h, h->p.tau, h->p.eps, h->beta,
                                      h->gamma, h->diag, h->W, h->partials,
                                      h->has_ghost ? &h->ghost : nullptr, h->stream);
    h->launches += 1;
    CK_LAUNCH("step_coef");
    h->has_coef = true;
    const bool mixed = h->p.precision == 1;
    SolveOut so;
    // with omega_adapt, every solve starts from params.omega and raises it
    // from its own residual history (so a step's result does not depend on
    // earlier steps' solves beyond u itself)
    double om = h->p.omega;
    seg4d_status st = solve_system(h, h->u, brec, h->p.omega, h->p.tol, h->p.max_iters,
                                   h->p.check_every, so, mixed, h->p.tol_inf,
                                   h->p.omega_adapt ? &om : nullptr);
    if (st) return st;
    sweeps += so.iters;
    if (info) {
        info->iters = so.iters;
        info->res_l2 = so.res;
        info->bnorm = so.bnorm;
        info->res_rel = so.bnorm > 0 ? so.res / so.bnorm : so.res;
        info->umin = so.umin;
        info->umax = so.umax;
        info->res_inf = so.res_inf;
        info->bmax = so.bmax;
        info->status = so.converged ? SEG4D_OK : SEG4D_ERR_NOT_CONVERGED;
    }
    if (!so.converged)
        return fail(h, SEG4D_ERR_NOT_CONVERGED, "step solve reached max_iters");
    return SEG4D_OK;
}

// check_finite: the split kernel flags non-finite values; the flag lands in
// host_flag[0] once the stream has reached this point
seg4d_status copy_in(seg4d *h, const float *src, size_t n, int on_device, float *dst_split,
                     bool check_finite = false)
{
    if (!src) return fail(h, SEG4D_ERR_INVALID, "NULL input pointer");
    if ((long long)n != nvox(h)) return fail(h, SEG4D_ERR_INVALID, "array size does not match dims");
    const float *nat = src;
    if (!on_device) {
        CK(cudaMemcpyAsync(h->stage, src, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        nat = h->stage;
    }
    if (check_finite) CK(cudaMemsetAsync(h->d_check, 0, sizeof(unsigned), h->stream));
    launch_split_from_natural(h->L, nat, dst_split, check_finite ? h->d_check : nullptr,
                              h->stream);
    h->launches += 1;
    CK_LAUNCH("split");
    if (check_finite)
        CK(cudaMemcpyAsync(h->host_flag, h->d_check, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           h->stream));
    return SEG4D_OK;
}

seg4d_status copy_out(seg4d *h, const float *split, float *dst, size_t n, int on_device)
{
    if (!dst) return fail(h, SEG4D_ERR_INVALID, "NULL output pointer");
    if ((long long)n != nvox(h)) return fail(h, SEG4D_ERR_INVALID, "array size does not match dims");
    float *nat = on_device ? dst : h->stage;
    launch_natural_from_split(h->L, split, nat, h->stream);
    h->launches += 1;
    CK_LAUNCH("unsplit");
    if (!on_device)
        CK(cudaMemcpyAsync(dst, h->stage, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SEG4D_OK;
}

struct CallTimer {
    seg4d *h;
    explicit CallTimer(seg4d *hh) : h(hh)
    {
        h->launches = 0;
        h->sweep_launches = 0;
        h->sweep_ms = 0.0;
        cudaEventRecord(h->ev0, h->stream);
    }
    float stop()
    {
        float ms = 0.0f;
        cudaEventRecord(h->ev1, h->stream);
        if (cudaEventSynchronize(h->ev1) == cudaSuccess) cudaEventElapsedTime(&ms, h->ev0, h->ev1);
        return ms;
    }
};

}  // namespace

// ====================================================================== ABI

extern "C" {

void seg4d_default_params(seg4d_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    for (int d = 0; d < 4; ++d) p->h[d] = 0.01;
    p->tau = 0.01;
    p->eps = 1.0;
    p->K = 1.0;
    p->delta = 0.5;
    p->vartheta = 0.5;
    p->lambda_th = 0.87;
    p->r_ball = 12.0;
    p->R_init = 12.0;
    p->v_init = 1.0;
    p->sigma_t = 0.01 * 0.01 / 8.0;
    p->omega = 1.6;
    p->omega_adapt = 1;
    p->omega_smooth = 1.0;
    p->tol = 1e-5;
    p->tol_inf = 1e-5;
    p->tol_smooth = 1e-6;
    p->max_iters = 20000;
    p->check_every = 10;
    p->sweep_variant = 1;
    p->precision = 0;
}

size_t seg4d_device_bytes(const seg4d_dims *dims) { return seg4d_device_bytes_ex(dims, 0); }

size_t seg4d_device_bytes_ex(const seg4d_dims *dims, int flags)
{
    if (!dims_ok(dims)) return 0;
    Layout L = make_layout(*dims);
    return bytes_for(L, (long long)dims->n1 * dims->n2 * dims->n3 * dims->n4,
                     (flags & SEG4D_CREATE_LEAN) != 0);
}

seg4d_status seg4d_create(const seg4d_dims *dims, void *cuda_stream, seg4d **out)
{
    return seg4d_create_ex(dims, cuda_stream, 0, out);
}

seg4d_status seg4d_create_ex(const seg4d_dims *dims, void *cuda_stream, int flags, seg4d **out)
{
    g_create_error.clear();
    if (flags & ~SEG4D_CREATE_LEAN) {
        g_create_error = "unknown creation flags";
        return SEG4D_ERR_INVALID;
    }
    if (!out) {
        g_create_error = "out is NULL";
        return SEG4D_ERR_INVALID;
    }
    *out = nullptr;
    if (!dims_ok(dims)) {
        g_create_error = "invalid dims (each >= 1, n3, n4 <= 65535, n1*n2*n3*n4 < 2^33)";
        return SEG4D_ERR_INVALID;
    }
    seg4d *h = new (std::nothrow) seg4d();
    if (!h) {
        g_create_error = "host allocation failed";
        return SEG4D_ERR_OOM;
    }
    h->dims = *dims;
    h->L = make_layout(*dims);
    h->stream = (cudaStream_t)cuda_stream;
    seg4d_default_params(&h->p);
    cudaGetDevice(&h->device);
    const Layout &L = h->L;
    const size_t S = (size_t)L.S;
    const long long nv = nvox(h);
    h->lean = (flags & SEG4D_CREATE_LEAN) != 0;
    struct A {
        void **p;
        size_t bytes;
    };
    std::vector<A> allocs = {
        {(void **)&h->u, 2 * S * 4},     {(void **)&h->beta, 2 * S * 4},
        {(void **)&h->gamma, 2 * S * 4}, {(void **)&h->diag, 2 * S * 4},
        {(void **)&h->W, 8 * S * 4},     {(void **)&h->G, (size_t)g_floats(L) * 4},
        {(void **)&h->owner, 2 * S * 4},
        {(void **)&h->partials, 4 * kPartCap * sizeof(double)},
        {(void **)&h->scal, 8 * sizeof(double)},
        {(void **)&h->d_check, 4 * sizeof(unsigned)},
    };
    if (h->lean) {
        // the solve's scratch exists from the start; staging and the image
        // fields live inside it and inside G (see run_setup)
        allocs.push_back({(void **)&h->ib, 2 * S * 4});
        allocs.push_back({(void **)&h->rho, 2 * S * 4});
        allocs.push_back({(void **)&h->dlt, 2 * S * 4});
    } else {
        allocs.push_back({(void **)&h->I0, 2 * S * 4});
        allocs.push_back({(void **)&h->ITH, 2 * S * 4});
        allocs.push_back({(void **)&h->Is0, 2 * S * 4});
        allocs.push_back({(void **)&h->IsTH, 2 * S * 4});
        allocs.push_back({(void **)&h->stage, (size_t)nv * 4});
    }
    for (auto &a : allocs) {
        if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            free_all(h);
            delete h;
            g_create_error = "device allocation failed (" + std::to_string(a.bytes) + " bytes)";
            return SEG4D_ERR_OOM;
        }
        // padding slots must read as zero in every array
        if (cudaMemsetAsync(*a.p, 0, a.bytes, h->stream) != cudaSuccess) {
            free_all(h);
            delete h;
            g_create_error = "cudaMemsetAsync failed";
            return SEG4D_ERR_CUDA;
        }
    }
    if (h->lean) {
        h->stage = h->rho;   // 2S >= n1 n2 n3 n4 floats
        h->I0 = h->G;        // plane 0 of G until the set-up computes G
    }
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (h->num_sms < 1) h->num_sms = 1;
    if (cudaMallocHost(&h->host_scal, 8 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&h->host_flag, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess ||
        cudaEventCreate(&h->evs0) != cudaSuccess || cudaEventCreate(&h->evs1) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        free_all(h);
        delete h;
        g_create_error = "pinned buffer / event creation failed";
        return SEG4D_ERR_CUDA;
    }
    *out = h;
    return SEG4D_OK;
}

seg4d_status seg4d_destroy(seg4d *h)
{
    if (!h) return SEG4D_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return SEG4D_OK;
}

seg4d_status seg4d_set_params(seg4d *h, const seg4d_params *p)
{
    if (!h) return SEG4D_ERR_INVALID;
    if (!p) return fail(h, SEG4D_ERR_INVALID, "params is NULL");
    for (int d = 0; d < 4; ++d)
        if (!finite_pos(p->h[d])) return fail(h, SEG4D_ERR_INVALID, "h must be finite and > 0");
    if (!finite_pos(p->tau) || !finite_pos(p->eps) || !finite_pos(p->sigma_t))
        return fail(h, SEG4D_ERR_INVALID, "tau, eps and sigma_t must be finite and > 0");
    if (!std::isfinite(p->K) || p->K < 0) return fail(h, SEG4D_ERR_INVALID, "K must be >= 0");
    if (!in01(p->delta) || !in01(p->vartheta) || !in01(p->lambda_th))
        return fail(h, SEG4D_ERR_INVALID, "delta, vartheta and lambda_th must lie in [0,1]");
    if (!finite_pos(p->r_ball) || !finite_pos(p->R_init) || !finite_pos(p->v_init))
        return fail(h, SEG4D_ERR_INVALID, "r_ball, R_init and v_init must be > 0");
    if (!(p->omega > 0 && p->omega < 2) || !(p->omega_smooth > 0 && p->omega_smooth < 2))
        return fail(h, SEG4D_ERR_INVALID, "omega and omega_smooth must lie in (0, 2)");
    if (!finite_pos(p->tol) || !finite_pos(p->tol_smooth))
        return fail(h, SEG4D_ERR_INVALID, "tol and tol_smooth must be finite and > 0");
    if (!std::isfinite(p->tol_inf) || p->tol_inf < 0)
        return fail(h, SEG4D_ERR_INVALID, "tol_inf must be finite and >= 0");
    if (p->max_iters < 1 || p->check_every < 1)
        return fail(h, SEG4D_ERR_INVALID, "max_iters and check_every must be >= 1");
    if (p->precision != 0 && p->precision != 1)
        return fail(h, SEG4D_ERR_INVALID, "precision must be 0 or 1");
    if (p->omega_adapt != 0 && p->omega_adapt != 1)
        return fail(h, SEG4D_ERR_INVALID, "omega_adapt must be 0 or 1");
    if ((p->sweep_variant != 1 && p->sweep_variant != 2) || p->ctas_per_sm != 0 ||
        p->wait_test != 0)
        return fail(h, SEG4D_ERR_INVALID,
                    "sweep_variant must be 1 or 2, ctas_per_sm and wait_test 0 (reserved)");
    const bool geom = std::memcmp(p->h, h->p.h, sizeof(p->h)) != 0 || p->K != h->p.K ||
                      p->delta != h->p.delta || p->vartheta != h->p.vartheta ||
                      p->lambda_th != h->p.lambda_th || p->r_ball != h->p.r_ball ||
                      p->sigma_t != h->p.sigma_t || p->R_init != h->p.R_init ||
                      p->omega_smooth != h->p.omega_smooth || p->tol_smooth != h->p.tol_smooth;
    h->p = *p;
    if (geom) h->setup_dirty = true;
    return SEG4D_OK;
}

seg4d_status seg4d_set_image(seg4d *h, const float *I0, size_t n, int on_device)
{
    if (!h) return SEG4D_ERR_INVALID;
    seg4d_status st = use_device(h);
    if (st) return st;
    if (h->lean) h->I0 = h->G;
    if ((st = copy_in(h, I0, n, on_device, h->I0, true))) return st;
    CK(cudaStreamSynchronize(h->stream));
    if (h->host_flag[0] != 0u) {   // the copy overwrote the old image
        h->has_image = false;
        h->setup_dirty = true;
        return fail(h, SEG4D_ERR_INVALID, "image has NaN/Inf; the handle has no image now");
    }
    h->has_image = true;
    h->img_live = true;
    h->setup_dirty = true;
    return SEG4D_OK;
}

seg4d_status seg4d_set_seed(seg4d *h, const seg4d_seed *seeds, int nseeds)
{
    if (!h) return SEG4D_ERR_INVALID;
    if (nseeds < 0 || (nseeds > 0 && !seeds))
        return fail(h, SEG4D_ERR_INVALID, "bad seed array");
    for (int m = 0; m < nseeds; ++m)
        if (!std::isfinite(seeds[m].x) || !std::isfinite(seeds[m].y) || !std::isfinite(seeds[m].z))
            return fail(h, SEG4D_ERR_INVALID, "seed coordinates must be finite");
    h->seeds.assign(seeds, seeds + nseeds);
    h->setup_dirty = true;
    h->need_u0 = true;
    return SEG4D_OK;
}

seg4d_status seg4d_set_u(seg4d *h, const float *u, size_t n, int on_device)
{
    if (!h) return SEG4D_ERR_INVALID;
    seg4d_status st = use_device(h);
    if (st) return st;
    if ((st = copy_in(h, u, n, on_device, h->u))) return st;
    CK(cudaStreamSynchronize(h->stream));
    h->has_u = true;
    h->need_u0 = false;
    h->has_coef = false;
    return SEG4D_OK;
}

size_t seg4d_dirichlet_count(const seg4d_dims *d)
{
    if (!dims_ok(d)) return 0;
    const long long np[4] = {d->n1 + 2LL, d->n2 + 2LL, d->n3 + 2LL, d->n4 + 2LL};
    long long total = 0;
    for (int a = 0; a < 4; ++a) total += 2 * (np[0] * np[1] * np[2] * np[3] / np[a]);
    return (size_t)total;
}

seg4d_status seg4d_set_dirichlet(seg4d *h, const float *g_prev, const float *g_now, size_t n,
                                 int on_device)
{
    if (!h) return SEG4D_ERR_INVALID;
    seg4d_status st = use_device(h);
    if (st) return st;
    if (!g_prev && !g_now) {
        h->has_ghost = false;
        return SEG4D_OK;
    }
    if (!g_prev || !g_now) return fail(h, SEG4D_ERR_INVALID, "give both ghost arrays, or neither");
    const size_t need = seg4d_dirichlet_count(&h->dims);
    if (n != need)
        return fail(h, SEG4D_ERR_INVALID,
                    "ghost data needs seg4d_dirichlet_count(dims) = " + std::to_string(need) +
                        " floats per time level");
    if (!h->gh_prev) {
        if (cudaMalloc(&h->gh_prev, n * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&h->gh_now, n * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(h->gh_prev);
            h->gh_prev = h->gh_now = nullptr;
            return fail(h, SEG4D_ERR_OOM, "ghost data: device allocation failed");
        }
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(h->gh_prev, g_prev, n * sizeof(float), kind, h->stream));
    CK(cudaMemcpyAsync(h->gh_now, g_now, n * sizeof(float), kind, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    Ghost &G = h->ghost;
    G.prev = h->gh_prev;
    G.now = h->gh_now;
    const int nd[4] = {h->dims.n1, h->dims.n2, h->dims.n3, h->dims.n4};
    long long off = 0;
    for (int a = 0; a < 4; ++a) G.np[a] = nd[a] + 2;
    for (int a = 0; a < 4; ++a) {
        long long sz = 1;
        for (int e = 0; e < 4; ++e)
            if (e != a) sz *= G.np[e];
        G.off[a] = off;
        G.size[a] = sz;
        off += 2 * sz;
    }
    h->has_ghost = true;
    h->has_coef = false;
    return SEG4D_OK;
}

seg4d_status seg4d_setup(seg4d *h, seg4d_info *info)
{
    if (!h) return SEG4D_ERR_INVALID;
    seg4d_status st = use_device(h);
    if (st) return st;
    if (info) std::memset(info, 0, sizeof(*info));
    CallTimer t(h);
    long long sweeps = 0;
    st = run_setup(h, sweeps);
    const float ms = t.stop();
    if (info) {
        info->sweeps_total = sweeps;
        info->ms = ms;
        info->sweep_ms = h->sweep_ms;
        info->launches = h->launches;
        info->sweep_launches = h->sweep_launches;
        info->status = st;
    }
    return st;
}

seg4d_status seg4d_solve(seg4d *h, seg4d_info *info)
{
    if (!h) return SEG4D_ERR_INVALID;
    seg4d_status st = use_device(h);
    if (st) return st;
    if (info) std::memset(info, 0, sizeof(*info));
    CallTimer t(h);
    long long sweeps = 0;
    st = run_setup(h, sweeps);
    if (!st) st = one_solve(h, info, sweeps);
    const float ms = t.stop();
    if (info) {
        info->sweeps_total = sweeps;
        info->ms = ms;
        info->sweep_ms = h->sweep_ms;
        info->launches = h->launches;
        info->sweep_launches = h->sweep_launches;
        info->status = st;
    }
    return st;
}

seg4d_status seg4d_step(seg4d *h, int nsteps, seg4d_info *info)
{
    if (!h) return SEG4D_ERR_INVALID;
    if (nsteps < 0) return fail(h, SEG4D_ERR_INVALID, "nsteps < 0");
    seg4d_status st = use_device(h);
    if (st) return st;
    if (info) std::memset(info, 0, sizeof(*info));
    CallTimer t(h);
    long long sweeps = 0;
    st = run_setup(h, sweeps);
    int done = 0;
    for (; !st && done < nsteps; ++done) {
        st = one_solve(h, info, sweeps);
        if (st) break;
        st = rescale(h);
    }
    const float ms = t.stop();
    if (info) {
        info->sweeps_total = sweeps;
        info->steps_done = done;
        info->ms = ms;
        info->sweep_ms = h->sweep_ms;
        info->launches = h->launches;
        info->sweep_launches = h->sweep_launches;
        info->status = st;
    }
    return st;
}

seg4d_status seg4d_read_u(seg4d *h, float *dst, size_t n, int on_device)
{
    if (!h) return SEG4D_ERR_INVALID;
    seg4d_status st = use_device(h);
    if (st) return st;
    if (!h->has_u && !h->need_u0) return fail(h, SEG4D_ERR_STATE, "u is not set");
    if (h->need_u0) {
        long long sweeps = 0;
        if ((st = run_setup(h, sweeps))) return st;
    }
    return copy_out(h, h->u, dst, n, on_device);
}

seg4d_status seg4d_read_field(seg4d *h, int field, float *dst, size_t n, int on_device)
{
    if (!h) return SEG4D_ERR_INVALID;
    seg4d_status st = use_device(h);
    if (st) return st;
    if (!dst) return fail(h, SEG4D_ERR_INVALID, "NULL output pointer");
    const long long nv = nvox(h);
    switch (field) {
    case SEG4D_FIELD_U:
        return seg4d_read_u(h, dst, n, on_device);
    case SEG4D_FIELD_I0:
        if (!h->has_image) return fail(h, SEG4D_ERR_STATE, "no image set");
        if (h->lean && !h->img_live)
            return fail(h, SEG4D_ERR_STATE, "a lean handle keeps no image after its set-up");
        return copy_out(h, h->I0, dst, n, on_device);
    case SEG4D_FIELD_ITH:
    case SEG4D_FIELD_ISIG0:
    case SEG4D_FIELD_ISIGTH:
        if (h->lean) return fail(h, SEG4D_ERR_STATE, "a lean handle keeps no image fields");
        [[fallthrough]];
    case SEG4D_FIELD_OWNER:
    case SEG4D_FIELD_G:
        if (!h->has_image || h->setup_dirty)
            return fail(h, SEG4D_ERR_STATE, "set-up not computed (call seg4d_setup)");
        break;
    case SEG4D_FIELD_DIAG:
    case SEG4D_FIELD_OFF:
        if (!h->has_coef) return fail(h, SEG4D_ERR_STATE, "no step coefficients computed");
        break;
    default:
        return fail(h, SEG4D_ERR_INVALID, "unknown field");
    }
    if (field == SEG4D_FIELD_ITH) return copy_out(h, h->ITH, dst, n, on_device);
    if (field == SEG4D_FIELD_ISIG0) return copy_out(h, h->Is0, dst, n, on_device);
    if (field == SEG4D_FIELD_ISIGTH) return copy_out(h, h->IsTH, dst, n, on_device);
    if (field == SEG4D_FIELD_DIAG) return copy_out(h, h->diag, dst, n, on_device);
    if (field == SEG4D_FIELD_OWNER) {
        if ((long long)n != nv) return fail(h, SEG4D_ERR_INVALID, "array size does not match dims");
        float *nat = on_device ? dst : h->stage;
        launch_owner_natural(h->L, h->owner, nat, h->stream);
        CK_LAUNCH("owner_natural");
        if (!on_device)
            CK(cudaMemcpyAsync(dst, h->stage, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return SEG4D_OK;
    }
    // 8 values per voxel: G or OFF
    if ((long long)n != 8 * nv)
        return fail(h, SEG4D_ERR_INVALID, "face fields need 8 * n1*n2*n3*n4 floats");
    float *nat8 = dst;
    if (!on_device) {
        if (cudaMallocAsync((void **)&nat8, n * sizeof(float), h->stream) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, SEG4D_ERR_OOM, "read_field: temporary allocation failed");
        }
    }
    if (field == SEG4D_FIELD_G)
        launch_G_natural(h->L, h->G, nat8, h->stream);
    else
        launch_off_natural(h->L, h->W, h->gamma, h->diag, nat8, h->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !on_device)
        e = cudaMemcpyAsync(dst, nat8, n * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (!on_device) cudaFreeAsync(nat8, h->stream);
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(h, SEG4D_ERR_CUDA, std::string("read_field: ") +
                                           cudaGetErrorString(e != cudaSuccess ? e : e2));
    return SEG4D_OK;
}

const char *seg4d_last_error(const seg4d *h)
{
    if (!h) return g_create_error.c_str();
    return h->err.c_str();
}

}  // extern "C"
