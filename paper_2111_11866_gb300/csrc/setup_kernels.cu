// setup_kernels.cu -- the work before the time loop (Section 3.6): local
// thresholding and ball owners (Section 3.1), presmoothing coefficients (the
// linear heat equation, Section 3.1), face edge coefficients G (Eq. 10th with
// g of Eq. eg1), the initial condition (Eq. initialcond) and local rescaling
// (Remark, Eq. 841); plus conversions between the caller's x-fastest arrays
// and the colour-split layout of seg4d_internal.cuh.
//
// Decisions that turn floating point into a discrete choice (ball membership,
// nearest seed, I0 >= TH) are taken in double precision with explicitly
// rounded operations (no contraction into FMA), in the same order as the
// plain definition, so that they do not depend on compiler contraction.
#include <cfloat>
#include <climits>
#include <cmath>

#include "stencil.cuh"

namespace seg4d_impl {

// ------------------------------------------------------------ conversions

// natural (x fastest) -> colour-split; one thread per natural voxel.  bad
// (nullable): set to 1 when a value is not finite.
__global__ void k_split_from_natural(Layout L, const float *__restrict__ nat,
                                     float *__restrict__ split, unsigned *__restrict__ bad)
{
    const long long n = (long long)L.n1 * L.R;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % L.n1);
        const long long row = v / L.n1;
        const int j = (int)(row % L.n2);
        const long long t = row / L.n2;
        const int k = (int)(t % L.n3);
        const int l = (int)(t / L.n3);
        int c;
        const long long s = slot_of(L, i, j, k, l, c);
        const float x = nat[v];
        split[c * L.S + s] = x;
        if (bad && !isfinite(x)) atomicOr(bad, 1u);
    }
}

__global__ void k_natural_from_split(Layout L, const float *__restrict__ split,
                                     float *__restrict__ nat, int nf)
{
    // nf = fields per voxel (1, or 8 for face arrays stored [c][f][S])
    const long long n = (long long)L.n1 * L.R;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % L.n1);
        const long long row = v / L.n1;
        const int j = (int)(row % L.n2);
        const long long t = row / L.n2;
        const int k = (int)(t % L.n3);
        const int l = (int)(t / L.n3);
        int c;
        const long long s = slot_of(L, i, j, k, l, c);
        for (int f = 0; f < nf; ++f) nat[v * nf + f] = split[((long long)c * nf + f) * L.S + s];
    }
}

__global__ void k_owner_natural(Layout L, const int *__restrict__ owner, float *__restrict__ nat)
{
    const long long n = (long long)L.n1 * L.R;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % L.n1);
        const long long row = v / L.n1;
        const int j = (int)(row % L.n2);
        const long long t = row / L.n2;
        const int k = (int)(t % L.n3);
        const int l = (int)(t / L.n3);
        int c;
        const long long s = slot_of(L, i, j, k, l, c);
        const int o = owner[c * L.S + s];
        nat[v] = o == kOwnerNone ? -1.0f : (float)o;
    }
}

// Off-diagonal magnitudes c*w_f per voxel and face (faces to the boundary: 0).
__global__ void k_off_natural(Layout L, const float *__restrict__ W,
                              const float *__restrict__ gamma, const float *__restrict__ diag,
                              float *__restrict__ nat8)
{
    const long long n = (long long)L.n1 * L.R;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int ci[4] = {(int)(v % L.n1), (int)((v / L.n1) % L.n2),
                           (int)((v / ((long long)L.n1 * L.n2)) % L.n3),
                           (int)(v / ((long long)L.n1 * L.n2 * L.n3))};
        const int nn[4] = {L.n1, L.n2, L.n3, L.n4};
        int c;
        const long long s = slot_of(L, ci[0], ci[1], ci[2], ci[3], c);
        const float cc = gamma[c * L.S + s] * diag[c * L.S + s];   // c = gamma * D
        for (int f = 0; f < 8; ++f) {
            const int d = f >> 1;
            int nb[4] = {ci[0], ci[1], ci[2], ci[3]};
            nb[d] += (f & 1) ? 1 : -1;
            float w = 0.0f;
            if (nb[d] >= 0 && nb[d] < nn[d]) {
                if (c == 0) {
                    w = W[(long long)f * L.S + s];
                } else {
                    int c2;
                    const long long s2 = slot_of(L, nb[0], nb[1], nb[2], nb[3], c2);
                    w = W[(long long)(f ^ 1) * L.S + s2];
                }
            }
            nat8[v * 8 + f] = cc * w;
        }
    }
}

static int conv_blocks(const Layout &L)
{
    const long long n = (long long)L.n1 * L.R;
    long long b = (n + 255) / 256;
    if (b > 152LL * 64) b = 152LL * 64;
    return (int)(b < 1 ? 1 : b);
}

void launch_split_from_natural(const Layout &L, const float *nat, float *split, unsigned *bad,
                               cudaStream_t st)
{
    k_split_from_natural<<<conv_blocks(L), 256, 0, st>>>(L, nat, split, bad);
}

void launch_natural_from_split(const Layout &L, const float *split, float *nat, cudaStream_t st)
{
    k_natural_from_split<<<conv_blocks(L), 256, 0, st>>>(L, split, nat, 1);
}

// G per voxel and face in x-fastest order ([voxel][8]) from its per-face
// storage (load_G8)
__global__ void k_G_natural(Layout L, const float *__restrict__ G, float *__restrict__ nat8)
{
    const long long n = (long long)L.n1 * L.R;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(v % L.n1);
        const int row = (int)(v / L.n1);
        RowPos rp;
        rp.j = row % L.n2;
        rp.k = (row / L.n2) % L.n3;
        rp.l = row / (L.n2 * L.n3);
        rp.p = (rp.j + rp.k + rp.l) & 1;
        const int s = i >> 1;
        float g[8];
        if (((i + rp.j + rp.k + rp.l) & 1) == 0)
            load_G8<0>(L, G, true, row, s, rp, g);
        else
            load_G8<1>(L, G, true, row, s, rp, g);
#pragma unroll
        for (int f = 0; f < 8; ++f) nat8[v * 8 + f] = g[f];
    }
}

void launch_G_natural(const Layout &L, const float *G, float *nat8, cudaStream_t st)
{
    k_G_natural<<<conv_blocks(L), 256, 0, st>>>(L, G, nat8);
}

void launch_owner_natural(const Layout &L, const int *owner, float *nat, cudaStream_t st)
{
    k_owner_natural<<<conv_blocks(L), 256, 0, st>>>(L, owner, nat);
}

void launch_off_natural(const Layout &L, const float *W, const float *gamma, const float *diag,
                        float *nat8, cudaStream_t st)
{
    k_off_natural<<<conv_blocks(L), 256, 0, st>>>(L, W, gamma, diag, nat8);
}

// ------------------------------------------------------------- seed balls

// squared spatial distance, evaluated as ((dx*dx + dy*dy) + dz*dz) with
// rounded double operations
__device__ inline double seed_d2(const SeedDev &sd, int i, int j, int k)
{
    const double dx = __dsub_rn((double)i, sd.x);
    const double dy = __dsub_rn((double)j, sd.y);
    const double dz = __dsub_rn((double)k, sd.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Iterate over the voxels of seed m's bounding box with the whole block.
#define FOR_BALL_BOX(sd, L, i, j, k, BODY)                                                 \
    {                                                                                      \
        const int nx_ = sd.bx1 - sd.bx0 + 1, ny_ = sd.by1 - sd.by0 + 1,                    \
                  nz_ = sd.bz1 - sd.bz0 + 1;                                               \
        const long long nb_ = (nx_ > 0 && ny_ > 0 && nz_ > 0 && sd.frame >= 0 &&           \
                               sd.frame < L.n4)                                            \
                                  ? (long long)nx_ * ny_ * nz_                             \
                                  : 0;                                                     \
        for (long long e_ = threadIdx.x; e_ < nb_; e_ += blockDim.x) {                     \
            const int i = sd.bx0 + (int)(e_ % nx_);                                        \
            const int j = sd.by0 + (int)((e_ / nx_) % ny_);                                \
            const int k = sd.bz0 + (int)(e_ / ((long long)nx_ * ny_));                     \
            BODY                                                                           \
        }                                                                                  \
    }

// pass 1: dkey = min over seeds of the ball distance (double bits are ordered
// like unsigned integers for non-negative values); pass 2: owner = lowest
// seed index attaining it.
__global__ void k_owner_dist(Layout L, const SeedDev *__restrict__ seeds, double r2,
                             unsigned long long *__restrict__ dkey)
{
    const SeedDev sd = seeds[blockIdx.x];
    FOR_BALL_BOX(sd, L, i, j, k, {
        const double d2 = seed_d2(sd, i, j, k);
        if (d2 <= r2) {
            int c;
            const long long s = slot_of(L, i, j, k, sd.frame, c);
            atomicMin(&dkey[c * L.S + s], (unsigned long long)__double_as_longlong(d2));
        }
    })
}

__global__ void k_owner_pick(Layout L, const SeedDev *__restrict__ seeds, double r2,
                             const unsigned long long *__restrict__ dkey, int *__restrict__ owner)
{
    const int m = blockIdx.x;
    const SeedDev sd = seeds[m];
    FOR_BALL_BOX(sd, L, i, j, k, {
        const double d2 = seed_d2(sd, i, j, k);
        if (d2 <= r2) {
            int c;
            const long long s = slot_of(L, i, j, k, sd.frame, c);
            if ((unsigned long long)__double_as_longlong(d2) == dkey[c * L.S + s])
                atomicMin(&owner[c * L.S + s], m);
        }
    })
}

void launch_owner(const Layout &L, const SeedDev *seeds, int nseeds, double r,
                  unsigned long long *dkey, int *owner, cudaStream_t st)
{
    if (nseeds <= 0) return;
    const double r2 = r * r;
    k_owner_dist<<<nseeds, 256, 0, st>>>(L, seeds, r2, dkey);
    k_owner_pick<<<nseeds, 256, 0, st>>>(L, seeds, r2, dkey, owner);
}

// min / max of a field over the whole ball of each seed (one block per seed)
__global__ void k_ball_minmax(Layout L, const SeedDev *__restrict__ seeds, double r2,
                              const float *__restrict__ field, SeedStat *__restrict__ out)
{
    const SeedDev sd = seeds[blockIdx.x];
    float mn = FLT_MAX, mx = -FLT_MAX;
    int cnt = 0;
    FOR_BALL_BOX(sd, L, i, j, k, {
        if (seed_d2(sd, i, j, k) <= r2) {
            int c;
            const long long s = slot_of(L, i, j, k, sd.frame, c);
            const float v = field[c * L.S + s];
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
            ++cnt;
        }
    })
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    __shared__ float smn[32], smx[32];
    __shared__ int scnt[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        smn[wid] = mn;
        smx[wid] = mx;
        scnt[wid] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mn = fminf(mn, smn[w]);
            mx = fmaxf(mx, smx[w]);
            cnt += scnt[w];
        }
        out[blockIdx.x] = SeedStat{mn, mx, cnt, 0};
    }
}

void launch_ball_minmax(const Layout &L, const SeedDev *seeds, int nseeds, double r,
                        const float *field, SeedStat *out, cudaStream_t st)
{
    if (nseeds <= 0) return;
    k_ball_minmax<<<nseeds, 256, 0, st>>>(L, seeds, r * r, field, out);
}

// Local thresholding (Section 3.1) on the voxels each seed owns:
// TH = lambda*alpha + (1-lambda)*beta in double; I0 >= TH -> beta, else alpha.
// ITH must hold a copy of I0 beforehand (voxels outside every ball keep I0).
__global__ void k_threshold_apply(Layout L, const SeedDev *__restrict__ seeds, double r2,
                                  double lambda, const SeedStat *__restrict__ stat,
                                  const int *__restrict__ owner, const float *__restrict__ I0,
                                  float *__restrict__ ITH)
{
    const int m = blockIdx.x;
    const SeedDev sd = seeds[m];
    const SeedStat ss = stat[m];
    if (ss.count == 0) return;
    const double alpha = (double)ss.mn, beta = (double)ss.mx;
    const double TH = __dadd_rn(__dmul_rn(lambda, alpha), __dmul_rn(__dsub_rn(1.0, lambda), beta));
    FOR_BALL_BOX(sd, L, i, j, k, {
        if (seed_d2(sd, i, j, k) <= r2) {
            int c;
            const long long s = slot_of(L, i, j, k, sd.frame, c);
            if (owner[c * L.S + s] == m)
                ITH[c * L.S + s] = ((double)I0[c * L.S + s] >= TH) ? ss.mx : ss.mn;
        }
    })
}

void launch_threshold_apply(const Layout &L, const SeedDev *seeds, int nseeds, double r,
                            double lambda, const SeedStat *stat, const int *owner,
                            const float *I0, float *ITH, cudaStream_t st)
{
    if (nseeds <= 0) return;
    k_threshold_apply<<<nseeds, 256, 0, st>>>(L, seeds, r * r, lambda, stat, owner, I0, ITH);
}

// u0 = 1/(d + v) - 1/(R + v) inside the ball of radius R, maximum over seeds
// (values are >= 0, so their float bits order like ints).  u must be zeroed.
__global__ void k_init_u(Layout L, const SeedDev *__restrict__ seeds, double R2, double R,
                         double v, float *__restrict__ u)
{
    const SeedDev sd = seeds[blockIdx.x];
    FOR_BALL_BOX(sd, L, i, j, k, {
        const double d2 = seed_d2(sd, i, j, k);
        if (d2 <= R2) {
            const double val = 1.0 / (sqrt(d2) + v) - 1.0 / (R + v);
            const float fv = val > 0.0 ? (float)val : 0.0f;
            int c;
            const long long s = slot_of(L, i, j, k, sd.frame, c);
            atomicMax((int *)&u[c * L.S + s], __float_as_int(fv));
        }
    })
}

void launch_init_u(const Layout &L, const SeedDev *seeds, int nseeds, double R, double v,
                   float *u, cudaStream_t st)
{
    if (nseeds <= 0) return;
    k_init_u<<<nseeds, 256, 0, st>>>(L, seeds, R * R, R, v, u);
}

// Local rescaling (Eq. 841) of the voxels each seed owns with the min/max of
// its whole ball, taken before any ball was rescaled.
__global__ void k_rescale_apply(Layout L, const SeedDev *__restrict__ seeds, double r2,
                                const SeedStat *__restrict__ stat, const int *__restrict__ owner,
                                float *__restrict__ u)
{
    const int m = blockIdx.x;
    const SeedDev sd = seeds[m];
    const SeedStat ss = stat[m];
    if (ss.count == 0) return;
    const double mu = ss.mn, span = (double)ss.mx - (double)ss.mn;
    if (!(span > 1e-30)) return;
    FOR_BALL_BOX(sd, L, i, j, k, {
        if (seed_d2(sd, i, j, k) <= r2) {
            int c;
            const long long s = slot_of(L, i, j, k, sd.frame, c);
            if (owner[c * L.S + s] == m)
                u[c * L.S + s] = (float)(((double)u[c * L.S + s] - mu) / span);
        }
    })
}

void launch_rescale_apply(const Layout &L, const SeedDev *seeds, int nseeds, double r,
                          const SeedStat *stat, const int *owner, float *u, cudaStream_t st)
{
    if (nseeds <= 0) return;
    k_rescale_apply<<<nseeds, 256, 0, st>>>(L, seeds, r * r, stat, owner, u);
}

// ------------------------------------------------------- face coefficients

struct GConst {
    float inv_h[4];
    float K, delta, vartheta;
};

// |grad^f I|^2 with replicated ghosts (reduced diamond cell, Section 3.2)
__device__ inline float face_grad_sq_img(const Layout &L, const float *__restrict__ I, const int *c,
                                         int f, const float *inv_h)
{
    const int d = f >> 1;
    int nb[4] = {c[0], c[1], c[2], c[3]};
    nb[d] += (f & 1) ? 1 : -1;
    const float u0 = ld_replicate(L, I, c[0], c[1], c[2], c[3]);
    const float un = ld_replicate(L, I, nb[0], nb[1], nb[2], nb[3]);
    const float nrm = (un - u0) * inv_h[d];
    float sum = nrm * nrm;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        if (t == d) continue;
        int a[4] = {c[0], c[1], c[2], c[3]};
        int b[4] = {nb[0], nb[1], nb[2], nb[3]};
        a[t] += 1;
        b[t] += 1;
        const float up = ld_replicate(L, I, a[0], a[1], a[2], a[3]) +
                         ld_replicate(L, I, b[0], b[1], b[2], b[3]);
        a[t] -= 2;
        b[t] -= 2;
        const float dn = ld_replicate(L, I, a[0], a[1], a[2], a[3]) +
                         ld_replicate(L, I, b[0], b[1], b[2], b[3]);
        const float comp = 0.25f * (up - dn) * inv_h[t];
        sum += comp * comp;
    }
    return sum;
}

// G_f = 1 / (1 + K s^2), s = delta |grad^f Is0| + vartheta |grad^f IsTH|,
// once per face: every red voxel's 8 faces in the planes, and a black
// voxel's faces to the Dirichlet ring in the side table (gb_offsets).  The
// face gradient is symmetric in the face's two cells, so the red end's value
// is the face's.
__global__ void k_face_G(Layout L, const float *__restrict__ Is0, const float *__restrict__ IsTH,
                         GConst K, float *__restrict__ G)
{
    const long long n = 2LL * L.S;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int C = e >= L.S ? 1 : 0;
        const long long q = e - (long long)C * L.S;
        const int row = (int)(q / L.P);
        const int s = (int)(q - (long long)row * L.P);
        const int j = row % L.n2;
        const int k = (row / L.n2) % L.n3;
        const int l = row / (L.n2 * L.n3);
        const int i = 2 * s + (C ^ ((j + k + l) & 1));
        if (i >= L.n1) continue;
        const int c[4] = {i, j, k, l};
        const int nn[4] = {L.n1, L.n2, L.n3, L.n4};
        const GbOff o = gb_offsets(L);
        for (int f = 0; f < 8; ++f) {
            const int nb = c[f >> 1] + ((f & 1) ? 1 : -1);
            const bool ring = nb < 0 || nb >= nn[f >> 1];
            if (C == 1 && !ring) continue;   // stored by the red end
            const float a0 = sqrtf(face_grad_sq_img(L, Is0, c, f, K.inv_h));
            const float a1 = sqrtf(face_grad_sq_img(L, IsTH, c, f, K.inv_h));
            const float sv = K.delta * a0 + K.vartheta * a1;
            const float g = 1.0f / (1.0f + K.K * sv * sv);
            if (C == 0)
                G[(long long)f * L.S + q] = g;
            else
                G[8 * L.S + gb_index(L, o, f, row, s, j, k, l)] = g;
        }
    }
}

void launch_face_G(const Layout &L, const float *Is0, const float *IsTH, const double *h,
                   double K, double delta, double vartheta, float *G, cudaStream_t st)
{
    GConst c;
    for (int d = 0; d < 4; ++d) c.inv_h[d] = (float)(1.0 / h[d]);
    c.K = (float)K;
    c.delta = (float)delta;
    c.vartheta = (float)vartheta;
    long long n = 2LL * L.S;
    long long b = (n + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    k_face_G<<<(int)(b < 1 ? 1 : b), 256, 0, st>>>(L, Is0, IsTH, c, G);
}

// ------------------------------------------------- presmoothing coefficients

// One implicit heat step of length sigma_t with zero-Neumann data:
//   v + sum_{faces inside the grid} sigma_t/h_d^2 (v - v_nb) = I,
// i.e. w_f = 1/h_d^2 on interior faces (0 on boundary faces), c = sigma_t,
// D = 1 + c sum_f w_f, beta = I (the right-hand side), gamma = c/D.
// Records: (sum I^2, min, max).
__global__ void __launch_bounds__(kPartThreads) k_smooth_coef(Layout L, const float *__restrict__ I,
                                                              float4 inv_h2, float sigma_t,
                                                              float *__restrict__ beta,
                                                              float *__restrict__ gamma,
                                                              float *__restrict__ diag,
                                                              float *__restrict__ W,
                                                              double *__restrict__ partials)
{
    const float ih2[4] = {inv_h2.x, inv_h2.y, inv_h2.z, inv_h2.w};
    const int nn[4] = {L.n1, L.n2, L.n3, L.n4};
    Rec3f a = rec3f_init();
    const long long n = 2LL * L.S;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int C = e >= L.S ? 1 : 0;
        const long long q = e - (long long)C * L.S;
        const int row = (int)(q / L.P);
        const int s = (int)(q - (long long)row * L.P);
        const int j = row % L.n2;
        const int k = (row / L.n2) % L.n3;
        const int l = row / (L.n2 * L.n3);
        const int i = 2 * s + (C ^ ((j + k + l) & 1));
        if (i >= L.n1) continue;
        const int c[4] = {i, j, k, l};
        float wsum = 0.0f;
        for (int f = 0; f < 8; ++f) {
            const int d = f >> 1;
            const int nb = c[d] + ((f & 1) ? 1 : -1);
            const float w = (nb >= 0 && nb < nn[d]) ? ih2[d] : 0.0f;
            wsum += w;
            if (C == 0) W[(long long)f * L.S + q] = w;
        }
        const float D = 1.0f + sigma_t * wsum;
        const float b = I[C * L.S + q];
        diag[C * L.S + q] = D;
        beta[C * L.S + q] = b;
        gamma[C * L.S + q] = sigma_t / D;
        rec3f_add(a, __fmul_rn(b, b), b);
    }
    const Acc3 ad = rec3f_acc(a);
    double ssum = ad.sum, mn = ad.mn, mx = ad.mx;
    // block reduction of (sum, min, max)
    for (int o = 16; o > 0; o >>= 1) {
        ssum += __shfl_down_sync(0xffffffffu, ssum, o);
        mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    __shared__ double sh[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = ssum;
        sh[1][wid] = mn;
        sh[2][wid] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            ssum += sh[0][w];
            mn = fmin(mn, sh[1][w]);
            mx = fmax(mx, sh[2][w]);
        }
        partials[3 * blockIdx.x + 0] = ssum;
        partials[3 * blockIdx.x + 1] = mn;
        partials[3 * blockIdx.x + 2] = mx;
    }
}

void launch_smooth_coef(const Layout &L, const float *I, const double *h, double sigma_t,
                        float *beta, float *gamma, float *diag, float *W, double *partials,
                        int nparts, cudaStream_t st)
{
    float4 ih2 = make_float4((float)(1.0 / (h[0] * h[0])), (float)(1.0 / (h[1] * h[1])),
                             (float)(1.0 / (h[2] * h[2])), (float)(1.0 / (h[3] * h[3])));
    k_smooth_coef<<<nparts, kPartThreads, 0, st>>>(L, I, ih2, (float)sigma_t, beta, gamma, diag, W,
                                                   partials);
}

}  // namespace seg4d_impl
