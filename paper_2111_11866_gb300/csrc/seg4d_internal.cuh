// seg4d_internal.cuh -- device data layout and kernel launchers of libseg4d.
//
// Layout ("colour-split rows").  The red-black ordering of Section 3.7 colours
// voxel (i,j,k,l) red when i+j+k+l is even.  Every array that a sweep touches
// is stored as two half arrays, red then black.  Row r = j + n2*(k + n3*l)
// holds the voxels of one x-line; inside a row the voxels of one colour are
// compacted along x: voxel i sits in slot i >> 1 of its colour.  A row has
// P = roundup(ceil(n1/2), 4) slots per colour; unused slots are padding that
// always holds zero.  Consequences used by the kernels:
//   - with p = (j+k+l) & 1, the red voxel of slot s is i = 2s + p and the
//     black one is i = 2s + 1 - p;
//   - the x-neighbours of red slot s are black slots s-1+p and s+p, those of
//     black slot s are red slots s-p and s+1-p; the y/z/t neighbours of any
//     slot are the other colour's same slot in rows r -+ 1, r -+ n2, r -+ n2*n3.
// So a half sweep reads each array with unit stride (coalesced) and no lane
// loads a value of its own colour except its own voxel.
//
// Face weights of the step system are stored once per face, by the face's red
// end: every face joins one red and one black voxel, so W[f][red slot] for the
// 8 faces f of every red voxel covers each interior face exactly once.  Faces
// to the Dirichlet ghost ring are only needed on the diagonal, which the
// coefficient kernel folds into D.
#pragma once

#include <cmath>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

namespace seg4d_impl {

struct Layout {
    int n1, n2, n3, n4;
    int P;          // slots per colour per row
    int nchunk;     // ceil(P / 32): 32-slot chunks per row
    int njb;        // ceil(n2 / 8): 8-row blocks along y
    int R;          // rows = n2*n3*n4
    long long S;    // slots per colour = R*P
    int kt;         // z-planes per tile of the plane traversal order
    int ntile;      // ceil(n3 / kt)
};

// Traversal order of the (k, l) planes in the stencil kernels: tiles of kt
// consecutive z-planes, l-major inside a tile (plane index c = tile n4 + l,
// then k = tile kt + kin, kin fastest), so that the t-neighbour planes of a
// plane are visited kt planes apart rather than n3 apart.  With kt chosen so
// that 2 kt planes of sweep traffic stay well inside L2, values read through
// the +-t faces are L2 hits on large grids too.  kt = n3 is the plain order
// (k fastest, then l).  Plane slots with k >= n3 (the last tile) are holes.
//
// kt for a grid: about 64 MB of sweep traffic (48 B per slot and colour)
// over 2 kt planes; grids whose frame-to-frame distance already fits keep
// kt = n3.  ntile n4 stays within a grid dimension (65535).  On 512x512x128
// planes, 38, 64 and 102 MB (kt = 3, 5, 8) swept within 0.5 % of each other.
#ifndef SEG4D_PLANE_TILE_BYTES
#define SEG4D_PLANE_TILE_BYTES 64.0e6
#endif
inline int plane_tile(int n2, int n3, int n4, int P)
{
    const double plane = 96.0 * (double)n2 * (double)P;
    int kt = (int)(SEG4D_PLANE_TILE_BYTES / plane);
    if (kt < 1) kt = 1;
    if (2 * kt >= n3) kt = n3;
    while (kt < n3 && (long long)((n3 + kt - 1) / kt) * n4 > 65535) ++kt;
    return kt;
}

// Face edge coefficients G are stored once per face, by the face's red end,
// as W is: G[f][S] for the 8 faces f of every red voxel (faces to the
// Dirichlet ring included).  A black voxel's faces to the ring have no red
// end; their G follow the planes in a side table (offsets from G + 8 S):
//   x: per row, [row][side] (i = 0 and i = n1-1);
//   y: rows j = 0 and j = n2-1, [side][k + n3 l][slot];
//   z: rows k = 0 and k = n3-1, [side][j + n2 l][slot];
//   t: rows l = 0 and l = n4-1, [side][j + n2 k][slot].
struct GbOff {
    long long x, y, z, t, total;
};

__host__ __device__ inline GbOff gb_offsets(const Layout &L)
{
    GbOff o;
    o.x = 0;
    o.y = 2LL * L.R;
    o.z = o.y + 2LL * L.n3 * L.n4 * L.P;
    o.t = o.z + 2LL * L.n2 * L.n4 * L.P;
    o.total = o.t + 2LL * L.n2 * L.n3 * L.P;
    return o;
}

// floats of the G array: the 8 planes and the side table
__host__ __device__ inline long long g_floats(const Layout &L)
{
    return 8LL * L.S + gb_offsets(L).total;
}

// side-table index of face f (to the ring) of the black voxel in slot s of
// row `row` at (j, k, l)
__host__ __device__ inline long long gb_index(const Layout &L, const GbOff &o, int f, int row,
                                              int s, int j, int k, int l)
{
    const int side = f & 1;
    switch (f >> 1) {
    case 0: return o.x + 2LL * row + side;
    case 1: return o.y + ((long long)side * L.n3 * L.n4 + k + (long long)L.n3 * l) * L.P + s;
    case 2: return o.z + ((long long)side * L.n2 * L.n4 + j + (long long)L.n2 * l) * L.P + s;
    default: return o.t + ((long long)side * L.n2 * L.n3 + j + (long long)L.n2 * k) * L.P + s;
    }
}

// Voxel coordinates -> colour and slot (caller guarantees the voxel exists).
__host__ __device__ inline long long slot_of(const Layout &L, int i, int j, int k, int l,
                                             int &colour)
{
    int row = j + L.n2 * (k + L.n3 * l);
    colour = (i + j + k + l) & 1;
    return (long long)row * L.P + (i >> 1);
}

__device__ inline int clampi(int a, int n) { return a < 0 ? 0 : (a >= n ? n - 1 : a); }

// image read with replicated ghosts (zero Neumann data for images).
__device__ inline float ld_replicate(const Layout &L, const float *__restrict__ a, int i, int j,
                                     int k, int l)
{
    i = clampi(i, L.n1);
    j = clampi(j, L.n2);
    k = clampi(k, L.n3);
    l = clampi(l, L.n4);
    int c;
    long long s = slot_of(L, i, j, k, l, c);
    return a[c * L.S + s];
}

// owner value of a voxel outside every ball (memset byte pattern 0x7F); larger
// than any seed index, so atomicMin picks real owners over it
constexpr int kOwnerNone = 0x7F7F7F7F;

struct SeedDev {
    double x, y, z;
    int frame;
    int bx0, bx1, by0, by1, bz0, bz1;   // bounding box of the ball, clipped to the grid
};

// Per-seed scalars produced on the device.
struct SeedStat {
    float mn, mx;     // min / max of a field over the ball
    int count;        // voxels in the ball (0 = empty ball)
    int pad;
};

// Dirichlet data on the ghost ring of the padded grid (indices -1 and n_d
// along an axis), as the 8 face slabs of that ring: slab (d, side) holds the
// values at padding index a_d = 0 (side 0) or n_d + 1 (side 1) for every
// padded position of the other three axes (0..n_e+1, x fastest), slabs in the
// order (0,0) (0,1) (1,0) ... (3,1).  Edges and corners of the ring lie in
// several slabs; the one of the first axis out of range is read.  `prev` is
// the data the coefficients see, `now` the data of the solve.
struct Ghost {
    const float *prev, *now;
    long long off[4];   // offset of slab (d, 0); slab (d, 1) follows it
    long long size[4];  // values per slab of axis d
    int np[4];          // padded extents n_d + 2
};

// ---------------------------------------------------------------- launchers
// set-up (setup_kernels.cu)
// bad (nullable): a device flag set to 1 when an input value is not finite
void launch_split_from_natural(const Layout &L, const float *nat, float *split, unsigned *bad,
                               cudaStream_t st);
void launch_natural_from_split(const Layout &L, const float *split, float *nat, cudaStream_t st);
// G ([8][S] planes by red end + side table) -> [voxel][8], x fastest
void launch_G_natural(const Layout &L, const float *G, float *nat8, cudaStream_t st);
void launch_owner_natural(const Layout &L, const int *owner, float *nat, cudaStream_t st);
void launch_off_natural(const Layout &L, const float *W, const float *gamma, const float *diag,
                        float *nat8, cudaStream_t st);
void launch_owner(const Layout &L, const SeedDev *seeds, int nseeds, double r,
                  unsigned long long *dkey, int *owner, cudaStream_t st);
void launch_ball_minmax(const Layout &L, const SeedDev *seeds, int nseeds, double r,
                        const float *field, SeedStat *out, cudaStream_t st);
void launch_threshold_apply(const Layout &L, const SeedDev *seeds, int nseeds, double r,
                            double lambda, const SeedStat *stat, const int *owner,
                            const float *I0, float *ITH, cudaStream_t st);
void launch_init_u(const Layout &L, const SeedDev *seeds, int nseeds, double R, double v,
                   float *u, cudaStream_t st);
void launch_rescale_apply(const Layout &L, const SeedDev *seeds, int nseeds, double r,
                          const SeedStat *stat, const int *owner, float *u, cudaStream_t st);
void launch_face_G(const Layout &L, const float *Is0, const float *IsTH, const double *h,
                   double K, double delta, double vartheta, float *G, cudaStream_t st);
void launch_smooth_coef(const Layout &L, const float *I, const double *h, double sigma_t,
                        float *beta, float *gamma, float *diag, float *W, double *partials,
                        int nparts, cudaStream_t st);

// step and solve (solve_kernels.cu)
// returns the number of per-block records (sum b^2, min b, max b) written;
// ghost: Dirichlet data on the ghost ring (NULL: zero)
int launch_step_coef(const Layout &L, const float *u, const float *G, const double *h,
                     double tau, double eps, float *beta, float *gamma, float *diag, float *W,
                     double *partials, const Ghost *ghost, cudaStream_t st);
// gamma = NULL: a unit-diagonal (scaled) system, G = 1; Wblack (nullable): the
// weights by black end, read by the black pass at its own slots
void launch_sweep(const Layout &L, int colour, float *x, const float *beta, const float *gamma,
                  const float *W, float omega, cudaStream_t st, const float *Wblack = nullptr);
// mixed precision (mixed_kernels.cu); Wb is a __nv_bfloat16 [8][S] array
void launch_mixed_prepare(const Layout &L, const float *W, const float *gamma, const float *diag,
                          void *Wb, float *gb, float *ib, cudaStream_t st);
// returns the number of per-block records written to `partials`
// amax: per-block max |r| (one double per record)
int launch_defect(const Layout &L, const float *u, const float *b, const float *gamma,
                  const float *diag, const float *W, const float *ib, float *rho, float *delta,
                  double *partials, double *amax, cudaStream_t st);
// red-black SOR on the BF16 correction system A_b delta = r (solve_kernels.cu)
void launch_sweep_mixed(const Layout &L, int colour, float *delta, const float *rho,
                        const float *gb, const void *Wb, float omega, cudaStream_t st);
void launch_apply(const Layout &L, float *u, const float *delta, cudaStream_t st);
// FP32 solves (see k_scaled_weights): scaled correction weights, per-voxel
// r = sqrt(gamma) and 1 / (D r); and u <- u + r delta
// Wsb (nullable): also write the weights by black end
void launch_scaled_weights(const Layout &L, const float *W, float *Ws, float *Wsb,
                           const float *gamma, cudaStream_t st);
void launch_plain_prepare(const Layout &L, const float *gamma, const float *diag, float *rs,
                          float *ib, cudaStream_t st);
void launch_apply_scaled(const Layout &L, float *u, const float *delta, const float *rs,
                         cudaStream_t st);
// out[0..2] = (sum, min, max) of the records; with amax, out[3] = max of amax
void launch_reduce_partials(const double *partials, int nparts, double *out, cudaStream_t st,
                            const double *amax = nullptr);

// Sweeps until the next stopping test of a solve.  After two checks with
// r_now < r_prev, rho = (r_now/r_prev)^(1/sweeps) and need = log(tol*||b|| /
// r_now) / log(rho) sweeps remain.  SOR contracts faster as it proceeds, so
// need over-estimates: the next batch is 0.8 * need, and at most the sweeps
// that cut the residual by the factor `gain` at rate rho, so that rho is
// re-measured on the way.  A mixed-precision cycle cannot gain much more than
// the inverse of the BF16 weight error (about 2^9) before the correction
// system's own error dominates, so mixed cycles aim at 1e-2, plain batches at
// 1e-3.  Batches are kept in [max(1, check_every/4), 8*check_every]; without
// two usable checks the batch is check_every.  The result depends only on the
// solve's own residual history.
// (host and device: the batch engine decides its checks on the device)
__host__ __device__ inline int next_check_batch(double rn, double prev_rn, int it, int prev_it,
                                                double tol, double bnorm, int check_every,
                                                bool mixed)
{
    if (!(prev_rn > 0.0 && rn < prev_rn && it > prev_it && rn > 0.0)) return check_every;
    const double gain = mixed ? 1e-2 : 1e-3;
    const double rho = pow(rn / prev_rn, 1.0 / (it - prev_it));
    const double need = log(tol * bnorm / rn) / log(rho);
    const double cap = log(gain) / log(rho);
    const int lo = check_every / 4 > 1 ? check_every / 4 : 1, hi = 8 * check_every;
    const double want = ceil(fmin(0.8 * need, cap));
    return isfinite(want) ? (int)fmin((double)hi, fmax((double)lo, want)) : check_every;
}

// Run-time choice of the SOR relaxation (Eq. 5.33 leaves omega open).  The
// red-black ordering makes the step matrix consistently ordered, so Young's
// relation ties the spectral radius lam of the SOR iteration at relaxation
// omega to the Jacobi radius mu: (lam + omega - 1)^2 = lam omega^2 mu^2, and
// the best relaxation is omega_b = 2 / (1 + sqrt(1 - mu^2)).  Given the
// residual contraction per sweep lam observed at omega, this returns the
// estimate of omega_b when lam shows omega below it (lam > omega - 1; at or
// past omega_b, lam = omega - 1 and there is nothing to learn), never less
// than omega and at most 1.95.  Host and device use it (single grid and
// batched windows).
__host__ __device__ inline double sor_omega_update(double omega, double lam)
{
    if (!(lam > 0.0 && lam < 1.0) || lam <= omega - 1.0 + 0.02) return omega;
    const double a = lam + omega - 1.0;
    const double mu2 = a * a / (lam * omega * omega);
    if (!(mu2 < 1.0)) return omega;
    const double wb = 2.0 / (1.0 + sqrt(1.0 - mu2));
    return fmin(fmax(wb, omega), 1.95);
}

// Stopping decision at a check of a solve.  The test has two parts:
// ||r||_2 <= tol ||b||_2 and, with tol_inf > 0, max |r| <= tol_inf max |b|
// (a per-voxel bound, ||A^-1||_inf <= 1).  When the 2-norm part holds but the
// per-voxel part does not, and max |r| has stopped falling -- less than 1 %
// per sweep over at least check_every sweeps since the previous check --
// the iterate has reached the floor that FP32 rounding of u sets for max |r|
// (about D ulp(u) at a voxel), and the solve stops there (kStopFloor; the
// achieved max |r| is what the caller reports).  Otherwise `batch` is the
// number of sweeps to the next check: from the 2-norm history, or, once the
// 2-norm part holds, from the max |r| history.  Only the solve's own
// residual history enters.
struct CheckState {
    double prev_rn = -1.0, prev_inf = -1.0;
    int prev_it = 0;
};
enum { kGoOn = 0, kStop = 1, kStopFloor = 2 };
__host__ __device__ inline int check_decision(CheckState &cs, double rn, double bn, double rinf,
                                              double bmax, int it, double tol, double tol_inf,
                                              int check_every, bool mixed, int &batch)
{
    const bool l2 = rn <= tol * bn;
    const bool inf = tol_inf <= 0.0 || rinf <= tol_inf * bmax;
    int res = kGoOn;
    if (l2 && inf) {
        res = kStop;
    } else if (l2 && cs.prev_inf > 0.0 && it - cs.prev_it >= check_every) {
        const double rho = pow(rinf / cs.prev_inf, 1.0 / (it - cs.prev_it));
        if (!(rho < 0.99)) res = kStopFloor;
    }
    if (res == kGoOn) {
        if (l2) {
            batch = next_check_batch(rinf, cs.prev_inf, it, cs.prev_it, tol_inf, bmax,
                                     check_every, mixed);
        } else {
            batch = next_check_batch(rn, cs.prev_rn, it, cs.prev_it, tol, bn, check_every, mixed);
        }
    }
    cs.prev_rn = rn;
    cs.prev_inf = rinf;
    cs.prev_it = it;
    return res;
}

// message of the last failed handle-free call of this thread (api.cu)
std::string &handle_free_error();

// number of per-block partial records (3 doubles each: sum, min, max) the
// reduction kernels use; the scratch array holds 4 * kPartCap doubles: the
// records, then one max |r| per record of the defect pass.
constexpr int kPartBlocks = 1024;
constexpr int kPartThreads = 256;
// blocks (records) of the item loops of the coefficient, defect and scaling
// kernels: 2048 was the fastest of 912 ... 65536 in whole medium time steps
// (more blocks cost more than their tail saves); the scratch array holds
// 3 * max(kPartBlocks, kResBlocks) doubles
#ifndef SEG4D_RES_BLOCKS
#define SEG4D_RES_BLOCKS 2048
#endif
constexpr int kResBlocks = SEG4D_RES_BLOCKS;
constexpr int kPartCap = kResBlocks > kPartBlocks ? kResBlocks : kPartBlocks;

}  // namespace seg4d_impl
