/*
 * seg4d.h -- C ABI of libseg4d, a single-GPU NVIDIA GB300 (sm_103a)
 * implementation of the semi-implicit finite-volume scheme for the 4D
 * generalized subjective-surface (GSUBSURF) segmentation of Uba, Mikula and
 * Park, "4D Segmentation Algorithm with application to 3D+time Image
 * Segmentation" (arXiv 2111.11866).
 *
 * Model (Section 3.1, Eq. first): u_t = |grad u| div(G0 grad u / |grad u|)
 * on a 3D+time grid with zero Dirichlet data, G0 = g(delta |grad I_sigma^0| +
 * vartheta |grad I_sigma^TH|), g(s) = 1/(1 + K s^2) (Eq. eg1).  Each time step
 * solves the linear system of Eq. new1 (Eq. new for equal h) built with the
 * reduced diamond-cell gradients of Section 3.2 and the coefficients of
 * Eq. 111th, by red-black SOR (Eqs. 5.33, gsee and the red-black ordering of
 * Section 3.7), and then rescales u locally (Remark, Eq. 841).
 *
 * Conventions shared by every entry point:
 *  - Arrays are 4D, x fastest: index ((l*n3 + k)*n2 + j)*n1 + i for 0-based
 *    interior voxel (i, j, k, l); l is the frame (time) axis.  This is the
 *    4D->1D map of Section 3.7 without the ghost ring.
 *  - The caller owns every pointer it passes.  The library copies on set and
 *    on read and keeps no caller pointer.  `on_device` = 1 means the pointer is
 *    device memory of the current CUDA device, 0 means host memory.
 *  - Every call enqueues its work on the stream given to seg4d_create and
 *    returns after that work has finished (the library synchronises the stream
 *    where it needs a device value on the host, e.g. for the stopping test).
 *  - Calls return a seg4d_status.  They never abort and never wait without a
 *    bound.  After an error, seg4d_last_error() describes it.  A handle is
 *    not thread safe: one host thread at a time per handle.
 */
#ifndef SEG4D_H
#define SEG4D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct seg4d seg4d;

typedef enum {
    SEG4D_OK = 0,
    SEG4D_ERR_INVALID = -1,       /* bad argument: sizes, NaN/Inf parameters, NULL */
    SEG4D_ERR_OOM = -2,           /* device allocation failed                       */
    SEG4D_ERR_STATE = -3,         /* call out of order (e.g. step before set_image) */
    SEG4D_ERR_NOT_CONVERGED = -4, /* a solve reached max_iters; u holds the last
                                     iterate and the info struct is filled          */
    SEG4D_ERR_CUDA = -5,          /* a CUDA call failed                             */
    SEG4D_ERR_TIMEOUT = -6        /* a bounded device wait ran out (no kernel of
                                     this version waits on another)              */
} seg4d_status;

/* interior grid sizes; n4 = number of frames */
typedef struct {
    int n1, n2, n3, n4;
} seg4d_dims;

/* Parameters.  seg4d_default_params() fills the values used throughout
 * Section 4 of the paper (delta = vartheta = 0.5, h = 0.01, tau = 0.01,
 * eps = 1, sigma = h^2/8, R = 12, lambda = 0.87) plus the readings for the
 * values the paper does not give (K = 1, v = 1, omega = 1.6 raised at run time
 * by omega_adapt, the stopping
 * rule below). */
typedef struct {
    double h[4];        /* voxel sizes h1..h4 (Eq. new1)                            */
    double tau;         /* segmentation time step                                   */
    double eps;         /* Evans-Spruck regularisation epsilon (Eq. 3rd)            */
    double K;           /* Perona-Malik g(s) = 1/(1 + K s^2) (Eq. eg1)              */
    double delta;       /* weight of the presmoothed original image (Eq. first)     */
    double vartheta;    /* weight of the presmoothed thresholded image (Eq. first)  */
    double lambda_th;   /* TH = lambda*min + (1-lambda)*max over a ball (Sec. 3.1)  */
    double r_ball;      /* radius (voxels) of the thresholding and rescaling balls  */
    double R_init;      /* radius (voxels) of the initial peak (Eq. initialcond)    */
    double v_init;      /* 1/v is the peak height of u0 (Eq. initialcond)           */
    double sigma_t;     /* presmoothing: one implicit heat step of this length      */
    double omega;       /* SOR relaxation of the step solves (Eq. 5.33); with
                           omega_adapt, the value each solve starts from        */
    double omega_smooth;/* SOR relaxation of the presmoothing solves                */
    double tol;         /* stop when ||b - A u||_2 <= tol ||b||_2 (step solves; see
                           also tol_inf)                                        */
    double tol_smooth;  /* the same for the presmoothing solves                     */
    int max_iters;      /* sweep cap per solve (SEG4D_ERR_NOT_CONVERGED beyond)     */
    int check_every;    /* sweeps before the first re-evaluation of the stopping
                           test; later gaps are predicted from the observed
                           residual decay, within [max(1, check_every/4),
                           8*check_every]                                           */
    int precision;      /* 0: FP32 throughout.  1: mixed -- the sweeps stream BF16
                           face weights (a BF16 system with its own consistent
                           diagonal) and every check is an exact FP32 defect
                           pass r = b - A u; the sweeps solve A_b delta = r and
                           u += delta, so the fixed point is the FP32 system's.
                           Presmoothing solves are always FP32.                    */
    int sweep_variant;  /* one launch per colour of each red-black sweep.  1
                           (default): the FP32 solve also keeps its scaled face
                           weights by black end (16 B/voxel more), so the black
                           pass reads them at its own slots as the red pass
                           does; 2: the black pass reads them across the faces
                           (less memory).  Both give identical bits; the lean
                           handle always works as 2                           */
    int ctas_per_sm;    /* reserved, must be 0                                   */
    int wait_test;      /* reserved, must be 0                                   */
    double tol_inf;     /* per-voxel part of the stopping test of the step solves:
                           with tol_inf > 0 a solve also needs
                           max |b - A u| <= tol_inf max |b|.  The step matrix is
                           an M-matrix with ||A^-1||_inf <= 1 (Theorem, Section
                           3.3), so every voxel is then within tol_inf max |b|
                           of the exact solve.  0 disables it; the default is
                           1e-5 (the FP32 floor of max |r| on the measured
                           workloads lies between 2e-6 and 5e-6 of max |b|)  */
    int omega_adapt;    /* 1: the step solves choose their SOR relaxation at run
                           time (Young's relation for the consistently ordered
                           red-black matrix: the contraction observed at omega
                           gives the Jacobi radius mu and the best relaxation
                           2 / (1 + sqrt(1 - mu^2))); each solve starts at
                           omega and only raises it.  0: omega is used as is  */
} seg4d_params;

/* a segmentation seed: centre c_m (voxel units, 0-based) inside frame `frame` */
typedef struct {
    double x, y, z;
    int frame;
    int reserved;
} seg4d_seed;

/* results of the last solve of a call */
typedef struct {
    int iters;              /* red-black sweeps of the last solve                    */
    int status;             /* seg4d_status of the last solve                        */
    double res_l2;          /* ||b - A u||_2 of the returned iterate                 */
    double res_rel;         /* res_l2 / ||b||_2                                      */
    double bnorm;           /* ||b||_2                                               */
    double umin, umax;      /* min / max of the solved u (before rescaling)          */
    long long sweeps_total; /* sweeps of every solve of the call (setup included)    */
    int steps_done;         /* time steps completed by the call                      */
    float ms;               /* device time of the call's work, milliseconds          */
    double sweep_ms;        /* device time spent in red-black sweeps (CUDA events on
                               the handle's stream around each batch of sweeps)      */
    long long launches;     /* kernels the call launched                             */
    long long sweep_launches; /* of which sweep kernels (timed by sweep_ms)          */
    double res_inf;         /* max |b - A u| of the returned iterate (last solve)    */
    double bmax;            /* max |b| of the last solve                             */
} seg4d_info;

/* fields readable with seg4d_read_field; G and OFF give 8 values per voxel,
 * face f = 2*d + (side > 0) for axis d = x1..x4, as array [voxel][8]. */
enum {
    SEG4D_FIELD_U = 0,        /* segmentation function u                          */
    SEG4D_FIELD_I0 = 1,       /* the image as set                                 */
    SEG4D_FIELD_ITH = 2,      /* locally thresholded image I^TH (Section 3.1)      */
    SEG4D_FIELD_ISIG0 = 3,    /* presmoothed I0                                    */
    SEG4D_FIELD_ISIGTH = 4,   /* presmoothed I^TH                                  */
    SEG4D_FIELD_G = 5,        /* face edge coefficients G_f (Eq. 10th), 8/voxel    */
    SEG4D_FIELD_OWNER = 6,    /* index of the seed ball a voxel follows, or -1     */
    SEG4D_FIELD_DIAG = 7,     /* diagonal of the current step system (Eq. new1)    */
    SEG4D_FIELD_OFF = 8       /* off-diagonal magnitudes tau*Abar*G_f/(A_f h_d^2)
                                 of the current system, 8/voxel; faces to the
                                 Dirichlet boundary read as 0                      */
};

/* Fill *p with the defaults described above. */
void seg4d_default_params(seg4d_params *p);

/* Allocate a handle and every device buffer for a grid of `dims` voxels on the
 * current CUDA device.  `cuda_stream` is a cudaStream_t (NULL = the legacy
 * default stream).  All n_d >= 1 and n1*n2*n3*n4 < 2^33.
 * Errors: INVALID (sizes), OOM, CUDA. */
seg4d_status seg4d_create(const seg4d_dims *dims, void *cuda_stream, seg4d **out);

/* seg4d_create with flags.  SEG4D_CREATE_LEAN: 64 instead of about 120 bytes
 * per voxel, for the largest grids (the paper's 567x577x147x70 zebrafish
 * stack, Section 4, needs 216 GB this way, 258 GB in mixed precision).  The image fields are kept inside the
 * G array until the set-up has used them (they cannot be read back after
 * it, and new seeds need set_image again; u serves as scratch during the
 * set-up, which therefore re-initialises it from the seeds); the FP32 solve
 * sweeps its
 * correction system unscaled (c/D streamed instead of stored scaled
 * weights: about 8 % slower per sweep).  Errors as seg4d_create, and INVALID
 * for unknown flags. */
enum { SEG4D_CREATE_LEAN = 1 };
seg4d_status seg4d_create_ex(const seg4d_dims *dims, void *cuda_stream, int flags, seg4d **out);

/* Free the handle and its device memory.  NULL is accepted. */
seg4d_status seg4d_destroy(seg4d *h);

/* Copy the parameters.  Errors: INVALID (non-finite or out of range:
 * h, tau, eps > 0; K >= 0; delta, vartheta, lambda in [0,1]; radii > 0;
 * 0 < omega, omega_smooth < 2; tol, tol_smooth > 0; tol_inf >= 0; omega_adapt 0 or 1;
 * max_iters >= 1;
 * check_every >= 1; precision 0). */
seg4d_status seg4d_set_params(seg4d *h, const seg4d_params *p);

/* Copy the 4D image I0 (n = n1*n2*n3*n4 floats).  Marks the image-derived
 * set-up (thresholding, presmoothing, G) for recomputation.
 * Errors: INVALID (n mismatch, NULL, non-finite values -- checked on the
 * device after the copy, so the handle then has no image until the next
 * successful call), CUDA. */
seg4d_status seg4d_set_image(seg4d *h, const float *I0, size_t n, int on_device);

/* Copy the seeds (Section 3.1, the centres C_theta).  Marks the set-up for
 * recomputation and u for re-initialisation from u0 (Eq. initialcond)
 * followed by a local rescale.  nseeds >= 0; a seed whose frame is outside
 * 0..n4-1 has an empty ball.  Errors: INVALID (NaN coordinates), OOM. */
seg4d_status seg4d_set_seed(seg4d *h, const seg4d_seed *seeds, int nseeds);

/* Overwrite u (checkpoint / resume, or a chosen initial guess); cancels a
 * pending re-initialisation from the seeds.  Errors: INVALID, CUDA. */
seg4d_status seg4d_set_u(seg4d *h, const float *u, size_t n, int on_device);

/* Dirichlet data on the ghost ring (Section 3.4, where the exact solution is
 * prescribed on the ghost cells of the padded grid; zero is the default, the
 * u^D = 0 of the segmentation runs).  The ring is given as its 8 face slabs:
 * slab (d, side) holds the values at padded index 0 (side 0) or n_d + 1
 * (side 1) along axis d (0 = x .. 3 = frame) for every padded position
 * 0..n_e+1 of the other three axes, x fastest; the slabs follow each other in
 * the order (0,0) (0,1) (1,0) (1,1) ... (3,1), and edges and corners repeat
 * in several slabs with the same value.  g_prev is the data at t_{n-1}, which
 * the face gradients of the coefficients see; g_now is the data at t_n, whose
 * columns go to the right-hand side of the solve.  Both are copied (n =
 * seg4d_dirichlet_count(dims) floats each) and used by every following
 * solve / step until replaced; both NULL returns to zero data.
 * Errors: INVALID (one NULL, n mismatch), OOM, CUDA. */
size_t seg4d_dirichlet_count(const seg4d_dims *dims);
seg4d_status seg4d_set_dirichlet(seg4d *h, const float *g_prev, const float *g_now, size_t n,
                                 int on_device);

/* Run the pending set-up now: thresholding, both presmoothing solves, face
 * coefficients G and, if pending, u0 and its rescale.  solve and step call it
 * themselves.  Errors: STATE (no image), NOT_CONVERGED (a presmoothing solve
 * hit max_iters), CUDA. */
seg4d_status seg4d_setup(seg4d *h, seg4d_info *info);

/* One linear solve without rescaling: build the coefficients of Eq. new1 from
 * the current u (= u^{resc,n-1}, also the right-hand side and the initial
 * guess) and iterate red-black SOR until the stopping rule holds.
 * Errors: STATE, NOT_CONVERGED, CUDA.  info may be NULL. */
seg4d_status seg4d_solve(seg4d *h, seg4d_info *info);

/* nsteps time steps, each {coefficients, solve, local rescale} (Section 3.6).
 * Stops at the first failing solve (u holds its last iterate).
 * Errors: INVALID (nsteps < 0), STATE, NOT_CONVERGED, CUDA. */
seg4d_status seg4d_step(seg4d *h, int nsteps, seg4d_info *info);

/* Copy u out (n floats).  Errors: INVALID, CUDA. */
seg4d_status seg4d_read_u(seg4d *h, float *dst, size_t n, int on_device);

/* Copy a field out: n = n1*n2*n3*n4 floats, or 8 times that for G and OFF.
 * Errors: INVALID (unknown field, n mismatch), STATE (field not computed yet),
 * CUDA. */
seg4d_status seg4d_read_field(seg4d *h, int field, float *dst, size_t n, int on_device);

/* Bytes of device memory a handle of these sizes allocates (_ex: with the
 * creation flags).  Mixed precision adds 12 bytes per voxel at its first
 * solve. */
size_t seg4d_device_bytes(const seg4d_dims *dims);
size_t seg4d_device_bytes_ex(const seg4d_dims *dims, int flags);

/* Message of the last error on this handle ("" if none); valid until the next
 * call on the handle.  h == NULL gives the message of the last failed
 * handle-free call of the calling thread (seg4d_create,
 * seg4d_residual_norms_noalloc). */
const char *seg4d_last_error(const seg4d *h);

/* Residual norms of a step system that lives entirely in the caller's device
 * memory, computed without allocating anything.  The paper has no counterpart:
 * this is a service for callers that cannot call cudaMalloc -- for example
 * code that hands all device memory to its own pooled allocator or fixed
 * budget (a serving loop that admits work by HBM budget), or that must not
 * take the device-wide synchronisation cudaMalloc/cudaFree can imply while
 * other work is in flight.  Such callers can still check a solve.
 *
 * Inputs (device pointers, x-fastest arrays of n = n1*n2*n3*n4 voxels): u, b,
 * diag (n floats each) and off (8n floats: for every voxel the magnitudes of
 * its 8 off-diagonal entries, face f = 2*d + (side > 0), exactly as
 * seg4d_read_field returns SEG4D_FIELD_DIAG and SEG4D_FIELD_OFF).  Faces whose
 * neighbour lies outside the grid are ignored (zero Dirichlet data).
 * Output: result[0] = ||b - A u||_2 and result[1] = ||b||_2, two doubles in
 * device memory, written on `cuda_stream`; the call returns after enqueueing.
 *
 * Scratch: per-block FP64 records in a fixed 256 KiB device array compiled
 * into the library, which every device that loads the library holds until the
 * process exits.  Grids with n2*n3*n4 > 4,194,304 x-lines (or n >= 2^33) are
 * rejected with SEG4D_ERR_INVALID.  Every call shares that array and leaves its
 * records there; each call writes all records it reads, so nothing needs
 * clearing, but calls that overlap on the GPU (other streams or host threads)
 * race on it.  The first call on a device looks up the array's device address
 * with that device current (cudaGetSymbolAddress); make that first call before
 * any stream capture.  A failed lookup is reported (SEG4D_ERR_CUDA) and tried
 * again by the next call.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  Errors: INVALID (dims, NULL, too large), CUDA; message via
 * seg4d_last_error(NULL). */
seg4d_status seg4d_residual_norms_noalloc(const seg4d_dims *dims, const float *u, const float *b,
                                          const float *diag, const float *off, double *result,
                                          void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batched windows.  Many independent problems (e.g. one window around each
 * nucleus, the windows of Section 4's third and fourth experiments) advanced
 * together: every hot kernel launch covers all active windows.  Each window
 * runs exactly the scheme above -- set-up, then per step coefficients, red-
 * black SOR to its own stopping rule, local rescale.  The solves run in
 * rounds of 4 sweeps.  Each window's checks, its check spacing (rounded up to
 * whole rounds) and its run-time SOR relaxation are decided on the device
 * from its own residuals, so its iterates do not depend on which other
 * windows share the batch.  max_iters is honoured to the round.
 * ------------------------------------------------------------------------ */

typedef struct seg4d_batch seg4d_batch;

/* what one seg4d_batch_advance call did */
typedef struct {
    int setup_windows;      /* windows whose set-up ran                           */
    int stepped_windows;    /* windows advanced by one time step                  */
    int active_windows;     /* windows still stepping after the call (pending incl.) */
    int done_windows;       /* windows that completed their nsteps                */
    int failed_windows;     /* windows whose solve failed (NOT_CONVERGED / NaN)    */
    int status;             /* seg4d_status of the call                           */
    long long window_sweeps;/* sum over windows of the red-black sweeps run      */
    long long launches;     /* kernels launched                                   */
    long long arena_used;   /* bytes of the arena in use                          */
    float ms;               /* device time of the call                            */
    float pad;
    double sweep_ms;        /* device time of the batched sweeps                  */
} seg4d_batch_info;

/* state of one window: 0 pending set-up, 1 active, 2 done, 3 failed */
typedef struct {
    int state, steps_done, nsteps, last_iters;
    long long sweeps;       /* red-black sweeps of its step solves so far          */
    long long device_bytes; /* arena bytes it holds                                */
    double last_res_rel;    /* ||b - A u|| / ||b|| at the end of its last solve     */
} seg4d_window_info;

/* Create a batch with a device arena of `arena_bytes` (allocated now) for at
 * most `max_windows` windows; work goes to `cuda_stream`.  Parameters start as
 * seg4d_default_params().  Errors: INVALID, OOM (message via
 * seg4d_batch_last_error(NULL)). */
seg4d_status seg4d_batch_create(size_t arena_bytes, int max_windows, void *cuda_stream,
                                seg4d_batch **out);
seg4d_status seg4d_batch_destroy(seg4d_batch *b);

/* Parameters shared by every window (validated as for seg4d_set_params); they
 * apply to work done after the call. */
seg4d_status seg4d_batch_set_params(seg4d_batch *b, const seg4d_params *p);

/* Admit a window: its dims, image (copied; x fastest, host or device) and
 * seeds (copied), and the number of time steps to run.  The window takes
 * seg4d_batch_window_bytes(dims, nseeds) bytes of the arena (the image part
 * is returned after its set-up).  SEG4D_ERR_OOM when the arena has no room:
 * admission control by device-memory budget -- retry after windows are
 * removed.  *id_out identifies the window.  Errors: INVALID, OOM, CUDA. */
seg4d_status seg4d_batch_add(seg4d_batch *b, const seg4d_dims *dims, const float *image,
                             int on_device, const seg4d_seed *seeds, int nseeds, int nsteps,
                             int *id_out);

/* One engine iteration: set-up of every window admitted since the last call
 * (thresholding, presmoothing, G, u0 + rescale; Section 3.6), then one time
 * step for every active window.  A window whose solve fails is marked failed
 * and the others go on.  Errors: CUDA (the batch is then not usable). */
seg4d_status seg4d_batch_advance(seg4d_batch *b, seg4d_batch_info *info);

/* State of window `id`.  Errors: INVALID (unknown id). */
seg4d_status seg4d_batch_poll(seg4d_batch *b, int id, seg4d_window_info *info);

/* Copy window `id`'s u out (n = its n1*n2*n3*n4 floats, x fastest).
 * Errors: INVALID, STATE (set-up not run yet), CUDA. */
seg4d_status seg4d_batch_read_u(seg4d_batch *b, int id, float *dst, size_t n, int on_device);

/* Retire window `id` and return its arena space.  Errors: INVALID. */
seg4d_status seg4d_batch_remove(seg4d_batch *b, int id);

/* Arena bytes a window of these sizes needs at admission in a batch of the
 * given precision (seg4d_params.precision). */
size_t seg4d_batch_window_bytes(const seg4d_dims *dims, int nseeds, int precision);

/* Message of the last error of the batch (NULL: of the last failed create). */
const char *seg4d_batch_last_error(const seg4d_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* SEG4D_H */
