/*
 * seg4d_oracle.c -- plain FP64 CPU oracle for the 4D generalized
 * subjective-surface (GSUBSURF) segmentation scheme of Uba, Mikula and Park,
 * "4D Segmentation Algorithm with application to 3D+time Image Segmentation"
 * (arXiv 2111.11866).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may build, load or call this file.
 * It shares no code, header, table or helper with the CUDA implementation.
 *
 * Style: slow, single-threaded and direct.  Every function follows the
 * formula it cites, in the paper's order and notation, so that it can be
 * checked against the paper by eye.  (A second library built from this file
 * with SEG4D_ORACLE_OMP splits the SOR sweeps' frame loop among OpenMP
 * threads, as the paper's OpenMP program does; it serves only as a timed CPU
 * baseline, and a test checks that it reaches the same solutions.)  All arithmetic is double precision; the
 * file is compiled with -ffp-contract=off so that x86 and Arm hosts give the
 * same bits.
 *
 * Grid (Section 3.7): interior voxels i=1..n1, j=1..n2, k=1..n3, l=1..n4 sit
 * inside a one-voxel ghost ring; the padded array is flattened x fastest,
 * T1D(i,j,k,l) = ((l*kMax + k)*jMax + j)*iMax + i with iMax = n1+2 etc.
 * Caller-visible arrays are compact interior arrays, x fastest, 0-based.
 *
 * Faces: f = 2*d + (s > 0), d = axis 0..3 (x1..x4), s = -1/+1 the side; this
 * enumerates the neighbour set N_ijkl of Section 3.2.
 *
 * Pins (tests/test_oracle_*.py): the EOC table (Table gridrefinementerr) for
 * the assembled scheme with G = 1; dense LU on tiny grids for the solver; the
 * exactness of the diamond gradient on quadratics; Neumann cosine eigenmodes
 * for presmoothing; the min-max principle (Theorem, Section 3.3); the two-level
 * image remark of Section 4 for thresholding; closed forms for u0 and rescale.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_NOT_CONVERGED 1
#define OR_ERR_ALLOC -2
#define OR_ERR_ARG -1

/* ------------------------------------------------------------------------ */
/* padded grid                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n[4];    /* interior sizes */
    long st[4];  /* strides of the padded array */
    long np;     /* padded element count */
    long nv;     /* interior element count */
} pgrid;

static int pg_init(pgrid *g, const int *dims)
{
    for (int d = 0; d < 4; ++d) {
        if (dims[d] < 1) return OR_ERR_ARG;
        g->n[d] = dims[d];
    }
    g->st[0] = 1;
    g->st[1] = (long)(dims[0] + 2);
    g->st[2] = g->st[1] * (long)(dims[1] + 2);
    g->st[3] = g->st[2] * (long)(dims[2] + 2);
    g->np = g->st[3] * (long)(dims[3] + 2);
    g->nv = (long)dims[0] * dims[1] * dims[2] * dims[3];
    return OR_OK;
}

/* padded index of the interior voxel with 0-based coordinates (i,j,k,l) */
static long pg_at(const pgrid *g, int i, int j, int k, int l)
{
    return (long)(i + 1) + (long)(j + 1) * g->st[1] + (long)(k + 1) * g->st[2] +
           (long)(l + 1) * g->st[3];
}

/* padded index from padded coordinates a[0..3] in 0..n+1 */
static long pg_atp(const pgrid *g, const int *a)
{
    return (long)a[0] + (long)a[1] * g->st[1] + (long)a[2] * g->st[2] + (long)a[3] * g->st[3];
}

static int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

/* Copy an interior array into a padded one whose ghost ring holds the value
 * `ghost` (zero Dirichlet data u^D = 0 of Eq. first11). */
static void pad_dirichlet(const pgrid *g, const double *in, double *out, double ghost)
{
    for (long p = 0; p < g->np; ++p) out[p] = ghost;
    long v = 0;
    for (int l = 0; l < g->n[3]; ++l)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) out[pg_at(g, i, j, k, l)] = in[v++];
}

/* Copy an interior image into a padded one whose ghost cells repeat the
 * nearest interior value (zero Neumann data for images, Eq. first2). */
static void pad_replicate(const pgrid *g, const double *in, double *out)
{
    int a[4];
    for (a[3] = 0; a[3] < g->n[3] + 2; ++a[3])
        for (a[2] = 0; a[2] < g->n[2] + 2; ++a[2])
            for (a[1] = 0; a[1] < g->n[1] + 2; ++a[1])
                for (a[0] = 0; a[0] < g->n[0] + 2; ++a[0]) {
                    int i = clampi(a[0] - 1, 0, g->n[0] - 1);
                    int j = clampi(a[1] - 1, 0, g->n[1] - 1);
                    int k = clampi(a[2] - 1, 0, g->n[2] - 1);
                    int l = clampi(a[3] - 1, 0, g->n[3] - 1);
                    long v = (((long)l * g->n[2] + k) * g->n[1] + j) * g->n[0] + i;
                    out[pg_atp(g, a)] = in[v];
                }
}

/* ------------------------------------------------------------------------ */
/* reduced diamond-cell face gradient (Section 3.2)                          */
/* ------------------------------------------------------------------------ */

/* |grad^{pqrs} v|^2 on face f of the voxel at padded index p.
 * The normal component is s (v_nb - v)/h_d; each tangential component t is
 * (v^{+t} - v^{-t})/h_t where v^{+-t} is the value at the diamond point
 * y^{pqrs}: the average of the four cells v, v_nb, v(+-e_t), v_nb(+-e_t). */
static double diamond_grad_sq(const pgrid *g, const double *v, long p, int f, const double *h)
{
    int d = f >> 1;
    long sd = (f & 1) ? g->st[d] : -g->st[d];
    double normal = (v[p + sd] - v[p]) / h[d];
    double sum = normal * normal;
    for (int t = 0; t < 4; ++t) {
        if (t == d) continue;
        long st = g->st[t];
        double y_plus = 0.25 * (v[p] + v[p + sd] + v[p + st] + v[p + sd + st]);
        double y_minus = 0.25 * (v[p] + v[p + sd] + v[p - st] + v[p + sd - st]);
        double comp = (y_plus - y_minus) / h[t];
        sum += comp * comp;
    }
    return sum;
}

/* Exported so that the tests can check the diamond gradient on its own:
 * g2[v*8 + f] = |grad^f u|^2 for the interior array u, with zero Dirichlet
 * ghosts (mode 0) or replicated ghosts (mode 1). */
int or_face_grad_sq(const int *dims, const double *u, const double *h, int mode, double *g2)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double *up = (double *)malloc(sizeof(double) * g.np);
    if (!up) return OR_ERR_ALLOC;
    if (mode == 0) pad_dirichlet(&g, u, up, 0.0);
    else pad_replicate(&g, u, up);
    long v = 0;
    for (int l = 0; l < g.n[3]; ++l)
        for (int k = 0; k < g.n[2]; ++k)
            for (int j = 0; j < g.n[1]; ++j)
                for (int i = 0; i < g.n[0]; ++i, ++v) {
                    long p = pg_at(&g, i, j, k, l);
                    for (int f = 0; f < 8; ++f) g2[v * 8 + f] = diamond_grad_sq(&g, up, p, f, h);
                }
    free(up);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* seeds, balls and their owners                                             */
/* ------------------------------------------------------------------------ */

/* squared spatial (3D) distance between interior voxel (i,j,k) and seed m */
static double seed_d2(const double *xyz, int m, int i, int j, int k)
{
    double dx = (double)i - xyz[3 * m + 0];
    double dy = (double)j - xyz[3 * m + 1];
    double dz = (double)k - xyz[3 * m + 2];
    double a = dx * dx;
    double b = dy * dy;
    double c = dz * dz;
    return (a + b) + c;
}

/* owner[v] = index of the nearest seed in the voxel's frame whose ball of
 * radius r contains the voxel (ties -> lowest index), or -1.  Balls
 * B(c_m, r) are spatial balls inside the seed's frame (Section 3.1). */
int or_owner(const int *dims, const double *xyz, const int *frame, int nseeds, double r, int *owner)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double r2 = r * r;
    long v = 0;
    for (int l = 0; l < g.n[3]; ++l)
        for (int k = 0; k < g.n[2]; ++k)
            for (int j = 0; j < g.n[1]; ++j)
                for (int i = 0; i < g.n[0]; ++i, ++v) {
                    int best = -1;
                    double bd = 0.0;
                    for (int m = 0; m < nseeds; ++m) {
                        if (frame[m] != l) continue;
                        double d2 = seed_d2(xyz, m, i, j, k);
                        if (d2 > r2) continue;
                        if (best < 0 || d2 < bd) { best = m; bd = d2; }
                    }
                    owner[v] = best;
                }
    return OR_OK;
}

/* min and max of a over the full ball B(c_m, r) of seed m */
static void ball_minmax(const pgrid *g, const double *a, const double *xyz, const int *frame, int m,
                        double r, double *mn, double *mx, int *count)
{
    double r2 = r * r;
    int l = frame[m];
    *count = 0;
    *mn = 0.0;
    *mx = 0.0;
    if (l < 0 || l >= g->n[3]) return;
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                if (seed_d2(xyz, m, i, j, k) > r2) continue;
                long v = (((long)l * g->n[2] + k) * g->n[1] + j) * g->n[0] + i;
                if (*count == 0 || a[v] < *mn) *mn = a[v];
                if (*count == 0 || a[v] > *mx) *mx = a[v];
                ++*count;
            }
}

/* ------------------------------------------------------------------------ */
/* local thresholding (Section 3.1)                                          */
/* ------------------------------------------------------------------------ */

/* alpha_m = min, beta_m = max of I0 over B(c_m, r); TH_m = lambda*alpha_m +
 * (1-lambda)*beta_m; inside the ball I^TH = beta_m where I0 >= TH_m, else
 * alpha_m.  A voxel inside several balls follows its owner; outside every
 * ball I^TH = I0. */
int or_threshold(const int *dims, const double *I0, const double *xyz, const int *frame, int nseeds,
                 double r, double lambda, double *ITH)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    int *owner = (int *)malloc(sizeof(int) * g.nv);
    double *alpha = (double *)malloc(sizeof(double) * (nseeds > 0 ? nseeds : 1));
    double *beta = (double *)malloc(sizeof(double) * (nseeds > 0 ? nseeds : 1));
    if (!owner || !alpha || !beta) { free(owner); free(alpha); free(beta); return OR_ERR_ALLOC; }
    or_owner(dims, xyz, frame, nseeds, r, owner);
    for (int m = 0; m < nseeds; ++m) {
        int cnt;
        ball_minmax(&g, I0, xyz, frame, m, r, &alpha[m], &beta[m], &cnt);
    }
    for (long v = 0; v < g.nv; ++v) {
        int m = owner[v];
        if (m < 0) { ITH[v] = I0[v]; continue; }
        double a = lambda * alpha[m];
        double b = (1.0 - lambda) * beta[m];
        double TH = a + b;
        ITH[v] = (I0[v] >= TH) ? beta[m] : alpha[m];
    }
    free(owner); free(alpha); free(beta);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* linear system: residual and SOR (Eqs. new, 5.33, gsee)                    */
/* ------------------------------------------------------------------------ */

/* Row v of the system:  diag[v]*u_v - sum_f off[v*8+f]*u_nb(f) = b_v, with
 * the neighbour value taken from the padded array (ghost = Dirichlet data).
 * off[] holds the positive coefficients; the matrix entries are -off. */

static double residual_norm_padded(const pgrid *g, const double *diag, const double *off,
                                   const double *b, const double *up)
{
    double s = 0.0;
    const long frame = (long)g->n[0] * g->n[1] * g->n[2];
#ifdef SEG4D_ORACLE_OMP
#pragma omp parallel for schedule(static) reduction(+ : s)
#endif
    for (int l = 0; l < g->n[3]; ++l) {
        long v = (long)l * frame;
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i, ++v) {
                    long p = pg_at(g, i, j, k, l);
                    double acc = b[v] - diag[v] * up[p];
                    for (int f = 0; f < 8; ++f) {
                        long sd = (f & 1) ? g->st[f >> 1] : -g->st[f >> 1];
                        acc += off[v * 8 + f] * up[p + sd];
                    }
                    s += acc * acc;
                }
    }
    return sqrt(s);
}

/* One relaxation (Eq. 5.33 with the Gauss-Seidel value of Eq. gsee) of the
 * interior voxel v at padded index p. */
static void relax_padded(const pgrid *g, const double *diag, const double *off, const double *b,
                         double *up, double omega, long v, long p)
{
    double acc = b[v];
    for (int f = 0; f < 8; ++f) {
        long sd = (f & 1) ? g->st[f >> 1] : -g->st[f >> 1];
        acc += off[v * 8 + f] * up[p + sd];
    }
    double ubar = acc / diag[v];
    up[p] = omega * ubar + (1.0 - omega) * up[p];
}

/* SOR in lexicographic order (Eq. 5.33 with the Gauss-Seidel value of
 * Eq. gsee): neighbours already visited in this sweep carry their new value.
 * Stops when ||b - A u||_2 <= tol * ||b||_2, tested before the first sweep and
 * then every check_every sweeps.
 *
 * Built with SEG4D_ORACLE_OMP (a separate library, used only as a timed CPU
 * baseline, never by the tests' pins), the sweep follows the paper's OpenMP
 * scheme instead: the frame loop is split among threads, and the RED-BLACK
 * ordering of Section 3.7 (red: even index sum) makes that split exact.  The
 * iterates differ from the lexicographic ones; the solution of the system is
 * the same. */
static int sor_padded(const pgrid *g, const double *diag, const double *off, const double *b,
                      double *up, double omega, double tol, int max_iters, int check_every,
                      int *iters, double *res_rel)
{
    double bn = 0.0;
    for (long v = 0; v < g->nv; ++v) bn += b[v] * b[v];
    bn = sqrt(bn);
    if (check_every < 1) check_every = 1;
    double rn = residual_norm_padded(g, diag, off, b, up);
    int it = 0;
    int status = OR_OK;
    if (!(rn <= tol * bn)) {
        status = OR_NOT_CONVERGED;
        for (it = 1; it <= max_iters; ++it) {
#ifdef SEG4D_ORACLE_OMP
            const long frame = (long)g->n[0] * g->n[1] * g->n[2];
            for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel for schedule(static)
                for (int l = 0; l < g->n[3]; ++l) {
                    long v = (long)l * frame;
                    for (int k = 0; k < g->n[2]; ++k)
                        for (int j = 0; j < g->n[1]; ++j)
                            for (int i = 0; i < g->n[0]; ++i, ++v)
                                if (((i + j + k + l) & 1) == colour)
                                    relax_padded(g, diag, off, b, up, omega, v,
                                                 pg_at(g, i, j, k, l));
                }
            }
#else
            long v = 0;
            for (int l = 0; l < g->n[3]; ++l)
                for (int k = 0; k < g->n[2]; ++k)
                    for (int j = 0; j < g->n[1]; ++j)
                        for (int i = 0; i < g->n[0]; ++i, ++v)
                            relax_padded(g, diag, off, b, up, omega, v, pg_at(g, i, j, k, l));
#endif
            if (it % check_every == 0 || it == max_iters) {
                rn = residual_norm_padded(g, diag, off, b, up);
                if (rn <= tol * bn) { status = OR_OK; break; }
            }
        }
        if (it > max_iters) it = max_iters;
    }
    if (iters) *iters = it;
    if (res_rel) *res_rel = bn > 0.0 ? rn / bn : rn;
    return status;
}

/* Threads the sweeps use: 1, or OpenMP's maximum in the SEG4D_ORACLE_OMP
 * build. */
#ifdef SEG4D_ORACLE_OMP
#include <omp.h>
int or_threads(void) { return omp_get_max_threads(); }
#else
int or_threads(void) { return 1; }
#endif

/* Solve diag/off system with zero Dirichlet ghosts; u holds the initial
 * guess on entry and the iterate on exit. */
int or_solve(const int *dims, const double *diag, const double *off, const double *b, double *u,
             double omega, double tol, int max_iters, int check_every, int *iters, double *res_rel)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double *up = (double *)malloc(sizeof(double) * g.np);
    if (!up) return OR_ERR_ALLOC;
    pad_dirichlet(&g, u, up, 0.0);
    int st = sor_padded(&g, diag, off, b, up, omega, tol, max_iters, check_every, iters, res_rel);
    long v = 0;
    for (int l = 0; l < g.n[3]; ++l)
        for (int k = 0; k < g.n[2]; ++k)
            for (int j = 0; j < g.n[1]; ++j)
                for (int i = 0; i < g.n[0]; ++i) u[v++] = up[pg_at(&g, i, j, k, l)];
    free(up);
    return st;
}

/* r = b - A u with zero Dirichlet ghosts */
int or_residual(const int *dims, const double *diag, const double *off, const double *b,
                const double *u, double *r)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double *up = (double *)malloc(sizeof(double) * g.np);
    if (!up) return OR_ERR_ALLOC;
    pad_dirichlet(&g, u, up, 0.0);
    long v = 0;
    for (int l = 0; l < g.n[3]; ++l)
        for (int k = 0; k < g.n[2]; ++k)
            for (int j = 0; j < g.n[1]; ++j)
                for (int i = 0; i < g.n[0]; ++i, ++v) {
                    long p = pg_at(&g, i, j, k, l);
                    double acc = b[v] - diag[v] * up[p];
                    for (int f = 0; f < 8; ++f) {
                        long sd = (f & 1) ? g.st[f >> 1] : -g.st[f >> 1];
                        acc += off[v * 8 + f] * up[p + sd];
                    }
                    r[v] = acc;
                }
    free(up);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* presmoothing: one implicit step of the linear heat equation (Section 3.1) */
/* ------------------------------------------------------------------------ */

/* The linear heat equation is the model with G = 1 (and no |grad u|
 * factors); one backward-Euler step of length sigma_t gives
 *   v + sum_{faces inside the grid} (sigma_t/h_d^2) (v - v_nb) = I,
 * with zero Neumann data (faces to ghost cells carry no flux). */
int or_presmooth(const int *dims, const double *I, const double *h, double sigma_t, double omega,
                 double tol, int max_iters, int check_every, double *out, int *iters, double *res_rel)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double *diag = (double *)malloc(sizeof(double) * g.nv);
    double *off = (double *)malloc(sizeof(double) * g.nv * 8);
    if (!diag || !off) { free(diag); free(off); return OR_ERR_ALLOC; }
    long v = 0;
    for (int l = 0; l < g.n[3]; ++l)
        for (int k = 0; k < g.n[2]; ++k)
            for (int j = 0; j < g.n[1]; ++j)
                for (int i = 0; i < g.n[0]; ++i, ++v) {
                    int c[4] = {i, j, k, l};
                    double dsum = 0.0;
                    for (int f = 0; f < 8; ++f) {
                        int d = f >> 1;
                        int nb = c[d] + ((f & 1) ? 1 : -1);
                        double a = 0.0;
                        if (nb >= 0 && nb < g.n[d]) a = sigma_t / (h[d] * h[d]);
                        off[v * 8 + f] = a;
                        dsum += a;
                    }
                    diag[v] = 1.0 + dsum;
                }
    for (v = 0; v < g.nv; ++v) out[v] = I[v];
    int st = or_solve(dims, diag, off, I, out, omega, tol, max_iters, check_every, iters, res_rel);
    free(diag); free(off);
    return st;
}

/* ------------------------------------------------------------------------ */
/* edge coefficients on faces (Eq. 10th with g of Eq. eg1)                   */
/* ------------------------------------------------------------------------ */

/* G[v*8+f] = g(delta |grad^f Isig0| + vartheta |grad^f IsigTH|), g(s) =
 * 1/(1 + K s^2); image ghosts repeat the edge (Neumann). */
int or_face_G(const int *dims, const double *Is0, const double *IsTH, const double *h, double K,
              double delta, double vartheta, double *G)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double *p0 = (double *)malloc(sizeof(double) * g.np);
    double *p1 = (double *)malloc(sizeof(double) * g.np);
    if (!p0 || !p1) { free(p0); free(p1); return OR_ERR_ALLOC; }
    pad_replicate(&g, Is0, p0);
    pad_replicate(&g, IsTH, p1);
    long v = 0;
    for (int l = 0; l < g.n[3]; ++l)
        for (int k = 0; k < g.n[2]; ++k)
            for (int j = 0; j < g.n[1]; ++j)
                for (int i = 0; i < g.n[0]; ++i, ++v) {
                    long p = pg_at(&g, i, j, k, l);
                    for (int f = 0; f < 8; ++f) {
                        double n0 = sqrt(diamond_grad_sq(&g, p0, p, f, h));
                        double n1 = sqrt(diamond_grad_sq(&g, p1, p, f, h));
                        double s = delta * n0 + vartheta * n1;
                        G[v * 8 + f] = 1.0 / (1.0 + K * s * s);
                    }
                }
    free(p0); free(p1);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* initial condition and local rescaling                                     */
/* ------------------------------------------------------------------------ */

/* u0 = 1/(d + v) - 1/(R + v) for spatial distance d <= R from a seed inside
 * its frame, else 0 (Eq. initialcond with the 1/(R+v) shift for zero
 * Dirichlet data); overlapping peaks take the maximum. */
int or_init_u(const int *dims, const double *xyz, const int *frame, int nseeds, double R, double vv,
              double *u)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double R2 = R * R;
    long v = 0;
    for (int l = 0; l < g.n[3]; ++l)
        for (int k = 0; k < g.n[2]; ++k)
            for (int j = 0; j < g.n[1]; ++j)
                for (int i = 0; i < g.n[0]; ++i, ++v) {
                    double best = 0.0;
                    for (int m = 0; m < nseeds; ++m) {
                        if (frame[m] != l) continue;
                        double d2 = seed_d2(xyz, m, i, j, k);
                        if (d2 > R2) continue;
                        double val = 1.0 / (sqrt(d2) + vv) - 1.0 / (R + vv);
                        if (val > best) best = val;
                    }
                    u[v] = best;
                }
    return OR_OK;
}

/* Remark "Local rescaling" (Eq. 841): mu_m, xi_m = min, max of u over
 * B(c_m, r), taken from u before any ball is rescaled; then owned voxels get
 * (u - mu)/(xi - mu).  A ball with xi - mu <= 1e-30 is left as it is. */
int or_rescale(const int *dims, double *u, const double *xyz, const int *frame, int nseeds, double r)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    int *owner = (int *)malloc(sizeof(int) * g.nv);
    double *mu = (double *)malloc(sizeof(double) * (nseeds > 0 ? nseeds : 1));
    double *xi = (double *)malloc(sizeof(double) * (nseeds > 0 ? nseeds : 1));
    if (!owner || !mu || !xi) { free(owner); free(mu); free(xi); return OR_ERR_ALLOC; }
    or_owner(dims, xyz, frame, nseeds, r, owner);
    for (int m = 0; m < nseeds; ++m) {
        int cnt;
        ball_minmax(&g, u, xyz, frame, m, r, &mu[m], &xi[m], &cnt);
    }
    for (long v = 0; v < g.nv; ++v) {
        int m = owner[v];
        if (m < 0) continue;
        double span = xi[m] - mu[m];
        if (!(span > 1e-30)) continue;
        u[v] = (u[v] - mu[m]) / span;
    }
    free(owner); free(mu); free(xi);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* coefficients of the step system (Eqs. 111th, new1 / new)                  */
/* ------------------------------------------------------------------------ */

/* From the padded u^{resc,n-1}: A_f = sqrt(eps^2 + |grad^f u|^2),
 * Abar = sqrt(eps^2 + (1/8) sum_f |grad^f u|^2), and for face f on axis d
 * off_f = tau/h_d^2 * Abar * G_f / A_f  (tau m(e)/(m(V) m(sigma)) of Eq. new1),
 * diag = 1 + sum_f off_f.  Faces to ghost cells keep their diagonal share;
 * the ghost's value enters through the padded array (Dirichlet data). */
static void assemble_padded(const pgrid *g, const double *up, const double *G, const double *h,
                            double tau, double eps, double *diag, double *off)
{
    long v = 0;
    for (int l = 0; l < g->n[3]; ++l)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i, ++v) {
                    long p = pg_at(g, i, j, k, l);
                    double g2[8];
                    double sum = 0.0;
                    for (int f = 0; f < 8; ++f) {
                        g2[f] = diamond_grad_sq(g, up, p, f, h);
                        sum += g2[f];
                    }
                    double Abar = sqrt(eps * eps + sum / 8.0);
                    double dsum = 0.0;
                    for (int f = 0; f < 8; ++f) {
                        int d = f >> 1;
                        double Af = sqrt(eps * eps + g2[f]);
                        double Gf = G ? G[v * 8 + f] : 1.0;
                        double a = tau / (h[d] * h[d]) * Abar * Gf / Af;
                        off[v * 8 + f] = a;
                        dsum += a;
                    }
                    diag[v] = 1.0 + dsum;
                }
}

/* Exported: coefficients from an interior u with zero Dirichlet ghosts.
 * Abar_out and Af_out may be NULL. */
int or_assemble(const int *dims, const double *u, const double *G, const double *h, double tau,
                double eps, double *diag, double *off)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double *up = (double *)malloc(sizeof(double) * g.np);
    if (!up) return OR_ERR_ALLOC;
    pad_dirichlet(&g, u, up, 0.0);
    assemble_padded(&g, up, G, h, tau, eps, diag, off);
    free(up);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* the whole segmentation (Section 3.5, "Brief overview")                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    double h[4];
    double tau, eps, K, delta, vartheta, lambda_th, r_ball, R_init, v_init, sigma_t, omega, tol;
    double omega_smooth; /* SOR relaxation used for the presmoothing solves */
    int max_iters, check_every;
} or_params;

/* u0 -> rescale -> threshold -> presmooth -> G -> nsteps x {coefficients,
 * solve with initial guess u^{resc,n-1}, rescale}.  iters_out[n] (optional)
 * receives the SOR sweeps of step n, res_out[n] the final relative residual.
 * Returns OR_NOT_CONVERGED if any solve hit max_iters (u is still valid). */
int or_segment(const int *dims, const double *I0, const double *xyz, const int *frame, int nseeds,
               const or_params *P, int nsteps, double *u, int *iters_out, double *res_out)
{
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    long nv = g.nv;
    double *ITH = (double *)malloc(sizeof(double) * nv);
    double *Is0 = (double *)malloc(sizeof(double) * nv);
    double *IsTH = (double *)malloc(sizeof(double) * nv);
    double *G = (double *)malloc(sizeof(double) * nv * 8);
    double *diag = (double *)malloc(sizeof(double) * nv);
    double *off = (double *)malloc(sizeof(double) * nv * 8);
    double *b = (double *)malloc(sizeof(double) * nv);
    int status = OR_OK;
    if (!ITH || !Is0 || !IsTH || !G || !diag || !off || !b) { status = OR_ERR_ALLOC; goto done; }

    or_init_u(dims, xyz, frame, nseeds, P->R_init, P->v_init, u);
    or_rescale(dims, u, xyz, frame, nseeds, P->r_ball);
    or_threshold(dims, I0, xyz, frame, nseeds, P->r_ball, P->lambda_th, ITH);
    {
        int it;
        double rr;
        int s1 = or_presmooth(dims, I0, P->h, P->sigma_t, P->omega_smooth, P->tol, P->max_iters,
                              P->check_every, Is0, &it, &rr);
        int s2 = or_presmooth(dims, ITH, P->h, P->sigma_t, P->omega_smooth, P->tol, P->max_iters,
                              P->check_every, IsTH, &it, &rr);
        if (s1 || s2) status = OR_NOT_CONVERGED;
    }
    or_face_G(dims, Is0, IsTH, P->h, P->K, P->delta, P->vartheta, G);
    for (int n = 0; n < nsteps; ++n) {
        or_assemble(dims, u, G, P->h, P->tau, P->eps, diag, off);
        memcpy(b, u, sizeof(double) * nv);
        int it = 0;
        double rr = 0.0;
        int s = or_solve(dims, diag, off, b, u, P->omega, P->tol, P->max_iters, P->check_every, &it, &rr);
        if (s) status = OR_NOT_CONVERGED;
        if (iters_out) iters_out[n] = it;
        if (res_out) res_out[n] = rr;
        or_rescale(dims, u, xyz, frame, nseeds, P->r_ball);
    }
done:
    free(ITH); free(Is0); free(IsTH); free(G); free(diag); free(off); free(b);
    return status;
}

/* ------------------------------------------------------------------------ */
/* experimental order of convergence (Section 3.4)                           */
/* ------------------------------------------------------------------------ */

/* exact solution u = (|x|^2 - 1)/6 + t of the level-set mean-curvature flow
 * (Eqs. exactsol, levelsetmcf) */
static double eoc_exact(const double *x, double t)
{
    double s = 0.0;
    for (int d = 0; d < 4; ++d) s += x[d] * x[d];
    return (s - 1.0) / 6.0 + t;
}

/* Coordinate of padded index a (0..n+1) on [-L, L]: x(a) = -L + (a + xoff) h.
 * xoff = -1/2 puts interior cell centres at -L + (i - 1/2) h (ghost-cell
 * centres half a cell outside the domain); other offsets place the ghost
 * values elsewhere (the paper does not state the placement). */
static double eoc_coord(int a, double L, double h, double xoff)
{
    return -L + ((double)a + xoff) * h;
}

static void eoc_fill_ghosts(const pgrid *g, double *up, double L, double h, double t, double xoff)
{
    int a[4];
    int n = g->n[0];
    for (a[3] = 0; a[3] < n + 2; ++a[3])
        for (a[2] = 0; a[2] < n + 2; ++a[2])
            for (a[1] = 0; a[1] < n + 2; ++a[1])
                for (a[0] = 0; a[0] < n + 2; ++a[0]) {
                    int ghost = 0;
                    for (int d = 0; d < 4; ++d)
                        if (a[d] == 0 || a[d] == n + 1) ghost = 1;
                    if (!ghost) continue;
                    double x[4];
                    for (int d = 0; d < 4; ++d) x[d] = eoc_coord(a[d], L, h, xoff);
                    up[pg_atp(g, a)] = eoc_exact(x, t);
                }
}

/* Runs the scheme with G = 1, no rescaling, eps = eps_factor * h^2, the exact
 * solution as Dirichlet data and initial condition, on [-L, L]^4 with n cells
 * per axis and nsteps steps of tau = T/nsteps.  err_out receives the
 * L2((0,T), L2(Omega)) error sqrt(sum_n tau sum_i h^4 (u_i^n - u(x_i,t_n))^2). */
int or_eoc(int n, int nsteps, double T, double L, double hdiv, double xoff, double eps_factor,
           double omega, double tol, int max_iters, double *err_out, double *err_steps,
           int *iters_total)
{
    int dims[4] = {n, n, n, n};
    pgrid g;
    if (pg_init(&g, dims)) return OR_ERR_ARG;
    double h = 2.0 * L / ((double)n + hdiv);
    double hv[4] = {h, h, h, h};
    double tau = T / nsteps;
    double eps = eps_factor * h * h;
    double *up = (double *)malloc(sizeof(double) * g.np);
    double *diag = (double *)malloc(sizeof(double) * g.nv);
    double *off = (double *)malloc(sizeof(double) * g.nv * 8);
    double *b = (double *)malloc(sizeof(double) * g.nv);
    if (!up || !diag || !off || !b) { free(up); free(diag); free(off); free(b); return OR_ERR_ALLOC; }
    int a[4];
    for (a[3] = 0; a[3] < n + 2; ++a[3])
        for (a[2] = 0; a[2] < n + 2; ++a[2])
            for (a[1] = 0; a[1] < n + 2; ++a[1])
                for (a[0] = 0; a[0] < n + 2; ++a[0]) {
                    double x[4];
                    for (int d = 0; d < 4; ++d) x[d] = eoc_coord(a[d], L, h, xoff);
                    up[pg_atp(&g, a)] = eoc_exact(x, 0.0);
                }
    double err2 = 0.0;
    int status = OR_OK;
    int total = 0;
    for (int s = 1; s <= nsteps; ++s) {
        double t_prev = (s - 1) * tau, t = s * tau;
        eoc_fill_ghosts(&g, up, L, h, t_prev, xoff);
        assemble_padded(&g, up, NULL, hv, tau, eps, diag, off);
        long v = 0;
        for (int l = 0; l < n; ++l)
            for (int k = 0; k < n; ++k)
                for (int j = 0; j < n; ++j)
                    for (int i = 0; i < n; ++i) b[v++] = up[pg_at(&g, i, j, k, l)];
        eoc_fill_ghosts(&g, up, L, h, t, xoff);
        int it = 0;
        double rr = 0.0;
        if (sor_padded(&g, diag, off, b, up, omega, tol, max_iters, 4, &it, &rr)) status = OR_NOT_CONVERGED;
        total += it;
        double e2 = 0.0;
        for (a[3] = 1; a[3] <= n; ++a[3])
            for (a[2] = 1; a[2] <= n; ++a[2])
                for (a[1] = 1; a[1] <= n; ++a[1])
                    for (a[0] = 1; a[0] <= n; ++a[0]) {
                        double x[4];
                        for (int d = 0; d < 4; ++d) x[d] = eoc_coord(a[d], L, h, xoff);
                        double e = up[pg_atp(&g, a)] - eoc_exact(x, t);
                        e2 += e * e;
                    }
        err2 += tau * h * h * h * h * e2;
        if (err_steps) err_steps[s - 1] = sqrt(h * h * h * h * e2);
    }
    *err_out = sqrt(err2);
    if (iters_total) *iters_total = total;
    free(up); free(diag); free(off); free(b);
    return status;
}
