/*
 * fv_oracle.c -- plain, slow FP64 CPU oracle for one explicit finite-volume
 * time step over a batch of Cartesian patches (Rusanov flux, compressible
 * Euler equations).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.  It shares no code, header or
 * table with the CUDA library and must never be reached from the product
 * path.
 *
 * What it follows (arXiv:2306.16731, "SYCL compute kernels for ExaHyPE"):
 *   - Sec. 2.2: each volume of a p^d patch carries N unknowns; the new value
 *     is the old one plus dt-scaled face fluxes; the face flux is Eq. 2
 *     (Rusanov); every patch carries a halo layer of width one; after the
 *     update the maximum eigenvalue over the new solution is reduced per
 *     patch and feeds the CFL condition (local time stepping).
 *   - Sec. 2.3: the kernel takes N (p+2)^d T values (with halo) and yields
 *     N p^d T values; Algorithm 1 orders the work as: copy Q to Q_new on the
 *     interior; directional fluxes F_x over [-1,p] x [0,p-1], F_y over
 *     [0,p-1] x [-1,p] (and F_z likewise in 3D); the update of every interior
 *     volume from the fluxes left and right of it; the directional
 *     eigenvalues.
 *   - Sec. 5: Euler equations, N = 2 + d, no non-conservative terms and no
 *     sources.  The paper prints no flux formulas; the textbook ideal-gas
 *     Euler system with adiabatic index gamma is used.
 *
 * Readings of garbled or silent passages (each is listed in the design notes
 * of the repository):
 *   R1  the update scale printed as "dt * h" is dt / h;
 *   R2  the "+-" of the update is minus the outward flux difference, i.e.
 *       Q_new = Q - dt/h * sum_n (Fhat_n(c+1/2) - Fhat_n(c-1/2)); the
 *       difference is formed first, summed over n in the order x, y, z and
 *       only then scaled;
 *   R3  the dissipation coefficient printed as "C/h" is 1/2:
 *       Fhat = 1/2 (F_n(Q_L) + F_n(Q_R)) - 1/2 max(lam_L, lam_R) (Q_R - Q_L),
 *       with L the lower-index volume and R the upper-index volume;
 *   R4  the eigenvalues that enter Eq. 2 are those of the current state (the
 *       position of the eigenvalue loop in Algorithm 1 is schematic);
 *   R5  the per-patch maximum runs over interior volumes of the new state
 *       and all d directions, neutral element 0;
 *   R6  the CFL condition is dt = CFL * h / (d * lambda_max);
 *   R7  halo width 1; edge and corner halo volumes are never read.  Fixed
 *       halos are copied from input to output; periodic halos are rebuilt
 *       from the wrapped interior before every step.
 *
 * Layout (Sec. 4, array of structures): Q[patch][z][y][x][k], x fastest,
 * the N unknowns of a volume contiguous; patch i starts at element
 * sum_{j<i} N (p_j+2)^d.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared [-fopenmp].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FVO_OK 0
#define FVO_EINVAL (-1)
#define FVO_ENOMEM (-2)

/* ---------------------------------------------------------------- layout */

static int64_t patch_cells(int dim, int p)
{
    int64_t e = (int64_t)p + 2;
    return dim == 2 ? e * e : e * e * e;
}

/* Halo-inclusive linear cell index of (i, j, k), each in [-1, p]. */
static int64_t cell_index(int dim, int p, int i, int j, int k)
{
    int64_t e = (int64_t)p + 2;
    if (dim == 2)
        return (int64_t)(j + 1) * e + (i + 1);
    return ((int64_t)(k + 1) * e + (j + 1)) * e + (i + 1);
}

/* ------------------------------------------------------- Euler physics */

/* Primitive state of one volume: velocity u[0..d-1], pressure, sound speed.
 * Ideal gas: p = (gamma-1) (E - 1/2 sum_k (rho u_k) u_k), c = sqrt(gamma p / rho). */
static void primitives(int dim, double gamma, const double *q,
                       double *u, double *pres, double *snd)
{
    double rho = q[0];
    double kin = 0.0;
    for (int a = 0; a < dim; ++a) {
        u[a] = q[1 + a] / rho;
        kin += q[1 + a] * u[a];
    }
    double E = q[dim + 1];
    *pres = (gamma - 1.0) * (E - 0.5 * kin);
    *snd = sqrt(gamma * (*pres) / rho);
}

/* Maximum eigenvalue of the flux Jacobian along axis n (Sec. 2.2): |u_n| + c. */
static double max_eigenvalue_along(int dim, double gamma, const double *q, int n)
{
    double u[3], pres, snd;
    primitives(dim, gamma, q, u, &pres, &snd);
    return fabs(u[n]) + snd;
}

/* Physical flux along axis n:
 * (rho u_n, rho u_1 u_n + delta_{1n} p, ..., rho u_d u_n + delta_{dn} p, (E + p) u_n). */
static void physical_flux(int dim, double gamma, const double *q, int n, double *F)
{
    double u[3], pres, snd;
    primitives(dim, gamma, q, u, &pres, &snd);
    F[0] = q[1 + n];
    for (int a = 0; a < dim; ++a)
        F[1 + a] = q[1 + a] * u[n] + (a == n ? pres : 0.0);
    F[dim + 1] = (q[dim + 1] + pres) * u[n];
}

/* Rusanov face flux (Eq. 2, reading R3) from the stored directional fluxes
 * and eigenvalues of the two volumes adjacent to the face. */
static void rusanov_face(int N, const double *QL, const double *QR,
                         const double *FL, const double *FR,
                         double lamL, double lamR, double *Fhat)
{
    double lam = lamL > lamR ? lamL : lamR;
    for (int k = 0; k < N; ++k)
        Fhat[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * lam * (QR[k] - QL[k]);
}

/* ---------------------------------------------------------- halo modes */

/* Periodic halo: axis by axis, halo index -1 takes the value at p-1 and
 * halo index p the value at 0.  Whole layers are copied (including the
 * halo ranges of the other axes), so edges and corners wrap too. */
static void fill_periodic_halo(int dim, int p, int N, double *Q)
{
    int kmin = dim == 3 ? -1 : 0, kmax = dim == 3 ? p : 0;
    for (int axis = 0; axis < dim; ++axis) {
        for (int k = kmin; k <= kmax; ++k)
            for (int j = -1; j <= p; ++j)
                for (int i = -1; i <= p; ++i) {
                    int idx[3] = {i, j, k};
                    if (idx[axis] != -1 && idx[axis] != p)
                        continue;
                    int src[3] = {i, j, k};
                    src[axis] = idx[axis] == -1 ? p - 1 : 0;
                    int64_t d = cell_index(dim, p, i, j, k);
                    int64_t s = cell_index(dim, p, src[0], src[1], src[2]);
                    memcpy(Q + d * N, Q + s * N, (size_t)N * sizeof(double));
                }
    }
}

/* ------------------------------------------------------------- one patch */

/* Maximum eigenvalue of one patch over its interior volumes and all d
 * directions (reading R5). */
static double patch_max_eigenvalue(int dim, int p, double gamma, const double *Q)
{
    int N = dim + 2;
    int kmax = dim == 3 ? p - 1 : 0;
    double lam = 0.0;
    for (int k = 0; k <= kmax; ++k)
        for (int j = 0; j < p; ++j)
            for (int i = 0; i < p; ++i) {
                const double *q = Q + cell_index(dim, p, i, j, k) * N;
                for (int n = 0; n < dim; ++n) {
                    double l = max_eigenvalue_along(dim, gamma, q, n);
                    if (l > lam)
                        lam = l;
                }
            }
    return lam;
}

/* One explicit step of one patch, in the order of Algorithm 1.
 * Qin and Qout both hold (p+2)^d volumes of N unknowns. */
static int patch_step(int dim, int p, double gamma, int periodic,
                      double h, double dt, const double *Qin, double *Qout)
{
    int N = dim + 2;
    int64_t nc = patch_cells(dim, p);
    double *Q = (double *)malloc((size_t)(nc * N) * sizeof(double));
    double *tmpF[3] = {NULL, NULL, NULL};
    double *tmpL[3] = {NULL, NULL, NULL};
    int rc = FVO_OK;
    if (!Q) return FVO_ENOMEM;
    for (int n = 0; n < dim; ++n) {
        tmpF[n] = (double *)calloc((size_t)(nc * N), sizeof(double));
        tmpL[n] = (double *)calloc((size_t)nc, sizeof(double));
        if (!tmpF[n] || !tmpL[n]) { rc = FVO_ENOMEM; goto done; }
    }

    memcpy(Q, Qin, (size_t)(nc * N) * sizeof(double));
    if (periodic)
        fill_periodic_halo(dim, p, N, Q);

    /* Q_new <- Q (halo volumes included: fixed halos stay as given). */
    memcpy(Qout, Q, (size_t)(nc * N) * sizeof(double));

    /* Directional fluxes and eigenvalues: along n over [-1, p], over
     * [0, p-1] along the other axes. */
    int kmin = dim == 3 ? -1 : 0, kmax = dim == 3 ? p : 0;
    for (int n = 0; n < dim; ++n)
        for (int k = kmin; k <= kmax; ++k)
            for (int j = -1; j <= p; ++j)
                for (int i = -1; i <= p; ++i) {
                    int idx[3] = {i, j, dim == 3 ? k : 0};
                    int ok = 1;
                    for (int a = 0; a < dim; ++a) {
                        int lo = a == n ? -1 : 0, hi = a == n ? p : p - 1;
                        if (idx[a] < lo || idx[a] > hi) ok = 0;
                    }
                    if (!ok) continue;
                    int64_t c = cell_index(dim, p, i, j, k);
                    physical_flux(dim, gamma, Q + c * N, n, tmpF[n] + c * N);
                    tmpL[n][c] = max_eigenvalue_along(dim, gamma, Q + c * N, n);
                }

    /* Update of every interior volume (readings R1, R2). */
    double scale = dt / h;
    int kin_lo = 0, kin_hi = dim == 3 ? p - 1 : 0;
    for (int k = kin_lo; k <= kin_hi; ++k)
        for (int j = 0; j < p; ++j)
            for (int i = 0; i < p; ++i) {
                int64_t c = cell_index(dim, p, i, j, k);
                double acc[5] = {0, 0, 0, 0, 0};
                for (int n = 0; n < dim; ++n) {
                    int lo[3] = {i, j, k}, hi[3] = {i, j, k};
                    lo[n] -= 1;
                    hi[n] += 1;
                    int64_t cl = cell_index(dim, p, lo[0], lo[1], lo[2]);
                    int64_t cr = cell_index(dim, p, hi[0], hi[1], hi[2]);
                    double Fleft[5], Fright[5];
                    rusanov_face(N, Q + cl * N, Q + c * N, tmpF[n] + cl * N,
                                 tmpF[n] + c * N, tmpL[n][cl], tmpL[n][c], Fleft);
                    rusanov_face(N, Q + c * N, Q + cr * N, tmpF[n] + c * N,
                                 tmpF[n] + cr * N, tmpL[n][c], tmpL[n][cr], Fright);
                    for (int q = 0; q < N; ++q)
                        acc[q] += Fright[q] - Fleft[q];
                }
                for (int q = 0; q < N; ++q)
                    Qout[c * N + q] = Q[c * N + q] - scale * acc[q];
            }

done:
    for (int n = 0; n < 3; ++n) { free(tmpF[n]); free(tmpL[n]); }
    free(Q);
    return rc;
}

/* --------------------------------------------------------------- batches */

static int check_batch(int dim, int T, const int32_t *p)
{
    if (dim != 2 && dim != 3) return FVO_EINVAL;
    if (T < 0 || (T > 0 && !p)) return FVO_EINVAL;
    for (int i = 0; i < T; ++i)
        if (p[i] < 1) return FVO_EINVAL;
    return FVO_OK;
}

/* Element offset of every patch (T+1 entries). */
static int64_t *patch_offsets(int dim, int T, const int32_t *p)
{
    int64_t *off = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    if (!off) return NULL;
    off[0] = 0;
    for (int i = 0; i < T; ++i)
        off[i + 1] = off[i] + (int64_t)(dim + 2) * patch_cells(dim, p[i]);
    return off;
}

/* Number of doubles of a halo-inclusive batch state. */
int64_t fvo_state_elems(int dim, int T, const int32_t *p)
{
    int64_t s = 0;
    for (int i = 0; i < T; ++i)
        s += (int64_t)(dim + 2) * patch_cells(dim, p[i]);
    return s;
}

/* One step over all patches: Qout = step(Qin) with per-patch h = dx[i] and
 * dt[i]; lambda_out[i] (may be NULL) = maximum eigenvalue of the new state. */
int fvo_batch_step(int dim, int T, const int32_t *p, const double *dx,
                   const double *dt, double gamma, int halo_mode,
                   const double *Qin, double *Qout, double *lambda_out)
{
    int rc = check_batch(dim, T, p);
    if (rc) return rc;
    int64_t *off = patch_offsets(dim, T, p);
    if (!off) return FVO_ENOMEM;
    int err = FVO_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) reduction(min : err)
#endif
    for (int i = 0; i < T; ++i) {
        int r = patch_step(dim, p[i], gamma, halo_mode == 1, dx[i], dt[i],
                           Qin + off[i], Qout + off[i]);
        if (r < err) err = r;
        if (lambda_out)
            lambda_out[i] = patch_max_eigenvalue(dim, p[i], gamma, Qout + off[i]);
    }
    free(off);
    return err;
}

/* Per-patch maximum eigenvalue (interior, all directions). */
int fvo_batch_max_eigenvalue(int dim, int T, const int32_t *p, double gamma,
                             const double *Q, double *lambda_out)
{
    int rc = check_batch(dim, T, p);
    if (rc) return rc;
    int64_t *off = patch_offsets(dim, T, p);
    if (!off) return FVO_ENOMEM;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int i = 0; i < T; ++i)
        lambda_out[i] = patch_max_eigenvalue(dim, p[i], gamma, Q + off[i]);
    free(off);
    return FVO_OK;
}

/* CFL time step (reading R6): dt = cfl * h / (d * lambda). */
void fvo_cfl_time_step(int dim, int T, const double *lambda, const double *dx,
                       double cfl, double *dt_out)
{
    for (int i = 0; i < T; ++i)
        dt_out[i] = (cfl * dx[i]) / ((double)dim * lambda[i]);
}

/* S steps with per-patch dt chaining: dt_0 from the eigenvalue of Q, then
 * dt_{s+1} from the eigenvalue of the new state.  Q is updated in place
 * (the halo follows halo_mode); lambda_out/dt_out receive the values after
 * the last step (may be NULL). */
int fvo_batch_run(int dim, int T, const int32_t *p, const double *dx,
                  double gamma, int halo_mode, double cfl, int steps,
                  double *Q, double *lambda_out, double *dt_out)
{
    int rc = check_batch(dim, T, p);
    if (rc) return rc;
    int64_t n = fvo_state_elems(dim, T, p);
    double *tmp = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *lam = (double *)malloc((size_t)(T > 0 ? T : 1) * sizeof(double));
    double *dt = (double *)malloc((size_t)(T > 0 ? T : 1) * sizeof(double));
    if (!tmp || !lam || !dt) { rc = FVO_ENOMEM; goto out; }
    rc = fvo_batch_max_eigenvalue(dim, T, p, gamma, Q, lam);
    if (rc) goto out;
    fvo_cfl_time_step(dim, T, lam, dx, cfl, dt);
    for (int s = 0; s < steps; ++s) {
        rc = fvo_batch_step(dim, T, p, dx, dt, gamma, halo_mode, Q, tmp, lam);
        if (rc) goto out;
        memcpy(Q, tmp, (size_t)n * sizeof(double));
        fvo_cfl_time_step(dim, T, lam, dx, cfl, dt);
    }
    if (lambda_out) memcpy(lambda_out, lam, (size_t)T * sizeof(double));
    if (dt_out) memcpy(dt_out, dt, (size_t)T * sizeof(double));
out:
    free(tmp);
    free(lam);
    free(dt);
    return rc;
}

/* Per-patch sums of every unknown over the interior volumes (conservation
 * diagnostics); totals_out has T * N entries. */
int fvo_batch_totals(int dim, int T, const int32_t *p, const double *Q,
                     double *totals_out)
{
    int rc = check_batch(dim, T, p);
    if (rc) return rc;
    int64_t *off = patch_offsets(dim, T, p);
    if (!off) return FVO_ENOMEM;
    int N = dim + 2;
    for (int i = 0; i < T; ++i) {
        int P = p[i];
        int kmax = dim == 3 ? P - 1 : 0;
        for (int q = 0; q < N; ++q) totals_out[(int64_t)i * N + q] = 0.0;
        for (int k = 0; k <= kmax; ++k)
            for (int j = 0; j < P; ++j)
                for (int ii = 0; ii < P; ++ii) {
                    const double *c = Q + off[i] + cell_index(dim, P, ii, j, k) * N;
                    for (int q = 0; q < N; ++q)
                        totals_out[(int64_t)i * N + q] += c[q];
                }
    }
    free(off);
    return FVO_OK;
}

/* Number of threads the batch loops use (1 without OpenMP). */
int fvo_num_threads(void)
{
#ifdef _OPENMP
    int n = 0;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}

/* Threads for the following batch loops (timing the oracle on one core or
 * on all of them); n < 1 restores the OpenMP default. */
void fvo_set_num_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n >= 1 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}

/* Halo fill from neighbouring patches (the step before the kernel call in
 * the paper's framework: patches are equipped with a halo layer of width one
 * taken from their neighbours, Sec. 2.2).  nbr has 2*dim entries per patch in
 * the order -x, +x, -y, +y[, -z, +z]: the index of the patch across that face
 * (same edge length), or -1 to leave that face's halo as it is.  For each
 * face with a neighbour, every face-halo volume (corners excluded) receives
 * the neighbour's interior volume that touches the face: across -x the
 * neighbour's column x = p-1, across +x its column x = 0, and likewise in y
 * and z.  Q is updated in place (only halo volumes are written). */
int fvo_halo_exchange(int dim, int T, const int32_t *p, const int32_t *nbr, double *Q)
{
    int rc = check_batch(dim, T, p);
    if (rc) return rc;
    for (int i = 0; i < T * 2 * dim; ++i) {
        int j = nbr[i];
        if (j < -1 || j >= T || (j >= 0 && p[j] != p[i / (2 * dim)])) return FVO_EINVAL;
    }
    int64_t *off = patch_offsets(dim, T, p);
    if (!off) return FVO_ENOMEM;
    int N = dim + 2;
    for (int i = 0; i < T; ++i) {
        int P = p[i];
        int kmax = dim == 3 ? P - 1 : 0;
        for (int face = 0; face < 2 * dim; ++face) {
            int j = nbr[i * 2 * dim + face];
            if (j < 0) continue;
            int axis = face / 2, upper = face % 2;
            /* halo coordinate along the axis and the neighbour's source index */
            int dst_a = upper ? P : -1, src_a = upper ? 0 : P - 1;
            for (int k = 0; k <= kmax; ++k)
                for (int t = 0; t < P; ++t) {
                    int dc[3], sc[3];
                    /* the two tangential coordinates run over the interior */
                    int tan[2] = {t, k};
                    int ti = 0;
                    for (int a = 0; a < dim; ++a) {
                        if (a == axis) { dc[a] = dst_a; sc[a] = src_a; }
                        else { dc[a] = tan[ti]; sc[a] = tan[ti]; ++ti; }
                    }
                    if (dim == 2) { dc[2] = 0; sc[2] = 0; }
                    int64_t d = off[i] + cell_index(dim, P, dc[0], dc[1], dc[2]) * N;
                    int64_t s = off[j] + cell_index(dim, P, sc[0], sc[1], sc[2]) * N;
                    for (int q = 0; q < N; ++q) Q[d + q] = Q[s + q];
                }
        }
    }
    free(off);
    return FVO_OK;
}

/* =====================================================================
 * Generic first-order hyperbolic PDE of Eq. 1,
 *     dQ/dt + div F(Q) + sum_n B_n(Q) dQ/dx_n = S(Q),
 * realised for the two-dimensional shallow water equations over a
 * bathymetry b with a Coriolis force (the paper states the PDE class in
 * Sec. 2 and studies only Euler, for which B = 0 and S = 0):
 *     Q = (h, hu, hv, b),  b a parameter (db/dt = 0), u = hu/h, v = hv/h,
 *     F_x = (hu, hu u + g h^2 / 2, hv u, 0),
 *     F_y = (hv, hu v, hv v + g h^2 / 2, 0),
 *     B_x(Q) dQ/dx = (0, g h db/dx, 0, 0),  B_y(Q) dQ/dy = (0, 0, g h db/dy, 0),
 *     S(Q) = (0, f hv, -f hu, 0),
 *     lambda_n = |u_n| + sqrt(g h).
 * Readings (the paper gives no discretisation of B and S):
 *   R13 the Rusanov flux of Eq. 2 (reading R3) acts on the evolved unknowns
 *       (h, hu, hv); the parameter b gets no flux and no dissipation and is
 *       copied unchanged;
 *   R14 the non-conservative product at a face L|R along n is
 *       D = B_n(Qbar) (Q_R - Q_L) with Qbar = (Q_L + Q_R) / 2, and half of it
 *       enters each of the two volumes;
 *   R15 the source is explicit and pointwise, evaluated on the old state.
 * One step of an interior volume c (faces l = c-1/2, r = c+1/2 along n):
 *     acc = sum_{n = x, y} ((Fhat_r - Fhat_l) + 1/2 (D_r + D_l)),
 *     Q_new = Q - (dt / h) acc + dt S(Q).
 * Halos follow R7.  The CFL step uses lambda_max as in R5/R6.
 * ===================================================================== */

#define SWE_N 4

static double swe_lambda(double g, const double *q, int n)
{
    double h = q[0];
    return fabs(q[1 + n] / h) + sqrt(g * h);
}

static void swe_flux(double g, const double *q, int n, double *F)
{
    double h = q[0], un = q[1 + n] / h;
    F[0] = q[1 + n];
    F[1] = q[1] * un + (n == 0 ? 0.5 * g * h * h : 0.0);
    F[2] = q[2] * un + (n == 1 ? 0.5 * g * h * h : 0.0);
    F[3] = 0.0;
}

/* D = B_n(Qbar) (Q_R - Q_L) (reading R14). */
static void swe_ncp(double g, const double *QL, const double *QR, int n, double *D)
{
    double hbar = 0.5 * (QL[0] + QR[0]);
    D[0] = 0.0;
    D[1] = n == 0 ? g * hbar * (QR[3] - QL[3]) : 0.0;
    D[2] = n == 1 ? g * hbar * (QR[3] - QL[3]) : 0.0;
    D[3] = 0.0;
}

/* Rusanov flux on the evolved unknowns (readings R3, R13). */
static void swe_face(double g, const double *QL, const double *QR, int n, double *Fhat)
{
    double FL[SWE_N], FR[SWE_N];
    swe_flux(g, QL, n, FL);
    swe_flux(g, QR, n, FR);
    double lL = swe_lambda(g, QL, n), lR = swe_lambda(g, QR, n);
    double lam = lL > lR ? lL : lR;
    for (int k = 0; k < 3; ++k)
        Fhat[k] = 0.5 * (FL[k] + FR[k]) - 0.5 * lam * (QR[k] - QL[k]);
    Fhat[3] = 0.0;
}

static double swe_patch_max_eigenvalue(int p, double g, const double *Q)
{
    double lam = 0.0;
    for (int j = 0; j < p; ++j)
        for (int i = 0; i < p; ++i) {
            const double *q = Q + cell_index(2, p, i, j, 0) * SWE_N;
            for (int n = 0; n < 2; ++n) {
                double l = swe_lambda(g, q, n);
                if (l > lam) lam = l;
            }
        }
    return lam;
}

static int swe_patch_step(int p, double g, double f, int periodic, double h, double dt,
                          const double *Qin, double *Qout)
{
    int64_t nc = patch_cells(2, p);
    double *Q = (double *)malloc((size_t)(nc * SWE_N) * sizeof(double));
    if (!Q) return FVO_ENOMEM;
    memcpy(Q, Qin, (size_t)(nc * SWE_N) * sizeof(double));
    if (periodic)
        fill_periodic_halo(2, p, SWE_N, Q);
    memcpy(Qout, Q, (size_t)(nc * SWE_N) * sizeof(double));
    double scale = dt / h;
    for (int j = 0; j < p; ++j)
        for (int i = 0; i < p; ++i) {
            int64_t c = cell_index(2, p, i, j, 0);
            const double *qc = Q + c * SWE_N;
            double acc[SWE_N] = {0, 0, 0, 0};
            for (int n = 0; n < 2; ++n) {
                int lo[2] = {i, j}, hi[2] = {i, j};
                lo[n] -= 1;
                hi[n] += 1;
                const double *ql = Q + cell_index(2, p, lo[0], lo[1], 0) * SWE_N;
                const double *qr = Q + cell_index(2, p, hi[0], hi[1], 0) * SWE_N;
                double Fl[SWE_N], Fr[SWE_N], Dl[SWE_N], Dr[SWE_N];
                swe_face(g, ql, qc, n, Fl);
                swe_face(g, qc, qr, n, Fr);
                swe_ncp(g, ql, qc, n, Dl);
                swe_ncp(g, qc, qr, n, Dr);
                for (int k = 0; k < SWE_N; ++k)
                    acc[k] += (Fr[k] - Fl[k]) + 0.5 * (Dr[k] + Dl[k]);
            }
            double S[SWE_N] = {0.0, f * qc[2], -f * qc[1], 0.0};
            for (int k = 0; k < 3; ++k)
                Qout[c * SWE_N + k] = qc[k] - scale * acc[k] + dt * S[k];
            Qout[c * SWE_N + 3] = qc[3];
        }
    free(Q);
    return FVO_OK;
}

/* One shallow water step over a batch of 2D patches (N = 4 unknowns per
 * volume, layout as for Euler); lambda_out (may be NULL) = maximum
 * eigenvalue of the new state per patch. */
int fvo_swe_batch_step(int T, const int32_t *p, const double *dx, const double *dt, double g, double f,
                       int halo_mode, const double *Qin, double *Qout, double *lambda_out)
{
    int rc = check_batch(2, T, p);
    if (rc) return rc;
    int64_t *off = (int64_t *)malloc((size_t)(T + 1) * sizeof(int64_t));
    if (!off) return FVO_ENOMEM;
    off[0] = 0;
    for (int i = 0; i < T; ++i) off[i + 1] = off[i] + SWE_N * patch_cells(2, p[i]);
    int err = FVO_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) reduction(min : err)
#endif
    for (int i = 0; i < T; ++i) {
        int r = swe_patch_step(p[i], g, f, halo_mode == 1, dx[i], dt[i], Qin + off[i], Qout + off[i]);
        if (r < err) err = r;
        if (lambda_out) lambda_out[i] = swe_patch_max_eigenvalue(p[i], g, Qout + off[i]);
    }
    free(off);
    return err;
}

int fvo_swe_batch_max_eigenvalue(int T, const int32_t *p, double g, const double *Q, double *lambda_out)
{
    int rc = check_batch(2, T, p);
    if (rc) return rc;
    int64_t o = 0;
    for (int i = 0; i < T; ++i) {
        lambda_out[i] = swe_patch_max_eigenvalue(p[i], g, Q + o);
        o += SWE_N * patch_cells(2, p[i]);
    }
    return FVO_OK;
}
