/*
 * FP64 CPU oracle for the RKL2 super-time-step of anisotropic (optionally
 * saturated) thermal conduction, Vaidya et al. 2017 (arXiv:1702.05487).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, obviously correct
 * statement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code,
 * header or constant with the CUDA library and includes nothing from it.
 *
 * Every routine follows the paper's definitions in the paper's order:
 *   - face fluxes: Eq. Fclass (classical anisotropic flux), Eq. Fclass_HD
 *     (isotropic / perpendicular part), Eqs. Fc and Fsat (harmonic blend with
 *     the saturated flux), with the normal gradient taken as a central
 *     difference across the face and the transverse gradients averaged to
 *     the face (Eqs. qN and qT, Appendix B);
 *   - conservative divergence: the equation after Eq. scalar_diffusion in
 *     Section 3 (one flux per face, shared by the two cells);
 *   - explicit parabolic step: Eq. dt_exp;
 *   - number of RKL2 stages: Eq. RKL-s, rounded as in Section 4.1;
 *   - RKL2 coefficients and stage recurrence: Appendix A, Eq. rkl2scheme.
 *
 * Readings where the paper is silent (stated once here, used throughout):
 *   - the state variable is T = rho*eps = p with rho = 1 and gamma = 2, so
 *     dT/dt = -div F (Section 4.1);
 *   - at a face, b and T are the arithmetic means of the two cells and the
 *     conductivity is kappa(T_face);
 *   - kappa_perp = kappa_perp_ratio * kappa_par;
 *   - the saturated flux uses c_iso = sqrt(T_face) (p/rho with rho = 1), or,
 *     with sat_upwind, the T of the cell the normal classical flux leaves;
 *   - |F_class| is the Euclidean norm of the full face vector;
 *   - Dirichlet ghosts (edges and corners included) hold T = bc_value and copy
 *     b from the nearest interior cell;
 *   - dt_expl bounds chi_d by kappa_par + kappa_perp in every direction;
 *   - with the limiter of Appendix C (Sharma & Hammett 2007) the transverse
 *     gradient at a face is MC(MC(up_L, down_L), MC(up_R, down_R)), the
 *     monotonised-central limiter applied first to the two one-sided
 *     differences of each cell and then across the two cells, used at faces
 *     whose lower temperature is below limiter_floor (Section 3.4: limiters
 *     only where T falls below a floor; an infinite floor limits everywhere).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int ndim;               /* 1, 2 or 3 active axes (x first)            */
    long n[3];              /* cells along x, y, z; inactive axes hold 1   */
    double dx[3];           /* mesh spacing along x, y, z                 */
    int bc;                 /* 0 periodic, 1 Dirichlet                    */
    double bc_value;        /* ghost temperature for Dirichlet            */
    int kappa_model;        /* 0 constant, 1 Spitzer kappa0 * T^(5/2)     */
    double kappa_par0;
    double kappa_perp_ratio;
    int saturate;           /* 1: harmonic blend with q = 5 phi rho c^3   */
    double phi;
    double rho;
    int sat_upwind;         /* 1: q from the upwind cell, 0: from T_face  */
    double cp;              /* parabolic Courant number of Eq. dt_exp     */
    int limiter;            /* 1: MC-limited transverse gradients          */
    double limiter_floor;   /* limit only faces with min(T_L, T_R) below   */
} orc_problem;

static long ncell(const orc_problem *P) { return P->n[0] * P->n[1] * P->n[2]; }

static long idx(const orc_problem *P, long i, long j, long k)
{
    return (k * P->n[1] + j) * P->n[0] + i;
}

/* T at a cell that may lie one or two cells outside the grid. */
static double T_at(const orc_problem *P, const double *T, long i, long j, long k)
{
    long c[3] = {i, j, k};
    for (int d = 0; d < 3; ++d) {
        if (c[d] >= 0 && c[d] < P->n[d]) continue;
        if (d >= P->ndim || P->bc == 0) {
            c[d] = ((c[d] % P->n[d]) + P->n[d]) % P->n[d];
        } else {
            return P->bc_value;
        }
    }
    return T[idx(P, c[0], c[1], c[2])];
}

/* Component e of the unit field b at a cell that may lie outside the grid. */
static double b_at(const orc_problem *P, const double *b, int e, long i, long j, long k)
{
    long c[3] = {i, j, k};
    for (int d = 0; d < 3; ++d) {
        if (c[d] >= 0 && c[d] < P->n[d]) continue;
        if (d >= P->ndim || P->bc == 0) {
            c[d] = ((c[d] % P->n[d]) + P->n[d]) % P->n[d];
        } else {
            c[d] = c[d] < 0 ? 0 : P->n[d] - 1;
        }
    }
    return b[(long)e * ncell(P) + idx(P, c[0], c[1], c[2])];
}

/* Monotonised-central limiter: 0 if a and b differ in sign, else the one of
 * 2a, 2b, (a+b)/2 smallest in magnitude (van Leer's MC slope). */
static double mc_limit(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    double m = fabs(0.5 * (a + b));
    if (2.0 * fabs(a) < m) m = 2.0 * fabs(a);
    if (2.0 * fabs(b) < m) m = 2.0 * fabs(b);
    return a > 0.0 ? m : -m;
}

/* Parallel conductivity kappa_par(T). */
static double kappa_par(const orc_problem *P, double T)
{
    if (P->kappa_model == 1) return P->kappa_par0 * pow(T, 2.5);
    return P->kappa_par0;
}

/*
 * Component d of the conduction flux on the face between cell (i,j,k) and
 * its +e_d neighbour.
 */
double orc_face_flux(const orc_problem *P, const double *T, const double *b,
                     int d, long i, long j, long k)
{
    long c0[3] = {i, j, k};
    long c1[3] = {i, j, k};
    c1[d] += 1;

    /* gradient of T at the face */
    double grad[3] = {0.0, 0.0, 0.0};
    double TL = T_at(P, T, c0[0], c0[1], c0[2]);
    double TR = T_at(P, T, c1[0], c1[1], c1[2]);
    grad[d] = (TR - TL) / P->dx[d];                         /* normal, Eq. qN */
    const int limit = P->limiter && (TL < TR ? TL : TR) < P->limiter_floor;
    for (int e = 0; e < P->ndim; ++e) {
        if (e == d) continue;
        long a0[3] = {c0[0], c0[1], c0[2]}, a1[3] = {c1[0], c1[1], c1[2]};
        long m0[3] = {c0[0], c0[1], c0[2]}, m1[3] = {c1[0], c1[1], c1[2]};
        a0[e] += 1; a1[e] += 1; m0[e] -= 1; m1[e] -= 1;
        double upL = T_at(P, T, a0[0], a0[1], a0[2]) - TL, downL = TL - T_at(P, T, m0[0], m0[1], m0[2]);
        double upR = T_at(P, T, a1[0], a1[1], a1[2]) - TR, downR = TR - T_at(P, T, m1[0], m1[1], m1[2]);
        if (limit)      /* limited transverse gradient, Appendix C */
            grad[e] = mc_limit(mc_limit(upL, downL), mc_limit(upR, downR)) / P->dx[e];
        else            /* mean of the four one-sided transverse differences, Eq. qT */
            grad[e] = (upL + downL + upR + downR) / (4.0 * P->dx[e]);
    }

    /* face values of b and T */
    double bf[3];
    for (int e = 0; e < 3; ++e)
        bf[e] = 0.5 * (b_at(P, b, e, c0[0], c0[1], c0[2]) + b_at(P, b, e, c1[0], c1[1], c1[2]));
    double Tf = 0.5 * (TL + TR);

    double kpar = kappa_par(P, Tf);
    double kperp = P->kappa_perp_ratio * kpar;

    /* classical flux, Eq. Fclass plus the perpendicular term of Eq. Fclass_HD */
    double bdotg = bf[0] * grad[0] + bf[1] * grad[1] + bf[2] * grad[2];
    double F[3];
    for (int e = 0; e < 3; ++e) F[e] = -kpar * bf[e] * bdotg - kperp * grad[e];

    if (!P->saturate) return F[d];

    /* saturated flux, Eq. Fsat, and the harmonic blend, Eq. Fc */
    double Fmag = sqrt(F[0] * F[0] + F[1] * F[1] + F[2] * F[2]);
    double Tq = Tf;
    if (P->sat_upwind) Tq = (F[d] >= 0.0) ? TL : TR;
    double ciso = sqrt(Tq);
    double q = 5.0 * P->phi * P->rho * ciso * ciso * ciso;
    return q / (q + Fmag) * F[d];
}

/* All face fluxes; F[d] holds, at cell c, the flux on the face c+1/2 e_d. */
void orc_flux(const orc_problem *P, const double *T, const double *b,
              double *Fx, double *Fy, double *Fz)
{
    double *F[3] = {Fx, Fy, Fz};
    for (int d = 0; d < P->ndim; ++d) {
        if (!F[d]) continue;
        #pragma omp parallel for collapse(2) schedule(static)
        for (long k = 0; k < P->n[2]; ++k)
            for (long j = 0; j < P->n[1]; ++j)
                for (long i = 0; i < P->n[0]; ++i)
                    F[d][idx(P, i, j, k)] = orc_face_flux(P, T, b, d, i, j, k);
    }
}

/*
 * Flux on face c - 1/2 e_d, from the array of c + 1/2 e_d fluxes.  Interior
 * and periodic faces are the neighbour's +face (one flux per face); the
 * Dirichlet face at the low boundary is computed from the ghost cell.
 */
static double low_face(const orc_problem *P, const double *T, const double *b,
                       const double *Fd, int d, long i, long j, long k)
{
    long c[3] = {i, j, k};
    c[d] -= 1;
    if (c[d] < 0) {
        if (P->bc == 0) c[d] += P->n[d];
        else return orc_face_flux(P, T, b, d, c[0], c[1], c[2]);
    }
    return Fd[idx(P, c[0], c[1], c[2])];
}

/* M(T) = -div F, the conservative divergence of Section 3. */
void orc_apply_M(const orc_problem *P, const double *T, const double *b, double *MT)
{
    long N = ncell(P);
    double *F[3] = {NULL, NULL, NULL};
    for (int d = 0; d < P->ndim; ++d) F[d] = (double *)malloc(sizeof(double) * N);
    orc_flux(P, T, b, F[0], F[1], F[2]);
    #pragma omp parallel for collapse(2) schedule(static)
    for (long k = 0; k < P->n[2]; ++k)
        for (long j = 0; j < P->n[1]; ++j)
            for (long i = 0; i < P->n[0]; ++i) {
                double div = 0.0;
                for (int d = 0; d < P->ndim; ++d) {
                    double Fhi = F[d][idx(P, i, j, k)];
                    double Flo = low_face(P, T, b, F[d], d, i, j, k);
                    div += (Fhi - Flo) / P->dx[d];
                }
                MT[idx(P, i, j, k)] = -div;
            }
    for (int d = 0; d < P->ndim; ++d) free(F[d]);
}

/* Eq. dt_exp with chi_d = (kappa_par + kappa_perp)(gamma-1)/rho, gamma = 2, rho = 1. */
double orc_dt_expl(const orc_problem *P, const double *T)
{
    long N = ncell(P);
    double inv = 0.0;
    for (int d = 0; d < P->ndim; ++d) inv += 1.0 / (P->dx[d] * P->dx[d]);
    double best = 0.0;
    #pragma omp parallel for reduction(max:best) schedule(static)
    for (long c = 0; c < N; ++c) {
        double chi = kappa_par(P, T[c]) * (1.0 + P->kappa_perp_ratio);
        double v = chi * inv;
        if (v > best) best = v;
    }
    return P->cp / best;
}

/* Eq. RKL-s for RKL2 solved for s, then s -> 1 + floor(s) (Section 4.1). */
int orc_num_stages(double ratio)
{
    double s = 0.5 * (-1.0 + sqrt(9.0 + 16.0 * ratio));
    return 1 + (int)floor(s);
}

/* Appendix A: b_j for the final stage count (b_0 = b_1 = b_2 = 1/3). */
static double rkl2_b(int j)
{
    if (j <= 2) return 1.0 / 3.0;
    return ((double)j * j + j - 2.0) / (2.0 * j * (j + 1.0));
}

/*
 * Appendix A coefficients, arrays of length s + 1 indexed by stage j.
 * mu[0], nu[0], nu[1], mu[1], gt[0], gt[1] are unused and set to 0;
 * mut[1] is mu~_1.
 */
void orc_coeffs(int s, double *mu, double *nu, double *mut, double *gt)
{
    double w1 = 4.0 / ((double)s * s + s - 2.0);
    for (int j = 0; j <= s; ++j) { mu[j] = nu[j] = mut[j] = gt[j] = 0.0; }
    mut[1] = rkl2_b(1) * w1;
    for (int j = 2; j <= s; ++j) {
        double bj = rkl2_b(j), bj1 = rkl2_b(j - 1), bj2 = rkl2_b(j - 2);
        double aj1 = 1.0 - bj1;
        mu[j] = (2.0 * j - 1.0) / j * bj / bj1;
        nu[j] = -((double)j - 1.0) / j * bj / bj2;
        mut[j] = mu[j] * w1;
        gt[j] = -aj1 * mut[j];
    }
}

/*
 * One stage of Eq. rkl2scheme with tau = dt.  j = 1 computes MY0 = M(Y0)
 * (stored into MY0) and Y1; j >= 2 uses Yjm1, Yjm2, Y0 and MY0.
 */
void orc_stage(const orc_problem *P, int j, int s, double dt, const double *b,
               const double *Y0, double *MY0, const double *Yjm1,
               const double *Yjm2, double *Yj)
{
    long N = ncell(P);
    double *mu = malloc(sizeof(double) * (s + 1)), *nu = malloc(sizeof(double) * (s + 1));
    double *mut = malloc(sizeof(double) * (s + 1)), *gt = malloc(sizeof(double) * (s + 1));
    orc_coeffs(s, mu, nu, mut, gt);
    if (j == 1) {
        orc_apply_M(P, Y0, b, MY0);
        for (long c = 0; c < N; ++c) Yj[c] = Y0[c] + mut[1] * dt * MY0[c];
    } else {
        double *MY = malloc(sizeof(double) * N);
        orc_apply_M(P, Yjm1, b, MY);
        for (long c = 0; c < N; ++c)
            Yj[c] = mu[j] * Yjm1[c] + nu[j] * Yjm2[c] + (1.0 - mu[j] - nu[j]) * Y0[c]
                  + mut[j] * dt * MY[c] + gt[j] * dt * MY0[c];
        free(MY);
    }
    free(mu); free(nu); free(mut); free(gt);
}

/*
 * One RKL2 super-step of length dt with s stages (s >= 2), T updated in
 * place.  If stage_min is not NULL it receives the minimum of T over all
 * cells and all stages Y_1..Y_s.  Returns s.
 */
int orc_super_step(const orc_problem *P, double dt, int s, double *T,
                   const double *b, double *stage_min)
{
    long N = ncell(P);
    size_t bytes = sizeof(double) * N;
    double *Y0 = malloc(bytes), *MY0 = malloc(bytes);
    double *buf[3] = {malloc(bytes), malloc(bytes), malloc(bytes)};
    memcpy(Y0, T, bytes);
    double mn = INFINITY;
    /* Y_j lives in buf[(j - 1) % 3]; Y_{j-2} of stage 2 is Y_0 */
    orc_stage(P, 1, s, dt, b, Y0, MY0, NULL, NULL, buf[0]);
    for (long c = 0; c < N; ++c) if (buf[0][c] < mn) mn = buf[0][c];
    double *Yjm2 = Y0, *Yjm1 = buf[0];
    for (int j = 2; j <= s; ++j) {
        double *Yj = buf[(j - 1) % 3];
        orc_stage(P, j, s, dt, b, Y0, MY0, Yjm1, Yjm2, Yj);
        for (long c = 0; c < N; ++c) if (Yj[c] < mn) mn = Yj[c];
        Yjm2 = Yjm1;
        Yjm1 = Yj;
    }
    memcpy(T, Yjm1, bytes);
    if (stage_min) *stage_min = mn;
    free(Y0); free(MY0); free(buf[0]); free(buf[1]); free(buf[2]);
    return s;
}

/* Forward Euler, the s = 1 case (Section 3.3): T <- T + dt M(T). */
void orc_euler_step(const orc_problem *P, double dt, double *T, const double *b)
{
    long N = ncell(P);
    double *MT = malloc(sizeof(double) * N);
    orc_apply_M(P, T, b, MT);
    for (long c = 0; c < N; ++c) T[c] += dt * MT[c];
    free(MT);
}

/* Total energy sum_c T_c dV (rho = 1, gamma = 2 so that E = T). */
double orc_energy(const orc_problem *P, const double *T)
{
    double dV = 1.0;
    for (int d = 0; d < P->ndim; ++d) dV *= P->dx[d];
    double sum = 0.0;
    long N = ncell(P);
    for (long c = 0; c < N; ++c) sum += T[c];
    return sum * dV;
}

/* Scalar form of Eq. rkl2scheme for dY/dt = lambda Y: returns R_s(z), z = dt*lambda. */
double orc_rkl2_scalar(int s, double z)
{
    double *mu = malloc(sizeof(double) * (s + 1)), *nu = malloc(sizeof(double) * (s + 1));
    double *mut = malloc(sizeof(double) * (s + 1)), *gt = malloc(sizeof(double) * (s + 1));
    orc_coeffs(s, mu, nu, mut, gt);
    double Y0 = 1.0, MY0 = z;                 /* tau * M * Y0 with tau*lambda = z */
    double Yjm2 = Y0, Yjm1 = Y0 + mut[1] * MY0;
    for (int j = 2; j <= s; ++j) {
        double Yj = mu[j] * Yjm1 + nu[j] * Yjm2 + (1.0 - mu[j] - nu[j]) * Y0
                  + mut[j] * z * Yjm1 + gt[j] * MY0;
        Yjm2 = Yjm1;
        Yjm1 = Yj;
    }
    free(mu); free(nu); free(mut); free(gt);
    return Yjm1;
}

/* ------------------------------------------------------------------------
 * First-order super-time-steppers of Section 3.3 (comparison methods).
 *
 * RKL1: the stability polynomial is P_s(1 + w1 z) with w1 = 2/(s^2 + s)
 * (Eq. stabpara with a_s = 0, b_s = 1), and Eq. RKL-s gives
 * dt / dt_expl = (s^2 + s)/2.  Writing the Legendre three-term recursion
 * (Eq. recLegP) at x = 1 + w1 tau M gives the stages
 *   Y_1 = Y_0 + w1 tau M(Y_0),
 *   Y_j = mu_j Y_{j-1} + nu_j Y_{j-2} + mu_j w1 tau M(Y_{j-1}),
 * with mu_j = (2j-1)/j and nu_j = -(j-1)/j.
 * ---------------------------------------------------------------------- */

/* Eq. RKL-s for RKL1 solved for s, then s -> 1 + floor(s) as for RKL2. */
int orc_num_stages_rkl1(double ratio)
{
    double s = 0.5 * (-1.0 + sqrt(1.0 + 8.0 * ratio));
    return 1 + (int)floor(s);
}

int orc_rkl1_super_step(const orc_problem *P, double dt, int s, double *T, const double *b)
{
    long N = ncell(P);
    size_t bytes = sizeof(double) * N;
    double w1 = 2.0 / ((double)s * s + s);
    double *Yjm2 = malloc(bytes), *Yjm1 = malloc(bytes), *Yj = malloc(bytes), *MY = malloc(bytes);
    memcpy(Yjm2, T, bytes);
    orc_apply_M(P, Yjm2, b, MY);
    for (long c = 0; c < N; ++c) Yjm1[c] = Yjm2[c] + w1 * dt * MY[c];
    for (int j = 2; j <= s; ++j) {
        double mu = (2.0 * j - 1.0) / j, nu = -((double)j - 1.0) / j;
        orc_apply_M(P, Yjm1, b, MY);
        for (long c = 0; c < N; ++c) Yj[c] = mu * Yjm1[c] + nu * Yjm2[c] + mu * w1 * dt * MY[c];
        double *t = Yjm2; Yjm2 = Yjm1; Yjm1 = Yj; Yj = t;
    }
    memcpy(T, Yjm1, bytes);
    free(Yjm2); free(Yjm1); free(Yj); free(MY);
    return s;
}

/* Scalar RKL1 on dY/dt = lambda Y: returns R_s(z), z = tau lambda. */
double orc_rkl1_scalar(int s, double z)
{
    double w1 = 2.0 / ((double)s * s + s);
    double Yjm2 = 1.0, Yjm1 = 1.0 + w1 * z;
    for (int j = 2; j <= s; ++j) {
        double mu = (2.0 * j - 1.0) / j, nu = -((double)j - 1.0) / j;
        double Yj = mu * Yjm1 + nu * Yjm2 + mu * w1 * z * Yjm1;
        Yjm2 = Yjm1;
        Yjm1 = Yj;
    }
    return Yjm1;
}

/* ------------------------------------------------------------------------
 * AAG-STS (Alexiades, Amiez & Gremaud 1996): N forward-Euler sub-steps with
 * damping nu,  tau_j = dt_p / ((nu - 1) cos((2j - 1) pi / (2N)) + 1 + nu),
 * whose sum is the super-step of Eq. AAG-STS,
 *   dt_h = dt_p N/(2 sqrt(nu)) [(1+sqrt nu)^(2N) - (1-sqrt nu)^(2N)]
 *                             / [(1+sqrt nu)^(2N) + (1-sqrt nu)^(2N)].
 * ---------------------------------------------------------------------- */

/* Eq. AAG-STS: dt_h / dt_p for N sub-steps. */
double orc_sts_gain(int N, double nu)
{
    double r = sqrt(nu);
    double a = pow(1.0 + r, 2.0 * N), c = pow(1.0 - r, 2.0 * N);
    return N / (2.0 * r) * (a - c) / (a + c);
}

/* Smallest N whose super-step reaches ratio * dt_p (Eq. AAG-STS). */
int orc_num_stages_sts(double ratio, double nu)
{
    int N = 1;
    while (orc_sts_gain(N, nu) < ratio && N < 100000) ++N;
    return N;
}

/* The N sub-steps of a super-step of length dt: dt_p is set to
 * dt / gain(N) (at most the explicit step) so that they sum to dt. */
void orc_sts_substeps(int N, double nu, double dt, double *tau)
{
    double dtp = dt / orc_sts_gain(N, nu);
    const double pi = 3.14159265358979323846;
    for (int j = 1; j <= N; ++j)
        tau[j - 1] = dtp / ((nu - 1.0) * cos((2.0 * j - 1.0) * pi / (2.0 * N)) + 1.0 + nu);
}

int orc_sts_super_step(const orc_problem *P, double dt, int N, double nu, double *T, const double *b)
{
    double *tau = malloc(sizeof(double) * N);
    orc_sts_substeps(N, nu, dt, tau);
    for (int j = 0; j < N; ++j) orc_euler_step(P, tau[j], T, b);
    free(tau);
    return N;
}

/* ------------------------------------------------------------------------
 * Operator splitting (Section 3): a hyperbolic step without the conduction
 * flux, then the conduction step of Eq. scalar_diffusion.  The hyperbolic
 * part here is the passive advection of the energy density by a given
 * cell-centred velocity u (3 arrays of grid size), dT/dt = -div(u T), by the
 * conservative first-order donor-cell scheme: the face velocity is the mean
 * of the two cells and the face flux carries T from the upwind cell.
 * ---------------------------------------------------------------------- */

/* Component e of u at a cell that may lie outside the grid (as b). */
static double u_at(const orc_problem *P, const double *u, int e, long i, long j, long k)
{
    return b_at(P, u, e, i, j, k);
}

/* Eq. dt_h with lambda_d = |u_d| (no sound or magnetosonic speed in a
 * passive advection): C_h / max_cells sum_d |u_d| / dx_d; 0 if u = 0. */
double orc_dt_hyp(const orc_problem *P, const double *u, double ch)
{
    long N = ncell(P);
    double best = 0.0;
    for (long c = 0; c < N; ++c) {
        double v = 0.0;
        for (int d = 0; d < P->ndim; ++d) v += fabs(u[(long)d * N + c]) / P->dx[d];
        if (v > best) best = v;
    }
    return best > 0.0 ? ch / best : 0.0;
}

/* Advective flux on the face between cell (i,j,k) and its +e_d neighbour. */
static double adv_flux(const orc_problem *P, const double *T, const double *u, int d, long i, long j, long k)
{
    long c1[3] = {i, j, k};
    c1[d] += 1;
    double uf = 0.5 * (u_at(P, u, d, i, j, k) + u_at(P, u, d, c1[0], c1[1], c1[2]));
    double Tup = uf >= 0.0 ? T_at(P, T, i, j, k) : T_at(P, T, c1[0], c1[1], c1[2]);
    return uf * Tup;
}

/* One donor-cell step: T_out = T - dt sum_d (F_d(c+1/2) - F_d(c-1/2)) / dx_d. */
void orc_advect(const orc_problem *P, double dt, const double *T, const double *u, double *Tout)
{
    #pragma omp parallel for collapse(2) schedule(static)
    for (long k = 0; k < P->n[2]; ++k)
        for (long j = 0; j < P->n[1]; ++j)
            for (long i = 0; i < P->n[0]; ++i) {
                double div = 0.0;
                for (int d = 0; d < P->ndim; ++d) {
                    long lo[3] = {i, j, k};
                    lo[d] -= 1;
                    div += (adv_flux(P, T, u, d, i, j, k) - adv_flux(P, T, u, d, lo[0], lo[1], lo[2])) / P->dx[d];
                }
                Tout[idx(P, i, j, k)] = T[idx(P, i, j, k)] - dt * div;
            }
}

int orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
