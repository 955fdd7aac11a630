/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle for the modified lattice BGK
 * model of Wang, Mi and Guo, "A modified lattice Bhatnagar-Gross-Krook model
 * for convection heat transfer in porous media" (arXiv 1505.02976).
 *
 * TEST INFRASTRUCTURE.  This file is the independent reference that the CUDA
 * path is checked against.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may build, load or call it.  It shares no
 * code, header, table or constant with the CUDA library: the lattice is built
 * here from the paper's own cos/sin definition (Sec. 3.1), every tensor
 * contraction is written out as an explicit loop over Cartesian indices, and
 * the 2x2 system for the temperature gradient is solved by Gaussian
 * elimination, never by a closed-form inverse.
 *
 * What it computes, in the paper's notation (lattice units dx = dt = 1):
 *   flow LBE                 Eq. (LBEeq)        Sec. 3.1
 *   flow EDF with eps, S     Eqs. (EQFIN), (EQTSHIN)
 *   forcing term F_i         Eq. (FtermF)
 *   total force F            Eq. (ForceEq),  G = g beta (T - T0) j + a
 *   Ergun F_eps and K        Sec. 2 (Ergun relations)
 *   p, u, quadratic solve    Sec. 3.1 (pressure / velocity definitions),
 *                            p closed forms of s_0 and F_0 in Appendix A
 *   thermal LBE + EDF        Eqs. (LBEHeq), (TeEDFEQ), P_i (Eq:Tforce), Q_i
 *   sigma T = sum g + Q/2    Sec. 3.2
 *   local shear rate S       Eq. (ShearEqCom)   Sec. 3.3
 *   local grad T             Eqs. (TeEqCom)-(MatrN)
 *   NEES velocity BC         Eqs. (FNEESEQFIN), (NEESVel)   Sec. 3.4
 *   NEES Dirichlet-T BC      Eqs. (TeEBounDFEQ), (TNEESAp)
 *   NEES Neumann-T BC        Eq. (TNEESApGra)
 *   A and B from Ra, Pr, Ma  Eq. (EQA&B)        Sec. 4
 *   Nusselt number           Eq. (Eq:AvNuss)
 *   steady-state criterion   Sec. 4 (relative change over 100 steps)
 *
 * Readings of points the paper leaves open (each one is listed, with its
 * reason, in the design notes of the repository):
 *   - the temperature lattice is D2Q9 with the flow weights;
 *   - wall nodes are the outermost lattice nodes, L = N - 1;
 *   - NEES rebuilds the post-streaming populations of a wall node from the
 *     post-streaming state of x_f, and the wall node is then collided with the
 *     same equilibrium it was rebuilt with; its force uses u_b and T_b;
 *   - on an adiabatic wall p(x_f) replaces p(x_b) and grad T_b is grad T(x_f)
 *     with its wall-normal component set to the prescribed value 0;
 *   - a corner takes the temperature and velocity of its x-wall when that wall
 *     is Dirichlet, else of its y-wall; x_f is the diagonal neighbour;
 *   - the local Nusselt number uses the second-order one-sided difference and
 *     the mean is the trapezoid rule over the wall nodes divided by H = N - 1.
 *
 * State layout: f[i][y][x] and g[i][y][x], i = 0..8, doubles, holding the
 * POST-COLLISION populations of the last completed step.  One step streams
 * (pull) and collides.  All nine populations are kept (f_0 only feeds the mass
 * diagnostic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* The same source builds twice: with real_t = double (the oracle), and with
 * real_t = double complex (-DORC_COMPLEX) for complex-step derivatives: a
 * tiny imaginary perturbation h of one input gives d(output)/d(input) as
 * Im(output)/h to machine precision, with no subtraction.  Comparisons and
 * pivot choices look at real parts only. */
#ifdef ORC_COMPLEX
#include <complex.h>
typedef double complex real_t;
#define RSQRT(x) csqrt(x)
#define RE(x) creal(x)
#else
typedef double real_t;
#define RSQRT(x) sqrt(x)
#define RE(x) (x)
#endif

/* ------------------------------------------------------------------ lattice */

static int CX[9], CY[9];
static double WGT[9];
static double VARPI[9];
static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2 / 3 with c = 1 */
static int lattice_ready = 0;

/* D2Q9 velocities from their definition in Sec. 3.1:
 * c_0 = 0; c_i = (cos((i-1)pi/2), sin((i-1)pi/2)) for i = 1..4;
 * c_i = sqrt(2) (cos((i-5)pi/2 + pi/4), sin((i-5)pi/2 + pi/4)) for i = 5..8.
 * Weights 4/9, 1/9, 1/36; varpi_i = w_i (i != 0), varpi_0 = -sum_{i!=0} varpi_i
 * (Eq. TeEDFEQ). */
static void lattice_init(void) {
    if (lattice_ready) return;
    const double pi = 3.14159265358979323846;
    CX[0] = 0; CY[0] = 0;
    for (int i = 1; i <= 4; ++i) {
        double a = (i - 1) * pi / 2.0;
        CX[i] = (int)lround(cos(a));
        CY[i] = (int)lround(sin(a));
    }
    for (int i = 5; i <= 8; ++i) {
        double a = (i - 5) * pi / 2.0 + pi / 4.0;
        CX[i] = (int)lround(sqrt(2.0) * cos(a));
        CY[i] = (int)lround(sqrt(2.0) * sin(a));
    }
    WGT[0] = 4.0 / 9.0;
    for (int i = 1; i <= 4; ++i) WGT[i] = 1.0 / 9.0;
    for (int i = 5; i <= 8; ++i) WGT[i] = 1.0 / 36.0;
    double s = 0.0;
    for (int i = 1; i < 9; ++i) { VARPI[i] = WGT[i]; s += VARPI[i]; }
    VARPI[0] = -s;
    lattice_ready = 1;
}

/* ----------------------------------------------------------- problem types */

enum { ORC_PERIODIC = 0, ORC_WALL_DIRICHLET = 1, ORC_WALL_ADIABATIC = 2 };
enum { SIDE_W = 0, SIDE_E = 1, SIDE_S = 2, SIDE_N = 3 };

/* Problem statement (Sec. 2 and Sec. 4).  A value of NaN in one of the
 * override fields means "derive it from the dimensionless groups". */
typedef struct {
    int32_t nx, ny;
    int32_t bc[4];        /* W, E, S, N */
    int32_t forchheimer;  /* 1: F_eps from the Ergun relation, 0: F_eps = 0 */
    int32_t da_infinite;  /* 1: K -> infinity, no drag */
    double Ra, Pr, Da, J, eps, sigma, Ma;
    double tau_f, tau_T;
    double Th, Tc, T_init, rho0, Q, ax, ay;
    double L;                            /* characteristic length; NaN: nx - 1 */
    double nu, alpha_e, gbeta, A, B, K;  /* overrides; NaN: derive */
    double T_bc[4];                      /* Dirichlet wall temperature per side */
    double u_bc[4][2];                   /* wall velocity per side */
    double T0;                           /* buoyancy reference; NaN: (Th + Tc) / 2 */
    double Ra_I;                         /* internal Rayleigh number, for Q = NaN */
} orc_problem;

/* Lattice constants derived from the problem statement. */
typedef struct {
    double L, T0, dT, U, gbeta, nu, nu_e, alpha_e, A, B, K, Feps, Q;
    double kappa_f, kappa_T; /* (1 - 1/(2 tau)) */
} orc_derived;

/* Porosity-dependent constants of one node, and the y-component of the
 * external acceleration a at the node's row. */
typedef struct {
    real_t eps, nu_over_K, Feps_over_sqrtK, c0, c1;
    double ay;
} orc_cell;

/* Optional external acceleration a_y(y) added to the problem's uniform a_y,
 * one value per row (the mixed-convection channel of Sec. 4.1 drives its
 * flow with such a profile).  Test infrastructure: one profile at a time. */
static double *g_ay_profile = NULL;
static int g_ay_rows = 0;
int orc_set_ay_profile(const double *ay, int ny) {
    free(g_ay_profile);
    g_ay_profile = NULL;
    g_ay_rows = 0;
    if (ay && ny > 0) {
        g_ay_profile = (double *)malloc(sizeof(double) * (size_t)ny);
        if (!g_ay_profile) return 100;
        memcpy(g_ay_profile, ay, sizeof(double) * (size_t)ny);
        g_ay_rows = ny;
    }
    return 0;
}

/* Everything a node update needs. */
typedef struct {
    const orc_problem *pb;
    orc_derived d;
    const real_t *eps_field; /* [ny][nx] or NULL */
} orc_ctx;

/* Moments of one node (or the boundary state of a wall node). */
typedef struct {
    real_t T, u[2], F[2], p, S[2][2], gradT[2];
} orc_state;

static int is_nan(real_t v) { return v != v; }

/* Threads for the loops over nodes.  Every node of a step is computed from
 * the previous state alone and written to its own slots, so the rows may be
 * shared among threads without changing a single bit of the result; the
 * sums (totals, residual, Nusselt mean) stay single-threaded, in node order.
 * 0 (the default) means one thread per processor. */
static int g_threads = 0;
int orc_set_threads(int n) { g_threads = n < 0 ? 0 : n; return 0; }
int orc_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_num_procs();
#else
    return 1;
#endif
}

/* Derivation of the lattice constants.  U = Ma c_s is the characteristic
 * velocity of Sec. 4; g beta, nu and alpha_e invert the definitions of Ra and
 * Pr (Sec. 2) with U^2 = g beta dT L; nu_e = J nu; A and B from
 * nu_e = c_s^2 (tau_f - A - 1/2) and alpha_e = sigma c_s^2 (tau_T - B - 1/2)
 * (Appendix A and Eq. Therdiff), which for J = 1 is exactly Eq. (EQA&B);
 * K = Da L^2 (Sec. 2); F_eps = 1.75 / RSQRT(150 eps^3) (Ergun). */
int orc_derive(const orc_problem *pb, orc_derived *d) {
    lattice_init();
    memset(d, 0, sizeof(*d));
    d->L = is_nan(pb->L) ? (real_t)(pb->nx - 1) : pb->L;
    d->T0 = is_nan(pb->T0) ? 0.5 * (pb->Th + pb->Tc) : pb->T0;
    d->dT = pb->Th - pb->Tc;
    d->U = pb->Ma * RSQRT(CS2);
    if (!is_nan(pb->gbeta)) d->gbeta = pb->gbeta;
    else d->gbeta = d->U * d->U / (d->dT * d->L);
    if (!is_nan(pb->nu)) d->nu = pb->nu;
    else if (!is_nan(pb->A)) d->nu = CS2 * (pb->tau_f - pb->A - 0.5) / pb->J;
    else d->nu = d->U * d->L * RSQRT(pb->Pr / pb->Ra);
    d->nu_e = pb->J * d->nu;
    if (!is_nan(pb->alpha_e)) d->alpha_e = pb->alpha_e;
    else if (!is_nan(pb->B)) d->alpha_e = pb->sigma * CS2 * (pb->tau_T - pb->B - 0.5);
    else d->alpha_e = d->nu / pb->Pr;
    d->A = is_nan(pb->A) ? pb->tau_f - 0.5 - d->nu_e / CS2 : pb->A;
    d->B = is_nan(pb->B) ? pb->tau_T - 0.5 - d->alpha_e / (pb->sigma * CS2) : pb->B;
    if (pb->da_infinite) d->K = INFINITY;
    else d->K = is_nan(pb->K) ? pb->Da * d->L * d->L : pb->K;
    d->Feps = pb->forchheimer ? 1.75 / RSQRT(150.0 * pb->eps * pb->eps * pb->eps) : 0.0;
    /* internal heat source of Sec. 4.4, Q = Ra_I alpha_e dT / (Ra L^2) */
    d->Q = is_nan(pb->Q) ? pb->Ra_I * d->alpha_e * d->dT / (pb->Ra * d->L * d->L) : pb->Q;
    d->kappa_f = 1.0 - 1.0 / (2.0 * pb->tau_f);
    d->kappa_T = 1.0 - 1.0 / (2.0 * pb->tau_T);
    /* admissibility (Sec. 4): 0 < eps <= 1, tau > 1/2, A < tau_f - 1/2,
     * B < tau_T - 1/2 */
    if (!(pb->eps > 0.0 && pb->eps <= 1.0)) return 1;
    if (!(pb->tau_f > 0.5 && pb->tau_T > 0.5)) return 2;
    if (!(d->A < pb->tau_f - 0.5)) return 3;
    if (!(d->B < pb->tau_T - 0.5)) return 4;
    if (!(pb->sigma > 0.0 && pb->rho0 > 0.0)) return 5;
    if (pb->nx < 1 || pb->ny < 1) return 6;
    if ((pb->bc[SIDE_W] == ORC_PERIODIC) != (pb->bc[SIDE_E] == ORC_PERIODIC)) return 7;
    if ((pb->bc[SIDE_S] == ORC_PERIODIC) != (pb->bc[SIDE_N] == ORC_PERIODIC)) return 7;
    if (pb->bc[SIDE_W] != ORC_PERIODIC && pb->nx < 4) return 6;
    if (pb->bc[SIDE_S] != ORC_PERIODIC && pb->ny < 4) return 6;
    return 0;
}

/* K and F_eps at porosity eps.  A porosity field scales K with the
 * Kozeny-Carman form of the Ergun permeability, K ~ eps^3 / (1 - eps)^2
 * (Sec. 2), anchored at K(eps_ref) = Da L^2 with eps_ref the scalar eps. */
static void cell_constants(const orc_ctx *cx, real_t eps, orc_cell *c) {
    const orc_problem *pb = cx->pb;
    real_t K = cx->d.K, Feps = cx->d.Feps;
    if (cx->eps_field && !pb->da_infinite) {
        real_t er = pb->eps;
        real_t kc = (eps * eps * eps / ((1.0 - eps) * (1.0 - eps)))
                  / (er * er * er / ((1.0 - er) * (1.0 - er)));
        K = cx->d.K * kc;
        Feps = pb->forchheimer ? 1.75 / RSQRT(150.0 * eps * eps * eps) : 0.0;
    }
    c->eps = eps;
    c->nu_over_K = isinf(RE(K)) ? 0.0 : cx->d.nu / K;
    c->Feps_over_sqrtK = isinf(RE(K)) ? 0.0 : Feps / RSQRT(K);
    c->c0 = 0.5 * (1.0 + eps * 0.5 * c->nu_over_K);
    c->c1 = eps * 0.5 * c->Feps_over_sqrtK;
    c->ay = pb->ay;
}

static real_t node_eps(const orc_ctx *cx, int x, int y) {
    return cx->eps_field ? cx->eps_field[(size_t)y * cx->pb->nx + x] : cx->pb->eps;
}

/* Constants of node (x, y): its porosity and its row's a_y. */
static void node_cell(const orc_ctx *cx, int x, int y, orc_cell *c) {
    cell_constants(cx, node_eps(cx, x, y), c);
    if (g_ay_profile && y < g_ay_rows) c->ay = cx->pb->ay + g_ay_profile[y];
}

/* ------------------------------------------------ per-direction functions */

/* X : (c_i c_i - c_s^2 I) for a 2x2 tensor X, index by index. */
static real_t contract_ccI(int i, real_t X[2][2]) {
    double c[2] = {(double)CX[i], (double)CY[i]};
    real_t s = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            s += X[a][b] * (c[a] * c[b] - CS2 * (a == b ? 1.0 : 0.0));
    return s;
}

static real_t dot_c(int i, const real_t v[2]) { return CX[i] * v[0] + CY[i] * v[1]; }

/* s_i(u) of Eq. (EQTSHIN). */
static real_t s_i(int i, const real_t u[2], real_t eps) {
    real_t uu[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) uu[a][b] = u[a] * u[b];
    return WGT[i] * (dot_c(i, u) / CS2 + contract_ccI(i, uu) / (2.0 * eps * CS2 * CS2));
}

/* r_i of Eq. (EQTSHIN) (dt = 1). */
static real_t r_i(int i, real_t A, real_t S[2][2]) {
    return WGT[i] * A * contract_ccI(i, S) / (2.0 * CS2);
}

/* Flow EDF, Eq. (EQFIN); with_r = 0 gives f^{e(0)} of Appendix A. */
static void flow_eq(const orc_ctx *cx, const orc_cell *c, real_t p, const real_t u[2],
                    real_t S[2][2], int with_r, real_t out[9]) {
    real_t rho0 = cx->pb->rho0, A = cx->d.A, eps = c->eps;
    for (int i = 0; i < 9; ++i) {
        real_t r = with_r ? r_i(i, A, S) : 0.0;
        if (i == 0)
            out[i] = rho0 - (1.0 - WGT[0]) * eps * p / CS2 + rho0 * s_i(0, u, eps) + rho0 * r;
        else
            out[i] = WGT[i] * eps * p / CS2 + rho0 * s_i(i, u, eps) + rho0 * r;
    }
}

/* Forcing term F_i, Eq. (FtermF). */
static void flow_force_terms(const orc_ctx *cx, const orc_cell *c, const real_t u[2],
                             const real_t F[2], real_t out[9]) {
    real_t rho0 = cx->pb->rho0, eps = c->eps, kf = cx->d.kappa_f;
    real_t uFFu[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) uFFu[a][b] = u[a] * F[b] + F[a] * u[b];
    for (int i = 0; i < 9; ++i)
        out[i] = WGT[i] * rho0 * kf *
                 (dot_c(i, F) / CS2 + contract_ccI(i, uFFu) / (2.0 * eps * CS2 * CS2));
}

/* Temperature EDF, Eq. (TeEDFEQ); with_grad = 0 gives g^{e(0)} of Sec. 3.2. */
static void thermal_eq(const orc_ctx *cx, const orc_cell *c, real_t T, const real_t u[2],
                       real_t p, const real_t gradT[2], int with_grad, real_t out[9]) {
    real_t sigma = cx->pb->sigma, rho0 = cx->pb->rho0, eps = c->eps, B = cx->d.B;
    real_t uu[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) uu[a][b] = u[a] * u[b];
    for (int i = 0; i < 9; ++i) {
        real_t v = WGT[i] * T *
                       (sigma + dot_c(i, u) / CS2 + contract_ccI(i, uu) / (2.0 * eps * CS2 * CS2)) +
                   VARPI[i] * T * eps * p / (CS2 * rho0);
        if (with_grad) v += sigma * WGT[i] * B * dot_c(i, gradT);
        out[i] = v;
    }
}

/* Source P_i, Eq. (Eq:Tforce). uu:(c_i gradT) = sum_ab u_a u_b c_a dT/dx_b. */
static void thermal_P(const orc_ctx *cx, const orc_cell *c, real_t T, const real_t u[2],
                      real_t p, const real_t F[2], const real_t gradT[2], real_t out[9]) {
    real_t sigma = cx->pb->sigma, rho0 = cx->pb->rho0, eps = c->eps, kT = cx->d.kappa_T;
    real_t w[2];
    for (int a = 0; a < 2; ++a) w[a] = T * F[a] + eps * p * gradT[a] / rho0;
    for (int i = 0; i < 9; ++i) {
        double ci[2] = {(double)CX[i], (double)CY[i]};
        real_t uuc = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) uuc += u[a] * u[b] * ci[a] * gradT[b];
        out[i] = WGT[i] * kT * (dot_c(i, w) / CS2 + (1.0 / eps - 1.0 / sigma) * uuc / CS2);
    }
}

/* Source Q_i of Sec. 3.2. */
static void thermal_Q(const orc_ctx *cx, const real_t u[2], real_t out[9]) {
    real_t sigma = cx->pb->sigma, kT = cx->d.kappa_T, Q = cx->d.Q;
    for (int i = 0; i < 9; ++i) out[i] = WGT[i] * kT * (1.0 + dot_c(i, u) / (sigma * CS2)) * Q;
}

/* Total force, Eq. (ForceEq), with G = g beta (T - T0) j + a. */
static void total_force(const orc_ctx *cx, const orc_cell *c, real_t T, const real_t u[2],
                        real_t F[2]) {
    real_t G[2] = {cx->pb->ax, cx->d.gbeta * (T - cx->d.T0) + c->ay};
    real_t umag = RSQRT(u[0] * u[0] + u[1] * u[1]);
    for (int a = 0; a < 2; ++a)
        F[a] = -c->eps * c->nu_over_K * u[a] - c->eps * c->Feps_over_sqrtK * umag * u[a] +
               c->eps * G[a];
}

/* Velocity from the temporary velocity v (Sec. 3.1). */
static void velocity_from_v(const orc_cell *c, const real_t v[2], real_t u[2]) {
    real_t vmag = RSQRT(v[0] * v[0] + v[1] * v[1]);
    real_t den = c->c0 + RSQRT(c->c0 * c->c0 + c->c1 * vmag);
    u[0] = v[0] / den;
    u[1] = v[1] / den;
}

/* Solve the 2x2 system M x = N by Gaussian elimination with partial
 * pivoting.  Returns 0, or 1 when M is singular. */
static int solve2(real_t M[2][2], const real_t N[2], real_t x[2]) {
    real_t a[2][3] = {{M[0][0], M[0][1], N[0]}, {M[1][0], M[1][1], N[1]}};
    if (fabs(RE(a[1][0])) > fabs(RE(a[0][0]))) {
        for (int k = 0; k < 3; ++k) { real_t t = a[0][k]; a[0][k] = a[1][k]; a[1][k] = t; }
    }
    if (RE(a[0][0]) == 0.0) return 1;
    real_t m = a[1][0] / a[0][0];
    for (int k = 0; k < 3; ++k) a[1][k] -= m * a[0][k];
    if (RE(a[1][1]) == 0.0) return 1;
    x[1] = a[1][2] / a[1][1];
    x[0] = (a[0][2] - a[0][1] * x[1]) / a[0][0];
    return 0;
}

/* Moments of one node from its post-streaming populations (Sec. 3.1-3.3):
 * T first (this step's g), then buoyancy, v, u, F, p, S, grad T. */
static void node_moments(const orc_ctx *cx, const orc_cell *c, const real_t fs[9],
                         const real_t gs[9], orc_state *m) {
    const orc_problem *pb = cx->pb;
    real_t rho0 = pb->rho0, eps = c->eps, sigma = pb->sigma;
    /* sigma T = sum_i g_i + (dt/2) Q */
    real_t sg = 0.0;
    for (int i = 0; i < 9; ++i) sg += gs[i];
    m->T = (sg + 0.5 * cx->d.Q) / sigma;
    /* v = sum_i c_i f_i / rho0 + (dt/2) eps G */
    real_t G[2] = {pb->ax, cx->d.gbeta * (m->T - cx->d.T0) + c->ay};
    real_t v[2] = {0.0, 0.0};
    for (int i = 0; i < 9; ++i) { v[0] += CX[i] * fs[i]; v[1] += CY[i] * fs[i]; }
    for (int a = 0; a < 2; ++a) v[a] = v[a] / rho0 + 0.5 * eps * G[a];
    velocity_from_v(c, v, m->u);
    total_force(cx, c, m->T, m->u, m->F);
    /* p = c_s^2 / (eps (1 - w_0)) [sum_{i!=0} f_i + tau_f dt F_0 + rho0 s_0(u)] */
    real_t Fi[9];
    flow_force_terms(cx, c, m->u, m->F, Fi);
    real_t sf = 0.0;
    for (int i = 1; i < 9; ++i) sf += fs[i];
    m->p = CS2 / (eps * (1.0 - WGT[0])) * (sf + pb->tau_f * Fi[0] + rho0 * s_i(0, m->u, eps));
    /* S, Eq. (ShearEqCom) */
    real_t fe0[9], zero[2][2] = {{0, 0}, {0, 0}};
    flow_eq(cx, c, m->p, m->u, zero, 0, fe0);
    real_t Pi[2][2] = {{0, 0}, {0, 0}};
    for (int i = 0; i < 9; ++i) {
        double ci[2] = {(double)CX[i], (double)CY[i]};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) Pi[a][b] += ci[a] * ci[b] * (fs[i] - fe0[i]);
    }
    real_t den = CS2 * rho0 * (cx->d.A - pb->tau_f);
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            m->S[a][b] = (Pi[a][b] + 0.5 * rho0 * (m->u[a] * m->F[b] + m->F[a] * m->u[b]) / eps) / den;
    /* grad T, Eqs. (TeEqCom)-(MatrN) */
    real_t ge0[9], g0[2] = {0.0, 0.0};
    thermal_eq(cx, c, m->T, m->u, m->p, g0, 0, ge0);
    real_t N[2] = {0.0, 0.0};
    for (int i = 0; i < 9; ++i) { N[0] += CX[i] * (gs[i] - ge0[i]); N[1] += CY[i] * (gs[i] - ge0[i]); }
    for (int a = 0; a < 2; ++a) N[a] += 0.5 * (m->T * m->F[a] + m->u[a] * cx->d.Q / sigma);
    real_t M[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            M[a][b] = (-eps * m->p / (2.0 * rho0) + CS2 * sigma * (cx->d.B - pb->tau_T)) * (a == b ? 1.0 : 0.0) -
                      0.5 * (1.0 / eps - 1.0 / sigma) * m->u[a] * m->u[b];
    if (solve2(M, N, m->gradT)) { m->gradT[0] = NAN; m->gradT[1] = NAN; }
}

/* ------------------------------------------------------------ the lattice */

static int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* Post-streaming population i at (x, y): the post-collision value that
 * streamed in from x - c_i (streaming step of Sec. 3.2, pull form). */
static real_t pull(const orc_ctx *cx, const real_t *h, int i, int x, int y) {
    int nx = cx->pb->nx, ny = cx->pb->ny;
    int xs = wrap(x - CX[i], nx), ys = wrap(y - CY[i], ny);
    return h[((size_t)i * ny + ys) * nx + xs];
}

typedef struct {
    int wall;
    int xf, yf, xff, yff;
    int dirichlet;
    real_t Tb;
    real_t ub[2];
    int fixed_grad[2]; /* wall-normal gradient components prescribed (= 0) */
} orc_wall;

#ifdef ORC_COMPLEX
/* Imaginary parts added to the Dirichlet wall temperatures (complex build). */
static double g_tbc_imag[4];
int orc_cs_set_tbc_imag(const double im[4]) {
    for (int k = 0; k < 4; ++k) g_tbc_imag[k] = im[k];
    return 0;
}
static real_t tbc_value(const orc_problem *pb, int side) { return pb->T_bc[side] + I * g_tbc_imag[side]; }
#else
static real_t tbc_value(const orc_problem *pb, int side) { return pb->T_bc[side]; }
#endif

static void classify(const orc_ctx *cx, int x, int y, orc_wall *w) {
    const orc_problem *pb = cx->pb;
    int onW = (x == 0 && pb->bc[SIDE_W] != ORC_PERIODIC);
    int onE = (x == pb->nx - 1 && pb->bc[SIDE_E] != ORC_PERIODIC);
    int onS = (y == 0 && pb->bc[SIDE_S] != ORC_PERIODIC);
    int onN = (y == pb->ny - 1 && pb->bc[SIDE_N] != ORC_PERIODIC);
    memset(w, 0, sizeof(*w));
    if (!(onW || onE || onS || onN)) return;
    w->wall = 1;
    int dx = onW ? 1 : (onE ? -1 : 0);
    int dy = onS ? 1 : (onN ? -1 : 0);
    w->xf = x + dx; w->yf = y + dy;
    w->xff = x + 2 * dx; w->yff = y + 2 * dy;
    int xs = onW ? SIDE_W : (onE ? SIDE_E : -1);
    int ys = onS ? SIDE_S : (onN ? SIDE_N : -1);
    int tside = -1;
    if (xs >= 0 && pb->bc[xs] == ORC_WALL_DIRICHLET) tside = xs;
    else if (ys >= 0 && pb->bc[ys] == ORC_WALL_DIRICHLET) tside = ys;
    if (tside >= 0) { w->dirichlet = 1; w->Tb = tbc_value(pb, tside); }
    else {
        w->dirichlet = 0;
        w->fixed_grad[0] = (xs >= 0);
        w->fixed_grad[1] = (ys >= 0);
    }
    int uside = xs >= 0 ? xs : ys;
    w->ub[0] = pb->u_bc[uside][0];
    w->ub[1] = pb->u_bc[uside][1];
}

/* Post-streaming state of node (x, y).  Interior nodes: their own moments.
 * Wall nodes: the boundary state used by NEES (Sec. 3.4): u_b, T_b, p(x_f),
 * S(x_f), grad T_b, F at (u_b, T_b).  When rebuilt is non-NULL the wall
 * node's rebuilt post-streaming populations (Eqs. NEESVel, TNEESAp) are
 * written there; for interior nodes the pulled populations are. */
static void node_state(const orc_ctx *cx, const real_t *f, const real_t *g, int x, int y,
                       orc_state *st, real_t fr[9], real_t gr[9]) {
    orc_wall w;
    classify(cx, x, y, &w);
    orc_cell c;
    node_cell(cx, x, y, &c);
    if (!w.wall) {
        real_t fs[9], gs[9];
        for (int i = 0; i < 9; ++i) { fs[i] = pull(cx, f, i, x, y); gs[i] = pull(cx, g, i, x, y); }
        node_moments(cx, &c, fs, gs, st);
        if (fr) for (int i = 0; i < 9; ++i) { fr[i] = fs[i]; gr[i] = gs[i]; }
        return;
    }
    /* state at x_f from its own post-streaming populations */
    orc_cell cf;
    node_cell(cx, w.xf, w.yf, &cf);
    real_t ff[9], gf[9];
    for (int i = 0; i < 9; ++i) { ff[i] = pull(cx, f, i, w.xf, w.yf); gf[i] = pull(cx, g, i, w.xf, w.yf); }
    orc_state sf;
    node_moments(cx, &cf, ff, gf, &sf);
    /* boundary values */
    st->u[0] = w.ub[0]; st->u[1] = w.ub[1];
    st->p = sf.p;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) st->S[a][b] = sf.S[a][b];
    st->gradT[0] = sf.gradT[0]; st->gradT[1] = sf.gradT[1];
    if (w.dirichlet) {
        st->T = w.Tb;
    } else {
        /* Eq. (TNEESApGra) with a zero prescribed normal gradient */
        orc_cell cff;
        node_cell(cx, w.xff, w.yff, &cff);
        real_t fff[9], gff[9];
        for (int i = 0; i < 9; ++i) { fff[i] = pull(cx, f, i, w.xff, w.yff); gff[i] = pull(cx, g, i, w.xff, w.yff); }
        orc_state sff;
        node_moments(cx, &cff, fff, gff, &sff);
        for (int a = 0; a < 2; ++a)
            if (w.fixed_grad[a]) st->gradT[a] = 0.0;
        real_t dl = 0.0; /* Delta . grad T_b, Delta = x_f - x_b */
        dl += (w.xf - x) * st->gradT[0] * w.fixed_grad[0];
        dl += (w.yf - y) * st->gradT[1] * w.fixed_grad[1];
        st->T = (4.0 * sf.T - sff.T - 2.0 * dl) / 3.0;
    }
    total_force(cx, &c, st->T, st->u, st->F);
    if (fr) {
        /* f(x_b) = f^eq(x_b) + [f(x_f) - f^eq(x_f)], Eq. (NEESVel) */
        real_t eqb[9], eqf[9];
        flow_eq(cx, &c, st->p, st->u, st->S, 1, eqb);
        flow_eq(cx, &cf, sf.p, sf.u, sf.S, 1, eqf);
        for (int i = 0; i < 9; ++i) fr[i] = eqb[i] + (ff[i] - eqf[i]);
        /* g(x_b) = g^eq(x_b) + [g(x_f) - g^eq(x_f)], Eq. (TNEESAp) */
        thermal_eq(cx, &c, st->T, st->u, st->p, st->gradT, 1, eqb);
        thermal_eq(cx, &cf, sf.T, sf.u, sf.p, sf.gradT, 1, eqf);
        for (int i = 0; i < 9; ++i) gr[i] = eqb[i] + (gf[i] - eqf[i]);
    }
}

/* One node of one time step: stream (pull), rebuild walls, collide
 * (Eqs. LBEeq and TEqColli). */
static void node_update(const orc_ctx *cx, const real_t *f, const real_t *g, int x, int y,
                        real_t fo[9], real_t go[9]) {
    orc_state st;
    real_t fr[9], gr[9];
    node_state(cx, f, g, x, y, &st, fr, gr);
    orc_cell c;
    node_cell(cx, x, y, &c);
    real_t feq[9], Fi[9], geq[9], Pi[9], Qi[9];
    flow_eq(cx, &c, st.p, st.u, st.S, 1, feq);
    flow_force_terms(cx, &c, st.u, st.F, Fi);
    thermal_eq(cx, &c, st.T, st.u, st.p, st.gradT, 1, geq);
    thermal_P(cx, &c, st.T, st.u, st.p, st.F, st.gradT, Pi);
    thermal_Q(cx, st.u, Qi);
    const orc_problem *pb = cx->pb;
    for (int i = 0; i < 9; ++i) {
        fo[i] = fr[i] - (fr[i] - feq[i]) / pb->tau_f + Fi[i];
        go[i] = gr[i] - (gr[i] - geq[i]) / pb->tau_T + Pi[i] + Qi[i];
    }
}

static int make_ctx(const orc_problem *pb, const real_t *eps_field, orc_ctx *cx) {
    cx->pb = pb;
    cx->eps_field = eps_field;
    return orc_derive(pb, &cx->d);
}

/* ------------------------------------------------------------ public API */

#ifndef ORC_COMPLEX
int orc_lattice(int32_t cx_out[9], int32_t cy_out[9], double w_out[9], double varpi_out[9]) {
    lattice_init();
    for (int i = 0; i < 9; ++i) { cx_out[i] = CX[i]; cy_out[i] = CY[i]; w_out[i] = WGT[i]; varpi_out[i] = VARPI[i]; }
    return 0;
}

/* derived: L, T0, dT, U, gbeta, nu, nu_e, alpha_e, A, B, K, Feps, Q (13 values) */
int orc_derived_values(const orc_problem *pb, double out[13]) {
    orc_derived d;
    int rc = orc_derive(pb, &d);
    double v[13] = {d.L, d.T0, d.dT, d.U, d.gbeta, d.nu, d.nu_e, d.alpha_e, d.A, d.B, d.K, d.Feps, d.Q};
    memcpy(out, v, sizeof(v));
    return rc;
}

/* One-cell building blocks, exposed for the identity tests.  S is row-major
 * [Sxx, Sxy, Syx, Syy]; which selects the function. */
int orc_cell_eval(const orc_problem *pb, int which, double eps, double T, const double u[2],
                  double p, const double S4[4], const double F[2], const double gradT[2],
                  double out[9]) {
    orc_ctx cx;
    int rc = make_ctx(pb, NULL, &cx);
    if (rc) return rc;
    orc_cell c;
    cell_constants(&cx, eps, &c);
    c.eps = eps;
    double S[2][2] = {{S4[0], S4[1]}, {S4[2], S4[3]}};
    switch (which) {
    case 0: flow_eq(&cx, &c, p, u, S, 0, out); break;        /* f^{e(0)} */
    case 1: flow_eq(&cx, &c, p, u, S, 1, out); break;        /* f^{eq} */
    case 2: flow_force_terms(&cx, &c, u, F, out); break;     /* F_i */
    case 3: thermal_eq(&cx, &c, T, u, p, gradT, 0, out); break; /* g^{e(0)} */
    case 4: thermal_eq(&cx, &c, T, u, p, gradT, 1, out); break; /* g^{eq} */
    case 5: thermal_P(&cx, &c, T, u, p, F, gradT, out); break;  /* P_i */
    case 6: thermal_Q(&cx, u, out); break;                      /* Q_i */
    default: return -1;
    }
    return 0;
}

/* Moments of one node from given post-streaming populations.
 * out = [T, ux, uy, Fx, Fy, p, Sxx, Sxy, Syx, Syy, dTdx, dTdy] */
int orc_cell_moments(const orc_problem *pb, double eps, const double fs[9], const double gs[9],
                     double out[12]) {
    orc_ctx cx;
    int rc = make_ctx(pb, NULL, &cx);
    if (rc) return rc;
    orc_cell c;
    cell_constants(&cx, eps, &c);
    orc_state m;
    node_moments(&cx, &c, fs, gs, &m);
    double v[12] = {m.T, m.u[0], m.u[1], m.F[0], m.F[1], m.p,
                    m.S[0][0], m.S[0][1], m.S[1][0], m.S[1][1], m.gradT[0], m.gradT[1]};
    memcpy(out, v, sizeof(v));
    return 0;
}

/* Velocity from the temporary velocity v at porosity eps: out = [ux, uy]. */
int orc_cell_velocity(const orc_problem *pb, double eps, const double v[2], double out[2],
                      double c01[2]) {
    orc_ctx cx;
    int rc = make_ctx(pb, NULL, &cx);
    if (rc) return rc;
    orc_cell c;
    cell_constants(&cx, eps, &c);
    velocity_from_v(&c, v, out);
    c01[0] = c.c0;
    c01[1] = c.c1;
    return 0;
}

#endif /* !ORC_COMPLEX */

/* Initial post-collision state from macroscopic fields (NULL = uniform):
 * f = f^{eq}(p = 0, u, S = 0), g = g^{eq}(T, u, p = 0, grad T = 0). */
int orc_init(const orc_problem *pb, const real_t *T, const real_t *ux, const real_t *uy,
             const real_t *eps_field, real_t *f, real_t *g) {
    orc_ctx cx;
    int rc = make_ctx(pb, eps_field, &cx);
    if (rc) return rc;
    int nx = pb->nx, ny = pb->ny;
    const int nth = orc_get_threads();
    (void)nth;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            real_t S[2][2] = {{0, 0}, {0, 0}}, z[2] = {0, 0};
            size_t k = (size_t)y * nx + x;
            orc_cell c;
            node_cell(&cx, x, y, &c);
            real_t u[2] = {ux ? ux[k] : 0.0, uy ? uy[k] : 0.0};
            real_t t = T ? T[k] : pb->T_init;
            real_t fe[9], ge[9];
            flow_eq(&cx, &c, 0.0, u, S, 1, fe);
            thermal_eq(&cx, &c, t, u, 0.0, z, 1, ge);
            for (int i = 0; i < 9; ++i) {
                f[(size_t)i * nx * ny + k] = fe[i];
                g[(size_t)i * nx * ny + k] = ge[i];
            }
        }
    return 0;
}

/* n time steps; f and g are updated in place (the oracle ping-pongs through
 * a private copy). */
int orc_run(const orc_problem *pb, const real_t *eps_field, real_t *f, real_t *g, int64_t n) {
    orc_ctx cx;
    int rc = make_ctx(pb, eps_field, &cx);
    if (rc) return rc;
    int nx = pb->nx, ny = pb->ny;
    size_t plane = (size_t)nx * ny, tot = 9 * plane;
    real_t *f2 = (real_t *)malloc(tot * sizeof(real_t));
    real_t *g2 = (real_t *)malloc(tot * sizeof(real_t));
    if (!f2 || !g2) { free(f2); free(g2); return 100; }
    real_t *fa = f, *ga = g, *fb = f2, *gb = g2;
    const int nth = orc_get_threads();
    (void)nth;
    for (int64_t s = 0; s < n; ++s) {
#pragma omp parallel for schedule(static) num_threads(nth)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                real_t fo[9], go[9];
                node_update(&cx, fa, ga, x, y, fo, go);
                size_t k = (size_t)y * nx + x;
                for (int i = 0; i < 9; ++i) { fb[i * plane + k] = fo[i]; gb[i * plane + k] = go[i]; }
            }
        real_t *t;
        t = fa; fa = fb; fb = t;
        t = ga; ga = gb; gb = t;
    }
    if (fa != f) { memcpy(f, fa, tot * sizeof(real_t)); memcpy(g, ga, tot * sizeof(real_t)); }
    free(f2);
    free(g2);
    return 0;
}

/* One step evaluated only at the listed nodes: fo/go[k][9] are the new
 * post-collision populations of node (xs[k], ys[k]). */
int orc_update_nodes(const orc_problem *pb, const real_t *eps_field, const real_t *f,
                     const real_t *g, int64_t n, const int32_t *xs, const int32_t *ys,
                     real_t *fo, real_t *go) {
    orc_ctx cx;
    int rc = make_ctx(pb, eps_field, &cx);
    if (rc) return rc;
    const int nth = orc_get_threads();
    (void)nth;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int64_t k = 0; k < n; ++k) node_update(&cx, f, g, xs[k], ys[k], fo + 9 * k, go + 9 * k);
    return 0;
}

/* Macroscopic fields of the state: the moments a next step would compute
 * after streaming (wall nodes: the NEES boundary state). */
int orc_moments(const orc_problem *pb, const real_t *eps_field, const real_t *f, const real_t *g,
                real_t *p, real_t *ux, real_t *uy, real_t *T) {
    orc_ctx cx;
    int rc = make_ctx(pb, eps_field, &cx);
    if (rc) return rc;
    int nx = pb->nx, ny = pb->ny;
    const int nth = orc_get_threads();
    (void)nth;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            orc_state st;
            node_state(&cx, f, g, x, y, &st, NULL, NULL);
            size_t k = (size_t)y * nx + x;
            if (p) p[k] = st.p;
            if (ux) ux[k] = st.u[0];
            if (uy) uy[k] = st.u[1];
            if (T) T[k] = st.T;
        }
    return 0;
}

/* Shear rate and temperature gradient fields (local schemes). */
int orc_gradients(const orc_problem *pb, const real_t *eps_field, const real_t *f,
                  const real_t *g, real_t *Sxx, real_t *Sxy, real_t *Syy, real_t *dTdx,
                  real_t *dTdy) {
    orc_ctx cx;
    int rc = make_ctx(pb, eps_field, &cx);
    if (rc) return rc;
    int nx = pb->nx, ny = pb->ny;
    const int nth = orc_get_threads();
    (void)nth;
#pragma omp parallel for schedule(static) num_threads(nth)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            orc_state st;
            node_state(&cx, f, g, x, y, &st, NULL, NULL);
            size_t k = (size_t)y * nx + x;
            Sxx[k] = st.S[0][0]; Sxy[k] = st.S[0][1]; Syy[k] = st.S[1][1];
            dTdx[k] = st.gradT[0]; dTdy[k] = st.gradT[1];
        }
    return 0;
}

/* Local and mean Nusselt number on one side (W, E, S, N) from a temperature
 * field, Eq. (Eq:AvNuss): Nu = -L (dT/dn)_wall / dT with the derivative taken
 * into the wall by the second-order one-sided difference; the mean is the
 * trapezoid rule over the wall's nodes divided by its length in lattice
 * units.  nu_local has ny entries (W, E) or nx entries (S, N). */
int orc_nusselt(const orc_problem *pb, const real_t *T, int side, real_t *nu_local,
                real_t *nu_mean) {
    orc_derived d;
    int rc = orc_derive(pb, &d);
    if (rc) return rc;
    int nx = pb->nx, ny = pb->ny;
    int n = (side <= SIDE_E) ? ny : nx;
    real_t acc = 0.0;
    for (int j = 0; j < n; ++j) {
        real_t t0, t1, t2;
        if (side == SIDE_W) { t0 = T[(size_t)j * nx + 0]; t1 = T[(size_t)j * nx + 1]; t2 = T[(size_t)j * nx + 2]; }
        else if (side == SIDE_E) { t0 = T[(size_t)j * nx + nx - 1]; t1 = T[(size_t)j * nx + nx - 2]; t2 = T[(size_t)j * nx + nx - 3]; }
        else if (side == SIDE_S) { t0 = T[j]; t1 = T[(size_t)nx + j]; t2 = T[(size_t)2 * nx + j]; }
        else { t0 = T[(size_t)(ny - 1) * nx + j]; t1 = T[(size_t)(ny - 2) * nx + j]; t2 = T[(size_t)(ny - 3) * nx + j]; }
        /* one-sided second-order derivative taken from the wall inward, then
         * turned into the derivative along +x (W, E) or +y (S, N) */
        real_t d_in = (-3.0 * t0 + 4.0 * t1 - t2) / 2.0;
        real_t d_axis = (side == SIDE_W || side == SIDE_S) ? d_in : -d_in;
        real_t nu = -d.L * d_axis / d.dT;
        if (nu_local) nu_local[j] = nu;
        real_t wt = (j == 0 || j == n - 1) ? 0.5 : 1.0;
        acc += wt * nu;
    }
    *nu_mean = acc / (real_t)(n - 1);
    return 0;
}

#ifndef ORC_COMPLEX
/* Steady-state criterion of Sec. 4: res_u = sum |u - u_old|_2 / sum |u|_2,
 * res_T = sum |T - T_old| / sum |T|. */
int orc_residual(int64_t n, const double *ux, const double *uy, const double *T,
                 const double *ux0, const double *uy0, const double *T0, double out[2]) {
    double nu_ = 0, du = 0, nT = 0, dT = 0;
    for (int64_t k = 0; k < n; ++k) {
        du += RSQRT((ux[k] - ux0[k]) * (ux[k] - ux0[k]) + (uy[k] - uy0[k]) * (uy[k] - uy0[k]));
        nu_ += RSQRT(ux[k] * ux[k] + uy[k] * uy[k]);
        dT += fabs(T[k] - T0[k]);
        nT += fabs(T[k]);
    }
    out[0] = du / nu_;
    out[1] = dT / nT;
    return 0;
}

/* Stream function of a velocity field [ny][nx] (Sec. 4.3, Table 3): u_x is
 * d psi / dy, psi vanishes on the bottom row, and each column is integrated
 * upward with the trapezoid rule (the paper does not state its quadrature). */
int orc_stream_function(int nx, int ny, const double *ux, double *psi) {
    for (int x = 0; x < nx; ++x) {
        psi[x] = 0.0;
        for (int y = 1; y < ny; ++y) {
            double du = 0.5 * (ux[(size_t)(y - 1) * nx + x] + ux[(size_t)y * nx + x]);
            psi[(size_t)y * nx + x] = psi[(size_t)(y - 1) * nx + x] + du;
        }
    }
    return 0;
}

#endif /* !ORC_COMPLEX */

/* Totals of the post-collision state: out = [sum f (all nine), sum g]. */
int orc_totals(const orc_problem *pb, const real_t *f, const real_t *g, real_t out[2]) {
    size_t tot = (size_t)9 * pb->nx * pb->ny;
    real_t sf = 0, sg = 0;
    for (size_t k = 0; k < tot; ++k) { sf += f[k]; sg += g[k]; }
    out[0] = sf;
    out[1] = sg;
    return 0;
}
