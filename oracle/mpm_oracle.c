/*
 * Plain FP64 CPU oracle of the explicit MPM time step of JAX-MPM (Du & He,
 * arXiv 2507.04192).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library; both sides are written independently from
 * the paper.
 *
 * The step follows the paper's order and notation (Sec. 2.2): particle-to-grid
 * transfer (Eq. update_m and the nodal momentum and force of Eq. semi), the
 * explicit grid update (Eq. semi_eq), the Coulomb wall contact of Eq.
 * coulomb_friction (Sec. 5.3), and the grid-to-particle transfer with the APIC
 * affine matrix B_p and moment matrix D_p (Appendix B), the velocity gradient
 * (Eq. update_v_gradient), the deformation gradient, the density update and the
 * stress update (Sec. 2.3, Appendix A), updated stress last (USL).
 *
 * Everything is written as plain loops over particles and stencil nodes with no
 * blocking, fusion or reordering.  The shape functions are the quadratic
 * B-spline of Sec. 2.1 evaluated from its piecewise definition; the moment
 * matrix D_p is built from its definition and inverted.
 *
 * Readings where the paper is silent or garbled are the same as stated in the
 * package's design notes: density update with tr(dd) (the paper prints det);
 * viscous stress from the rate of deformation; Tait EOS (gamma = 1 is the
 * paper's linear EOS); walls at the domain faces with one ghost node beyond;
 * contact applied only to approaching nodes (v.n > 0); friction segment index
 * floor(x_i / L * n_seg) clamped; Drucker-Prager corner guard.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_WALLS 6

typedef struct {
    int dim;
    int n_cells[3];
    double dx, dt;
    double gravity[3];
    int material;               /* 0 = weakly compressible Newtonian fluid, 1 = Drucker-Prager */
    int dp_literal;             /* 1 = Appendix A exactly as printed, no corner guard */
    double rho0;                /* reference (fluid) or initial (sand) density */
    double bulk_K, gamma, viscosity;                     /* fluid */
    double E, nu, phi_deg, psi_deg, cohesion, sigma_t;   /* Drucker-Prager */
    double particle_volume;     /* initial volume V_p^0; mass m_p = rho0 V_p^0 */
    int n_seg[ORC_MAX_WALLS][2];
    const double *mu[ORC_MAX_WALLS];   /* per wall: mu[s1 * n_seg0 + s0], NULL = slip */
} orc_params;

/* ------------------------------------------------------------------------- */
/* Quadratic B-spline of Sec. 2.1 and its derivative.                        */
/* ------------------------------------------------------------------------- */

double orc_phi_bar(double xi)
{
    double a = fabs(xi);
    if (a < 0.5) return -a * a + 0.75;
    if (a < 1.5) return 0.5 * a * a - 1.5 * a + 9.0 / 8.0;
    return 0.0;
}

/* d phi_bar / d xi */
double orc_dphi_bar(double xi)
{
    double a = fabs(xi);
    double s = xi < 0.0 ? -1.0 : 1.0;
    if (a < 0.5) return -2.0 * xi;
    if (a < 1.5) return s * (a - 1.5);
    return 0.0;
}

/* ------------------------------------------------------------------------- */
/* Grid indexing: N_a + 3 nodes per axis, node j at coordinate (j - 1) dx.   */
/* ------------------------------------------------------------------------- */

static int nodes_axis(const orc_params *P, int a) { return P->n_cells[a] + 3; }

long orc_num_nodes(const orc_params *P)
{
    long g = 1;
    for (int a = 0; a < P->dim; ++a) g *= nodes_axis(P, a);
    return g;
}

static long node_index(const orc_params *P, const int j[3])
{
    long idx = 0;
    for (int a = P->dim - 1; a >= 0; --a) idx = idx * nodes_axis(P, a) + j[a];
    return idx;
}

/* The 3^d nodes whose shape function can be nonzero at x_p. */
typedef struct {
    int count;
    long node[27];
    double xi[27][3];      /* node coordinates */
    double phi[27];
    double grad[27][3];    /* gradient of phi_i at x_p */
} stencil_t;

static void build_stencil(const orc_params *P, const double *xp, stencil_t *S)
{
    int d = P->dim;
    int base[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) base[a] = (int)floor(xp[a] / P->dx - 0.5);
    int total = d == 2 ? 9 : 27;
    S->count = total;
    for (int k = 0; k < total; ++k) {
        int off[3] = {k % 3, (k / 3) % 3, k / 9};
        int j[3] = {0, 0, 0};
        double fa[3], dfa[3];
        for (int a = 0; a < d; ++a) {
            int cell = base[a] + off[a];          /* node coordinate = cell * dx */
            j[a] = cell + 1;
            S->xi[k][a] = cell * P->dx;
            double xi = (xp[a] - S->xi[k][a]) / P->dx;
            fa[a] = orc_phi_bar(xi);
            dfa[a] = orc_dphi_bar(xi) / P->dx;
        }
        double phi = 1.0;
        for (int a = 0; a < d; ++a) phi *= fa[a];
        S->phi[k] = phi;
        for (int a = 0; a < d; ++a) {
            double g = dfa[a];
            for (int b = 0; b < d; ++b) if (b != a) g *= fa[b];
            S->grad[k][a] = g;
        }
        S->node[k] = node_index(P, j);
    }
}

/* Small dense linear algebra on d x d row-major matrices. */
static int invert(int d, const double *A, double *inv)
{
    if (d == 2) {
        double det = A[0] * A[3] - A[1] * A[2];
        if (det == 0.0) return -1;
        inv[0] = A[3] / det; inv[1] = -A[1] / det;
        inv[2] = -A[2] / det; inv[3] = A[0] / det;
        return 0;
    }
    double c00 = A[4] * A[8] - A[5] * A[7];
    double c01 = A[5] * A[6] - A[3] * A[8];
    double c02 = A[3] * A[7] - A[4] * A[6];
    double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    if (det == 0.0) return -1;
    inv[0] = c00 / det;
    inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    inv[3] = c01 / det;
    inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    inv[6] = c02 / det;
    inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    return 0;
}

static void matmul(int d, const double *A, const double *B, double *C)
{
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) s += A[i * d + k] * B[k * d + j];
            C[i * d + j] = s;
        }
}

/* Moment matrix D_p = sum_i phi_ip (x_i - x_p) (x_i - x_p)^T (Appendix B). */
static void moment_matrix(const orc_params *P, const double *xp, const stencil_t *S, double *D)
{
    int d = P->dim;
    for (int q = 0; q < d * d; ++q) D[q] = 0.0;
    for (int k = 0; k < S->count; ++k)
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b)
                D[a * d + b] += S->phi[k] * (S->xi[k][a] - xp[a]) * (S->xi[k][b] - xp[b]);
}

double orc_particle_mass(const orc_params *P) { return P->rho0 * P->particle_volume; }

/* ------------------------------------------------------------------------- */
/* P2G (Sec. 2.2): lumped mass, APIC momentum, internal and body force.      */
/* sigma is stored as a full 3 x 3 row-major matrix per particle; in 2D the  */
/* in-plane 2 x 2 block acts on the grid.                                    */
/* ------------------------------------------------------------------------- */

void orc_p2g(const orc_params *P, long n, const double *x, const double *v, const double *B,
             const double *rho, const double *sigma, double *gm, double *gq, double *gf)
{
    int d = P->dim;
    double mp = orc_particle_mass(P);
    stencil_t S;
    for (long p = 0; p < n; ++p) {
        const double *xp = x + p * d;
        const double *vp = v + p * d;
        const double *Bp = B + p * d * d;
        const double *sp = sigma + p * 9;
        double Vp = mp / rho[p];
        build_stencil(P, xp, &S);
        double D[9], Dinv[9], M[9];
        moment_matrix(P, xp, &S, D);
        invert(d, D, Dinv);
        matmul(d, Bp, Dinv, M);                         /* B_p D_p^{-1} */
        for (int k = 0; k < S.count; ++k) {
            long i = S.node[k];
            double phi = S.phi[k];
            gm[i] += mp * phi;                          /* Eq. update_m */
            for (int a = 0; a < d; ++a) {
                double aff = 0.0;
                for (int b = 0; b < d; ++b) aff += M[a * d + b] * (S.xi[k][b] - xp[b]);
                gq[i * d + a] += phi * mp * (vp[a] + aff);
            }
            for (int a = 0; a < d; ++a) {
                double fint = 0.0;
                for (int b = 0; b < d; ++b) fint += S.grad[k][b] * sp[b * 3 + a];
                gf[i * d + a] += -Vp * fint + phi * mp * P->gravity[a];
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Coulomb frictional contact with a stationary rigid wall (Eq.              */
/* coulomb_friction, Bardenhagen et al. 2001), written with the cross        */
/* products of the paper in 3D.  v_cm = 0 for a stationary wall.             */
/* ------------------------------------------------------------------------- */

static void cross3(const double *a, const double *b, double *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_friction(const double *v, const double *n, double mu, double *out)
{
    double dv[3] = {v[0], v[1], v[2]};             /* Delta v = v - v_cm, v_cm = 0 */
    double dvn = dv[0] * n[0] + dv[1] * n[1] + dv[2] * n[2];
    for (int a = 0; a < 3; ++a) out[a] = v[a];
    if (dvn <= 0.0) return;                        /* not approaching the wall */
    double c[3];
    cross3(dv, n, c);
    double cn = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    double mup = 0.0, nxw[3] = {0.0, 0.0, 0.0};
    if (cn > 0.0) {
        double omega[3] = {c[0] / cn, c[1] / cn, c[2] / cn};
        mup = cn / dvn < mu ? cn / dvn : mu;       /* mu' = min(mu, |dv x n| / dv.n) */
        cross3(n, omega, nxw);
    }
    for (int a = 0; a < 3; ++a) out[a] = v[a] - dvn * (n[a] + mup * nxw[a]);
}

/* Friction coefficient of the wall segment containing node j. */
static double wall_mu(const orc_params *P, int w, const int j[3])
{
    if (P->mu[w] == NULL) return 0.0;
    int a = w / 2, d = P->dim;
    int t[2], nt = 0;
    for (int b = 0; b < d; ++b) if (b != a) t[nt++] = b;
    int s[2] = {0, 0};
    for (int q = 0; q < nt; ++q) {
        int ns = P->n_seg[w][q];
        /* s = floor(x_i / L * n_seg) with x_i / L = (j - 1) / N, evaluated exactly */
        long num = (long)(j[t[q]] - 1) * ns;
        long den = P->n_cells[t[q]];
        long sq = num >= 0 ? num / den : -1;
        if (sq < 0) sq = 0;
        if (sq > ns - 1) sq = ns - 1;
        s[q] = (int)sq;
    }
    return P->mu[w][s[1] * P->n_seg[w][0] + s[0]];
}

/* ------------------------------------------------------------------------- */
/* Grid update (Sec. 2.2): a_i = f_i / m_i, v_i^{n+1} = v_i^n + dt a_i, then   */
/* the walls.  Walls sit at the domain faces; wall and ghost nodes (node      */
/* coordinate <= 0 or >= L) take the contact correction.  Order: x-, x+,     */
/* y-, y+, z-, z+ with the floor (the low wall of the last axis) last.       */
/* ------------------------------------------------------------------------- */

void orc_grid_update(const orc_params *P, const double *gm, const double *gq, const double *gf,
                     double *gv)
{
    int d = P->dim;
    long G = orc_num_nodes(P);
    double m_eps = 1e-10 * P->rho0 * pow(P->dx, d);
    int order[ORC_MAX_WALLS], nw = 0;
    int floor_w = 2 * (d - 1);
    for (int w = 0; w < 2 * d; ++w) if (w != floor_w) order[nw++] = w;
    order[nw++] = floor_w;
    for (long i = 0; i < G; ++i) {
        int j[3] = {0, 0, 0};
        long r = i;
        for (int a = 0; a < d; ++a) { j[a] = (int)(r % nodes_axis(P, a)); r /= nodes_axis(P, a); }
        double vi[3] = {0.0, 0.0, 0.0};
        if (gm[i] > m_eps) {
            for (int a = 0; a < d; ++a) {
                double vn = gq[i * d + a] / gm[i];
                double an = gf[i * d + a] / gm[i];
                vi[a] = vn + P->dt * an;
            }
        }
        for (int q = 0; q < nw; ++q) {
            int w = order[q], a = w / 2, hi = w % 2;
            double coord = (j[a] - 1) * P->dx;
            double L = P->n_cells[a] * P->dx;
            int on_wall = hi ? (coord >= L) : (coord <= 0.0);
            if (!on_wall) continue;
            double nrm[3] = {0.0, 0.0, 0.0};
            nrm[a] = hi ? 1.0 : -1.0;                  /* outward normal */
            double out[3];
            orc_friction(vi, nrm, wall_mu(P, w, j), out);
            for (int b = 0; b < 3; ++b) vi[b] = out[b];
        }
        for (int a = 0; a < d; ++a) gv[i * d + a] = vi[a];
    }
}

/* ------------------------------------------------------------------------- */
/* Constitutive updates (Sec. 2.3, Appendix A).                              */
/* ------------------------------------------------------------------------- */

/* Tait equation of state; gamma = 1 gives the paper's c^2 (rho - rho0) with c^2 = K / rho0. */
double orc_tait_pressure(const orc_params *P, double rho)
{
    return P->bulk_K / P->gamma * (pow(rho / P->rho0, P->gamma) - 1.0);
}

typedef struct { double K, G, q_phi, k_phi, q_psi, sig_t, tau_P, alpha_P; } dp_consts;

static void dp_constants(const orc_params *P, dp_consts *c)
{
    const double pi = 3.14159265358979323846;
    double phi = P->phi_deg * pi / 180.0, psi = P->psi_deg * pi / 180.0;
    c->K = P->E / (3.0 * (1.0 - 2.0 * P->nu));
    c->G = P->E / (2.0 * (1.0 + P->nu));
    c->q_phi = 6.0 * sin(phi) / (sqrt(3.0) * (3.0 + sin(phi)));
    c->k_phi = 6.0 * P->cohesion * cos(phi) / (sqrt(3.0) * (3.0 + sin(phi)));
    c->q_psi = 6.0 * sin(psi) / (sqrt(3.0) * (3.0 + sin(psi)));
    c->sig_t = P->sigma_t;
    if (c->q_phi > 0.0 && c->k_phi / c->q_phi < c->sig_t) c->sig_t = c->k_phi / c->q_phi;
    c->tau_P = c->k_phi - c->q_phi * c->sig_t;
    c->alpha_P = sqrt(1.0 + c->q_phi * c->q_phi) - c->q_phi;
}

void orc_dp_constants(const orc_params *P, double *out8)
{
    dp_consts c;
    dp_constants(P, &c);
    out8[0] = c.K; out8[1] = c.G; out8[2] = c.q_phi; out8[3] = c.k_phi;
    out8[4] = c.q_psi; out8[5] = c.sig_t; out8[6] = c.tau_P; out8[7] = c.alpha_P;
}

/*
 * Drucker-Prager update of Appendix A for one particle.  dd and dw are the
 * 3 x 3 strain and vorticity increments, s the 3 x 3 stress (in/out), eps the
 * equivalent plastic strain (in/out).  Returns the zone (1, 2 or 3).
 */
int orc_dp_update(const orc_params *P, const double *dd, const double *dw, double *s, double *eps)
{
    dp_consts c;
    dp_constants(P, &c);
    double lam = c.K - 2.0 * c.G / 3.0;
    /* (1) Jaumann-rotated stress: sR_ij = s_ij + s_ik dw_jk + s_jk dw_ik */
    double sR[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = s[i * 3 + j];
            for (int k = 0; k < 3; ++k) v += s[i * 3 + k] * dw[j * 3 + k] + s[j * 3 + k] * dw[i * 3 + k];
            sR[i * 3 + j] = v;
        }
    /* trial stress: sR_ij + C_ijkl dd_kl, isotropic C_ijkl = lam d_ij d_kl + G (d_ik d_jl + d_il d_jk) */
    double st[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = sR[i * 3 + j];
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    double C = lam * (i == j) * (k == l) + c.G * ((i == k) * (j == l) + (i == l) * (j == k));
                    v += C * dd[k * 3 + l];
                }
            st[i * 3 + j] = v;
        }
    /* (2) trial invariants */
    double sm = (st[0] + st[4] + st[8]) / 3.0;
    double sdev[9];
    for (int q = 0; q < 9; ++q) sdev[q] = st[q] - (q % 4 == 0 ? sm : 0.0);
    double ss = 0.0;
    for (int q = 0; q < 9; ++q) ss += sdev[q] * sdev[q];
    double tau = sqrt(0.5 * ss);
    /* (3) yield functions */
    double fs = tau - c.k_phi + c.q_phi * sm;
    double ft = sm - c.sig_t;
    double h = tau - c.tau_P - c.alpha_P * (sm - c.sig_t);
    if (fs <= 0.0 && ft < 0.0) {                                     /* Zone I */
        for (int q = 0; q < 9; ++q) s[q] = st[q];
        return 1;
    }
    if ((fs > 0.0 && ft < 0.0) || (h > 0.0 && ft >= 0.0)) {          /* Zone II */
        double dl = fs / (c.G + c.K * c.q_phi * c.q_psi);
        double sm_n = sm - c.K * c.q_psi * dl;
        double tau_n = c.k_phi - c.q_phi * sm_n;
        if (!P->dp_literal && sm_n > c.sig_t) {    /* return lands past the tension cutoff: corner */
            sm_n = c.sig_t;
            tau_n = c.tau_P;
        }
        double r = tau > 0.0 ? tau_n / tau : 0.0;
        for (int q = 0; q < 9; ++q) s[q] = r * sdev[q] + (q % 4 == 0 ? sm_n : 0.0);
        *eps += dl * sqrt(1.0 / 3.0 + 2.0 / 9.0 * c.q_psi * c.q_psi);
        return 2;
    }
    /* Zone III: tension cutoff */
    for (int q = 0; q < 9; ++q) s[q] = st[q] + (q % 4 == 0 ? (c.sig_t - sm) : 0.0);
    double dlt = (sm - c.sig_t) / c.K;
    *eps += sqrt(2.0) / 3.0 * dlt;
    if (!P->dp_literal && tau > c.tau_P) {          /* deviator still outside the cone: corner */
        double r = c.tau_P / tau;
        for (int q = 0; q < 9; ++q) s[q] = r * sdev[q] + (q % 4 == 0 ? c.sig_t : 0.0);
    }
    return 3;
}

/* ------------------------------------------------------------------------- */
/* G2P (Sec. 2.2, Appendix B): velocity, affine matrix B_p, velocity         */
/* gradient, position, deformation gradient, density and stress (USL).       */
/* ------------------------------------------------------------------------- */

void orc_g2p(const orc_params *P, long n, const double *gv, double *x, double *v, double *B,
             double *F, double *rho, double *sigma, double *eps)
{
    int d = P->dim;
    double dt = P->dt;
    stencil_t S;
    for (long p = 0; p < n; ++p) {
        double *xp = x + p * d;
        build_stencil(P, xp, &S);
        double vp[3] = {0.0, 0.0, 0.0}, Bp[9] = {0.0}, L[9] = {0.0};
        for (int k = 0; k < S.count; ++k) {
            const double *vi = gv + S.node[k] * d;
            for (int a = 0; a < d; ++a) {
                vp[a] += S.phi[k] * vi[a];
                for (int b = 0; b < d; ++b) {
                    Bp[a * d + b] += S.phi[k] * vi[a] * (S.xi[k][b] - xp[b]);
                    L[a * d + b] += vi[a] * S.grad[k][b];        /* Eq. update_v_gradient */
                }
            }
        }
        for (int a = 0; a < d; ++a) {
            v[p * d + a] = vp[a];
            double xn = xp[a] + dt * vp[a];
            double Lmax = P->n_cells[a] * P->dx;
            if (xn < 0.0) xn = 0.0;
            if (xn > Lmax) xn = Lmax;
            xp[a] = xn;
        }
        for (int q = 0; q < d * d; ++q) B[p * d * d + q] = Bp[q];
        /* F <- (I + dt L) F */
        double A[9], Fn[9];
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) A[a * d + b] = (a == b) + dt * L[a * d + b];
        matmul(d, A, F + p * d * d, Fn);
        for (int q = 0; q < d * d; ++q) F[p * d * d + q] = Fn[q];
        /* increments embedded in 3 x 3 */
        double dd[9] = {0.0}, dw[9] = {0.0};
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                dd[a * 3 + b] = 0.5 * (L[a * d + b] + L[b * d + a]) * dt;
                dw[a * 3 + b] = 0.5 * (L[a * d + b] - L[b * d + a]) * dt;
            }
        double trdd = dd[0] + dd[4] + dd[8];
        rho[p] = rho[p] / (1.0 + trdd);
        double *sp = sigma + p * 9;
        if (P->material == 0) {
            double pr = orc_tait_pressure(P, rho[p]);
            double mu = P->viscosity;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double rate = dd[a * 3 + b] / dt;          /* rate of deformation */
                    double tr_rate = trdd / dt;
                    sp[a * 3 + b] = (a == b ? -pr - 2.0 / 3.0 * mu * tr_rate : 0.0) + 2.0 * mu * rate;
                }
        } else {
            orc_dp_update(P, dd, dw, sp, eps + p);
        }
    }
}

/* C_p = B_p D_p^{-1} with D_p at the current position (what the next P2G uses). */
void orc_affine_C(const orc_params *P, long n, const double *x, const double *B, double *C)
{
    int d = P->dim;
    stencil_t S;
    for (long p = 0; p < n; ++p) {
        build_stencil(P, x + p * d, &S);
        double D[9], Dinv[9];
        moment_matrix(P, x + p * d, &S, D);
        invert(d, D, Dinv);
        matmul(d, B + p * d * d, Dinv, C + p * d * d);
    }
}

/* Full steps: grid reset, P2G, grid update, G2P.  Returns 0, or -1 on allocation failure. */
int orc_step(const orc_params *P, long n, double *x, double *v, double *B, double *F, double *rho,
             double *sigma, double *eps, int n_steps)
{
    int d = P->dim;
    long G = orc_num_nodes(P);
    double *gm = (double *)malloc(sizeof(double) * G);
    double *gq = (double *)malloc(sizeof(double) * G * d);
    double *gf = (double *)malloc(sizeof(double) * G * d);
    double *gv = (double *)malloc(sizeof(double) * G * d);
    if (!gm || !gq || !gf || !gv) { free(gm); free(gq); free(gf); free(gv); return -1; }
    for (int s = 0; s < n_steps; ++s) {
        memset(gm, 0, sizeof(double) * G);                   /* grid reset */
        memset(gq, 0, sizeof(double) * G * d);
        memset(gf, 0, sizeof(double) * G * d);
        orc_p2g(P, n, x, v, B, rho, sigma, gm, gq, gf);
        orc_grid_update(P, gm, gq, gf, gv);
        orc_g2p(P, n, gv, x, v, B, F, rho, sigma, eps);
    }
    free(gm); free(gq); free(gf); free(gv);
    return 0;
}
