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
 * floor(x_i / L * n_seg) clamped; Drucker-Prager corner guard.  Rigid obstacles
 * (Sec. 4.1, 3D dam break) are stationary axis-aligned boxes with frictionless
 * contact, applied before the walls: a node inside a box (within 1e-9 dx) takes
 * the outward normal of the nearest box face that lies inside the domain and,
 * when it moves into the box, loses its normal velocity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_WALLS 6
#define ORC_MAX_OBSTACLES 8

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
    int transfer;               /* 0 = APIC, 1 = TPIC, 2 = PIC, 3 = FLIP / PIC blend (Sec. 2.2 G2P transfer) */
    double flip_alpha;          /* FLIP share of the blended particle velocity (transfer 3) */
    const double *flip_grid;    /* transfer 3: grid velocity before the update, set inside orc_step */
    int n_obstacles;            /* stationary rigid boxes, frictionless contact (Sec. 4.1) */
    double obstacle[ORC_MAX_OBSTACLES][2][3];   /* [o][0] = low corner, [o][1] = high corner (m) */
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
    /* The pragmas take effect only in the OpenMP build of this file (a timing
       baseline); the build the checks use is serial and ignores them. */
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        stencil_t S;
        const double *xp = x + p * d;
        const double *vp = v + p * d;
        const double *Bp = B + p * d * d;
        const double *sp = sigma + p * 9;
        double Vp = mp / rho[p];
        build_stencil(P, xp, &S);
        double D[9], Dinv[9], M[9];
        if (P->transfer == 1) {
            for (int q = 0; q < d * d; ++q) M[q] = Bp[q];   /* TPIC: the stored quantity is grad v_p */
        } else {
            moment_matrix(P, xp, &S, D);
            invert(d, D, Dinv);
            matmul(d, Bp, Dinv, M);                     /* B_p D_p^{-1} (zero for PIC) */
        }
        for (int k = 0; k < S.count; ++k) {
            long i = S.node[k];
            double phi = S.phi[k];
#pragma omp atomic
            gm[i] += mp * phi;                          /* Eq. update_m */
            for (int a = 0; a < d; ++a) {
                double aff = 0.0;
                for (int b = 0; b < d; ++b) aff += M[a * d + b] * (S.xi[k][b] - xp[b]);
#pragma omp atomic
                gq[i * d + a] += phi * mp * (vp[a] + aff);
            }
            for (int a = 0; a < d; ++a) {
                double fint = 0.0;
                for (int b = 0; b < d; ++b) fint += S.grad[k][b] * sp[b * 3 + a];
#pragma omp atomic
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

/* Contact normal of node j (oracle index, coordinate (j - 1) dx) with obstacle o:
 * returns 1 and the outward normal of the nearest box face when the node lies in
 * the closed box.  Box extents are taken in node units, ceil(lo / dx - 1e-9) ..
 * floor(hi / dx + 1e-9); faces on or beyond the domain boundary are not contact
 * faces; ties go to the first face in the order x-, x+, y-, y+, z-, z+. */
int orc_obstacle_normal(const orc_params *P, int o, const int j[3], double nrm[3])
{
    int d = P->dim, best = -1;
    long best_dist = 0;
    for (int a = 0; a < d; ++a) {
        long lo = (long)ceil(P->obstacle[o][0][a] / P->dx - 1e-9);
        long hi = (long)floor(P->obstacle[o][1][a] / P->dx + 1e-9);
        long c = j[a] - 1;
        if (c < lo || c > hi) return 0;
    }
    for (int a = 0; a < d; ++a) {
        long lo = (long)ceil(P->obstacle[o][0][a] / P->dx - 1e-9);
        long hi = (long)floor(P->obstacle[o][1][a] / P->dx + 1e-9);
        long c = j[a] - 1;
        if (lo > 0 && (best < 0 || c - lo < best_dist)) { best = 2 * a; best_dist = c - lo; }
        if (hi < P->n_cells[a] && (best < 0 || hi - c < best_dist)) { best = 2 * a + 1; best_dist = hi - c; }
    }
    if (best < 0) return 0;
    nrm[0] = nrm[1] = nrm[2] = 0.0;
    nrm[best / 2] = (best % 2) ? 1.0 : -1.0;
    return 1;
}

/* Frictionless contact with a stationary obstacle: v <- v - (v.n) n for a node
 * moving into the box (v.n < 0).  Returns 1 when applied. */
static int obstacle_contact(const double nrm[3], double v[3])
{
    double vn = v[0] * nrm[0] + v[1] * nrm[1] + v[2] * nrm[2];
    if (!(vn < 0.0)) return 0;
    for (int a = 0; a < 3; ++a) v[a] -= vn * nrm[a];
    return 1;
}

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
#pragma omp parallel for schedule(static)
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
        for (int o = 0; o < P->n_obstacles; ++o) {
            double nrm[3];
            if (orc_obstacle_normal(P, o, j, nrm)) obstacle_contact(nrm, vi);
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

/*
 * Vector-Jacobian product of orc_dp_update (Appendix A) for one particle: given
 * the stress s before the update, the increments dd and dw, and the adjoint sb1
 * of the updated stress (all 3 x 3, every entry independent), adds the adjoints
 * of s, dd and dw to sb0, ddb, dwb.  The zone and corner branches taken by the
 * forward update are held fixed (derivative of the branch taken).
 */
void orc_dp_vjp(const orc_params *P, const double *dd, const double *dw, const double *s, const double *sb1,
                double *sb0, double *ddb, double *dwb)
{
    dp_consts c;
    dp_constants(P, &c);
    double lam = c.K - 2.0 * c.G / 3.0;
    /* forward replay */
    double sR[9], st[9], sdev[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = s[i * 3 + j];
            for (int k = 0; k < 3; ++k) v += s[i * 3 + k] * dw[j * 3 + k] + s[j * 3 + k] * dw[i * 3 + k];
            sR[i * 3 + j] = v;
        }
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
    double sm = (st[0] + st[4] + st[8]) / 3.0;
    double ss = 0.0;
    for (int q = 0; q < 9; ++q) {
        sdev[q] = st[q] - (q % 4 == 0 ? sm : 0.0);
        ss += sdev[q] * sdev[q];
    }
    double tau = sqrt(0.5 * ss);
    double fs = tau - c.k_phi + c.q_phi * sm;
    double ft = sm - c.sig_t;
    double h = tau - c.tau_P - c.alpha_P * (sm - c.sig_t);
    /* reverse: adjoints of the trial stress (stb), its mean (smb) and deviator (sdevb) */
    double stb[9] = {0.0}, sdevb[9] = {0.0}, smb = 0.0, taub = 0.0;
    double trb = sb1[0] + sb1[4] + sb1[8];
    if (fs <= 0.0 && ft < 0.0) {                                     /* Zone I: s' = st */
        for (int q = 0; q < 9; ++q) stb[q] = sb1[q];
    } else if ((fs > 0.0 && ft < 0.0) || (h > 0.0 && ft >= 0.0)) {   /* Zone II */
        double A = c.G + c.K * c.q_phi * c.q_psi;
        double dl = fs / A;
        double sm_n = sm - c.K * c.q_psi * dl;
        double tau_n = c.k_phi - c.q_phi * sm_n;
        int corner = !P->dp_literal && sm_n > c.sig_t;
        if (corner) tau_n = c.tau_P;
        double r = tau > 0.0 ? tau_n / tau : 0.0;
        /* s'_q = r sdev_q + sm_n delta_q */
        double rb = 0.0;
        for (int q = 0; q < 9; ++q) {
            rb += sb1[q] * sdev[q];
            sdevb[q] += r * sb1[q];
        }
        double sm_nb = corner ? 0.0 : trb;
        double tau_nb = 0.0;
        if (tau > 0.0) {
            if (!corner) tau_nb = rb / tau;
            taub += -rb * tau_n / (tau * tau);
        }
        sm_nb += -c.q_phi * tau_nb;
        /* sm_n = sm - K q_psi (tau - k_phi + q_phi sm) / A */
        smb += sm_nb * (1.0 - c.K * c.q_psi * c.q_phi / A);
        taub += sm_nb * (-c.K * c.q_psi / A);
    } else {                                                         /* Zone III */
        int corner = !P->dp_literal && tau > c.tau_P;
        if (corner) {
            /* s' = (tau_P / tau) sdev + sig_t I */
            double r = c.tau_P / tau, rb = 0.0;
            for (int q = 0; q < 9; ++q) {
                rb += sb1[q] * sdev[q];
                sdevb[q] += r * sb1[q];
            }
            taub += -rb * c.tau_P / (tau * tau);
        } else {
            /* s' = st + (sig_t - sm) I */
            for (int q = 0; q < 9; ++q) stb[q] = sb1[q];
            smb += -trb;
        }
    }
    /* tau = sqrt(sdev:sdev / 2), sdev = st - sm I, sm = tr(st) / 3 */
    if (tau > 0.0)
        for (int q = 0; q < 9; ++q) sdevb[q] += taub * 0.5 * sdev[q] / tau;
    double sdev_tr = sdevb[0] + sdevb[4] + sdevb[8];
    for (int q = 0; q < 9; ++q) stb[q] += sdevb[q];
    smb += -sdev_tr;
    for (int a = 0; a < 3; ++a) stb[a * 4] += smb / 3.0;
    /* st = sR + C:dd */
    double trstb = stb[0] + stb[4] + stb[8];
    for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l)
            ddb[k * 3 + l] += lam * trstb * (k == l) + c.G * (stb[k * 3 + l] + stb[l * 3 + k]);
    /* sR_ij = s_ij + s_ik dw_jk + s_jk dw_ik */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double g = stb[i * 3 + j];
            sb0[i * 3 + j] += g;
            for (int k = 0; k < 3; ++k) {
                sb0[i * 3 + k] += g * dw[j * 3 + k];
                dwb[j * 3 + k] += g * s[i * 3 + k];
                sb0[j * 3 + k] += g * dw[i * 3 + k];
                dwb[i * 3 + k] += g * s[j * 3 + k];
            }
        }
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
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n; ++p) {
        stencil_t S;
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
        /* FLIP: v_p += sum phi (v_i^{n+1} - v_i^n), blended with PIC: v_p = vp + alpha (v_p - sum phi v_i^n) */
        double vflip[3] = {vp[0], vp[1], vp[2]};
        if (P->transfer == 3 && P->flip_grid) {
            double vo[3] = {0.0, 0.0, 0.0};
            for (int k = 0; k < S.count; ++k)
                for (int a = 0; a < d; ++a) vo[a] += S.phi[k] * P->flip_grid[S.node[k] * d + a];
            for (int a = 0; a < d; ++a) vflip[a] = vp[a] + P->flip_alpha * (v[p * d + a] - vo[a]);
        }
        for (int a = 0; a < d; ++a) {
            v[p * d + a] = vflip[a];
            double xn = xp[a] + dt * vp[a];
            double Lmax = P->n_cells[a] * P->dx;
            if (xn < 0.0) xn = 0.0;
            if (xn > Lmax) xn = Lmax;
            xp[a] = xn;
        }
        /* APIC keeps B_p; TPIC keeps the velocity gradient; PIC keeps nothing */
        for (int q = 0; q < d * d; ++q)
            B[p * d * d + q] = P->transfer == 1 ? L[q] : (P->transfer >= 2 ? 0.0 : Bp[q]);
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
        if (P->transfer == 1) {
            for (int q = 0; q < d * d; ++q) C[p * d * d + q] = B[p * d * d + q];
            continue;
        }
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
    double *gvo = P->transfer == 3 ? (double *)malloc(sizeof(double) * G * d) : NULL;
    orc_params Q = *P;
    Q.flip_grid = gvo;
    double m_eps = 1e-10 * P->rho0 * pow(P->dx, d);
    for (int s = 0; s < n_steps; ++s) {
        memset(gm, 0, sizeof(double) * G);                   /* grid reset */
        memset(gq, 0, sizeof(double) * G * d);
        memset(gf, 0, sizeof(double) * G * d);
        orc_p2g(P, n, x, v, B, rho, sigma, gm, gq, gf);
        orc_grid_update(P, gm, gq, gf, gv);
        if (gvo)                                             /* FLIP: the grid velocity before the update */
            for (long i = 0; i < G; ++i)
                for (int a = 0; a < d; ++a) gvo[i * d + a] = gm[i] > m_eps ? gq[i * d + a] / gm[i] : 0.0;
        orc_g2p(&Q, n, gv, x, v, B, F, rho, sigma, eps);
    }
    free(gvo);
    free(gm); free(gq); free(gf); free(gv);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of one step (reverse mode), weakly compressible fluid.            */
/*                                                                           */
/* A separately hand-derived vector-Jacobian product of the step above for   */
/* the state S = (x, v, B, rho) (the fluid's stress is -p(rho) I, a function */
/* of rho; F does not feed back).  Given the adjoint of S^{t+1}, returns the */
/* adjoint of S^t and adds d<adj, S^{t+1}>/d mu to mu_bar for every wall     */
/* with a friction field (the recursion of Eq. dzda, Sec. 3.1).  D_p is      */
/* constant in x_p for quadratic B-splines, so it is not differentiated.     */
/* Branches (clamp, contact, stick/slide, mass threshold) follow the forward */
/* pass.  mu_bar[w] points to n_seg0*n_seg1 doubles (NULL for slip walls).   */
/* ------------------------------------------------------------------------- */

/* Hessian of phi_i at x_p: H_ab = d^2 phi_i / dx_a dx_b. */
static void stencil_hessian(const orc_params *P, const double *xp, const stencil_t *S, int k, double *H)
{
    int d = P->dim;
    double f[3], df[3], ddf[3];
    for (int a = 0; a < d; ++a) {
        double xi = (xp[a] - S->xi[k][a]) / P->dx;
        f[a] = orc_phi_bar(xi);
        df[a] = orc_dphi_bar(xi) / P->dx;
        double ax = fabs(xi);
        ddf[a] = (ax < 0.5 ? -2.0 : (ax < 1.5 ? 1.0 : 0.0)) / (P->dx * P->dx);
    }
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double h = 1.0;
            for (int c = 0; c < d; ++c) {
                int na = (c == a) + (c == b);
                h *= na == 0 ? f[c] : (na == 1 ? df[c] : ddf[c]);
            }
            H[a * d + b] = h;
        }
}

/* Contact with one wall in the closed form of Eq. coulomb_friction (v_n > 0):
 * v_t = v - v_n n; stick if |v_t| <= mu v_n; else slide v_t (1 - mu v_n / |v_t|).
 * Reverse of that map for the adjoint ob of its output; returns the adjoint of
 * its input in ib and adds d<ob, out>/d mu to *mub. */
static void wall_vjp(const double *v, const double *n, double mu, const double *ob, double *ib, double *mub)
{
    double vn = v[0] * n[0] + v[1] * n[1] + v[2] * n[2];
    for (int a = 0; a < 3; ++a) ib[a] = ob[a];
    if (vn <= 0.0) return;
    double vt[3], vtn = 0.0;
    for (int a = 0; a < 3; ++a) { vt[a] = v[a] - vn * n[a]; vtn += vt[a] * vt[a]; }
    vtn = sqrt(vtn);
    /* output = P_t v (slip), 0 (stick), or s P_t v with s = 1 - mu vn / |vt| */
    double obt[3], obn = ob[0] * n[0] + ob[1] * n[1] + ob[2] * n[2];
    for (int a = 0; a < 3; ++a) obt[a] = ob[a] - obn * n[a];            /* P_t^T ob = P_t ob */
    if (mu == 0.0) { for (int a = 0; a < 3; ++a) ib[a] = obt[a]; return; }
    if (vtn <= mu * vn) { for (int a = 0; a < 3; ++a) ib[a] = 0.0; return; }
    double s = 1.0 - mu * vn / vtn;
    double dot = obt[0] * vt[0] + obt[1] * vt[1] + obt[2] * vt[2];      /* ob . vt */
    /* d(s vt)/dv applied transposed: s P_t ob + vt (ob.vt) * ds/dv, with
     * ds/dv = -mu (n / |vt| - vn vt / |vt|^3) */
    for (int a = 0; a < 3; ++a)
        ib[a] = s * obt[a] - mu * dot * (n[a] / vtn - vn * vt[a] / (vtn * vtn * vtn));
    if (mub) *mub += -dot * vn / vtn;
}

static int wall_segment_index(const orc_params *P, int w, const int j[3])
{
    int a = w / 2, d = P->dim, t[2], nt = 0;
    for (int b = 0; b < d; ++b) if (b != a) t[nt++] = b;
    int s[2] = {0, 0};
    for (int q = 0; q < nt; ++q) {
        int ns = P->n_seg[w][q];
        long num = (long)(j[t[q]] - 1) * ns;
        long den = P->n_cells[t[q]];
        long sq = num >= 0 ? num / den : -1;
        if (sq < 0) sq = 0;
        if (sq > ns - 1) sq = ns - 1;
        s[q] = (int)sq;
    }
    return s[1] * P->n_seg[w][0] + s[0];
}

/* dp/drho of the Tait equation of state */
static double tait_dpdrho(const orc_params *P, double rho)
{
    return P->bulk_K / P->rho0 * pow(rho / P->rho0, P->gamma - 1.0);
}

int orc_step_vjp(const orc_params *P, long n, const double *x, const double *v, const double *B,
                 const double *rho, const double *sigma,
                 const double *xb1, const double *vb1, const double *Bb1, const double *rhob1,
                 const double *sigb1,
                 double *xb0, double *vb0, double *Bb0, double *rhob0, double *sigb0, double **mu_bar)
{
    const int sand = P->material == 1;
    if (sand && (!sigma || !sigb1 || !sigb0)) return -2;
    if (P->transfer != 0) return -3;            /* the adjoint follows the APIC transfer */
    int d = P->dim;
    long G = orc_num_nodes(P);
    double dt = P->dt;
    double mp = orc_particle_mass(P);
    double m_eps = 1e-10 * P->rho0 * pow(P->dx, d);
    double *gm = calloc(G, sizeof(double)), *gq = calloc(G * d, sizeof(double)), *gf = calloc(G * d, sizeof(double));
    double *gu = calloc(G * 3, sizeof(double)), *gv = calloc(G * 3, sizeof(double));
    double *gvb = calloc(G * 3, sizeof(double)), *gqb = calloc(G * d, sizeof(double)), *gfb = calloc(G * d, sizeof(double));
    double *gmb = calloc(G, sizeof(double));
    if (!gm || !gq || !gf || !gu || !gv || !gvb || !gqb || !gfb || !gmb) return -1;
    double *sig = calloc(n * 9, sizeof(double));
    for (long p = 0; p < n; ++p) {
        if (sand) {
            for (int q = 0; q < 9; ++q) sig[p * 9 + q] = sigma[p * 9 + q];
        } else {
            double pr = orc_tait_pressure(P, rho[p]);
            for (int a = 0; a < 3; ++a) sig[p * 9 + a * 4] = -pr;
        }
    }
    /* forward: P2G and grid update, keeping the pre-wall velocity u */
    orc_p2g(P, n, x, v, B, rho, sig, gm, gq, gf);
    int order[ORC_MAX_WALLS], nw = 0, floor_w = 2 * (d - 1);
    for (int w = 0; w < 2 * d; ++w) if (w != floor_w) order[nw++] = w;
    order[nw++] = floor_w;
    for (long i = 0; i < G; ++i) {
        if (gm[i] > m_eps)
            for (int a = 0; a < d; ++a) gu[i * 3 + a] = gq[i * d + a] / gm[i] + dt * gf[i * d + a] / gm[i];
    }
    {
        /* walls on a copy */
        double *tmp = malloc(sizeof(double) * G * d);
        for (long i = 0; i < G; ++i) for (int a = 0; a < d; ++a) tmp[i * d + a] = 0.0;
        orc_grid_update(P, gm, gq, gf, tmp);
        for (long i = 0; i < G; ++i) for (int a = 0; a < d; ++a) gv[i * 3 + a] = tmp[i * d + a];
        free(tmp);
    }
    /* reverse G2P */
    stencil_t S;
    for (long p = 0; p < n; ++p) {
        const double *xp = x + p * d;
        build_stencil(P, xp, &S);
        double vp[3] = {0, 0, 0}, L[9] = {0};
        for (int k = 0; k < S.count; ++k)
            for (int a = 0; a < d; ++a) {
                vp[a] += S.phi[k] * gv[S.node[k] * 3 + a];
                for (int b = 0; b < d; ++b) L[a * d + b] += gv[S.node[k] * 3 + a] * S.grad[k][b];
            }
        double trL = 0.0;
        for (int a = 0; a < d; ++a) trL += L[a * d + a];
        double vbt[3] = {0, 0, 0};
        for (int a = 0; a < d; ++a) {
            double xn = xp[a] + dt * vp[a];
            int clamped = xn < 0.0 || xn > P->n_cells[a] * P->dx;
            xb0[p * d + a] = clamped ? 0.0 : xb1[p * d + a];
            vbt[a] = vb1[p * d + a] + (clamped ? 0.0 : dt * xb1[p * d + a]);
        }
        double den = 1.0 + dt * trL;
        rhob0[p] = rhob1[p] / den;
        double trLb = -rhob1[p] * rho[p] * dt / (den * den);
        /* adjoint of L through the Drucker-Prager update: dd = dt sym(L), dw = dt skew(L) */
        double Lb[9] = {0.0};
        if (sand) {
            double dd[9] = {0.0}, dw[9] = {0.0}, ddb[9] = {0.0}, dwb[9] = {0.0};
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    dd[a * 3 + b] = 0.5 * (L[a * d + b] + L[b * d + a]) * dt;
                    dw[a * 3 + b] = 0.5 * (L[a * d + b] - L[b * d + a]) * dt;
                }
            orc_dp_vjp(P, dd, dw, sigma + p * 9, sigb1 + p * 9, sigb0 + p * 9, ddb, dwb);
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b)
                    Lb[a * d + b] = 0.5 * dt * (ddb[a * 3 + b] + ddb[b * 3 + a] + dwb[a * 3 + b] - dwb[b * 3 + a]);
        }
        for (int a = 0; a < d; ++a) Lb[a * d + a] += trLb;
        const double *Bb = Bb1 + p * d * d;
        for (int k = 0; k < S.count; ++k) {
            long i = S.node[k];
            double phi = S.phi[k], r[3];
            for (int b = 0; b < d; ++b) r[b] = S.xi[k][b] - xp[b];
            double phib = 0.0, gradb[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) {
                double via = gv[i * 3 + a];
                double Br = 0.0;
                for (int b = 0; b < d; ++b) Br += Bb[a * d + b] * r[b];
                double Lg = 0.0;
                for (int b = 0; b < d; ++b) {
                    Lg += Lb[a * d + b] * S.grad[k][b];
                    gradb[b] += Lb[a * d + b] * via;
                }
                gvb[i * 3 + a] += phi * vbt[a] + phi * Br + Lg;
                phib += vbt[a] * via + Br * via;
                for (int b = 0; b < d; ++b) xb0[p * d + b] += -Bb[a * d + b] * phi * via;
            }
            double H[9];
            stencil_hessian(P, xp, &S, k, H);
            for (int b = 0; b < d; ++b) {
                double hb = 0.0;
                for (int a = 0; a < d; ++a) hb += H[b * d + a] * gradb[a];
                xb0[p * d + b] += phib * S.grad[k][b] + hb;
            }
        }
    }
    /* reverse grid update */
    for (long i = 0; i < G; ++i) {
        if (!(gm[i] > m_eps)) continue;
        int j[3] = {0, 0, 0};
        long r = i;
        for (int a = 0; a < d; ++a) { j[a] = (int)(r % nodes_axis(P, a)); r /= nodes_axis(P, a); }
        /* forward through the obstacles (projections, kept with their normals),
         * then the walls, keeping each wall's input */
        double chain[ORC_MAX_WALLS + 1][3];
        for (int a = 0; a < 3; ++a) chain[0][a] = gu[i * 3 + a];
        double onrm[ORC_MAX_OBSTACLES][3];
        int oapplied[ORC_MAX_OBSTACLES];
        for (int o = 0; o < P->n_obstacles; ++o)
            oapplied[o] = orc_obstacle_normal(P, o, j, onrm[o]) && obstacle_contact(onrm[o], chain[0]);
        int applied[ORC_MAX_WALLS];
        for (int q = 0; q < nw; ++q) {
            int w = order[q], a = w / 2, hi = w % 2;
            double coord = (j[a] - 1) * P->dx, Lw = P->n_cells[a] * P->dx;
            applied[q] = hi ? (coord >= Lw) : (coord <= 0.0);
            for (int b = 0; b < 3; ++b) chain[q + 1][b] = chain[q][b];
            if (applied[q]) {
                double nrm[3] = {0, 0, 0};
                nrm[a] = hi ? 1.0 : -1.0;
                orc_friction(chain[q], nrm, wall_mu(P, w, j), chain[q + 1]);
            }
        }
        double ob[3] = {gvb[i * 3], gvb[i * 3 + 1], gvb[i * 3 + 2]};
        for (int q = nw - 1; q >= 0; --q) {
            if (!applied[q]) continue;
            int w = order[q], a = w / 2, hi = w % 2;
            double nrm[3] = {0, 0, 0}, ib[3];
            nrm[a] = hi ? 1.0 : -1.0;
            double *mub = NULL;
            if (P->mu[w] && mu_bar && mu_bar[w]) mub = mu_bar[w] + wall_segment_index(P, w, j);
            wall_vjp(chain[q], nrm, wall_mu(P, w, j), ob, ib, mub);
            for (int b = 0; b < 3; ++b) ob[b] = ib[b];
        }
        for (int o = P->n_obstacles - 1; o >= 0; --o) {     /* a projection is its own transpose */
            if (!oapplied[o]) continue;
            double obn = ob[0] * onrm[o][0] + ob[1] * onrm[o][1] + ob[2] * onrm[o][2];
            for (int b = 0; b < 3; ++b) ob[b] -= obn * onrm[o][b];
        }
        for (int a = 0; a < d; ++a) {
            gqb[i * d + a] = ob[a] / gm[i];
            gfb[i * d + a] = dt * ob[a] / gm[i];
            gmb[i] += -ob[a] * (gq[i * d + a] + dt * gf[i * d + a]) / (gm[i] * gm[i]);
        }
    }
    /* reverse P2G */
    for (long p = 0; p < n; ++p) {
        const double *xp = x + p * d;
        const double *vpp = v + p * d;
        build_stencil(P, xp, &S);
        double D[9], Dinv[9], M[9], Mb[9] = {0};
        moment_matrix(P, xp, &S, D);
        invert(d, D, Dinv);
        matmul(d, B + p * d * d, Dinv, M);
        double Vp = mp / rho[p], pr = sand ? 0.0 : orc_tait_pressure(P, rho[p]);
        double Vb = 0.0, prb = 0.0;
        const double *sp = sig + p * 9;
        for (int k = 0; k < S.count; ++k) {
            long i = S.node[k];
            double phi = S.phi[k], r[3];
            for (int b = 0; b < d; ++b) r[b] = S.xi[k][b] - xp[b];
            double phib = mp * gmb[i], gradb[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) {
                double qa = vpp[a];
                for (int b = 0; b < d; ++b) qa += M[a * d + b] * r[b];
                double qb = gqb[i * d + a], fb = gfb[i * d + a];
                phib += mp * qb * qa + mp * fb * P->gravity[a];
                vb0[p * d + a] += phi * mp * qb;
                for (int b = 0; b < d; ++b) {
                    Mb[a * d + b] += phi * mp * qb * r[b];
                    xb0[p * d + b] += -phi * mp * qb * M[a * d + b];
                }
                /* f_a = -V sigma_ab grad_b (fluid: sigma = -p I, f_a = V p grad_a) */
                if (sand) {
                    for (int b = 0; b < d; ++b) {
                        gradb[b] += -Vp * sp[a * 3 + b] * fb;
                        Vb += -sp[a * 3 + b] * S.grad[k][b] * fb;
                        sigb0[p * 9 + a * 3 + b] += -Vp * S.grad[k][b] * fb;
                    }
                } else {
                    gradb[a] += Vp * pr * fb;
                    Vb += pr * fb * S.grad[k][a];
                    prb += Vp * fb * S.grad[k][a];
                }
            }
            double H[9];
            stencil_hessian(P, xp, &S, k, H);
            for (int b = 0; b < d; ++b) {
                double hb = 0.0;
                for (int a = 0; a < d; ++a) hb += H[b * d + a] * gradb[a];
                xb0[p * d + b] += phib * S.grad[k][b] + hb;
            }
        }
        /* M = B Dinv -> Bbar = Mbar Dinv^T */
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double s = 0.0;
                for (int c = 0; c < d; ++c) s += Mb[a * d + c] * Dinv[b * d + c];
                Bb0[p * d * d + a * d + b] = s;
            }
        rhob0[p] += Vb * (-mp / (rho[p] * rho[p])) + (sand ? 0.0 : prb * tait_dpdrho(P, rho[p]));
    }
    free(gm); free(gq); free(gf); free(gu); free(gv); free(gvb); free(gqb); free(gfb); free(gmb); free(sig);
    return 0;
}
