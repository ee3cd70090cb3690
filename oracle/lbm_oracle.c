/*
 * FP64 CPU oracle of the two-component pseudo-potential lattice Boltzmann
 * step on D3Q19 (and, for the paper's two-dimensional experiments of
 * Sec. III, on D2Q9) with the multiscale models of arXiv 2512.21696.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
 * leg of the benchmark call this file; the library path never does.  It shares
 * no code, header, table or constant with the CUDA library: everything below
 * is written from the paper's equations, cell by cell, in the paper's order,
 * with no blocking, fusion or storage tricks.
 *
 * What it computes (sections/equations of the paper):
 *   - LB equation, D3Q19, Eq. 2 (Sec. II); streaming with halfway bounce-back
 *     at solid cells (walls of Sec. I.B, III.B).
 *   - Collision projected on the Hermite basis (Sec. II, ref. [20]) to second
 *     order, with the force term of Eq. 3.  Reading: the non-equilibrium
 *     second moment carries the half-step force correction
 *     Pi1 = sum c c (f - feq) + (uF + Fu)/2 and the post-collision state is
 *     feq + (1 - 1/tau) w Q:Pi1 / (2 cs^4) + Fi/2, which has the zeroth,
 *     first and second moments of BGK with the same force term (Guo-consistent
 *     reading of Eq. 3 with u = (j + F/2)/rho).
 *   - Shan-Chen inter-component force with psi = rho (Sec. II, refs. [15,16]);
 *     solid neighbours carry virtual wall densities rho_wall.
 *   - CSF surface-tension control, Eq. 4, with phi^a = rho^{other}.  Reading
 *     of the divergence of the unit normal: with g = grad phi, H its Hessian
 *     and the regularised normal n = g / s, s = sqrt(|g|^2 + eps_n^2),
 *     div n = tr(H)/s - g.H.g / s^3 (curvature identity), evaluated with the
 *     isotropic D3Q19 gradient and the D3Q19 moment Hessian of the cell's own
 *     neighbourhood (solid neighbours carry rho_wall).  The other reading,
 *     selectable for the pins that bound the choice (csf_div = 1), is the
 *     isotropic divergence (1/cs^2) sum_i w_i n(x + c_i) . c_i of the unit
 *     normals n = g / max(|g|, eps_n) at the neighbours (zero at solid
 *     neighbours and outside).
 *   - Multiscale force of Eq. 1 in gray cells: capillary term
 *     -Pc(Sw) rho_r n H and the viscous resistance, the latter made tensorial
 *     by Eqs. 6-7 (principal axis from the Hessian and gradient of porosity,
 *     abstract and Sec. II) and solved semi-implicitly for the velocity.
 *     Reading: the top eigenvector of M = H H + c_g grad phi grad phi^T is
 *     the low-permeability axis, a tie of the two largest eigenvalues
 *     (within 1e-12 of the largest, floor 1e-30) means no axis, and the
 *     gradient is summed over opposite velocity pairs so that a flat
 *     neighbourhood gives M = 0 exactly.
 *   - Residual components (Sec. II, Eq. 5 and Fig. 6): crossings of the
 *     Leverett-scaled Pc(Sw; phi) with Pc_ref,max / Pc_ref,min give the
 *     residual water / oil amounts, switched on by a hysteresis on the local
 *     normalised wetting density and counted separately from the lattice.
 *   - Constitutive curves: Kozeny-Carman K0(phi) (Appendix), Corey Kr(Sw),
 *     and Pc(Sw) either Brooks-Corey or the Thomeer hyperbola the Appendix
 *     fits (its coefficients are in the paper's ref. [12]; here the pore-
 *     geometrical factor is an input).  Reading of the Thomeer form: the
 *     normalised non-wetting saturation 1 - Se obeys
 *     ln(1 - Se) log10(Pc / Pe) = -G with the entry pressure Pe = lamL Pd,
 *     i.e. Pc = Pe 10^(-G / ln(1 - Se)), capped at 10 Pe (the cap the
 *     Brooks-Corey clamp Se >= 1e-2 gives at lambda = 2).
 *
 *   - Pressure boundaries (the imbibition set-ups of Sec. I and the Appendix:
 *     a pressure difference between two boundaries of the domain, lowered in
 *     steps).  Reading: inlet / outlet cells are reservoirs held at given
 *     component densities at rest.  In every step such a cell takes its
 *     prescribed densities as its moments (so the force stencils of its
 *     neighbours see them), carries no force and no velocity, and leaves the
 *     collision as the rest equilibrium of those densities, which then
 *     streams into the domain.  The pressure of a reservoir is
 *     p = cs^2 (rhoA + rhoB) + G rhoA rhoB.
 *
 *   - Mass-sink-source (the Appendix's relative-permeability runs move the
 *     saturation between stages by injecting water near the oil-water
 *     interface; its definition is in the paper's refs. [12, 15]).  Reading:
 *     in every fluid cell that is not a reservoir, the collision adds the
 *     rest equilibrium w_i dm to the wetting component and w_i (-dm) to the
 *     other, dm = m I, with m the run's rate (lattice density per step) and
 *     I = max(0, (4 r_w r_n - I_b) / (1 - I_b)), r = rho^a / (rho^w + rho^n),
 *     I_b = 4 r_lo r_hi the value in either bulk: zero in the bulks, one in
 *     the middle of an interface.  Cell mass and momentum are unchanged.
 *   - D2Q9: the same step on one plane with the nine-velocity set (weights
 *     4/9, 1/9, 1/36, cs^2 = 1/3); every formula above is written for
 *     three-component vectors whose z parts vanish, and the identity in the
 *     density Hessian of Eq. 4 is that of the plane.
 *
 * Order inside one step: stream; moments at all cells; residual update;
 * density gradients at all cells; forces and velocity; collide.
 * Every force reads neighbour densities of the same time level.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_TYPES 16

enum { PORE = 0, SOLID = 1, GRAY = 2, INLET = 3, OUTLET = 4 };
enum { T_SC = 0, T_CSF = 1, T_CAP = 2, T_DRAG = 3, T_BODY = 4, N_TERM = 5 };

typedef struct {
    int nx, ny, nz;
    int periodic[3];
    double tau[2];
    double G;
    double kappa;
    double phi_avg[2];
    double phi_max[2];
    int csf_everywhere;
    double rho_wall[2];
    double accel[2][3];
    int wet;
    double rho_hi, rho_lo;
    double s_lo, s_hi, at_cut, eps_n, kr_min, c_g;
    double rho_in[2], rho_out[2]; /* densities held in inlet / outlet cells */
    int lattice;                  /* 0: D3Q19; 1: D2Q9 (nz = 1) */
    double mss;                   /* mass-sink-source rate m (0: off) */
    int csf_div;                  /* Eq. 4 divergence: 0 curvature identity, 1 neighbour normals */
} orc_params;

typedef struct {
    double kc_d, pd, lambda, swr, nw, nn, phi_ref, f_max, f_min, aniso;
    double thomeer_g; /* > 0: Thomeer Pc with this factor; 0: Brooks-Corey */
} orc_curve;

/* D3Q19 velocities: rest, the 6 faces, the 12 edges. */
static const int CV19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
/* D2Q9 velocities (the plane z = 0): rest, the 4 faces, the 4 diagonals. */
static const int CV9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};

static const double CS2 = 1.0 / 3.0;

/* A velocity set: Q velocities in `dim` dimensions (z components zero in 2-D),
 * their weights and opposites.  Both sets have cs^2 = 1/3. */
typedef struct {
    int Q, dim;
    int cv[19][3];
    double w[19];
    int opp[19];
} lattice;

static void make_lattice(lattice *L, int d2q9)
{
    L->Q = d2q9 ? 9 : 19;
    L->dim = d2q9 ? 2 : 3;
    for (int i = 0; i < L->Q; ++i)
        for (int d = 0; d < 3; ++d) L->cv[i][d] = d2q9 ? CV9[i][d] : CV19[i][d];
    for (int i = 0; i < L->Q; ++i) {
        int len2 = L->cv[i][0] * L->cv[i][0] + L->cv[i][1] * L->cv[i][1] + L->cv[i][2] * L->cv[i][2];
        if (d2q9)
            L->w[i] = len2 == 0 ? 4.0 / 9.0 : (len2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        else
            L->w[i] = len2 == 0 ? 1.0 / 3.0 : (len2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        L->opp[i] = -1;
        for (int k = 0; k < L->Q; ++k)
            if (L->cv[k][0] == -L->cv[i][0] && L->cv[k][1] == -L->cv[i][1] && L->cv[k][2] == -L->cv[i][2])
                L->opp[i] = k;
    }
}

typedef struct orc_state {
    orc_params p;
    lattice L;
    long n;
    uint8_t *type, *ptype;
    double *phi;
    orc_curve curve[ORC_MAX_TYPES];
    int ncurve;
    /* per gray cell, from the geometry */
    double *K0, *lamL, *swirr, *sores, *kinv, *e1;
    int *iso;
    /* residual components */
    double *Rw, *Ro;
    int *wetflag;
    /* populations [a][i][cell]: post-collision f, streamed fs */
    double *f, *fs;
    /* fields of the last step */
    double *rho[2], *j, *u, *sw, *s;
    double *grad[2];
    double *term[N_TERM][2];
    double *F[2];
    long steps;
} orc_state;

static long cell_index(const orc_state *st, int x, int y, int z)
{
    return (long)x + (long)st->p.nx * ((long)y + (long)st->p.ny * (long)z);
}

static void cell_coords(const orc_state *st, long c, int *x, int *y, int *z)
{
    *x = (int)(c % st->p.nx);
    *y = (int)((c / st->p.nx) % st->p.ny);
    *z = (int)(c / ((long)st->p.nx * st->p.ny));
}

/* Index of (x+dx, y+dy, z+dz), wrapped on periodic axes, -1 if outside. */
static long neighbour(const orc_state *st, long c, int dx, int dy, int dz)
{
    int x, y, z;
    cell_coords(st, c, &x, &y, &z);
    int q[3] = {x + dx, y + dy, z + dz};
    int N[3] = {st->p.nx, st->p.ny, st->p.nz};
    for (int d = 0; d < 3; ++d) {
        if (q[d] < 0 || q[d] >= N[d]) {
            if (!st->p.periodic[d]) return -1;
            q[d] = ((q[d] % N[d]) + N[d]) % N[d];
        }
    }
    return cell_index(st, q[0], q[1], q[2]);
}

static int is_wall(const orc_state *st, long m) { return m < 0 || st->type[m] == SOLID; }

/* Density of component a as seen by a stencil at cell m (virtual wall value). */
static double rho_seen(const orc_state *st, long m, int a)
{
    return is_wall(st, m) ? st->p.rho_wall[a] : st->rho[a][m];
}

static double phi_seen(const orc_state *st, long m) { return m < 0 ? 0.0 : st->phi[m]; }

/* Prescribed density of component a in pressure cell c (inlet or outlet). */
static int is_pressure(const orc_state *st, long c) { return st->type[c] == INLET || st->type[c] == OUTLET; }
static double rho_held(const orc_state *st, long c, int a)
{
    return st->type[c] == INLET ? st->p.rho_in[a] : st->p.rho_out[a];
}

static double *alloc0(long count) { return (double *)calloc((size_t)count, sizeof(double)); }

/* ---------------------------------------------------------------------- */
/* Constitutive curves                                                       */
/* ---------------------------------------------------------------------- */

/* Kozeny-Carman absolute permeability (Appendix: fitted K0(phi)). */
static double kozeny_carman(const orc_curve *cv, double phi)
{
    return cv->kc_d * cv->kc_d * phi * phi * phi / (180.0 * (1.0 - phi) * (1.0 - phi));
}

/* Leverett J-function similarity, Eq. 5: Pc sqrt(K0/phi) is the same for all
 * phi, so Pc(Sw; phi) = Pc(Sw; phi_ref) * sqrt((K0_ref/phi_ref)/(K0/phi)). */
static double leverett_factor(const orc_curve *cv, double phi)
{
    double kref = kozeny_carman(cv, cv->phi_ref);
    double k = kozeny_carman(cv, phi);
    return sqrt((kref / cv->phi_ref) / (k / phi));
}

/* Water saturation on the capillary-pressure curve at pressure p (the
 * inverse of the curve, without its cap; Se = 1 at or below entry):
 * Brooks-Corey Se = (p/Pe)^(-lambda); Thomeer 1 - Se = exp(-G / log10(p/Pe)). */
static double sw_at_pressure(const orc_curve *cv, double lamL, double p)
{
    double ratio = p / (lamL * cv->pd);
    double se;
    if (cv->thomeer_g > 0.0)
        se = ratio <= 1.0 ? 1.0 : 1.0 - exp(-cv->thomeer_g / log10(ratio));
    else
        se = pow(ratio, -cv->lambda);
    if (se > 1.0) se = 1.0;
    return cv->swr + (1.0 - cv->swr) * se;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Capillary pressure, Se clamped to [1e-2, 1]: Brooks-Corey Pe Se^(-1/lambda),
 * or Thomeer Pe 10^min(-G / ln(1 - Se), 1). */
static double capillary_pressure(const orc_curve *cv, double lamL, double sw)
{
    double se = clampd((sw - cv->swr) / (1.0 - cv->swr), 1e-2, 1.0);
    if (cv->thomeer_g > 0.0) {
        double e = -cv->thomeer_g / log(1.0 - se); /* 0 at se = 1 */
        return lamL * cv->pd * pow(10.0, e < 1.0 ? e : 1.0);
    }
    return lamL * cv->pd * pow(se, -1.0 / cv->lambda);
}

/* ---------------------------------------------------------------------- */
/* Symmetric 3x3 eigen-decomposition: cyclic Jacobi rotations              */
/* ---------------------------------------------------------------------- */
static void jacobi3(double A[3][3], double evals[3], double V[3][3])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) V[r][c] = (r == c) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        double dia = A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2];
        if (off <= 1e-32 * dia || off == 0.0) break;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0);
                double s = t * c;
                /* A <- J^T A J with J the (p,q) rotation */
                for (int k = 0; k < 3; ++k) {
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int k = 0; k < 3; ++k) evals[k] = A[k][k];
}

/* Hessian of the density of component a at fluid cell c from the lattice
 * moments: since sum_i w_i (c_i c_i - cs^2 I) c_i c_i : X = 2 cs^4 X for
 * symmetric X on D3Q19 (and on D2Q9 in its plane), H = (1/cs^4) sum_i w_i
 * (c_i c_i - cs^2 I) (rho(x + c_i) - rho(x)), I the identity of the lattice's
 * dimensions, solid neighbours carrying rho_wall. */
static void density_hessian(const orc_state *st, long c, int a, double H[3][3])
{
    const lattice *L = &st->L;
    double fc = st->rho[a][c];
    for (int d = 0; d < 3; ++d)
        for (int e = 0; e < 3; ++e) H[d][e] = 0.0;
    for (int i = 1; i < L->Q; ++i) {
        double df = rho_seen(st, neighbour(st, c, L->cv[i][0], L->cv[i][1], L->cv[i][2]), a) - fc;
        for (int d = 0; d < 3; ++d)
            for (int e = 0; e < 3; ++e)
                H[d][e] += L->w[i] * (L->cv[i][d] * L->cv[i][e] - (d == e && d < L->dim ? CS2 : 0.0)) * df /
                           (CS2 * CS2);
    }
}

/* Geometry precompute for gray cell c (Eqs. 5-7). */
static void gray_static(orc_state *st, long c)
{
    const orc_curve *cv = &st->curve[st->ptype[c]];
    double phi = st->phi[c];
    /* gradient with the isotropic stencil of the lattice, written as central
     * differences over the opposite pairs (i < opp[i]): the same sum, and a
     * flat neighbourhood gives exactly zero */
    const lattice *L = &st->L;
    double g[3] = {0, 0, 0};
    for (int i = 1; i < L->Q; ++i) {
        if (L->opp[i] < i) continue;
        double vp = phi_seen(st, neighbour(st, c, L->cv[i][0], L->cv[i][1], L->cv[i][2]));
        double vm = phi_seen(st, neighbour(st, c, -L->cv[i][0], -L->cv[i][1], -L->cv[i][2]));
        for (int d = 0; d < 3; ++d) g[d] += L->w[i] * (vp - vm) * L->cv[i][d] / CS2;
    }
    /* Hessian: second differences on the faces, four-point cross terms */
    double H[3][3];
    for (int a = 0; a < 3; ++a) {
        int ea[3] = {0, 0, 0};
        ea[a] = 1;
        double fp = phi_seen(st, neighbour(st, c, ea[0], ea[1], ea[2]));
        double fm = phi_seen(st, neighbour(st, c, -ea[0], -ea[1], -ea[2]));
        H[a][a] = fp - 2.0 * phi + fm;
        for (int b = a + 1; b < 3; ++b) {
            int eb[3] = {0, 0, 0};
            eb[b] = 1;
            double pp = phi_seen(st, neighbour(st, c, ea[0] + eb[0], ea[1] + eb[1], ea[2] + eb[2]));
            double pm = phi_seen(st, neighbour(st, c, ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]));
            double mp = phi_seen(st, neighbour(st, c, -ea[0] + eb[0], -ea[1] + eb[1], -ea[2] + eb[2]));
            double mm = phi_seen(st, neighbour(st, c, -ea[0] - eb[0], -ea[1] - eb[1], -ea[2] - eb[2]));
            H[a][b] = H[b][a] = 0.25 * (pp - pm - mp + mm);
        }
    }
    /* M = H H + c_g g g^T; its top eigenvector is the low-permeability axis */
    double M[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += H[a][k] * H[k][b];
            M[a][b] = acc + st->p.c_g * g[a] * g[b];
        }
    double ev[3], V[3][3];
    jacobi3(M, ev, V);
    int top = 0;
    for (int k = 1; k < 3; ++k)
        if (ev[k] > ev[top]) top = k;
    double second = -INFINITY;
    for (int k = 0; k < 3; ++k)
        if (k != top && ev[k] > second) second = ev[k];
    double mu1 = ev[top];
    int iso = (mu1 - second) <= 1e-12 * fmax(mu1, 1e-30);
    double e[3] = {V[0][top], V[1][top], V[2][top]};
    double K0 = kozeny_carman(cv, phi);
    st->K0[c] = K0;
    st->iso[c] = iso;
    for (int d = 0; d < 3; ++d) st->e1[3 * c + d] = iso ? 0.0 : e[d];
    /* K = B K^D B^-1 with K^D = diag(K0/a, K0, K0); B orthonormal.  Its
     * inverse is (1/K0) (I + (a-1) e1 e1^T). */
    double am1 = cv->aniso - 1.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = (a == b) ? 1.0 : 0.0;
            if (!iso) v += am1 * e[a] * e[b];
            st->kinv[9 * c + 3 * a + b] = v / K0;
        }
    double lamL = leverett_factor(cv, phi);
    st->lamL[c] = lamL;
    double pc_pm = cv->pd; /* critical pressure of the typical region (phi_ref) */
    st->swirr[c] = sw_at_pressure(cv, lamL, cv->f_max * pc_pm);
    st->sores[c] = 1.0 - sw_at_pressure(cv, lamL, cv->f_min * pc_pm);
}

/* ---------------------------------------------------------------------- */
/* Collision of one component at one cell                                  */
/* ---------------------------------------------------------------------- */
static void equilibrium(const lattice *L, double rho, const double u[3], double feq[19])
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->Q; ++i) {
        double cu = L->cv[i][0] * u[0] + L->cv[i][1] * u[1] + L->cv[i][2] * u[2];
        feq[i] = L->w[i] * rho * (1.0 + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
    }
}

/* Eq. 3 force term F_i for force F at velocity u (in 2-D, u and F have no
 * z component, so the zz entry of c c - cs^2 I meets zeros). */
static double force_term(const lattice *L, int i, const double u[3], const double F[3])
{
    double cF = 0.0, sec = 0.0;
    for (int a = 0; a < 3; ++a) cF += L->cv[i][a] * F[a];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double Q = L->cv[i][a] * L->cv[i][b] - (a == b ? CS2 : 0.0);
            sec += (u[a] * F[b] + F[a] * u[b]) * Q;
        }
    return L->w[i] * (cF / CS2 + sec / (2.0 * CS2 * CS2));
}

static void collide_cell(const lattice *L, const double *fin, const double u[3], const double F[3], double tau,
                         double *fout)
{
    double rho = 0.0;
    for (int i = 0; i < L->Q; ++i) rho += fin[i];
    double feq[19];
    equilibrium(L, rho, u, feq);
    double P[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int i = 0; i < L->Q; ++i) acc += L->cv[i][a] * L->cv[i][b] * (fin[i] - feq[i]);
            P[a][b] = acc + 0.5 * (u[a] * F[b] + F[a] * u[b]);
        }
    for (int i = 0; i < L->Q; ++i) {
        double QP = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) QP += (L->cv[i][a] * L->cv[i][b] - (a == b ? CS2 : 0.0)) * P[a][b];
        fout[i] = feq[i] + (1.0 - 1.0 / tau) * L->w[i] * QP / (2.0 * CS2 * CS2) + 0.5 * force_term(L, i, u, F);
    }
}

/* One D3Q19 cell (exported for the moment-identity tests). */
void orc_collide_cell(const double fin[19], const double u[3], const double F[3], double tau,
                      double fout[19])
{
    lattice L;
    make_lattice(&L, 0);
    collide_cell(&L, fin, u, F, tau, fout);
}

/* Solve A x = b (3x3) by Gaussian elimination with partial pivoting. */
static void solve3(double A[3][3], const double b[3], double x[3])
{
    double M[3][4];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) M[r][c] = A[r][c];
        M[r][3] = b[r];
    }
    for (int k = 0; k < 3; ++k) {
        int piv = k;
        for (int r = k + 1; r < 3; ++r)
            if (fabs(M[r][k]) > fabs(M[piv][k])) piv = r;
        if (piv != k)
            for (int c = 0; c < 4; ++c) {
                double t = M[k][c];
                M[k][c] = M[piv][c];
                M[piv][c] = t;
            }
        for (int r = k + 1; r < 3; ++r) {
            double fct = M[r][k] / M[k][k];
            for (int c = k; c < 4; ++c) M[r][c] -= fct * M[k][c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double acc = M[r][3];
        for (int c = r + 1; c < 3; ++c) acc -= M[r][c] * x[c];
        x[r] = acc / M[r][r];
    }
}

/* ---------------------------------------------------------------------- */
/* State management                                                         */
/* ---------------------------------------------------------------------- */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_destroy(orc_state *st)
{
    if (!st) return;
    free(st->type); free(st->ptype); free(st->phi);
    free(st->K0); free(st->lamL); free(st->swirr); free(st->sores); free(st->kinv); free(st->e1);
    free(st->iso); free(st->Rw); free(st->Ro); free(st->wetflag);
    free(st->f); free(st->fs);
    for (int a = 0; a < 2; ++a) {
        free(st->rho[a]); free(st->grad[a]); free(st->F[a]);
        for (int t = 0; t < N_TERM; ++t) free(st->term[t][a]);
    }
    free(st->j); free(st->u); free(st->sw); free(st->s);
    free(st);
}

/* type: cell codes; phi: porosity of gray cells (pore is 1, solid 0 whatever
 * is passed); ptype: pore-type index of each cell into `curves`. */
orc_state *orc_create(const orc_params *p, const orc_curve *curves, int ncurve,
                      const uint8_t *type, const double *phi, const uint8_t *ptype)
{
    if (ncurve < 1 || ncurve > ORC_MAX_TYPES) return NULL;
    if (p->lattice == 1 && p->nz != 1) return NULL;
    orc_state *st = (orc_state *)calloc(1, sizeof(orc_state));
    st->p = *p;
    make_lattice(&st->L, p->lattice == 1);
    if (p->lattice == 1) st->p.periodic[2] = 1; /* one plane: z-invariant stencils */
    st->n = (long)p->nx * p->ny * p->nz;
    long n = st->n;
    st->ncurve = ncurve;
    memcpy(st->curve, curves, sizeof(orc_curve) * (size_t)ncurve);
    st->type = (uint8_t *)malloc((size_t)n);
    st->ptype = (uint8_t *)malloc((size_t)n);
    memcpy(st->type, type, (size_t)n);
    for (long c = 0; c < n; ++c) st->ptype[c] = ptype ? ptype[c] : 0;
    st->phi = alloc0(n);
    for (long c = 0; c < n; ++c)
        st->phi[c] = type[c] == SOLID ? 0.0 : (type[c] == GRAY ? phi[c] : 1.0);
    st->K0 = alloc0(n); st->lamL = alloc0(n); st->swirr = alloc0(n); st->sores = alloc0(n);
    st->kinv = alloc0(9 * n); st->e1 = alloc0(3 * n);
    st->iso = (int *)calloc((size_t)n, sizeof(int));
    st->Rw = alloc0(n); st->Ro = alloc0(n);
    st->wetflag = (int *)calloc((size_t)n, sizeof(int));
    st->f = alloc0(2 * (long)st->L.Q * n);
    st->fs = alloc0(2 * (long)st->L.Q * n);
    for (int a = 0; a < 2; ++a) {
        st->rho[a] = alloc0(n); st->grad[a] = alloc0(3 * n);
        st->F[a] = alloc0(3 * n);
        for (int t = 0; t < N_TERM; ++t) st->term[t][a] = alloc0(3 * n);
    }
    st->j = alloc0(3 * n); st->u = alloc0(3 * n); st->sw = alloc0(n); st->s = alloc0(n);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c)
        if (st->type[c] == GRAY) gray_static(st, c);
    return st;
}

static double rel_wet(const orc_state *st, double rw, double rn)
{
    (void)st;
    return rw / (rw + rn);
}

static double normalised_wet(const orc_state *st, double rho_w, double rho_n)
{
    double r_lo = st->p.rho_lo / (st->p.rho_hi + st->p.rho_lo);
    double r_hi = st->p.rho_hi / (st->p.rho_hi + st->p.rho_lo);
    return clampd((rel_wet(st, rho_w, rho_n) - r_lo) / (r_hi - r_lo), 0.0, 1.0);
}

/* Equilibrium populations of the given densities and velocity (u may be
 * NULL for rest).  The residual flag starts from the local normalised wetting
 * density: wet when s >= 1/2; no residual amount is held yet. */
void orc_init_fields(orc_state *st, const double *rhoA, const double *rhoB, const double *u)
{
    long n = st->n;
    int w = st->p.wet;
    for (long c = 0; c < n; ++c) {
        double uc[3] = {0, 0, 0};
        if (u)
            for (int d = 0; d < 3; ++d) uc[d] = u[d * n + c];
        double r[2] = {rhoA[c], rhoB[c]};
        for (int a = 0; a < 2; ++a) {
            double feq[19];
            const int Q = st->L.Q;
            equilibrium(&st->L, r[a], uc, feq);
            for (int i = 0; i < Q; ++i) st->f[((long)a * Q + i) * n + c] = st->type[c] == SOLID ? 0.0 : feq[i];
            st->rho[a][c] = st->type[c] == SOLID ? 0.0 : r[a];
        }
        for (int d = 0; d < 3; ++d) st->u[d * n + c] = st->type[c] == SOLID ? 0.0 : uc[d];
        st->Rw[c] = st->Ro[c] = 0.0;
        if (st->type[c] != SOLID) {
            double s = normalised_wet(st, r[w], r[1 - w]);
            st->s[c] = s;
            st->sw[c] = s;
            st->wetflag[c] = s >= 0.5;
        } else {
            st->s[c] = st->sw[c] = 0.0;
            st->wetflag[c] = 0;
        }
    }
    st->steps = 0;
}

/* New mass-sink-source rate, used from the next step on. */
void orc_set_mss(orc_state *st, double rate) { st->p.mss = rate; }

/* New reservoir densities, used from the next step on. */
void orc_set_pressure(orc_state *st, const double rho_in[2], const double rho_out[2])
{
    for (int a = 0; a < 2; ++a) {
        st->p.rho_in[a] = rho_in[a];
        st->p.rho_out[a] = rho_out[a];
    }
}

/* Populations [2][Q][n] (Q = 19 or 9). */
void orc_set_populations(orc_state *st, const double *f) { memcpy(st->f, f, sizeof(double) * 2 * st->L.Q * (size_t)st->n); }
void orc_get_populations(const orc_state *st, double *f) { memcpy(f, st->f, sizeof(double) * 2 * st->L.Q * (size_t)st->n); }
int orc_q(const orc_state *st) { return st->L.Q; }
void orc_set_residual(orc_state *st, const double *Rw, const double *Ro, const int *wet)
{
    memcpy(st->Rw, Rw, sizeof(double) * (size_t)st->n);
    memcpy(st->Ro, Ro, sizeof(double) * (size_t)st->n);
    memcpy(st->wetflag, wet, sizeof(int) * (size_t)st->n);
}
void orc_get_residual(const orc_state *st, double *Rw, double *Ro, int *wet)
{
    memcpy(Rw, st->Rw, sizeof(double) * (size_t)st->n);
    memcpy(Ro, st->Ro, sizeof(double) * (size_t)st->n);
    memcpy(wet, st->wetflag, sizeof(int) * (size_t)st->n);
}

/* ---------------------------------------------------------------------- */
/* One time step                                                            */
/* ---------------------------------------------------------------------- */
static void one_step(orc_state *st)
{
    const long n = st->n;
    const orc_params *p = &st->p;
    const int w = p->wet;
    const lattice *L = &st->L;
    const int Q = L->Q;
    const int *opp = L->opp;

    /* (1) streaming with halfway bounce-back, (2) moments */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        if (st->type[c] == SOLID) continue;
        double jc[3] = {0, 0, 0};
        for (int a = 0; a < 2; ++a) {
            double r = 0.0;
            for (int i = 0; i < Q; ++i) {
                long src = neighbour(st, c, -L->cv[i][0], -L->cv[i][1], -L->cv[i][2]);
                double v = is_wall(st, src) ? st->f[((long)a * Q + opp[i]) * n + c]
                                            : st->f[((long)a * Q + i) * n + src];
                st->fs[((long)a * Q + i) * n + c] = v;
                r += v;
                for (int d = 0; d < 3; ++d) jc[d] += L->cv[i][d] * v;
            }
            st->rho[a][c] = is_pressure(st, c) ? rho_held(st, c, a) : r;
        }
        for (int d = 0; d < 3; ++d) st->j[d * n + c] = is_pressure(st, c) ? 0.0 : jc[d];
    }

    /* (3) residual components: hysteresis on the normalised wetting density */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        if (st->type[c] == SOLID) continue;
        double s = normalised_wet(st, st->rho[w][c], st->rho[1 - w][c]);
        st->s[c] = s;
        if (st->type[c] == GRAY) {
            if (st->wetflag[c] && s < p->s_lo) {
                st->Rw[c] = st->swirr[c];
                st->Ro[c] = 0.0;
                st->wetflag[c] = 0;
            } else if (!st->wetflag[c] && s > p->s_hi) {
                st->Ro[c] = st->sores[c];
                st->Rw[c] = 0.0;
                st->wetflag[c] = 1;
            }
            st->sw[c] = st->Rw[c] + (1.0 - st->Rw[c] - st->Ro[c]) * s;
        } else {
            st->sw[c] = s;
        }
    }

    /* (4a) gradient of phi^a = rho^{other} at every fluid cell */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        for (int a = 0; a < 2; ++a) {
            double g[3] = {0, 0, 0};
            if (st->type[c] != SOLID) {
                for (int i = 0; i < Q; ++i) {
                    long m = neighbour(st, c, L->cv[i][0], L->cv[i][1], L->cv[i][2]);
                    double v = rho_seen(st, m, 1 - a);
                    for (int d = 0; d < 3; ++d) g[d] += L->w[i] * v * L->cv[i][d] / CS2;
                }
            }
            for (int d = 0; d < 3; ++d) st->grad[a][d * n + c] = g[d];
        }
    }

    /* (4b) forces and velocity */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        for (int t = 0; t < N_TERM; ++t)
            for (int a = 0; a < 2; ++a)
                for (int d = 0; d < 3; ++d) st->term[t][a][d * n + c] = 0.0;
        if (st->type[c] == SOLID || is_pressure(st, c)) {
            for (int d = 0; d < 3; ++d) st->u[d * n + c] = 0.0;
            for (int a = 0; a < 2; ++a)
                for (int d = 0; d < 3; ++d) st->F[a][d * n + c] = 0.0;
            continue;
        }
        const int gray = st->type[c] == GRAY;
        double r[2] = {st->rho[0][c], st->rho[1][c]};
        double rt = r[0] + r[1];
        double T[N_TERM][2][3];
        memset(T, 0, sizeof(T));
        for (int a = 0; a < 2; ++a) {
            for (int d = 0; d < 3; ++d) {
                double ga = st->grad[a][d * n + c];
                /* Shan-Chen: -G psi^a sum_i w_i psi^other(x+c_i) c_i / cs^2 */
                T[T_SC][a][d] = -p->G * r[a] * ga;
                T[T_BODY][a][d] = r[a] * p->accel[a][d];
            }
            if (p->kappa != 0.0 && (p->csf_everywhere || gray)) {
                /* Eq. 4: kappa (-div n^a) (grad phi^a / phi_avg) (rho^a / phi_max),
                 * div n = tr(H)/s - g.H.g/s^3, s = sqrt(|g|^2 + eps_n^2) */
                double div = 0.0;
                if (p->csf_div == 1) {
                    /* divergence of the neighbours' unit normals g / max(|g|, eps_n) */
                    for (int i = 1; i < Q; ++i) {
                        long m = neighbour(st, c, L->cv[i][0], L->cv[i][1], L->cv[i][2]);
                        if (m < 0) continue;
                        double gm[3], mag2 = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            gm[d] = st->grad[a][d * n + m];
                            mag2 += gm[d] * gm[d];
                        }
                        double den = fmax(sqrt(mag2), p->eps_n);
                        for (int d = 0; d < 3; ++d) div += L->w[i] * (gm[d] / den) * L->cv[i][d] / CS2;
                    }
                } else {
                    double H[3][3], g[3];
                    density_hessian(st, c, 1 - a, H);
                    for (int d = 0; d < 3; ++d) g[d] = st->grad[a][d * n + c];
                    double s = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2] + p->eps_n * p->eps_n);
                    double gHg = 0.0;
                    for (int d = 0; d < 3; ++d)
                        for (int e = 0; e < 3; ++e) gHg += g[d] * H[d][e] * g[e];
                    div = (H[0][0] + H[1][1] + H[2][2]) / s - gHg / (s * s * s);
                }
                for (int d = 0; d < 3; ++d)
                    T[T_CSF][a][d] = p->kappa * (-div) * (st->grad[a][d * n + c] / p->phi_avg[a]) *
                                     (r[a] / p->phi_max[a]);
            }
        }
        double jc[3] = {st->j[c], st->j[n + c], st->j[2 * n + c]};
        double uc[3];
        if (gray) {
            const orc_curve *cv = &st->curve[st->ptype[c]];
            /* Atwood number of wetting vs non-wetting, its gradient and normal */
            double At_c = (r[w] - r[1 - w]) / (r[w] + r[1 - w]);
            double dAt[3] = {0, 0, 0};
            for (int i = 0; i < Q; ++i) {
                long m = neighbour(st, c, L->cv[i][0], L->cv[i][1], L->cv[i][2]);
                double rw = rho_seen(st, m, w), rn = rho_seen(st, m, 1 - w);
                double At = (rw + rn > 0.0) ? (rw - rn) / (rw + rn) : 0.0;
                for (int d = 0; d < 3; ++d) dAt[d] += L->w[i] * At * L->cv[i][d] / CS2;
            }
            double mag = sqrt(dAt[0] * dAt[0] + dAt[1] * dAt[1] + dAt[2] * dAt[2]);
            double H = (fabs(At_c) <= p->at_cut) ? 0.5 * mag : 0.0;
            if (H > 0.0) {
                double Pc = capillary_pressure(cv, st->lamL[c], st->sw[c]);
                for (int a = 0; a < 2; ++a)
                    for (int d = 0; d < 3; ++d)
                        T[T_CAP][a][d] = -Pc * (r[a] / rt) * (dAt[d] / fmax(mag, p->eps_n)) * H;
            }
            /* Eq. 1 viscous resistance, tensorial by Eq. 7 */
            double se = clampd((st->sw[c] - cv->swr) / (1.0 - cv->swr), 0.0, 1.0);
            double kr[2];
            kr[w] = pow(se, cv->nw);
            kr[1 - w] = pow(1.0 - se, cv->nn);
            double coef = 0.0;
            for (int b = 0; b < 2; ++b) {
                double nu = (p->tau[b] - 0.5) / 3.0;
                if (r[b] != 0.0) coef += r[b] * nu / fmax(kr[b], p->kr_min);
            }
            double R[3][3], A[3][3], rhs[3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    R[a][b] = coef * st->kinv[9 * c + 3 * a + b];
                    A[a][b] = (a == b ? rt : 0.0) + 0.5 * R[a][b];
                }
            for (int d = 0; d < 3; ++d) {
                double Fo = 0.0;
                for (int a = 0; a < 2; ++a) Fo += T[T_SC][a][d] + T[T_CSF][a][d] + T[T_CAP][a][d] + T[T_BODY][a][d];
                rhs[d] = jc[d] + 0.5 * Fo;
            }
            /* semi-implicit velocity: (rho I + R/2) u = j + F_other/2 */
            solve3(A, rhs, uc);
            for (int a = 0; a < 2; ++a)
                for (int d = 0; d < 3; ++d) {
                    double Ru = R[d][0] * uc[0] + R[d][1] * uc[1] + R[d][2] * uc[2];
                    T[T_DRAG][a][d] = -(r[a] / rt) * Ru;
                }
        } else {
            for (int d = 0; d < 3; ++d) {
                double Ft = 0.0;
                for (int a = 0; a < 2; ++a) Ft += T[T_SC][a][d] + T[T_CSF][a][d] + T[T_BODY][a][d];
                uc[d] = (jc[d] + 0.5 * Ft) / rt;
            }
        }
        for (int d = 0; d < 3; ++d) st->u[d * n + c] = uc[d];
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 3; ++d) {
                double tot = 0.0;
                for (int t = 0; t < N_TERM; ++t) {
                    st->term[t][a][d * n + c] = T[t][a][d];
                    tot += T[t][a][d];
                }
                st->F[a][d * n + c] = tot;
            }
    }

    /* (5) collision */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < n; ++c) {
        if (st->type[c] == SOLID) continue;
        double uc[3] = {st->u[c], st->u[n + c], st->u[2 * n + c]};
        if (is_pressure(st, c)) {
            /* reservoir: the rest equilibrium of the held densities */
            for (int a = 0; a < 2; ++a) {
                double feq[19];
                equilibrium(L, st->rho[a][c], uc, feq);
                for (int i = 0; i < Q; ++i) st->f[((long)a * Q + i) * n + c] = feq[i];
            }
            continue;
        }
        /* mass-sink-source: dm = m I moved from the non-wetting to the wetting component */
        double dm = 0.0;
        if (p->mss != 0.0) {
            double rt = st->rho[0][c] + st->rho[1][c];
            double rw = st->rho[w][c] / rt, rn = st->rho[1 - w][c] / rt;
            double rlo = p->rho_lo / (p->rho_hi + p->rho_lo), rhi = p->rho_hi / (p->rho_hi + p->rho_lo);
            double Ib = 4.0 * rlo * rhi;
            double I = (4.0 * rw * rn - Ib) / (1.0 - Ib);
            dm = p->mss * (I > 0.0 ? I : 0.0);
        }
        for (int a = 0; a < 2; ++a) {
            double fin[19], fout[19], Fa[3];
            for (int i = 0; i < Q; ++i) fin[i] = st->fs[((long)a * Q + i) * n + c];
            for (int d = 0; d < 3; ++d) Fa[d] = st->F[a][d * n + c];
            collide_cell(L, fin, uc, Fa, p->tau[a], fout);
            double sgn = a == w ? 1.0 : -1.0;
            for (int i = 0; i < Q; ++i) st->f[((long)a * Q + i) * n + c] = fout[i] + sgn * L->w[i] * dm;
        }
    }
    st->steps += 1;
}

void orc_step(orc_state *st, int nsteps)
{
    for (int k = 0; k < nsteps; ++k) one_step(st);
}

/* ---------------------------------------------------------------------- */
/* Read-back                                                                */
/* ---------------------------------------------------------------------- */
/* rhoA, rhoB [n]; u [3][n]; sw [n]: fields of the last step (or of init). */
void orc_fields(const orc_state *st, double *rhoA, double *rhoB, double *u, double *sw)
{
    long n = st->n;
    if (rhoA) memcpy(rhoA, st->rho[0], sizeof(double) * (size_t)n);
    if (rhoB) memcpy(rhoB, st->rho[1], sizeof(double) * (size_t)n);
    if (u) memcpy(u, st->u, sizeof(double) * 3 * (size_t)n);
    if (sw) memcpy(sw, st->sw, sizeof(double) * (size_t)n);
}

/* Force term `term` of component a in the last step, [3][n]. */
void orc_force_term(const orc_state *st, int term, int a, double *out)
{
    memcpy(out, st->term[term][a], sizeof(double) * 3 * (size_t)st->n);
}

/* Geometry results: kinv [9][n] row-major per cell, K0, Leverett factor,
 * residual bounds, isotropic flag; zero outside gray cells. */
void orc_static(const orc_state *st, double *kinv, double *K0, double *lamL, double *swirr,
                double *sores, int *iso)
{
    long n = st->n;
    for (long c = 0; c < n; ++c)
        for (int k = 0; k < 9; ++k) kinv[(long)k * n + c] = st->kinv[9 * c + k];
    memcpy(K0, st->K0, sizeof(double) * (size_t)n);
    memcpy(lamL, st->lamL, sizeof(double) * (size_t)n);
    memcpy(swirr, st->swirr, sizeof(double) * (size_t)n);
    memcpy(sores, st->sores, sizeof(double) * (size_t)n);
    memcpy(iso, st->iso, sizeof(int) * (size_t)n);
}

/* Observables (S8) of fields given as arrays over an nx x ny x nz grid
 * (x fastest): out[0..1] mass of A and B; out[2] saturation
 * sum(phi_c Sw)/sum(phi_c) (phi_c = 1 in pore, phi in gray, pressure cells
 * left out); out[3] mean u_x over the outlet plane x = nx-1; out[4..6] volume
 * mean of u; out[7] max |u|; out[8] mean pressure inside radius r_in minus
 * outside r_out about the probe centre, p = cs^2 (rhoA+rhoB) + G rhoA rhoB;
 * out[9] count of non-finite density or velocity values (such cells are left
 * out of every sum).  probe = {cx, cy, cz, r_in, r_out}; u is [3][n]. */
void orc_observables_of(int nx, int ny, int nz, const unsigned char *type, const double *phi, const double *rhoA,
                        const double *rhoB, const double *u, const double *sw, double G, const double probe[5],
                        double out[10])
{
    long n = (long)nx * ny * nz;
    double mass[2] = {0, 0}, satn = 0, satd = 0, fout = 0, fv[3] = {0, 0, 0}, umax = 0;
    double pin = 0, nin = 0, pout = 0, nout = 0, bad = 0;
    for (long c = 0; c < n; ++c) {
        if (type[c] == SOLID) continue;
        int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long)nx * ny));
        double ra = rhoA[c], rb = rhoB[c];
        double u0 = u[c], u1 = u[n + c], u2 = u[2 * n + c];
        if (!isfinite(ra) || !isfinite(rb) || !isfinite(u0) || !isfinite(u1) || !isfinite(u2)) {
            bad += 1;
            continue;
        }
        mass[0] += ra;
        mass[1] += rb;
        if (type[c] != INLET && type[c] != OUTLET) {
            double phc = type[c] == GRAY ? phi[c] : 1.0;
            satn += phc * sw[c];
            satd += phc;
        }
        if (x == nx - 1) fout += u0;
        fv[0] += u0; fv[1] += u1; fv[2] += u2;
        double um = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
        if (um > umax) umax = um;
        double dx = x - probe[0], dy = y - probe[1], dz = z - probe[2];
        double r2 = dx * dx + dy * dy + dz * dz;
        double pr = CS2 * (ra + rb) + G * ra * rb;
        if (r2 < probe[3] * probe[3]) { pin += pr; nin += 1; }
        if (r2 > probe[4] * probe[4]) { pout += pr; nout += 1; }
    }
    out[0] = mass[0];
    out[1] = mass[1];
    out[2] = satd > 0 ? satn / satd : 0.0;
    out[3] = fout / ((double)ny * nz);
    for (int d = 0; d < 3; ++d) out[4 + d] = fv[d] / (double)n;
    out[7] = umax;
    out[8] = (nin > 0 ? pin / nin : 0.0) - (nout > 0 ? pout / nout : 0.0);
    out[9] = bad;
}

/* The observables of the oracle's own fields. */
void orc_observables(const orc_state *st, const double probe[5], double out[10])
{
    orc_observables_of(st->p.nx, st->p.ny, st->p.nz, st->type, st->phi, st->rho[0], st->rho[1], st->u, st->sw,
                       st->p.G, probe, out);
}

long orc_steps(const orc_state *st) { return st->steps; }
