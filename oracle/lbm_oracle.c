/*
 * FP64 CPU oracle of the progressive-mesh two-component pseudo-potential
 * lattice Boltzmann step (Duchateau et al., "A Progressive Mesh Method for
 * Physical Simulations Using Lattice Boltzmann Method on Single-Node
 * multi-GPU Architectures", arXiv:1510.03560).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or constant with the CUDA library; the two only ever see
 * the same seeded inputs.
 *
 * It is written to be read against the paper, not to be fast: a dense
 * [comp][cell][19] layout, one loop per algorithmic step, every cell
 * treated on its own.  Blocks exist only as an activation mask.
 *
 * What each step follows:
 *   lattice            Sec. 2.1, Fig. 1(b), Eq. 3 (c_s^2 = 1/3)
 *   equilibrium        Eq. 2
 *   streaming          Eq. 1 / Eq. 10 left-hand side (pull form)
 *   macroscopics      Eqs. 4-5, per component (Sec. 2.2, end)
 *   EOS                Eq. 7 (Peng-Robinson)
 *   pseudo-potential   Eq. 6
 *   cohesion           Eq. 8 (beta-mixed)
 *   inter-component    Eq. 9
 *   extra forces       Sec. 2.2 after Eq. 9 (gravity, fluid-solid)
 *   forced collision   Eqs. 10-12 (exact-difference forcing)
 *   criterion          Eq. 13, Sec. 4.2, Fig. 4
 *   block creation     Sec. 4.1-4.3
 *
 * Readings taken where the text is garbled or silent (all are listed with
 * their reasons in the design notes of the repository):
 *   R1  collision sign: standard BGK, f - (f - feq)/tau.
 *   R2  D3Q19 weights 1/3, 1/18 (axes), 1/36 (face diagonals).
 *   R3  Eq. 7 denominator 1 + 2 b rho - b^2 rho^2; theta(T) the standard
 *       Peng-Robinson alpha function; Tc = 0.0778 a / (0.45724 b R).
 *   R4  Eq. 8: F = -beta g psi(x) sum w psi(x+e) e
 *                  - (1-beta)/2 g sum w psi(x+e)^2 e,
 *       psi from Eq. 6 with the same g; the argument of the square root
 *       is clamped at zero.
 *   R5  Eq. 9 uses the other component's effective mass; the second
 *       component is an ideal gas (p = c_s^2 rho, psi = 0), so the
 *       effective mass of both components in Eq. 9 is rho itself.
 *   R6  u_alpha in feq is each component's own velocity (Eq. 5).
 *   R7  gravity F = (rho - rho_ref) g.
 *   R8  adhesion F = -g_ads max(0, rho - rho_amb) sum w s(x+e) e.
 *   R9  reported velocity u + F / (2 rho).
 *   R10 halfway bounce-back at solid cells; a solid neighbour lends the
 *       centre cell's own psi / rho to Eqs. 8-9; cells outside a
 *       non-periodic axis are solid.
 *   R11 criterion fires when ||u(t) - u(t-1)||_2 > S for any component
 *       (compared as squares).
 *   R12 targets: every inactive block, not fully solid, holding a D3Q19
 *       neighbour of a firing cell.
 *   R13 the criterion runs after streaming of step t (u(t) is known) and
 *       before that step's collision; new blocks take part in step t.  The
 *       velocity "before step 0" is the initial velocity field.
 *   R14 a new block starts from the ambient equilibrium w_i rho_amb.
 *   R15 blocks are never removed; fully solid blocks never activate.
 *   R16 "held" cells (inlet / outlet) keep their initial populations.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* ---- lattice: Sec. 2.1, Fig. 1(b) ------------------------------------- */

/* The 19 velocities: rest, the 6 axis neighbours, the 12 face diagonals. */
static const int EV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* Weight from |e|^2 (R2). */
static double weight_of(int i)
{
    int n2 = EV[i][0] * EV[i][0] + EV[i][1] * EV[i][1] + EV[i][2] * EV[i][2];
    if (n2 == 0) return 1.0 / 3.0;
    if (n2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* Index of -e_i. */
static int opposite_of(int i)
{
    for (int k = 0; k < Q; ++k)
        if (EV[k][0] == -EV[i][0] && EV[k][1] == -EV[i][1] && EV[k][2] == -EV[i][2])
            return k;
    return -1;
}

/* The two functions above, tabulated once (filled before any parallel
 * region runs). */
static double W_TAB[Q];
static int OPP_TAB[Q];
static int tables_ready = 0;

static void init_tables(void)
{
    if (tables_ready) return;
    for (int i = 0; i < Q; ++i) {
        W_TAB[i] = weight_of(i);
        OPP_TAB[i] = opposite_of(i);
    }
    tables_ready = 1;
}

static double weight(int i) { return W_TAB[i]; }
static int opposite(int i) { return OPP_TAB[i]; }

static const double CS2 = 1.0 / 3.0; /* Eq. 3 with dx = dt = 1 */

/* ---- parameters -------------------------------------------------------- */

typedef struct {
    int nx, ny, nz;
    int ncomp;              /* 1 or 2 */
    int bx, by, bz;         /* block shape (activation unit) */
    int periodic[3];
    int progressive;        /* 0: static mesh, 1: progressive mesh */
    double tau, beta;
    double pr_a, pr_b, pr_R, pr_omega, T_over_Tc;
    double g_self, g_cross;
    double g_ads[2];
    double grav[3];
    double rho_ref[2];
    double S;
} orc_params;

enum { CELL_FLUID = 0, CELL_SOLID = 1, CELL_HELD = 2 };

typedef struct {
    orc_params p;
    long ncell;
    int nbx, nby, nbz;
    long nblock;
    unsigned char *type;      /* [cell] */
    long *nbr;                /* [cell][Q] index of x + e_i, -1 outside */
    long *blk;                /* [cell] block holding the cell */
    double *f[2];             /* [comp][cell][Q] post-collision populations */
    int cur;                  /* buffer holding the latest post-collision state */
    double *fin;              /* [comp][cell][Q] streamed populations of this step */
    double *rho;              /* [comp][cell] */
    double *u;                /* [comp][cell][3] bare velocity, Eq. 5 */
    double *psi;              /* [cell] Eq. 6, component 0 */
    double *force;            /* [comp][cell][3] */
    double *uprev;            /* [comp][cell][3] u of the previous step */
    unsigned char *active;    /* [block] */
    unsigned char *allsolid;  /* [block] */
    unsigned char *mark;      /* [block] scratch for the criterion */
    double *crit;             /* [block] largest ||du||^2 seen at a cell bordering it */
    double rho_amb[2];
    double psi_amb;
    long t;                   /* completed steps */
    /* Peng-Robinson constants (R3) */
    double Tc, T, kappa, theta;
} orc_sim;

/* ---- equilibrium: Eq. 2 ------------------------------------------------ */

static double feq(int i, double rho, const double u[3])
{
    double eu = EV[i][0] * u[0] + EV[i][1] * u[1] + EV[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return weight(i) * rho *
           (1.0 + eu / CS2 + (eu * eu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* ---- EOS and pseudo-potential: Eqs. 6-7 -------------------------------- */

static void pr_constants(const orc_params *p, double *Tc, double *T, double *kappa,
                         double *theta)
{
    *Tc = 0.0778 * p->pr_a / (0.45724 * p->pr_b * p->pr_R);
    *T = p->T_over_Tc * (*Tc);
    *kappa = 0.37464 + 1.54226 * p->pr_omega - 0.26992 * p->pr_omega * p->pr_omega;
    double s = 1.0 + (*kappa) * (1.0 - sqrt(*T / *Tc));
    *theta = s * s;
}

static double pr_pressure(const orc_params *p, double T, double theta, double rho)
{
    double a = p->pr_a, b = p->pr_b;
    return rho * p->pr_R * T / (1.0 - b * rho) -
           a * theta * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

static double pseudo_potential(const orc_params *p, double T, double theta, double rho)
{
    if (p->g_self == 0.0) return 0.0;
    double arg = 2.0 * (pr_pressure(p, T, theta, rho) - CS2 * rho) / (CS2 * p->g_self);
    if (arg < 0.0) arg = 0.0;
    return sqrt(arg);
}

/* ---- geometry helpers -------------------------------------------------- */

static long cell_index(const orc_sim *s, int x, int y, int z)
{
    return (long)x + (long)s->p.nx * ((long)y + (long)s->p.ny * z);
}

/* Cell at (x,y,z)+d, or -1 if it leaves a non-periodic axis. */
static long neighbour(const orc_sim *s, int x, int y, int z, int dx, int dy, int dz)
{
    int c[3] = {x + dx, y + dy, z + dz};
    int n[3] = {s->p.nx, s->p.ny, s->p.nz};
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= n[a]) {
            if (!s->p.periodic[a]) return -1;
            c[a] = (c[a] + n[a]) % n[a];
        }
    }
    return cell_index(s, c[0], c[1], c[2]);
}

static long block_of_cell_slow(const orc_sim *s, long cell)
{
    int x = (int)(cell % s->p.nx);
    int y = (int)((cell / s->p.nx) % s->p.ny);
    int z = (int)(cell / ((long)s->p.nx * s->p.ny));
    int bxi = x / s->p.bx, byi = y / s->p.by, bzi = z / s->p.bz;
    return (long)bxi + (long)s->nbx * ((long)byi + (long)s->nby * bzi);
}

static long block_of_cell(const orc_sim *s, long cell) { return s->blk[cell]; }

/* Cell x + e_i (tabulated at creation), -1 when it leaves the domain. */
static long step_to(const orc_sim *s, long cell, int i) { return s->nbr[cell * Q + i]; }

static int is_solid(const orc_sim *s, long cell)
{
    return cell < 0 || s->type[cell] == CELL_SOLID;
}

static int cell_active(const orc_sim *s, long cell)
{
    return s->active[block_of_cell(s, cell)];
}

static double *fcell(const orc_sim *s, int buf, int comp, long cell)
{
    return s->f[buf] + ((long)comp * s->ncell + cell) * Q;
}

/* ---- step pieces -------------------------------------------------------- */

/* Pull streaming (Eq. 10 left side) and macroscopics (Eqs. 4-5) for one
 * cell of an active block.  The populations arriving from direction i come
 * from x - e_i: bounce-back if that cell is solid or outside (R10), the
 * ambient equilibrium if it lies in an inactive block (the unmeshed
 * region), the stored post-collision value otherwise.  Held cells keep
 * their own populations. */
static void stream_and_moments(orc_sim *s, long cell, int x, int y, int z)
{
    for (int a = 0; a < s->p.ncomp; ++a) {
        const double *own = fcell(s, s->cur, a, cell);
        double *fi = s->fin + ((long)a * s->ncell + cell) * Q;
        for (int i = 0; i < Q; ++i) {
            if (s->type[cell] == CELL_HELD) {
                fi[i] = own[i];
                continue;
            }
            long src = step_to(s, cell, opposite(i)); /* x - e_i */
            if (is_solid(s, src))
                fi[i] = own[opposite(i)];
            else if (!cell_active(s, src))
                fi[i] = weight(i) * s->rho_amb[a];
            else
                fi[i] = fcell(s, s->cur, a, src)[i];
        }
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            rho += fi[i];
            for (int d = 0; d < 3; ++d) j[d] += fi[i] * EV[i][d];
        }
        s->rho[(long)a * s->ncell + cell] = rho;
        for (int d = 0; d < 3; ++d) s->u[((long)a * s->ncell + cell) * 3 + d] = j[d] / rho;
    }
}

/* Value of a per-cell scalar as seen from the centre cell for the force
 * sums of Eqs. 8-9: the centre's own value behind a solid (R10), the
 * ambient value in an inactive block, the neighbour's value otherwise. */
static double seen(const orc_sim *s, long centre, long nb, const double *field,
                   double ambient)
{
    if (is_solid(s, nb)) return field[centre];
    if (!cell_active(s, nb)) return ambient;
    return field[nb];
}

/* Forces on one fluid cell: Eqs. 8-9, gravity (R7), adhesion (R8). */
static void cell_forces(orc_sim *s, long cell, int x, int y, int z)
{
    const orc_params *p = &s->p;
    long nc = s->ncell;
    double sum_psi[3] = {0, 0, 0}, sum_psi2[3] = {0, 0, 0};
    double sum_rho[2][3] = {{0, 0, 0}, {0, 0, 0}}, sum_solid[3] = {0, 0, 0};
    for (int i = 1; i < Q; ++i) {
        long nb = step_to(s, cell, i);
        double w = weight(i);
        double ps = seen(s, cell, nb, s->psi, s->psi_amb);
        double sol = is_solid(s, nb) ? 1.0 : 0.0;
        for (int d = 0; d < 3; ++d) {
            sum_psi[d] += w * ps * EV[i][d];
            sum_psi2[d] += w * ps * ps * EV[i][d];
            sum_solid[d] += w * sol * EV[i][d];
        }
        for (int a = 0; a < p->ncomp; ++a) {
            double r = seen(s, cell, nb, s->rho + (long)a * nc, s->rho_amb[a]);
            for (int d = 0; d < 3; ++d) sum_rho[a][d] += w * r * EV[i][d];
        }
    }
    for (int a = 0; a < p->ncomp; ++a) {
        double rho = s->rho[(long)a * nc + cell];
        double *F = s->force + ((long)a * nc + cell) * 3;
        for (int d = 0; d < 3; ++d) F[d] = 0.0;
        if (a == 0 && p->g_self != 0.0) {
            double psi = s->psi[cell];
            for (int d = 0; d < 3; ++d)
                F[d] += -p->beta * p->g_self * psi * sum_psi[d] -
                        (1.0 - p->beta) / 2.0 * p->g_self * sum_psi2[d];
        }
        if (p->ncomp == 2) {
            int o = 1 - a;
            for (int d = 0; d < 3; ++d) F[d] += -p->g_cross * rho * sum_rho[o][d];
        }
        double excess = rho - s->rho_amb[a];
        if (excess < 0.0) excess = 0.0;
        for (int d = 0; d < 3; ++d) F[d] += -p->g_ads[a] * excess * sum_solid[d];
        for (int d = 0; d < 3; ++d) F[d] += (rho - p->rho_ref[a]) * p->grav[d];
    }
}

/* Forced BGK collision, Eqs. 10-12 with the R1 sign. */
static void collide_cell(double tau, double rho, const double u[3], const double F[3],
                         const double *fin, double *fout)
{
    double du[3], u2[3];
    for (int d = 0; d < 3; ++d) {
        du[d] = F[d] / rho;       /* Eq. 12, dt = 1 */
        u2[d] = u[d] + du[d];
    }
    for (int i = 0; i < Q; ++i) {
        double e0 = feq(i, rho, u);
        double dfi = feq(i, rho, u2) - e0; /* Eq. 11 */
        fout[i] = fin[i] - (fin[i] - e0) / tau + dfi;
    }
}

static void block_coords(const orc_sim *s, long b, int *bxi, int *byi, int *bzi)
{
    *bxi = (int)(b % s->nbx);
    *byi = (int)((b / s->nbx) % s->nby);
    *bzi = (int)(b / ((long)s->nbx * s->nby));
}

/* Loop helper: run fn on every cell of every block whose flag is set. */
typedef void (*cell_fn)(orc_sim *, long, int, int, int);

static void for_cells_of_blocks(orc_sim *s, const unsigned char *flag, cell_fn fn)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (long b = 0; b < s->nblock; ++b) {
        if (!flag[b]) continue;
        int bxi, byi, bzi;
        block_coords(s, b, &bxi, &byi, &bzi);
        for (int z = bzi * s->p.bz; z < (bzi + 1) * s->p.bz; ++z)
            for (int y = byi * s->p.by; y < (byi + 1) * s->p.by; ++y)
                for (int x = bxi * s->p.bx; x < (bxi + 1) * s->p.bx; ++x) {
                    long c = cell_index(s, x, y, z);
                    fn(s, c, x, y, z);
                }
    }
}

static void macro_cell(orc_sim *s, long c, int x, int y, int z)
{
    if (s->type[c] == CELL_SOLID) return;
    stream_and_moments(s, c, x, y, z);
}

static void psi_cell(orc_sim *s, long c, int x, int y, int z)
{
    (void)x; (void)y; (void)z;
    if (s->type[c] == CELL_SOLID) return;
    s->psi[c] = pseudo_potential(&s->p, s->T, s->theta, s->rho[c]);
}

static void force_cell(orc_sim *s, long c, int x, int y, int z)
{
    if (s->type[c] != CELL_FLUID) return;
    cell_forces(s, c, x, y, z);
}

static void collide_and_store(orc_sim *s, long c, int x, int y, int z)
{
    (void)x; (void)y; (void)z;
    if (s->type[c] == CELL_SOLID) return;
    int nxt = 1 - s->cur;
    for (int a = 0; a < s->p.ncomp; ++a) {
        double *out = fcell(s, nxt, a, c);
        const double *fi = s->fin + ((long)a * s->ncell + c) * Q;
        if (s->type[c] == CELL_HELD) {
            for (int i = 0; i < Q; ++i) out[i] = fi[i];
        } else {
            collide_cell(s->p.tau, s->rho[(long)a * s->ncell + c],
                         s->u + ((long)a * s->ncell + c) * 3,
                         s->force + ((long)a * s->ncell + c) * 3, fi, out);
        }
        for (int d = 0; d < 3; ++d)
            s->uprev[((long)a * s->ncell + c) * 3 + d] = s->u[((long)a * s->ncell + c) * 3 + d];
    }
}

/* Reset a block to the ambient equilibrium at rest (R14) in the buffer that
 * holds the previous post-collision state. */
static void ambient_cell(orc_sim *s, long c, int x, int y, int z)
{
    (void)x; (void)y; (void)z;
    for (int a = 0; a < s->p.ncomp; ++a) {
        double *f = fcell(s, s->cur, a, c);
        for (int i = 0; i < Q; ++i) f[i] = weight(i) * s->rho_amb[a];
    }
}

/* Eq. 13 on the cells that border the unmeshed region; marks target blocks
 * (R11, R12).  Evaluated on the blocks that were active when the step
 * started. */
static void criterion(orc_sim *s)
{
    long nc = s->ncell;
    double S2 = s->p.S * s->p.S;
    memset(s->mark, 0, (size_t)s->nblock);
    for (long b = 0; b < s->nblock; ++b) s->crit[b] = -1.0;
    for (long b = 0; b < s->nblock; ++b) {
        if (!s->active[b]) continue;
        int bxi, byi, bzi;
        block_coords(s, b, &bxi, &byi, &bzi);
        for (int z = bzi * s->p.bz; z < (bzi + 1) * s->p.bz; ++z)
            for (int y = byi * s->p.by; y < (byi + 1) * s->p.by; ++y)
                for (int x = bxi * s->p.bx; x < (bxi + 1) * s->p.bx; ++x) {
                    long c = cell_index(s, x, y, z);
                    if (s->type[c] != CELL_FLUID) continue;
                    double c2 = 0.0;
                    for (int a = 0; a < s->p.ncomp; ++a) {
                        double n2 = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            double du = s->u[((long)a * nc + c) * 3 + d] -
                                        s->uprev[((long)a * nc + c) * 3 + d];
                            n2 += du * du;
                        }
                        if (n2 > c2) c2 = n2;
                    }
                    for (int i = 1; i < Q; ++i) {
                        long nb = step_to(s, c, i);
                        if (nb < 0) continue;
                        long tb = block_of_cell(s, nb);
                        if (s->active[tb] || s->allsolid[tb]) continue;
                        if (c2 > s->crit[tb]) s->crit[tb] = c2;
                        if (c2 > S2) s->mark[tb] = 1;
                    }
                }
    }
}

/* ---- public API ---------------------------------------------------------- */

void orc_lattice(int *e, double *w, int *opp)
{
    init_tables();
    for (int i = 0; i < Q; ++i) {
        for (int d = 0; d < 3; ++d) e[i * 3 + d] = EV[i][d];
        w[i] = weight(i);
        if (opp) opp[i] = opposite(i);
    }
}

void orc_feq(double rho, const double *u, double *out)
{
    init_tables();
    for (int i = 0; i < Q; ++i) out[i] = feq(i, rho, u);
}

void orc_collide(double tau, double rho, const double *u, const double *F, const double *fin,
                 double *fout)
{
    init_tables();
    collide_cell(tau, rho, u, F, fin, fout);
}

void orc_eos_constants(const orc_params *p, double *out4)
{
    pr_constants(p, &out4[0], &out4[1], &out4[2], &out4[3]);
}

/* Pressure of Eq. 7 at temperature T_over_Tc * Tc. */
double orc_pressure(const orc_params *p, double rho)
{
    double Tc, T, k, th;
    pr_constants(p, &Tc, &T, &k, &th);
    return pr_pressure(p, T, th, rho);
}

double orc_psi(const orc_params *p, double rho)
{
    double Tc, T, k, th;
    pr_constants(p, &Tc, &T, &k, &th);
    return pseudo_potential(p, T, th, rho);
}

orc_sim *orc_create(const orc_params *p, const unsigned char *type, const double *rho_init,
                    const double *u_init, const double *rho_amb)
{
    init_tables();
    if (p->ncomp < 1 || p->ncomp > 2) return NULL;
    if (p->nx % p->bx || p->ny % p->by || p->nz % p->bz) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->p = *p;
    s->ncell = (long)p->nx * p->ny * p->nz;
    s->nbx = p->nx / p->bx;
    s->nby = p->ny / p->by;
    s->nbz = p->nz / p->bz;
    s->nblock = (long)s->nbx * s->nby * s->nbz;
    long nc = s->ncell, na = p->ncomp;
    s->type = (unsigned char *)malloc((size_t)nc);
    memcpy(s->type, type, (size_t)nc);
    s->nbr = (long *)malloc(sizeof(long) * (size_t)(nc * Q));
    s->blk = (long *)malloc(sizeof(long) * (size_t)nc);
    for (int z = 0; z < p->nz; ++z)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                long c = cell_index(s, x, y, z);
                s->blk[c] = block_of_cell_slow(s, c);
                for (int i = 0; i < Q; ++i)
                    s->nbr[c * Q + i] = neighbour(s, x, y, z, EV[i][0], EV[i][1], EV[i][2]);
            }
    for (int b = 0; b < 2; ++b) s->f[b] = (double *)calloc((size_t)(na * nc * Q), sizeof(double));
    s->fin = (double *)calloc((size_t)(na * nc * Q), sizeof(double));
    s->rho = (double *)calloc((size_t)(na * nc), sizeof(double));
    s->u = (double *)calloc((size_t)(na * nc * 3), sizeof(double));
    s->psi = (double *)calloc((size_t)nc, sizeof(double));
    s->force = (double *)calloc((size_t)(na * nc * 3), sizeof(double));
    s->uprev = (double *)calloc((size_t)(na * nc * 3), sizeof(double));
    s->active = (unsigned char *)calloc((size_t)s->nblock, 1);
    s->allsolid = (unsigned char *)calloc((size_t)s->nblock, 1);
    s->mark = (unsigned char *)calloc((size_t)s->nblock, 1);
    s->crit = (double *)calloc((size_t)s->nblock, sizeof(double));
    for (int a = 0; a < 2; ++a) s->rho_amb[a] = a < p->ncomp ? rho_amb[a] : 0.0;
    pr_constants(p, &s->Tc, &s->T, &s->kappa, &s->theta);
    s->psi_amb = pseudo_potential(p, s->T, s->theta, s->rho_amb[0]);
    s->cur = 0;
    s->t = 0;

    for (long b = 0; b < s->nblock; ++b) s->allsolid[b] = 1;
    for (long c = 0; c < nc; ++c) {
        long b = block_of_cell(s, c);
        if (type[c] != CELL_SOLID) s->allsolid[b] = 0;
        if (type[c] == CELL_SOLID) continue;
        int differs = 0;
        for (int a = 0; a < na; ++a) {
            double u[3] = {0, 0, 0};
            if (u_init)
                for (int d = 0; d < 3; ++d) u[d] = u_init[((long)a * 3 + d) * nc + c];
            double r = rho_init[(long)a * nc + c];
            if (r != s->rho_amb[a] || u[0] != 0.0 || u[1] != 0.0 || u[2] != 0.0) differs = 1;
            for (int d = 0; d < 3; ++d) s->uprev[((long)a * nc + c) * 3 + d] = u[d];
            for (int i = 0; i < Q; ++i) {
                double v = feq(i, r, u);
                fcell(s, 0, a, c)[i] = v;
                fcell(s, 1, a, c)[i] = v;
            }
        }
        if (differs) s->active[b] = 1;
    }
    for (long b = 0; b < s->nblock; ++b) {
        if (s->allsolid[b]) s->active[b] = 0;
        else if (!p->progressive) s->active[b] = 1;
    }
    return s;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->type);
    free(s->nbr);
    free(s->blk);
    free(s->f[0]);
    free(s->f[1]);
    free(s->fin);
    free(s->rho);
    free(s->u);
    free(s->psi);
    free(s->force);
    free(s->uprev);
    free(s->active);
    free(s->allsolid);
    free(s->mark);
    free(s->crit);
    free(s);
}

/* One time step, in the order reconstructed from Sec. 4.3 (R13). */
static void one_step(orc_sim *s)
{
    /* 1. streaming and macroscopics on the meshed blocks */
    for_cells_of_blocks(s, s->active, macro_cell);

    /* 2. progressive mesh: criterion, new blocks, their streaming */
    if (s->p.progressive) {
        criterion(s);
        long added = 0;
        for (long b = 0; b < s->nblock; ++b) added += s->mark[b];
        if (added) {
            for_cells_of_blocks(s, s->mark, ambient_cell);
            for (long b = 0; b < s->nblock; ++b)
                if (s->mark[b]) s->active[b] = 1;
            for_cells_of_blocks(s, s->mark, macro_cell);
        }
    }

    /* 3. pseudo-potential, 4. forces, 5. collision (+ stored velocity) */
    for_cells_of_blocks(s, s->active, psi_cell);
    for_cells_of_blocks(s, s->active, force_cell);
    for_cells_of_blocks(s, s->active, collide_and_store);

    /* 6. the new post-collision state becomes current */
    s->cur = 1 - s->cur;
    s->t += 1;
}

void orc_step(orc_sim *s, int n)
{
    for (int k = 0; k < n; ++k) one_step(s);
}

/* Macroscopic fields of the current state: what the next step would see
 * after streaming.  Fluid cells report the physical velocity u + F/(2 rho)
 * (R9); held cells their own moments; solid cells zero; cells of inactive
 * blocks the ambient state. */
void orc_macro(orc_sim *s, int comp, double *rho, double *ux, double *uy, double *uz)
{
    for_cells_of_blocks(s, s->active, macro_cell);
    for_cells_of_blocks(s, s->active, psi_cell);
    for_cells_of_blocks(s, s->active, force_cell);
    long nc = s->ncell;
    for (long c = 0; c < nc; ++c) {
        double r = 0.0, v[3] = {0, 0, 0};
        if (s->type[c] == CELL_SOLID) {
        } else if (!cell_active(s, c)) {
            r = s->rho_amb[comp];
        } else {
            r = s->rho[(long)comp * nc + c];
            for (int d = 0; d < 3; ++d) {
                v[d] = s->u[((long)comp * nc + c) * 3 + d];
                if (s->type[c] == CELL_FLUID)
                    v[d] += s->force[((long)comp * nc + c) * 3 + d] / (2.0 * r);
            }
        }
        rho[c] = r;
        ux[c] = v[0];
        uy[c] = v[1];
        uz[c] = v[2];
    }
}

/* Forces of the current state (same evaluation as orc_macro), [cell][3]. */
void orc_forces(orc_sim *s, int comp, double *F)
{
    for_cells_of_blocks(s, s->active, macro_cell);
    for_cells_of_blocks(s, s->active, psi_cell);
    for_cells_of_blocks(s, s->active, force_cell);
    long nc = s->ncell;
    for (long c = 0; c < nc; ++c)
        for (int d = 0; d < 3; ++d)
            F[c * 3 + d] = (s->type[c] == CELL_FLUID && cell_active(s, c))
                               ? s->force[((long)comp * nc + c) * 3 + d]
                               : 0.0;
}

long orc_active_blocks(const orc_sim *s, int *ids)
{
    long n = 0;
    for (long b = 0; b < s->nblock; ++b)
        if (s->active[b]) {
            if (ids) ids[n] = (int)b;
            ++n;
        }
    return n;
}

/* Per-component mass: sum of the populations of every non-solid cell, the
 * unmeshed cells counted at the ambient equilibrium.  The per-cell sums are
 * accumulated with compensated (Kahan) summation so that the total is
 * accurate to a few ulps whatever the grid size. */
void orc_mass(const orc_sim *s, double *mass)
{
    for (int a = 0; a < s->p.ncomp; ++a) {
        double m = 0.0, comp = 0.0;
        for (long c = 0; c < s->ncell; ++c) {
            if (s->type[c] == CELL_SOLID) continue;
            double cellsum = 0.0;
            if (cell_active(s, c)) {
                const double *f = fcell(s, s->cur, a, c);
                for (int i = 0; i < Q; ++i) cellsum += f[i];
            } else {
                for (int i = 0; i < Q; ++i) cellsum += weight(i) * s->rho_amb[a];
            }
            double y = cellsum - comp;
            double t = m + y;
            comp = (t - m) - y;
            m = t;
        }
        mass[a] = m;
    }
}

/* Largest squared velocity change seen by the last criterion pass at a
 * cell bordering each inactive block (-1 where none). */
void orc_crit(const orc_sim *s, double *out)
{
    for (long b = 0; b < s->nblock; ++b) out[b] = s->crit[b];
}

/* Raw access to the current post-collision populations, [cell][19]. */
void orc_get_f(const orc_sim *s, int comp, double *out)
{
    memcpy(out, fcell(s, s->cur, comp, 0), sizeof(double) * (size_t)(s->ncell * Q));
}

void orc_set_f(orc_sim *s, int comp, const double *in)
{
    memcpy(fcell(s, s->cur, comp, 0), in, sizeof(double) * (size_t)(s->ncell * Q));
}

void orc_set_active(orc_sim *s, const unsigned char *act)
{
    for (long b = 0; b < s->nblock; ++b) s->active[b] = act[b] && !s->allsolid[b];
}

void orc_set_time(orc_sim *s, long t) { s->t = t; }

long orc_time(const orc_sim *s) { return s->t; }
