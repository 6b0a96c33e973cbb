/*
 * FP64 CPU oracle for the D3Q19 lattice Boltzmann sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The
 * product path (the CUDA library in paper_1007_1388_gb300/) never links,
 * loads or calls it, and the two share no code, tables or headers.
 *
 * It is a plain, slow, direct transcription of the method of Sec. 2.1:
 *   - D3Q19 stencil with weights 1/3, 1/18, 1/36 (Sec. 2.1);
 *   - shifted PDFs  f~_i = f_i - f_i^eq(rho0, 0) = f_i - w_i rho0  (Sec. 2.1),
 *     stored in two full grids (src/dst) and updated by the pull scheme;
 *   - moments rho = rho0 + drho = rho0 + sum f~_i, rho0 u = sum e_i f~_i
 *     (Sec. 2.1, with the +F/2 shift of the forcing reading below);
 *   - incompressible equilibrium of Eq. (2), shifted:
 *       f~_i^eq = w_i [drho + rho0 (3 e_i.u + 4.5 (e_i.u)^2 - 1.5 u.u)];
 *   - single-relaxation-time collision of Eq. (1) (BGK), or the
 *     two-relaxation-time variant (not in the paper, standard Ginzburg TRT);
 *   - half-way bounce-back with wall velocity (Sec. 2.1), read with the
 *     momentum-consistent sign: for an incoming direction i whose source
 *     x - e_i is a wall,  f~_i(x) = f~*_opp(i)(x) + 6 w_i rho0 (e_i . u_w).
 *   - Guo forcing (not in the paper): S_i split into a symmetric part
 *     relaxed with omega+ and an antisymmetric part relaxed with omega-.
 *
 * Where the paper is silent, garbled or inconsistent, the reading taken is
 * stated beside the code that takes it.  No blocking, fusion or reordering is
 * applied; every cell is updated by the same straight loop.  orc_step may
 * spread its z planes over OpenMP threads (orc_set_threads): each cell is
 * still computed by the same code from the same inputs, so the result does
 * not depend on the thread count.
 *
 * Grid convention: interior cells only, index c = (z*ny + y)*nx + x, PDF
 * arrays q-major: f[q*N + c].  Anything outside the interior is either a
 * periodic image (index wrap) or a wall of the face it lies beyond.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 19

enum { ORC_FLUID = 0, ORC_NOSLIP = 1, ORC_MOVING = 2, ORC_PRESSURE = 3 };
enum { ORC_BGK = 0, ORC_TRT = 1 };

/* D3Q19 velocities: 0 rest, 1..6 the axis neighbours, 7..18 the twelve
 * face diagonals.  Opposite pairs are (1,2) (3,4) ... (17,18). */
static const int E[ORC_Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
};

static double weight(int i)
{
    int n2 = E[i][0] * E[i][0] + E[i][1] * E[i][1] + E[i][2] * E[i][2];
    if (n2 == 0) return 1.0 / 3.0;
    if (n2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int opposite(int i)
{
    for (int j = 0; j < ORC_Q; ++j)
        if (E[j][0] == -E[i][0] && E[j][1] == -E[i][1] && E[j][2] == -E[i][2]) return j;
    return -1;
}

typedef struct {
    int n[3];          /* interior cells along x, y, z */
    int periodic[3];   /* 1 = periodic along that axis */
    int face_bc[6];    /* wall kind beyond -x,+x,-y,+y,-z,+z (non-periodic axes) */
    int collision;     /* ORC_BGK or ORC_TRT */
    double tau;        /* relaxation time, omega+ = 1/tau */
    double magic;      /* TRT parameter Lambda = (1/w+ - 1/2)(1/w- - 1/2) */
    double rho0;       /* reference density */
    double force[3];   /* body force density F */
    double wall_u[3];  /* velocity of every ORC_MOVING wall */
    double rho_b;      /* density of every ORC_PRESSURE boundary */
    const double *qw;  /* curved walls: [19][N] wall distances, NULL = half-way everywhere */
} orc_problem;

static int classify(const orc_problem *p, const uint8_t *flags, int x, int y, int z, long *c);

/* Curved resting walls (not in the paper, which leaves further boundary
 * conditions to future work, Sec. 6): the linear interpolated bounce-back of
 * Bouzidi, Firdaouss and Lallemand (2001).  For the pull of direction i at
 * fluid cell x whose source x - e_i is an ORC_NOSLIP node, qw[i][x] = q in
 * (0, 1] places the wall at x - q e_i (q = 1/2: half-way).  The value that
 * returns to x along e_i is interpolated from post-collision populations
 * moving towards the wall (direction ibar = opposite(i)):
 *   q <  1/2: 2q f*_ibar(x) + (1 - 2q) f*_ibar(x + e_i)  (the fluid neighbour
 *             on the far side; if it is not fluid, half-way bounce-back)
 *   q >= 1/2: f*_ibar(x) / (2q) + (1 - 1/(2q)) f*_i(x)
 * Both reduce to f*_ibar(x) at q = 1/2.  The weights sum to one, so the rule
 * holds for the shifted f~ as it stands. */
static double curved_pull(const orc_problem *p, const uint8_t *flags, const double *src, long N, long c,
                          int x, int y, int z, int i)
{
    const int ib = opposite(i);
    const double q = p->qw[i * N + c];
    if (q < 0.5) {
        long s = -1;
        if (classify(p, flags, x + E[i][0], y + E[i][1], z + E[i][2], &s) != ORC_FLUID)
            return src[ib * N + c];
        return 2.0 * q * src[ib * N + c] + (1.0 - 2.0 * q) * src[ib * N + s];
    }
    return src[ib * N + c] / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * src[i * N + c];
}

/* Pressure boundary (not in the paper, which leaves further boundary
 * conditions to future work, Sec. 6): anti-bounce-back with the velocity
 * correction.  A population leaving the fluid cell x towards an ORC_PRESSURE
 * node returns as
 *   f_ibar = -f*_i + 2 w_i [rho_b + rho0 (4.5 (e_i.u_b)^2 - 1.5 u_b^2)],
 * twice the symmetric part of the equilibrium of Eq. (2) at (rho_b, u_b); it
 * holds the density halfway between x and the boundary node at rho_b.  u_b
 * is the velocity of cell x's last collision, read from its stored
 * populations: rho0 u_b = sum_j e_j f~*_j(x) - F/2.  In shifted variables
 * (f~ = f - w rho0): f~_ibar = -f~*_i + 2 w_i [(rho_b - rho0) + rho0 (...)]. */
static void stored_velocity(const orc_problem *p, const double *src, long N, long c, double ub[3])
{
    for (int a = 0; a < 3; ++a) {
        double j = 0.0;
        for (int q = 0; q < ORC_Q; ++q) j += E[q][a] * src[q * N + c];
        ub[a] = (j - 0.5 * p->force[a]) / p->rho0;
    }
}

/* the anti-bounce-back source of direction i for boundary velocity ub, shifted */
static double abb_term(const orc_problem *p, int i, const double ub[3])
{
    double eu = E[i][0] * ub[0] + E[i][1] * ub[1] + E[i][2] * ub[2];
    double usq = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
    return 2.0 * weight(i) * ((p->rho_b - p->rho0) + p->rho0 * (4.5 * eu * eu - 1.5 * usq));
}

/* ------------------------------------------------------------------ */
/* exported lattice and equilibrium, so that tests can pin them        */

void orc_lattice(int *e, double *w, int *opp)
{
    for (int i = 0; i < ORC_Q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = E[i][a];
        w[i] = weight(i);
        opp[i] = opposite(i);
    }
}

/* Shifted incompressible equilibrium, Eq. (2) minus f_i^eq(rho0, 0). */
void orc_equilibrium(double drho, const double u[3], double rho0, double *feq)
{
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < ORC_Q; ++i) {
        double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
        feq[i] = weight(i) * (drho + rho0 * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq));
    }
}

/* ------------------------------------------------------------------ */
/* collision of one cell (pre-collision f~ in, post-collision out)     */

static double omega_minus(const orc_problem *p)
{
    /* Lambda = (tau - 1/2)(1/w- - 1/2)  =>  1/w- = 1/2 + Lambda/(tau - 1/2) */
    return 1.0 / (0.5 + p->magic / (p->tau - 0.5));
}

/* Writes the collided PDFs to fout and the velocity used to u. */
void orc_collide(const orc_problem *p, const double *f, double *fout, double *u_out)
{
    const double *F = p->force;
    double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < ORC_Q; ++i) {
        drho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += E[i][a] * f[i];
    }
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / p->rho0;
    double feq[ORC_Q];
    orc_equilibrium(drho, u, p->rho0, feq);

    double wp = 1.0 / p->tau;
    double wm = (p->collision == ORC_TRT) ? omega_minus(p) : wp;
    double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];

    for (int i = 0; i < ORC_Q; ++i) {
        double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
        double eF = E[i][0] * F[0] + E[i][1] * F[1] + E[i][2] * F[2];
        /* Guo source: w_i [3(e_i - u) + 9 (e_i.u) e_i] . F, split into its
         * even part w_i (9 eu eF - 3 uF) and its odd part 3 w_i eF. */
        double s_even = weight(i) * (9.0 * eu * eF - 3.0 * uF);
        double s_odd = weight(i) * 3.0 * eF;
        if (p->collision == ORC_BGK) {
            fout[i] = f[i] - wp * (f[i] - feq[i]) + (1.0 - 0.5 * wp) * (s_even + s_odd);
        } else {
            int ib = opposite(i);
            double fp = 0.5 * (f[i] + f[ib]), fm = 0.5 * (f[i] - f[ib]);
            double ep = 0.5 * (feq[i] + feq[ib]), em = 0.5 * (feq[i] - feq[ib]);
            fout[i] = f[i] - wp * (fp - ep) - wm * (fm - em)
                      + (1.0 - 0.5 * wp) * s_even + (1.0 - 0.5 * wm) * s_odd;
        }
    }
    if (u_out)
        for (int a = 0; a < 3; ++a) u_out[a] = u[a];
}

/* ------------------------------------------------------------------ */
/* the domain: what lies at a (possibly outside) lattice position      */

static long cell_index(const orc_problem *p, int x, int y, int z)
{
    return ((long)z * p->n[1] + y) * p->n[0] + x;
}

/* Classifies the lattice position (x,y,z).  Periodic axes wrap.  A position
 * beyond exactly one non-periodic face is that face's wall; beyond two or
 * three (an edge or corner of the wall shell) it is a resting wall.  Inside,
 * it is the cell's own flag.  On return *c is the wrapped interior index
 * when the position is inside. */
static int classify(const orc_problem *p, const uint8_t *flags, int x, int y, int z, long *c)
{
    int pos[3] = {x, y, z};
    int outside = 0, face = -1;
    for (int a = 0; a < 3; ++a) {
        int n = p->n[a];
        if (pos[a] < 0 || pos[a] >= n) {
            if (p->periodic[a]) {
                pos[a] = ((pos[a] % n) + n) % n;
            } else {
                ++outside;
                face = 2 * a + (pos[a] >= n ? 1 : 0);
            }
        }
    }
    if (outside >= 2) return ORC_NOSLIP;
    if (outside == 1) return p->face_bc[face];
    *c = cell_index(p, pos[0], pos[1], pos[2]);
    return flags ? flags[*c] : ORC_FLUID;
}

/* ------------------------------------------------------------------ */
/* one time step, pull form (Sec. 2.1): src holds post-collision f~ of
 * step n-1, dst receives post-collision f~ of step n.  Solid cells are
 * not updated and hold 0.  If u_used is given it receives, per cell, the
 * velocity the collision used (3 x N, component-major). */
static int orc_threads = 1;

/* Threads used by orc_step (1 = serial; ignored without OpenMP). */
void orc_set_threads(int n) { orc_threads = n > 0 ? n : 1; }

void orc_step(const orc_problem *p, const uint8_t *flags, const double *src, double *dst,
              double *u_used)
{
    long N = (long)p->n[0] * p->n[1] * p->n[2];
#pragma omp parallel for schedule(static) num_threads(orc_threads) if (orc_threads > 1)
    for (int z = 0; z < p->n[2]; ++z)
        for (int y = 0; y < p->n[1]; ++y)
            for (int x = 0; x < p->n[0]; ++x) {
                long c = cell_index(p, x, y, z);
                if (flags && flags[c] != ORC_FLUID) {
                    for (int i = 0; i < ORC_Q; ++i) dst[i * N + c] = 0.0;
                    if (u_used)
                        for (int a = 0; a < 3; ++a) u_used[a * N + c] = 0.0;
                    continue;
                }
                double f[ORC_Q], fout[ORC_Q], u[3];
                for (int i = 0; i < ORC_Q; ++i) {
                    long s = -1;
                    int kind = classify(p, flags, x - E[i][0], y - E[i][1], z - E[i][2], &s);
                    if (kind == ORC_FLUID) {
                        f[i] = src[i * N + s];
                    } else if (kind == ORC_PRESSURE) {
                        double ub[3];
                        stored_velocity(p, src, N, c, ub);
                        f[i] = -src[opposite(i) * N + c] + abb_term(p, i, ub);
                    } else if (kind == ORC_NOSLIP && p->qw) {
                        f[i] = curved_pull(p, flags, src, N, c, x, y, z, i);
                    } else {
                        double bb = src[opposite(i) * N + c];
                        if (kind == ORC_MOVING) {
                            double eu = E[i][0] * p->wall_u[0] + E[i][1] * p->wall_u[1] +
                                        E[i][2] * p->wall_u[2];
                            bb += 6.0 * weight(i) * p->rho0 * eu;
                        }
                        f[i] = bb;
                    }
                }
                orc_collide(p, f, fout, u);
                for (int i = 0; i < ORC_Q; ++i) dst[i * N + c] = fout[i];
                if (u_used)
                    for (int a = 0; a < 3; ++a) u_used[a * N + c] = u[a];
            }
}

/* n steps starting from f (in place; uses one temporary grid). */
int orc_run(const orc_problem *p, const uint8_t *flags, double *f, int nsteps)
{
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    double *tmp = (double *)malloc(sizeof(double) * ORC_Q * N);
    if (!tmp) return -1;
    double *a = f, *b = tmp;
    for (int s = 0; s < nsteps; ++s) {
        orc_step(p, flags, a, b, NULL);
        double *t = a;
        a = b;
        b = t;
    }
    if (a != f) memcpy(f, a, sizeof(double) * ORC_Q * N);
    free(tmp);
    return 0;
}

/* One pull step evaluated only at the listed interior cells (used to check
 * large GPU runs cell by cell).  out[k*19 + i] = post-collision f~_i. */
void orc_step_cells(const orc_problem *p, const uint8_t *flags, const double *src,
                    const long *cells, long ncells, double *out)
{
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    for (long k = 0; k < ncells; ++k) {
        long c = cells[k];
        int x = (int)(c % p->n[0]);
        int y = (int)((c / p->n[0]) % p->n[1]);
        int z = (int)(c / ((long)p->n[0] * p->n[1]));
        if (flags && flags[c] != ORC_FLUID) {
            for (int i = 0; i < ORC_Q; ++i) out[k * ORC_Q + i] = 0.0;
            continue;
        }
        double f[ORC_Q];
        for (int i = 0; i < ORC_Q; ++i) {
            long s = -1;
            int kind = classify(p, flags, x - E[i][0], y - E[i][1], z - E[i][2], &s);
            if (kind == ORC_FLUID) {
                f[i] = src[i * N + s];
            } else if (kind == ORC_PRESSURE) {
                double ub[3];
                stored_velocity(p, src, N, c, ub);
                f[i] = -src[opposite(i) * N + c] + abb_term(p, i, ub);
            } else if (kind == ORC_NOSLIP && p->qw) {
                f[i] = curved_pull(p, flags, src, N, c, x, y, z, i);
            } else {
                double bb = src[opposite(i) * N + c];
                if (kind == ORC_MOVING) {
                    double eu = E[i][0] * p->wall_u[0] + E[i][1] * p->wall_u[1] +
                                E[i][2] * p->wall_u[2];
                    bb += 6.0 * weight(i) * p->rho0 * eu;
                }
                f[i] = bb;
            }
        }
        orc_collide(p, f, out + k * ORC_Q, NULL);
    }
}

/* ------------------------------------------------------------------ */
/* macroscopic fields of a stored (post-collision) state (Sec. 2.1).
 * The stored f~* of a fluid cell satisfies sum f~* = drho and
 * sum e f~* = rho0 u + F/2, so u = (sum e f~* - F/2)/rho0 is the velocity
 * that cell's last collision used.  Solid cells report rho0 and 0. */
void orc_macroscopic(const orc_problem *p, const uint8_t *flags, const double *f, double *rho,
                     double *u)
{
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    for (long c = 0; c < N; ++c) {
        if (flags && flags[c] != ORC_FLUID) {
            rho[c] = p->rho0;
            for (int a = 0; a < 3; ++a) u[a * N + c] = 0.0;
            continue;
        }
        double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < ORC_Q; ++i) {
            drho += f[i * N + c];
            for (int a = 0; a < 3; ++a) j[a] += E[i][a] * f[i * N + c];
        }
        rho[c] = p->rho0 + drho;
        for (int a = 0; a < 3; ++a) u[a * N + c] = (j[a] - 0.5 * p->force[a]) / p->rho0;
    }
}

/* Sets every fluid cell to f~^eq(rho - rho0, u); solid cells to 0. */
void orc_init_equilibrium(const orc_problem *p, const uint8_t *flags, const double *rho,
                          const double *u, double *f)
{
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    for (long c = 0; c < N; ++c) {
        double feq[ORC_Q];
        if (flags && flags[c] != ORC_FLUID) {
            for (int i = 0; i < ORC_Q; ++i) f[i * N + c] = 0.0;
            continue;
        }
        double uc[3] = {u[c], u[N + c], u[2 * N + c]};
        orc_equilibrium(rho[c] - p->rho0, uc, p->rho0, feq);
        for (int i = 0; i < ORC_Q; ++i) f[i * N + c] = feq[i];
    }
}

/* Total mass sum(rho0 + sum f~) and momentum sum(rho0 u) over fluid cells. */
void orc_invariants(const orc_problem *p, const uint8_t *flags, const double *f, double *mass,
                    double mom[3])
{
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    double m = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (long c = 0; c < N; ++c) {
        if (flags && flags[c] != ORC_FLUID) continue;
        m += p->rho0;
        for (int i = 0; i < ORC_Q; ++i) {
            m += f[i * N + c];
            for (int a = 0; a < 3; ++a) j[a] += E[i][a] * f[i * N + c];
        }
        for (int a = 0; a < 3; ++a) j[a] -= 0.5 * p->force[a];
    }
    *mass = m;
    for (int a = 0; a < 3; ++a) mom[a] = j[a];
}

/* One-step velocity residual ||u_n - u_{n-1}||_2 / ||u_n||_2 over fluid
 * cells, from the stored states of steps n-1 (prev) and n (cur).  Returns 0
 * when both norms vanish. */
double orc_residual(const orc_problem *p, const uint8_t *flags, const double *prev,
                    const double *cur)
{
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    double num = 0.0, den = 0.0;
    for (long c = 0; c < N; ++c) {
        if (flags && flags[c] != ORC_FLUID) continue;
        for (int a = 0; a < 3; ++a) {
            double jc = 0.0, jp = 0.0;
            for (int i = 0; i < ORC_Q; ++i) {
                jc += E[i][a] * cur[i * N + c];
                jp += E[i][a] * prev[i * N + c];
            }
            double uc = (jc - 0.5 * p->force[a]) / p->rho0;
            double up = (jp - 0.5 * p->force[a]) / p->rho0;
            num += (uc - up) * (uc - up);
            den += uc * uc;
        }
    }
    if (den == 0.0) return num == 0.0 ? 0.0 : INFINITY;
    return sqrt(num) / sqrt(den);
}

/* Change per step over an interval of k steps, the convergence criterion
 * taken for sphere-packed channels (not in the paper; the one-step residual
 * above stalls there on an undamped period-2 mode of the scheme):
 *   r = ||u_n - u_{n-k}||_2 / (k ||u_n||_2)   over fluid cells,
 * from the stored states of steps n-k (prev) and n (cur).  It is the one-step
 * residual's quotient of norms, now between states k steps apart, divided
 * by k.  Returns 0 when both norms vanish. */
double orc_interval_residual(const orc_problem *p, const uint8_t *flags, const double *prev,
                             const double *cur, int k)
{
    if (k <= 0) return NAN;
    return orc_residual(p, flags, prev, cur) / (double)k;
}

/* ------------------------------------------------------------------ */
/* An independently written push-form step on UNSHIFTED populations,
 * used only to pin orc_step by brute force on tiny grids.  The stored
 * post-collision state is converted to full populations f = f~ + w rho0;
 * every fluid cell then scatters each population to its downstream
 * neighbour, or reflects it back into itself (with the moving-wall term)
 * when that neighbour is a wall or solid; finally every fluid cell collides
 * what it received, and the result is shifted back.  This computes the same
 * map as the pull step (stream, then collide) by the opposite route, and it
 * shares only the lattice table with it. */

static int push_target(const orc_problem *p, const uint8_t *flags, const int at[3], long *t)
{
    int q[3];
    int beyond = 0, which = -1;
    for (int a = 0; a < 3; ++a) {
        q[a] = at[a];
        if (q[a] < 0 || q[a] >= p->n[a]) {
            if (!p->periodic[a]) {
                beyond++;
                which = 2 * a + (q[a] < 0 ? 0 : 1);
            } else if (q[a] < 0) {
                q[a] += p->n[a];
            } else {
                q[a] -= p->n[a];
            }
        }
    }
    if (beyond > 1) return ORC_NOSLIP;
    if (beyond == 1) return p->face_bc[which];
    *t = (long)q[0] + (long)p->n[0] * ((long)q[1] + (long)p->n[1] * q[2]);
    return flags ? flags[*t] : ORC_FLUID;
}

void orc_push_step(const orc_problem *p, const uint8_t *flags, const double *src, double *dst)
{
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    double *recv = (double *)malloc(sizeof(double) * ORC_Q * N);
    const double wF = 1.0 / p->tau;
    const double wM = (p->collision == ORC_TRT) ? 1.0 / (0.5 + p->magic / (p->tau - 0.5)) : wF;
    for (long c = 0; c < ORC_Q * N; ++c) recv[c] = NAN;
    /* scatter or reflect */
    for (int z = 0; z < p->n[2]; ++z)
        for (int y = 0; y < p->n[1]; ++y)
            for (int x = 0; x < p->n[0]; ++x) {
                long c = (long)x + (long)p->n[0] * ((long)y + (long)p->n[1] * z);
                if (flags && flags[c] != ORC_FLUID) continue;
                for (int i = 0; i < ORC_Q; ++i) {
                    double g = src[i * N + c] + weight(i) * p->rho0;
                    int at[3] = {x + E[i][0], y + E[i][1], z + E[i][2]};
                    long t = -1;
                    int kind = push_target(p, flags, at, &t);
                    if (kind == ORC_FLUID) {
                        recv[i * N + t] = g;
                    } else if (kind == ORC_PRESSURE) {
                        /* anti-bounce-back, unshifted: 2 w [rho_b + rho0 (4.5 (e.u)^2 - 1.5 u^2)] - g,
                         * u the velocity this cell's stored populations carry */
                        double jx = 0.0, jy = 0.0, jz = 0.0;
                        for (int q = 0; q < ORC_Q; ++q) {
                            double gq = src[q * N + c] + weight(q) * p->rho0;
                            jx += E[q][0] * gq;
                            jy += E[q][1] * gq;
                            jz += E[q][2] * gq;
                        }
                        double ux = (jx - 0.5 * p->force[0]) / p->rho0, uy = (jy - 0.5 * p->force[1]) / p->rho0,
                               uz = (jz - 0.5 * p->force[2]) / p->rho0;
                        double eu = E[i][0] * ux + E[i][1] * uy + E[i][2] * uz;
                        double usq = ux * ux + uy * uy + uz * uz;
                        recv[opposite(i) * N + c] =
                            2.0 * weight(i) * (p->rho_b + p->rho0 * (4.5 * eu * eu - 1.5 * usq)) - g;
                    } else if (kind == ORC_NOSLIP && p->qw) {
                        /* the wall sits at x + q e_i; the reflected population
                         * (direction k) mixes g_i of x with g_i of the upstream
                         * neighbour x - e_i (q < 1/2) or with g_k of x (q >= 1/2) */
                        int k = opposite(i);
                        double q = p->qw[k * N + c], r;
                        if (q < 0.5) {
                            int up[3] = {x - E[i][0], y - E[i][1], z - E[i][2]};
                            long u = -1;
                            if (push_target(p, flags, up, &u) == ORC_FLUID)
                                r = 2.0 * q * g + (1.0 - 2.0 * q) * (src[i * N + u] + weight(i) * p->rho0);
                            else
                                r = g;
                        } else {
                            r = g / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * (src[k * N + c] + weight(k) * p->rho0);
                        }
                        recv[k * N + c] = r;
                    } else {
                        int k = opposite(i);
                        double ew = E[k][0] * p->wall_u[0] + E[k][1] * p->wall_u[1] +
                                    E[k][2] * p->wall_u[2];
                        recv[k * N + c] = g + (kind == ORC_MOVING ? 6.0 * weight(k) * p->rho0 * ew : 0.0);
                    }
                }
            }
    /* collide what arrived, in unshifted variables:
     * rho = sum f, rho0 v = sum e f + F/2 */
    for (long c = 0; c < N; ++c) {
        if (flags && flags[c] != ORC_FLUID) {
            for (int i = 0; i < ORC_Q; ++i) dst[i * N + c] = 0.0;
            continue;
        }
        double g[ORC_Q], rho = 0.0, m[3] = {0, 0, 0};
        for (int i = 0; i < ORC_Q; ++i) {
            g[i] = recv[i * N + c];
            rho += g[i];
            m[0] += g[i] * E[i][0];
            m[1] += g[i] * E[i][1];
            m[2] += g[i] * E[i][2];
        }
        double v[3];
        for (int a = 0; a < 3; ++a) v[a] = (m[a] + p->force[a] / 2.0) / p->rho0;
        double vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        double vF = v[0] * p->force[0] + v[1] * p->force[1] + v[2] * p->force[2];
        double geq[ORC_Q];
        for (int i = 0; i < ORC_Q; ++i) {
            double ev = E[i][0] * v[0] + E[i][1] * v[1] + E[i][2] * v[2];
            geq[i] = weight(i) * rho + weight(i) * p->rho0 * (3.0 * ev + 4.5 * ev * ev - 1.5 * vv);
        }
        for (int i = 0; i < ORC_Q; ++i) {
            int k = opposite(i);
            double ev = E[i][0] * v[0] + E[i][1] * v[1] + E[i][2] * v[2];
            double eF = E[i][0] * p->force[0] + E[i][1] * p->force[1] + E[i][2] * p->force[2];
            /* relax the symmetric and antisymmetric halves separately */
            double sym = (g[i] + g[k]) / 2.0 - (geq[i] + geq[k]) / 2.0;
            double asym = (g[i] - g[k]) / 2.0 - (geq[i] - geq[k]) / 2.0;
            double src_sym = (1.0 - wF / 2.0) * weight(i) * (9.0 * ev * eF - 3.0 * vF);
            double src_asym = (1.0 - wM / 2.0) * weight(i) * (3.0 * eF);
            double post = g[i] - wF * sym - wM * asym + src_sym + src_asym;
            dst[i * N + c] = post - weight(i) * p->rho0;
        }
    }
    free(recv);
}
