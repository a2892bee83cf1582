/*
 * pic_oracle.c -- plain FP64 CPU oracle for one timestep of the fully
 * relativistic electromagnetic particle-in-cell (EM-PIC) method of
 * Fonseca et al., "Exploiting multi-scale parallelism for large scale
 * numerical modelling of laser wakefield accelerators" (Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * What one step computes (Sec. 2, Sec. 5.2 steps i-v):
 *   1. B-spline weights of order p at the particle (Sec. 5.2 step i),
 *   2. gather of E and B, each component at its own Yee location (Sec. 5.1,
 *      Sec. 5.2 step ii),
 *   3. relativistic push, read as the Boris scheme (Sec. 2, Sec. 5.2 step iii),
 *   4. position update,
 *   5. charge-conserving current deposit, read as Esirkepov's density
 *      decomposition on the full straight segment (Sec. 5.2, the
 *      charge-conserving method it cites),
 *   6. Yee FDTD update of E and B (Sec. 2; Sec. 3: a local field solver).
 * The deposit runs the paper's shared-memory algorithm literally: n_T threads
 * each own a private copy of the current grid, followed by a threaded
 * reduction of the copies (Sec. 3.1).
 *
 * Conventions (normalised units, c = 1):
 *   positions are in cell units: node i of axis a sits at x_a = i; the
 *   physical coordinate is x_a * d[a];
 *   arrays are component-major, x fastest: idx = i + n0*(j + n1*k);
 *   Yee locations (cell units): E0 (1/2,0,0) E1 (0,1/2,0) E2 (0,0,1/2)
 *                               B0 (0,1/2,1/2) B1 (1/2,0,1/2) B2 (1/2,1/2,0);
 *   in 2D the third axis is absent (no z offset, no z derivative);
 *   Maxwell: dE/dt = curl B - J, dB/dt = -curl E, div E = rho;
 *   particle weight w is a density (n / ppc): rho(node) = sum q w S.
 * Parity status of every exported function is listed in oracle/__init__.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t dim;          /* 2 or 3 */
    int32_t n[3];         /* cells per axis; n[2] == 1 in 2D */
    double d[3];          /* cell size per axis */
    double dt;
    int32_t order;        /* B-spline order, 1..4 */
    int32_t open_last;    /* 1: last axis has Mur field and absorbing particle boundaries */
    double q, m;          /* species charge and mass */
    /* laser antenna (one-way plane source on the last axis) */
    int32_t laser_on;
    int32_t laser_plane;  /* node index along the last axis */
    int32_t laser_pol;    /* polarisation axis */
    int32_t pad0;
    double a0, omega0, waist, fwhm, t_peak;
    /* moving window along the last axis */
    int32_t window_on;
    int32_t ppc[3];       /* particles per cell per axis for injection */
    double window_v, window_t0;
    double density;       /* injected density when n_knots == 0 */
    int32_t n_knots;
    int32_t pad1;
    const double *knots;  /* piecewise-linear density over lab z in [z0, z1] */
    double z0, z1;
    /* evolving state */
    double time;
    int64_t step;
    int64_t shifts;
    int32_t nthreads;
    int32_t pad2;
    /* deposit of each move: 0 = one charge-conserving deposit of the whole */
    /* straight move; 1 = virtual trajectories (or_deposit_current_split)    */
    int32_t split;
    int32_t pad3;
} or_sim;

/* ------------------------------------------------------------------ */
/* B-spline shape functions (Sec. 5.2 step i; Table 3 varies the order  */
/* from 1 to 4).  S_p is the p-fold convolution of the unit box.        */
/* ------------------------------------------------------------------ */
double or_bspline(int p, double t)
{
    double a = fabs(t);
    switch (p) {
    case 1:
        return a < 1.0 ? 1.0 - a : 0.0;
    case 2:
        if (a <= 0.5) return 0.75 - a * a;
        if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
        return 0.0;
    case 3:
        if (a <= 1.0) return (4.0 - 6.0 * a * a + 3.0 * a * a * a) / 6.0;
        if (a < 2.0) return (2.0 - a) * (2.0 - a) * (2.0 - a) / 6.0;
        return 0.0;
    case 4:
        if (a <= 0.5) return (115.0 - 120.0 * a * a + 48.0 * a * a * a * a) / 192.0;
        if (a <= 1.5)
            return (55.0 + 20.0 * a - 120.0 * a * a + 80.0 * a * a * a - 16.0 * a * a * a * a) / 96.0;
        if (a < 2.5) {
            double b = 2.5 - a;
            return b * b * b * b / 24.0;
        }
        return 0.0;
    default:
        return 0.0;
    }
}

static inline int64_t wrap(int64_t i, int64_t n)
{
    int64_t r = i % n;
    return r < 0 ? r + n : r;
}

static inline int64_t cell_index(const or_sim *s, int64_t i, int64_t j, int64_t k)
{
    int64_t n0 = s->n[0], n1 = s->n[1], n2 = s->n[2];
    return wrap(i, n0) + n0 * (wrap(j, n1) + n1 * wrap(k, n2));
}

static inline int64_t ncells(const or_sim *s)
{
    return (int64_t)s->n[0] * s->n[1] * s->n[2];
}

/* Yee location of field component c (0..2 E, 3..5 B) along axis a, in cells. */
static double yee_offset(int c, int a)
{
    static const double off[6][3] = {
        {0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5},
        {0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};
    return off[c][a];
}

/* ------------------------------------------------------------------ */
/* Gather (Sec. 5.1, Sec. 5.2 step ii): every component is interpolated  */
/* from its own staggered nodes with the same order-p weights.          */
/* Written as the plain sum over every node whose weight can be nonzero. */
/* ------------------------------------------------------------------ */
void or_gather(const or_sim *s, const double *E, const double *B, const double *x, double *out)
{
    const int64_t nc = ncells(s);
    const int p = s->order;
    const double half = 0.5 * (p + 1);
    for (int c = 0; c < 6; ++c) {
        const double *F = c < 3 ? E + (int64_t)c * nc : B + (int64_t)(c - 3) * nc;
        int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        for (int a = 0; a < s->dim; ++a) {
            double xa = x[a] - yee_offset(c, a);
            lo[a] = (int64_t)floor(xa - half);
            hi[a] = (int64_t)floor(xa + half) + 1;
        }
        double sum = 0.0;
        for (int64_t k = lo[2]; k <= hi[2]; ++k) {
            double wz = s->dim == 3 ? or_bspline(p, x[2] - (k + yee_offset(c, 2))) : 1.0;
            if (wz == 0.0) continue;
            for (int64_t j = lo[1]; j <= hi[1]; ++j) {
                double wy = or_bspline(p, x[1] - (j + yee_offset(c, 1)));
                if (wy == 0.0) continue;
                for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                    double wx = or_bspline(p, x[0] - (i + yee_offset(c, 0)));
                    if (wx == 0.0) continue;
                    sum += wx * wy * wz * F[cell_index(s, i, j, k)];
                }
            }
        }
        out[c] = sum;
    }
}

/* ------------------------------------------------------------------ */
/* Relativistic push (Sec. 2: the relativistic equations of motion;     */
/* Sec. 5.2 step iii), read as the Boris scheme: half electric kick,     */
/* magnetic rotation with tan(theta/2) = |t|, half electric kick.        */
/* u = gamma*beta; eb = (E0,E1,E2,B0,B1,B2) at the particle.            */
/* ------------------------------------------------------------------ */
void or_boris(double qm, double dt, const double *eb, double *u)
{
    double h = 0.5 * qm * dt;
    double um[3], up[3], t[3], sv[3], uprime[3];
    for (int a = 0; a < 3; ++a) um[a] = u[a] + h * eb[a];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int a = 0; a < 3; ++a) t[a] = h * eb[3 + a] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; ++a) sv[a] = 2.0 * t[a] / (1.0 + t2);
    uprime[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    uprime[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    uprime[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    up[0] = um[0] + (uprime[1] * sv[2] - uprime[2] * sv[1]);
    up[1] = um[1] + (uprime[2] * sv[0] - uprime[0] * sv[2]);
    up[2] = um[2] + (uprime[0] * sv[1] - uprime[1] * sv[0]);
    for (int a = 0; a < 3; ++a) u[a] = up[a] + h * eb[a];
}

/* ------------------------------------------------------------------ */
/* Charge density (Sec. 2): rho(node) += q w S(x - node).  Used for     */
/* diagnostics and to pin the deposit through discrete continuity.      */
/* ------------------------------------------------------------------ */
void or_deposit_rho(const or_sim *s, double qw, const double *x, double *rho)
{
    const int p = s->order;
    const double half = 0.5 * (p + 1);
    int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int a = 0; a < s->dim; ++a) {
        lo[a] = (int64_t)floor(x[a] - half);
        hi[a] = (int64_t)floor(x[a] + half) + 1;
    }
    for (int64_t k = lo[2]; k <= hi[2]; ++k) {
        double wz = s->dim == 3 ? or_bspline(p, x[2] - k) : 1.0;
        for (int64_t j = lo[1]; j <= hi[1]; ++j) {
            double wy = or_bspline(p, x[1] - j);
            for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                double wx = or_bspline(p, x[0] - i);
                double w = wx * wy * wz;
                if (w != 0.0) rho[cell_index(s, i, j, k)] += qw * w;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Charge-conserving current deposit (Sec. 5.2, the charge-conserving    */
/* method it cites: Esirkepov's density decomposition).                 */
/*   S0 = S(x_old - node), S1 = S(x_new - node), DS = S1 - S0 per axis.  */
/*   3D: W_x = DSx (S0y S0z + DSy S0z / 2 + S0y DSz / 2 + DSy DSz / 3),  */
/*       cyclically for W_y, W_z;                                        */
/*   2D: W_x = DSx (S0y + DSy / 2), W_y = DSy (S0x + DSx / 2),           */
/*       J_z = q w v_z (S0x S0y + DSx S0y / 2 + S0x DSy / 2 + DSx DSy / 3).*/
/*   J_a(node + 1/2 along a) = J_a(node - 1/2) - q w (d_a / dt) W_a(node),*/
/*   starting from zero below the window.                                */
/* x_old / x_new are unwrapped (the move is less than one cell); indices */
/* are wrapped only when writing.  J is component-major.                 */
/* ------------------------------------------------------------------ */
#define OR_WMAX 12
void or_deposit_current(const or_sim *s, double qw, const double *x_old, const double *x_new,
                        double vz, double *J)
{
    const int p = s->order;
    const int dim = s->dim;
    const int64_t nc = ncells(s);
    const double half = 0.5 * (p + 1);
    int64_t lo[3] = {0, 0, 0};
    int len[3] = {1, 1, 1};
    double S0[3][OR_WMAX], DS[3][OR_WMAX];
    for (int a = 0; a < 3; ++a)
        for (int q = 0; q < OR_WMAX; ++q) {
            S0[a][q] = a < dim ? 0.0 : 1.0;
            DS[a][q] = 0.0;
        }
    for (int a = 0; a < dim; ++a) {
        double mn = x_old[a] < x_new[a] ? x_old[a] : x_new[a];
        double mx = x_old[a] < x_new[a] ? x_new[a] : x_old[a];
        lo[a] = (int64_t)floor(mn - half);
        int64_t hi = (int64_t)floor(mx + half) + 1;
        len[a] = (int)(hi - lo[a] + 1);
        if (len[a] > OR_WMAX) len[a] = OR_WMAX; /* cannot happen for |move| < 1 cell, p <= 4 */
        for (int q = 0; q < len[a]; ++q) {
            double node = (double)(lo[a] + q);
            double s0 = or_bspline(p, x_old[a] - node);
            double s1 = or_bspline(p, x_new[a] - node);
            S0[a][q] = s0;
            DS[a][q] = s1 - s0;
        }
    }
    double *Jx = J, *Jy = J + nc, *Jz = J + 2 * nc;
    if (dim == 3) {
        /* W_a over the window, then prefix sums along a. */
        for (int comp = 0; comp < 3; ++comp) {
            int a = comp, b = (comp + 1) % 3, c = (comp + 2) % 3;
            double coef = -qw * s->d[a] / s->dt;
            double *Ja = comp == 0 ? Jx : (comp == 1 ? Jy : Jz);
            for (int qb = 0; qb < len[b]; ++qb)
                for (int qc = 0; qc < len[c]; ++qc) {
                    double fac = S0[b][qb] * S0[c][qc] + 0.5 * DS[b][qb] * S0[c][qc] +
                                 0.5 * S0[b][qb] * DS[c][qc] + DS[b][qb] * DS[c][qc] / 3.0;
                    double run = 0.0;
                    for (int qa = 0; qa < len[a]; ++qa) {
                        run += coef * DS[a][qa] * fac;
                        int64_t idx3[3];
                        idx3[a] = lo[a] + qa;
                        idx3[b] = lo[b] + qb;
                        idx3[c] = lo[c] + qc;
                        if (run != 0.0) Ja[cell_index(s, idx3[0], idx3[1], idx3[2])] += run;
                    }
                }
        }
    } else {
        double cx = -qw * s->d[0] / s->dt, cy = -qw * s->d[1] / s->dt;
        for (int qy = 0; qy < len[1]; ++qy) {
            double run = 0.0;
            for (int qx = 0; qx < len[0]; ++qx) {
                run += cx * DS[0][qx] * (S0[1][qy] + 0.5 * DS[1][qy]);
                if (run != 0.0) Jx[cell_index(s, lo[0] + qx, lo[1] + qy, 0)] += run;
            }
        }
        for (int qx = 0; qx < len[0]; ++qx) {
            double run = 0.0;
            for (int qy = 0; qy < len[1]; ++qy) {
                run += cy * DS[1][qy] * (S0[0][qx] + 0.5 * DS[0][qx]);
                if (run != 0.0) Jy[cell_index(s, lo[0] + qx, lo[1] + qy, 0)] += run;
            }
        }
        for (int qy = 0; qy < len[1]; ++qy)
            for (int qx = 0; qx < len[0]; ++qx) {
                double f = S0[0][qx] * S0[1][qy] + 0.5 * DS[0][qx] * S0[1][qy] +
                           0.5 * S0[0][qx] * DS[1][qy] + DS[0][qx] * DS[1][qy] / 3.0;
                double v = qw * vz * f;
                if (v != 0.0) Jz[cell_index(s, lo[0] + qx, lo[1] + qy, 0)] += v;
            }
    }
}

/* ------------------------------------------------------------------ */
/* Virtual trajectories (Sec. 5.2 step iv: up to four per particle in    */
/* 3D).  The straight move is cut at every point where it crosses a      */
/* boundary between the grid points nearest the particle -- the          */
/* half-integer positions for even orders, the cell faces for odd ones   */
/* -- along any axis, and each piece is deposited by or_deposit_current  */
/* as a move of its own, its out-of-plane current (2D) weighted by the   */
/* piece's share of the time step.  Each piece conserves charge, so the  */
/* sum does; for linear shapes every piece stays in one cell and its     */
/* current is Villasenor and Buneman's.                                  */
/* ------------------------------------------------------------------ */
void or_deposit_current_split(const or_sim *s, double qw, const double *x_old, const double *x_new,
                              double vz, double *J)
{
    const int dim = s->dim;
    const double off = (s->order % 2 == 0) ? 0.5 : 0.0; /* boundaries at j + off */
    double ts[3];
    int nt = 0;
    for (int a = 0; a < dim; ++a) {
        const double lo = x_old[a] < x_new[a] ? x_old[a] : x_new[a];
        const double hi = x_old[a] < x_new[a] ? x_new[a] : x_old[a];
        const double b = floor(lo - off) + 1.0 + off; /* first boundary above lo */
        if (b < hi) ts[nt++] = (b - x_old[a]) / (x_new[a] - x_old[a]);
    }
    for (int i = 1; i < nt; ++i) /* ascending */
        for (int j = i; j > 0 && ts[j] < ts[j - 1]; --j) {
            double t = ts[j];
            ts[j] = ts[j - 1];
            ts[j - 1] = t;
        }
    double xs[3] = {x_old[0], x_old[1], x_old[2]}, t0 = 0.0;
    for (int i = 0; i <= nt; ++i) {
        const double t1 = i < nt ? ts[i] : 1.0;
        double xe[3];
        for (int a = 0; a < 3; ++a) xe[a] = i < nt ? x_old[a] + t1 * (x_new[a] - x_old[a]) : x_new[a];
        if (t1 > t0) or_deposit_current(s, qw, xs, xe, vz * (t1 - t0), J);
        for (int a = 0; a < 3; ++a) xs[a] = xe[a];
        t0 = t1;
    }
}

/* ------------------------------------------------------------------ */
/* Laser antenna: a one-way plane source on the last axis (total-field / */
/* scattered-field split at node plane s).  The incident wave travels    */
/* towards +last axis, polarised along laser_pol, with                   */
/*   E_inc = a0 exp(-r^2/w0^2) exp(-2 ln2 (xi - t_peak)^2 / fwhm^2)      */
/*           cos(omega0 (xi - t_peak)),  xi = t - (z - z_plane),         */
/* the envelope being Gaussian in intensity with the given FWHM (Sec. 2: */
/* the laser drives the wake; Sec. 6 names the lasers; the shape is a   */
/* reading).                                                             */
/* ------------------------------------------------------------------ */
static double laser_field(const or_sim *s, double r2, double xi)
{
    double env = exp(-2.0 * log(2.0) * (xi - s->t_peak) * (xi - s->t_peak) / (s->fwhm * s->fwhm));
    return s->a0 * exp(-r2 / (s->waist * s->waist)) * env * cos(s->omega0 * (xi - s->t_peak));
}

/* radius^2 from the box axis of the transverse location of E_pol on the plane */
static double laser_r2(const or_sim *s, int64_t i, int64_t j)
{
    int last = s->dim - 1;
    double r2 = 0.0;
    int64_t idx[2] = {i, j};
    for (int a = 0; a < last; ++a) {
        double pos = ((double)idx[a] + yee_offset(s->laser_pol, a)) * s->d[a];
        double ctr = 0.5 * s->n[a] * s->d[a];
        r2 += (pos - ctr) * (pos - ctr);
    }
    return r2;
}

/* The B component carrying the incident wave and its sign: E_pol x B_b
 * points along +last axis.  3D (pol 0, last 2): B1 = +E.  2D (pol 0,
 * last 1): B2 = -E. */
static void laser_b_component(const or_sim *s, int *bcomp, double *sgn)
{
    if (s->dim == 3) {
        *bcomp = s->laser_pol == 0 ? 1 : 0;
        *sgn = s->laser_pol == 0 ? 1.0 : -1.0;
    } else {
        *bcomp = 2;
        *sgn = -1.0;
    }
}

static int laser_active(const or_sim *s)
{
    return s->laser_on && s->shifts == 0;
}

/* ------------------------------------------------------------------ */
/* Yee FDTD (Sec. 2; Sec. 3: a local field solver; Sec. 5.1: Yee mesh):  */
/* B -= h curl E with forward differences of E.  h = dt/2 per half step.*/
/* On an open last axis the B components at half-integer positions with */
/* index n-1 lie outside the domain and stay zero.                      */
/* ------------------------------------------------------------------ */
void or_yee_b(const or_sim *s, const double *E, double *B, double h)
{
    const int64_t nc = ncells(s);
    const int64_t n0 = s->n[0], n1 = s->n[1], n2 = s->n[2];
    const double *Ex = E, *Ey = E + nc, *Ez = E + 2 * nc;
    double *Bx = B, *By = B + nc, *Bz = B + 2 * nc;
    const int three = s->dim == 3;
    const double idx_ = 1.0 / s->d[0], idy = 1.0 / s->d[1], idz = three ? 1.0 / s->d[2] : 0.0;
    const int last = s->dim - 1;
    const int64_t nl = s->n[last];
    for (int64_t k = 0; k < n2; ++k)
        for (int64_t j = 0; j < n1; ++j)
            for (int64_t i = 0; i < n0; ++i) {
                int64_t c = cell_index(s, i, j, k);
                int64_t cx = cell_index(s, i + 1, j, k), cy = cell_index(s, i, j + 1, k);
                int64_t cz = three ? cell_index(s, i, j, k + 1) : c;
                double dEz_dy = (Ez[cy] - Ez[c]) * idy, dEy_dz = three ? (Ey[cz] - Ey[c]) * idz : 0.0;
                double dEx_dz = three ? (Ex[cz] - Ex[c]) * idz : 0.0, dEz_dx = (Ez[cx] - Ez[c]) * idx_;
                double dEy_dx = (Ey[cx] - Ey[c]) * idx_, dEx_dy = (Ex[cy] - Ex[c]) * idy;
                int64_t il = last == 2 ? k : j;
                /* half-integer positions along the last axis: B0,B1 in 3D; B0,B2 in 2D */
                int outside = s->open_last && il == nl - 1;
                if (three) {
                    if (!outside) {
                        Bx[c] -= h * (dEz_dy - dEy_dz);
                        By[c] -= h * (dEx_dz - dEz_dx);
                    }
                    Bz[c] -= h * (dEy_dx - dEx_dy);
                } else {
                    if (!outside) {
                        Bx[c] -= h * (dEz_dy - dEy_dz);
                        Bz[c] -= h * (dEy_dx - dEx_dy);
                    }
                    By[c] -= h * (dEx_dz - dEz_dx);
                }
            }
    if (laser_active(s)) {
        /* B_b at plane-1 saw total E_pol at plane: remove the incident part. */
        int bc;
        double sgn;
        laser_b_component(s, &bc, &sgn);
        double *Bb = B + (int64_t)bc * nc;
        int64_t ps = s->laser_plane;
        double xi = s->time; /* incident wave evaluated at the plane itself */
        if (three) {
            for (int64_t j = 0; j < n1; ++j)
                for (int64_t i = 0; i < n0; ++i)
                    Bb[cell_index(s, i, j, ps - 1)] += sgn * h * idz * laser_field(s, laser_r2(s, i, j), xi);
        } else {
            for (int64_t i = 0; i < n0; ++i)
                Bb[cell_index(s, i, ps - 1, 0)] += sgn * h * idy * laser_field(s, laser_r2(s, i, 0), xi);
        }
    }
}

/* E += dt (curl B - J) with backward differences of B; Mur first-order  */
/* absorbing update for the tangential E at both ends of an open last    */
/* axis; the laser correction on the total-field side of the plane.     */
void or_yee_e(const or_sim *s, double *E, const double *B, const double *J)
{
    const int64_t nc = ncells(s);
    const int64_t n0 = s->n[0], n1 = s->n[1], n2 = s->n[2];
    double *Ex = E, *Ey = E + nc, *Ez = E + 2 * nc;
    const double *Bx = B, *By = B + nc, *Bz = B + 2 * nc;
    const double *Jx = J, *Jy = J + nc, *Jz = J + 2 * nc;
    const int three = s->dim == 3;
    const double dt = s->dt;
    const double idx_ = 1.0 / s->d[0], idy = 1.0 / s->d[1], idz = three ? 1.0 / s->d[2] : 0.0;
    const int last = s->dim - 1;
    const int64_t nl = s->n[last];
    /* tangential components on the last axis: (0,1) in 3D, (0,2) in 2D */
    const int tan0 = 0, tan1 = three ? 1 : 2, normal = three ? 2 : 1;
    double *old = NULL;
    int64_t plane = three ? n0 * n1 : n0;
    if (s->open_last) {
        /* keep E^n on planes 0,1,nl-2,nl-1 for the Mur update */
        old = (double *)malloc(sizeof(double) * 2 * 4 * plane);
        for (int t = 0; t < 2; ++t) {
            const double *F = E + (int64_t)(t == 0 ? tan0 : tan1) * nc;
            int64_t pl[4] = {0, 1, nl - 2, nl - 1};
            for (int q = 0; q < 4; ++q)
                for (int64_t r = 0; r < plane; ++r) {
                    int64_t i = r % n0, jj = r / n0;
                    int64_t c = three ? cell_index(s, i, jj, pl[q]) : cell_index(s, i, pl[q], 0);
                    old[(t * 4 + q) * plane + r] = F[c];
                }
        }
    }
    for (int64_t k = 0; k < n2; ++k)
        for (int64_t j = 0; j < n1; ++j)
            for (int64_t i = 0; i < n0; ++i) {
                int64_t c = cell_index(s, i, j, k);
                int64_t mx = cell_index(s, i - 1, j, k), my = cell_index(s, i, j - 1, k);
                int64_t mz = three ? cell_index(s, i, j, k - 1) : c;
                double dBz_dy = (Bz[c] - Bz[my]) * idy, dBy_dz = three ? (By[c] - By[mz]) * idz : 0.0;
                double dBx_dz = three ? (Bx[c] - Bx[mz]) * idz : 0.0, dBz_dx = (Bz[c] - Bz[mx]) * idx_;
                double dBy_dx = (By[c] - By[mx]) * idx_, dBx_dy = (Bx[c] - Bx[my]) * idy;
                double nx_ = Ex[c] + dt * (dBz_dy - dBy_dz - Jx[c]);
                double ny_ = Ey[c] + dt * (dBx_dz - dBz_dx - Jy[c]);
                double nz_ = Ez[c] + dt * (dBy_dx - dBx_dy - Jz[c]);
                if (s->open_last) {
                    int64_t il = last == 2 ? k : j;
                    int bnd = il == 0 || il == nl - 1;
                    double *dst[3] = {&nx_, &ny_, &nz_};
                    double cur[3] = {Ex[c], Ey[c], Ez[c]};
                    if (bnd) { /* tangential: Mur below; keep the old value for now */
                        *dst[tan0] = cur[tan0];
                        *dst[tan1] = cur[tan1];
                    }
                    if (il == nl - 1) *dst[normal] = 0.0; /* half-integer position outside */
                }
                Ex[c] = nx_;
                Ey[c] = ny_;
                Ez[c] = nz_;
            }
    if (laser_active(s)) {
        /* E_pol at the plane saw scattered B_b at plane-1: add the incident B. */
        double *Ep = E + (int64_t)s->laser_pol * nc;
        int64_t ps = s->laser_plane;
        double t_half = s->time + 0.5 * dt;
        if (three) {
            double xi = t_half + 0.5 * s->d[2];
            for (int64_t j = 0; j < n1; ++j)
                for (int64_t i = 0; i < n0; ++i)
                    Ep[cell_index(s, i, j, ps)] += dt * idz * laser_field(s, laser_r2(s, i, j), xi);
        } else {
            double xi = t_half + 0.5 * s->d[1];
            for (int64_t i = 0; i < n0; ++i)
                Ep[cell_index(s, i, ps, 0)] += dt * idy * laser_field(s, laser_r2(s, i, 0), xi);
        }
    }
    if (s->open_last) {
        double dl = s->d[last];
        double coef = (dt - dl) / (dt + dl);
        for (int t = 0; t < 2; ++t) {
            double *F = E + (int64_t)(t == 0 ? tan0 : tan1) * nc;
            for (int64_t r = 0; r < plane; ++r) {
                int64_t i = r % n0, jj = r / n0;
                int64_t c0, c1, cm, cm1;
                if (three) {
                    c0 = cell_index(s, i, jj, 0);
                    c1 = cell_index(s, i, jj, 1);
                    cm = cell_index(s, i, jj, nl - 1);
                    cm1 = cell_index(s, i, jj, nl - 2);
                } else {
                    c0 = cell_index(s, i, 0, 0);
                    c1 = cell_index(s, i, 1, 0);
                    cm = cell_index(s, i, nl - 1, 0);
                    cm1 = cell_index(s, i, nl - 2, 0);
                }
                double o0 = old[(t * 4 + 0) * plane + r], o1 = old[(t * 4 + 1) * plane + r];
                double om1 = old[(t * 4 + 2) * plane + r], om = old[(t * 4 + 3) * plane + r];
                F[c0] = o1 + coef * (F[c1] - o0);
                F[cm] = om1 + coef * (F[cm1] - om);
            }
        }
        free(old);
    }
}

/* ------------------------------------------------------------------ */
/* Particle boundary on an open last axis: particles are kept while     */
/* g <= x_last < n_last - g, g = order + 1, so that no shape reaches the */
/* two boundary nodes' far side.                                         */
/* ------------------------------------------------------------------ */
static int particle_kept(const or_sim *s, const double *xp)
{
    if (!s->open_last) return 1;
    int last = s->dim - 1;
    double g = (double)(s->order + 1);
    return xp[last] >= g && xp[last] < (double)s->n[last] - g;
}

/* Plasma density at lab coordinate zlab along the last axis. */
static double profile_density(const or_sim *s, double zlab)
{
    if (s->n_knots <= 0 || s->knots == NULL) return s->density;
    if (s->n_knots == 1) return s->knots[0];
    double f = (zlab - s->z0) / (s->z1 - s->z0) * (s->n_knots - 1);
    if (f <= 0.0) return s->knots[0];
    if (f >= s->n_knots - 1) return s->knots[s->n_knots - 1];
    int i = (int)floor(f);
    double r = f - i;
    return s->knots[i] * (1.0 - r) + s->knots[i + 1] * r;
}

/* Moving window (Sec. 2: the box moves along with the laser pulse):    */
/* shift every field one cell back along the last axis, zero the new     */
/* front plane, move every particle one cell back, drop those leaving    */
/* the kept region and inject a cold, regularly placed layer at the      */
/* front.                                                                */
static void window_shift(or_sim *s, double *E, double *B, double *x, double *u, double *w,
                         int64_t *np, int64_t cap)
{
    const int64_t nc = ncells(s);
    const int last = s->dim - 1;
    const int64_t nl = s->n[last];
    const int64_t plane = nc / nl;
    for (int comp = 0; comp < 6; ++comp) {
        double *F = comp < 3 ? E + (int64_t)comp * nc : B + (int64_t)(comp - 3) * nc;
        memmove(F, F + plane, sizeof(double) * (size_t)(plane * (nl - 1)));
        memset(F + plane * (nl - 1), 0, sizeof(double) * (size_t)plane);
    }
    s->shifts += 1;
    int64_t n = *np, keep = 0;
    for (int64_t p = 0; p < n; ++p) {
        x[(int64_t)last * cap + p] -= 1.0;
        double xp[3] = {x[p], x[cap + p], s->dim == 3 ? x[2 * cap + p] : 0.0};
        if (!particle_kept(s, xp)) continue;
        for (int a = 0; a < 3; ++a) {
            x[(int64_t)a * cap + keep] = x[(int64_t)a * cap + p];
            u[(int64_t)a * cap + keep] = u[(int64_t)a * cap + p];
        }
        w[keep] = w[p];
        ++keep;
    }
    /* inject one layer of cells at last-axis cell index nl - g - 1 */
    int64_t g = s->order + 1;
    int64_t kcell = nl - g - 1;
    int ppc_tot = s->ppc[0] * s->ppc[1] * (s->dim == 3 ? s->ppc[2] : 1);
    int64_t ntr0 = s->n[0], ntr1 = s->dim == 3 ? s->n[1] : 1;
    for (int64_t c1 = 0; c1 < ntr1; ++c1)
        for (int64_t c0 = 0; c0 < ntr0; ++c0)
            for (int m2 = 0; m2 < (s->dim == 3 ? s->ppc[2] : 1); ++m2)
                for (int m1 = 0; m1 < s->ppc[1]; ++m1)
                    for (int m0 = 0; m0 < s->ppc[0]; ++m0) {
                        if (keep >= cap) break;
                        double pos[3];
                        pos[0] = c0 + (m0 + 0.5) / s->ppc[0];
                        if (s->dim == 3) {
                            pos[1] = c1 + (m1 + 0.5) / s->ppc[1];
                            pos[2] = kcell + (m2 + 0.5) / s->ppc[2];
                        } else {
                            pos[1] = kcell + (m1 + 0.5) / s->ppc[1];
                            pos[2] = 0.0;
                        }
                        double zlab = (pos[last] + (double)s->shifts) * s->d[last];
                        for (int a = 0; a < 3; ++a) {
                            x[(int64_t)a * cap + keep] = pos[a];
                            u[(int64_t)a * cap + keep] = 0.0;
                        }
                        w[keep] = profile_density(s, zlab) / ppc_tot;
                        ++keep;
                    }
    *np = keep;
}

/* ------------------------------------------------------------------ */
/* One full timestep, repeated nsteps times (Sec. 2 loop order):         */
/*   particles: gather E^n,B^n at x^n -> Boris u^{n+1/2} -> x^{n+1} ->    */
/*   deposit J^{n+1/2} into the thread's private copy (Sec. 3.1);         */
/*   reduce the copies; drop absorbed particles;                          */
/*   fields: B^{n+1/2} = B^n - dt/2 curl E^n; E^{n+1} = E^n + dt (curl    */
/*   B^{n+1/2} - J^{n+1/2}); B^{n+1} = B^{n+1/2} - dt/2 curl E^{n+1};     */
/*   t += dt; moving-window shift when due.                               */
/* x,u: [3][cap] component-major (unused axes ignored); w: [cap].         */
/* ------------------------------------------------------------------ */
int or_step(or_sim *s, double *E, double *B, double *J, double *x, double *u, double *w,
            int64_t *np, int64_t cap, int nsteps)
{
    const int64_t nc = ncells(s);
    const int dim = s->dim;
    int nt = s->nthreads > 0 ? s->nthreads : 1;
#ifndef _OPENMP
    nt = 1;
#endif
    double *copies = (double *)calloc((size_t)nt * 3 * (size_t)nc, sizeof(double));
    unsigned char *keep = NULL;
    if (!copies) return -1;
    for (int st = 0; st < nsteps; ++st) {
        int64_t n = *np;
        free(keep);
        keep = (unsigned char *)malloc((size_t)(n > 0 ? n : 1));
        memset(copies, 0, sizeof(double) * (size_t)nt * 3 * (size_t)nc);
#pragma omp parallel num_threads(nt)
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            double *Jt = copies + (int64_t)tid * 3 * nc;
            /* even division of particles across threads (Sec. 3.1) */
            int64_t b0 = n * tid / nt, b1 = n * (tid + 1) / nt;
            for (int64_t p = b0; p < b1; ++p) {
                double xo[3], xn[3], up[3], eb[6];
                for (int a = 0; a < 3; ++a) {
                    xo[a] = a < dim ? x[(int64_t)a * cap + p] : 0.0;
                    up[a] = u[(int64_t)a * cap + p];
                }
                or_gather(s, E, B, xo, eb);
                or_boris(s->q / s->m, s->dt, eb, up);
                double gam = sqrt(1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
                for (int a = 0; a < 3; ++a) xn[a] = a < dim ? xo[a] + s->dt * up[a] / (gam * s->d[a]) : 0.0;
                if (s->split) or_deposit_current_split(s, s->q * w[p], xo, xn, up[2] / gam, Jt);
                else or_deposit_current(s, s->q * w[p], xo, xn, up[2] / gam, Jt);
                keep[p] = (unsigned char)particle_kept(s, xn);
                for (int a = 0; a < 3; ++a) {
                    u[(int64_t)a * cap + p] = up[a];
                    if (a < dim) {
                        double v = xn[a];
                        if (!(s->open_last && a == dim - 1)) { /* periodic wrap */
                            double L = (double)s->n[a];
                            v = fmod(v, L);
                            if (v < 0.0) v += L;
                            if (v >= L) v -= L;
                        }
                        x[(int64_t)a * cap + p] = v;
                    }
                }
            }
        }
        /* threaded reduction of the n_T current copies (Sec. 3.1) */
#pragma omp parallel for num_threads(nt) schedule(static)
        for (int64_t c = 0; c < 3 * nc; ++c) {
            double acc = 0.0;
            for (int t = 0; t < nt; ++t) acc += copies[(int64_t)t * 3 * nc + c];
            J[c] = acc;
        }
        if (s->open_last) {
            int64_t kept = 0;
            for (int64_t p = 0; p < n; ++p) {
                if (!keep[p]) continue;
                for (int a = 0; a < 3; ++a) {
                    x[(int64_t)a * cap + kept] = x[(int64_t)a * cap + p];
                    u[(int64_t)a * cap + kept] = u[(int64_t)a * cap + p];
                }
                w[kept] = w[p];
                ++kept;
            }
            *np = kept;
        }
        or_yee_b(s, E, B, 0.5 * s->dt);
        or_yee_e(s, E, B, J);
        s->time += s->dt; /* second half of B sees E^{n+1} at t^{n+1} */
        or_yee_b(s, E, B, 0.5 * s->dt);
        s->step += 1;
        if (s->window_on && s->time >= s->window_t0) {
            double travelled = s->window_v * (s->time - s->window_t0);
            if (travelled >= (double)(s->shifts + 1) * s->d[dim - 1])
                window_shift(s, E, B, x, u, w, np, cap);
        }
    }
    free(keep);
    free(copies);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Diagnostics.                                                         */
/* ------------------------------------------------------------------ */
/* div E at every node (backward differences of the staggered E). */
void or_div_e(const or_sim *s, const double *E, double *out)
{
    const int64_t nc = ncells(s);
    const int three = s->dim == 3;
    for (int64_t k = 0; k < s->n[2]; ++k)
        for (int64_t j = 0; j < s->n[1]; ++j)
            for (int64_t i = 0; i < s->n[0]; ++i) {
                int64_t c = cell_index(s, i, j, k);
                double v = (E[c] - E[cell_index(s, i - 1, j, k)]) / s->d[0] +
                           (E[nc + c] - E[nc + cell_index(s, i, j - 1, k)]) / s->d[1];
                if (three) v += (E[2 * nc + c] - E[2 * nc + cell_index(s, i, j, k - 1)]) / s->d[2];
                out[c] = v;
            }
}

/* out[0] = W_E = 1/2 sum E^2 V, out[1] = W_B, out[2] = W_kin = V sum w m (gamma-1). */
void or_energies(const or_sim *s, const double *E, const double *B, const double *u, const double *w,
                 int64_t n, int64_t cap, double *out)
{
    const int64_t nc = ncells(s);
    double V = s->d[0] * s->d[1] * (s->dim == 3 ? s->d[2] : 1.0);
    double we = 0.0, wb = 0.0, wk = 0.0;
    for (int64_t c = 0; c < 3 * nc; ++c) {
        we += E[c] * E[c];
        wb += B[c] * B[c];
    }
    for (int64_t p = 0; p < n; ++p) {
        double ux = u[p], uy = u[cap + p], uz = u[2 * cap + p];
        wk += w[p] * s->m * (sqrt(1.0 + ux * ux + uy * uy + uz * uz) - 1.0);
    }
    out[0] = 0.5 * we * V;
    out[1] = 0.5 * wb * V;
    out[2] = wk * V;
}

/* rho of all particles (charge q w each) added into rho[ncells]. */
void or_charge(const or_sim *s, const double *x, const double *w, int64_t n, int64_t cap, double *rho)
{
    for (int64_t p = 0; p < n; ++p) {
        double xp[3] = {x[p], x[cap + p], s->dim == 3 ? x[2 * cap + p] : 0.0};
        or_deposit_rho(s, s->q * w[p], xp, rho);
    }
}

int or_abi_size(void)
{
    return (int)sizeof(or_sim);
}
