/*
 * FP64 CPU oracle of the implicit regularized enthalpy based method (IREBM).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  It shares no
 * code, header, table or constant with the CUDA library: lattice tables, the
 * boundary closures, the Newton solve and the adjoint are all written here
 * again, on purpose, in the plainest form.
 *
 * Source: F. Luddens, C. Lothode, I. Danaila, "An implicit regularized
 * enthalpy Lattice Boltzmann Method for the Stefan problem" (arXiv 2505.13097).
 * Equation numbers follow the paper's order of numbered equations:
 *   (12) def_qi_omegai   Omega_i = (1-1/tau) f_i + f_i^eq / tau, q_i = streamed Omega_i
 *   (13) rhs_fl_stag     f_i(t+1) = q_i + (w_i/Ste)(phi(theta) - phi(theta~))
 *   (14) rhs_fl_2        theta~ = M0(q) + (phi(theta) - phi(theta~))/Ste
 *   (15) Dirichlet       closure on M0(q) at a Dirichlet node
 *   (16) Dir_on_q        single-unknown form of (15) (D1Q3, D2Q5)
 *   (17) Neu_on_q        Neumann closure through the inner neighbour's M0(q) (D2Q5)
 * One step, as the paper states the method (Sec. 4, Algorithm 3), written here
 * from the equations: theta = M0(f); the collision of Eq. (12); pull
 * streaming of Omega into q; the closures of Sec. 4.2 on the q that streaming
 * leaves undefined (Eqs. 15-17, and the bounce-back q_ix = q_{bar ix} of
 * Sec. 4.2.2); the local nonlinear equation (14) for theta~, solved by
 * Newton's method from theta; the source and update of Eq. (13).  Each of
 * these is one pass over the lattice, in that order.
 *
 * Storage: the oracle stores the distributions f_i (q planes of nx*ny doubles,
 * x fastest) and recomputes theta = M0(f) at the start of every step.  No
 * blocking, fusion or reordering of those passes.
 *
 * Readings where the paper is silent:
 *  - weights: D1Q3 (2/3, 1/6, 1/6), D2Q5 (1/3, 1/6 x4), D2Q9 (4/9, 1/9 x4,
 *    1/36 x4), c_s^2 = 1/3 on all three.
 *  - Newton stopping: |x_{k+1}-x_k| <= tol*max(1,|x_k|) (x_{k+1} kept), or
 *    F(x_k) = 0, or a bracket narrower than that; at most maxit iterations.
 *  - Newton safeguard: the root lies in [m0 + (phi(theta)-1)/Ste, m0 + phi(theta)/Ste]
 *    (0 <= phi <= 1 and F increasing); an iterate that leaves the current
 *    bracket, or does not at least halve the update before last, is replaced
 *    by the bracket midpoint.
 *  - Dirichlet on D2Q9: the unknown q_i share R = m0_target - sum(known q)
 *    in proportion to w_i.  m0_target follows from Eq. (14) with
 *    theta~ = theta_D (see orc_dirichlet_m0 for the sign of the phi term).
 *  - A node on a Dirichlet wall is a Dirichlet node, corners included
 *    ("Dirichlet beats Neumann"); its value is that of the first Dirichlet
 *    wall in the order W, E, S, N.
 *  - Bounce-back: mirror q_i = q_{bar i} (Sec. 4.2.2) where q_{bar i} is known,
 *    else (corner diagonals, thin domains) link-wise q_i = Omega_{bar i} at the
 *    node.  bb_mode = 1 uses the link-wise form for every unknown direction.
 *  - bb_mode = 2 (D2Q5, nx and ny >= 3): the Neumann closure of Eq. (17),
 *    M0(q) at a wall node = M0(q) at the node one step inwards; at a corner of
 *    two adiabatic walls that is the diagonal interior node, and the two
 *    unknowns share the remainder by weight (equally).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXQ 9   /* D2Q9; D2Q5 and D1Q3 use the first 5 / 3 entries */

typedef struct {
    int lattice;          /* 1 = D1Q3, 2 = D2Q9, 3 = D2Q5 */
    int nx, ny;           /* ny = 1 for D1Q3 */
    double tau, delta, ste;
    double newton_tol;
    int newton_max_iter;
    int bb_mode;          /* 0 = mirror (Sec. 4.2.2), 1 = link-wise */
    int wall_kind[4];     /* W, E, S, N: 0 = adiabatic, 1 = Dirichlet */
    double wall_theta[4];
} orc_params;

typedef struct {          /* per-step diagnostics */
    double energy_before; /* sum_x theta + phi(theta)/Ste at time t   */
    double energy_after;  /* same at time t+1 (theta = M0(f(t+1)))    */
    double flux;          /* sum of filled q minus Omega leaving the lattice */
    int max_iter;         /* largest Newton iteration count            */
    int failed;           /* number of nodes where Newton did not converge */
} orc_diag;

/* ---- lattice tables (Sec. 3.2; weights are the standard ones) ---- */
static int lat_q(const orc_params* p) { return p->lattice == 1 ? 3 : (p->lattice == 3 ? 5 : 9); }

static void lat_vec(const orc_params* p, int i, int* ex, int* ey, double* w)
{
    if (p->lattice == 1) {
        static const int e1[3] = {0, 1, -1};
        static const double w1[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};
        *ex = e1[i]; *ey = 0; *w = w1[i];
    } else if (p->lattice == 3) {
        /* D2Q5: rest, +x, +y, -x, -y; weights 1/3 and 1/6 (c_s^2 = 1/3) */
        static const int e5x[5] = {0, 1, 0, -1, 0};
        static const int e5y[5] = {0, 0, 1, 0, -1};
        static const double w5[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
        *ex = e5x[i]; *ey = e5y[i]; *w = w5[i];
    } else {
        static const int e2x[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        static const int e2y[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        static const double w2[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                                     1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
        *ex = e2x[i]; *ey = e2y[i]; *w = w2[i];
    }
}

/* index of the direction opposite to i: e_{bar i} = -e_i */
static int lat_opp(const orc_params* p, int i)
{
    int ex, ey, jx, jy, j, q = lat_q(p);
    double w;
    lat_vec(p, i, &ex, &ey, &w);
    for (j = 0; j < q; j++) {
        lat_vec(p, j, &jx, &jy, &w);
        if (jx == -ex && jy == -ey) return j;
    }
    return -1;
}

/* ---- regularized liquid fraction, Sec. 4.1: phi_d = (1 + tanh(x/d))/2 ---- */
double orc_phi(double x, double delta) { return 0.5 * (1.0 + tanh(x / delta)); }

double orc_dphi(double x, double delta)
{
    double t = tanh(x / delta);
    return 0.5 * (1.0 - t * t) / delta;
}

/*
 * Local Newton solve of Eq. (14): find x with
 *     F(x) = (x - m0) + (phi(x) - phi(theta))/Ste = 0,
 * using the update of Algorithm 3 started at x = theta.  F' = 1 + phi'/Ste >= 1,
 * so the root is unique.  The two phi terms of Algorithm 3's update are
 * grouped as (phi(theta) - phi(x))/Ste so that they cancel before the division
 * by Ste (same algebra, no loss of the low bits of m0 when 1/Ste is large).
 * Stops when a Newton update moves x by at most tol*max(1,|x|) (that update
 * is kept; the test comes before the safeguard, so a last correction that
 * rounds just outside the bracket is not mistaken for a wild step), when F(x)
 * is exactly 0, or when the safeguard bracket has shrunk below that size.  Returns the root; *iters = iterations used; *ok = 0 if
 * maxit was reached first.
 */
double orc_newton(double m0, double theta, double ste, double delta, double tol, int maxit,
                  int* iters, int* ok)
{
    double pth = orc_phi(theta, delta);
    double lo = m0 + (pth - 1.0) / ste, hi = m0 + pth / ste;   /* F(lo) <= 0 <= F(hi): 0 <= phi <= 1 */
    double x = theta;
    double step_old = hi - lo, step = step_old;   /* sizes of the last two updates */
    int k;
    *ok = 0;
    for (k = 0; k < maxit; k++) {
        double t = tanh(x / delta);
        double ph = 0.5 * (1.0 + t), dph = 0.5 * (1.0 - t * t) / delta;
        double F = (x - m0) + (ph - pth) / ste;
        double xn;
        if (F == 0.0) { *ok = 1; break; }
        if (F < 0.0) { if (x > lo) lo = x; } else { if (x < hi) hi = x; }
        /* Algorithm 3: theta^(k+1) = (m0 + phi(theta)/Ste + phi'(x) x/Ste - phi(x)/Ste) / (1 + phi'(x)/Ste) */
        xn = (m0 + (pth - ph) / ste + dph * x / ste) / (1.0 + dph / ste);
        if (fabs(xn - x) <= tol * fmax(1.0, fabs(x))) { x = xn; *ok = 1; k++; break; }
        /* safeguard: bisect the bracket when the Newton iterate leaves it or does
           not at least halve the update before last (this also breaks cycles) */
        if (!(xn >= lo && xn <= hi) || fabs(xn - x) > 0.5 * step_old) {
            step_old = step;
            step = 0.5 * (hi - lo);
            xn = lo + step;
            if (step <= tol * fmax(1.0, fabs(xn))) { x = xn; *ok = 1; k++; break; }
        } else {
            step_old = step;
            step = fabs(xn - x);
        }
        x = xn;
    }
    *iters = k;
    return x;
}

/* ---- node classification for the boundary closures (Sec. 4.2) ---- */
static int inside(const orc_params* p, int x, int y) { return x >= 0 && x < p->nx && y >= 0 && y < p->ny; }

/* walls touching node (x,y): bit 0 = W, 1 = E, 2 = S, 3 = N */
static int node_walls(const orc_params* p, int x, int y)
{
    int m = 0;
    if (x == 0) m |= 1;
    if (x == p->nx - 1) m |= 2;
    if (p->lattice != 1) {
        if (y == 0) m |= 4;
        if (y == p->ny - 1) m |= 8;
    }
    return m;
}

/* 1 and the wall value if the node lies on a Dirichlet wall (first in W, E, S, N) */
static int node_dirichlet(const orc_params* p, int x, int y, double* theta_d, int* wall)
{
    int m = node_walls(p, x, y), k;
    for (k = 0; k < 4; k++)
        if ((m >> k & 1) && p->wall_kind[k] == 1) {
            *theta_d = p->wall_theta[k];
            if (wall) *wall = k;
            return 1;
        }
    return 0;
}

/*
 * Target of M0(q) at a Dirichlet node.  Eq. (14) with theta~ = theta_D gives
 *     M0(q) = theta_D + (phi(theta_D) - phi(theta))/Ste,
 * theta being the node's current temperature.  Eq. (15) prints the phi
 * difference with the opposite sign; both coincide when theta = theta_D,
 * which holds at every step once the wall node starts at theta_D.
 */
static double orc_dirichlet_m0(const orc_params* p, double theta_d, double theta)
{
    return theta_d + (orc_phi(theta_d, p->delta) - orc_phi(theta, p->delta)) / p->ste;
}

/* ---- initial state: f_i = w_i theta0 (equilibrium); Dirichlet nodes at theta_D ---- */
void orc_init(const orc_params* p, const double* theta0, double* f)
{
    int q = lat_q(p), n = p->nx * p->ny, x, y, i, ex, ey;
    double w;
    for (y = 0; y < p->ny; y++)
        for (x = 0; x < p->nx; x++) {
            double th = theta0[y * p->nx + x], td;
            if (node_dirichlet(p, x, y, &td, NULL)) th = td;
            for (i = 0; i < q; i++) {
                lat_vec(p, i, &ex, &ey, &w);
                f[i * n + y * p->nx + x] = w * th;
            }
        }
}

/* theta = M0(f) (Algorithm 3, line "moments") */
void orc_theta(const orc_params* p, const double* f, double* theta)
{
    int q = lat_q(p), n = p->nx * p->ny, k, i;
    for (k = 0; k < n; k++) {
        double s = 0.0;
        for (i = 0; i < q; i++) s += f[i * n + k];
        theta[k] = s;
    }
}

double orc_energy(const orc_params* p, const double* f)
{
    int q = lat_q(p), n = p->nx * p->ny, k, i;
    double e = 0.0;
    for (k = 0; k < n; k++) {
        double th = 0.0;
        for (i = 0; i < q; i++) th += f[i * n + k];
        e += th + orc_phi(th, p->delta) / p->ste;
    }
    return e;
}

/* M0 of the streamed populations at node (x, y): sum_i Omega_i(x - e_i) over
 * the lattice (every x - e_i inside for an interior node) */
static double orc_pulled_m0(const orc_params* p, const double* Om, int x, int y)
{
    const int n = p->nx * p->ny;
    double s = 0.0, w;
    int i, ex, ey;
    for (i = 0; i < lat_q(p); i++) {
        lat_vec(p, i, &ex, &ey, &w);
        if (inside(p, x - ex, y - ey)) s += Om[i * n + (y - ey) * p->nx + (x - ex)];
    }
    return s;
}

/*
 * One IREBM time step, Algorithm 3, f -> fn.
 * Optional outputs (may be NULL): per-node m0, theta (time t), theta~ (root),
 * Newton iterations, and the step diagnostics.
 */
int orc_step(const orc_params* p, const double* f, double* fn, double* m0_out, double* theta_out,
             double* root_out, int* iters_out, orc_diag* diag)
{
    const int q = lat_q(p), nx = p->nx, ny = p->ny, n = nx * ny;
    const double omega = 1.0 / p->tau;
    double* theta = (double*)malloc(sizeof(double) * n);
    double* Om = (double*)malloc(sizeof(double) * q * n);
    double flux = 0.0, e0 = 0.0, e1 = 0.0;
    int x, y, i, failed = 0, maxit_seen = 0;
    int ex[ORC_MAXQ], ey[ORC_MAXQ], opp[ORC_MAXQ];
    double w[ORC_MAXQ];
    if (!theta || !Om) { free(theta); free(Om); return -1; }
    for (i = 0; i < q; i++) { lat_vec(p, i, &ex[i], &ey[i], &w[i]); opp[i] = lat_opp(p, i); }

    /* moments: theta <- M0(f) */
    orc_theta(p, f, theta);
    if (diag)
        for (x = 0; x < n; x++) e0 += theta[x] + orc_phi(theta[x], p->delta) / p->ste;

    /* equilibrium and collision, Eq. (12): Omega_i = (1-1/tau) f_i + w_i theta / tau */
    for (i = 0; i < q; i++)
        for (x = 0; x < n; x++) Om[i * n + x] = (1.0 - omega) * f[i * n + x] + omega * w[i] * theta[x];

    /* Omega leaving the lattice (for the energy balance) */
    for (y = 0; y < ny; y++)
        for (x = 0; x < nx; x++)
            for (i = 0; i < q; i++)
                if (!inside(p, x + ex[i], y + ey[i])) flux -= Om[i * n + y * nx + x];

    for (y = 0; y < ny; y++)
        for (x = 0; x < nx; x++) {
            const int k = y * nx + x;
            double qv[ORC_MAXQ];
            int known[ORC_MAXQ], nunk = 0;
            double m0, root, td, g;
            int it, ok;

            /* streaming: q_i(y) = Omega_i(y - e_i) where y - e_i is in the lattice */
            for (i = 0; i < q; i++) {
                int sx = x - ex[i], sy = y - ey[i];
                known[i] = inside(p, sx, sy);
                qv[i] = known[i] ? Om[i * n + sy * nx + sx] : 0.0;
                if (!known[i]) nunk++;
            }

            /* boundary closures on q (Sec. 4.2) */
            if (nunk > 0) {
                if (node_dirichlet(p, x, y, &td, NULL)) {
                    /* Eq. (15): M0(q) = m0_target; unknowns share the rest by weight */
                    double rest = orc_dirichlet_m0(p, td, theta[k]), wu = 0.0;
                    for (i = 0; i < q; i++) {
                        if (known[i]) rest -= qv[i];
                        else wu += w[i];
                    }
                    for (i = 0; i < q; i++)
                        if (!known[i]) qv[i] = w[i] * rest / wu;
                } else if (p->bb_mode == 2) {
                    /* Eq. (17): M0(q) of the node equals M0(q) of the interior node
                     * one lattice step inwards (the diagonal one at a corner); the
                     * unknowns share the rest by weight, as at a Dirichlet node */
                    const int sx = x + (x == 0 ? 1 : (x == nx - 1 ? -1 : 0));
                    const int sy = y + (y == 0 ? 1 : (y == ny - 1 ? -1 : 0));
                    double rest = orc_pulled_m0(p, Om, sx, sy), wu = 0.0;
                    for (i = 0; i < q; i++) {
                        if (known[i]) rest -= qv[i];
                        else wu += w[i];
                    }
                    for (i = 0; i < q; i++)
                        if (!known[i]) qv[i] = w[i] * rest / wu;
                } else {
                    /* bounce-back, Sec. 4.2.2 */
                    for (i = 0; i < q; i++)
                        if (!known[i]) {
                            if (p->bb_mode == 0 && known[opp[i]]) qv[i] = qv[opp[i]];
                            else qv[i] = Om[opp[i] * n + k];
                        }
                }
                for (i = 0; i < q; i++)
                    if (!known[i]) flux += qv[i];
            }

            /* Newton initialization and loop (Algorithm 3) */
            m0 = 0.0;
            for (i = 0; i < q; i++) m0 += qv[i];
            root = orc_newton(m0, theta[k], p->ste, p->delta, p->newton_tol, p->newton_max_iter, &it, &ok);
            if (!ok) failed++;
            if (it > maxit_seen) maxit_seen = it;

            /* source term and update, Eq. (13) */
            g = (orc_phi(theta[k], p->delta) - orc_phi(root, p->delta)) / p->ste;
            for (i = 0; i < q; i++) fn[i * n + k] = qv[i] + w[i] * g;

            if (m0_out) m0_out[k] = m0;
            if (theta_out) theta_out[k] = theta[k];
            if (root_out) root_out[k] = root;
            if (iters_out) iters_out[k] = it;
        }

    if (diag) {
        double th;
        for (x = 0; x < n; x++) {
            th = 0.0;
            for (i = 0; i < q; i++) th += fn[i * n + x];
            e1 += th + orc_phi(th, p->delta) / p->ste;
        }
        diag->energy_before = e0;
        diag->energy_after = e1;
        diag->flux = flux;
        diag->max_iter = maxit_seen;
        diag->failed = failed;
    }
    free(theta);
    free(Om);
    return failed;
}

/* nsteps steps from theta0; final f and theta. Returns the number of Newton failures. */
int orc_run(const orc_params* p, const double* theta0, int nsteps, double* f_out, double* theta_out)
{
    int q = lat_q(p), n = p->nx * p->ny, s, failed = 0;
    double* a = (double*)malloc(sizeof(double) * q * n);
    double* b = (double*)malloc(sizeof(double) * q * n);
    if (!a || !b) { free(a); free(b); return -1; }
    orc_init(p, theta0, a);
    for (s = 0; s < nsteps; s++) {
        double* t;
        int r = orc_step(p, a, b, NULL, NULL, NULL, NULL, NULL);
        if (r < 0) { failed = -1; break; }
        failed += r;
        t = a; a = b; b = t;
    }
    if (f_out) memcpy(f_out, a, sizeof(double) * q * n);
    if (theta_out) orc_theta(p, a, theta_out);
    free(a);
    free(b);
    return failed;
}

/* ------------------------------------------------------------------------
 * Liquid-fraction misfit and its FP64 discrete adjoint.
 *
 * Loss: L = 1/2 sum_x (phi(theta_T(x)) - phi_target(x))^2 with theta_T = M0(f_T).
 * The adjoint is the exact transpose of the oracle's own step (the f storage
 * above), by reverse accumulation over a tape of theta(t) and the Newton
 * roots.  The Newton root enters through the implicit function theorem on
 * F(x) = x + phi(x)/Ste - m0 - phi(theta)/Ste:
 *   d root/d m0 = 1/F',  d root/d theta = phi'(theta)/(Ste F'),
 *   d root/d Ste = (phi(root) - phi(theta))/(Ste^2 F'),  F' = 1 + phi'(root)/Ste.
 * ------------------------------------------------------------------------ */
double orc_loss(const orc_params* p, const double* theta0, int nsteps, const double* phi_target)
{
    int n = p->nx * p->ny, k;
    double* th = (double*)malloc(sizeof(double) * n);
    double L = 0.0;
    if (!th) return NAN;
    orc_run(p, theta0, nsteps, NULL, th);
    for (k = 0; k < n; k++) {
        double d = orc_phi(th[k], p->delta) - phi_target[k];
        L += 0.5 * d * d;
    }
    free(th);
    return L;
}

/*
 * Gradient of orc_loss with respect to theta0 (n values; zero at Dirichlet
 * nodes, whose initial value is the wall's), the four wall temperatures
 * (only Dirichlet walls receive a value) and Ste.  Returns L.
 */
double orc_adjoint(const orc_params* p, const double* theta0, int nsteps, const double* phi_target,
                   double* g_theta0, double* g_wall, double* g_ste)
{
    const int q = lat_q(p), nx = p->nx, ny = p->ny, n = nx * ny;
    const double omega = 1.0 / p->tau, ste = p->ste, dl = p->delta;
    double *f = NULL, *fn = NULL, *tape_th = NULL, *tape_root = NULL, *fb = NULL, *fbn = NULL;
    double *Ob = NULL, *thb = NULL;
    double L = 0.0, gste = 0.0, gw[4] = {0, 0, 0, 0};
    int ex[ORC_MAXQ], ey[ORC_MAXQ], opp[ORC_MAXQ];
    double w[ORC_MAXQ];
    int s, x, y, i, k;

    for (i = 0; i < q; i++) { lat_vec(p, i, &ex[i], &ey[i], &w[i]); opp[i] = lat_opp(p, i); }
    f = (double*)malloc(sizeof(double) * q * n);
    fn = (double*)malloc(sizeof(double) * q * n);
    tape_th = (double*)malloc(sizeof(double) * (size_t)n * (nsteps + 1));
    tape_root = (double*)malloc(sizeof(double) * (size_t)n * (nsteps > 0 ? nsteps : 1));
    fb = (double*)malloc(sizeof(double) * q * n);
    fbn = (double*)malloc(sizeof(double) * q * n);
    Ob = (double*)malloc(sizeof(double) * q * n);
    thb = (double*)malloc(sizeof(double) * n);
    if (!f || !fn || !tape_th || !tape_root || !fb || !fbn || !Ob || !thb) { L = NAN; goto done; }

    /* forward sweep, recording theta(t) and the roots */
    orc_init(p, theta0, f);
    for (s = 0; s < nsteps; s++) {
        double* t;
        orc_step(p, f, fn, NULL, tape_th + (size_t)s * n, tape_root + (size_t)s * n, NULL, NULL);
        t = f; f = fn; fn = t;
    }
    orc_theta(p, f, tape_th + (size_t)nsteps * n);

    /* seed: dL/df_i(T) = (phi(theta_T) - phi*) phi'(theta_T) for every i */
    for (k = 0; k < n; k++) {
        double thT = tape_th[(size_t)nsteps * n + k];
        double d = orc_phi(thT, dl) - phi_target[k];
        L += 0.5 * d * d;
        for (i = 0; i < q; i++) fb[i * n + k] = d * orc_dphi(thT, dl);
    }

    for (s = nsteps - 1; s >= 0; s--) {
        const double* th = tape_th + (size_t)s * n;
        const double* rt = tape_root + (size_t)s * n;
        memset(Ob, 0, sizeof(double) * q * n);
        memset(thb, 0, sizeof(double) * n);
        for (y = 0; y < ny; y++)
            for (x = 0; x < nx; x++) {
                const int kk = y * nx + x;
                double qb[ORC_MAXQ], S = 0.0, rb, Fp, m0b, td;
                int known[ORC_MAXQ], nunk = 0;
                for (i = 0; i < q; i++) {
                    known[i] = inside(p, x - ex[i], y - ey[i]);
                    if (!known[i]) nunk++;
                }
                /* f(t+1)_i = q_i + w_i g,  g = (phi(theta) - phi(root))/Ste */
                for (i = 0; i < q; i++) { qb[i] = fb[i * n + kk]; S += w[i] * fb[i * n + kk]; }
                S /= ste;
                thb[kk] += S * orc_dphi(th[kk], dl);
                rb = -S * orc_dphi(rt[kk], dl);
                gste += -S * (orc_phi(th[kk], dl) - orc_phi(rt[kk], dl)) / ste;
                /* Newton root, implicit function theorem */
                Fp = 1.0 + orc_dphi(rt[kk], dl) / ste;
                m0b = rb / Fp;
                thb[kk] += rb * orc_dphi(th[kk], dl) / (ste * Fp);
                gste += rb * (orc_phi(rt[kk], dl) - orc_phi(th[kk], dl)) / (ste * ste * Fp);
                for (i = 0; i < q; i++) qb[i] += m0b;
                /* boundary closures, transposed */
                if (nunk > 0) {
                    int wall = -1;
                    if (node_dirichlet(p, x, y, &td, &wall)) {
                        double wu = 0.0, A = 0.0;
                        for (i = 0; i < q; i++)
                            if (!known[i]) wu += w[i];
                        for (i = 0; i < q; i++)
                            if (!known[i]) A += qb[i] * w[i] / wu;
                        for (i = 0; i < q; i++)
                            if (known[i]) qb[i] -= A;
                        gw[wall] += A * (1.0 + orc_dphi(td, dl) / ste);
                        thb[kk] += -A * orc_dphi(th[kk], dl) / ste;
                        gste += -A * (orc_phi(td, dl) - orc_phi(th[kk], dl)) / (ste * ste);
                    } else {
                        for (i = 0; i < q; i++)
                            if (!known[i]) {
                                if (p->bb_mode == 0 && known[opp[i]]) qb[opp[i]] += qb[i];
                                else Ob[opp[i] * n + kk] += qb[i];
                            }
                    }
                }
                /* streaming, transposed: q_i(y) = Omega_i(y - e_i) */
                for (i = 0; i < q; i++)
                    if (known[i]) Ob[i * n + (y - ey[i]) * nx + (x - ex[i])] += qb[i];
            }
        /* collision Omega_i = (1-omega) f_i + omega w_i theta and theta = M0(f), transposed */
        for (k = 0; k < n; k++) {
            double tb = thb[k];
            for (i = 0; i < q; i++) tb += omega * w[i] * Ob[i * n + k];
            for (i = 0; i < q; i++) fbn[i * n + k] = (1.0 - omega) * Ob[i * n + k] + tb;
        }
        { double* t = fb; fb = fbn; fbn = t; }
    }

    /* initial state f_i = w_i theta0 (or w_i theta_D on Dirichlet nodes) */
    for (y = 0; y < ny; y++)
        for (x = 0; x < nx; x++) {
            const int kk = y * nx + x;
            double s0 = 0.0, td;
            int wall = -1;
            for (i = 0; i < q; i++) s0 += w[i] * fb[i * n + kk];
            if (node_dirichlet(p, x, y, &td, &wall)) {
                gw[wall] += s0;
                if (g_theta0) g_theta0[kk] = 0.0;
            } else if (g_theta0) {
                g_theta0[kk] = s0;
            }
        }
    if (g_wall) for (k = 0; k < 4; k++) g_wall[k] = gw[k];
    if (g_ste) *g_ste = gste;
done:
    free(f); free(fn); free(tape_th); free(tape_root); free(fb); free(fbn); free(Ob); free(thb);
    return L;
}

/* ======================================================================
 * Explicit enthalpy based method (EEBM), Algorithm 2 and Sec. 3.4 of the
 * paper: the distributions carry the enthalpy, H = M0(f); the temperature
 * follows explicitly from H through Theta (no source term, no Newton):
 *     Theta(H) = H if H < 0,  0 if 0 <= H <= 1/Ste,  H - 1/Ste if H > 1/Ste;
 * equilibrium f_i^eq = w_i theta (i != 0), f_0^eq = H - (1 - w_0) theta, so
 * that M0(f^eq) = H; collision Omega_i = f_i - (f_i - f_i^eq)/tau; streaming
 * f~_i(y) = Omega_i(y - e_i).
 * Boundary closures (the paper leaves EEBM's to standard techniques): the
 * same as IREBM's on the streamed distributions, with the Dirichlet target
 * M0(f~) = H(theta_D) = theta_D + [theta_D > 0]/Ste (the enthalpy of the wall
 * value; a wall at exactly 0 is taken solid), bounce-back unchanged, and on
 * D2Q5 the Neumann closure of Eq. (17) on H (bb_mode 2).
 * ====================================================================== */
double orc_eebm_theta(double H, double ste)
{
    if (H < 0.0) return H;
    if (H > 1.0 / ste) return H - 1.0 / ste;
    return 0.0;
}

double orc_eebm_enthalpy(double theta, double ste) { return theta + (theta > 0.0 ? 1.0 / ste : 0.0); }

/* equilibrium state of theta0 (Dirichlet nodes at their wall value) */
void orc_eebm_init(const orc_params* p, const double* theta0, double* f)
{
    int q = lat_q(p), n = p->nx * p->ny, x, y, i, ex, ey;
    double w, w0;
    lat_vec(p, 0, &ex, &ey, &w0);
    for (y = 0; y < p->ny; y++)
        for (x = 0; x < p->nx; x++) {
            double th = theta0[y * p->nx + x], td, H;
            if (node_dirichlet(p, x, y, &td, NULL)) th = td;
            H = orc_eebm_enthalpy(th, p->ste);
            for (i = 0; i < q; i++) {
                lat_vec(p, i, &ex, &ey, &w);
                f[i * n + y * p->nx + x] = i == 0 ? H - (1.0 - w0) * th : w * th;
            }
        }
}

/* theta = Theta(M0(f)) */
void orc_eebm_fields(const orc_params* p, const double* f, double* theta, double* H)
{
    int q = lat_q(p), n = p->nx * p->ny, k, i;
    for (k = 0; k < n; k++) {
        double s = 0.0;
        for (i = 0; i < q; i++) s += f[i * n + k];
        if (H) H[k] = s;
        if (theta) theta[k] = orc_eebm_theta(s, p->ste);
    }
}

/* One EEBM step, Algorithm 2, f -> fn; diag (may be NULL): sum of H before
 * and after, and the boundary flux of H (filled distributions minus the
 * post-collision ones that leave the lattice). */
int orc_eebm_step(const orc_params* p, const double* f, double* fn, orc_diag* diag)
{
    const int q = lat_q(p), nx = p->nx, ny = p->ny, n = nx * ny;
    const double omega = 1.0 / p->tau;
    double* Om = (double*)malloc(sizeof(double) * q * n);
    double flux = 0.0, e0 = 0.0, e1 = 0.0;
    int x, y, i, k;
    int ex[ORC_MAXQ], ey[ORC_MAXQ], opp[ORC_MAXQ];
    double w[ORC_MAXQ];
    if (!Om) return -1;
    for (i = 0; i < q; i++) { lat_vec(p, i, &ex[i], &ey[i], &w[i]); opp[i] = lat_opp(p, i); }

    /* moments, equilibrium and collision */
    for (k = 0; k < n; k++) {
        double H = 0.0, th;
        for (i = 0; i < q; i++) H += f[i * n + k];
        e0 += H;
        th = orc_eebm_theta(H, p->ste);
        for (i = 0; i < q; i++) {
            const double feq = i == 0 ? H - (1.0 - w[0]) * th : w[i] * th;
            Om[i * n + k] = f[i * n + k] - (f[i * n + k] - feq) / p->tau;
        }
    }
    (void)omega;
    for (y = 0; y < ny; y++)
        for (x = 0; x < nx; x++)
            for (i = 0; i < q; i++)
                if (!inside(p, x + ex[i], y + ey[i])) flux -= Om[i * n + y * nx + x];

    /* streaming and the closures of the unknown streamed distributions */
    for (y = 0; y < ny; y++)
        for (x = 0; x < nx; x++) {
            double qv[ORC_MAXQ], td;
            int known[ORC_MAXQ], nunk = 0;
            k = y * nx + x;
            for (i = 0; i < q; i++) {
                int sx = x - ex[i], sy = y - ey[i];
                known[i] = inside(p, sx, sy);
                qv[i] = known[i] ? Om[i * n + sy * nx + sx] : 0.0;
                if (!known[i]) nunk++;
            }
            if (nunk > 0) {
                if (node_dirichlet(p, x, y, &td, NULL) || p->bb_mode == 2) {
                    /* Dirichlet: M0 = H(theta_D); Eq. (17): M0 = M0 of the streamed
                     * distributions one node inwards (the diagonal one at a corner) */
                    double rest, wu = 0.0;
                    if (node_dirichlet(p, x, y, &td, NULL)) {
                        rest = orc_eebm_enthalpy(td, p->ste);
                    } else {
                        const int sx = x + (x == 0 ? 1 : (x == nx - 1 ? -1 : 0));
                        const int sy = y + (y == 0 ? 1 : (y == ny - 1 ? -1 : 0));
                        rest = orc_pulled_m0(p, Om, sx, sy);
                    }
                    for (i = 0; i < q; i++) {
                        if (known[i]) rest -= qv[i];
                        else wu += w[i];
                    }
                    for (i = 0; i < q; i++)
                        if (!known[i]) qv[i] = w[i] * rest / wu;
                } else {
                    for (i = 0; i < q; i++)
                        if (!known[i]) {
                            if (p->bb_mode == 0 && known[opp[i]]) qv[i] = qv[opp[i]];
                            else qv[i] = Om[opp[i] * n + k];
                        }
                }
                for (i = 0; i < q; i++)
                    if (!known[i]) flux += qv[i];
            }
            for (i = 0; i < q; i++) fn[i * n + k] = qv[i];
        }
    if (diag) {
        for (k = 0; k < n; k++)
            for (i = 0; i < q; i++) e1 += fn[i * n + k];
        diag->energy_before = e0;
        diag->energy_after = e1;
        diag->flux = flux;
        diag->max_iter = 0;
        diag->failed = 0;
    }
    free(Om);
    return 0;
}

/* nsteps EEBM steps from the equilibrium state of theta0: final f and theta */
int orc_eebm_run(const orc_params* p, const double* theta0, int nsteps, double* f_out, double* theta_out)
{
    const int q = lat_q(p), n = p->nx * p->ny;
    double* a = (double*)malloc(sizeof(double) * q * n);
    double* b = (double*)malloc(sizeof(double) * q * n);
    int s;
    if (!a || !b) { free(a); free(b); return -1; }
    orc_eebm_init(p, theta0, a);
    for (s = 0; s < nsteps; s++) {
        double* t;
        if (orc_eebm_step(p, a, b, NULL) < 0) { free(a); free(b); return -1; }
        t = a; a = b; b = t;
    }
    if (f_out) memcpy(f_out, a, sizeof(double) * q * n);
    if (theta_out) orc_eebm_fields(p, a, theta_out, NULL);
    free(a);
    free(b);
    return 0;
}

/* ======================================================================
 * Implicit liquid fraction based method (ILFBM), Algorithm 1 (Sec. 3.3),
 * the paper's second comparison scheme.  The distributions carry the
 * temperature, theta = M0(f), f_i^eq = w_i theta; a separate field l (the
 * liquid fraction) enters through the source g_i = (w_i/Ste)(l - l~), and l~
 * is found by an inner loop of collision, streaming and the lever rule
 *     l(H) = 0 if H < 0,  Ste H if 0 <= H <= 1/Ste,  1 if H > 1/Ste.
 * One step from (f, l):
 *     theta = M0(f); l^(0) = l; for k = 1, 2, ...:
 *         Omega_i = f_i - (f_i - w_i theta)/tau + (w_i/Ste)(l - l^(k-1))
 *         f^(k)_i(y) = Omega_i(y - e_i), closures on the unknown ones
 *         H^(k) = M0(f^(k)) + l^(k-1)/Ste,   l^(k) = l(H^(k))
 *     until max_y |l^(k) - l^(k-1)| <= tol (or k = maxit: not converged);
 *     f~ = f^(k), l~ = l^(k).
 * Readings (the algorithm names the loop's test but not its form):
 *  - the printed first line of Algorithm 1 ("H <- phi(theta)") is not used:
 *    H is formed in the loop;
 *  - convergence: the largest change of l over the lattice is at most tol
 *    (f^(k) depends on l^(k-1) only through the source, so it settles with l);
 *  - closures on the streamed f: Dirichlet makes M0(f~) = theta_D, the
 *    unknowns sharing the rest by weight; bounce-back as for IREBM; a
 *    Dirichlet node's liquid fraction is that of its wall value, [theta_D > 0];
 *  - initial l = [theta0 > 0] (the phase of the initial temperature).
 * ====================================================================== */
double orc_ilfbm_lever(double H, double ste)
{
    if (H < 0.0) return 0.0;
    if (H > 1.0 / ste) return 1.0;
    return ste * H;
}

void orc_ilfbm_init(const orc_params* p, const double* theta0, double* f, double* ell)
{
    int q = lat_q(p), n = p->nx * p->ny, x, y, i, ex, ey;
    double w;
    for (y = 0; y < p->ny; y++)
        for (x = 0; x < p->nx; x++) {
            double th = theta0[y * p->nx + x], td;
            if (node_dirichlet(p, x, y, &td, NULL)) th = td;
            for (i = 0; i < q; i++) {
                lat_vec(p, i, &ex, &ey, &w);
                f[i * n + y * p->nx + x] = w * th;
            }
            ell[y * p->nx + x] = th > 0.0 ? 1.0 : 0.0;
        }
}

/* sum_x theta + l/Ste with theta = M0(f) */
double orc_ilfbm_energy(const orc_params* p, const double* f, const double* ell)
{
    int q = lat_q(p), n = p->nx * p->ny, k, i;
    double e = 0.0;
    for (k = 0; k < n; k++) {
        double th = 0.0;
        for (i = 0; i < q; i++) th += f[i * n + k];
        e += th + ell[k] / p->ste;
    }
    return e;
}

/* One ILFBM step (f, ell) -> (fn, elln).  Returns 0 when the inner loop
 * converged, 1 when it reached maxit, -1 on allocation failure; *iters gets
 * the number of inner iterations; diag (may be NULL): energies before and
 * after and the boundary flux of the last inner iteration. */
int orc_ilfbm_step(const orc_params* p, const double* f, const double* ell, double* fn, double* elln, double tol,
                   int maxit, int* iters, orc_diag* diag)
{
    const int q = lat_q(p), nx = p->nx, ny = p->ny, n = nx * ny;
    double* theta = (double*)malloc(sizeof(double) * n);
    double* Om = (double*)malloc(sizeof(double) * q * n);
    double* lprev = (double*)malloc(sizeof(double) * n);
    double flux = 0.0;
    int x, y, i, k, it = 0, converged = 0;
    int ex[ORC_MAXQ], ey[ORC_MAXQ], opp[ORC_MAXQ];
    double w[ORC_MAXQ];
    if (!theta || !Om || !lprev) { free(theta); free(Om); free(lprev); return -1; }
    for (i = 0; i < q; i++) { lat_vec(p, i, &ex[i], &ey[i], &w[i]); opp[i] = lat_opp(p, i); }

    /* moments: theta = M0(f); inner loop initialization l^(0) = l */
    orc_theta(p, f, theta);
    memcpy(lprev, ell, sizeof(double) * n);
    while (!converged && it < maxit) {
        double change = 0.0;
        it++;
        /* collision with the source of the current liquid-fraction iterate */
        for (i = 0; i < q; i++)
            for (k = 0; k < n; k++)
                Om[i * n + k] = f[i * n + k] - (f[i * n + k] - w[i] * theta[k]) / p->tau +
                                w[i] / p->ste * (ell[k] - lprev[k]);
        /* streaming and closures */
        flux = 0.0;
        for (y = 0; y < ny; y++)
            for (x = 0; x < nx; x++)
                for (i = 0; i < q; i++)
                    if (!inside(p, x + ex[i], y + ey[i])) flux -= Om[i * n + y * nx + x];
        for (y = 0; y < ny; y++)
            for (x = 0; x < nx; x++) {
                double qv[ORC_MAXQ], td;
                int known[ORC_MAXQ], nunk = 0;
                k = y * nx + x;
                for (i = 0; i < q; i++) {
                    int sx = x - ex[i], sy = y - ey[i];
                    known[i] = inside(p, sx, sy);
                    qv[i] = known[i] ? Om[i * n + sy * nx + sx] : 0.0;
                    if (!known[i]) nunk++;
                }
                if (nunk > 0) {
                    if (node_dirichlet(p, x, y, &td, NULL)) {
                        double rest = td, wu = 0.0;
                        for (i = 0; i < q; i++) {
                            if (known[i]) rest -= qv[i];
                            else wu += w[i];
                        }
                        for (i = 0; i < q; i++)
                            if (!known[i]) qv[i] = w[i] * rest / wu;
                    } else {
                        for (i = 0; i < q; i++)
                            if (!known[i]) {
                                if (p->bb_mode == 0 && known[opp[i]]) qv[i] = qv[opp[i]];
                                else qv[i] = Om[opp[i] * n + k];
                            }
                    }
                    for (i = 0; i < q; i++)
                        if (!known[i]) flux += qv[i];
                }
                for (i = 0; i < q; i++) fn[i * n + k] = qv[i];
            }
        /* enthalpy and lever rule; Dirichlet nodes keep the phase of their wall value */
        for (y = 0; y < ny; y++)
            for (x = 0; x < nx; x++) {
                double m0 = 0.0, td, lk;
                k = y * nx + x;
                for (i = 0; i < q; i++) m0 += fn[i * n + k];
                if (node_dirichlet(p, x, y, &td, NULL)) lk = td > 0.0 ? 1.0 : 0.0;
                else lk = orc_ilfbm_lever(m0 + lprev[k] / p->ste, p->ste);
                if (fabs(lk - lprev[k]) > change) change = fabs(lk - lprev[k]);
                elln[k] = lk;
            }
        converged = change <= tol;
        memcpy(lprev, elln, sizeof(double) * n);
    }
    if (iters) *iters = it;
    if (diag) {
        diag->energy_before = orc_ilfbm_energy(p, f, ell);
        diag->energy_after = orc_ilfbm_energy(p, fn, elln);
        diag->flux = flux;
        diag->max_iter = it;
        diag->failed = !converged;
    }
    free(theta);
    free(Om);
    free(lprev);
    return converged ? 0 : 1;
}

/* nsteps ILFBM steps from (w_i theta0, [theta0 > 0]): final f, l and theta;
 * the number of steps whose inner loop did not converge, -1 on allocation
 * failure; *max_iters the largest inner iteration count */
int orc_ilfbm_run(const orc_params* p, const double* theta0, int nsteps, double tol, int maxit, double* f_out,
                  double* ell_out, double* theta_out, int* max_iters)
{
    const int q = lat_q(p), n = p->nx * p->ny;
    double* a = (double*)malloc(sizeof(double) * q * n);
    double* b = (double*)malloc(sizeof(double) * q * n);
    double* la = (double*)malloc(sizeof(double) * n);
    double* lb = (double*)malloc(sizeof(double) * n);
    int s, failed = 0, mx = 0;
    if (!a || !b || !la || !lb) { free(a); free(b); free(la); free(lb); return -1; }
    orc_ilfbm_init(p, theta0, a, la);
    for (s = 0; s < nsteps; s++) {
        double* t;
        int it = 0, r = orc_ilfbm_step(p, a, la, b, lb, tol, maxit, &it, NULL);
        if (r < 0) { failed = -1; break; }
        failed += r;
        if (it > mx) mx = it;
        t = a; a = b; b = t;
        t = la; la = lb; lb = t;
    }
    if (f_out) memcpy(f_out, a, sizeof(double) * q * n);
    if (ell_out) memcpy(ell_out, la, sizeof(double) * n);
    if (theta_out) orc_theta(p, a, theta_out);
    if (max_iters) *max_iters = mx;
    free(a);
    free(b);
    free(la);
    free(lb);
    return failed;
}
