/*
 * FP64 CPU oracle for the sparse lattice-Boltzmann (LBGK) collide-and-stream
 * path.  TEST INFRASTRUCTURE ONLY: it is called by the tests, by the smoke
 * check and by the timed CPU baseline of the benchmark, never by the product
 * library, and it shares no code, header, table or helper with it.
 *
 * What the paper fixes (HemeLB, arXiv 1906.11925):
 *   Section 2: the fluid is a lattice of sparse fluid sites, each holding a
 *     single-particle distribution over a finite set of lattice vectors; a
 *     time step is a collision followed by propagation to the neighbouring
 *     site along each vector; the lattice is D3Q19 (Fig. 1).
 *   Section 4: walls use simple bounce-back.
 * Everything else is a stated reading (the paper gives no equation):
 *   - single-relaxation-time (LBGK) collision toward the compressible
 *     second-order equilibrium
 *       feq_i = w_i rho (1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 |u|^2),
 *   - D3Q15 as a second velocity set (textbook weights 2/9, 1/9, 1/72),
 *   - halfway bounce-back: a population that would leave x through a wall
 *     link i comes back to x as population opp(i) at the next step,
 *   - density (pressure) iolets: a link from x into iolet k returns the
 *     equilibrium population feq_opp(i)(rho_k(t), u(x,t)) with the iolet's
 *     prescribed density and the site's own velocity,
 *     rho_k(t) = mean_k + amp_k sin(2 pi t / period_k + phase_k),
 *   - wall shear stress from the non-equilibrium stress
 *       sigma = -(1 - 1/(2 tau)) sum_i (f_i - feq_i) c_i c_i,
 *     traction t = sigma n, WSS = |t - (n.t) n|, with the wall normal
 *     n = -normalize(sum of c_i over the site's wall links).
 *   Section 3.3.2: the visualisation renders a volume by ray marching with a
 *     transfer-function look-up table; orc_render states its readings.
 *
 * Direction order: 0 is the rest vector; after it, opposite vectors are
 * adjacent (opp(i) = i + 1 for odd i, i - 1 for even i > 0).
 *
 * Layouts: populations f[q][n] (direction-major), caller site order;
 * nbr[q][n] int32 (index of the site x + c_i, -1 if none); link[q][n] uint8
 * (0 fluid, 1 wall, 2 + k iolet k); u[n][3].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- lattices */

static const int E15[15][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}};

static const int E19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

typedef struct {
    int q;
    int e[19][3];
    double w[19];
    int opp[19];
} lattice_t;

static int get_lattice(int q, lattice_t *L) {
    if (q != 15 && q != 19) return -1;
    L->q = q;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) L->e[i][a] = (q == 15) ? E15[i][a] : E19[i][a];
        int len2 = L->e[i][0] * L->e[i][0] + L->e[i][1] * L->e[i][1] + L->e[i][2] * L->e[i][2];
        if (q == 15) L->w[i] = len2 == 0 ? 2.0 / 9.0 : (len2 == 1 ? 1.0 / 9.0 : 1.0 / 72.0);
        else         L->w[i] = len2 == 0 ? 1.0 / 3.0 : (len2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        L->opp[i] = (i == 0) ? 0 : ((i & 1) ? i + 1 : i - 1);
    }
    return 0;
}

/* Export of the velocity set, so that tests can check it against the
 * isotropy conditions that define it. */
int orc_lattice(int q, int32_t *e, double *w, int32_t *opp) {
    lattice_t L;
    if (get_lattice(q, &L)) return -1;
    for (int i = 0; i < q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
        w[i] = L.w[i];
        opp[i] = L.opp[i];
    }
    return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int nt) {
#ifdef _OPENMP
    if (nt > 0) omp_set_num_threads(nt);
#else
    (void)nt;
#endif
}

/* ------------------------------------------------------------- equilibrium */

static void equilibrium(const lattice_t *L, double rho, const double u[3], double *feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->q; ++i) {
        double cu = L->e[i][0] * u[0] + L->e[i][1] * u[1] + L->e[i][2] * u[2];
        feq[i] = L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

int orc_equilibrium(int q, double rho, const double *u, double *feq) {
    lattice_t L;
    if (get_lattice(q, &L)) return -1;
    equilibrium(&L, rho, u, feq);
    return 0;
}

/* density and velocity moments of one site's populations */
static void moments(const lattice_t *L, const double *g, double *rho, double u[3]) {
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->q; ++i) {
        r += g[i];
        for (int a = 0; a < 3; ++a) j[a] += L->e[i][a] * g[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = j[a] / r;
}

/* prescribed iolet density at the start of step t */
static double iolet_rho(int k, int64_t t, const double *mean, const double *amp,
                        const double *period, const double *phase) {
    double r = mean[k];
    if (period[k] != 0.0 && amp[k] != 0.0)
        r += amp[k] * sin(2.0 * M_PI * (double)t / period[k] + phase[k]);
    return r;
}

/* ---------------------------------------------------------------- links */

#define KB 21
#define KOFF (1LL << 20)

static int64_t vkey(int64_t x, int64_t y, int64_t z) {
    return ((z + KOFF) << (2 * KB)) | ((y + KOFF) << KB) | (x + KOFF);
}

typedef struct {
    int64_t key;
    int64_t val;
} kv_t;

static int kv_cmp(const void *a, const void *b) {
    int64_t ka = ((const kv_t *)a)->key, kb = ((const kv_t *)b)->key;
    return (ka > kb) - (ka < kb);
}

/* binary search of a sorted key array; -1 if absent */
static int64_t kv_find(const kv_t *t, int64_t n, int64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (t[mid].key < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < n && t[lo].key == key) ? t[lo].val : -1;
}

/*
 * Neighbour-link table (Section 2: each fluid site propagates to the
 * neighbouring site along every lattice vector).  For site x and direction i
 * the target voxel is y = x + c_i (wrapped per axis where periodic[a] > 0).
 * nbr[i][x] = index of y if y is a fluid site, else -1.
 * link[i][x] = 0 if y is fluid; 2 + k if y is an iolet-k voxel; else 1 (wall).
 * Returns 0, or -1 on a bad lattice, -2 on duplicate fluid voxels, -3 on an
 * iolet id outside [0, 253], -4 on a coordinate outside the key range.
 */
int orc_links_build(int q, int64_t n, const int32_t *xyz, int64_t n_io,
                    const int32_t *io_xyz, const int32_t *io_id,
                    const int32_t *periodic, int32_t *nbr, uint8_t *link) {
    lattice_t L;
    if (get_lattice(q, &L)) return -1;
    for (int64_t m = 0; m < n_io; ++m)
        if (io_id[m] < 0 || io_id[m] > 253) return -3;
    for (int64_t x = 0; x < n; ++x)
        for (int a = 0; a < 3; ++a)
            if (xyz[3 * x + a] < -(1 << 19) || xyz[3 * x + a] >= (1 << 19)) return -4;
    kv_t *fl = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
    kv_t *io = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n_io > 0 ? n_io : 1));
    if (!fl || !io) { free(fl); free(io); return -5; }
    for (int64_t x = 0; x < n; ++x) {
        fl[x].key = vkey(xyz[3 * x], xyz[3 * x + 1], xyz[3 * x + 2]);
        fl[x].val = x;
    }
    for (int64_t m = 0; m < n_io; ++m) {
        io[m].key = vkey(io_xyz[3 * m], io_xyz[3 * m + 1], io_xyz[3 * m + 2]);
        io[m].val = io_id[m];
    }
    qsort(fl, (size_t)n, sizeof(kv_t), kv_cmp);
    qsort(io, (size_t)n_io, sizeof(kv_t), kv_cmp);
    for (int64_t x = 1; x < n; ++x)
        if (fl[x].key == fl[x - 1].key) { free(fl); free(io); return -2; }
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < n; ++x) {
        for (int i = 0; i < q; ++i) {
            int64_t y[3];
            for (int a = 0; a < 3; ++a) {
                y[a] = (int64_t)xyz[3 * x + a] + L.e[i][a];
                if (periodic && periodic[a] > 0) y[a] = ((y[a] % periodic[a]) + periodic[a]) % periodic[a];
            }
            int64_t key = vkey(y[0], y[1], y[2]);
            int64_t j = kv_find(fl, n, key);
            if (j >= 0) {
                nbr[(int64_t)i * n + x] = (int32_t)j;
                link[(int64_t)i * n + x] = 0;
            } else {
                int64_t k = kv_find(io, n_io, key);
                nbr[(int64_t)i * n + x] = -1;
                link[(int64_t)i * n + x] = (uint8_t)(k >= 0 ? 2 + k : 1);
            }
        }
    }
    free(fl);
    free(io);
    return 0;
}

/* ------------------------------------------------------------------ step */

/*
 * One time step t -> t+1 in push form (Section 2: collision, then
 * propagation).  f and fout are [q][n]; every slot of fout is written
 * exactly once for a consistent (symmetric) link table.
 *   1. rho = sum_i f_i, u = sum_i c_i f_i / rho, feq_i(rho, u);
 *   2. post-collision f*_i = f_i - (f_i - feq_i) / tau;
 *   3. for each i: fluid link -> fout_i(nbr) = f*_i;
 *                  wall link  -> fout_opp(i)(x) = f*_i   (halfway bounce-back);
 *                  iolet k    -> fout_opp(i)(x) = feq_opp(i)(rho_k(t), u)
 *                                (density iolet), or
 *                  iolet k    -> fout_opp(i)(x) = f*_i - 6 w_i rho (c_i . u_b)
 *                                (velocity iolet: bounce-back from a boundary
 *                                moving with u_b = weight[x] U_k(t) n_k, Ladd's
 *                                moving-wall rule with c_s^2 = 1/3; the paper
 *                                drives its inlet this way, Sections 2 and 3.2,
 *                                Table I).
 * The schedule mean/amp/period/phase gives rho_k(t) for a density iolet and
 * the velocity magnitude U_k(t) for a velocity iolet (io_kind[k] = 1, unit
 * inward normal io_normal[3k..3k+2]); weight may be NULL (all 1).
 *
 * Interpolated walls (the paper's BFL wall boundary, Section 3.2: Bouzidi,
 * Firdaouss & Lallemand, Phys. Fluids 13, 3452 (2001)): wall_q[i][x] in
 * (0, 1] is the fraction of the link from x along c_i that lies in the fluid
 * (1/2: the wall half-way, the plain bounce-back above).  With xb = x - c_i:
 *   q <  1/2, xb fluid: fout_opp(i)(x) = 2q f*_i(x) + (1 - 2q) f*_i(xb),
 *   q >= 1/2:           fout_opp(i)(x) = f*_i(x) / (2q) + (1 - 1/(2q)) f*_opp(i)(x),
 *   q <  1/2, xb not fluid: the plain bounce-back (a reading: the
 *   interpolation has no second fluid point).
 * wall_q NULL: every wall is half-way.
 */
/* Post-collision population i at site x (the collision written once more,
 * for the BFL upstream point). */
static double post_collision(const lattice_t *L, const double *f, int64_t n, int64_t x, int i,
                             double tau) {
    double h[19], he[19], r, v[3];
    for (int j = 0; j < L->q; ++j) h[j] = f[(int64_t)j * n + x];
    moments(L, h, &r, v);
    equilibrium(L, r, v, he);
    return h[i] - (h[i] - he[i]) / tau;
}

int orc_step_bc(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
                int n_io, const double *rho_mean, const double *amp,
                const double *period, const double *phase, const int32_t *io_kind,
                const double *io_normal, const double *weight, const double *wall_q,
                int64_t t, const double *f, double *fout) {
    lattice_t L;
    if (get_lattice(q, &L)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < n; ++x) {
        double g[19], feq[19], rho, u[3];
        for (int i = 0; i < q; ++i) g[i] = f[(int64_t)i * n + x];
        moments(&L, g, &rho, u);
        equilibrium(&L, rho, u, feq);
        double fsa[19];
        for (int i = 0; i < q; ++i) fsa[i] = g[i] - (g[i] - feq[i]) / tau;
        for (int i = 0; i < q; ++i) {
            double fs = fsa[i];
            int lk = link[(int64_t)i * n + x];
            double qw = (lk == 1 && wall_q) ? wall_q[(int64_t)i * n + x] : 0.5;
            if (lk == 0) {
                fout[(int64_t)i * n + nbr[(int64_t)i * n + x]] = fs;
            } else if (lk == 1 && qw == 0.5) {
                fout[(int64_t)L.opp[i] * n + x] = fs;
            } else if (lk == 1 && qw < 0.5) {
                int64_t ob = (int64_t)L.opp[i] * n + x;  /* the link toward xb = x - c_i */
                double val = fs;
                if (link[ob] == 0) val = 2.0 * qw * fs + (1.0 - 2.0 * qw) * post_collision(&L, f, n, nbr[ob], i, tau);
                fout[(int64_t)L.opp[i] * n + x] = val;
            } else if (lk == 1) {
                fout[(int64_t)L.opp[i] * n + x] = fs / (2.0 * qw) + (1.0 - 1.0 / (2.0 * qw)) * fsa[L.opp[i]];
            } else if (io_kind && io_kind[lk - 2] == 1) {
                int k = lk - 2;
                double U = iolet_rho(k, t, rho_mean, amp, period, phase);
                double wx = weight ? weight[x] : 1.0;
                double cub = 0.0;
                for (int a = 0; a < 3; ++a) cub += L.e[i][a] * wx * U * io_normal[3 * k + a];
                fout[(int64_t)L.opp[i] * n + x] = fs - 6.0 * L.w[i] * rho * cub;
            } else {
                int k = lk - 2;
                double feq_k[19];
                double rk = iolet_rho(k, t, rho_mean, amp, period, phase);
                equilibrium(&L, rk, u, feq_k);
                fout[(int64_t)L.opp[i] * n + x] = feq_k[L.opp[i]];
            }
        }
    }
    (void)n_io;
    return 0;
}

int orc_step(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
             int n_io, const double *rho_mean, const double *amp,
             const double *period, const double *phase, int64_t t,
             const double *f, double *fout) {
    return orc_step_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, NULL, NULL, NULL,
                       NULL, t, f, fout);
}

/* nsteps steps from time t0; f holds the state on entry and on exit;
 * work is scratch of the same size. */
int orc_run_bc(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
               int n_io, const double *rho_mean, const double *amp, const double *period,
               const double *phase, const int32_t *io_kind, const double *io_normal,
               const double *weight, const double *wall_q, int64_t t0, int64_t nsteps, double *f,
               double *work) {
    double *a = f, *b = work;
    for (int64_t s = 0; s < nsteps; ++s) {
        int r = orc_step_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, io_kind,
                            io_normal, weight, wall_q, t0 + s, a, b);
        if (r) return r;
        double *tmp = a; a = b; b = tmp;
    }
    if (a != f) memcpy(f, a, sizeof(double) * (size_t)q * (size_t)n);
    return 0;
}

int orc_run(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
            int n_io, const double *rho_mean, const double *amp, const double *period,
            const double *phase, int64_t t0, int64_t nsteps, double *f, double *work) {
    return orc_run_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, NULL, NULL, NULL,
                      NULL, t0, nsteps, f, work);
}

/* --------------------------------------------------------------- macros */

/*
 * Density, velocity and wall shear stress of the state f (pre-collision
 * populations at time t).  u is [n][3].  Sites without wall links, or whose
 * wall-link vectors sum to zero, get wss = 0.
 */
int orc_macros(int q, int64_t n, const uint8_t *link, double tau, const double *f,
               double *rho_out, double *u_out, double *wss_out) {
    lattice_t L;
    if (get_lattice(q, &L)) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < n; ++x) {
        double g[19], feq[19], rho, u[3];
        for (int i = 0; i < q; ++i) g[i] = f[(int64_t)i * n + x];
        moments(&L, g, &rho, u);
        if (rho_out) rho_out[x] = rho;
        if (u_out) for (int a = 0; a < 3; ++a) u_out[3 * x + a] = u[a];
        if (!wss_out) continue;
        double s[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < q; ++i)
            if (link[(int64_t)i * n + x] == 1)
                for (int a = 0; a < 3; ++a) s[a] += L.e[i][a];
        double sn = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
        if (sn == 0.0) { wss_out[x] = 0.0; continue; }
        double nv[3] = {-s[0] / sn, -s[1] / sn, -s[2] / sn};
        equilibrium(&L, rho, u, feq);
        double pi[3][3] = {{0}};
        for (int i = 0; i < q; ++i) {
            double d = g[i] - feq[i];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) pi[a][b] += d * L.e[i][a] * L.e[i][b];
        }
        double coef = -(1.0 - 1.0 / (2.0 * tau));
        double tr[3];
        for (int a = 0; a < 3; ++a) {
            tr[a] = 0.0;
            for (int b = 0; b < 3; ++b) tr[a] += coef * pi[a][b] * nv[b];
        }
        double tn = tr[0] * nv[0] + tr[1] * nv[1] + tr[2] * nv[2];
        double w2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double c = tr[a] - tn * nv[a];
            w2 += c * c;
        }
        wss_out[x] = sqrt(w2);
    }
    return 0;
}

/* total mass sum_x sum_i f_i(x), summed in site order */
double orc_mass(int q, int64_t n, const double *f) {
    double m = 0.0;
    for (int64_t x = 0; x < n; ++x)
        for (int i = 0; i < q; ++i) m += f[(int64_t)i * n + x];
    return m;
}

/* ---------------------------------------------------------------- adjoint
 *
 * Discrete adjoint of orc_step (reverse mode, float64).  With the step
 * written as f(t+1) = F_t(f(t); tau, iolet schedule) and an objective
 * J = scale * sum_{t in window} sum_x m_x q(x, t), the adjoint variable
 * lam(t) = dJ/df(t) obeys lam(t) = (dF_t/df)^T lam(t+1) + dj_t/df(t).
 *
 * Per site x, with lam*_i the adjoint of the post-collision population:
 *   fluid link i: lam*_i = lam_i(x + c_i, t+1);  wall link i: lam*_i =
 *   lam_opp(i)(x, t+1);  iolet link i: lam*_i = 0 (f*_i leaves the domain)
 *   and the returning population feq_opp(i)(rho_k(t), u) feeds back into u
 *   and rho_k(t).
 * Collision f*_i = (1 - w) f_i + w feq_i(rho, u), w = 1/tau, with
 *   d feq_i / d rho = feq_i / rho,
 *   d feq_i / d u   = w_i rho (3 c_i + 9 (c_i.u) c_i - 3 u),
 *   d rho / d f_j = 1,  d u / d f_j = (c_j - u) / rho,
 * gives lam_j(x, t) = (1 - w) lam*_j + w (a + b.(c_j - u)/rho)
 *                     + g.(c_j - u)/rho,
 *   a = sum_i lam*_i feq_i / rho,  b = sum_i lam*_i d feq_i / d u,
 *   g = sum over iolet links i of lam_opp(i)(x, t+1) d feq_opp(i) / d u.
 * Parameter derivatives accumulated here:
 *   dJ/dtau      += sum_i lam*_i (f_i - feq_i) / tau^2,
 *   dJ/drho_k(t) += sum over iolet-k links of lam_opp(i)(x, t+1) feq_opp(i)/rho_k,
 * and, through rho_k(t) = mean + amp sin(2 pi t / period + phase), the
 * derivatives with respect to mean, amp and phase of every iolet.
 */

static void dfeq_du(const lattice_t *L, int i, double rho, const double u[3], double out[3]) {
    double cu = L->e[i][0] * u[0] + L->e[i][1] * u[1] + L->e[i][2] * u[2];
    for (int a = 0; a < 3; ++a) out[a] = L->w[i] * rho * (3.0 * L->e[i][a] + 9.0 * cu * L->e[i][a] - 3.0 * u[a]);
}

/* The adjoint of orc_step_bc, with velocity iolets and interpolated walls.
 * Every outgoing population f*_i(x) enters the next state through its link
 * (see orc_step_bc); lam*_i(x) collects lam of every population it feeds,
 * with the same weights:
 *   fluid link:             lam*_i(x)    += lam_i(x + c_i)
 *   half-way wall:          lam*_i(x)    += lam_opp(i)(x)
 *   BFL wall, q < 1/2, xb = x - c_i fluid:
 *                           lam*_i(x)    += 2q lam_opp(i)(x),
 *                           lam*_i(xb)   += (1 - 2q) lam_opp(i)(x)
 *   BFL wall, q >= 1/2:     lam*_i(x)    += lam_opp(i)(x) / (2q),
 *                           lam*_opp(i)(x) += (1 - 1/(2q)) lam_opp(i)(x)
 *   velocity iolet k:       lam*_i(x)    += lam_opp(i)(x), and the moving-wall
 *     term -6 w_i rho c_i.u_b (u_b = weight(x) U_k(t) n_k) feeds back through
 *     rho: every lam_j(x) gains -6 w_i (c_i.u_b) lam_opp(i)(x), and
 *     dJ/dU_k(t) gains -6 w_i rho weight(x) (c_i.n_k) lam_opp(i)(x);
 *   density iolet:          as in orc_adjoint_step.
 * Because the BFL upstream term adds to another site, all lam* are formed
 * first (a pass over the sites), then each site's collision is reversed. */
static void chain_schedule(int k, int64_t t, const double *amp, const double *period,
                           const double *phase, double d, double *dmean, double *damp, double *dphase) {
    dmean[k] += d;
    if (period[k] != 0.0 && amp[k] != 0.0) {
        double arg = 2.0 * M_PI * (double)t / period[k] + phase[k];
        damp[k] += d * sin(arg);
        dphase[k] += d * amp[k] * cos(arg);
    } else if (period[k] != 0.0) {
        damp[k] += d * sin(2.0 * M_PI * (double)t / period[k] + phase[k]);
    }
}

int orc_adjoint_step_bc(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
                        int n_io, const double *rho_mean, const double *amp, const double *period,
                        const double *phase, const int32_t *io_kind, const double *io_normal,
                        const double *weight, const double *wall_q, int64_t t, const double *f,
                        const double *lam_next, double *lam, double *dtau, double *dmean,
                        double *damp, double *dphase) {
    lattice_t L;
    if (get_lattice(q, &L)) return -1;
    const double om = 1.0 / tau;
    const size_t sz = (size_t)q * (size_t)n;
    double *ls = (double *)calloc(sz ? sz : 1, sizeof(double));    /* lam*[i][x] */
    double *gu = (double *)calloc(n ? 3 * (size_t)n : 1, sizeof(double)); /* density-iolet term */
    double *gv = (double *)calloc(n ? (size_t)n : 1, sizeof(double));     /* velocity-iolet term */
    if (!ls || !gu || !gv) { free(ls); free(gu); free(gv); return -5; }
    for (int64_t x = 0; x < n; ++x) {
        double g[19], rho, u[3];
        for (int i = 0; i < q; ++i) g[i] = f[(int64_t)i * n + x];
        moments(&L, g, &rho, u);
        for (int i = 0; i < q; ++i) {
            const int64_t o = (int64_t)L.opp[i] * n + x;  /* slot of population opp(i) at x */
            const int lk = link[(int64_t)i * n + x];
            if (lk == 0) {
                ls[(int64_t)i * n + x] += lam_next[(int64_t)i * n + nbr[(int64_t)i * n + x]];
            } else if (lk == 1) {
                const double qw = wall_q ? wall_q[(int64_t)i * n + x] : 0.5;
                const double lo = lam_next[o];
                if (qw == 0.5) {
                    ls[(int64_t)i * n + x] += lo;
                } else if (qw < 0.5) {
                    if (link[o] == 0) {
                        ls[(int64_t)i * n + x] += 2.0 * qw * lo;
                        ls[(int64_t)i * n + nbr[o]] += (1.0 - 2.0 * qw) * lo;
                    } else {
                        ls[(int64_t)i * n + x] += lo;
                    }
                } else {
                    ls[(int64_t)i * n + x] += lo / (2.0 * qw);
                    ls[o] += (1.0 - 1.0 / (2.0 * qw)) * lo;
                }
            } else if (io_kind && io_kind[lk - 2] == 1) {
                const int k = lk - 2;
                const double lo = lam_next[o];
                const double U = iolet_rho(k, t, rho_mean, amp, period, phase);
                const double wx = weight ? weight[x] : 1.0;
                double cn = 0.0;
                for (int a = 0; a < 3; ++a) cn += L.e[i][a] * io_normal[3 * k + a];
                ls[(int64_t)i * n + x] += lo;
                gv[x] += -6.0 * L.w[i] * wx * U * cn * lo;
                chain_schedule(k, t, amp, period, phase, -6.0 * L.w[i] * rho * wx * cn * lo, dmean, damp, dphase);
            } else {
                const int k = lk - 2, oi = L.opp[i];
                const double lo = lam_next[o];
                const double rk = iolet_rho(k, t, rho_mean, amp, period, phase);
                double feq_k[19], d[3];
                equilibrium(&L, rk, u, feq_k);
                dfeq_du(&L, oi, rk, u, d);
                for (int a = 0; a < 3; ++a) gu[3 * x + a] += lo * d[a];
                chain_schedule(k, t, amp, period, phase, lo * feq_k[oi] / rk, dmean, damp, dphase);
            }
        }
    }
    double acc_tau = 0.0;
    for (int64_t x = 0; x < n; ++x) {
        double g[19], feq[19], rho, u[3];
        for (int i = 0; i < q; ++i) g[i] = f[(int64_t)i * n + x];
        moments(&L, g, &rho, u);
        equilibrium(&L, rho, u, feq);
        double a = 0.0, b[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < q; ++i) {
            const double li = ls[(int64_t)i * n + x];
            double d[3];
            a += li * feq[i] / rho;
            dfeq_du(&L, i, rho, u, d);
            for (int c = 0; c < 3; ++c) b[c] += li * d[c];
            acc_tau += li * (g[i] - feq[i]) / (tau * tau);
        }
        for (int j = 0; j < q; ++j) {
            double s = a, h = 0.0;
            for (int c = 0; c < 3; ++c) {
                double dj = (L.e[j][c] - u[c]) / rho;
                s += b[c] * dj;
                h += gu[3 * x + c] * dj;
            }
            lam[(int64_t)j * n + x] = (1.0 - om) * ls[(int64_t)j * n + x] + om * s + h + gv[x];
        }
    }
    *dtau += acc_tau;
    free(ls);
    free(gu);
    free(gv);
    (void)n_io;
    return 0;
}

int orc_adjoint_step(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
                     int n_io, const double *rho_mean, const double *amp, const double *period,
                     const double *phase, int64_t t, const double *f, const double *lam_next,
                     double *lam, double *dtau, double *dmean, double *damp, double *dphase) {
    return orc_adjoint_step_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, NULL, NULL, NULL,
                               NULL, t, f, lam_next, lam, dtau, dmean, damp, dphase);
}

/* Objective terms.  kind 0: wall shear stress (as orc_macros), kind 1:
 * density.  q(x) is weighted by m[x]. */
enum { ORC_OBJ_WSS = 0, ORC_OBJ_DENSITY = 1 };

/* wall normal of site x (unit, from its wall links); returns 0 if none */
static int wall_normal(const lattice_t *L, int64_t n, const uint8_t *link, int64_t x, double nv[3]) {
    double s[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->q; ++i)
        if (link[(int64_t)i * n + x] == 1)
            for (int a = 0; a < 3; ++a) s[a] += L->e[i][a];
    double sn = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (sn == 0.0) return 0;
    for (int a = 0; a < 3; ++a) nv[a] = -s[a] / sn;
    return 1;
}

/* sum_x m_x q(x) of the state f; optional explicit d/dtau and d/df (both
 * multiplied by scale and added to *dtau and lam) */
double orc_objective(int q, int64_t n, const uint8_t *link, double tau, int kind,
                     const double *m, const double *f, double scale, double *lam, double *dtau) {
    lattice_t L;
    if (get_lattice(q, &L)) return NAN;
    double J = 0.0, jt = 0.0;
    /* without a gradient the site loop is independent: sum it in parallel */
#pragma omp parallel for schedule(static) reduction(+ : J, jt) if (lam == NULL)
    for (int64_t x = 0; x < n; ++x) {
        if (m[x] == 0.0) continue;
        double g[19], feq[19], rho, u[3];
        for (int i = 0; i < q; ++i) g[i] = f[(int64_t)i * n + x];
        moments(&L, g, &rho, u);
        if (kind == ORC_OBJ_DENSITY) {
            J += m[x] * rho;
            if (lam)
                for (int j = 0; j < q; ++j) lam[(int64_t)j * n + x] += scale * m[x];
            continue;
        }
        double nv[3];
        if (!wall_normal(&L, n, link, x, nv)) continue;
        equilibrium(&L, rho, u, feq);
        double pi[3][3] = {{0}};
        for (int i = 0; i < q; ++i)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) pi[a][b] += (g[i] - feq[i]) * L.e[i][a] * L.e[i][b];
        double coef = -(1.0 - 1.0 / (2.0 * tau));
        double tr[3], tn = 0.0, v[3], w2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            tr[a] = 0.0;
            for (int b = 0; b < 3; ++b) tr[a] += coef * pi[a][b] * nv[b];
            tn += tr[a] * nv[a];
        }
        for (int a = 0; a < 3; ++a) {
            v[a] = tr[a] - tn * nv[a];
            w2 += v[a] * v[a];
        }
        double wss = sqrt(w2);
        J += m[x] * wss;
        if (wss == 0.0) continue;
        /* explicit tau dependence of the factor (1 - 1/(2 tau)) */
        jt += m[x] * wss * (1.0 / (2.0 * tau * tau)) / (1.0 - 1.0 / (2.0 * tau));
        if (!lam) continue;
        /* d wss / d f_j = coef [M_j - (A + B.(c_j - u)/rho)],
         * M_i = (c_i.vh)(c_i.n), A = sum M_i feq_i/rho, B = sum M_i dfeq_i/du */
        double vh[3] = {v[0] / wss, v[1] / wss, v[2] / wss};
        double M[19], A = 0.0, B[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < q; ++i) {
            double cv = L.e[i][0] * vh[0] + L.e[i][1] * vh[1] + L.e[i][2] * vh[2];
            double cn = L.e[i][0] * nv[0] + L.e[i][1] * nv[1] + L.e[i][2] * nv[2];
            double d[3];
            M[i] = cv * cn;
            A += M[i] * feq[i] / rho;
            dfeq_du(&L, i, rho, u, d);
            for (int c = 0; c < 3; ++c) B[c] += M[i] * d[c];
        }
        for (int j = 0; j < q; ++j) {
            double s = A;
            for (int c = 0; c < 3; ++c) s += B[c] * (L.e[j][c] - u[c]) / rho;
            lam[(int64_t)j * n + x] += scale * m[x] * coef * (M[j] - s);
        }
    }
    if (dtau) *dtau += scale * jt;
    return J;
}

/*
 * Objective and its gradient by storing every state (small inputs only).
 * Runs nsteps steps from f0 at time t0; J = scale * sum over the states
 * f(t), t0 <= t <= t0 + nsteps, with t_begin <= t < t_end, of sum_x m_x q(x,t).
 * Outputs: J, dJ/dtau, per-iolet dJ/dmean, dJ/damp, dJ/dphase ([n_io] each,
 * overwritten) and, if lam0 != NULL, dJ/df(t0) ([q][n]).
 */
/* Objective and gradient over a run, with velocity iolets and interpolated
 * walls (io_kind, io_normal, weight, wall_q as in orc_step_bc; all NULL: the
 * plain step). */
int orc_gradient_bc(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
                    int n_io, const double *rho_mean, const double *amp, const double *period,
                    const double *phase, const int32_t *io_kind, const double *io_normal,
                    const double *weight, const double *wall_q, int64_t t0, int64_t nsteps,
                    const double *f0, int kind, const double *m, int64_t t_begin, int64_t t_end,
                    double scale, double *J_out, double *dtau_out, double *dmean, double *damp,
                    double *dphase, double *lam0) {
    const size_t sz = (size_t)q * (size_t)n;
    double *states = (double *)malloc(sizeof(double) * sz * (size_t)(nsteps + 1));
    double *la = (double *)malloc(sizeof(double) * (sz ? sz : 1));
    double *lb = (double *)malloc(sizeof(double) * (sz ? sz : 1));
    if (!states || !la || !lb) { free(states); free(la); free(lb); return -5; }
    memcpy(states, f0, sizeof(double) * sz);
    for (int64_t s = 0; s < nsteps; ++s) {
        int r = orc_step_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, io_kind, io_normal,
                            weight, wall_q, t0 + s, states + sz * (size_t)s, states + sz * (size_t)(s + 1));
        if (r) { free(states); free(la); free(lb); return r; }
    }
    double J = 0.0, dtau = 0.0;
    for (int k = 0; k < n_io; ++k) dmean[k] = damp[k] = dphase[k] = 0.0;
    /* lam(t0 + nsteps) = dj/df at the last state */
    memset(lb, 0, sizeof(double) * sz);
    int64_t T = t0 + nsteps;
    if (T >= t_begin && T < t_end)
        J += orc_objective(q, n, link, tau, kind, m, states + sz * (size_t)nsteps, scale, lb, &dtau);
    for (int64_t s = nsteps - 1; s >= 0; --s) {
        int64_t t = t0 + s;
        int r = orc_adjoint_step_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, io_kind,
                                    io_normal, weight, wall_q, t, states + sz * (size_t)s, lb, la, &dtau,
                                    dmean, damp, dphase);
        if (r) { free(states); free(la); free(lb); return r; }
        if (t >= t_begin && t < t_end)
            J += orc_objective(q, n, link, tau, kind, m, states + sz * (size_t)s, scale, la, &dtau);
        double *tmp = la; la = lb; lb = tmp;
    }
    *J_out = scale * J;
    *dtau_out = dtau;
    if (lam0) memcpy(lam0, lb, sizeof(double) * sz);
    free(states);
    free(la);
    free(lb);
    return 0;
}

int orc_gradient(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
                 int n_io, const double *rho_mean, const double *amp, const double *period,
                 const double *phase, int64_t t0, int64_t nsteps, const double *f0, int kind,
                 const double *m, int64_t t_begin, int64_t t_end, double scale, double *J_out,
                 double *dtau_out, double *dmean, double *damp, double *dphase, double *lam0) {
    return orc_gradient_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, NULL, NULL, NULL, NULL,
                           t0, nsteps, f0, kind, m, t_begin, t_end, scale, J_out, dtau_out, dmean, damp,
                           dphase, lam0);
}

double orc_objective_run_bc(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
                            int n_io, const double *rho_mean, const double *amp, const double *period,
                            const double *phase, const int32_t *io_kind, const double *io_normal,
                            const double *weight, const double *wall_q, int64_t t0, int64_t nsteps,
                            const double *f0, int kind, const double *m, int64_t t_begin, int64_t t_end,
                            double scale) {
    const size_t sz = (size_t)q * (size_t)n;
    double *a = (double *)malloc(sizeof(double) * (sz ? sz : 1));
    double *b = (double *)malloc(sizeof(double) * (sz ? sz : 1));
    if (!a || !b) { free(a); free(b); return NAN; }
    memcpy(a, f0, sizeof(double) * sz);
    double J = 0.0;
    for (int64_t s = 0; s <= nsteps; ++s) {
        int64_t t = t0 + s;
        if (t >= t_begin && t < t_end) J += orc_objective(q, n, link, tau, kind, m, a, scale, NULL, NULL);
        if (s < nsteps) {
            orc_step_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, io_kind, io_normal, weight,
                        wall_q, t, a, b);
            double *tmp = a; a = b; b = tmp;
        }
    }
    free(a);
    free(b);
    return scale * J;
}

double orc_objective_run(int q, int64_t n, const int32_t *nbr, const uint8_t *link, double tau,
                         int n_io, const double *rho_mean, const double *amp, const double *period,
                         const double *phase, int64_t t0, int64_t nsteps, const double *f0, int kind,
                         const double *m, int64_t t_begin, int64_t t_end, double scale) {
    return orc_objective_run_bc(q, n, nbr, link, tau, n_io, rho_mean, amp, period, phase, NULL, NULL, NULL,
                                NULL, t0, nsteps, f0, kind, m, t_begin, t_end, scale);
}

/* ------------------------------------------------------------- rendering
 *
 * Direct volume rendering by ray marching (Section 3.3.2: the renderer marches
 * rays through a volume held in a 3D texture, with the view parameters and the
 * transfer-function look-up table in constant memory; zoom, rotation and the
 * scale and offset of the transfer function are steerable).  Readings, taken
 * identically by the CUDA renderer:
 *   - volume: float vol[nz][ny][nx], voxel (i, j, k) centred at (i, j, k) in
 *     volume coordinates; samples are trilinear between voxel centres, clamped
 *     to the edge voxels; the box is [-0.5, n - 0.5] per axis;
 *   - camera: pinhole at eye looking at center, up vector up, vertical field of
 *     view fov_y (radians); pixel (px, py) of a W x H image looks through
 *     ((px + 0.5) / W * 2 - 1) * tan(fov_y/2) * W/H along the right axis and
 *     (1 - (py + 0.5) / H * 2) * tan(fov_y/2) along the up axis;
 *   - the ray's intersection [t_near, t_far] with the box (slab method; t_near
 *     is raised to 0 when the eye is inside) is cut into segments of length dt
 *     from t_near, the last one shorter; each segment takes one sample at its
 *     midpoint, and its length l enters the opacity (so the image is continuous
 *     in the view: a segment that appears at the far end starts with l = 0);
 *   - transfer function: s = clamp((v - offset) * scale, 0, 1), LUT index
 *     s * (L - 1) linearly interpolated between entries (L = 256 RGBA entries,
 *     alpha = opacity per unit length); opacity of a sample a = min(1, alpha l);
 *   - front to back: C += (1 - A) a c, A += (1 - A) a, before each sample the
 *     ray stops once A >= a_stop (early ray termination; a_stop = 1 never
 *     stops before A reaches 1).
 * Output rgba[H][W][4] = (C_r, C_g, C_b, A).
 */
static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static double trilinear(const float *vol, int nx, int ny, int nz, double x, double y, double z) {
    x = clampd(x, 0.0, nx - 1.0);
    y = clampd(y, 0.0, ny - 1.0);
    z = clampd(z, 0.0, nz - 1.0);
    int i0 = (int)floor(x), j0 = (int)floor(y), k0 = (int)floor(z);
    int i1 = i0 + 1 < nx ? i0 + 1 : i0, j1 = j0 + 1 < ny ? j0 + 1 : j0, k1 = k0 + 1 < nz ? k0 + 1 : k0;
    double fx = x - i0, fy = y - j0, fz = z - k0;
#define V(i, j, k) ((double)vol[((int64_t)(k) * ny + (j)) * nx + (i)])
    double c00 = V(i0, j0, k0) * (1 - fx) + V(i1, j0, k0) * fx;
    double c10 = V(i0, j1, k0) * (1 - fx) + V(i1, j1, k0) * fx;
    double c01 = V(i0, j0, k1) * (1 - fx) + V(i1, j0, k1) * fx;
    double c11 = V(i0, j1, k1) * (1 - fx) + V(i1, j1, k1) * fx;
#undef V
    double c0 = c00 * (1 - fy) + c10 * fy, c1 = c01 * (1 - fy) + c11 * fy;
    return c0 * (1 - fz) + c1 * fz;
}

/* Pixels (px, py) = pix[2k], pix[2k + 1] of a W x H image into out[k][4]
 * (pix NULL: every pixel in row-major order, npix = W H). */
int orc_render_pixels(const float *vol, int nx, int ny, int nz, int W, int H, const double *eye,
                      const double *center, const double *up, double fov_y, double dt,
                      double tf_scale, double tf_offset, double a_stop,
                      const float *lut /*[256][4]*/, int64_t npix, const int32_t *pix,
                      float *out) {
    if (W <= 0 || H <= 0 || nx <= 0 || ny <= 0 || nz <= 0 || !(dt > 0)) return -1;
    double f[3], r[3], u[3];
    for (int a = 0; a < 3; ++a) f[a] = center[a] - eye[a];
    double fn = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (int a = 0; a < 3; ++a) f[a] /= fn;
    r[0] = f[1] * up[2] - f[2] * up[1];
    r[1] = f[2] * up[0] - f[0] * up[2];
    r[2] = f[0] * up[1] - f[1] * up[0];
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int a = 0; a < 3; ++a) r[a] /= rn;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    const double th = tan(0.5 * fov_y), aspect = (double)W / (double)H;
    const double lo[3] = {-0.5, -0.5, -0.5}, hi[3] = {nx - 0.5, ny - 0.5, nz - 0.5};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < npix; ++k) {
        {
            const int px = pix ? pix[2 * k] : (int)(k % W), py = pix ? pix[2 * k + 1] : (int)(k / W);
            double sx = ((px + 0.5) / W * 2.0 - 1.0) * th * aspect;
            double sy = (1.0 - (py + 0.5) / H * 2.0) * th;
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = f[a] + sx * r[a] + sy * u[a];
            double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            for (int a = 0; a < 3; ++a) d[a] /= dn;
            double tn = -1e300, tf = 1e300;
            int hit = 1;
            for (int a = 0; a < 3; ++a) {
                if (d[a] == 0.0) {
                    if (eye[a] < lo[a] || eye[a] > hi[a]) hit = 0;
                    continue;
                }
                double t0 = (lo[a] - eye[a]) / d[a], t1 = (hi[a] - eye[a]) / d[a];
                if (t0 > t1) { double tmp = t0; t0 = t1; t1 = tmp; }
                if (t0 > tn) tn = t0;
                if (t1 < tf) tf = t1;
            }
            if (tn < 0.0) tn = 0.0;
            double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
            if (hit && tn < tf) {
                for (int64_t m = 0;; ++m) {
                    double t0 = tn + m * dt;
                    if (t0 >= tf || A >= a_stop) break;
                    double l = tf - t0 < dt ? tf - t0 : dt;
                    double t = t0 + 0.5 * l;
                    double v = trilinear(vol, nx, ny, nz, eye[0] + t * d[0], eye[1] + t * d[1],
                                         eye[2] + t * d[2]);
                    double s = clampd((v - tf_offset) * tf_scale, 0.0, 1.0) * 255.0;
                    int l0 = (int)floor(s);
                    int l1 = l0 < 255 ? l0 + 1 : 255;
                    double fl = s - l0, e[4];
                    for (int c = 0; c < 4; ++c) e[c] = lut[4 * l0 + c] * (1 - fl) + lut[4 * l1 + c] * fl;
                    double a = e[3] * l;
                    if (a > 1.0) a = 1.0;
                    for (int c = 0; c < 3; ++c) C[c] += (1.0 - A) * a * e[c];
                    A += (1.0 - A) * a;
                }
            }
            float *o = out + 4 * k;
            o[0] = (float)C[0];
            o[1] = (float)C[1];
            o[2] = (float)C[2];
            o[3] = (float)A;
        }
    }
    return 0;
}

int orc_render(const float *vol, int nx, int ny, int nz, int W, int H, const double *eye,
               const double *center, const double *up, double fov_y, double dt, double tf_scale,
               double tf_offset, double a_stop, const float *lut /*[256][4]*/,
               float *rgba /*[H][W][4]*/) {
    return orc_render_pixels(vol, nx, ny, nz, W, H, eye, center, up, fov_y, dt, tf_scale,
                             tf_offset, a_stop, lut, (int64_t)W * H, NULL, rgba);
}
