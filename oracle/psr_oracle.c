/*
 * FP64 CPU oracle for the truncated short-range particle-particle (P2P)
 * gravity of the PM-FMM method (Wang & Meng, PhotoNs-GPU, arXiv:2107.14008).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: it is written from the
 * paper's definitions, slowly and plainly, in double precision.
 *
 * Definitions followed (paper, Section 2):
 *   split radius     r_s = 1.2 * BOXSIZE / N_PM            (passed in)
 *   x                = r / (2 r_s)
 *   truncation       T(x) = erfc(x) + (r / (r_s sqrt(pi))) exp(-r^2 / 4 r_s^2)
 *                         = erfc(x) + (2 x / sqrt(pi)) exp(-x^2)        (Eq. tr)
 *   pair force       F_s(r) = -(r / |r|^3) T                         (Section 2)
 *   cutoff           the short-range sum is truncated at r_c         (Section 2)
 * Acceleration of target i (G times force per unit target mass), periodic box
 * of side L, images n in Z^3:
 *   a_i = G sum_j sum_n [j != i or n != 0] [0 < |d| < r_c] m_j d T(|d|/2r_s) / |d|^3,
 *   d   = x_j + n L - x_i.
 * Because the caller guarantees r_c <= L and positions lie in [0, L), only
 * n in {-1,0,1}^3 can satisfy |d| < r_c; the per-axis loops below enumerate
 * exactly the images whose component along that axis is below r_c, which is
 * the same set of non-zero terms as the definition.
 *
 * The adjoint (dL/dx, dL/dm of L = sum_i c_i . a_i) is not in the paper; it is
 * derived here from the pair force and from the paper's general truncated
 * prefactor f_(n)(x) (Section 2, the M2L prefactor equation) at n = 2, which
 * gives the radial derivative term of the tidal tensor:
 *   d/dx_k (g(r) d) = g I + (g'(r)/r) d d^T,   g = T / r^3 = -f_(1),
 *   g'(r)/r = -f_(2),
 *   dL/dx_k = G sum_j K(d_kj) (m_k c_j - m_j c_k),  K = g I - f_(2) d d^T,
 *   dL/dm_k = -G sum_j g(r_kj) d_kj . c_j.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- T(x) -- */

/* Eq. (tr) written in x = r / (2 r_s): r/(r_s sqrt(pi)) = 2x/sqrt(pi). */
double oracle_T(double x)
{
    return erfc(x) + 2.0 * x / sqrt(M_PI) * exp(-x * x);
}

/* E(x) = -4 exp(-x^2) / sqrt(pi), the factor of the Taylor terms (Eq. int). */
double oracle_E(double x)
{
    return -4.0 * exp(-x * x) / sqrt(M_PI);
}

static double dfact_odd(int k) /* (2k-1)!! with (-1)!! = 1 */
{
    double p = 1.0;
    for (int i = 2 * k - 1; i > 1; i -= 2) p *= (double)i;
    return p;
}

/*
 * Truncated prefactor f_(n) at separation r (Section 2):
 *   (-1)^n r_s^{2n+1} f_(n)(x) = (2n-1)!!/2^{2n+1} erfc(x)/x^{2n+1}
 *        + sum_{q=1..n} 2^{-q-n} (2n-1)!!/(2n-2q+1)!! exp(-x^2)/(sqrt(pi) x^{2q})
 */
double oracle_prefactor(int n, double r, double r_s)
{
    double x = r / (2.0 * r_s);
    double s = dfact_odd(n) / pow(2.0, 2 * n + 1) * erfc(x) / pow(x, 2 * n + 1);
    for (int q = 1; q <= n; ++q)
        s += pow(2.0, -q - n) * dfact_odd(n) / dfact_odd(n - q + 1) * exp(-x * x) /
             (sqrt(M_PI) * pow(x, 2 * q));
    double sign = (n % 2) ? -1.0 : 1.0;
    return sign * s / pow(r_s, 2 * n + 1);
}

/* Newtonian prefactor f^inv_(n) = (-1)^n (2n-1)!! / r^{2n+1} (Section 2). */
double oracle_prefactor_newton(int n, double r)
{
    double sign = (n % 2) ? -1.0 : 1.0;
    return sign * dfact_odd(n) / pow(r, 2 * n + 1);
}

/*
 * Interpolated T, for the precision study of the interpolation table
 * (Section 3.3).  Modes:
 *   0: exact T (Eq. tr)
 *   1: linear interpolation between nodes x_k = k x_c / N, k = 0..N
 *   2: cubic Hermite on (T_k, T'_k) with T'_k = x_k^2 E_k (the two tabulated
 *      quantities of Section 3.3)
 *   3: the paper's Taylor table (Eq. int) of level `level` (0..4) about the
 *      nearest node of a uniform grid of N nodes x_k = k x_c / N
 * Modes 1 and 2 return 0 for x >= x_c (the hard cutoff); mode 3 evaluates the
 * expansion at the nearest node for any x in [0, x_c] and returns 0 beyond.
 */
double oracle_T_interp(double x, int mode, int N, double x_c, int level)
{
    if (mode == 0) return oracle_T(x);
    if (!(x < x_c) || x < 0.0) return 0.0;
    double h = x_c / (double)N;
    if (mode == 1 || mode == 2) {
        int k = (int)floor(x / h);
        if (k > N - 1) k = N - 1;
        double x0 = k * h, x1 = (k + 1) * h;
        double t0 = oracle_T(x0), t1 = oracle_T(x1);
        if (mode == 1) return t0 + (x - x0) / h * (t1 - t0);
        double d0 = x0 * x0 * oracle_E(x0), d1 = x1 * x1 * oracle_E(x1);
        double s = (x - x0) / h;
        double h00 = (1 + 2 * s) * (1 - s) * (1 - s);
        double h10 = s * (1 - s) * (1 - s);
        double h01 = s * s * (3 - 2 * s);
        double h11 = s * s * (s - 1);
        return h00 * t0 + h10 * h * d0 + h01 * t1 + h11 * h * d1;
    }
    if (mode == 3) {
        int k = (int)floor(x / h + 0.5);
        if (k > N) k = N;
        double xi = k * h, e = x - xi;
        double Ei = oracle_E(xi);
        double Ti = erfc(xi) - xi * Ei / 2.0; /* = T(x_i) */
        double v = Ti;
        if (level >= 1) v += xi * xi * Ei * e;
        if (level >= 2) v -= xi * (xi * xi - 1.0) * Ei * e * e;
        if (level >= 3) v += (2.0 / 3.0 * pow(xi, 4) - 5.0 / 3.0 * xi * xi + 1.0 / 3.0) * Ei * e * e * e;
        if (level >= 4) v -= xi * (pow(xi, 4) / 3.0 - 1.5 * xi * xi + 1.0) * Ei * e * e * e * e;
        return v;
    }
    return NAN;
}

/* ------------------------------------------------------- pair summation -- */

typedef struct {
    int64_t n;
    const double* pos;   /* n x 3, in [0, L) */
    const double* mass;  /* n */
    const double* cot;   /* n x 3 or NULL (adjoint only) */
    double L, r_s, r_c, G;
    int t_mode, t_n, t_level; /* see oracle_T_interp */
    const int64_t* targets;   /* n_t indices or NULL for 0..n-1 */
    int64_t n_t;
    double* out_a;       /* n_t x 3 */
    double* out_gm;      /* n_t (adjoint) */
    int64_t* out_pairs;  /* n_t: within-cutoff pair count per target */
    int64_t* out_zero;   /* n_t: distinct pairs at r == 0 (contribute 0) */
    int adjoint;
    /* cell lists (NULL = brute force over all sources) */
    int nc;
    const int64_t* cell_start; /* nc^3 + 1 */
    const int64_t* cell_items; /* n, source indices grouped by cell */
    int64_t next;              /* work counter, guarded by lock */
    pthread_mutex_t lock;
} job_t;

static double Tsel(const job_t* jb, double x)
{
    if (jb->t_mode == 0) return oracle_T(x);
    return oracle_T_interp(x, jb->t_mode, jb->t_n, jb->r_c / (2.0 * jb->r_s), jb->t_level);
}

/* One (target i, source j) term over every periodic image within r_c. */
static void pair_terms(const job_t* jb, int64_t i, int64_t j, double acc[3], double* gm,
                       int64_t* npairs, int64_t* nzero)
{
    const double* xi = jb->pos + 3 * i;
    const double* xj = jb->pos + 3 * j;
    double L = jb->L, rc = jb->r_c;
    for (int nx = -1; nx <= 1; ++nx) {
        double dx = xj[0] + nx * L - xi[0];
        if (fabs(dx) >= rc) continue;
        for (int ny = -1; ny <= 1; ++ny) {
            double dy = xj[1] + ny * L - xi[1];
            if (fabs(dy) >= rc) continue;
            for (int nz = -1; nz <= 1; ++nz) {
                double dz = xj[2] + nz * L - xi[2];
                if (fabs(dz) >= rc) continue;
                if (j == i && nx == 0 && ny == 0 && nz == 0) continue; /* self */
                double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < rc * rc)) continue;
                if (r2 == 0.0) { (*nzero)++; continue; }
                (*npairs)++;
                double r = sqrt(r2);
                double x = r / (2.0 * jb->r_s);
                double T = Tsel(jb, x);
                double g = T / (r2 * r); /* T / r^3 = -f_(1) */
                double d[3] = {dx, dy, dz};
                if (!jb->adjoint) {
                    for (int a = 0; a < 3; ++a) acc[a] += jb->mass[j] * g * d[a];
                } else {
                    /* f_(2) from the paper's general prefactor, -f_(2) = g'(r)/r */
                    double f2 = oracle_prefactor(2, r, jb->r_s);
                    const double* cj = jb->cot + 3 * j;
                    const double* ck = jb->cot + 3 * i;
                    double mk = jb->mass[i], mj = jb->mass[j];
                    double v[3], dv = 0.0, dc = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        v[a] = mk * cj[a] - mj * ck[a];
                        dv += d[a] * v[a];
                        dc += d[a] * cj[a];
                    }
                    for (int a = 0; a < 3; ++a) acc[a] += g * v[a] - f2 * d[a] * dv;
                    *gm += -g * dc;
                }
            }
        }
    }
}

static void do_target(job_t* jb, int64_t t)
{
    int64_t i = jb->targets ? jb->targets[t] : t;
    double acc[3] = {0, 0, 0}, gm = 0.0;
    int64_t np = 0, nz = 0;
    if (!jb->cell_start) {
        for (int64_t j = 0; j < jb->n; ++j) pair_terms(jb, i, j, acc, &gm, &np, &nz);
    } else {
        int nc = jb->nc;
        const double* xi = jb->pos + 3 * i;
        int c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = (int)floor(xi[a] / jb->L * nc);
            if (c[a] < 0) c[a] = 0;
            if (c[a] > nc - 1) c[a] = nc - 1;
        }
        for (int ox = -1; ox <= 1; ++ox)
            for (int oy = -1; oy <= 1; ++oy)
                for (int oz = -1; oz <= 1; ++oz) {
                    int cx = (c[0] + ox + nc) % nc, cy = (c[1] + oy + nc) % nc,
                        cz = (c[2] + oz + nc) % nc;
                    int64_t cell = ((int64_t)cx * nc + cy) * nc + cz;
                    for (int64_t s = jb->cell_start[cell]; s < jb->cell_start[cell + 1]; ++s)
                        pair_terms(jb, i, jb->cell_items[s], acc, &gm, &np, &nz);
                }
    }
    for (int a = 0; a < 3; ++a) jb->out_a[3 * t + a] = jb->G * acc[a];
    if (jb->out_gm) jb->out_gm[t] = jb->G * gm;
    if (jb->out_pairs) jb->out_pairs[t] = np;
    if (jb->out_zero) jb->out_zero[t] = nz;
}

static void* worker(void* arg)
{
    job_t* jb = (job_t*)arg;
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        int64_t t0 = jb->next;
        jb->next += 64;
        pthread_mutex_unlock(&jb->lock);
        if (t0 >= jb->n_t) break;
        int64_t t1 = t0 + 64 < jb->n_t ? t0 + 64 : jb->n_t;
        for (int64_t t = t0; t < t1; ++t) do_target(jb, t);
    }
    return NULL;
}

static int run(job_t* jb, int use_cells, int nthreads)
{
    int64_t* cstart = NULL;
    int64_t* citems = NULL;
    jb->cell_start = NULL;
    jb->cell_items = NULL;
    if (use_cells) {
        int nc = (int)floor(jb->L / jb->r_c);
        if (nc > 256) nc = 256;
        if (nc >= 3) {
            int64_t ncell = (int64_t)nc * nc * nc;
            cstart = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
            citems = (int64_t*)malloc((size_t)(jb->n > 0 ? jb->n : 1) * sizeof(int64_t));
            int64_t* cid = (int64_t*)malloc((size_t)(jb->n > 0 ? jb->n : 1) * sizeof(int64_t));
            if (!cstart || !citems || !cid) { free(cstart); free(citems); free(cid); return -1; }
            for (int64_t j = 0; j < jb->n; ++j) {
                int c[3];
                for (int a = 0; a < 3; ++a) {
                    c[a] = (int)floor(jb->pos[3 * j + a] / jb->L * nc);
                    if (c[a] < 0) c[a] = 0;
                    if (c[a] > nc - 1) c[a] = nc - 1;
                }
                cid[j] = ((int64_t)c[0] * nc + c[1]) * nc + c[2];
                cstart[cid[j] + 1]++;
            }
            for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
            int64_t* fill = (int64_t*)malloc((size_t)ncell * sizeof(int64_t));
            if (!fill) { free(cstart); free(citems); free(cid); return -1; }
            memcpy(fill, cstart, (size_t)ncell * sizeof(int64_t));
            for (int64_t j = 0; j < jb->n; ++j) citems[fill[cid[j]]++] = j;
            free(fill);
            free(cid);
            jb->nc = nc;
            jb->cell_start = cstart;
            jb->cell_items = citems;
        }
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    jb->next = 0;
    pthread_mutex_init(&jb->lock, NULL);
    pthread_t th[512];
    int started = 0;
    for (int k = 1; k < nthreads; ++k)
        if (pthread_create(&th[started], NULL, worker, jb) == 0) started++;
    worker(jb);
    for (int k = 0; k < started; ++k) pthread_join(th[k], NULL);
    pthread_mutex_destroy(&jb->lock);
    free(cstart);
    free(citems);
    return 0;
}

/*
 * Accelerations of the listed targets (all particles if targets == NULL).
 * Returns 0, or -1 on bad arguments (r_c must satisfy 0 < r_c <= L,
 * positions must lie in [0, L)), -2 on allocation failure.
 * use_cells = 1 prunes sources with a periodic grid of cells of side >= r_c;
 * it visits every source that can lie within r_c, so the set of terms is that
 * of the brute force.
 */
int oracle_forces(int64_t n, const double* pos, const double* mass, double L, double r_s,
                  double r_c, double G, int t_mode, int t_n, int t_level, int64_t n_t,
                  const int64_t* targets, double* out_a, int64_t* out_pairs, int64_t* out_zero,
                  int use_cells, int nthreads)
{
    if (n < 0 || !(L > 0) || !(r_s > 0) || !(r_c > 0) || r_c > L) return -1;
    for (int64_t j = 0; j < 3 * n; ++j)
        if (!(pos[j] >= 0.0 && pos[j] < L)) return -1;
    job_t jb;
    memset(&jb, 0, sizeof jb);
    jb.n = n; jb.pos = pos; jb.mass = mass; jb.L = L; jb.r_s = r_s; jb.r_c = r_c; jb.G = G;
    jb.t_mode = t_mode; jb.t_n = t_n; jb.t_level = t_level;
    jb.targets = targets; jb.n_t = targets ? n_t : n;
    jb.out_a = out_a; jb.out_pairs = out_pairs; jb.out_zero = out_zero;
    return run(&jb, use_cells, nthreads) ? -2 : 0;
}

/*
 * Gradients of L = sum_i c_i . a_i with respect to the positions and masses of
 * the listed particles, exact T only.  out_gx: n_t x 3, out_gm: n_t.
 */
int oracle_adjoint(int64_t n, const double* pos, const double* mass, const double* cot, double L,
                   double r_s, double r_c, double G, int64_t n_t, const int64_t* targets,
                   double* out_gx, double* out_gm, int use_cells, int nthreads)
{
    if (n < 0 || !(L > 0) || !(r_s > 0) || !(r_c > 0) || r_c > L) return -1;
    for (int64_t j = 0; j < 3 * n; ++j)
        if (!(pos[j] >= 0.0 && pos[j] < L)) return -1;
    job_t jb;
    memset(&jb, 0, sizeof jb);
    jb.n = n; jb.pos = pos; jb.mass = mass; jb.cot = cot;
    jb.L = L; jb.r_s = r_s; jb.r_c = r_c; jb.G = G;
    jb.targets = targets; jb.n_t = targets ? n_t : n;
    jb.out_a = out_gx; jb.out_gm = out_gm; jb.adjoint = 1;
    return run(&jb, use_cells, nthreads) ? -2 : 0;
}

/* Vectorised T for the pins: out[k] = oracle_T_interp(x[k], mode, N, x_c, level). */
void oracle_T_array(int64_t n, const double* x, double* out, int mode, int N, double x_c, int level)
{
    for (int64_t k = 0; k < n; ++k) out[k] = oracle_T_interp(x[k], mode, N, x_c, level);
}
