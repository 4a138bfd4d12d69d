/*
 * ljmd_oracle.c -- plain, slow FP64 reference for truncated Lennard-Jones MD.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library.  The CUDA
 * product path shares no code, header, table or helper with it.
 *
 * What it computes, and where the paper states it (arXiv 2406.04210):
 *   - particles in a periodic cubic/orthorhombic box, Hamiltonian equations of
 *     motion integrated in time steps (Sec. 1, Introduction);
 *   - Lennard-Jones pair forces (Sec. 4, the first workload), truncated at a
 *     cutoff so that only close pairs contribute (Sec. 3, Code structure);
 *   - Verlet neighbour lists built with a spatial decomposition ("particle
 *     binning", Sec. 3, Code structure);
 *   - the velocity-Verlet integrator split into `integrate` (half kick +
 *     drift) and `finalize` (half kick) around the force evaluation (Sec. 3,
 *     Code structure; Fig. 1).
 * The paper prints no formulas; the textbook forms (Allen & Tildesley, cited
 * in Sec. 1 and Sec. 3) are written out here.  Where the paper is silent the
 * reading taken is stated beside the function that takes it (reduced units
 * and unit mass, a strict cutoff test, a full list with skin, 3N - 3 degrees
 * of freedom).
 *
 * Conventions: reduced LJ units, unit mass (m = 1), k_B = 1.  Arrays are
 * n x 3 row-major (AoS) FP64 in user order.  Pair parameter tables are
 * ntypes x ntypes row-major and symmetric.  All sums run sequentially in
 * index order.  Compiled with -ffp-contract=off so that a*b+c is two
 * roundings, exactly as written.
 *
 * Parity status (every function below is pinned by tests/test_oracle.py):
 *   or_pair                 closed forms (minimum at 2^(1/6) sigma, U(sigma)=shift,
 *                           F(sigma)=24 eps/sigma) and FD of U
 *   or_forces_brute/_list   Newton III, FD of E_pot, virial = -dU/dlambda
 *   or_nlist                cell list == brute force, brute force == definition
 *   or_run                  momentum, NVE drift ~ dt^2, time reversibility
 *   or_hvp, or_dforce_dparam  central differences of the forces
 *   or_hist, or_hist_grad   normalisation sum and central differences
 *   or_adjoint              central differences of a trajectory loss
 *   or_fire                 monotone descent to max|F| < ftol (input relaxation)
 *   or_philox4x32           the published known-answer vectors of Philox4x32-10
 *                           (Random123), uniformity and stream independence
 *                           (chi-square), Gaussian moments of the Box-Muller draws
 *   or_run with a thermostat  collision frequency = rate dt (binomial), canonical
 *                           <E_kin> = 3/2 (N - 1) T, velocity distribution
 *   or_run, all pairs       forces == or_forces_brute with rc = inf, NVE drift
 *
 * The all-to-all workload (Sec. 4: untruncated LJ forces between all pairs,
 * velocity-Verlet, and a stochastic Andersen-like "Boltzmann" thermostat) is
 * or_run with every cutoff infinite: forces by brute force over all pairs
 * with the minimum image, no lists.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_CAPACITY 4
#define OR_ERR_BOX 5
#define OR_ERR_OOM 3

/* ------------------------------------------------------------------ */
/* Pair potential.                                                     */
/* U(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - U_shift for r < rc,    */
/* zero otherwise; U_shift = 4 eps [(sigma/rc)^12 - (sigma/rc)^6] when */
/* `shift` is set (energy only; the force is the plain LJ force,       */
/* truncated at rc).  The force on i from j is F_ij = f * d_ij with    */
/* d_ij = x_i - x_j and f = -U'(r)/r = 48 eps/r^2 [s^12 - s^6/2].      */
/* Also returned: phi'' and phi'/r for the Hessian.                    */
/* ------------------------------------------------------------------ */
void or_pair(double eps, double sigma, double rc, int32_t shift, double r2,
             double out[4])
{
    out[0] = out[1] = out[2] = out[3] = 0.0;
    if (!(r2 < rc * rc)) return;
    double s2 = (sigma * sigma) / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double u = 4.0 * eps * (s12 - s6);
    if (shift) {
        double c2 = (sigma * sigma) / (rc * rc);
        double c6 = c2 * c2 * c2;
        u -= 4.0 * eps * (c6 * c6 - c6);
    }
    /* phi'(r) = -(24 eps / r) (2 s^12 - s^6)                              */
    /* phi''(r) = (24 eps / r^2) (26 s^12 - 7 s^6)                        */
    double f = 48.0 * eps / r2 * (s12 - 0.5 * s6);
    out[0] = f;                                    /* -phi'(r)/r */
    out[1] = u;
    out[2] = 24.0 * eps / r2 * (26.0 * s12 - 7.0 * s6); /* phi''(r) */
    out[3] = -f;                                   /* phi'(r)/r */
}

/* Minimum-image component, Sec. 1: periodic boundary conditions. */
double or_min_image(double d, double L)
{
    return d - L * nearbyint(d / L);
}

static double r2_min_image(const double* xi, const double* xj, const double L[3],
                           double d[3])
{
    d[0] = or_min_image(xi[0] - xj[0], L[0]);
    d[1] = or_min_image(xi[1] - xj[1], L[1]);
    d[2] = or_min_image(xi[2] - xj[2], L[2]);
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

static double max_rcut(int32_t nt, const double* rcut)
{
    double m = 0.0;
    for (int32_t k = 0; k < nt * nt; ++k)
        if (rcut[k] > m) m = rcut[k];
    return m;
}

/* ------------------------------------------------------------------ */
/* Forces, potential energy and virial by brute force over all pairs  */
/* i<j with the minimum image (the all-to-all form of Sec. 4/5).      */
/* W = sum_{i<j} d_ij . F_ij.                                          */
/* ------------------------------------------------------------------ */
int32_t or_forces_brute(int64_t n, const double L[3], int32_t nt,
                        const int32_t* type, const double* pos,
                        const double* eps, const double* sigma,
                        const double* rcut, int32_t shift, double* force,
                        double* epot, double* virial)
{
    double e = 0.0, w = 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) force[i] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double d[3];
            double r2 = r2_min_image(pos + 3 * i, pos + 3 * j, L, d);
            int32_t p = type[i] * nt + type[j];
            double o[4];
            or_pair(eps[p], sigma[p], rcut[p], shift, r2, o);
            for (int c = 0; c < 3; ++c) {
                force[3 * i + c] += o[0] * d[c];
                force[3 * j + c] -= o[0] * d[c];
            }
            e += o[1];
            w += o[0] * r2;
        }
    }
    if (epot) *epot = e;
    if (virial) *virial = w;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11): a counter-based generator.  Each of the  */
/* ten rounds multiplies words 0 and 2 of the counter by two fixed odd   */
/* constants, swaps the high/low halves across the words and mixes in   */
/* the key; the key advances by two Weyl constants between rounds.      */
/* ------------------------------------------------------------------ */
void or_philox4x32(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Uniform in (0, 1) from a 32-bit word: (x + 1/2) / 2^32.              */
static double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* ------------------------------------------------------------------ */
/* Andersen-like ("Boltzmann") thermostat, applied after the finalize   */
/* half kick of step s (reading of Sec. 4, which names the thermostat   */
/* only).  Particle u (user index) collides with the bath when word 0   */
/* of philox(ctr = (u, s lo, s hi, 0), key = seed) is below             */
/* floor(rate dt 2^32); its velocity is then redrawn from the           */
/* Maxwell-Boltzmann distribution at T_bath (unit mass): three          */
/* Gaussians by Box-Muller, g0, g1 from words 1, 2 and g2 from words    */
/* 0, 1 of philox(ctr = (u, s lo, s hi, 1)), v = sqrt(T_bath) g.        */
/* Returns the number of collisions.                                    */
/* ------------------------------------------------------------------ */
static uint32_t collide_threshold(double rate, double dt)
{
    double t = floor(rate * dt * 4294967296.0);
    if (!(t > 0.0)) return 0u;
    if (t >= 4294967295.0) return 4294967295u;
    return (uint32_t)t;
}

int64_t or_thermostat(int64_t n, double* vel, double T_bath, double rate, double dt,
                      uint64_t seed, int64_t step)
{
    const uint32_t thr = collide_threshold(rate, dt);
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const double sd = sqrt(T_bath);
    const double two_pi = 6.283185307179586476925286766559;
    int64_t hits = 0;
    for (int64_t u = 0; u < n; ++u) {
        uint32_t c[4] = {(uint32_t)u, (uint32_t)step, (uint32_t)((uint64_t)step >> 32), 0u};
        uint32_t x[4];
        or_philox4x32(c, key, x);
        if (!(x[0] < thr)) continue;
        c[3] = 1u;
        uint32_t y[4];
        or_philox4x32(c, key, y);
        double r1 = sqrt(-2.0 * log(u01(x[1]))), a1 = two_pi * u01(x[2]);
        double r2 = sqrt(-2.0 * log(u01(y[0]))), a2 = two_pi * u01(y[1]);
        vel[3 * u + 0] = sd * (r1 * cos(a1));
        vel[3 * u + 1] = sd * (r1 * sin(a1));
        vel[3 * u + 2] = sd * (r2 * cos(a2));
        ++hits;
    }
    return hits;
}

/* ------------------------------------------------------------------ */
/* Verlet neighbour list (Sec. 3): L_i = { j != i : |d_ij|^2 < rl^2 }, */
/* full (both directions), each list sorted ascending by j.            */
/* use_cells = 0: test every pair.  use_cells = 1: particle binning   */
/* into nc = floor(L/rl) cells per dimension and a 27-cell search,    */
/* which needs nc >= 3 (otherwise the brute-force form is used).      */
/* count[i] gets the true list length; at most cap entries are stored */
/* in list[i*cap ...].  Returns the largest length (a return above    */
/* cap means the list is truncated and must be redone).               */
/* ------------------------------------------------------------------ */
static int cmp_i64(const void* a, const void* b)
{
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

int64_t or_nlist(int64_t n, const double L[3], const double* pos, double rl,
                 int32_t use_cells, int64_t cap, int32_t* count, int64_t* list)
{
    double rl2 = rl * rl;
    int64_t maxc = 0;
    int64_t nc[3];
    for (int c = 0; c < 3; ++c) nc[c] = (int64_t)floor(L[c] / rl);
    if (use_cells && (nc[0] < 3 || nc[1] < 3 || nc[2] < 3)) use_cells = 0;

    if (!use_cells) {
        for (int64_t i = 0; i < n; ++i) {
            int64_t k = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double d[3];
                if (r2_min_image(pos + 3 * i, pos + 3 * j, L, d) < rl2) {
                    if (k < cap) list[i * cap + k] = j;
                    ++k;
                }
            }
            count[i] = (int32_t)k;
            if (k > maxc) maxc = k;
        }
        return maxc;
    }

    /* binning: head/next linked lists over cells */
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    if (!head || !next || !cand || !cell) {
        free(head); free(next); free(cand); free(cell);
        return -1;
    }
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t ci[3];
        for (int c = 0; c < 3; ++c) {
            double x = pos[3 * i + c] - L[c] * floor(pos[3 * i + c] / L[c]);
            int64_t q = (int64_t)floor(x / (L[c] / (double)nc[c]));
            if (q < 0) q = 0;
            if (q >= nc[c]) q = nc[c] - 1;
            ci[c] = q;
            cell[3 * i + c] = q;
        }
        int64_t lin = ci[0] + nc[0] * (ci[1] + nc[1] * ci[2]);
        next[i] = head[lin];
        head[lin] = i;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t cx = (cell[3 * i + 0] + dx + nc[0]) % nc[0];
                    int64_t cy = (cell[3 * i + 1] + dy + nc[1]) % nc[1];
                    int64_t cz = (cell[3 * i + 2] + dz + nc[2]) % nc[2];
                    for (int64_t j = head[cx + nc[0] * (cy + nc[1] * cz)]; j >= 0;
                         j = next[j]) {
                        if (j == i) continue;
                        double d[3];
                        if (r2_min_image(pos + 3 * i, pos + 3 * j, L, d) < rl2)
                            cand[k++] = j;
                    }
                }
        qsort(cand, (size_t)k, sizeof(int64_t), cmp_i64);
        for (int64_t m = 0; m < k && m < cap; ++m) list[i * cap + m] = cand[m];
        count[i] = (int32_t)k;
        if (k > maxc) maxc = k;
    }
    free(head); free(next); free(cand); free(cell);
    return maxc;
}

/* ------------------------------------------------------------------ */
/* Forces over a full neighbour list: F_i = sum_{j in L_i, r<rc} f d_ij; */
/* E_pot = 1/2 sum_i sum_j U, W = 1/2 sum_i sum_j f r^2 (each pair is  */
/* seen twice in a full list).                                        */
/* ------------------------------------------------------------------ */
int32_t or_forces_list(int64_t n, const double L[3], int32_t nt,
                       const int32_t* type, const double* pos,
                       const double* eps, const double* sigma,
                       const double* rcut, int32_t shift,
                       const int32_t* count, const int64_t* list, int64_t cap,
                       double* force, double* epot, double* virial)
{
    double e = 0.0, w = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double f[3] = {0.0, 0.0, 0.0};
        for (int64_t m = 0; m < count[i]; ++m) {
            int64_t j = list[i * cap + m];
            double d[3];
            double r2 = r2_min_image(pos + 3 * i, pos + 3 * j, L, d);
            int32_t p = type[i] * nt + type[j];
            double o[4];
            or_pair(eps[p], sigma[p], rcut[p], shift, r2, o);
            for (int c = 0; c < 3; ++c) f[c] += o[0] * d[c];
            e += 0.5 * o[1];
            w += 0.5 * o[0] * r2;
        }
        for (int c = 0; c < 3; ++c) force[3 * i + c] = f[c];
    }
    if (epot) *epot = e;
    if (virial) *virial = w;
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Hessian-vector product of U_tot over a full list:                  */
/* (H u)_i = sum_j [phi'' rh (rh.u_ij) + (phi'/r)(u_ij - rh (rh.u_ij))] */
/* with rh = d_ij/r and u_ij = u_i - u_j, for r < rc (the cutoff is   */
/* held fixed, so no boundary term).                                  */
/* ------------------------------------------------------------------ */
int32_t or_hvp(int64_t n, const double L[3], int32_t nt, const int32_t* type,
               const double* pos, const double* eps, const double* sigma,
               const double* rcut, const int32_t* count, const int64_t* list,
               int64_t cap, const double* u, double* hu)
{
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t m = 0; m < count[i]; ++m) {
            int64_t j = list[i * cap + m];
            double d[3];
            double r2 = r2_min_image(pos + 3 * i, pos + 3 * j, L, d);
            int32_t p = type[i] * nt + type[j];
            double o[4];
            or_pair(eps[p], sigma[p], rcut[p], 0, r2, o);
            if (!(r2 < rcut[p] * rcut[p])) continue;
            double r = sqrt(r2);
            double rh[3] = {d[0] / r, d[1] / r, d[2] / r};
            double uij[3];
            for (int c = 0; c < 3; ++c) uij[c] = u[3 * i + c] - u[3 * j + c];
            double ru = (rh[0] * uij[0] + rh[1] * uij[1]) + rh[2] * uij[2];
            for (int c = 0; c < 3; ++c)
                acc[c] += o[2] * rh[c] * ru + o[3] * (uij[c] - rh[c] * ru);
        }
        for (int c = 0; c < 3; ++c) hu[3 * i + c] = acc[c];
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Parameter derivatives of the forces, contracted with a vector lam: */
/* g_eps[a,b]   = sum_i lam_i . dF_i/d eps_ab                          */
/* g_sigma[a,b] = sum_i lam_i . dF_i/d sigma_ab                        */
/* at fixed rc.  dF_ij/d eps = F_ij/eps;                               */
/* dF_ij/d sigma = 48 eps/r^3 (12 s^11 - 3 s^5) d_ij, s = sigma/r.     */
/* eps_ab and sigma_ab are single symmetric parameters: both (a,b) and */
/* (b,a) pairs add into [a,b], and the table is written symmetric.    */
/* ------------------------------------------------------------------ */
int32_t or_dforce_dparam(int64_t n, const double L[3], int32_t nt,
                         const int32_t* type, const double* pos,
                         const double* eps, const double* sigma,
                         const double* rcut, const int32_t* count,
                         const int64_t* list, int64_t cap, const double* lam,
                         double* g_eps, double* g_sigma)
{
    for (int32_t k = 0; k < nt * nt; ++k) g_eps[k] = g_sigma[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t m = 0; m < count[i]; ++m) {
            int64_t j = list[i * cap + m];
            double d[3];
            double r2 = r2_min_image(pos + 3 * i, pos + 3 * j, L, d);
            int32_t a = type[i], b = type[j];
            int32_t p = a * nt + b;
            if (!(r2 < rcut[p] * rcut[p])) continue;
            double o[4];
            or_pair(eps[p], sigma[p], rcut[p], 0, r2, o);
            double r = sqrt(r2);
            double s = sigma[p] / r;
            double s5 = s * s * s * s * s;
            double s11 = s5 * s5 * s;
            double dfs = 48.0 * eps[p] / (r2 * r) * (12.0 * s11 - 3.0 * s5);
            double ld = (lam[3 * i + 0] * d[0] + lam[3 * i + 1] * d[1]) +
                        lam[3 * i + 2] * d[2];
            int32_t lo = a < b ? a : b, hi = a < b ? b : a;
            g_eps[lo * nt + hi] += o[0] / eps[p] * ld;
            g_sigma[lo * nt + hi] += dfs * ld;
        }
    }
    for (int32_t a = 0; a < nt; ++a)
        for (int32_t b = a + 1; b < nt; ++b) {
            g_eps[b * nt + a] = g_eps[a * nt + b];
            g_sigma[b * nt + a] = g_sigma[a * nt + b];
        }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Velocity-Verlet MD (Sec. 3, Fig. 1: integrate = half kick + drift,  */
/* force, finalize = half kick).                                      */
/*   v <- v + dt/2 F;  x <- x + dt v;  wrap x into [0,L), count images;*/
/*   rebuild the list if max_i |x_i - x_i(build)| > skin/2 (unwrapped);*/
/*   F <- F(x);  v <- v + dt/2 F.                                      */
/* thermo (nullable) gets, per step after finalize: E_pot, E_kin, W,  */
/* T = 2 E_kin / (3N - 3).  traj (nullable) gets the (wrapped)        */
/* positions after every step, (nsteps+1) x n x 3, index 0 = input.   */
/* Returns the number of list builds (including the initial one) or a */
/* negative value on error.                                           */
/* ------------------------------------------------------------------ */
static int64_t build_list(int64_t n, const double L[3], const double* pos,
                          double rl, int32_t** count, int64_t** list,
                          int64_t* cap)
{
    for (;;) {
        int64_t m = or_nlist(n, L, pos, rl, 1, *cap, *count, *list);
        if (m < 0) return -1;
        if (m <= *cap) return 0;
        *cap = m + 16;
        free(*list);
        *list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * (*cap) + 1));
        if (!*list) return -1;
    }
}

/* Thermostat (rate > 0): or_thermostat after the finalize of step s,  */
/* s = 0, 1, ...; energies are taken after it.  Every cutoff infinite:  */
/* the all-to-all form, forces by brute force over all pairs.          */
int64_t or_run(int64_t n, const double L[3], int32_t nt, const int32_t* type,
               double* pos, double* vel, int32_t* img, const double* eps,
               const double* sigma, const double* rcut, int32_t shift,
               double skin, double dt, int64_t nsteps, double* thermo,
               double* traj, double T_bath, double rate, uint64_t seed)
{
    double rl = max_rcut(nt, rcut) + skin;
    const int all_pairs = isinf(rl);
    for (int c = 0; c < 3; ++c)
        if (!all_pairs && !(rl < 0.5 * L[c])) return -OR_ERR_BOX;
    int64_t cap = 64;
    int32_t* count = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * cap + 1));
    double* f = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* disp = (double*)calloc((size_t)(3 * n + 1), sizeof(double));
    if (!count || !list || !f || !disp) return -OR_ERR_OOM;
    int64_t builds = 0;
    double e = 0.0, w = 0.0;

    if (all_pairs) {
        or_forces_brute(n, L, nt, type, pos, eps, sigma, rcut, shift, f, &e, &w);
    } else {
        if (build_list(n, L, pos, rl, &count, &list, &cap) < 0) return -OR_ERR_OOM;
        ++builds;
        or_forces_list(n, L, nt, type, pos, eps, sigma, rcut, shift, count, list,
                       cap, f, &e, &w);
    }
    if (traj) memcpy(traj, pos, sizeof(double) * (size_t)(3 * n));

    for (int64_t s = 0; s < nsteps; ++s) {
        /* integrate: half kick + drift */
        double dmax2 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            for (int c = 0; c < 3; ++c) {
                int64_t k = 3 * i + c;
                vel[k] = vel[k] + 0.5 * dt * f[k];
                double dx = dt * vel[k];
                pos[k] = pos[k] + dx;
                disp[k] += dx;
                double q = floor(pos[k] / L[c]);
                if (q != 0.0) {
                    pos[k] = pos[k] - L[c] * q;
                    if (img) img[k] += (int32_t)q;
                }
            }
            double d2 = (disp[3 * i] * disp[3 * i] + disp[3 * i + 1] * disp[3 * i + 1]) +
                        disp[3 * i + 2] * disp[3 * i + 2];
            if (d2 > dmax2) dmax2 = d2;
        }
        if (!all_pairs && dmax2 > 0.25 * skin * skin) {
            if (build_list(n, L, pos, rl, &count, &list, &cap) < 0)
                return -OR_ERR_OOM;
            ++builds;
            memset(disp, 0, sizeof(double) * (size_t)(3 * n));
        }
        /* force */
        if (all_pairs)
            or_forces_brute(n, L, nt, type, pos, eps, sigma, rcut, shift, f, &e, &w);
        else
            or_forces_list(n, L, nt, type, pos, eps, sigma, rcut, shift, count,
                           list, cap, f, &e, &w);
        /* finalize: half kick */
        double ek = 0.0;
        for (int64_t k = 0; k < 3 * n; ++k) {
            vel[k] = vel[k] + 0.5 * dt * f[k];
        }
        if (rate > 0.0) or_thermostat(n, vel, T_bath, rate, dt, seed, s);
        for (int64_t i = 0; i < n; ++i)
            ek += 0.5 * ((vel[3 * i] * vel[3 * i] + vel[3 * i + 1] * vel[3 * i + 1]) +
                         vel[3 * i + 2] * vel[3 * i + 2]);
        if (thermo) {
            thermo[4 * s + 0] = e;
            thermo[4 * s + 1] = ek;
            thermo[4 * s + 2] = w;
            thermo[4 * s + 3] = n > 1 ? 2.0 * ek / (3.0 * (double)n - 3.0) : 0.0;
        }
        if (traj) memcpy(traj + 3 * n * (s + 1), pos, sizeof(double) * (size_t)(3 * n));
    }
    free(count); free(list); free(f); free(disp);
    return builds;
}

/* ------------------------------------------------------------------ */
/* Pair-distance histogram with Gaussian smoothing over pairs i<j with */
/* r < rmax_pairs:  h_k = (1/N) sum_{i<j} exp(-(r_ij - c_k)^2/(2 w^2)), */
/* c_k = (k + 1/2) * rbin, k = 0..nbins-1, rbin = rhist/nbins.          */
/* Pairs come from a full list (each i<j pair once: j > i).            */
/* ------------------------------------------------------------------ */
int32_t or_hist(int64_t n, const double L[3], const double* pos,
                const int32_t* count, const int64_t* list, int64_t cap,
                double rmax_pairs, int32_t nbins, double rhist, double w,
                double* h)
{
    double rbin = rhist / (double)nbins;
    for (int32_t k = 0; k < nbins; ++k) h[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t m = 0; m < count[i]; ++m) {
            int64_t j = list[i * cap + m];
            if (j <= i) continue;
            double d[3];
            double r2 = r2_min_image(pos + 3 * i, pos + 3 * j, L, d);
            if (!(r2 < rmax_pairs * rmax_pairs)) continue;
            double r = sqrt(r2);
            for (int32_t k = 0; k < nbins; ++k) {
                double c = ((double)k + 0.5) * rbin;
                h[k] += exp(-(r - c) * (r - c) / (2.0 * w * w));
            }
        }
    }
    for (int32_t k = 0; k < nbins; ++k) h[k] /= (double)n;
    return OR_OK;
}

/* Gradient of sum_k coef_k h_k with respect to the positions:          */
/* dh_k/dx_i = (1/N) sum_j g_k'(r_ij) d_ij/r_ij, g_k'(r) = -(r-c_k)/w^2 g_k. */
int32_t or_hist_grad(int64_t n, const double L[3], const double* pos,
                     const int32_t* count, const int64_t* list, int64_t cap,
                     double rmax_pairs, int32_t nbins, double rhist, double w,
                     const double* coef, double* grad)
{
    double rbin = rhist / (double)nbins;
    for (int64_t i = 0; i < 3 * n; ++i) grad[i] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t m = 0; m < count[i]; ++m) {
            int64_t j = list[i * cap + m];
            if (j <= i) continue;
            double d[3];
            double r2 = r2_min_image(pos + 3 * i, pos + 3 * j, L, d);
            if (!(r2 < rmax_pairs * rmax_pairs)) continue;
            double r = sqrt(r2);
            double dg = 0.0;
            for (int32_t k = 0; k < nbins; ++k) {
                double c = ((double)k + 0.5) * rbin;
                double g = exp(-(r - c) * (r - c) / (2.0 * w * w));
                dg += coef[k] * (-(r - c) / (w * w)) * g;
            }
            for (int c = 0; c < 3; ++c) {
                grad[3 * i + c] += dg * d[c] / r / (double)n;
                grad[3 * j + c] -= dg * d[c] / r / (double)n;
            }
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Adjoint of velocity-Verlet (unit mass, a = F).  Forward step k:      */
/*   vh = v_k + h/2 a(x_k); x_{k+1} = x_k + h vh; v_{k+1} = vh + h/2 a(x_{k+1}). */
/* Reverse, with J_a = -H (H = Hessian of U_tot):                       */
/*   lx~ = lx_{k+1} - h/2 H(x_{k+1}) lv_{k+1}                            */
/*   lvh = lv_{k+1} + h lx~                                              */
/*   lx_k = lx~ - h/2 H(x_k) lvh ;  lv_k = lvh                           */
/*   dL/dtheta += h/2 lv_{k+1}.da(x_{k+1})/dtheta + h/2 lvh.da(x_k)/dtheta */
/* Written plainly with two HVPs per step and a fresh list at every    */
/* state (the forces do not depend on which valid list is used).       */
/* traj holds x_0..x_T ((nsteps+1) x n x 3).  Wrapping is a constant    */
/* shift of x and does not enter the derivatives.                      */
/* ------------------------------------------------------------------ */
int32_t or_adjoint(int64_t n, const double L[3], int32_t nt,
                   const int32_t* type, const double* traj,
                   const double* eps, const double* sigma, const double* rcut,
                   double dt, int64_t nsteps, const double* lx_T,
                   const double* lv_T, double* lx_0, double* lv_0,
                   double* g_eps, double* g_sigma)
{
    double rl = max_rcut(nt, rcut);
    int64_t cap = 64;
    int32_t* count = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * cap + 1));
    double* lx = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* lv = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* hv = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* ge = (double*)malloc(sizeof(double) * (size_t)(nt * nt));
    double* gs = (double*)malloc(sizeof(double) * (size_t)(nt * nt));
    if (!count || !list || !lx || !lv || !hv || !ge || !gs) return OR_ERR_OOM;
    memcpy(lx, lx_T, sizeof(double) * (size_t)(3 * n));
    memcpy(lv, lv_T, sizeof(double) * (size_t)(3 * n));
    for (int32_t k = 0; k < nt * nt; ++k) g_eps[k] = g_sigma[k] = 0.0;
    double h = dt;

    for (int64_t k = nsteps - 1; k >= 0; --k) {
        const double* x1 = traj + 3 * n * (k + 1);
        const double* x0 = traj + 3 * n * k;
        /* terms at x_{k+1} with lv_{k+1} */
        if (build_list(n, L, x1, rl, &count, &list, &cap) < 0) return OR_ERR_OOM;
        or_hvp(n, L, nt, type, x1, eps, sigma, rcut, count, list, cap, lv, hv);
        or_dforce_dparam(n, L, nt, type, x1, eps, sigma, rcut, count, list,
                         cap, lv, ge, gs);
        for (int32_t q = 0; q < nt * nt; ++q) {
            g_eps[q] += 0.5 * h * ge[q];
            g_sigma[q] += 0.5 * h * gs[q];
        }
        for (int64_t q = 0; q < 3 * n; ++q) {
            lx[q] = lx[q] - 0.5 * h * hv[q];   /* lx~ */
            lv[q] = lv[q] + h * lx[q];         /* lvh */
        }
        /* terms at x_k with lvh */
        if (build_list(n, L, x0, rl, &count, &list, &cap) < 0) return OR_ERR_OOM;
        or_hvp(n, L, nt, type, x0, eps, sigma, rcut, count, list, cap, lv, hv);
        or_dforce_dparam(n, L, nt, type, x0, eps, sigma, rcut, count, list,
                         cap, lv, ge, gs);
        for (int32_t q = 0; q < nt * nt; ++q) {
            g_eps[q] += 0.5 * h * ge[q];
            g_sigma[q] += 0.5 * h * gs[q];
        }
        for (int64_t q = 0; q < 3 * n; ++q) lx[q] = lx[q] - 0.5 * h * hv[q];
    }
    memcpy(lx_0, lx, sizeof(double) * (size_t)(3 * n));
    memcpy(lv_0, lv, sizeof(double) * (size_t)(3 * n));
    free(count); free(list); free(lx); free(lv); free(hv); free(ge); free(gs);
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* FIRE relaxation (Bitzek, Koskinen, Gaehler, Moseler, Gumbsch, Phys.  */
/* Rev. Lett. 97, 170201 (2006)) of U_tot, used to prepare the relaxed  */
/* random configurations of the binary-mixture workload.  Euler-type   */
/* MD steps with velocity mixing v <- (1-a) v + a |v| F/|F| while the  */
/* power P = F.v is positive; on P <= 0 the velocities are zeroed, the */
/* step is halved and a is reset.  Stops when max_i |F_i| < ftol.      */
/* Returns the number of iterations done.                              */
/* ------------------------------------------------------------------ */
int64_t or_fire(int64_t n, const double L[3], int32_t nt, const int32_t* type,
                double* pos, const double* eps, const double* sigma,
                const double* rcut, int64_t maxit, double ftol, double dt0,
                double* fmax_out)
{
    const double finc = 1.1, fdec = 0.5, a0 = 0.1, fa = 0.99;
    const int64_t nmin = 5;
    double dtmax = 10.0 * dt0, dt = dt0, a = a0;
    int64_t npos = 0;
    double rl = max_rcut(nt, rcut);
    int64_t cap = 64;
    int32_t* count = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * cap + 1));
    double* f = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* v = (double*)calloc((size_t)(3 * n + 1), sizeof(double));
    if (!count || !list || !f || !v) return -OR_ERR_OOM;
    int64_t it = 0;
    double fmax = 0.0;
    for (; it < maxit; ++it) {
        if (build_list(n, L, pos, rl, &count, &list, &cap) < 0) return -OR_ERR_OOM;
        or_forces_list(n, L, nt, type, pos, eps, sigma, rcut, 0, count, list,
                       cap, f, NULL, NULL);
        fmax = 0.0;
        double P = 0.0, vn = 0.0, fn = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double f2 = (f[3 * i] * f[3 * i] + f[3 * i + 1] * f[3 * i + 1]) +
                        f[3 * i + 2] * f[3 * i + 2];
            if (f2 > fmax) fmax = f2;
        }
        fmax = sqrt(fmax);
        if (fmax < ftol) break;
        for (int64_t q = 0; q < 3 * n; ++q) {
            P += f[q] * v[q];
            vn += v[q] * v[q];
            fn += f[q] * f[q];
        }
        vn = sqrt(vn);
        fn = sqrt(fn);
        if (P > 0.0) {
            for (int64_t q = 0; q < 3 * n; ++q)
                v[q] = (1.0 - a) * v[q] + a * vn * f[q] / fn;
            if (++npos > nmin) {
                dt = dt * finc < dtmax ? dt * finc : dtmax;
                a *= fa;
            }
        } else {
            for (int64_t q = 0; q < 3 * n; ++q) v[q] = 0.0;
            dt *= fdec;
            a = a0;
            npos = 0;
        }
        /* semi-implicit Euler step, displacement capped at 0.1 sigma */
        for (int64_t i = 0; i < n; ++i) {
            double dx[3];
            for (int c = 0; c < 3; ++c) {
                v[3 * i + c] += dt * f[3 * i + c];
                dx[c] = dt * v[3 * i + c];
            }
            double dn = sqrt((dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2]);
            double sc = dn > 0.1 ? 0.1 / dn : 1.0;
            for (int c = 0; c < 3; ++c) {
                double x = pos[3 * i + c] + sc * dx[c];
                pos[3 * i + c] = x - L[c] * floor(x / L[c]);
            }
        }
    }
    if (fmax_out) *fmax_out = fmax;
    free(count); free(list); free(f); free(v);
    return it;
}
