/*
 * oracle.c -- plain CPU reference ("oracle") for the short-range MD hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA library; the two meet only through the seeded
 * input generators (package `synth`) and the values they return.
 *
 * Everything here is the plain definition, in FP64, O(N^2) over all pairs
 * with the minimum-image convention in an orthorhombic periodic box whose
 * origin is 0 -- except the marked O(N) cell-list section, a second route to
 * the same LJ sums kept as the CPU baseline figure of an O(N) code (pinned
 * against the definition in the tests).  Loops over i may run in parallel (OpenMP) because every
 * per-atom quantity is written by the one thread that owns atom i; sums over
 * atoms are then taken sequentially in index order, so results do not depend
 * on the thread count.
 *
 * What the method computes (the paper, Trott/Winterfeld/Crozier,
 * "General-purpose molecular dynamics simulations on GPU-based clusters"):
 *   - pair forces summed over each atom's neighbour list (Sec. III.B, the
 *     thread-per-atom / block-per-atom listings): F_i = sum_j f(x_i, x_j);
 *   - the benchmark potentials of App. A: cut-off Lennard-Jones ("lj/cut")
 *     and EAM.  The paper prints neither formula; the LJ form is the textbook
 *     12-6 potential truncated at r_c, and the EAM form is the analytic
 *     Finnis-Sinclair variant fixed for the EAM workload:
 *         rho(r) = (rc - r)^2, F(rho) = -A sqrt(rho),
 *         phi(r) = (rc - r)^2 (c0 + c1 r + c2 r^2), all for r < rc;
 *   - NVE time integration on the GPU (Sec. II) -- velocity Verlet, the
 *     integrator of LAMMPS' "fix nve";
 *   - Verlet neighbour lists with a skin (Sec. III.B): the list of j with
 *     |x_i - x_j| < rc + skin, rebuilt once an atom has moved more than
 *     skin/2 since the last build.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - cut-off tests are strict: pair (i,j) interacts iff r^2 < rc^2, and is a
 *     list neighbour iff r^2 < (rc+skin)^2;
 *   - LJ energy is unshifted unless `shift` is set, then U(r) - U(rc);
 *   - EAM: F(0) = F'(0) = 0 (the square root is singular at rho = 0);
 *   - virial W_ab = sum_{i<j} d_a f_b with d = x_i - x_j (minimum image) and
 *     f the force on i due to j.
 *
 * Status codes: 0 ok, -1 invalid argument (box smaller than twice the
 * cut-off, non-positive sizes), -2 capacity exceeded.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* helpers                                                             */
/* ------------------------------------------------------------------ */

/* minimum-image separation along one axis of a periodic box of edge L */
static double min_image(double d, double L) { return d - L * floor(d / L + 0.5); }

/* d = x_i - x_j under the minimum image; returns |d|^2 */
static double separation(const double *x, int64_t i, int64_t j, const double box[3], double d[3]) {
    double r2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        d[a] = min_image(x[3 * i + a] - x[3 * j + a], box[a]);
        r2 += d[a] * d[a];
    }
    return r2;
}

static int box_ok(const double box[3], double rcut) {
    for (int a = 0; a < 3; ++a)
        if (!(box[a] >= 2.0 * rcut)) return 0;
    return 1;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Neighbour sets (Sec. III.B: numneigh[i], neighbors[i][jj])          */
/* ------------------------------------------------------------------ */

/*
 * Full neighbour sets of the atoms listed in `idx` (m of them; idx == NULL
 * means all n atoms in order): every j != i with r^2 < rl^2, ascending j.
 * counts[k] receives the set size of atom idx[k]; the sets are stored back to
 * back in nbr (CSR order), at most `cap` entries in total.
 * Returns the total number of entries, or -2 if cap was too small (counts are
 * still filled), -1 on bad input.
 */
int64_t oracle_neighbors(int64_t n, const double *x, const double box[3], double rl,
                         int64_t m, const int64_t *idx, int32_t *counts, int32_t *nbr, int64_t cap) {
    if (n <= 0 || rl <= 0.0 || !box_ok(box, rl)) return -1;
    if (idx == NULL) m = n;
    const double rl2 = rl * rl;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        int32_t c = 0;
        double d[3];
        for (int64_t j = 0; j < n; ++j)
            if (j != i && separation(x, i, j, box, d) < rl2) ++c;
        counts[k] = c;
    }
    int64_t total = 0;
    for (int64_t k = 0; k < m; ++k) total += counts[k];
    if (total > cap) return -2;
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
    if (!offs) return -1;
    offs[0] = 0;
    for (int64_t k = 0; k < m; ++k) offs[k + 1] = offs[k] + counts[k];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        int64_t p = offs[k];
        double d[3];
        for (int64_t j = 0; j < n; ++j)
            if (j != i && separation(x, i, j, box, d) < rl2) nbr[p++] = (int32_t)j;
    }
    free(offs);
    return total;
}

/*
 * Smallest | |x_i - x_j| - rl | over all pairs that involve one of the listed
 * atoms (idx == NULL: all atoms).  Used to certify that an input keeps every
 * pair away from the list radius, so that the list is unique.
 */
double oracle_min_gap(int64_t n, const double *x, const double box[3], double rl,
                      int64_t m, const int64_t *idx) {
    if (n <= 0 || !box_ok(box, rl)) return -1.0;
    if (idx == NULL) m = n;
    double best = INFINITY;
#pragma omp parallel for schedule(dynamic, 16) reduction(min : best)
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx ? idx[k] : k;
        double d[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double g = fabs(sqrt(separation(x, i, j, box, d)) - rl);
            if (g < best) best = g;
        }
    }
    return best;
}

/* ------------------------------------------------------------------ */
/* Lennard-Jones (App. A, "lj/cut")                                    */
/* ------------------------------------------------------------------ */

/* U(r) = 4 eps [(sig/r)^12 - (sig/r)^6] */
static double lj_energy(double r2, double eps, double sig) {
    double sr2 = sig * sig / r2;
    double sr6 = sr2 * sr2 * sr2;
    return 4.0 * eps * (sr6 * sr6 - sr6);
}

/* -U'(r)/r = 24 eps [2 (sig/r)^12 - (sig/r)^6] / r^2, so the force on i is this times d */
static double lj_force_over_r(double r2, double eps, double sig) {
    double sr2 = sig * sig / r2;
    double sr6 = sr2 * sr2 * sr2;
    return 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
}

/*
 * Forces, potential energy and virial of a (multi-type) LJ system.
 *   type[i] in [0, nt); eps, sig: nt*nt row-major, symmetric.
 *   f (n*3, may be NULL), energy (may be NULL), w6 = {xx,yy,zz,xy,xz,yz} (may be NULL).
 * E = sum_{i<j, r<rc} [U(r) - shift*U(rc)], F_i = sum_{j != i, r<rc} (-U'(r)/r) d_ij.
 */
int oracle_lj(int64_t n, const double *x, const int32_t *type, int32_t nt,
              const double *eps, const double *sig, const double box[3], double rc,
              int32_t shift, double *f, double *energy, double *w6) {
    if (n <= 0 || nt <= 0 || rc <= 0.0 || !box_ok(box, rc)) return -1;
    const double rc2 = rc * rc;
    double *e_i = (double *)calloc((size_t)n, sizeof(double));
    double *w_i = (double *)calloc((size_t)n * 6, sizeof(double));
    if (!e_i || !w_i) { free(e_i); free(w_i); return -1; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        double d[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = separation(x, i, j, box, d);
            if (!(r2 < rc2)) continue;
            int p = type[i] * nt + type[j];
            double s = lj_force_over_r(r2, eps[p], sig[p]);
            for (int a = 0; a < 3; ++a) fi[a] += s * d[a];
            if (j > i) { /* each unordered pair once for E and W */
                double u = lj_energy(r2, eps[p], sig[p]);
                if (shift) u -= lj_energy(rc2, eps[p], sig[p]);
                e_i[i] += u;
                double fv[3] = {s * d[0], s * d[1], s * d[2]};
                w_i[6 * i + 0] += d[0] * fv[0];
                w_i[6 * i + 1] += d[1] * fv[1];
                w_i[6 * i + 2] += d[2] * fv[2];
                w_i[6 * i + 3] += d[0] * fv[1];
                w_i[6 * i + 4] += d[0] * fv[2];
                w_i[6 * i + 5] += d[1] * fv[2];
            }
        }
        if (f) for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];
    }
    if (energy) { double e = 0.0; for (int64_t i = 0; i < n; ++i) e += e_i[i]; *energy = e; }
    if (w6) {
        for (int c = 0; c < 6; ++c) w6[c] = 0.0;
        for (int64_t i = 0; i < n; ++i) for (int c = 0; c < 6; ++c) w6[c] += w_i[6 * i + c];
    }
    free(e_i); free(w_i);
    return 0;
}

/*
 * LJ forces on the m atoms idx[k] only (each O(n)); for checking very large
 * systems one sampled atom at a time.  Also returns each atom's number of
 * interacting partners (r < rc) and its half-share of the pair energy.
 */
int oracle_lj_at(int64_t n, const double *x, const int32_t *type, int32_t nt,
                 const double *eps, const double *sig, const double box[3], double rc,
                 int32_t shift, int64_t m, const int64_t *idx, double *f, double *e_half, int32_t *ninter) {
    if (n <= 0 || nt <= 0 || rc <= 0.0 || !box_ok(box, rc)) return -1;
    const double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx[k];
        double fi[3] = {0.0, 0.0, 0.0}, e = 0.0, d[3];
        int32_t c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = separation(x, i, j, box, d);
            if (!(r2 < rc2)) continue;
            int p = type[i] * nt + type[j];
            double s = lj_force_over_r(r2, eps[p], sig[p]);
            for (int a = 0; a < 3; ++a) fi[a] += s * d[a];
            double u = lj_energy(r2, eps[p], sig[p]);
            if (shift) u -= lj_energy(rc2, eps[p], sig[p]);
            e += 0.5 * u;
            ++c;
        }
        for (int a = 0; a < 3; ++a) f[3 * k + a] = fi[a];
        if (e_half) e_half[k] = e;
        if (ninter) ninter[k] = c;
    }
    return 0;
}

/*
 * Vector-Jacobian product of the LJ forces (the backward pass of a
 * force-matching loss).  With L = sum_i g_i . F_i:
 *   dL/dx_k = sum_{j != k, r<rc} M_kj (g_k - g_j),
 *       M = dF_pair/dd = s(r) I + (s'(r)/r) d d^T,  s = -U'(r)/r;
 *   dL/deps_ab = sum_i sum_{j: {t_i,t_j} = {a,b}} g_i . f_ij / eps_ab,
 *   dL/dsig_ab = sum_i sum_{j: {t_i,t_j} = {a,b}} g_i . (ds/dsig) d.
 * eps_ab is ONE parameter shared by the (a,b) and (b,a) entries; both entries
 * of grad_eps / grad_sig receive dL/deps_ab.  grad_x (n*3) may be NULL;
 * grad_eps / grad_sig (nt*nt) may be NULL.
 */
int oracle_lj_vjp(int64_t n, const double *x, const int32_t *type, int32_t nt,
                  const double *eps, const double *sig, const double box[3], double rc,
                  const double *g, double *grad_x, double *grad_eps, double *grad_sig) {
    if (n <= 0 || nt <= 0 || rc <= 0.0 || !box_ok(box, rc)) return -1;
    const double rc2 = rc * rc;
    const int np = nt * nt;
    double *ge = (double *)calloc((size_t)n * np, sizeof(double));
    double *gs = (double *)calloc((size_t)n * np, sizeof(double));
    if (!ge || !gs) { free(ge); free(gs); return -1; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < n; ++k) {
        double acc[3] = {0.0, 0.0, 0.0}, d[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == k) continue;
            double r2 = separation(x, k, j, box, d);
            if (!(r2 < rc2)) continue;
            int p = type[k] * nt + type[j];
            double e = eps[p], sg = sig[p];
            double sg2 = sg * sg, sg6 = sg2 * sg2 * sg2, sg12 = sg6 * sg6;
            double ir2 = 1.0 / r2, ir6 = ir2 * ir2 * ir2, ir8 = ir6 * ir2, ir14 = ir6 * ir6 * ir2;
            double s = 24.0 * e * (2.0 * sg12 * ir14 - sg6 * ir8);
            double sp_over_r = 24.0 * e * (-28.0 * sg12 * ir14 * ir2 + 8.0 * sg6 * ir8 * ir2);
            double dg[3] = {g[3 * k] - g[3 * j], g[3 * k + 1] - g[3 * j + 1], g[3 * k + 2] - g[3 * j + 2]};
            double ddg = d[0] * dg[0] + d[1] * dg[1] + d[2] * dg[2];
            for (int a = 0; a < 3; ++a) acc[a] += s * dg[a] + sp_over_r * d[a] * ddg;
            double gd = g[3 * k] * d[0] + g[3 * k + 1] * d[1] + g[3 * k + 2] * d[2];
            /* unordered pair index: both (a,b) and (b,a) map to min/max */
            int ta = type[k] < type[j] ? type[k] : type[j];
            int tb = type[k] < type[j] ? type[j] : type[k];
            int q = ta * nt + tb;
            ge[(size_t)k * np + q] += gd * s / e;
            double ds_dsig = 24.0 * e * (24.0 * sg12 / sg * ir14 - 6.0 * sg6 / sg * ir8);
            gs[(size_t)k * np + q] += gd * ds_dsig;
        }
        if (grad_x) for (int a = 0; a < 3; ++a) grad_x[3 * k + a] = acc[a];
    }
    for (int q = 0; q < np; ++q) {
        double se = 0.0, ss = 0.0;
        for (int64_t k = 0; k < n; ++k) { se += ge[(size_t)k * np + q]; ss += gs[(size_t)k * np + q]; }
        int a = q / nt, b = q % nt;
        if (a > b) continue; /* filled from the (min,max) slot below */
        if (grad_eps) { grad_eps[a * nt + b] = se; grad_eps[b * nt + a] = se; }
        if (grad_sig) { grad_sig[a * nt + b] = ss; grad_sig[b * nt + a] = ss; }
    }
    free(ge); free(gs);
    return 0;
}

/* ------------------------------------------------------------------ */
/* EAM, Finnis-Sinclair analytic form (App. A "EAM"; form of the EAM   */
/* workload): p = {rc, A, c0, c1, c2}                                  */
/* ------------------------------------------------------------------ */

static double fs_rho(double r, double rc) { double t = rc - r; return t * t; }
static double fs_drho(double r, double rc) { return -2.0 * (rc - r); }
static double fs_phi(double r, const double *p) {
    double t = p[0] - r;
    return t * t * (p[2] + p[3] * r + p[4] * r * r);
}
static double fs_dphi(double r, const double *p) {
    double t = p[0] - r;
    return -2.0 * t * (p[2] + p[3] * r + p[4] * r * r) + t * t * (p[3] + 2.0 * p[4] * r);
}
static double fs_embed(double rho, double A) { return rho > 0.0 ? -A * sqrt(rho) : 0.0; }
static double fs_dembed(double rho, double A) { return rho > 0.0 ? -0.5 * A / sqrt(rho) : 0.0; }

/* host density of atom i: rho_i = sum_{j != i, r<rc} rho(r_ij) */
static double fs_density(int64_t n, const double *x, int64_t i, const double box[3], double rc) {
    double rho = 0.0, d[3];
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double r2 = separation(x, i, j, box, d);
        if (r2 < rc * rc) rho += fs_rho(sqrt(r2), rc);
    }
    return rho;
}

/*
 * E = sum_i F(rho_i) + sum_{i<j} phi(r_ij);
 * F_i = -sum_{j != i, r<rc} [phi'(r) + (F'(rho_i) + F'(rho_j)) rho'(r)] d_ij / r.
 * rho_out, fp_out (n each) may be NULL; f (n*3), energy, w6 may be NULL.
 */
int oracle_eam(int64_t n, const double *x, const double box[3], const double *p,
               double *f, double *energy, double *w6, double *rho_out, double *fp_out) {
    const double rc = p[0], A = p[1];
    if (n <= 0 || rc <= 0.0 || !box_ok(box, rc)) return -1;
    const double rc2 = rc * rc;
    double *rho = (double *)malloc(sizeof(double) * (size_t)n);
    double *fp = (double *)malloc(sizeof(double) * (size_t)n);
    double *e_i = (double *)calloc((size_t)n, sizeof(double));
    double *w_i = (double *)calloc((size_t)n * 6, sizeof(double));
    if (!rho || !fp || !e_i || !w_i) { free(rho); free(fp); free(e_i); free(w_i); return -1; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        rho[i] = fs_density(n, x, i, box, rc);
        fp[i] = fs_dembed(rho[i], A);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0}, d[3];
        double e = fs_embed(rho[i], A);
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = separation(x, i, j, box, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            double c = -(fs_dphi(r, p) + (fp[i] + fp[j]) * fs_drho(r, rc)) / r;
            for (int a = 0; a < 3; ++a) fi[a] += c * d[a];
            if (j > i) {
                e += fs_phi(r, p);
                w_i[6 * i + 0] += d[0] * c * d[0];
                w_i[6 * i + 1] += d[1] * c * d[1];
                w_i[6 * i + 2] += d[2] * c * d[2];
                w_i[6 * i + 3] += d[0] * c * d[1];
                w_i[6 * i + 4] += d[0] * c * d[2];
                w_i[6 * i + 5] += d[1] * c * d[2];
            }
        }
        e_i[i] = e;
        if (f) for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];
    }
    if (energy) { double e = 0.0; for (int64_t i = 0; i < n; ++i) e += e_i[i]; *energy = e; }
    if (w6) {
        for (int c = 0; c < 6; ++c) w6[c] = 0.0;
        for (int64_t i = 0; i < n; ++i) for (int c = 0; c < 6; ++c) w6[c] += w_i[6 * i + c];
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    if (fp_out) memcpy(fp_out, fp, sizeof(double) * (size_t)n);
    free(rho); free(fp); free(e_i); free(w_i);
    return 0;
}

/*
 * EAM forces (and host densities) on the m atoms idx[k] only.  Each needs
 * rho of the atom and of every partner, each O(n): O(n * partners) per atom.
 */
int oracle_eam_at(int64_t n, const double *x, const double box[3], const double *p,
                  int64_t m, const int64_t *idx, double *f, double *rho_out) {
    const double rc = p[0], A = p[1];
    if (n <= 0 || rc <= 0.0 || !box_ok(box, rc)) return -1;
    const double rc2 = rc * rc;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx[k];
        double rho_i = fs_density(n, x, i, box, rc);
        double fp_i = fs_dembed(rho_i, A);
        double fx = 0.0, fy = 0.0, fz = 0.0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : fx, fy, fz)
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            double r2 = separation(x, i, j, box, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            double fp_j = fs_dembed(fs_density(n, x, j, box, rc), A);
            double c = -(fs_dphi(r, p) + (fp_i + fp_j) * fs_drho(r, rc)) / r;
            fx += c * d[0]; fy += c * d[1]; fz += c * d[2];
        }
        f[3 * k] = fx; f[3 * k + 1] = fy; f[3 * k + 2] = fz;
        if (rho_out) rho_out[k] = rho_i;
    }
    return 0;
}

/*
 * Backward of the EAM forces for the loss L = sum_i g_i . F_i (the
 * vector-Jacobian product that force matching needs; the forward is
 * oracle_eam).  Derivation, with d = x_i - x_j, r = |d|, u = d / r,
 * G = g_i - g_j, w = G . u, and per pair
 *     s = phi'(r) + (F'_i + F'_j) rho'(r)      so that F_i = -sum_j s u,
 *     k = phi''(r) + (F'_i + F'_j) rho''(r)    (ds/dr with F' held fixed):
 *   1. L depends on F'_m explicitly through s: dL/dF'_m = -lambda_m with
 *      lambda_m = sum_j w_mj rho'(r_mj);
 *   2. F'_m depends on rho_m: dL/drho_m = -mu_m, mu_m = lambda_m F''(rho_m);
 *   3. positions, through s and u at fixed F', and through every rho:
 *      dL/dx_i = -sum_j [ (s/r) G + w (k - s/r) u + (mu_i + mu_j) rho'(r) u ];
 *   4. parameters: dL/dA = -sum_m lambda_m dF'_m/dA with dF'/dA = -1/(2 sqrt(rho)),
 *      dL/dc_q = -sum_i sum_j (g_i . u) d phi'(r)/dc_q.
 * grad_p has the layout of p; its cut-off slot grad_p[0] is not a
 * derivative (the cut-off is not differentiated) and is written as 0.
 * g, grad_x: n*3.  grad_x or grad_p may be NULL.
 */
static double fs_d2phi(double r, const double *p) {
    double t = p[0] - r;
    return 2.0 * (p[2] + p[3] * r + p[4] * r * r) - 4.0 * t * (p[3] + 2.0 * p[4] * r) + t * t * 2.0 * p[4];
}
static double fs_d2rho(void) { return 2.0; }
static double fs_d2embed(double rho, double A) { return rho > 0.0 ? 0.25 * A / (rho * sqrt(rho)) : 0.0; }
static double fs_dembed_dA(double rho) { return rho > 0.0 ? -0.5 / sqrt(rho) : 0.0; }
/* d phi'(r) / d c_q for q = 0, 1, 2 */
static void fs_dphi_dc(double r, double rc, double out[3]) {
    double t = rc - r;
    out[0] = -2.0 * t;
    out[1] = -2.0 * t * r + t * t;
    out[2] = -2.0 * t * r * r + 2.0 * r * t * t;
}

int oracle_eam_vjp(int64_t n, const double *x, const double box[3], const double *p, const double *g,
                   double *grad_x, double *grad_p) {
    const double rc = p[0], A = p[1];
    if (n <= 0 || rc <= 0.0 || !box_ok(box, rc)) return -1;
    const double rc2 = rc * rc;
    double *rho = (double *)malloc(sizeof(double) * (size_t)n);
    double *fp = (double *)malloc(sizeof(double) * (size_t)n);
    double *lam = (double *)malloc(sizeof(double) * (size_t)n);
    double *mu = (double *)malloc(sizeof(double) * (size_t)n);
    double *gc_i = (double *)calloc((size_t)n * 3, sizeof(double));
    if (!rho || !fp || !lam || !mu || !gc_i) { free(rho); free(fp); free(lam); free(mu); free(gc_i); return -1; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        rho[i] = fs_density(n, x, i, box, rc);
        fp[i] = fs_dembed(rho[i], A);
    }
    /* step 1: lambda_i = sum_j ((g_i - g_j) . u_ij) rho'(r_ij) */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double l = 0.0, d[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = separation(x, i, j, box, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2), w = 0.0;
            for (int a = 0; a < 3; ++a) w += (g[3 * i + a] - g[3 * j + a]) * d[a] / r;
            l += w * fs_drho(r, rc);
        }
        lam[i] = l;
    }
    /* step 2 */
    for (int64_t i = 0; i < n; ++i) mu[i] = lam[i] * fs_d2embed(rho[i], A);
    /* steps 3 and 4 (c part) */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0}, d[3];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double r2 = separation(x, i, j, box, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2), u[3], G[3], w = 0.0, gu = 0.0;
            for (int a = 0; a < 3; ++a) {
                u[a] = d[a] / r;
                G[a] = g[3 * i + a] - g[3 * j + a];
                w += G[a] * u[a];
                gu += g[3 * i + a] * u[a];
            }
            double s = fs_dphi(r, p) + (fp[i] + fp[j]) * fs_drho(r, rc);
            double k = fs_d2phi(r, p) + (fp[i] + fp[j]) * fs_d2rho();
            double emb = (mu[i] + mu[j]) * fs_drho(r, rc);
            for (int a = 0; a < 3; ++a) acc[a] -= (s / r) * G[a] + w * (k - s / r) * u[a] + emb * u[a];
            double dc[3];
            fs_dphi_dc(r, rc, dc);
            for (int q = 0; q < 3; ++q) gc_i[3 * i + q] -= gu * dc[q];
        }
        if (grad_x) for (int a = 0; a < 3; ++a) grad_x[3 * i + a] = acc[a];
    }
    if (grad_p) {
        double gA = 0.0, gc[3] = {0.0, 0.0, 0.0};
        for (int64_t i = 0; i < n; ++i) {
            gA -= lam[i] * fs_dembed_dA(rho[i]);
            for (int q = 0; q < 3; ++q) gc[q] += gc_i[3 * i + q];
        }
        grad_p[0] = 0.0;
        grad_p[1] = gA;
        for (int q = 0; q < 3; ++q) grad_p[2 + q] = gc[q];
    }
    free(rho); free(fp); free(lam); free(mu); free(gc_i);
    return 0;
}

/* ------------------------------------------------------------------ */
/* O(N) cell-list CPU baseline (not the oracle's definition)           */
/* ------------------------------------------------------------------ */
/*
 * A plain cell-list evaluation of the same single-type LJ forces, for the
 * CPU baseline figure that an O(N) CPU code would give (the O(N^2) loops
 * above are the definition; this is a second route to the same sums, pinned
 * against them in the tests).  Cells of edge >= rc, at least 3 per axis (so
 * the 27 neighbour cells are distinct); atoms counting-sorted into cells;
 * each atom sums over the atoms of its 27 neighbour cells, minimum image per
 * pair.  Loops over atoms run in parallel; each atom's force is written by
 * its own thread.  Returns -1 if the box is too small for 3 cells of rc.
 */
typedef struct { int nb[3]; double inv[3]; int *start, *order; } cells_t;

static int cells_build(int64_t n, const double *x, const double box[3], double rc, cells_t *c) {
    for (int a = 0; a < 3; ++a) {
        c->nb[a] = (int)floor(box[a] / rc);
        if (c->nb[a] < 3) return -1;
        c->inv[a] = c->nb[a] / box[a];
    }
    const int64_t nc = (int64_t)c->nb[0] * c->nb[1] * c->nb[2];
    int *cell = (int *)malloc(sizeof(int) * (size_t)n);
    c->start = (int *)calloc((size_t)nc + 1, sizeof(int));
    c->order = (int *)malloc(sizeof(int) * (size_t)n);
    if (!cell || !c->start || !c->order) { free(cell); free(c->start); free(c->order); return -1; }
    for (int64_t i = 0; i < n; ++i) {
        int b[3];
        for (int a = 0; a < 3; ++a) {
            double w = x[3 * i + a] - box[a] * floor(x[3 * i + a] / box[a]);
            b[a] = (int)(w * c->inv[a]);
            if (b[a] >= c->nb[a]) b[a] = c->nb[a] - 1;
            if (b[a] < 0) b[a] = 0;
        }
        cell[i] = (b[2] * c->nb[1] + b[1]) * c->nb[0] + b[0];
        c->start[cell[i] + 1]++;
    }
    for (int64_t k = 0; k < nc; ++k) c->start[k + 1] += c->start[k];
    int *fill = (int *)malloc(sizeof(int) * (size_t)nc);
    if (!fill) { free(cell); free(c->start); free(c->order); return -1; }
    memcpy(fill, c->start, sizeof(int) * (size_t)nc);
    for (int64_t i = 0; i < n; ++i) c->order[fill[cell[i]]++] = (int)i;
    free(fill);
    free(cell);
    return 0;
}

static void cells_free(cells_t *c) { free(c->start); free(c->order); }

static void lj_cells_forces(int64_t n, const double *x, const double box[3], double rc, const cells_t *c,
                            double *f) {
    const double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        int b[3];
        for (int a = 0; a < 3; ++a) {
            double w = x[3 * i + a] - box[a] * floor(x[3 * i + a] / box[a]);
            b[a] = (int)(w * c->inv[a]);
            if (b[a] >= c->nb[a]) b[a] = c->nb[a] - 1;
            if (b[a] < 0) b[a] = 0;
        }
        double fi[3] = {0.0, 0.0, 0.0}, d[3];
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int q[3] = {b[0] + dx, b[1] + dy, b[2] + dz};
                    for (int a = 0; a < 3; ++a) q[a] = (q[a] + c->nb[a]) % c->nb[a];
                    const int k = (q[2] * c->nb[1] + q[1]) * c->nb[0] + q[0];
                    for (int s = c->start[k]; s < c->start[k + 1]; ++s) {
                        const int j = c->order[s];
                        if (j == i) continue;
                        const double r2 = separation(x, i, j, box, d);
                        if (!(r2 < rc2)) continue;
                        const double sc = lj_force_over_r(r2, 1.0, 1.0);
                        for (int a = 0; a < 3; ++a) fi[a] += sc * d[a];
                    }
                }
        for (int a = 0; a < 3; ++a) f[3 * i + a] = fi[a];
    }
}

/* single-type LJ (eps = sigma = 1) forces by cell lists */
int oracle_lj_cells(int64_t n, const double *x, const double box[3], double rc, double *f) {
    if (n <= 0 || rc <= 0.0) return -1;
    cells_t c;
    if (cells_build(n, x, box, rc, &c)) return -1;
    lj_cells_forces(n, x, box, rc, &c, f);
    cells_free(&c);
    return 0;
}

/* velocity-Verlet NVE (mass m) with cell-list forces, cells rebuilt every step;
 * f (n*3) holds the forces of x on entry (computed here if `have_f` is 0) and
 * of the final x on return */
int oracle_nve_cells(int64_t n, double *x, double *v, const double box[3], double rc, double dt, double m,
                     int64_t nsteps, double *f, int32_t have_f) {
    if (n <= 0 || nsteps < 0) return -1;
    if (!have_f && oracle_lj_cells(n, x, box, rc, f)) return -1;
    const double hk = 0.5 * dt / m;
    for (int64_t s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                v[3 * i + a] += hk * f[3 * i + a];
                x[3 * i + a] += dt * v[3 * i + a];
            }
        if (oracle_lj_cells(n, x, box, rc, f)) return -1;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) v[3 * i + a] += hk * f[3 * i + a];
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Kinetic energy and velocity-Verlet NVE (Sec. II)                    */
/* ------------------------------------------------------------------ */

/* KE = sum_i m_i v_i^2 / (2 ftm2v): ftm2v converts force/mass to acceleration */
double oracle_kinetic(int64_t n, const double *v, const int32_t *type, const double *mass, double ftm2v) {
    double ke = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double m = mass[type[i]];
        ke += 0.5 * m * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]) / ftm2v;
    }
    return ke;
}

/*
 * Velocity-Verlet NVE for `nsteps` steps with forces from the LJ (pot = 0,
 * params = eps[nt*nt] then sig[nt*nt]) or the EAM (pot = 1, params = {rc, A,
 * c0, c1, c2}) definitions above:
 *     v += (dt/2) a(x);  x += dt v;  [list check];  v += (dt/2) a(x_new),
 * with a = ftm2v F / m.  x, v (n*3) are advanced in place; f (n*3) returns
 * the final forces.  Positions are not wrapped (the minimum image makes the
 * forces independent of wrapping).
 * The list policy is tracked for reference: after each drift, if any atom is
 * farther than skin/2 from its position at the last build, a rebuild is
 * counted there and the build positions reset.  The forces never use a list
 * (all pairs are examined), so the trajectory does not depend on this policy.
 * epot / ekin (nsteps+1 each, may be NULL) record the energies at every step.
 * Returns the number of rebuilds, or -1.
 */
int64_t oracle_nve(int64_t n, double *x, double *v, const int32_t *type, int32_t nt,
                   const double *mass, double ftm2v, const double box[3], int32_t pot,
                   const double *params, double rc, int32_t shift, double skin, double dt,
                   int64_t nsteps, double *f, double *epot, double *ekin) {
    if (n <= 0 || nsteps < 0) return -1;
    double *xb = (double *)malloc(sizeof(double) * (size_t)n * 3);
    if (!xb) return -1;
    memcpy(xb, x, sizeof(double) * (size_t)n * 3);
    const double *eps = params, *sig = params + nt * nt;
    int rc_ok;
    double e;
#define ORACLE_FORCES()                                                             \
    (pot == 0 ? oracle_lj(n, x, type, nt, eps, sig, box, rc, shift, f, &e, NULL)    \
              : oracle_eam(n, x, box, params, f, &e, NULL, NULL, NULL))
    rc_ok = ORACLE_FORCES();
    if (rc_ok) { free(xb); return -1; }
    if (epot) epot[0] = e;
    if (ekin) ekin[0] = oracle_kinetic(n, v, type, mass, ftm2v);
    int64_t rebuilds = 0;
    const double half2 = 0.25 * skin * skin;
    for (int64_t s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < n; ++i) {
            double a = ftm2v / mass[type[i]];
            for (int c = 0; c < 3; ++c) {
                v[3 * i + c] += 0.5 * dt * a * f[3 * i + c];
                x[3 * i + c] += dt * v[3 * i + c];
            }
        }
        double dmax2 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double d2 = 0.0;
            for (int c = 0; c < 3; ++c) { double t = x[3 * i + c] - xb[3 * i + c]; d2 += t * t; }
            if (d2 > dmax2) dmax2 = d2;
        }
        if (dmax2 > half2) { ++rebuilds; memcpy(xb, x, sizeof(double) * (size_t)n * 3); }
        rc_ok = ORACLE_FORCES();
        if (rc_ok) { free(xb); return -1; }
        for (int64_t i = 0; i < n; ++i) {
            double a = ftm2v / mass[type[i]];
            for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt * a * f[3 * i + c];
        }
        if (epot) epot[s] = e;
        if (ekin) ekin[s] = oracle_kinetic(n, v, type, mass, ftm2v);
    }
#undef ORACLE_FORCES
    free(xb);
    return rebuilds;
}
