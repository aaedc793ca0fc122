/*
 * FP64 CPU oracle for the Voronoi-cell-list CGMD hot path of OpenRBC
 * (arXiv 1701.02059).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA product path
 * never calls it, and it shares no code, header or constant table with it.
 *
 * Plain, slow, obviously correct: every quantity in double precision,
 * compiled with -ffp-contract=off so that no multiply-add is fused, loops in
 * the order the paper states them.  OpenMP only splits independent
 * per-particle or per-cell work; every sum that mixes particles is taken in
 * a fixed serial order.
 *
 * What each part follows (paper sections):
 *   - Voronoi cell = set of points whose closest centroid (L2, minimum image)
 *     is that centroid ("Spatial Searching Algorithm", Voronoi definition);
 *     the k-d tree search with the previous particle's centroid as the
 *     initial guess is the paper's own search structure (same section).
 *   - k-means initial clustering followed by an EM update of centroid
 *     location and ownership, then the two-level reorder: centroids along a
 *     Morton curve, particles by cell ("Spatial Searching Algorithm",
 *     two-step procedure).
 *   - Quad loop over cell, neighbouring cell, particle, particle, reusing the
 *     lipid cells with a wider cutoff for proteins, bond list for linked
 *     proteins ("Force Evaluation").
 *   - Newton's 3rd law half-list versus per-particle double computation
 *     ("Force Evaluation", patch decomposition): both are provided so tests
 *     can check they agree.
 *   - Time stepping: force and torque, then position and orientation update
 *     ("Software Overview", flow chart).
 *   - Harmonic volume constraint and the upper-rim height map for the
 *     membrane fluctuation ("Validation and Benchmark", the whole-cell run):
 *     readings V1, V2 and H1 beside the code.
 *
 * Readings where the paper is silent (pair potential, integrator, cell
 * adjacency rule, tie-breaks, fixed-point scales) are stated beside the code
 * that implements them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_LIPID 0
#define OR_BAND3 3
#define OR_GLYCOPHORIN 4

/* Reading P1 (the two-component model's membrane proteins: the paper places
 * band-3 and glycophorin particles in the membrane, "Initial structure
 * generation", but prints none of the cited model's constants): band-3 and
 * glycophorin sit in the bilayer and carry a director like the lipids; any
 * two bilayer particles interact through the lipid potential with the well
 * depth and cutoff of their species pair (lipid, band-3, glycophorin), all
 * other constants shared.  With every pair at the lipid-lipid values a
 * membrane protein is a lipid with another label. */
static inline int or_membrane(int t) { return t == OR_LIPID || t == OR_BAND3 || t == OR_GLYCOPHORIN; }
static inline int or_species(int t) { return t == OR_BAND3 ? 1 : (t == OR_GLYCOPHORIN ? 2 : 0); }

/* ---------------------------------------------------------------- model */

typedef struct {
    double eps;          /* lipid-lipid well depth                       */
    double rmin;         /* lipid-lipid potential minimum (2^(1/6) sigma) */
    double rc;           /* lipid-lipid cutoff                           */
    double mu;           /* orientation coupling                          */
    double sin_theta0;   /* spontaneous-curvature angle                   */
    int    zeta;         /* attractive-tail exponent (cos^(2 zeta))       */
    int    pad0;
    double eps_wca;      /* protein excluded-volume strength              */
    double sigma_wca;    /* lipid-protein excluded-volume size            */
    double sigma_pp;     /* protein-protein excluded-volume size          */
    double box[3];
    int    periodic[3];
    int    pad1;
    double mem_eps[9];   /* bilayer species pairs [3 s_i + s_j]: well depth */
    double mem_rc[9];    /* ... and cutoff (the lipid-lipid pair: eps, rc)  */
} or_model;

/* 2^(1/6), correctly rounded. */
static const double OR_TWO_SIXTH = 1.122462048309373;

static double or_wca_cut(const or_model* m) { return OR_TWO_SIXTH * m->sigma_wca; }
static double or_wca_pp_cut(const or_model* m) { return OR_TWO_SIXTH * m->sigma_pp; }

/* Search cutoff: the widest type-pair cutoff. */
double or_search_cutoff(const or_model* m)
{
    double a = m->rc, b = or_wca_cut(m), c = or_wca_pp_cut(m);
    double r = a > b ? a : b;
    r = r > c ? r : c;
    for (int q = 0; q < 9; q++) r = m->mem_rc[q] > r ? m->mem_rc[q] : r;
    return r;
}

/* Minimum image along one axis: d - L * rint(d / L). */
static inline double or_minimg(double d, double L, int per)
{
    if (!per) return d;
    double q = d / L;
    double r = rint(q);
    double p = L * r;
    return d - p;
}

/* Squared distance, evaluated as ((dx*dx + dy*dy) + dz*dz), with the
 * displacement a - b under the minimum image. */
static inline double or_dist2(const double* a, const double* b, const double* box, const int* per,
                              double d[3])
{
    for (int k = 0; k < 3; k++) d[k] = or_minimg(a[k] - b[k], box[k], per[k]);
    double s = d[0] * d[0];
    s = s + d[1] * d[1];
    s = s + d[2] * d[2];
    return s;
}

/* Wrap into [0, L) on a periodic axis. */
static inline double or_wrap(double c, double L, int per)
{
    if (!per) return c;
    double t = c / L;
    double f = floor(t);
    double p = L * f;
    double w = c - p;
    if (w < 0.0) w = w + L;
    if (w >= L) w = w - L;
    return w;
}

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
 * SC'11): ten rounds of two 32x32->64 multiplies with the key bumped by the
 * Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (r < 9) { k0 += W0; k1 += W1; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Unit-variance uniform noise from one 32-bit word:
 * u = (w + 1/2) 2^-32 in (0,1), xi = sqrt(12) (u - 1/2). */
static const double OR_SQRT12 = 3.4641016151377544;
static inline double or_uniform_noise(uint32_t w)
{
    double u = ((double)w + 0.5) * 2.3283064365386963e-10;
    return OR_SQRT12 * (u - 0.5);
}

/* Noise triple for (seed, instance; particle id, step, substream). */
void or_noise3(uint64_t seed, uint32_t instance, uint32_t id, uint64_t step, uint32_t sub, double xi[3])
{
    uint32_t ctr[4] = { id, (uint32_t)step, (uint32_t)(step >> 32), sub };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) ^ instance };
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    for (int k = 0; k < 3; k++) xi[k] = or_uniform_noise(w[k]);
}

/* ---------------------------------------------------------------- pair terms */

static inline double dot3(const double* a, const double* b)
{
    double s = a[0] * b[0];
    s = s + a[1] * b[1];
    s = s + a[2] * b[2];
    return s;
}
static inline void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/*
 * Lipid-lipid orientation-dependent pair potential of the one-particle-thick
 * membrane model (Yuan, Huang, Li, Lykotrafitis & Zhang, PRE 82, 011905,
 * 2010), on which the two-component red-cell model the paper simulates
 * builds.  With r_ij = x_i - x_j, r = |r_ij|, rh = r_ij / r:
 *   a   = (n_i x rh).(n_j x rh) + s0 (n_j - n_i).rh - s0^2,  s0 = sin(theta0)
 *   phi = 1 + mu (a - 1)
 *   U   = u_R(r) + (1 - phi) eps                 r <  rmin
 *   U   = u_A(r) phi                             rmin <= r < rc
 *   u_R = eps [(rmin/r)^4 - 2 (rmin/r)^2]
 *   u_A = -eps cos^(2 zeta)( (pi/2)(r - rmin)/(rc - rmin) )
 * Written as U = f(r) + g(r) phi.  Returns U; force on i (force on j is its
 * negative) and the torques n x (-dU/dn) on i and j.
 *
 * d is x_j - x_i (minimum image), as produced by the pair search.
 */
double or_lipid_pair(const or_model* m, const double d[3], double r2, const double* ni, const double* nj,
                     double Fi[3], double Ti[3], double Tj[3])
{
    double r = sqrt(r2);
    double rh[3] = { -d[0] / r, -d[1] / r, -d[2] / r };
    double s0 = m->sin_theta0;
    double nin = dot3(ni, nj), nir = dot3(ni, rh), njr = dot3(nj, rh);
    double a = nin - nir * njr + s0 * (njr - nir) - s0 * s0;
    double phi = 1.0 + m->mu * (a - 1.0);
    double f, fp, g, gp;
    if (r < m->rmin) {
        double q = m->rmin / r;
        double q2 = q * q, q4 = q2 * q2;
        f = m->eps * (q4 - 2.0 * q2) + m->eps;
        fp = m->eps * (-4.0 * q4 / r + 4.0 * q2 / r);
        g = -m->eps;
        gp = 0.0;
    } else {
        double w = (M_PI / 2.0) / (m->rc - m->rmin);
        double th = w * (r - m->rmin);
        double c = cos(th), s = sin(th);
        double cp = 1.0;                       /* c^(2 zeta - 1) */
        for (int k = 0; k < 2 * m->zeta - 1; k++) cp = cp * c;
        f = 0.0;
        fp = 0.0;
        g = -m->eps * cp * c;
        gp = m->eps * (double)(2 * m->zeta) * cp * s * w;
    }
    double U = f + g * phi;
    /* da/drh = -(n_j.rh) n_i - (n_i.rh) n_j + s0 (n_j - n_i) */
    double w3[3];
    for (int k = 0; k < 3; k++) w3[k] = -njr * ni[k] - nir * nj[k] + s0 * (nj[k] - ni[k]);
    double wr = dot3(w3, rh);
    double radial = fp + gp * phi;
    double gm = g * m->mu;
    for (int k = 0; k < 3; k++) {
        double wperp = w3[k] - wr * rh[k];
        Fi[k] = -radial * rh[k] - gm * wperp / r;
    }
    /* da/dn_i = n_j - (n_j.rh) rh - s0 rh ; da/dn_j = n_i - (n_i.rh) rh + s0 rh */
    double gi[3], gj[3], ci[3], cj[3];
    for (int k = 0; k < 3; k++) {
        gi[k] = nj[k] - njr * rh[k] - s0 * rh[k];
        gj[k] = ni[k] - nir * rh[k] + s0 * rh[k];
    }
    cross3(ni, gi, ci);
    cross3(nj, gj, cj);
    for (int k = 0; k < 3; k++) {
        Ti[k] = -gm * ci[k];
        Tj[k] = -gm * cj[k];
    }
    return U;
}

/* Purely repulsive Weeks-Chandler-Andersen term for every pair that is not
 * lipid-lipid: 4 e [(s/r)^12 - (s/r)^6] + e for r < 2^(1/6) s, with
 * s = sigma_wca for lipid-protein pairs and s = sigma_pp for
 * protein-protein pairs.  Reading: the workloads' spectrin chains (bond
 * lengths 0.45-1 sigma, several chains meeting at each junction) put beads
 * of neighbouring chains ~0.7 sigma apart, so the protein-protein size is a
 * parameter of its own. */
double or_wca_pair_s(const or_model* m, double sig, const double d[3], double r2, double Fi[3])
{
    double s2 = sig * sig / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double U = 4.0 * m->eps_wca * (s12 - s6) + m->eps_wca;
    /* -dU/dr / r, force on i along r_ij = -d */
    double fr = 4.0 * m->eps_wca * (12.0 * s12 - 6.0 * s6) / r2;
    for (int k = 0; k < 3; k++) Fi[k] = -fr * d[k];
    return U;
}

double or_wca_pair(const or_model* m, const double d[3], double r2, double Fi[3])
{
    return or_wca_pair_s(m, m->sigma_wca, d, r2, Fi);
}

/* Two bilayer particles (reading P1): the lipid potential with the well
 * depth and cutoff of their species pair. */
double or_membrane_pair(const or_model* m, int si, int sj, const double d[3], double r2, const double* ni,
                        const double* nj, double Fi[3], double Ti[3], double Tj[3])
{
    or_model q = *m;
    q.eps = m->mem_eps[3 * si + sj];
    q.rc = m->mem_rc[3 * si + sj];
    return or_lipid_pair(&q, d, r2, ni, nj, Fi, Ti, Tj);
}

/* Cutoff of a type pair: the species pair's for two bilayer particles, the
 * WCA range for a bilayer particle and a cytoskeleton protein, the
 * protein-protein WCA range for two cytoskeleton proteins. */
static inline double or_pair_cut(const or_model* m, int ti, int tj)
{
    if (or_membrane(ti) && or_membrane(tj)) return m->mem_rc[3 * or_species(ti) + or_species(tj)];
    if (or_membrane(ti) || or_membrane(tj)) return or_wca_cut(m);
    return or_wca_pp_cut(m);
}

/* Full pair evaluation for a type pair (no exclusion test). */
double or_pair_terms(const or_model* m, int ti, int tj, const double d[3], double r2,
                     const double* ni, const double* nj, double Fi[3], double Ti[3], double Tj[3])
{
    if (or_membrane(ti) && or_membrane(tj))
        return or_membrane_pair(m, or_species(ti), or_species(tj), d, r2, ni, nj, Fi, Ti, Tj);
    for (int k = 0; k < 3; k++) { Ti[k] = 0.0; Tj[k] = 0.0; }
    double sig = (or_membrane(ti) || or_membrane(tj)) ? m->sigma_wca : m->sigma_pp;
    return or_wca_pair_s(m, sig, d, r2, Fi);
}

/* Harmonic bond 1/2 kb (r - r0)^2; d = x_b - x_a; returns U and force on a. */
double or_bond_pair(const double d[3], double kb, double r0, double Fa[3])
{
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double dr = r - r0;
    double c = kb * dr / r;
    for (int k = 0; k < 3; k++) Fa[k] = c * d[k];
    return 0.5 * kb * dr * dr;
}

/* ---------------------------------------------------------------- bonded-exclusion lookup */

typedef struct {
    int n;             /* number of particle ids                 */
    int* ptr;          /* CSR over ids                           */
    int* nbr;          /* partner ids, ascending within a row    */
} or_bondmap;

static int or_int_cmp(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

static void or_bondmap_build(or_bondmap* bm, int n_ids, int nb, const int* ij)
{
    bm->n = n_ids;
    bm->ptr = (int*)calloc((size_t)n_ids + 1, sizeof(int));
    bm->nbr = (int*)malloc(sizeof(int) * (size_t)(2 * nb + 1));
    for (int b = 0; b < nb; b++) { bm->ptr[ij[2 * b] + 1]++; bm->ptr[ij[2 * b + 1] + 1]++; }
    for (int i = 0; i < n_ids; i++) bm->ptr[i + 1] += bm->ptr[i];
    int* fill = (int*)calloc((size_t)n_ids, sizeof(int));
    for (int b = 0; b < nb; b++) {
        int a = ij[2 * b], c = ij[2 * b + 1];
        bm->nbr[bm->ptr[a] + fill[a]++] = c;
        bm->nbr[bm->ptr[c] + fill[c]++] = a;
    }
    free(fill);
    for (int i = 0; i < n_ids; i++) qsort(bm->nbr + bm->ptr[i], (size_t)(bm->ptr[i + 1] - bm->ptr[i]), sizeof(int), or_int_cmp);
}

static void or_bondmap_free(or_bondmap* bm)
{
    free(bm->ptr); free(bm->nbr);
    bm->ptr = bm->nbr = NULL;
}

/* Reading of the bonded exclusions (the paper keeps a bond list for linked
 * proteins but states no non-bonded exclusion rule): pairs that are bonded
 * (1-2) or share a bond partner (1-3) carry no excluded-volume term, as in
 * bead-spring chain models; chains of 0.55 sigma bonds meeting at a junction
 * would otherwise start inside each other's repulsive core. */
static inline int or_excluded(const or_bondmap* bm, int ida, int idb)
{
    if (!bm || !bm->ptr) return 0;
    for (int q = bm->ptr[ida]; q < bm->ptr[ida + 1]; q++) {
        int c = bm->nbr[q];
        if (c == idb) return 1;
        for (int w = bm->ptr[idb]; w < bm->ptr[idb + 1]; w++)
            if (bm->nbr[w] == c) return 1;
    }
    return 0;
}

/* Does pair (i, j) interact?  Strict FP64 inclusion d^2 < rc^2 with the
 * type-pair cutoff; 1-2 and 1-3 bonded pairs are excluded from the
 * excluded-volume term (the cytoskeleton's chains, and a membrane protein
 * anchored to them: reading P3); two bilayer particles never are. */
static inline int or_interacts(const or_model* m, const or_bondmap* bm, int ti, int tj, int idi, int idj,
                               double r2)
{
    double rc = or_pair_cut(m, ti, tj);
    if (!(r2 < rc * rc)) return 0;
    if (!(or_membrane(ti) && or_membrane(tj)) && or_excluded(bm, idi, idj)) return 0;
    return 1;
}

/* ---------------------------------------------------------------- brute-force pair search */

/* All interacting pairs (i < j, storage indices), O(N^2).  Writes up to cap
 * pairs; returns the total count. */
long long or_pairs_brute(const or_model* m, int n, const double* x, const unsigned char* type,
                         const unsigned* id, int nb, const int* bonds, long long cap, int* pairs)
{
    or_bondmap bm = {0};
    int maxid = 0;
    for (int i = 0; i < n; i++) if ((int)id[i] > maxid) maxid = (int)id[i];
    if (nb > 0) or_bondmap_build(&bm, maxid + 1, nb, bonds);
    long long cnt = 0;
    for (int i = 0; i < n; i++) {
        for (int j = i + 1; j < n; j++) {
            double d[3];
            double r2 = or_dist2(x + 3 * j, x + 3 * i, m->box, m->periodic, d);
            if (or_interacts(m, nb > 0 ? &bm : NULL, type[i], type[j], (int)id[i], (int)id[j], r2)) {
                if (cnt < cap) { pairs[2 * cnt] = i; pairs[2 * cnt + 1] = j; }
                cnt++;
            }
        }
    }
    if (nb > 0) or_bondmap_free(&bm);
    return cnt;
}

/* Forces and energies from an explicit half pair list, Newton's 3rd law
 * (serial accumulation), plus bonds.  energies: [U_pair, U_bond, 0, 0, W]
 * with W the pair+bond virial sum of r_ij . F_ij. */
void or_forces_from_pairs(const or_model* m, int n, const double* x, const double* ori,
                          const unsigned char* type, long long npairs, const int* pairs,
                          int nb, const int* bond_idx, const double* r0, const double* kb,
                          double* F, double* T, double* energies)
{
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    memset(T, 0, sizeof(double) * 3 * (size_t)n);
    double up = 0.0, ub = 0.0, w = 0.0;
    for (long long p = 0; p < npairs; p++) {
        int i = pairs[2 * p], j = pairs[2 * p + 1];
        double d[3], Fi[3], Ti[3], Tj[3];
        double r2 = or_dist2(x + 3 * j, x + 3 * i, m->box, m->periodic, d);
        double U = or_pair_terms(m, type[i], type[j], d, r2, ori + 3 * i, ori + 3 * j, Fi, Ti, Tj);
        up += U;
        for (int k = 0; k < 3; k++) {
            F[3 * i + k] += Fi[k];
            F[3 * j + k] -= Fi[k];
            T[3 * i + k] += Ti[k];
            T[3 * j + k] += Tj[k];
            w += -d[k] * Fi[k];
        }
    }
    for (int b = 0; b < nb; b++) {
        int a = bond_idx[2 * b], c = bond_idx[2 * b + 1];
        double d[3], Fa[3];
        or_dist2(x + 3 * c, x + 3 * a, m->box, m->periodic, d);
        ub += or_bond_pair(d, kb[b], r0[b], Fa);
        for (int k = 0; k < 3; k++) {
            F[3 * a + k] += Fa[k];
            F[3 * c + k] -= Fa[k];
            w += -d[k] * Fa[k];
        }
    }
    if (energies) { energies[0] = up; energies[1] = ub; energies[2] = 0.0; energies[3] = 0.0; energies[4] = w; }
}

/* ---------------------------------------------------------------- nearest centroid */

/* Plain definition: argmin_k d^2(x_i, c_k) over all centroids, exact FP64
 * comparison, ties to the lowest centroid index. */
void or_assign_brute(int n, const double* x, int K, const double* c, const double* box, const int* per,
                     int* cell)
{
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < n; i++) {
        double best = INFINITY;
        int bk = -1;
        for (int k = 0; k < K; k++) {
            double d[3];
            double d2 = or_dist2(x + 3 * i, c + 3 * k, box, per, d);
            if (d2 < best) { best = d2; bk = k; }
        }
        cell[i] = bk;
    }
}

/* k-d tree over the centroids (the paper's nearest-centroid structure):
 * recursive median split on the widest axis, bounding boxes per node,
 * nearest search visiting the closer child first, pruning a node whose box
 * is farther than the current best.  Candidates are always scored with the
 * exact minimum-image distance, so the result equals or_assign_brute. */
typedef struct { double lo[3], hi[3]; int begin, end, left, right; } or_kdnode;
typedef struct { or_kdnode* nodes; int nnodes, cap; int* idx; const double* c; int K; } or_kdtree;

typedef struct { double key; int idx; } or_keyidx;
static int or_keyidx_cmp(const void* a, const void* b)
{
    const or_keyidx* p = (const or_keyidx*)a;
    const or_keyidx* q = (const or_keyidx*)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

static int or_kd_build_rec(or_kdtree* t, int begin, int end)
{
    int me = t->nnodes++;
    or_kdnode* nd = &t->nodes[me];
    nd->begin = begin; nd->end = end; nd->left = nd->right = -1;
    for (int k = 0; k < 3; k++) { nd->lo[k] = INFINITY; nd->hi[k] = -INFINITY; }
    for (int q = begin; q < end; q++) {
        const double* p = t->c + 3 * t->idx[q];
        for (int k = 0; k < 3; k++) {
            if (p[k] < nd->lo[k]) nd->lo[k] = p[k];
            if (p[k] > nd->hi[k]) nd->hi[k] = p[k];
        }
    }
    if (end - begin <= 8) return me;
    int ax = 0;
    double wmax = -1.0;
    for (int k = 0; k < 3; k++) if (nd->hi[k] - nd->lo[k] > wmax) { wmax = nd->hi[k] - nd->lo[k]; ax = k; }
    int n = end - begin;
    or_keyidx* tmp = (or_keyidx*)malloc(sizeof(or_keyidx) * (size_t)n);
    for (int q = 0; q < n; q++) { tmp[q].idx = t->idx[begin + q]; tmp[q].key = t->c[3 * tmp[q].idx + ax]; }
    qsort(tmp, (size_t)n, sizeof(or_keyidx), or_keyidx_cmp);
    for (int q = 0; q < n; q++) t->idx[begin + q] = tmp[q].idx;
    free(tmp);
    int mid = begin + n / 2;
    int l = or_kd_build_rec(t, begin, mid);
    int r = or_kd_build_rec(t, mid, end);
    t->nodes[me].left = l;
    t->nodes[me].right = r;
    return me;
}

static void or_kd_build(or_kdtree* t, int K, const double* c)
{
    t->K = K; t->c = c;
    t->cap = 2 * K + 8;
    t->nodes = (or_kdnode*)malloc(sizeof(or_kdnode) * (size_t)t->cap);
    t->nnodes = 0;
    t->idx = (int*)malloc(sizeof(int) * (size_t)K);
    for (int k = 0; k < K; k++) t->idx[k] = k;
    or_kd_build_rec(t, 0, K);
}

static void or_kd_free(or_kdtree* t) { free(t->nodes); free(t->idx); }

static inline double or_box_dist(const or_kdnode* nd, const double* q)
{
    double s = 0.0;
    for (int k = 0; k < 3; k++) {
        double e = 0.0;
        if (q[k] < nd->lo[k]) e = nd->lo[k] - q[k];
        else if (q[k] > nd->hi[k]) e = q[k] - nd->hi[k];
        s += e * e;
    }
    return sqrt(s);
}

static void or_kd_search(const or_kdtree* t, int node, const double* q, const double* x,
                         const double* box, const int* per, double* best, int* bk)
{
    const or_kdnode* nd = &t->nodes[node];
    /* prune with a 1e-9 sigma margin: image-shifted query boxes and exact
     * minimum-image scores differ only by rounding */
    if (or_box_dist(nd, q) > sqrt(*best) + 1e-9) return;
    if (nd->left < 0) {
        for (int p = nd->begin; p < nd->end; p++) {
            int k = t->idx[p];
            double d[3];
            double d2 = or_dist2(x, t->c + 3 * k, box, per, d);
            if (d2 < *best || (d2 == *best && k < *bk)) { *best = d2; *bk = k; }
        }
        return;
    }
    double dl = or_box_dist(&t->nodes[nd->left], q), dr = or_box_dist(&t->nodes[nd->right], q);
    if (dl <= dr) {
        or_kd_search(t, nd->left, q, x, box, per, best, bk);
        or_kd_search(t, nd->right, q, x, box, per, best, bk);
    } else {
        or_kd_search(t, nd->right, q, x, box, per, best, bk);
        or_kd_search(t, nd->left, q, x, box, per, best, bk);
    }
}

/* Nearest centroid of every particle through the k-d tree, seeding each
 * search with the previous particle's answer (the paper's last-particle
 * guess).  Periodic axes are searched through the three images of the
 * wrapped query.  Result identical to or_assign_brute. */
void or_assign_kdtree(int n, const double* x, int K, const double* c, const double* box, const int* per,
                      int* cell)
{
    or_kdtree t;
    or_kd_build(&t, K, c);
    #pragma omp parallel
    {
        int guess = 0;
        #pragma omp for schedule(static)
        for (int i = 0; i < n; i++) {
            const double* xi = x + 3 * i;
            double d[3];
            double best = or_dist2(xi, c + 3 * guess, box, per, d);
            int bk = guess;
            double w[3];
            for (int k = 0; k < 3; k++) w[k] = or_wrap(xi[k], box[k], per[k]);
            int nx = per[0] ? 3 : 1, ny = per[1] ? 3 : 1, nz = per[2] ? 3 : 1;
            for (int a = 0; a < nx; a++) for (int b = 0; b < ny; b++) for (int e = 0; e < nz; e++) {
                double q[3] = { w[0] + (per[0] ? (a - 1) * box[0] : 0.0),
                                w[1] + (per[1] ? (b - 1) * box[1] : 0.0),
                                w[2] + (per[2] ? (e - 1) * box[2] : 0.0) };
                if (!per[0]) q[0] = xi[0];
                if (!per[1]) q[1] = xi[1];
                if (!per[2]) q[2] = xi[2];
                or_kd_search(&t, 0, q, xi, box, per, &best, &bk);
            }
            cell[i] = bk;
            guess = bk;
        }
    }
    or_kd_free(&t);
}

/* ---------------------------------------------------------------- the 2^-40 grid */

/* Reading: the state lives on a grid of 2^-40 (sigma for positions, the
 * matching units for velocities, directors and angular velocities).  Input
 * values are rounded to it (round-half-even), and centroids are kept on it,
 * so centroid arithmetic is exact integer arithmetic and every grid value
 * is an exact double. */
static const double OR_GRID = 1099511627776.0;          /* 2^40 */
static const double OR_GRID_INV = 9.094947017729282e-13; /* 2^-40 */

long long or_to_grid(double v) { return llrint(v * OR_GRID); }
double or_from_grid(long long q) { return (double)q * OR_GRID_INV; }

static inline long long or_floor_div(long long a, long long b)   /* b > 0 */
{
    long long q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}
static inline long long or_floor_mod(long long a, long long b) { return a - b * or_floor_div(a, b); }

/* Minimum image on the grid: d - L round(d / L), ties rounding up. */
static inline long long or_minimg_grid(long long d, long long L, int per)
{
    if (!per) return d;
    return d - L * or_floor_div(2 * d + L, 2 * L);
}

/* ---------------------------------------------------------------- EM centroid update */

/* M-step of the continuous k-means update: each centroid moves to the mean
 * of its bilayer particles, the lipids and the membrane proteins (the lipid
 * cells are reused for the cytoskeleton's proteins, "Force Evaluation").
 * Reading, exact integer arithmetic on the 2^-40 grid:
 *   S_k = sum_{bilayer i in k} minimg(x_i - c_k),  n_k = their count,
 *   c_k <- c_k + floor((2 S_k + n_k) / (2 n_k))   (mean, ties rounding up);
 * cells without bilayer particles keep their centroid; periodic axes wrap into
 * [0, L).  Positions off the grid are rounded to it first. */
void or_lloyd(int n, const double* x, const unsigned char* type, const int* cell, int K, const double* c_in,
              double* c_out, const double* box, const int* per)
{
    long long* S = (long long*)calloc((size_t)3 * K, sizeof(long long));
    int* cnt = (int*)calloc((size_t)K, sizeof(int));
    long long L[3];
    for (int a = 0; a < 3; a++) L[a] = per[a] ? or_to_grid(box[a]) : 0;
    for (int i = 0; i < n; i++) {
        if (!or_membrane(type[i])) continue;
        int k = cell[i];
        for (int a = 0; a < 3; a++) {
            long long d = or_to_grid(x[3 * i + a]) - or_to_grid(c_in[3 * k + a]);
            S[3 * k + a] += or_minimg_grid(d, L[a], per[a]);
        }
        cnt[k]++;
    }
    for (int k = 0; k < K; k++) {
        for (int a = 0; a < 3; a++) {
            long long cq = or_to_grid(c_in[3 * k + a]);
            if (cnt[k] > 0) cq += or_floor_div(2 * S[3 * k + a] + cnt[k], 2 * (long long)cnt[k]);
            if (per[a]) cq = or_floor_mod(cq, L[a]);
            c_out[3 * k + a] = or_from_grid(cq);
        }
    }
    free(S); free(cnt);
}

/* Centroid as given, rounded to the grid and wrapped on periodic axes. */
static double or_centroid_on_grid(double c, double L, int per)
{
    long long q = or_to_grid(c);
    if (per) q = or_floor_mod(q, or_to_grid(L));
    return or_from_grid(q);
}

/* ---------------------------------------------------------------- Morton order of centroids */

/* Reading: centroid bounding box, 21 bits per axis,
 * q = min(2^21 - 1, floor((c - lo) * s)), s = 2^21 / (hi - lo) (0 on a
 * degenerate axis), bits interleaved x,y,z from the least significant bit;
 * stable order by (key, old index).  order[new] = old. */
static uint64_t or_spread3(uint64_t v)
{
    uint64_t r = 0;
    for (int b = 0; b < 21; b++) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

typedef struct { uint64_t key; int idx; } or_u64idx;
static int or_u64idx_cmp(const void* a, const void* b)
{
    const or_u64idx* p = (const or_u64idx*)a;
    const or_u64idx* q = (const or_u64idx*)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

void or_morton_keys(int K, const double* c, uint64_t* keys)
{
    double lo[3], hi[3], s[3];
    for (int a = 0; a < 3; a++) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int k = 0; k < K; k++) for (int a = 0; a < 3; a++) {
        if (c[3 * k + a] < lo[a]) lo[a] = c[3 * k + a];
        if (c[3 * k + a] > hi[a]) hi[a] = c[3 * k + a];
    }
    for (int a = 0; a < 3; a++) s[a] = (hi[a] > lo[a]) ? 2097152.0 / (hi[a] - lo[a]) : 0.0;
    for (int k = 0; k < K; k++) {
        uint64_t key = 0;
        for (int a = 0; a < 3; a++) {
            double t = (c[3 * k + a] - lo[a]) * s[a];
            double f = floor(t);
            uint64_t q = (f >= 2097151.0) ? 2097151ull : (uint64_t)f;
            key |= or_spread3(q) << a;
        }
        keys[k] = key;
    }
}

void or_morton_order(int K, const double* c, int* order)
{
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)K);
    or_morton_keys(K, c, keys);
    or_u64idx* t = (or_u64idx*)malloc(sizeof(or_u64idx) * (size_t)K);
    for (int k = 0; k < K; k++) { t[k].key = keys[k]; t[k].idx = k; }
    qsort(t, (size_t)K, sizeof(or_u64idx), or_u64idx_cmp);
    for (int k = 0; k < K; k++) order[k] = t[k].idx;
    free(t); free(keys);
}

/* ---------------------------------------------------------------- stable counting sort */

/* Particles by cell, stable on the current storage order.  perm[new] = old,
 * start[K + 1] = first storage slot of each cell. */
void or_counting_sort(int n, const int* cell, int K, int* perm, int* start)
{
    int* cnt = (int*)calloc((size_t)K + 1, sizeof(int));
    for (int i = 0; i < n; i++) cnt[cell[i] + 1]++;
    for (int k = 0; k < K; k++) cnt[k + 1] += cnt[k];
    memcpy(start, cnt, sizeof(int) * ((size_t)K + 1));
    for (int i = 0; i < n; i++) perm[cnt[cell[i]]++] = i;
    free(cnt);
}

/* ---------------------------------------------------------------- cell radius and adjacency */

/* R_k = max over particles of cell k of |x_i - c_k| (all types); particles
 * sorted by cell. */
void or_cell_radius(const double* x, int K, const int* start, const double* c, const double* box,
                    const int* per, double* R)
{
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < K; k++) {
        double r = 0.0;
        for (int i = start[k]; i < start[k + 1]; i++) {
            double d[3];
            double v = sqrt(or_dist2(x + 3 * i, c + 3 * k, box, per, d));
            if (v > r) r = v;
        }
        R[k] = r;
    }
}

/* Reading of the neighbouring-cell rule (the paper's supplementary
 * algorithm is not available): cells j and k are neighbours when their
 * bounding spheres, widened by the search cutoff and twice the skin, meet:
 *   |c_k - c_j| < (R_k + R_j + r_s + 2 delta)(1 + 1e-12).
 * By the triangle inequality every pair closer than r_s is then found.
 * Every cell is its own neighbour.  Rows ascending.  Returns the number of
 * entries (writes up to cap). */
long long or_adjacency(int K, const double* c, const double* R, double rs, double skin, const double* box,
                       const int* per, int* ptr, int* adj, long long cap)
{
    int* cnt = (int*)calloc((size_t)K, sizeof(int));
    #pragma omp parallel for schedule(dynamic, 64)
    for (int k = 0; k < K; k++) {
        int m = 0;
        for (int j = 0; j < K; j++) {
            double d[3];
            double dist = sqrt(or_dist2(c + 3 * k, c + 3 * j, box, per, d));
            double t = R[k] + R[j];
            t = t + rs;
            t = t + (skin + skin);
            t = t * (1.0 + 1e-12);
            if (dist < t) m++;
        }
        cnt[k] = m;
    }
    ptr[0] = 0;
    for (int k = 0; k < K; k++) ptr[k + 1] = ptr[k] + cnt[k];
    long long total = ptr[K];
    if (total <= cap) {
        #pragma omp parallel for schedule(dynamic, 64)
        for (int k = 0; k < K; k++) {
            int o = ptr[k];
            for (int j = 0; j < K; j++) {
                double d[3];
                double dist = sqrt(or_dist2(c + 3 * k, c + 3 * j, box, per, d));
                double t = R[k] + R[j];
                t = t + rs;
                t = t + (skin + skin);
                t = t * (1.0 + 1e-12);
                if (dist < t) adj[o++] = j;
            }
        }
    }
    free(cnt);
    return total;
}

/* ---------------------------------------------------------------- the system */

typedef struct {
    double dt, kT, gamma_t, gamma_r, mass, inertia;
    double skin;
    unsigned long long seed;
    unsigned instance;
    int rebuild_every;
    int n_centroids;
    int n_lloyd_init;
    int n_protein_centroids;   /* > 0: a separate cell set for the proteins (reading D1) */
} or_run;

typedef struct {
    or_model m;
    or_run r;
    int n, K, nb;
    /* storage-order state */
    double *x, *v, *n_, *w;
    unsigned char* type;
    unsigned* id;
    int* cell;
    /* cell list */
    double *c, *R;
    int* start;
    int *adj_ptr, *adj;
    long long adj_len;
    double* xref;          /* positions at the last rebuild (skin trigger) */
    /* bonds (ids) */
    int* bond_ids;
    double *r0, *kb;
    or_bondmap bm;
    int* slot_of_id;
    int max_id;
    /* forces in storage order */
    double *F, *T;
    int forces_valid;
    double energies[5];
    long long step;
    int cells_valid;
    long long n_rebuilds;
    /* harmonic volume constraint (reading V1-V2) */
    int vol_on;
    double kv, v0, a_vol, xc[3];
    double vol, u_vol;
} or_sys;

or_sys* or_sys_create(const or_model* m, const or_run* r)
{
    or_sys* s = (or_sys*)calloc(1, sizeof(or_sys));
    s->m = *m;
    s->r = *r;
    return s;
}

static void or_free_state(or_sys* s)
{
    free(s->x); free(s->v); free(s->n_); free(s->w); free(s->type); free(s->id); free(s->cell);
    free(s->F); free(s->T); free(s->xref); free(s->slot_of_id);
    s->x = s->v = s->n_ = s->w = s->F = s->T = s->xref = NULL;
    s->type = NULL; s->id = NULL; s->cell = NULL; s->slot_of_id = NULL;
}

void or_sys_destroy(or_sys* s)
{
    if (!s) return;
    or_free_state(s);
    free(s->c); free(s->R); free(s->start); free(s->adj_ptr); free(s->adj);
    free(s->bond_ids); free(s->r0); free(s->kb);
    or_bondmap_free(&s->bm);
    free(s);
}

int or_sys_set_particles(or_sys* s, int n, const double* pos, const double* vel, const double* ori,
                         const double* angvel, const unsigned char* type, const unsigned* id)
{
    or_free_state(s);
    s->n = n;
    s->x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    s->v = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    s->n_ = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    s->w = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    s->F = (double*)calloc(3 * (size_t)n, sizeof(double));
    s->T = (double*)calloc(3 * (size_t)n, sizeof(double));
    s->xref = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    s->type = (unsigned char*)malloc((size_t)n);
    s->id = (unsigned*)malloc(sizeof(unsigned) * (size_t)n);
    s->cell = (int*)calloc((size_t)n, sizeof(int));
    for (size_t q = 0; q < 3 * (size_t)n; q++) {
        s->x[q] = or_from_grid(or_to_grid(pos[q]));
        s->v[q] = or_from_grid(or_to_grid(vel[q]));
    }
    memcpy(s->type, type, (size_t)n);
    memcpy(s->id, id, sizeof(unsigned) * (size_t)n);
    for (int i = 0; i < n; i++) for (int k = 0; k < 3; k++) {
        int lip = or_membrane(type[i]);
        s->n_[3 * i + k] = lip ? or_from_grid(or_to_grid(ori[3 * i + k])) : 0.0;
        s->w[3 * i + k] = lip ? or_from_grid(or_to_grid(angvel[3 * i + k])) : 0.0;
    }
    s->max_id = 0;
    for (int i = 0; i < n; i++) if ((int)id[i] > s->max_id) s->max_id = (int)id[i];
    s->slot_of_id = (int*)malloc(sizeof(int) * ((size_t)s->max_id + 1));
    for (int i = 0; i <= s->max_id; i++) s->slot_of_id[i] = -1;
    for (int i = 0; i < n; i++) s->slot_of_id[id[i]] = i;
    s->forces_valid = 0;
    s->cells_valid = 0;
    s->step = 0;
    return 0;
}

int or_sys_set_bonds(or_sys* s, int nb, const int* ij, const double* r0, const double* kb)
{
    free(s->bond_ids); free(s->r0); free(s->kb);
    or_bondmap_free(&s->bm);
    s->nb = nb;
    s->bond_ids = (int*)malloc(sizeof(int) * 2 * (size_t)(nb > 0 ? nb : 1));
    s->r0 = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    s->kb = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
    if (nb > 0) {
        memcpy(s->bond_ids, ij, sizeof(int) * 2 * (size_t)nb);
        memcpy(s->r0, r0, sizeof(double) * (size_t)nb);
        memcpy(s->kb, kb, sizeof(double) * (size_t)nb);
    }
    or_bondmap_build(&s->bm, s->max_id + 1, nb, s->bond_ids);
    s->forces_valid = 0;
    return 0;
}

/* Apply a storage permutation (perm[new] = old) to the whole state. */
static void or_permute(or_sys* s, const int* perm)
{
    int n = s->n;
    double* t3 = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* arrs[6] = { s->x, s->v, s->n_, s->w, s->F, s->T };
    for (int a = 0; a < 6; a++) {
        for (int p = 0; p < n; p++) for (int k = 0; k < 3; k++) t3[3 * p + k] = arrs[a][3 * perm[p] + k];
        memcpy(arrs[a], t3, sizeof(double) * 3 * (size_t)n);
    }
    for (int p = 0; p < n; p++) for (int k = 0; k < 3; k++) t3[3 * p + k] = s->xref[3 * perm[p] + k];
    memcpy(s->xref, t3, sizeof(double) * 3 * (size_t)n);
    free(t3);
    unsigned char* tt = (unsigned char*)malloc((size_t)n);
    unsigned* ti = (unsigned*)malloc(sizeof(unsigned) * (size_t)n);
    int* tc = (int*)malloc(sizeof(int) * (size_t)n);
    for (int p = 0; p < n; p++) { tt[p] = s->type[perm[p]]; ti[p] = s->id[perm[p]]; tc[p] = s->cell[perm[p]]; }
    memcpy(s->type, tt, (size_t)n);
    memcpy(s->id, ti, sizeof(unsigned) * (size_t)n);
    memcpy(s->cell, tc, sizeof(int) * (size_t)n);
    free(tt); free(ti); free(tc);
    for (int p = 0; p < n; p++) s->slot_of_id[s->id[p]] = p;
}

/* Separate protein cells ("Force Evaluation": for a cell whose cytoskeleton
 * is partly or fully detached, the proteins get a Voronoi cell set of their
 * own).  Reading D1: with K_P = n_protein_centroids > 0, cells 0..K_L-1
 * cluster the bilayer (lipids and membrane proteins) and K_L..K_L+K_P-1 the
 * cytoskeleton's proteins; each particle belongs
 * to the nearest centroid of its own set, and each centroid moves to the
 * mean of its own members.  Reading D2: the neighbouring-cell rule is the
 * same over both sets together, so the quad loop over a cell and its
 * neighbours finds lipid-lipid, lipid-protein and protein-protein pairs.
 * Reading D3: each set is numbered along its own Morton curve (the box of
 * its own centroids), lipid cells first. */
static int or_kp(const or_sys* s) { return s->r.n_protein_centroids > 0 ? s->r.n_protein_centroids : 0; }

/* E-step: the nearest centroid of each particle's own set. */
static void or_assign_sets(or_sys* s)
{
    const int KP = or_kp(s), KL = s->K - KP, n = s->n;
    if (KP == 0) {
        or_assign_kdtree(n, s->x, s->K, s->c, s->m.box, s->m.periodic, s->cell);
        return;
    }
    double* xs = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    int* idx = (int*)malloc(sizeof(int) * (size_t)n);
    int* cs = (int*)malloc(sizeof(int) * (size_t)n);
    for (int set = 0; set < 2; set++) {
        int m = 0;
        for (int i = 0; i < n; i++) {
            if ((!or_membrane(s->type[i])) != set) continue;
            for (int a = 0; a < 3; a++) xs[3 * m + a] = s->x[3 * i + a];
            idx[m++] = i;
        }
        const int Ks = set ? KP : KL, k0 = set ? KL : 0;
        if (m > 0) or_assign_kdtree(m, xs, Ks, s->c + 3 * (size_t)k0, s->m.box, s->m.periodic, cs);
        for (int q = 0; q < m; q++) s->cell[idx[q]] = k0 + cs[q];
    }
    free(xs); free(idx); free(cs);
}

/* M-step: bilayer particles only for the shared cells; with separate sets every
 * particle is a member of its own set's cell. */
static void or_mstep_sets(or_sys* s, double* c_out)
{
    if (or_kp(s) == 0) {
        or_lloyd(s->n, s->x, s->type, s->cell, s->K, s->c, c_out, s->m.box, s->m.periodic);
        return;
    }
    unsigned char* all = (unsigned char*)calloc((size_t)s->n, 1);   /* every particle counted */
    or_lloyd(s->n, s->x, all, s->cell, s->K, s->c, c_out, s->m.box, s->m.periodic);
    free(all);
}

/* Morton order of each set's centroids, order[new] = old. */
static void or_morton_sets(const or_sys* s, int* order)
{
    const int KP = or_kp(s), KL = s->K - KP;
    or_morton_order(KL, s->c, order);
    if (KP > 0) {
        or_morton_order(KP, s->c + 3 * (size_t)KL, order + KL);
        for (int k = KL; k < s->K; k++) order[k] += KL;
    }
}

/* Morton relabel of the centroids, E-step, stable sort, radii, adjacency. */
static int or_finish_cells(or_sys* s)
{
    int K = s->K, n = s->n;
    int* order = (int*)malloc(sizeof(int) * (size_t)K);
    or_morton_sets(s, order);
    double* cn = (double*)malloc(sizeof(double) * 3 * (size_t)K);
    for (int k = 0; k < K; k++) for (int a = 0; a < 3; a++) cn[3 * k + a] = s->c[3 * order[k] + a];
    memcpy(s->c, cn, sizeof(double) * 3 * (size_t)K);
    free(cn); free(order);
    or_assign_sets(s);
    int* perm = (int*)malloc(sizeof(int) * (size_t)n);
    or_counting_sort(n, s->cell, K, perm, s->start);
    or_permute(s, perm);
    free(perm);
    or_cell_radius(s->x, K, s->start, s->c, s->m.box, s->m.periodic, s->R);
    double rs = or_search_cutoff(&s->m);
    long long tot = or_adjacency(K, s->c, s->R, rs, s->r.skin, s->m.box, s->m.periodic, s->adj_ptr, s->adj, 0);
    free(s->adj);
    s->adj = (int*)malloc(sizeof(int) * (size_t)(tot > 0 ? tot : 1));
    s->adj_len = or_adjacency(K, s->c, s->R, rs, s->r.skin, s->m.box, s->m.periodic, s->adj_ptr, s->adj, tot);
    memcpy(s->xref, s->x, sizeof(double) * 3 * (size_t)n);
    s->cells_valid = 1;
    s->forces_valid = 0;
    s->n_rebuilds++;
    return 0;
}

/* Seeds centroids c[0..K) from the particles of one set in id order
 * (c_k = member floor(k M / K)). */
static int or_seed_set(or_sys* s, int proteins, int K, double* c)
{
    int m = 0;
    for (int i = 0; i < s->n; i++) if ((!or_membrane(s->type[i])) == proteins) m++;
    if (m < K) return -1;
    int* mem = (int*)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    int q = 0;
    for (int idv = 0; idv <= s->max_id; idv++) {
        int slot = s->slot_of_id[idv];
        if (slot >= 0 && (!or_membrane(s->type[slot])) == proteins) mem[q++] = slot;
    }
    for (int k = 0; k < K; k++) {
        long long pick = ((long long)k * m) / K;
        for (int a = 0; a < 3; a++) c[3 * k + a] = s->x[3 * mem[pick] + a];
    }
    free(mem);
    return 0;
}

/* Initial k-means: centroids given, or seeded from the bilayer particles in
 * id order (c_k = bilayer particle floor(k N_L / K)), with separate protein
 * cells the protein centroids likewise from the cytoskeleton's proteins; then
 * n_lloyd_init rounds of [E-step, M-step] (shared cells: E over all
 * particles, M over the bilayer);
 * then the two-level reorder. */
int or_sys_init_cells(or_sys* s, const double* centroids)
{
    int K = s->r.n_centroids + or_kp(s), n = s->n;
    if (s->r.n_centroids <= 0) return -1;
    s->K = K;
    free(s->c); free(s->R); free(s->start); free(s->adj_ptr);
    s->c = (double*)malloc(sizeof(double) * 3 * (size_t)K);
    s->R = (double*)malloc(sizeof(double) * (size_t)K);
    s->start = (int*)malloc(sizeof(int) * ((size_t)K + 1));
    s->adj_ptr = (int*)malloc(sizeof(int) * ((size_t)K + 1));
    if (centroids) {
        memcpy(s->c, centroids, sizeof(double) * 3 * (size_t)K);
    } else {
        if (or_seed_set(s, 0, s->r.n_centroids, s->c) != 0) return -1;
        if (or_kp(s) > 0 && or_seed_set(s, 1, or_kp(s), s->c + 3 * (size_t)s->r.n_centroids) != 0) return -1;
    }
    for (int k = 0; k < K; k++) for (int a = 0; a < 3; a++)
        s->c[3 * k + a] = or_centroid_on_grid(s->c[3 * k + a], s->m.box[a], s->m.periodic[a]);
    double* cn = (double*)malloc(sizeof(double) * 3 * (size_t)K);
    for (int it = 0; it < s->r.n_lloyd_init; it++) {
        or_assign_sets(s);
        or_mstep_sets(s, cn);
        memcpy(s->c, cn, sizeof(double) * 3 * (size_t)K);
    }
    (void)n;
    free(cn);
    return or_finish_cells(s);
}

/* One rebuild: M-step from the current ownership, then the two-level
 * reorder. */
int or_sys_rebuild(or_sys* s)
{
    if (!s->cells_valid) return -1;
    double* cn = (double*)malloc(sizeof(double) * 3 * (size_t)s->K);
    or_mstep_sets(s, cn);
    memcpy(s->c, cn, sizeof(double) * 3 * (size_t)s->K);
    free(cn);
    return or_finish_cells(s);
}

/* Per-particle pair loop through the Voronoi cells (every pair computed from
 * both sides, as the paper does across patch boundaries), then bonds.
 * Energies: [U_pair, U_bond, K_trans, K_rot, W]. */
static void or_compute(or_sys* s)
{
    int n = s->n, K = s->K;
    const or_model* m = &s->m;
    double* up = (double*)calloc((size_t)n, sizeof(double));
    double* wp = (double*)calloc((size_t)n, sizeof(double));
    #pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < K; k++) {
        for (int p = s->start[k]; p < s->start[k + 1]; p++) {
            double f[3] = {0, 0, 0}, t[3] = {0, 0, 0}, u = 0.0, vir = 0.0;
            for (int a = s->adj_ptr[k]; a < s->adj_ptr[k + 1]; a++) {
                int j = s->adj[a];
                for (int q = s->start[j]; q < s->start[j + 1]; q++) {
                    if (q == p) continue;
                    double d[3];
                    double r2 = or_dist2(s->x + 3 * q, s->x + 3 * p, m->box, m->periodic, d);
                    if (!or_interacts(m, &s->bm, s->type[p], s->type[q], (int)s->id[p], (int)s->id[q], r2)) continue;
                    double Fi[3], Ti[3], Tj[3];
                    double U = or_pair_terms(m, s->type[p], s->type[q], d, r2, s->n_ + 3 * p, s->n_ + 3 * q, Fi, Ti, Tj);
                    u += 0.5 * U;
                    for (int c = 0; c < 3; c++) {
                        f[c] += Fi[c];
                        t[c] += Ti[c];
                        vir += 0.5 * (-d[c] * Fi[c]);
                    }
                }
            }
            for (int c = 0; c < 3; c++) { s->F[3 * p + c] = f[c]; s->T[3 * p + c] = t[c]; }
            up[p] = u;
            wp[p] = vir;
        }
    }
    double ub = 0.0, wb = 0.0;
    for (int b = 0; b < s->nb; b++) {
        int a = s->slot_of_id[s->bond_ids[2 * b]], c = s->slot_of_id[s->bond_ids[2 * b + 1]];
        double d[3], Fa[3];
        or_dist2(s->x + 3 * c, s->x + 3 * a, m->box, m->periodic, d);
        ub += or_bond_pair(d, s->kb[b], s->r0[b], Fa);
        for (int k = 0; k < 3; k++) {
            s->F[3 * a + k] += Fa[k];
            s->F[3 * c + k] -= Fa[k];
            wb += -d[k] * Fa[k];
        }
    }
    /* harmonic volume constraint ("Validation and Benchmark": a harmonic
     * volume constraint keeps the cell's surface-to-volume ratio; the form
     * is not given).  Reading V1: the enclosed volume of a particle
     * membrane by the divergence theorem over the bilayer particles' area
     * elements (lipids and membrane proteins), V = (1/3) sum a
     * (x_i - x_c).n_i, a the area per particle, x_c a fixed
     * reference point inside.  Reading V2: U_V = k_V (V - V0)^2 / 2 acts as
     * the uniform pressure P = -k_V (V - V0) on each area element,
     * F_i += P a n_i (moving one element by delta along its normal changes
     * the enclosed volume by a delta), and exerts no torque (a uniform
     * pressure has no moment about the element's own centre).  U_V is
     * reported with the bond energy and adds nothing to the virial. */
    s->vol = 0.0;
    s->u_vol = 0.0;
    if (s->vol_on) {
        double V = 0.0;
        for (int i = 0; i < n; i++) {
            if (!or_membrane(s->type[i])) continue;
            double d[3] = { s->x[3 * i] - s->xc[0], s->x[3 * i + 1] - s->xc[1], s->x[3 * i + 2] - s->xc[2] };
            V += s->a_vol * dot3(d, s->n_ + 3 * i) / 3.0;
        }
        const double Pa = -s->kv * (V - s->v0) * s->a_vol;
        for (int i = 0; i < n; i++) {
            if (!or_membrane(s->type[i])) continue;
            for (int c = 0; c < 3; c++) s->F[3 * i + c] += Pa * s->n_[3 * i + c];
        }
        s->vol = V;
        s->u_vol = 0.5 * s->kv * (V - s->v0) * (V - s->v0);
        ub += s->u_vol;
    }
    double U = 0.0, W = 0.0, kt = 0.0, kr = 0.0;
    for (int i = 0; i < n; i++) {
        U += up[i];
        W += wp[i];
        kt += 0.5 * s->r.mass * dot3(s->v + 3 * i, s->v + 3 * i);
        if (or_membrane(s->type[i])) kr += 0.5 * s->r.inertia * dot3(s->w + 3 * i, s->w + 3 * i);
    }
    s->energies[0] = U;
    s->energies[1] = ub;
    s->energies[2] = kt;
    s->energies[3] = kr;
    s->energies[4] = W + wb;
    free(up); free(wp);
    s->forces_valid = 1;
}

void or_sys_set_volume(or_sys* s, double kv, double v0, double area, const double* xc)
{
    s->vol_on = kv > 0.0;
    s->kv = kv;
    s->v0 = v0;
    s->a_vol = area;
    for (int c = 0; c < 3; c++) s->xc[c] = xc[c];
    s->forces_valid = 0;
}

/* The enclosed volume (reading V1) of the current state, whether or not the
 * constraint acts. */
double or_sys_volume(or_sys* s, double area, const double* xc)
{
    double V = 0.0;
    for (int i = 0; i < s->n; i++) {
        if (!or_membrane(s->type[i])) continue;
        double d[3] = { s->x[3 * i] - xc[0], s->x[3 * i + 1] - xc[1], s->x[3 * i + 2] - xc[2] };
        V += area * dot3(d, s->n_ + 3 * i) / 3.0;
    }
    return V;
}

/* Height map for the membrane fluctuation measurement ("Validation and
 * Benchmark": the instantaneous vertical fluctuation dh(x, y) along the
 * upper rim of a fixed cell; reading H1): bilayer particles above z_min whose distance
 * rho from the axis through (ax, ay) lies in [rho_in, rho_out) are binned on
 * the grid [x0 + i dx, x0 + (i + 1) dx) x [y0 + j dy, ...), i < nx, j < ny;
 * h[j nx + i] = their mean z (0 where the bin is empty), count = their
 * number.  dh over time is h(t) minus its time mean, bin by bin. */
void or_height_map(const or_sys* s, double x0, double y0, double dx, double dy, int nx, int ny, double z_min,
                   double ax, double ay, double rho_in, double rho_out, double* h, int* count)
{
    for (int q = 0; q < nx * ny; q++) { h[q] = 0.0; count[q] = 0; }
    for (int i = 0; i < s->n; i++) {
        if (!or_membrane(s->type[i])) continue;
        const double* x = s->x + 3 * i;
        if (!(x[2] > z_min)) continue;
        const double rx = x[0] - ax, ry = x[1] - ay;
        const double rho = sqrt(rx * rx + ry * ry);
        if (!(rho >= rho_in && rho < rho_out)) continue;
        const double fx = floor((x[0] - x0) / dx), fy = floor((x[1] - y0) / dy);
        if (!(fx >= 0.0 && fy >= 0.0 && fx < nx && fy < ny)) continue;
        const int q = (int)fy * nx + (int)fx;
        h[q] += x[2];
        count[q]++;
    }
    for (int q = 0; q < nx * ny; q++)
        if (count[q] > 0) h[q] /= count[q];
}

int or_sys_compute_forces(or_sys* s, double* energies)
{
    if (!s->cells_valid) return -1;
    or_compute(s);
    if (energies) memcpy(energies, s->energies, sizeof(double) * 5);
    return 0;
}

/* Cayley rotation of a unit vector by the rotation vector th (angle |th|):
 * a = th / 2, n' = n + 2/(1 + |a|^2) (a x n + a x (a x n)), renormalised. */
static void or_cayley(double* n, const double* th)
{
    double a[3] = { 0.5 * th[0], 0.5 * th[1], 0.5 * th[2] };
    double a2 = dot3(a, a);
    double k = 2.0 / (1.0 + a2);
    double an[3], aan[3];
    cross3(a, n, an);
    cross3(a, an, aan);
    for (int c = 0; c < 3; c++) n[c] = n[c] + k * (an[c] + aan[c]);
    double nn = sqrt(dot3(n, n));
    for (int c = 0; c < 3; c++) n[c] = n[c] / nn;
}

static void or_kick(or_sys* s, double h)
{
    double hm = h / s->r.mass, hi = h / s->r.inertia;
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < s->n; i++) {
        for (int c = 0; c < 3; c++) s->v[3 * i + c] += hm * s->F[3 * i + c];
        if (or_membrane(s->type[i])) {
            const double* nn = s->n_ + 3 * i;
            const double* t = s->T + 3 * i;
            double tn = dot3(t, nn);
            for (int c = 0; c < 3; c++) s->w[3 * i + c] += hi * (t[c] - tn * nn[c]);
        }
    }
}

static void or_drift(or_sys* s, double h)
{
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < s->n; i++) {
        for (int c = 0; c < 3; c++) s->x[3 * i + c] += h * s->v[3 * i + c];
        if (or_membrane(s->type[i])) {
            double* nn = s->n_ + 3 * i;
            double* w = s->w + 3 * i;
            double th[3] = { h * w[0], h * w[1], h * w[2] };
            or_cayley(nn, th);
            double wn = dot3(w, nn);
            for (int c = 0; c < 3; c++) w[c] = w[c] - wn * nn[c];
        }
    }
}

static void or_thermostat(or_sys* s)
{
    double ct = exp(-s->r.gamma_t * s->r.dt), cr = exp(-s->r.gamma_r * s->r.dt);
    double st = sqrt((1.0 - ct * ct) * s->r.kT / s->r.mass);
    double sr = sqrt((1.0 - cr * cr) * s->r.kT / s->r.inertia);
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < s->n; i++) {
        double xi[3];
        or_noise3(s->r.seed, s->r.instance, s->id[i], (uint64_t)s->step, 0u, xi);
        for (int c = 0; c < 3; c++) s->v[3 * i + c] = ct * s->v[3 * i + c] + st * xi[c];
        if (or_membrane(s->type[i])) {
            const double* nn = s->n_ + 3 * i;
            or_noise3(s->r.seed, s->r.instance, s->id[i], (uint64_t)s->step, 1u, xi);
            double xn = dot3(xi, nn);
            for (int c = 0; c < 3; c++) s->w[3 * i + c] = cr * s->w[3 * i + c] + sr * (xi[c] - xn * nn[c]);
        }
    }
}

static double or_max_displacement(or_sys* s)
{
    double mx = 0.0;
    for (int i = 0; i < s->n; i++) {
        double d[3];
        double v = sqrt(or_dist2(s->x + 3 * i, s->xref + 3 * i, s->m.box, s->m.periodic, d));
        if (v > mx) mx = v;
    }
    return mx;
}

/* BAOAB Langevin steps (Leimkuhler & Matthews 2013), translational for all
 * particles and rotational for the bilayer's (lipids and membrane proteins):
 *   B: v += dt/2 F/m, w += dt/2 (tau - (tau.n) n)/I
 *   A: x += dt/2 v, n rotated by dt/2 w (Cayley), w projected onto n-perp
 *   O: v = c v + sqrt((1-c^2) kT/m) xi, w = c w + sqrt((1-c^2) kT/I) P_perp xi
 *   A, [rebuild when due], forces, B.
 * The noise of step s is drawn with the step counter s.  A rebuild is due
 * every rebuild_every steps, or as soon as a particle has moved more than the
 * skin since the last rebuild. */
int or_sys_integrate(or_sys* s, int nsteps)
{
    if (!s->cells_valid) return -1;
    if (!s->forces_valid) or_compute(s);
    double h = 0.5 * s->r.dt;
    for (int it = 0; it < nsteps; it++) {
        or_kick(s, h);
        or_drift(s, h);
        or_thermostat(s);
        or_drift(s, h);
        int due = (s->r.rebuild_every > 0) && (((s->step + 1) % s->r.rebuild_every) == 0);
        if (!due && or_max_displacement(s) > s->r.skin) due = 1;
        if (due) or_sys_rebuild(s);
        or_compute(s);
        or_kick(s, h);
        s->step++;
    }
    return 0;
}

/* Velocity quench ("Initial structure generation": the generated system is
 * optimised by velocity quenching to remove collisions; reading M7 of the
 * mesh oracle): per step, with the current forces,
 *   v += dt F/m, then v <- (v.F) F / |F|^2 when v.F > 0, else v <- 0,
 *   scaled down so that |dt v| <= max_move; x += dt v;
 *   for bilayer particles w += dt tau_perp / I with tau_perp = tau - (tau.n) n, then
 *   w <- (w.tau_perp) tau_perp / |tau_perp|^2 when positive, else 0,
 *   scaled down so that |dt w| <= max_turn; n rotated by dt w (Cayley map,
 *   renormalised);
 * then the cells are rebuilt and the forces evaluated.  Velocities and
 * angular velocities are zero at the end; the step counter does not move.
 * fmax (nullable): the largest |F| after the last step. */
int or_sys_quench(or_sys* s, int nsteps, double dt, double max_move, double max_turn, double* fmax)
{
    if (!s->cells_valid) return -1;
    if (!s->forces_valid) or_compute(s);
    for (int it = 0; it < nsteps; it++) {
        for (int i = 0; i < s->n; i++) {
            double* v = s->v + 3 * i;
            const double* F = s->F + 3 * i;
            for (int c = 0; c < 3; c++) v[c] = v[c] + dt * F[c] / s->r.mass;
            const double vf = dot3(v, F), ff = dot3(F, F);
            for (int c = 0; c < 3; c++) v[c] = (vf > 0.0 && ff > 0.0) ? (vf / ff) * F[c] : 0.0;
            const double mv = dt * sqrt(dot3(v, v));
            if (mv > max_move)
                for (int c = 0; c < 3; c++) v[c] = v[c] * (max_move / mv);
            for (int c = 0; c < 3; c++) s->x[3 * i + c] = s->x[3 * i + c] + dt * v[c];
            if (or_membrane(s->type[i])) {
                double* w = s->w + 3 * i;
                double* nn = s->n_ + 3 * i;
                const double* t = s->T + 3 * i;
                const double tn = dot3(t, nn);
                double tp[3];
                for (int c = 0; c < 3; c++) tp[c] = t[c] - tn * nn[c];
                for (int c = 0; c < 3; c++) w[c] = w[c] + dt * tp[c] / s->r.inertia;
                const double wt = dot3(w, tp), tt = dot3(tp, tp);
                for (int c = 0; c < 3; c++) w[c] = (wt > 0.0 && tt > 0.0) ? (wt / tt) * tp[c] : 0.0;
                const double mw = dt * sqrt(dot3(w, w));
                if (mw > max_turn)
                    for (int c = 0; c < 3; c++) w[c] = w[c] * (max_turn / mw);
                double th[3] = { dt * w[0], dt * w[1], dt * w[2] };
                or_cayley(nn, th);
            }
        }
        or_sys_rebuild(s);
        or_compute(s);
    }
    double m = 0.0;
    for (int i = 0; i < s->n; i++) {
        double f = sqrt(dot3(s->F + 3 * i, s->F + 3 * i));
        if (f > m) m = f;
        for (int c = 0; c < 3; c++) { s->v[3 * i + c] = 0.0; s->w[3 * i + c] = 0.0; }
    }
    if (fmax) *fmax = m;
    return 0;
}

/* ---------------------------------------------------------------- getters (id order) */

int or_sys_n(const or_sys* s) { return s->n; }
int or_sys_k(const or_sys* s) { return s->K; }
long long or_sys_adj_len(const or_sys* s) { return s->adj_len; }
long long or_sys_rebuilds(const or_sys* s) { return s->n_rebuilds; }

int or_sys_get_state(const or_sys* s, double* pos, double* vel, double* ori, double* angvel, long long* step)
{
    for (int p = 0; p < s->n; p++) {
        int i = (int)s->id[p];
        for (int c = 0; c < 3; c++) {
            if (pos) pos[3 * i + c] = s->x[3 * p + c];
            if (vel) vel[3 * i + c] = s->v[3 * p + c];
            if (ori) ori[3 * i + c] = s->n_[3 * p + c];
            if (angvel) angvel[3 * i + c] = s->w[3 * p + c];
        }
    }
    if (step) *step = s->step;
    return 0;
}

int or_sys_get_forces(const or_sys* s, double* f, double* t)
{
    for (int p = 0; p < s->n; p++) {
        int i = (int)s->id[p];
        for (int c = 0; c < 3; c++) {
            if (f) f[3 * i + c] = s->F[3 * p + c];
            if (t) t[3 * i + c] = s->T[3 * p + c];
        }
    }
    return 0;
}

/* cell_of_id[id], perm[slot] = id at that storage slot, centroids[3K],
 * start[K+1], radius[K], adjacency CSR. */
int or_sys_get_cells(const or_sys* s, int* cell_of_id, unsigned* slot_ids, double* centroids, int* start,
                     double* radius, int* adj_ptr, int* adj)
{
    for (int p = 0; p < s->n; p++) {
        if (cell_of_id) cell_of_id[s->id[p]] = s->cell[p];
        if (slot_ids) slot_ids[p] = s->id[p];
    }
    if (centroids) memcpy(centroids, s->c, sizeof(double) * 3 * (size_t)s->K);
    if (start) memcpy(start, s->start, sizeof(int) * ((size_t)s->K + 1));
    if (radius) memcpy(radius, s->R, sizeof(double) * (size_t)s->K);
    if (adj_ptr) memcpy(adj_ptr, s->adj_ptr, sizeof(int) * ((size_t)s->K + 1));
    if (adj) memcpy(adj, s->adj, sizeof(int) * (size_t)s->adj_len);
    return 0;
}

/* Interacting pairs found by the quad loop, as (id_lo, id_hi) with
 * id_lo < id_hi; sorted.  Returns the count (writes up to cap). */
static int or_pair_cmp(const void* a, const void* b)
{
    const unsigned* p = (const unsigned*)a;
    const unsigned* q = (const unsigned*)b;
    if (p[0] != q[0]) return (p[0] > q[0]) - (p[0] < q[0]);
    return (p[1] > q[1]) - (p[1] < q[1]);
}

long long or_sys_pairs(const or_sys* s, long long cap, unsigned* pairs)
{
    const or_model* m = &s->m;
    long long cnt = 0;
    for (int k = 0; k < s->K; k++)
        for (int a = s->adj_ptr[k]; a < s->adj_ptr[k + 1]; a++) {
            int j = s->adj[a];
            for (int p = s->start[k]; p < s->start[k + 1]; p++)
                for (int q = s->start[j]; q < s->start[j + 1]; q++) {
                    if (s->id[q] <= s->id[p]) continue;   /* each pair once */
                    double d[3];
                    double r2 = or_dist2(s->x + 3 * q, s->x + 3 * p, m->box, m->periodic, d);
                    if (!or_interacts(m, &s->bm, s->type[p], s->type[q], (int)s->id[p], (int)s->id[q], r2)) continue;
                    if (cnt < cap) { pairs[2 * cnt] = s->id[p]; pairs[2 * cnt + 1] = s->id[q]; }
                    cnt++;
                }
        }
    if (cnt <= cap) qsort(pairs, (size_t)cnt, 2 * sizeof(unsigned), or_pair_cmp);
    return cnt;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
