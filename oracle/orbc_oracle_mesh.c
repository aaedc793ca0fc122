/*
 * FP64 CPU oracle: initial structure of a two-component membrane from a
 * triangular mesh, and the velocity quench that follows it (arXiv
 * 1701.02059, "Initial structure generation").
 *
 * TEST INFRASTRUCTURE ONLY (see orbc_oracle.c).  Plain, serial, in the
 * order the paper states the steps:
 *   1. protein particles on the mesh: actin/glycophorin on the vertices,
 *      spectrin along the edges (with the bonds of each spectrin chain);
 *   2. lipid particles placed at random on each triangular face by uniform
 *      sampling of the triangle (Osada, Funkhouser, Chazelle & Dobkin 2002):
 *      p = (1 - sqrt(r1)) a + sqrt(r1) (1 - r2) b + sqrt(r1) r2 c;
 *   3. a minimum distance between protein and lipid particles enforced;
 *   4. a velocity quench removes the remaining collisions (or_sys_quench).
 *
 * Readings where the paper is silent (stated again in the design notes):
 *   M1 lipid areal density: one lipid per (sqrt(3)/2) s^2 (hexagonal packing
 *      at spacing s); face f holds floor(A_f / a) + [u_f < frac(A_f / a)]
 *      lipids, u_f the uniform variate of Philox4x32-10 word 0 at counter
 *      (f, 0, 0, 2);
 *   M2 sample k of face f uses words 0 and 1 at counter (f, k, 0, 3) as r1,
 *      r2, each (w + 1/2) 2^-32; the lipid's director is the face's unit
 *      normal (e1 x e2)/|e1 x e2|, e1 = b - a, e2 = c - a (outward for a
 *      mesh wound counter-clockwise seen from outside);
 *   M3 vertex normal: the sum over the vertex's faces of round(2^32 (e1 x
 *      e2)) as exact 64-bit integers, normalised; the protein network sits
 *      `offset` sigma inside the surface: junction = v - offset n_v;
 *   M4 each undirected edge once: by its half-edge with the smaller source
 *      vertex when both directions exist, else by its only half-edge;
 *      edges numbered by the index 3 f + i of that half-edge; `beads`
 *      spectrin particles evenly spaced on the straight line between the
 *      two junctions, bonds junction-bead-...-bead-junction with rest
 *      length slack |J_b - J_a| / (beads + 1);
 *   M5 ids: surviving lipids (face order, then sample order), then
 *      junctions (vertex order), then spectrin (edge order, from a to b);
 *   M6 a lipid candidate is dropped when a protein particle lies closer
 *      than d_min, or when an earlier lipid candidate (in candidate order,
 *      kept or not) lies closer than d_ll (FP64 ((dx dx + dy dy) + dz dz)
 *      against the squared distance): uniform random points at membrane
 *      density would otherwise put pairs so close that a single pair term
 *      leaves the range of the force sums;
 *   M8 glycophorin (when asked for): one per vertex, at the vertex itself
 *      with the vertex normal as director, bonded to its junction (rest
 *      length |v - J_v|, constant kb_anchor);
 *   M9 immobile band-3 (when asked for, beads >= 1): one per edge at the
 *      midpoint (a + b) / 2 of its two vertices, director the normalised
 *      FP64 sum of the two vertices' exact normal sums, bonded to the
 *      chain's bead floor((beads - 1) / 2) (rest length the distance at
 *      construction, constant kb_anchor);
 *   M10 mobile band-3: face sample k of face f is a band-3 instead of a
 *      lipid when word 2 at counter (f, k, 0, 3), as (w + 1/2) 2^-32, is
 *      below band3_fraction; it is kept or dropped by the lipids' rules;
 *   M11 glycophorin and immobile band-3 are protein particles for the
 *      minimum distance d_min of the face samples; the bilayer comes first
 *      in id order: kept face samples, glycophorin (vertex order), immobile
 *      band-3 (edge order), then junctions and spectrin as in M5; the
 *      anchor bonds follow the chains' bonds, glycophorin's first;
 *   M7 the velocity quench (the paper names no scheme): quick-min with
 *      rotations -- v += dt F/m, then v is replaced by its component along
 *      F, or zero when it points against F, and scaled down so that
 *      |dt v| <= max_move; x += dt v; likewise w += dt tau_perp / I, w
 *      replaced by its component along tau_perp (zero when against), scaled
 *      so that |dt w| <= max_turn, n rotated by the Cayley map of dt w;
 *      cells rebuilt and forces evaluated every step; velocities zero at
 *      the end.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);

static double or_u01(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

static void or_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t sub, uint32_t w[4])
{
    uint32_t ctr[4] = { c0, c1, 0u, sub };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    or_philox4x32_10(ctr, key, w);
}

static void or_sub3(const double* a, const double* b, double* c)
{
    c[0] = a[0] - b[0];
    c[1] = a[1] - b[1];
    c[2] = a[2] - b[2];
}

static void or_cross(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double or_norm(const double* a)
{
    double s = a[0] * a[0];
    s = s + a[1] * a[1];
    s = s + a[2] * a[2];
    return sqrt(s);
}

/* Builds the particles and bonds of a mesh.  Outputs may be NULL (counts
 * only); cap / bcap bound what is written.  Returns 0, or -1 for an invalid
 * mesh (a vertex index out of range, a degenerate face). */
int or_mesh_build(int nv, const double* verts, int nf, const int* faces, double spacing, int beads, double slack,
                  double kb, double offset, double d_min, double d_ll, uint64_t seed, double band3_fraction,
                  int glycophorin, int band3_edges, double kb_anchor, long long cap, double* pos, double* ori,
                  unsigned char* type, long long* n_out, long long bcap, int* bonds, double* r0, double* kbo,
                  long long* nb_out)
{
    if (band3_edges && beads < 1) return -1;
    const double a_lip = 0.8660254037844386 * spacing * spacing;   /* sqrt(3)/2 s^2 */
    for (int q = 0; q < 3 * nf; q++)
        if (faces[q] < 0 || faces[q] >= nv) return -1;

    /* 1. proteins: vertex normals (exact integer sums), junctions */
    long long* nacc = calloc((size_t)3 * nv, sizeof(long long));
    double* junc = malloc(sizeof(double) * 3 * (size_t)(nv > 0 ? nv : 1));
    for (int f = 0; f < nf; f++) {
        const double *a = verts + 3 * faces[3 * f], *b = verts + 3 * faces[3 * f + 1], *c = verts + 3 * faces[3 * f + 2];
        double e1[3], e2[3], cr[3];
        or_sub3(b, a, e1);
        or_sub3(c, a, e2);
        or_cross(e1, e2, cr);
        for (int i = 0; i < 3; i++)
            for (int k = 0; k < 3; k++) nacc[3 * faces[3 * f + i] + k] += llrint(cr[k] * 4294967296.0);
    }
    for (int v = 0; v < nv; v++) {
        double n[3] = { (double)nacc[3 * v], (double)nacc[3 * v + 1], (double)nacc[3 * v + 2] };
        double l = or_norm(n);
        for (int k = 0; k < 3; k++) {
            double nk = l > 0.0 ? n[k] / l : 0.0;
            junc[3 * v + k] = verts[3 * v + k] - offset * nk;
        }
    }
    /* edges: owned half-edges in half-edge order */
    int* owner = malloc(sizeof(int) * (size_t)(3 * nf > 0 ? 3 * nf : 1));
    long long ne = 0;
    for (int h = 0; h < 3 * nf; h++) {
        const int f = h / 3, i = h % 3;
        const int a = faces[3 * f + i], b = faces[3 * f + (i + 1) % 3];
        int twin = 0;
        for (int g = 0; g < 3 * nf && !twin; g++) {
            const int fg = g / 3, ig = g % 3;
            if (faces[3 * fg + ig] == b && faces[3 * fg + (ig + 1) % 3] == a) twin = 1;
        }
        if (a < b || !twin) owner[ne++] = h;
    }

    /* 2. lipid candidates, face by face */
    long long ncand = 0;
    long long* fcount = malloc(sizeof(long long) * (size_t)(nf > 0 ? nf : 1));
    for (int f = 0; f < nf; f++) {
        const double *a = verts + 3 * faces[3 * f], *b = verts + 3 * faces[3 * f + 1], *c = verts + 3 * faces[3 * f + 2];
        double e1[3], e2[3], cr[3];
        or_sub3(b, a, e1);
        or_sub3(c, a, e2);
        or_cross(e1, e2, cr);
        const double area = 0.5 * or_norm(cr);
        if (!(area > 0.0)) { free(nacc); free(junc); free(owner); free(fcount); return -1; }
        const double lam = area / a_lip;
        const double fl = floor(lam);
        uint32_t w[4];
        or_words(seed, (uint32_t)f, 0u, 2u, w);
        fcount[f] = (long long)fl + (or_u01(w[0]) < lam - fl ? 1 : 0);
        ncand += fcount[f];
    }
    const long long ncyt = nv + ne * beads;                       /* junctions and spectrin */
    const long long ngly = glycophorin ? nv : 0, nb3e = band3_edges ? ne : 0;
    const long long nprot = ncyt + ngly + nb3e;                    /* every protein particle */
    double* prot = malloc(sizeof(double) * 3 * (size_t)(nprot > 0 ? nprot : 1));
    double* pdir = malloc(sizeof(double) * 3 * (size_t)(ngly + nb3e > 0 ? ngly + nb3e : 1));
    for (int v = 0; v < nv; v++)
        for (int k = 0; k < 3; k++) prot[3 * v + k] = junc[3 * v + k];
    for (long long e = 0; e < ne; e++) {
        const int h = owner[e], f = h / 3, i = h % 3;
        const int a = faces[3 * f + i], b = faces[3 * f + (i + 1) % 3];
        double d[3];
        or_sub3(junc + 3 * b, junc + 3 * a, d);
        for (int j = 1; j <= beads; j++) {
            const double t = (double)j / (double)(beads + 1);
            for (int k = 0; k < 3; k++) prot[3 * (nv + e * beads + (j - 1)) + k] = junc[3 * a + k] + d[k] * t;
        }
    }
    /* glycophorin on the vertices, band-3 on the edges' midpoints (M8, M9) */
    for (long long v = 0; v < ngly; v++) {
        double n[3] = { (double)nacc[3 * v], (double)nacc[3 * v + 1], (double)nacc[3 * v + 2] };
        double l = or_norm(n);
        for (int k = 0; k < 3; k++) {
            prot[3 * (ncyt + v) + k] = verts[3 * v + k];
            pdir[3 * v + k] = l > 0.0 ? n[k] / l : 0.0;
        }
    }
    for (long long e = 0; e < nb3e; e++) {
        const int h = owner[e], f = h / 3, i = h % 3;
        const int a = faces[3 * f + i], b = faces[3 * f + (i + 1) % 3];
        double n[3];
        for (int k = 0; k < 3; k++) n[k] = (double)nacc[3 * a + k] + (double)nacc[3 * b + k];
        double l = or_norm(n);
        for (int k = 0; k < 3; k++) {
            prot[3 * (ncyt + ngly + e) + k] = (verts[3 * a + k] + verts[3 * b + k]) * 0.5;
            pdir[3 * (ngly + e) + k] = l > 0.0 ? n[k] / l : 0.0;
        }
    }

    /* 2. lipid candidates: uniform samples of every face, in candidate order
     *    (some of them mobile band-3, M10) */
    double* cand = malloc(sizeof(double) * 6 * (size_t)(ncand > 0 ? ncand : 1));
    unsigned char* ctype = malloc((size_t)(ncand > 0 ? ncand : 1));
    long long ic = 0;
    for (int f = 0; f < nf; f++) {
        const double *a = verts + 3 * faces[3 * f], *b = verts + 3 * faces[3 * f + 1], *c = verts + 3 * faces[3 * f + 2];
        double e1[3], e2[3], cr[3];
        or_sub3(b, a, e1);
        or_sub3(c, a, e2);
        or_cross(e1, e2, cr);
        const double l = or_norm(cr);
        for (long long s = 0; s < fcount[f]; s++, ic++) {
            uint32_t w[4];
            or_words(seed, (uint32_t)f, (uint32_t)s, 3u, w);
            const double sr1 = sqrt(or_u01(w[0])), r2 = or_u01(w[1]);
            ctype[ic] = or_u01(w[2]) < band3_fraction ? 3 : 0;
            const double ca = 1.0 - sr1, cb = sr1 * (1.0 - r2), cc = sr1 * r2;
            for (int k = 0; k < 3; k++) {
                cand[6 * ic + k] = (ca * a[k] + cb * b[k]) + cc * c[k];
                cand[6 * ic + 3 + k] = cr[k] / l;
            }
        }
    }
    /* 3. minimum distances: to every protein particle, to earlier candidates */
    const double dmin2 = d_min * d_min, dll2 = d_ll * d_ll;
    long long nl = 0;
    for (long long i = 0; i < ncand; i++) {
        const double* p = cand + 6 * i;
        int keep = 1;
        for (long long q = 0; q < nprot && keep; q++) {
            double d[3];
            or_sub3(p, prot + 3 * q, d);
            double d2 = d[0] * d[0];
            d2 = d2 + d[1] * d[1];
            d2 = d2 + d[2] * d[2];
            if (d2 < dmin2) keep = 0;
        }
        for (long long j = 0; j < i && keep; j++) {
            double d[3];
            or_sub3(p, cand + 6 * j, d);
            double d2 = d[0] * d[0];
            d2 = d2 + d[1] * d[1];
            d2 = d2 + d[2] * d[2];
            if (d2 < dll2) keep = 0;
        }
        if (!keep) continue;
        if (pos && nl < cap) {
            for (int k = 0; k < 3; k++) { pos[3 * nl + k] = p[k]; ori[3 * nl + k] = p[3 + k]; }
            type[nl] = ctype[i];
        }
        nl++;
    }
    free(cand);
    free(ctype);
    /* 5. the bilayer's proteins after the face samples, then the
     *    cytoskeleton (M11) */
    const long long nbil = nl + ngly + nb3e;
    const long long n = nbil + ncyt;
    if (pos) {
        for (long long q = 0; q < ngly + nb3e && nl + q < cap; q++) {
            for (int k = 0; k < 3; k++) {
                pos[3 * (nl + q) + k] = prot[3 * (ncyt + q) + k];
                ori[3 * (nl + q) + k] = pdir[3 * q + k];
            }
            type[nl + q] = q < ngly ? 4 : 3;
        }
        for (long long q = 0; q < ncyt && nbil + q < cap; q++) {
            for (int k = 0; k < 3; k++) { pos[3 * (nbil + q) + k] = prot[3 * q + k]; ori[3 * (nbil + q) + k] = 0.0; }
            type[nbil + q] = q < nv ? 1 : 2;
        }
    }
    /* bonds of every chain */
    long long nb = 0;
    for (long long e = 0; e < ne; e++) {
        const int h = owner[e], f = h / 3, i = h % 3;
        const int a = faces[3 * f + i], b = faces[3 * f + (i + 1) % 3];
        double d[3];
        or_sub3(junc + 3 * b, junc + 3 * a, d);
        const double rest = slack * or_norm(d) / (double)(beads + 1);
        for (int j = 0; j <= beads; j++) {
            const long long u = j == 0 ? nbil + a : nbil + nv + e * beads + (j - 1);
            const long long w = j == beads ? nbil + b : nbil + nv + e * beads + j;
            if (bonds && nb < bcap) {
                bonds[2 * nb] = (int)u;
                bonds[2 * nb + 1] = (int)w;
                r0[nb] = rest;
                kbo[nb] = kb;
            }
            nb++;
        }
    }
    /* anchors: glycophorin to its junction, band-3 to its chain's middle bead */
    for (long long q = 0; q < ngly + nb3e; q++) {
        const long long u = nl + q;
        const long long pw = q < ngly ? q : nv + (q - ngly) * beads + (beads - 1) / 2;
        double d[3];
        or_sub3(prot + 3 * (ncyt + q), prot + 3 * pw, d);
        if (bonds && nb < bcap) {
            bonds[2 * nb] = (int)u;
            bonds[2 * nb + 1] = (int)(nbil + pw);
            r0[nb] = or_norm(d);
            kbo[nb] = kb_anchor;
        }
        nb++;
    }
    *n_out = n;
    *nb_out = nb;
    free(pdir);
    free(nacc);
    free(junc);
    free(owner);
    free(fcount);
    free(prot);
    return 0;
}
