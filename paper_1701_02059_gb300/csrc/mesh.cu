// Initial structure of a two-component membrane from a triangular mesh
// (arXiv 1701.02059, "Initial structure generation"): actin/glycophorin
// (junction) particles on the vertices, spectrin along the edges with the
// bonds of each chain, lipids placed at random on each face by uniform
// sampling of the triangle (Osada et al. 2002), a minimum distance between
// lipid and protein particles (and between lipids) enforced.
//
// Every step is a kernel over faces, half-edges, vertices, edges or lipid
// candidates; the random variates come from Philox4x32-10 keyed by the seed
// and counted by (face, sample), so the output does not depend on the launch
// shape.  FP64 arithmetic is written operation by operation without fused
// multiply-adds, so the positions are exact functions of the inputs.
// Readings where the paper is silent:
//   - lipid areal density: one lipid per (sqrt(3)/2) s^2, s the lipid
//     spacing; face f holds floor(A_f/a) + [u_f < frac(A_f/a)] candidates,
//     u_f = (w + 1/2) 2^-32 from word 0 at counter (f, 0, 0, 2);
//   - sample k of face f: words 0 and 1 at counter (f, k, 0, 3) give r1, r2;
//     p = ((1 - sqrt r1) a + sqrt r1 (1 - r2) b) + sqrt r1 r2 c; the lipid's
//     director is the face's unit normal (b - a) x (c - a) / |...|;
//   - vertex normal: the exact 64-bit sum of round(2^32 (b - a) x (c - a))
//     over the vertex's faces, normalised; junction = v - offset n_v;
//   - each undirected edge once, listed by its half-edge with the smaller
//     source vertex when both directions exist (else its only half-edge),
//     numbered in half-edge order 3 f + i; `beads` spectrin particles evenly
//     spaced between the two junctions; bonds junction-bead-...-junction with
//     rest length slack |J_b - J_a| / (beads + 1);
//   - a candidate is dropped when a protein particle lies closer than d_min,
//     or an earlier candidate (kept or not) closer than d_ll;
//   - the bilayer's proteins, when asked for: glycophorin on every vertex
//     (at the vertex, director n_v) bonded to its junction; immobile band-3
//     on every edge (at the midpoint (a + b) / 2, director the normalised
//     FP64 sum of the two vertices' exact normal sums) bonded to the chain's
//     bead floor((beads - 1) / 2); each anchor's rest length its length at
//     construction, constant kb_anchor; a face sample is a mobile band-3
//     instead of a lipid when word 2 at counter (f, k, 0, 3) is below
//     band3_fraction; glycophorin and edge band-3 count as proteins for
//     d_min;
//   - ids: the bilayer first (kept face samples in candidate order,
//     glycophorin, edge band-3), then junctions, then spectrin; bonds: the
//     chains', then the anchors (glycophorin's first).
#include "abi_common.cuh"

#include <algorithm>
#include <cmath>

namespace orbc {

__global__ void k_scan_block(const int* __restrict__ in, int* __restrict__ out, long long n, int* __restrict__ sums);
__global__ void k_scan_add(int* __restrict__ out, long long n, const int* __restrict__ offs);
__global__ void k_scan_single(const int* __restrict__ in, int* __restrict__ out, int m);

namespace {

constexpr int kBlk = 1024;   // elements per k_scan_block
inline int nb(long long n, int t) { return (int)((n + t - 1) / t); }

// Exclusive scan of n ints with a caller scratch of 2 * ceil(n / 1024) + 2.
void scan_ex(const int* in, int* out, long long n, int* tmp, cudaStream_t st) {
    if (n <= 0) return;
    const int blocks = nb(n, kBlk);
    k_scan_block<<<blocks, 256, 0, st>>>(in, out, n, tmp);
    if (blocks > 1) {
        k_scan_single<<<1, 1024, 0, st>>>(tmp, tmp + blocks + 1, blocks);
        k_scan_add<<<nb(n, 256), 256, 0, st>>>(out, n, tmp + blocks + 1);
    }
    CK(cudaGetLastError());
}

struct MeshDev {
    const double* v;       // [V][3]
    const int* f;          // [F][3]
    int V, F;
};

__device__ inline void cross_d(const double* a, const double* b, const double* c, double* cr) {
    const double e1[3] = {__dsub_rn(b[0], a[0]), __dsub_rn(b[1], a[1]), __dsub_rn(b[2], a[2])};
    const double e2[3] = {__dsub_rn(c[0], a[0]), __dsub_rn(c[1], a[1]), __dsub_rn(c[2], a[2])};
    cr[0] = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
    cr[1] = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
    cr[2] = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
}

__device__ inline double norm_d(const double* a) {
    double s = __dmul_rn(a[0], a[0]);
    s = __dadd_rn(s, __dmul_rn(a[1], a[1]));
    s = __dadd_rn(s, __dmul_rn(a[2], a[2]));
    return __dsqrt_rn(s);
}

__device__ inline double dist2_d(const double* p, const double* q) {
    const double dx = __dsub_rn(p[0], q[0]), dy = __dsub_rn(p[1], q[1]), dz = __dsub_rn(p[2], q[2]);
    double s = __dmul_rn(dx, dx);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    return s;
}

__device__ inline double u01(unsigned w) { return __dmul_rn(__dadd_rn(__uint2double_rn(w), 0.5), 2.3283064365386963e-10); }

__device__ inline uint4 words(unsigned long long seed, unsigned c0, unsigned c1, unsigned sub) {
    return philox4x32_10(make_uint4(c0, c1, 0u, sub), make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

// Per face: validity, lipid count, exact vertex-normal sums.
__global__ void k_mesh_faces(MeshDev m, double a_lip, unsigned long long seed, int* __restrict__ count,
                             long long* __restrict__ nacc, unsigned* __restrict__ bad) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= m.F) return;
    int id[3];
    for (int i = 0; i < 3; i++) {
        id[i] = m.f[3 * f + i];
        if (id[i] < 0 || id[i] >= m.V) { atomicOr(bad, 1u); count[f] = 0; return; }
    }
    double cr[3];
    cross_d(m.v + 3 * id[0], m.v + 3 * id[1], m.v + 3 * id[2], cr);
    const double area = __dmul_rn(0.5, norm_d(cr));
    if (!(area > 0.0)) { atomicOr(bad, 2u); count[f] = 0; return; }
    const double lam = __ddiv_rn(area, a_lip);
    const double fl = floor(lam);
    const uint4 w = words(seed, (unsigned)f, 0u, 2u);
    count[f] = (int)fl + (u01(w.x) < __dsub_rn(lam, fl) ? 1 : 0);
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++)
            atomicAdd((unsigned long long*)&nacc[3 * id[i] + k],
                      (unsigned long long)__double2ll_rn(__dmul_rn(cr[k], 4294967296.0)));
}

// Junctions: v - offset n_v.
__global__ void k_mesh_junctions(MeshDev m, const long long* __restrict__ nacc, double offset,
                                 double* __restrict__ prot) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= m.V) return;
    const double n[3] = {__ll2double_rn(nacc[3 * v]), __ll2double_rn(nacc[3 * v + 1]), __ll2double_rn(nacc[3 * v + 2])};
    const double l = norm_d(n);
    for (int k = 0; k < 3; k++) {
        const double nk = l > 0.0 ? __ddiv_rn(n[k], l) : 0.0;
        prot[3 * v + k] = __dsub_rn(m.v[3 * v + k], __dmul_rn(offset, nk));
    }
}

// Half-edges by source vertex: counts, then targets.
__global__ void k_half_count(MeshDev m, int* __restrict__ cnt) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * m.F) return;
    atomicAdd(&cnt[m.f[h]], 1);
}
__global__ void k_half_fill(MeshDev m, const int* __restrict__ start, int* __restrict__ cur, int* __restrict__ dst) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * m.F) return;
    const int f = h / 3, i = h % 3;
    const int a = m.f[h], b = m.f[3 * f + (i + 1) % 3];
    dst[start[a] + atomicAdd(&cur[a], 1)] = b;
}
// A half-edge a -> b lists its edge when a < b or when no b -> a exists.
__global__ void k_edge_owner(MeshDev m, const int* __restrict__ start, const int* __restrict__ dst,
                             int* __restrict__ own) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * m.F) return;
    const int f = h / 3, i = h % 3;
    const int a = m.f[h], b = m.f[3 * f + (i + 1) % 3];
    bool twin = false;
    for (int q = start[b]; q < start[b + 1] && !twin; q++) twin = dst[q] == a;
    own[h] = (a < b || !twin) ? 1 : 0;
}

// Spectrin beads and the rest length of each chain's bonds.
__global__ void k_mesh_beads(MeshDev m, const int* __restrict__ own, const int* __restrict__ eidx, int beads,
                             double slack, double* __restrict__ prot, double* __restrict__ rest, int* __restrict__ ends) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * m.F || !own[h]) return;
    const int f = h / 3, i = h % 3;
    const int a = m.f[h], b = m.f[3 * f + (i + 1) % 3];
    const long long e = eidx[h];
    const double* Ja = prot + 3 * a;
    const double* Jb = prot + 3 * b;
    const double d[3] = {__dsub_rn(Jb[0], Ja[0]), __dsub_rn(Jb[1], Ja[1]), __dsub_rn(Jb[2], Ja[2])};
    for (int j = 1; j <= beads; j++) {
        const double t = __ddiv_rn((double)j, (double)(beads + 1));
        double* p = prot + 3 * ((long long)m.V + e * beads + (j - 1));
        for (int k = 0; k < 3; k++) p[k] = __dadd_rn(Ja[k], __dmul_rn(d[k], t));
    }
    const double r = __ddiv_rn(__dmul_rn(slack, norm_d(d)), (double)(beads + 1));
    for (int j = 0; j <= beads; j++) {
        const long long q = e * (beads + 1) + j;
        rest[q] = r;
        ends[2 * q] = j == 0 ? a : (int)((long long)m.V + e * beads + (j - 1));
        ends[2 * q + 1] = j == beads ? b : (int)((long long)m.V + e * beads + j);
    }
}

// The bilayer's proteins: glycophorin on the vertices, band-3 on the edges'
// midpoints, after the ncyt cytoskeleton particles in prot, with their
// directors in dir.
__global__ void k_mesh_surface(MeshDev m, const long long* __restrict__ nacc, const int* __restrict__ own,
                               const int* __restrict__ eidx, long long ncyt, int ngly, int band3_edges,
                               double* __restrict__ prot, double* __restrict__ dir) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ngly) {
        const double n[3] = {__ll2double_rn(nacc[3 * t]), __ll2double_rn(nacc[3 * t + 1]), __ll2double_rn(nacc[3 * t + 2])};
        const double l = norm_d(n);
        for (int k = 0; k < 3; k++) {
            prot[3 * (ncyt + t) + k] = m.v[3 * t + k];
            dir[3 * t + k] = l > 0.0 ? __ddiv_rn(n[k], l) : 0.0;
        }
    }
    if (band3_edges && t < 3 * m.F && own[t]) {
        const int f = t / 3, i = t % 3;
        const int a = m.f[t], b = m.f[3 * f + (i + 1) % 3];
        const long long q = ngly + (long long)eidx[t];
        double n[3];
        for (int k = 0; k < 3; k++) n[k] = __dadd_rn(__ll2double_rn(nacc[3 * a + k]), __ll2double_rn(nacc[3 * b + k]));
        const double l = norm_d(n);
        for (int k = 0; k < 3; k++) {
            prot[3 * (ncyt + q) + k] = __dmul_rn(__dadd_rn(m.v[3 * a + k], m.v[3 * b + k]), 0.5);
            dir[3 * q + k] = l > 0.0 ? __ddiv_rn(n[k], l) : 0.0;
        }
    }
}

// Anchor bonds: surface protein q (output id nl + q) to its junction or to
// its edge chain's middle bead (output id nbil + that particle).
__global__ void k_mesh_anchors(const double* __restrict__ prot, long long ncyt, int ngly, long long nsurf, int V,
                               int beads, long long nl, long long nbil, int* __restrict__ ends,
                               double* __restrict__ rest) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nsurf) return;
    const long long pw = q < ngly ? q : (long long)V + (q - ngly) * beads + (beads - 1) / 2;
    const double* x = prot + 3 * (ncyt + q);
    const double* y = prot + 3 * pw;
    const double d[3] = {__dsub_rn(x[0], y[0]), __dsub_rn(x[1], y[1]), __dsub_rn(x[2], y[2])};
    ends[2 * q] = (int)(nl + q);
    ends[2 * q + 1] = (int)(nbil + pw);
    rest[q] = norm_d(d);
}

// Lipid candidates: sample k of face f, director = unit face normal; type 3
// (mobile band-3) when word 2 is below b3, else 0.
__global__ void k_mesh_samples(MeshDev m, const int* __restrict__ foff, long long nc, unsigned long long seed,
                               double b3, double* __restrict__ cand, unsigned char* __restrict__ ctype) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    int lo = 0, hi = m.F - 1;                 // the face: foff[f] <= i < foff[f + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (foff[mid] <= i) lo = mid; else hi = mid - 1;
    }
    const int f = lo;
    const int s = (int)(i - foff[f]);
    const double* a = m.v + 3 * m.f[3 * f];
    const double* b = m.v + 3 * m.f[3 * f + 1];
    const double* c = m.v + 3 * m.f[3 * f + 2];
    double cr[3];
    cross_d(a, b, c, cr);
    const double l = norm_d(cr);
    const uint4 w = words(seed, (unsigned)f, (unsigned)s, 3u);
    const double sr1 = __dsqrt_rn(u01(w.x)), r2 = u01(w.y);
    ctype[i] = u01(w.z) < b3 ? 3 : 0;
    const double ca = __dsub_rn(1.0, sr1), cb = __dmul_rn(sr1, __dsub_rn(1.0, r2)), cc = __dmul_rn(sr1, r2);
    for (int k = 0; k < 3; k++) {
        cand[6 * i + k] = __dadd_rn(__dadd_rn(__dmul_rn(ca, a[k]), __dmul_rn(cb, b[k])), __dmul_rn(cc, c[k]));
        cand[6 * i + 3 + k] = __ddiv_rn(cr[k], l);
    }
}

// Spatial hash over cells of edge h (at least the largest minimum distance):
// every point within h of a point lies in one of the 27 cells around it.
struct Hash {
    double h;
    unsigned mask;
    __device__ long long cell(double x) const { return (long long)floor(__ddiv_rn(x, h)); }
    __device__ unsigned key(long long ix, long long iy, long long iz) const {
        const unsigned long long u = (unsigned long long)ix * 73856093ull ^ (unsigned long long)iy * 19349663ull ^
                                     (unsigned long long)iz * 83492791ull;
        return (unsigned)(u ^ (u >> 32)) & mask;
    }
};
__global__ void k_hash_count(Hash H, const double* __restrict__ p, int stride, long long n, int* __restrict__ cnt,
                             int* __restrict__ key) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* x = p + stride * i;
    const unsigned k = H.key(H.cell(x[0]), H.cell(x[1]), H.cell(x[2]));
    key[i] = (int)k;
    atomicAdd(&cnt[k], 1);
}
__global__ void k_hash_fill(long long n, const int* __restrict__ key, const int* __restrict__ start,
                            int* __restrict__ cur, int* __restrict__ item) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = key[i];
    item[start[k] + atomicAdd(&cur[k], 1)] = (int)i;
}

// Keep a candidate unless a protein lies within d_min or an earlier
// candidate within d_ll (the FP64 squared distance against the square).
__global__ void k_mesh_reject(Hash H, const double* __restrict__ cand, long long nc, const double* __restrict__ prot,
                              const int* __restrict__ ps, const int* __restrict__ pi, const int* __restrict__ cs,
                              const int* __restrict__ ci, double dmin2, double dll2, int* __restrict__ keep) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc) return;
    const double* p = cand + 6 * i;
    const long long c0 = H.cell(p[0]), c1 = H.cell(p[1]), c2 = H.cell(p[2]);
    bool ok = true;
    for (int dz = -1; dz <= 1 && ok; dz++)
        for (int dy = -1; dy <= 1 && ok; dy++)
            for (int dx = -1; dx <= 1 && ok; dx++) {
                const unsigned k = H.key(c0 + dx, c1 + dy, c2 + dz);
                if (dmin2 > 0.0)
                    for (int q = ps[k]; q < ps[k + 1] && ok; q++)
                        if (dist2_d(p, prot + 3 * (long long)pi[q]) < dmin2) ok = false;
                if (dll2 > 0.0)
                    for (int q = cs[k]; q < cs[k + 1] && ok; q++) {
                        const int j = ci[q];
                        if (j < i && dist2_d(p, cand + 6 * (long long)j) < dll2) ok = false;
                    }
            }
    keep[i] = ok ? 1 : 0;
}

// Output in id order: kept face samples, the bilayer's proteins (after
// the ncyt cytoskeleton particles in prot), then the cytoskeleton.
__global__ void k_mesh_out(const double* __restrict__ cand, const unsigned char* __restrict__ ctype, long long nc,
                           const int* __restrict__ keep, const int* __restrict__ kidx, long long nl,
                           const double* __restrict__ prot, const double* __restrict__ dir, long long ncyt, int ngly,
                           long long nsurf, int V, double* __restrict__ pos, double* __restrict__ ori,
                           unsigned char* __restrict__ type) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nbil = nl + nsurf;
    if (i < nc && keep[i]) {
        const long long o = kidx[i];
        for (int k = 0; k < 3; k++) { pos[3 * o + k] = cand[6 * i + k]; ori[3 * o + k] = cand[6 * i + 3 + k]; }
        type[o] = ctype[i];
    }
    if (i < ncyt) {
        const long long o = nbil + i;
        for (int k = 0; k < 3; k++) { pos[3 * o + k] = prot[3 * i + k]; ori[3 * o + k] = 0.0; }
        type[o] = i < V ? 1 : 2;
    }
    if (i < nsurf) {
        const long long o = nl + i;
        for (int k = 0; k < 3; k++) { pos[3 * o + k] = prot[3 * (ncyt + i) + k]; ori[3 * o + k] = dir[3 * i + k]; }
        type[o] = i < ngly ? 4 : 3;
    }
}

__global__ void k_shift_ends(int* __restrict__ ends, long long n2, int by) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n2) ends[i] += by;
}

// Device buffers of one build, released together.
struct Scratch {
    std::vector<void*> ptrs;
    cudaStream_t st;
    explicit Scratch(cudaStream_t s) : st(s) {}
    template <typename T> T* get(size_t n) {
        void* p = nullptr;
        if (cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(T), st) != cudaSuccess) {
            cudaGetLastError();
            throw CudaError(cudaErrorMemoryAllocation, "mesh build: device allocation failed");
        }
        ptrs.push_back(p);
        CK(cudaMemsetAsync(p, 0, std::max<size_t>(n, 1) * sizeof(T), st));
        return (T*)p;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
    }
};

}  // namespace
}  // namespace orbc

using namespace orbc;

extern "C" int orbc_mesh_build(const orbc_mesh_params* mp, int nv, const double* verts, int nf, const int* faces,
                               long long cap, double* pos, double* ori, unsigned char* type, long long* n_out,
                               long long bond_cap, int* bonds, double* r0, double* kb, long long* nb_out,
                               void* cuda_stream) {
    if (!mp || !verts || !faces || !n_out || !nb_out || nv < 3 || nf < 1) return ORBC_E_ARG;
    if (!(mp->spacing > 0) || mp->beads < 0 || mp->beads > 64 || !(mp->slack > 0) || !(mp->kb >= 0) ||
        !(mp->d_min >= 0) || !(mp->d_ll >= 0) || !std::isfinite(mp->offset))
        return ORBC_E_ARG;
    if (!(mp->band3_fraction >= 0 && mp->band3_fraction <= 1) || !(mp->kb_anchor >= 0) ||
        !std::isfinite(mp->kb_anchor) || (mp->band3_edges && mp->beads < 1))
        return ORBC_E_ARG;
    if ((cap > 0 && (!pos || !ori || !type)) || (bond_cap > 0 && (!bonds || !r0 || !kb))) return ORBC_E_ARG;
    for (long long q = 0; q < 3ll * nv; q++)
        if (!std::isfinite(verts[q]) || std::fabs(verts[q]) >= 4096.0) return ORBC_E_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    try {
        Scratch S(st);
        double* dv = S.get<double>(3 * (size_t)nv);
        int* df = S.get<int>(3 * (size_t)nf);
        CK(cudaMemcpyAsync(dv, verts, sizeof(double) * 3 * nv, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(df, faces, sizeof(int) * 3 * (size_t)nf, cudaMemcpyHostToDevice, st));
        MeshDev m{dv, df, nv, nf};
        const long long nh = 3ll * nf;
        int* scan_tmp = S.get<int>(2 * (size_t)nb(std::max<long long>({nh, (long long)nv + 1, 1}), kBlk) + 8);
        unsigned* bad = S.get<unsigned>(1);
        // faces: counts and vertex-normal sums
        const double a_lip = 0.8660254037844386 * mp->spacing * mp->spacing;
        int* fcnt = S.get<int>((size_t)nf + 1);
        long long* nacc = S.get<long long>(3 * (size_t)nv);
        k_mesh_faces<<<nb(nf, 256), 256, 0, st>>>(m, a_lip, mp->seed, fcnt, nacc, bad);
        CK(cudaGetLastError());
        unsigned hbad = 0;
        CK(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (hbad) return ORBC_E_ARG;
        int* foff = S.get<int>((size_t)nf + 1);
        scan_ex(fcnt, foff, nf + 1, scan_tmp, st);
        int hnc = 0;
        CK(cudaMemcpyAsync(&hnc, foff + nf, sizeof(int), cudaMemcpyDeviceToHost, st));
        // edges
        int* hcnt = S.get<int>((size_t)nv + 1);
        int* hstart = S.get<int>((size_t)nv + 1);
        int* hcur = S.get<int>((size_t)nv);
        int* hdst = S.get<int>((size_t)nh);
        k_half_count<<<nb(nh, 256), 256, 0, st>>>(m, hcnt);
        scan_ex(hcnt, hstart, nv + 1, scan_tmp, st);
        k_half_fill<<<nb(nh, 256), 256, 0, st>>>(m, hstart, hcur, hdst);
        int* own = S.get<int>((size_t)nh + 1);
        int* eidx = S.get<int>((size_t)nh + 1);
        k_edge_owner<<<nb(nh, 256), 256, 0, st>>>(m, hstart, hdst, own);
        scan_ex(own, eidx, nh + 1, scan_tmp, st);
        int hne = 0;
        CK(cudaMemcpyAsync(&hne, eidx + nh, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const long long nc = hnc, ne = hne, beads = mp->beads;
        // cytoskeleton (junctions, beads), then the bilayer's proteins
        const int ngly = mp->glycophorin ? nv : 0;
        const long long ncyt = nv + ne * beads, nsurf = ngly + (mp->band3_edges ? ne : 0);
        const long long np = ncyt + nsurf, nchain = ne * (beads + 1), nbond = nchain + nsurf;
        if (nc + np > (1ll << 30)) return ORBC_E_ARG;
        // proteins
        double* prot = S.get<double>(3 * (size_t)np);
        double* pdir = S.get<double>(3 * (size_t)nsurf);
        double* rest = S.get<double>((size_t)nbond);
        int* ends = S.get<int>(2 * (size_t)nbond);
        k_mesh_junctions<<<nb(nv, 256), 256, 0, st>>>(m, nacc, mp->offset, prot);
        k_mesh_beads<<<nb(nh, 256), 256, 0, st>>>(m, own, eidx, mp->beads, mp->slack, prot, rest, ends);
        if (nsurf > 0)
            k_mesh_surface<<<nb(std::max<long long>(nh, nv), 256), 256, 0, st>>>(m, nacc, own, eidx, ncyt, ngly,
                                                                                 mp->band3_edges, prot, pdir);
        CK(cudaGetLastError());
        // lipid candidates and the minimum distances
        double* cand = S.get<double>(6 * (size_t)nc);
        unsigned char* ctype = S.get<unsigned char>((size_t)nc);
        if (nc > 0) k_mesh_samples<<<nb(nc, 256), 256, 0, st>>>(m, foff, nc, mp->seed, mp->band3_fraction, cand, ctype);
        int* keep = S.get<int>((size_t)nc + 1);
        int* kidx = S.get<int>((size_t)nc + 1);
        const double dmin2 = mp->d_min * mp->d_min, dll2 = mp->d_ll * mp->d_ll;
        const double hcell = std::max(mp->d_min, mp->d_ll);
        if (nc > 0 && hcell > 0.0) {
            unsigned T = 1024;
            while ((long long)T < 2 * (np + nc) && T < (1u << 30)) T <<= 1;
            Hash H{hcell, T - 1};
            int* tmp2 = S.get<int>(2 * (size_t)nb((long long)T + 1, kBlk) + 8);
            int* pc = S.get<int>((size_t)T + 1);
            int* ps = S.get<int>((size_t)T + 1);
            int* pcur = S.get<int>((size_t)T);
            int* pkey = S.get<int>((size_t)np);
            int* pitem = S.get<int>((size_t)np);
            int* cc = S.get<int>((size_t)T + 1);
            int* cs = S.get<int>((size_t)T + 1);
            int* ccur = S.get<int>((size_t)T);
            int* ckey = S.get<int>((size_t)nc);
            int* citem = S.get<int>((size_t)nc);
            if (np > 0) k_hash_count<<<nb(np, 256), 256, 0, st>>>(H, prot, 3, np, pc, pkey);
            scan_ex(pc, ps, (long long)T + 1, tmp2, st);
            if (np > 0) k_hash_fill<<<nb(np, 256), 256, 0, st>>>(np, pkey, ps, pcur, pitem);
            k_hash_count<<<nb(nc, 256), 256, 0, st>>>(H, cand, 6, nc, cc, ckey);
            scan_ex(cc, cs, (long long)T + 1, tmp2, st);
            k_hash_fill<<<nb(nc, 256), 256, 0, st>>>(nc, ckey, cs, ccur, citem);
            k_mesh_reject<<<nb(nc, 256), 256, 0, st>>>(H, cand, nc, prot, ps, pitem, cs, citem, dmin2, dll2, keep);
        } else if (nc > 0) {
            std::vector<int> ones((size_t)nc, 1);
            CK(cudaMemcpyAsync(keep, ones.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
            CK(cudaStreamSynchronize(st));
        }
        CK(cudaGetLastError());
        int* scan_c = S.get<int>(2 * (size_t)nb(nc + 1, kBlk) + 8);
        scan_ex(keep, kidx, nc + 1, scan_c, st);
        int hnl = 0;
        CK(cudaMemcpyAsync(&hnl, kidx + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        const long long nl = hnl, nbil = nl + nsurf, n = nl + np;
        *n_out = n;
        *nb_out = nbond;
        if (cap >= n && pos) {
            double* dpos = S.get<double>(3 * (size_t)n);
            double* dori = S.get<double>(3 * (size_t)n);
            unsigned char* dty = S.get<unsigned char>((size_t)n);
            const long long span = std::max(nc, np);
            if (span > 0)
                k_mesh_out<<<nb(span, 256), 256, 0, st>>>(cand, ctype, nc, keep, kidx, nl, prot, pdir, ncyt, ngly,
                                                          nsurf, nv, dpos, dori, dty);
            CK(cudaMemcpyAsync(pos, dpos, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(ori, dori, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(type, dty, (size_t)n, cudaMemcpyDeviceToHost, st));
        }
        if (bond_cap >= nbond && bonds && nbond > 0) {
            if (nchain > 0) k_shift_ends<<<nb(2 * nchain, 256), 256, 0, st>>>(ends, 2 * nchain, (int)nbil);
            if (nsurf > 0)
                k_mesh_anchors<<<nb(nsurf, 256), 256, 0, st>>>(prot, ncyt, ngly, nsurf, nv, mp->beads, nl, nbil,
                                                               ends + 2 * nchain, rest + nchain);
            CK(cudaMemcpyAsync(bonds, ends, sizeof(int) * 2 * nbond, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(r0, rest, sizeof(double) * nbond, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (long long q = 0; q < nbond; q++) kb[q] = q < nchain ? mp->kb : mp->kb_anchor;
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(st));
        if ((cap > 0 && cap < n) || (bond_cap > 0 && bond_cap < nbond)) return ORBC_E_ARG;
        return ORBC_OK;
    } catch (const CudaError& e) {
        return e.code == cudaErrorMemoryAllocation ? ORBC_E_NOMEM : ORBC_E_CUDA;
    } catch (const std::exception&) {
        return ORBC_E_CUDA;
    }
}
