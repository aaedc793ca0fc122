// Adaptive Voronoi cell list (arXiv 1701.02059, "Spatial Searching
// Algorithm"): centroid M-step, Morton relabel of the centroids, exact
// nearest-centroid E-step on a centroid grid, stable counting sort of the
// particles with the state gather, cell radii and neighbouring-cell lists.
//
// Every discrete output (cell of each particle, storage permutation,
// centroids, neighbouring cells) equals the FP64 definition bit for bit:
// integer arithmetic where the definition is integer (M-step, sort), FP32
// prefilters with a proven rounding band and an FP64 re-decision inside the
// band where the definition compares FP64 distances.
#include "ensemble.cuh"

#include <algorithm>

namespace orbc {

// ============================================================== M-step
// S_k = sum over the members (lipids; every particle of a protein cell set)
// of minimg(x_i - c_k) on the 2^-40 grid (int64, exact, order-independent),
// n_k = their count.  Warp-aggregated 64-bit atomics.
__global__ void k_mstep_accum(View v, const int* __restrict__ cell_of, long long* __restrict__ S,
                              int* __restrict__ cnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = i < v.N;
    int c = -1;
    long long d[3] = {0, 0, 0};
    if (act) {
        const int ci = cell_of[i];
        const Inst& I = v.inst[find_inst(v.inst_k0, v.B, ci)];
        if (centroid_member(I, v.type[i])) {
            c = ci;
            for (int a = 0; a < 3; a++)
                d[a] = minimg_q(v.xq[(size_t)a * v.N + i] - v.cq[(size_t)a * v.Ktot + c], I.boxq[a], I.periodic[a]);
        }
    }
    const unsigned full = 0xffffffffu;   // every lane of the warp reaches this point
    unsigned grp = __match_any_sync(full, c);
    int leader = __ffs(grp) - 1;
    int lane = threadIdx.x & 31;
    long long s0 = d[0], s1 = d[1], s2 = d[2];
    int n = (c >= 0) ? 1 : 0;
    // the group leader sums its members (exact integers, any order)
    long long a0 = 0, a1 = 0, a2 = 0;
    int an = 0;
    unsigned m = grp;
    while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        a0 += __shfl_sync(grp, s0, src);
        a1 += __shfl_sync(grp, s1, src);
        a2 += __shfl_sync(grp, s2, src);
        an += __shfl_sync(grp, n, src);
    }
    if (c >= 0 && lane == leader) {
        atomicAdd((unsigned long long*)&S[(size_t)0 * v.Ktot + c], (unsigned long long)a0);
        atomicAdd((unsigned long long*)&S[(size_t)1 * v.Ktot + c], (unsigned long long)a1);
        atomicAdd((unsigned long long*)&S[(size_t)2 * v.Ktot + c], (unsigned long long)a2);
        atomicAdd(&cnt[c], an);
    }
}

// c_k <- c_k + floor((2 S_k + n_k) / (2 n_k)); periodic axes wrap into [0, L).
// dmax (nullable): the largest move of an instance's centroids, as FP32 bits
// rounded up (warp-reduced before the atomics).
__global__ void k_mstep_finish(View v, long long* __restrict__ S, int* __restrict__ cnt, int iter,
                               unsigned* __restrict__ dmax, float* __restrict__ cmove) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.Ktot) return;
    int b = find_inst(v.inst_k0, v.B, k);
    const Inst& I = v.inst[b];
    int n = (iter < 0 || iter < I.n_lloyd) ? cnt[k] : 0;   // instances past their k-means rounds keep c
    float mv2 = 0.f;
    for (int a = 0; a < 3; a++) {
        long long c = v.cq[(size_t)a * v.Ktot + k];
        long long step = 0;
        if (n > 0) step = floor_div_ll(2 * S[(size_t)a * v.Ktot + k] + n, 2 * (long long)n);
        const float sf = ll_to_float(step) * (float)kGridInv;
        mv2 = fmaf(sf, sf, mv2);
        c += step;
        if (I.periodic[a]) c = floor_mod_ll(c, I.boxq[a]);
        v.cq[(size_t)a * v.Ktot + k] = c;
        S[(size_t)a * v.Ktot + k] = 0;
    }
    cnt[k] = 0;
    if (cmove) cmove[k] = sqrtf(mv2) * 1.0001f + 1e-6f;
    if (dmax) {
        const unsigned grp = __match_any_sync(__activemask(), b);
        const unsigned mv = __reduce_max_sync(grp, __float_as_uint(sqrtf(mv2) * 1.0001f + 1e-6f));
        if ((int)(threadIdx.x & 31) == __ffs(grp) - 1) atomicMax(&dmax[b], mv);
    }
}

// Rebuild M-step on cell-sorted particles: one warp per cell sums its members'
// grid displacements (exact int64, shuffles), updates the centroid and
// folds it into the instance bounding box (block-level, then atomics).
__global__ void k_mstep_sorted(View v, long long* __restrict__ bb, unsigned* __restrict__ dmax) {
    __shared__ long long wmin[8][3], wmax[8][3];
    __shared__ int winst[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * 8 + warp;
    int b = -1;
    long long c[3] = {0, 0, 0};
    if (k < v.Ktot) {
        b = find_inst(v.inst_k0, v.B, k);
        const Inst& I = v.inst[b];
        const int s = v.cell_start[k], e = v.cell_start[k + 1];
        for (int a = 0; a < 3; a++) c[a] = v.cq[(size_t)a * v.Ktot + k];
        long long S0 = 0, S1 = 0, S2 = 0;
        int n = 0;
        const size_t N = v.N;
        for (int p = s + lane; p < e; p += 32) {
            if (!centroid_member(I, v.type[p])) continue;
            S0 += minimg_q(v.xq[p] - c[0], I.boxq[0], I.periodic[0]);
            S1 += minimg_q(v.xq[N + p] - c[1], I.boxq[1], I.periodic[1]);
            S2 += minimg_q(v.xq[2 * N + p] - c[2], I.boxq[2], I.periodic[2]);
            n++;
        }
        for (int off = 16; off; off >>= 1) {
            S0 += __shfl_xor_sync(0xffffffffu, S0, off);
            S1 += __shfl_xor_sync(0xffffffffu, S1, off);
            S2 += __shfl_xor_sync(0xffffffffu, S2, off);
            n += __shfl_xor_sync(0xffffffffu, n, off);
        }
        long long S[3] = {S0, S1, S2};
        float mv2 = 0.f;
        for (int a = 0; a < 3; a++) {
            long long step = 0;
            if (n > 0) step = floor_div_ll(2 * S[a] + n, 2 * (long long)n);
            const float sf = ll_to_float(step) * (float)kGridInv;
            mv2 = fmaf(sf, sf, mv2);
            c[a] += step;
            if (I.periodic[a]) c[a] = floor_mod_ll(c[a], I.boxq[a]);
        }
        if (lane == 0) {
            for (int a = 0; a < 3; a++) v.cq[(size_t)a * v.Ktot + k] = c[a];
            if (dmax) atomicMax(&dmax[b], __float_as_uint(sqrtf(mv2) * 1.0001f + 1e-6f));
        }
    }
    if (lane == 0) {
        winst[warp] = b;
        for (int a = 0; a < 3; a++) { wmin[warp][a] = c[a]; wmax[warp][a] = c[a]; }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int cur = -1;
        long long mn[3], mx[3];
        for (int w = 0; w <= 8; w++) {
            int bw = (w < 8) ? winst[w] : -2;
            if (bw != cur) {
                if (cur >= 0)
                    for (int a = 0; a < 3; a++) { atomicMin(&bb[cur * 6 + a], mn[a]); atomicMax(&bb[cur * 6 + 3 + a], mx[a]); }
                cur = bw;
                if (bw >= 0) for (int a = 0; a < 3; a++) { mn[a] = wmin[w][a]; mx[a] = wmax[w][a]; }
            } else if (bw >= 0) {
                for (int a = 0; a < 3; a++) { mn[a] = min(mn[a], wmin[w][a]); mx[a] = max(mx[a], wmax[w][a]); }
            }
        }
    }
}

// M-step from the sums the B-A-O-A launch accumulated (same terms as
// k_mstep_sorted, so the same centroids): one thread per cell updates c_k,
// clears the sums for the next step and folds the centroid into the
// instance's bounding box and its largest move (warp-reduced before the
// atomics).
__global__ void __launch_bounds__(256) k_mstep_apply(View v, long long* __restrict__ S, int* __restrict__ cnt,
                                                     long long* __restrict__ bb, unsigned* __restrict__ dmax) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.Ktot) return;
    const size_t K = v.Ktot;
    const int b = find_inst(v.inst_k0, v.B, k);
    const Inst& I = v.inst[b];
    const int n = cnt[k];
    long long c[3];
    float mv2 = 0.f;
    for (int a = 0; a < 3; a++) {
        c[a] = v.cq[a * K + k];
        long long step = 0;
        if (n > 0) step = floor_div_ll(2 * S[a * K + k] + n, 2 * (long long)n);
        const float sf = ll_to_float(step) * (float)kGridInv;
        mv2 = fmaf(sf, sf, mv2);
        c[a] += step;
        if (I.periodic[a]) c[a] = floor_mod_ll(c[a], I.boxq[a]);
        v.cq[a * K + k] = c[a];
        S[a * K + k] = 0;
    }
    cnt[k] = 0;
    const unsigned grp = __match_any_sync(__activemask(), b);
    const unsigned mv = __reduce_max_sync(grp, __float_as_uint(sqrtf(mv2) * 1.0001f + 1e-6f));
    long long mn[3] = {c[0], c[1], c[2]}, mx[3] = {c[0], c[1], c[2]};
    if (grp == 0xffffffffu) {
        for (int off = 16; off; off >>= 1)
            for (int a = 0; a < 3; a++) {
                mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], off));
                mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], off));
            }
    }
    const bool leader = (int)(threadIdx.x & 31) == __ffs(grp) - 1;
    if (leader && dmax) atomicMax(&dmax[b], mv);
    if (grp != 0xffffffffu || leader)
        for (int a = 0; a < 3; a++) { atomicMin(&bb[b * 6 + a], mn[a]); atomicMax(&bb[b * 6 + 3 + a], mx[a]); }
}

// ============================================================== Morton relabel
__global__ void k_fill_bbox(long long* bb, int B) {
    for (int t = threadIdx.x; t < B * 6; t += blockDim.x) bb[t] = ((t % 6) < 3) ? 0x7fffffffffffffffll : (-0x7fffffffffffffffll - 1);
}

// Bounding box of each instance's centroids (exact int64 min/max), reduced
// per block before the atomics.
__global__ void k_bbox(View v, long long* __restrict__ bb /* [B][6] */) {
    __shared__ long long smin[256][3], smax[256][3];
    __shared__ int sb[256];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = threadIdx.x;
    sb[t] = -1;
    if (k < v.Ktot) {
        sb[t] = find_inst(v.inst_k0, v.B, k);
        for (int a = 0; a < 3; a++) smin[t][a] = smax[t][a] = v.cq[(size_t)a * v.Ktot + k];
    }
    __syncthreads();
    if (t == 0) {
        int cur = -2;
        long long mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
        for (int q = 0; q <= 256; q++) {
            int bq = (q < 256) ? sb[q] : -3;
            if (bq != cur) {
                if (cur >= 0)
                    for (int a = 0; a < 3; a++) { atomicMin(&bb[cur * 6 + a], mn[a]); atomicMax(&bb[cur * 6 + 3 + a], mx[a]); }
                cur = bq;
                if (bq >= 0) for (int a = 0; a < 3; a++) { mn[a] = smin[q][a]; mx[a] = smax[q][a]; }
            } else if (bq >= 0) {
                for (int a = 0; a < 3; a++) { mn[a] = min(mn[a], smin[q][a]); mx[a] = max(mx[a], smax[q][a]); }
            }
        }
    }
}

__device__ inline unsigned long long spread3(unsigned long long x) {
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Key: 21 bits per axis, q = min(2^21 - 1, floor((c - lo) * 2^21 / (hi - lo)))
// in FP64 exactly as the definition (c - lo is exact on the grid).
__global__ void k_morton_keys(View v, const long long* __restrict__ bb, unsigned long long* __restrict__ key) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.Ktot) return;
    int b = find_inst(v.inst_k0, v.B, k);
    unsigned long long kk = 0;
    for (int a = 0; a < 3; a++) {
        double lo = grid_to_double(bb[b * 6 + a]), hi = grid_to_double(bb[b * 6 + 3 + a]);
        double s = (hi > lo) ? __ddiv_rn(2097152.0, __dsub_rn(hi, lo)) : 0.0;
        double t = __dmul_rn(__dsub_rn(grid_to_double(v.cq[(size_t)a * v.Ktot + k]), lo), s);
        double f = floor(t);
        unsigned long long q = (f >= 2097151.0) ? 2097151ull : (unsigned long long)f;
        kk |= spread3(q) << a;
    }
    key[k] = kk;
}

// Sort of (instance, key, index): bitonic sort of 1024-element tiles in
// shared memory, then each element's rank inside its instance is its rank in
// its own tile plus, for every other tile of the instance, the number of
// smaller elements there (binary search).  Keys are unique with the index.
constexpr int kTile = 1024;

struct SortRec { unsigned long long key; int idx; int inst; };

__device__ inline bool rec_less(const SortRec& a, const SortRec& b) {
    if (a.inst != b.inst) return a.inst < b.inst;
    if (a.key != b.key) return a.key < b.key;
    return a.idx < b.idx;
}

// One tile of kTile records sorted by a block of kTile threads (bitonic):
// exchanges across warps go through shared memory, the strides below 32
// through shuffles.
__device__ inline SortRec shfl_rec(const SortRec& r, int m) {
    SortRec o;
    o.key = __shfl_xor_sync(0xffffffffu, r.key, m);
    o.idx = __shfl_xor_sync(0xffffffffu, r.idx, m);
    o.inst = __shfl_xor_sync(0xffffffffu, r.inst, m);
    return o;
}

__global__ void __launch_bounds__(kTile) k_tile_sort(View v, const unsigned long long* __restrict__ key,
                                                    SortRec* __restrict__ out) {
    __shared__ SortRec sh[kTile];
    const int t = threadIdx.x;
    const int k = blockIdx.x * kTile + t;
    SortRec r;
    if (k < v.Ktot) { r.key = key[k]; r.idx = k; r.inst = find_inst(v.inst_k0, v.B, k); }
    else { r.key = ~0ull; r.idx = 0x7fffffff; r.inst = 0x7fffffff; }
    for (int size = 2; size <= kTile; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            SortRec o;
            if (stride >= 32) {
                sh[t] = r;
                __syncthreads();
                o = sh[t ^ stride];
                __syncthreads();
            } else {
                o = shfl_rec(r, stride);
            }
            // the lower slot of an ascending pair keeps the smaller record
            const bool up = (t & size) == 0, lower = (t & stride) == 0;
            const bool take = (lower == up) ? rec_less(o, r) : rec_less(r, o);
            if (take) r = o;
        }
    }
    out[blockIdx.x * kTile + t] = r;
}

// rank -> new cell index; writes order[new] = old and the permuted centroids.
// Tiles wholly below or above a record need no search (nearly sorted keys
// between rebuilds make this the common case).
constexpr int kBoundTiles = 1024;   // tiles whose bounds a block keeps in shared memory

__global__ void k_rank_scatter(View v, const SortRec* __restrict__ tiles, int ntiles, const long long* __restrict__ cq_old,
                               int* __restrict__ new_of_old) {
    // first and last record of every tile (most tiles lie wholly below or
    // above a record, which these settle without a search)
    __shared__ SortRec tb[2][kBoundTiles];
    const bool cached = ntiles <= kBoundTiles;
    if (cached)
        for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
            tb[0][t] = tiles[(size_t)t * kTile];
            tb[1][t] = tiles[(size_t)t * kTile + kTile - 1];
        }
    __syncthreads();
    int pos = blockIdx.x * blockDim.x + threadIdx.x;   // position in the tiled array
    if (pos >= ntiles * kTile) return;
    SortRec me = tiles[pos];
    if (me.idx >= v.Ktot) return;
    const Inst& I = v.inst[me.inst];
    // rank inside the instance: over every tile holding part of the instance,
    // (records smaller than me) - (records of smaller instances)
    SortRec first;
    first.inst = me.inst; first.key = 0; first.idx = -1;
    int rank = 0;
    int t0 = I.k0 / kTile, t1 = (I.k0 + I.K - 1) / kTile;
    for (int t = t0; t <= t1; t++) {
        const SortRec* T = tiles + (size_t)t * kTile;
        const SortRec tmin = cached ? tb[0][t] : T[0], tmax = cached ? tb[1][t] : T[kTile - 1];
        int lo, lo2;
        if (rec_less(tmax, me)) lo = kTile;
        else if (!rec_less(tmin, me)) lo = 0;
        else {
            int a = 0, c = kTile;
            while (a < c) { int mid = (a + c) >> 1; if (rec_less(T[mid], me)) a = mid + 1; else c = mid; }
            lo = a;
        }
        if (rec_less(tmax, first)) lo2 = kTile;
        else if (!rec_less(tmin, first)) lo2 = 0;
        else {
            int a = 0, c = kTile;
            while (a < c) { int mid = (a + c) >> 1; if (rec_less(T[mid], first)) a = mid + 1; else c = mid; }
            lo2 = a;
        }
        rank += lo - lo2;
    }
    int nk = I.k0 + rank;
    new_of_old[me.idx] = nk;
    for (int a = 0; a < 3; a++) v.cq[(size_t)a * v.Ktot + nk] = cq_old[(size_t)a * v.Ktot + me.idx];
}

// ============================================================== centroid grid
// Fixed per-instance geometry (origin, edge, dims); edge cells extend to
// infinity, so the face-distance bound of the shell search stays valid for
// centroids and particles outside the box.
__device__ inline int grid_coord(long long xq, const Inst& I, int a, float& rel) {
    long long d = xq - I.gorg[a];
    if (I.periodic[a]) d = floor_mod_ll(d, I.boxq[a]);
    // >> 20: units of 2^-20 sigma, |.| < 2^31 for |d| < 2048 sigma
    long long s = d >> 20;
    if (s > 2147483647ll) s = 2147483647ll;
    if (s < -2147483647ll) s = -2147483647ll;
    rel = (float)(int)s * 9.5367431640625e-07f;
    int g = (int)floorf(rel * I.ginv[a]);
    if (g < 0) g = 0;
    if (g >= I.gdim[a]) g = I.gdim[a] - 1;
    return g;
}

__global__ void k_grid_count(View v, int* __restrict__ gcount, int* __restrict__ gidx) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.Ktot) return;
    int b = find_inst(v.inst_k0, v.B, k);
    const Inst& I = v.inst[b];
    float r[3];
    int gx = grid_coord(v.cq[k], I, 0, r[0]);
    int gy = grid_coord(v.cq[(size_t)v.Ktot + k], I, 1, r[1]);
    int gz = grid_coord(v.cq[(size_t)2 * v.Ktot + k], I, 2, r[2]);
    long long g = I.g0 + ((long long)gz * I.gdim[1] + gy) * I.gdim[0] + gx;
    gidx[k] = (int)g;
    atomicAdd(&gcount[g], 1);
}

__global__ void k_grid_fill(View v, const int* __restrict__ gidx, int* __restrict__ cursor, float4* __restrict__ cf) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.Ktot) return;
    int b = find_inst(v.inst_k0, v.B, k);
    const Inst& I = v.inst[b];
    int g = gidx[k];
    int pos = v.gstart[g] + atomicAdd(&cursor[g], 1);
    float r[3];
    grid_coord(v.cq[k], I, 0, r[0]);
    grid_coord(v.cq[(size_t)v.Ktot + k], I, 1, r[1]);
    grid_coord(v.cq[(size_t)2 * v.Ktot + k], I, 2, r[2]);
    v.gcent[pos] = k;
    v.gcf[pos] = make_float4(r[0], r[1], r[2], __int_as_float(k));
    if (cf) cf[k] = make_float4(r[0], r[1], r[2], 0.f);
}

// ============================================================== E-step
// Exact nearest centroid (ties to the lowest index) of every particle.
// FP32 distances relative to the grid origin have an absolute error below
// kBand (coordinates < 2048 sigma carry <= 1.3e-4 sigma each); the shell
// search stops once the unexplored region is farther than best + band, and
// every centroid within band of the FP32 best is re-scored in FP64 with the
// definition's operation order.  A single candidate in the band is the
// exact answer without FP64.
constexpr float kBandE = 2e-3f;
// margin of the FP32 certificates of the E-steps (coordinates up to ~2000 sigma)
constexpr float kCertMargin = 4e-3f;

__device__ inline float axis_dist(float p, float c, const Inst& I, int a) {
    float d = p - c;
    if (I.periodic[a]) d -= I.boxf[a] * rintf(d / I.boxf[a]);
    return d;
}

__device__ inline int wrap_idx(int x, int n) { x %= n; return x < 0 ? x + n : x; }

// Is grid index w (wrapped) inside the cube of Chebyshev radius r around g?
__device__ inline bool in_cube(const int w[3], const int g[3], int r, const Inst& I) {
    for (int a = 0; a < 3; a++) {
        if (I.periodic[a]) {
            if (2 * r + 1 >= I.gdim[a]) continue;
            int d = wrap_idx(w[a] - g[a], I.gdim[a]);
            if (min(d, I.gdim[a] - d) > r) return false;
        } else {
            if (w[a] < g[a] - r || w[a] > g[a] + r) return false;
        }
    }
    return true;
}

// Visit every grid cell of cube(r) \ cube(r - 1) exactly once (periodic axes
// wrap; once an axis is fully covered it is enumerated without repeats).
template <typename F>
__device__ inline void for_shell(const int g[3], int r, const Inst& I, F&& f) {
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        if (I.periodic[a]) {
            if (2 * r + 1 >= I.gdim[a]) { lo[a] = 0; hi[a] = I.gdim[a] - 1; }
            else { lo[a] = g[a] - r; hi[a] = g[a] + r; }
        } else {
            lo[a] = max(0, g[a] - r);
            hi[a] = min(I.gdim[a] - 1, g[a] + r);
        }
    }
    for (int z = lo[2]; z <= hi[2]; z++)
        for (int y = lo[1]; y <= hi[1]; y++)
            for (int x = lo[0]; x <= hi[0]; x++) {
                int w[3] = { I.periodic[0] ? wrap_idx(x, I.gdim[0]) : x, I.periodic[1] ? wrap_idx(y, I.gdim[1]) : y,
                             I.periodic[2] ? wrap_idx(z, I.gdim[2]) : z };
                if (r > 0 && in_cube(w, g, r - 1, I)) continue;
                long long gg = I.g0 + ((long long)w[2] * I.gdim[1] + w[1]) * I.gdim[0] + w[0];
                f(gg);
            }
}

// lower bound of the distance from p to anything outside the searched cube
__device__ inline float shell_bound(const float p[3], const int g[3], int r, const Inst& I, bool& exhausted) {
    float lb = 3.0e38f;
    exhausted = true;
    for (int a = 0; a < 3; a++) {
        if (I.periodic[a]) {
            if (2 * r + 1 >= I.gdim[a]) continue;
            float h = I.gh[a];
            float lo = p[a] - (g[a] - r) * h, hi = (g[a] + r + 1) * h - p[a];
            lb = fminf(lb, fminf(lo, hi));
            exhausted = false;
        } else {
            if (g[a] - r > 0) { lb = fminf(lb, p[a] - (g[a] - r) * I.gh[a]); exhausted = false; }
            if (g[a] + r < I.gdim[a] - 1) { lb = fminf(lb, (g[a] + r + 1) * I.gh[a] - p[a]); exhausted = false; }
        }
    }
    return lb;
}

// lbound (nullable) receives a lower bound on the distance from the particle
// to every centroid but the one it is assigned: the second-best scanned
// distance or the bound on the unscanned shells, whichever is smaller (0
// when the winner was decided inside the tie band).
__device__ void estep_one(const View& v, int i, int* __restrict__ cell_out, float* __restrict__ lbound = nullptr) {
    int b = find_inst(v.inst_p0, v.B, i);
    const Inst& I = v.inst[b];
    long long xq[3] = { v.xq[i], v.xq[(size_t)v.N + i], v.xq[(size_t)2 * v.N + i] };
    float p[3];
    int g[3];
    for (int a = 0; a < 3; a++) g[a] = grid_coord(xq[a], I, a, p[a]);
    float best = 3.0e38f, second = 3.0e38f;     // FP32 distances squared
    float lbx = 3.0e38f;                         // bound on the unscanned shells
    int r = 0;
    const int rmax = max(I.gdim[0], max(I.gdim[1], I.gdim[2]));
    for (;; r++) {
        for_shell(g, r, I, [&](long long gg) {
            for (int q = v.gstart[gg]; q < v.gstart[gg + 1]; q++) {
                float4 c = v.gcf[q];
                float dx = axis_dist(p[0], c.x, I, 0), dy = axis_dist(p[1], c.y, I, 1), dz = axis_dist(p[2], c.z, I, 2);
                float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                second = fminf(second, fmaxf(best, d2));
                best = fminf(best, d2);
            }
        });
        bool ex;
        float lb = shell_bound(p, g, r, I, ex);
        if (ex || r >= rmax) break;
        if (best < 3.0e38f && lb > sqrtf(best) + kBandE) { lbx = lb; break; }
    }
    // second pass over the searched cube: candidates within the band
    float lim = sqrtf(best) + kBandE;
    float lim2 = lim * lim;
    int ncand = 0, k1 = -1, bestk = -1;
    double best64 = 0.0;
    for (int rr = 0; rr <= r; rr++) {
        for_shell(g, rr, I, [&](long long gg) {
            for (int q = v.gstart[gg]; q < v.gstart[gg + 1]; q++) {
                float4 c = v.gcf[q];
                float dx = axis_dist(p[0], c.x, I, 0), dy = axis_dist(p[1], c.y, I, 1), dz = axis_dist(p[2], c.z, I, 2);
                float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (d2 <= lim2) {
                    int k = __float_as_int(c.w);
                    ncand++;
                    if (ncand == 1) { k1 = k; continue; }
                    if (ncand == 2) {
                        best64 = dist2_grid_d(xq[0], xq[1], xq[2], v.cq[k1], v.cq[(size_t)v.Ktot + k1],
                                              v.cq[(size_t)2 * v.Ktot + k1], I);
                        bestk = k1;
                    }
                    double d64 = dist2_grid_d(xq[0], xq[1], xq[2], v.cq[k], v.cq[(size_t)v.Ktot + k],
                                              v.cq[(size_t)2 * v.Ktot + k], I);
                    if (d64 < best64 || (d64 == best64 && k < bestk)) { best64 = d64; bestk = k; }
                }
            }
        });
    }
    if (ncand == 0) {   // unreachable for finite input: the search covers every centroid
        flag_inst(v, I, kStatusGridRange);
        cell_out[i] = I.k0;
        if (lbound) lbound[i] = 0.f;
        return;
    }
    cell_out[i] = (ncand == 1) ? k1 : bestk;
    if (lbound) lbound[i] = (ncand == 1) ? fminf(sqrtf(second), lbx) : 0.f;
}

// ---- warp-cooperative search for instances without periodic axes: the
// 32 queries of a warp (consecutive storage slots, hence neighbours in space)
// share one grid region [lo - r, hi + r]; every lane scores every centroid
// of the region (broadcast loads), and the region grows by one ring until
// each lane's unexplored space is provably farther than its band.
template <typename F>
__device__ inline void region_ring(const Inst& I, const int lo[3], const int hi[3], int r, F&& f) {
    int a0[3], a1[3];
    for (int a = 0; a < 3; a++) { a0[a] = max(0, lo[a] - r); a1[a] = min(I.gdim[a] - 1, hi[a] + r); }
    for (int z = a0[2]; z <= a1[2]; z++)
        for (int y = a0[1]; y <= a1[1]; y++)
            for (int x = a0[0]; x <= a1[0]; x++) {
                if (r > 0 && x >= lo[0] - r + 1 && x <= hi[0] + r - 1 && y >= lo[1] - r + 1 && y <= hi[1] + r - 1 &&
                    z >= lo[2] - r + 1 && z <= hi[2] + r - 1)
                    continue;
                f(I.g0 + ((long long)z * I.gdim[1] + y) * I.gdim[0] + x);
            }
}

__device__ inline float region_bound(const Inst& I, const float p[3], const int lo[3], const int hi[3], int r,
                                     bool& exhausted) {
    float lb = 3.0e38f;
    exhausted = true;
    for (int a = 0; a < 3; a++) {
        if (lo[a] - r > 0) { lb = fminf(lb, p[a] - (lo[a] - r) * I.gh[a]); exhausted = false; }
        if (hi[a] + r < I.gdim[a] - 1) { lb = fminf(lb, (hi[a] + r + 1) * I.gh[a] - p[a]); exhausted = false; }
    }
    return lb;
}

__device__ inline void warp_box(const int g[3], bool valid, int lo[3], int hi[3]) {
    for (int a = 0; a < 3; a++) {
        int l = valid ? g[a] : 0x7fffffff, h = valid ? g[a] : -1;
        for (int off = 16; off; off >>= 1) {
            l = min(l, __shfl_xor_sync(0xffffffffu, l, off));
            h = max(h, __shfl_xor_sync(0xffffffffu, h, off));
        }
        lo[a] = l;
        hi[a] = h;
    }
}

// list (nullable): search only the *count particles listed (in list order,
// which keeps the lanes of a warp close in space)
__global__ void k_estep_warp(View v, int* __restrict__ cell_out, float* __restrict__ lbound,
                             const int* __restrict__ list, const int* __restrict__ count) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = list ? q < *count : q < v.N;
    const int i = valid ? (list ? list[q] : q) : 0;
    const int b = valid ? find_inst(v.inst_p0, v.B, i) : -1;
    int b0 = __shfl_sync(0xffffffffu, b, 0);
    const int bfirst = __reduce_max_sync(0xffffffffu, valid ? b : -1);
    if (b0 < 0) b0 = bfirst;
    const bool same = __all_sync(0xffffffffu, !valid || b == b0);
    if (b0 < 0) return;
    const Inst& I = v.inst[b0];
    const bool periodic = I.periodic[0] | I.periodic[1] | I.periodic[2];
    if (!same || periodic) {
        // mixed instances or periodic axes: per-thread shell search
        if (valid) estep_one(v, i, cell_out, lbound);
        return;
    }
    long long xq[3] = {0, 0, 0};
    float p[3] = {0, 0, 0};
    int g[3] = {0, 0, 0};
    if (valid) {
        xq[0] = v.xq[i]; xq[1] = v.xq[(size_t)v.N + i]; xq[2] = v.xq[(size_t)2 * v.N + i];
        for (int a = 0; a < 3; a++) g[a] = grid_coord(xq[a], I, a, p[a]);
    }
    int lo[3], hi[3];
    warp_box(g, valid, lo, hi);
    if (hi[0] - lo[0] > 2 || hi[1] - lo[1] > 2 || hi[2] - lo[2] > 2) {
        // queries not clustered in space (e.g. input order): per-thread search
        if (valid) estep_one(v, i, cell_out, lbound);
        return;
    }
    float best = 3.0e38f, second = 3.0e38f;
    float lbr = 3.0e38f;    // bound on the unscanned region after the last ring
    int bk = -1;
    int r = 0;
    for (;; r++) {
        region_ring(I, lo, hi, r, [&](long long gg) {
            const int q1 = v.gstart[gg + 1];
            for (int q = v.gstart[gg]; q < q1; q++) {
                const float4 c = v.gcf[q];
                const float dx = p[0] - c.x, dy = p[1] - c.y, dz = p[2] - c.z;
                const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (d2 < best) { second = best; best = d2; bk = __float_as_int(c.w); }
                else if (d2 < second) second = d2;
            }
        });
        bool ex;
        const float lb = region_bound(I, p, lo, hi, r, ex);
        lbr = ex ? 3.0e38f : lb;
        const bool done = !valid || ex || (best < 3.0e38f && lb > sqrtf(best) + kBandE);
        if (__all_sync(0xffffffffu, done)) break;
    }
    // tie band: every centroid within the band of the FP32 best is re-scored in FP64
    const float lim = sqrtf(best) + kBandE;
    const bool amb = valid && second <= lim * lim;
    if (__any_sync(0xffffffffu, amb)) {
        double best64 = 1e300;
        int bk64 = -1;
        for (int rr = 0; rr <= r; rr++)
            region_ring(I, lo, hi, rr, [&](long long gg) {
                const int q1 = v.gstart[gg + 1];
                for (int q = v.gstart[gg]; q < q1; q++) {
                    const float4 c = v.gcf[q];
                    const float dx = p[0] - c.x, dy = p[1] - c.y, dz = p[2] - c.z;
                    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (amb && d2 <= lim * lim) {
                        const int k = __float_as_int(c.w);
                        const double d64 = dist2_grid_d(xq[0], xq[1], xq[2], v.cq[k], v.cq[(size_t)v.Ktot + k],
                                                        v.cq[(size_t)2 * v.Ktot + k], I);
                        if (d64 < best64 || (d64 == best64 && k < bk64)) { best64 = d64; bk64 = k; }
                    }
                }
            });
        if (amb) bk = bk64;
    }
    if (valid) {
        if (bk < 0) { flag_inst(v, I, kStatusGridRange); bk = I.k0; }
        cell_out[i] = bk;
        if (lbound) lbound[i] = amb ? 0.f : fminf(sqrtf(second), lbr);
    }
}

__global__ void k_estep(View v, int* __restrict__ cell_out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < v.N) estep_one(v, i, cell_out);
}

// Grid search for the particles the certified E-step could not decide.
__global__ void k_estep_list(View v, const int* __restrict__ fb_list, const int* __restrict__ fb_count,
                             int* __restrict__ cell_out, float* __restrict__ lbound = nullptr) {
    const int n = *fb_count;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
        estep_one(v, fb_list[q], cell_out, lbound);
}

// Largest move of the centroids now in each grid cell (FP32 bits:
// non-negative floats order like their bit patterns).
__global__ void k_grid_move(View v, const int* __restrict__ gidx, const float* __restrict__ cmove,
                            unsigned* __restrict__ gmove) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < v.Ktot) atomicMax(&gmove[gidx[k]], __float_as_uint(cmove[k]));
}

// k-means E-step after the first round (Hamerly's bound): the particle's
// centroid of the previous round is still its nearest when the distance to
// it is below the previous lower bound on every other centroid, less the
// largest move of the M-step in between (FP32 with a margin); the bound is
// carried on, the others are listed for the grid search.  When the bound is
// below the grid edge, every centroid that could now be nearer lies in the
// 27 grid cells around the particle, and the largest move among those
// replaces the instance's largest move.
__global__ void __launch_bounds__(256) k_estep_bound(View v, const int* __restrict__ cell, float* __restrict__ lbound,
                                                     const float4* __restrict__ cf, const unsigned* __restrict__ dmax,
                                                     const unsigned* __restrict__ gmove, int* __restrict__ list,
                                                     int* __restrict__ count) {
    __shared__ int wcount[8], wbase[8], bbase;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool need = false;
    if (i < v.N) {
        const int b = find_inst(v.inst_p0, v.B, i);
        const Inst& I = v.inst[b];
        float p[3];
        int g[3];
        for (int a = 0; a < 3; a++) g[a] = grid_coord(v.xq[(size_t)a * v.N + i], I, a, p[a]);
        const float4 c = cf[cell[i]];
        const float dx = axis_dist(p[0], c.x, I, 0), dy = axis_dist(p[1], c.y, I, 1), dz = axis_dist(p[2], c.z, I, 2);
        const float l0 = lbound[i];
        float dm = __uint_as_float(dmax[b]);
        if (gmove && l0 <= fminf(I.gh[0], fminf(I.gh[1], I.gh[2]))) {
            unsigned m = 0;
            for (int zz = -1; zz <= 1; zz++)
                for (int yy = -1; yy <= 1; yy++)
                    for (int xx = -1; xx <= 1; xx++) {
                        int w[3] = {g[0] + xx, g[1] + yy, g[2] + zz};
                        for (int a = 0; a < 3; a++)
                            w[a] = I.periodic[a] ? wrap_idx(w[a], I.gdim[a]) : min(max(w[a], 0), I.gdim[a] - 1);
                        m = max(m, gmove[I.g0 + ((long long)w[2] * I.gdim[1] + w[1]) * I.gdim[0] + w[0]]);
                    }
            dm = __uint_as_float(m);
        }
        const float l = l0 - dm;
        if (sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))) + kCertMargin < l) lbound[i] = l;
        else need = true;
    }
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (lane == 0) wcount[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < 8; w++) { wbase[w] = tot; tot += wcount[w]; }
        bbase = tot ? atomicAdd(count, tot) : 0;
    }
    __syncthreads();
    if (need) list[bbase + wbase[warp] + __popc(m & ((1u << lane) - 1u))] = i;
}

// The previous rows with their cells renumbered and the renumbered cells'
// FP32 centroids (w = new index), so the E-step reads one record per
// candidate instead of three dependent loads.
__global__ void k_cand_rows(const int* __restrict__ cnt_old, int Ktot, const int* __restrict__ pad_old,
                            const int* __restrict__ new_of_old, const float4* __restrict__ cf,
                            float4* __restrict__ rows) {
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // one thread per row slot
    if (q >= (long long)Ktot * kAdjRow || (int)(q % kAdjRow) >= cnt_old[q / kAdjRow]) return;
    const int j = new_of_old[pad_old[q]];
    float4 c = cf[j];
    c.w = __int_as_float(j);
    rows[q] = c;
}

// Rebuild E-step from the previous cell list (the paper's guess from the
// previous particle, made exact), one thread per particle: the candidates
// are the particle's previous cell and its previous neighbouring cells (one
// row; the lanes of a warp mostly share it), renumbered by the Morton
// relabel.  Every centroid outside the row was at least rho_k from the old
// centroid c_k when the list was built (rho_k: distance to the nearest
// non-neighbour), and every centroid has since moved at most dmax, so none
// of them is within best + band of the particle when
//   sqrt(best) + band < rho_k - 2 dmax - |x - c_k|   (FP32 with margins).
// Particles that fail the test take the grid search.
__global__ void __launch_bounds__(128, 16) k_estep_rows(View v, const int* __restrict__ cell_old,
                                                    const int* __restrict__ cnt_old, const float4* __restrict__ rows,
                                                    const float* __restrict__ rho_old, const int* __restrict__ new_of_old,
                                                    const unsigned* __restrict__ dmax, int* __restrict__ cell_out,
                                                    int* __restrict__ fb_list, int* __restrict__ fb_count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool fail = false;
    if (i < v.N) {
        const int b = find_inst(v.inst_p0, v.B, i);
        const Inst& I = v.inst[b];
        long long xq[3];
        float p[3];
        for (int a = 0; a < 3; a++) {
            xq[a] = v.xq[(size_t)a * v.N + i];
            grid_coord(xq[a], I, a, p[a]);
        }
        const int ko = cell_old[i], kn = new_of_old[ko];
        const int a0 = ko * kAdjRow, a1 = a0 + min(cnt_old[ko], kAdjRow);
        float best = 3.0e38f, second = 3.0e38f, dself2 = 3.0e38f;
        int bk = -1;
        for (int r = a0; r < a1; r++) {
            const float4 c = rows[r];
            const int j = __float_as_int(c.w);
            if (j < I.k0 || j >= I.k0 + I.K) continue;    // a cell of the other set
            const float dx = axis_dist(p[0], c.x, I, 0), dy = axis_dist(p[1], c.y, I, 1), dz = axis_dist(p[2], c.z, I, 2);
            const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (j == kn) dself2 = d2;
            if (d2 < best || (d2 == best && j < bk)) { second = best; best = d2; bk = j; }
            else if (d2 < second) second = d2;
        }
        const float lim = sqrtf(best) + kBandE;
        const float cert = rho_old[ko] - 2.0f * __uint_as_float(dmax[b]) - sqrtf(dself2) - kCertMargin;
        fail = bk < 0 || dself2 >= 3.0e38f || !(lim < cert);
        if (!fail) {
            if (second > lim * lim) {
                cell_out[i] = bk;
            } else {
                // tie band: FP64 among the row's candidates within it
                double best64 = 1e300;
                int bk64 = -1;
                for (int r = a0; r < a1; r++) {
                    const float4 c = rows[r];
                    const int j = __float_as_int(c.w);
                    if (j < I.k0 || j >= I.k0 + I.K) continue;
                    const float dx = axis_dist(p[0], c.x, I, 0), dy = axis_dist(p[1], c.y, I, 1),
                                dz = axis_dist(p[2], c.z, I, 2);
                    if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= lim * lim) {
                        const double d64 = dist2_grid_d(xq[0], xq[1], xq[2], v.cq[j], v.cq[(size_t)v.Ktot + j],
                                                        v.cq[(size_t)2 * v.Ktot + j], I);
                        if (d64 < best64 || (d64 == best64 && j < bk64)) { best64 = d64; bk64 = j; }
                    }
                }
                cell_out[i] = bk64;
            }
        }
    }
    // the rare failures to the grid search's list, one atomic per warp
    const unsigned m = __ballot_sync(0xffffffffu, fail);
    if (m) {
        const int lane = threadIdx.x & 31, first = __ffs(m) - 1;
        int base = 0;
        if (lane == first) base = atomicAdd(fb_count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, first);
        if (fail) fb_list[base + __popc(m & ((1u << lane) - 1u))] = i;
    }
}

// ============================================================== stable counting sort
// Consecutive particles mostly share a cell: one atomic per distinct cell of
// a warp (lanes with the same cell found with a match).
__global__ void k_hist(int N, const int* __restrict__ cell, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (i < N) ? cell[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int lane = threadIdx.x & 31;
    if (c >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[c], __popc(peers));
}

// Slot of each particle inside its cell's range (in any order across warps;
// the per-cell sort that follows restores the storage order).
__global__ void k_scatter(int N, const int* __restrict__ cell, const int* __restrict__ start, int* __restrict__ cursor,
                          int* __restrict__ tmp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = (i < N) ? cell[i] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (c >= 0 && lane == leader) base = atomicAdd(&cursor[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    if (c >= 0) tmp[start[c] + base + __popc(peers & ((1u << lane) - 1u))] = i;
}

// Sort each cell's slot list ascending (= old storage order), which makes the
// scatter stable.  One block per cell, bitonic in shared memory.
constexpr int kSegMax = 2048;
__global__ void k_segsort(int Ktot, const int* __restrict__ start, int* __restrict__ tmp, unsigned* status) {
    __shared__ int sh[kSegMax];
    for (int k = blockIdx.x; k < Ktot; k += gridDim.x) {
    int s = start[k], e = start[k + 1], n = e - s;
    if (n <= 128 || n > kSegMax) continue;   // warp kernel / k_segrank
    int m = 1;
    while (m < n) m <<= 1;
    for (int t = threadIdx.x; t < m; t += blockDim.x) sh[t] = (t < n) ? tmp[s + t] : 0x7fffffff;
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                int p = t ^ stride;
                if (p > t) {
                    bool up = (t & size) == 0;
                    int a = sh[t], c = sh[p];
                    if ((c < a) == up) { sh[t] = c; sh[p] = a; }
                }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < n; t += blockDim.x) tmp[s + t] = sh[t];
    __syncthreads();
    }
}

// Cells of up to 128 particles: one warp, bitonic network over 4 values per
// lane (element e = lane + 32 q), shuffles for strides < 32.
__global__ void k_segsort_warp(int Ktot, const int* __restrict__ start, int* __restrict__ tmp) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= Ktot) return;
    const int s = start[k], n = start[k + 1] - s;
    if (n <= 1 || n > 128) return;
    int val[4];
#pragma unroll
    for (int q = 0; q < 4; q++) val[q] = (lane + 32 * q < n) ? tmp[s + lane + 32 * q] : 0x7fffffff;
#pragma unroll
    for (int size = 2; size <= 128; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int qs = stride >> 5;
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    if (q & qs) continue;
                    const int e = lane + 32 * q;
                    const bool up = (e & size) == 0;
                    const int a = val[q], c = val[q | qs];
                    val[q] = up ? min(a, c) : max(a, c);
                    val[q | qs] = up ? max(a, c) : min(a, c);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int e = lane + 32 * q;
                    const int other = __shfl_xor_sync(0xffffffffu, val[q], stride);
                    const bool up = (e & size) == 0;
                    const bool lower = (e & stride) == 0;
                    val[q] = (lower == up) ? min(val[q], other) : max(val[q], other);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (lane + 32 * q < n) tmp[s + lane + 32 * q] = val[q];
}

// Cells larger than kSegMax: each slot's rank among its cell's (distinct)
// old indices, O(n^2) per such cell; writes the ordered list to out.
__global__ void k_segrank(int N, const int* __restrict__ cell, const int* __restrict__ start, const int* __restrict__ tmp,
                          int* __restrict__ out) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;   // slot in the scattered order
    if (q >= N) return;
    int c = cell[tmp[q]];
    int s = start[c], e = start[c + 1];
    if (e - s <= kSegMax) return;
    int me = tmp[q], r = 0;
    for (int t = s; t < e; t++) r += (tmp[t] < me);
    out[s + r] = me;
}

__global__ void k_segcopy(int N, const int* __restrict__ cell, const int* __restrict__ start, const int* __restrict__ src,
                          int* __restrict__ tmp) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= N) return;
    int c = cell[tmp[q]];
    if (start[c + 1] - start[c] > kSegMax) tmp[q] = src[q];
}

// Cells that the warp sort cannot take: 128 < n <= kSegMax into list A
// (block bitonic), n > kSegMax into list B (exact rank); counts in cnt[0..1].
__global__ void k_seglist(int Ktot, const int* __restrict__ start, int* __restrict__ la, int* __restrict__ lb,
                          int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = (k < Ktot) ? start[k + 1] - start[k] : 0;
    const bool a = n > 128 && n <= kSegMax, bb = n > kSegMax;
    const int lane = threadIdx.x & 31;
    const unsigned ma = __ballot_sync(0xffffffffu, a), mb = __ballot_sync(0xffffffffu, bb);
    int baseA = 0, baseB = 0;
    if (ma && lane == __ffs(ma) - 1) baseA = atomicAdd(&cnt[0], __popc(ma));
    if (mb && lane == __ffs(mb) - 1) baseB = atomicAdd(&cnt[1], __popc(mb));
    baseA = __shfl_sync(0xffffffffu, baseA, ma ? __ffs(ma) - 1 : 0);
    baseB = __shfl_sync(0xffffffffu, baseB, mb ? __ffs(mb) - 1 : 0);
    const unsigned lt = (1u << lane) - 1u;
    if (a) la[baseA + __popc(ma & lt)] = k;
    if (bb) lb[baseB + __popc(mb & lt)] = k;
}

// List A: one block per cell, bitonic sort of its slot list in shared memory.
__global__ void k_segsort_list(const int* __restrict__ start, const int* __restrict__ la, const int* __restrict__ cnt,
                               int* __restrict__ tmp) {
    __shared__ int sh[kSegMax];
    const int nl = cnt[0];
    for (int e = blockIdx.x; e < nl; e += gridDim.x) {
        const int k = la[e];
        const int s0 = start[k], n = start[k + 1] - s0;
        int m = 1;
        while (m < n) m <<= 1;
        for (int t = threadIdx.x; t < m; t += blockDim.x) sh[t] = (t < n) ? tmp[s0 + t] : 0x7fffffff;
        __syncthreads();
        for (int size = 2; size <= m; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int t = threadIdx.x; t < m; t += blockDim.x) {
                    const int p = t ^ stride;
                    if (p > t) {
                        const bool up = (t & size) == 0;
                        const int a = sh[t], c = sh[p];
                        if ((c < a) == up) { sh[t] = c; sh[p] = a; }
                    }
                }
                __syncthreads();
            }
        for (int t = threadIdx.x; t < n; t += blockDim.x) tmp[s0 + t] = sh[t];
        __syncthreads();
    }
}

// List B: one block per cell; every slot's rank among the cell's slots (they
// are distinct), written to out, then copied back.
__global__ void k_segrank_list(const int* __restrict__ start, const int* __restrict__ lb, const int* __restrict__ cnt,
                               int* __restrict__ tmp, int* __restrict__ out) {
    const int nl = cnt[1];
    for (int e = blockIdx.x; e < nl; e += gridDim.x) {
        const int k = lb[e];
        const int s0 = start[k], s1 = start[k + 1];
        for (int q = s0 + threadIdx.x; q < s1; q += blockDim.x) {
            const int me = tmp[q];
            int r = 0;
            for (int t = s0; t < s1; t++) r += (tmp[t] < me);
            out[s0 + r] = me;
        }
        __syncthreads();
        for (int q = s0 + threadIdx.x; q < s1; q += blockDim.x) tmp[q] = out[q];
        __syncthreads();
    }
}

// ============================================================== gather + mirrors
// The mirrors hold x - c~ at 2^-26 sigma, where c~ is the centroid rounded to
// a multiple of 2^-26 sigma: then round(x - c~) = round(x) - c~ exactly, and
// a pair's integer displacement m_j + (c~_l - c~_k) - m_i depends on the two
// positions alone (and, on a periodic axis, on the image), not on which
// cells hold them, so FP32 pair forces do not change when the cell list is
// rebuilt.
__device__ inline long long mirror_ref(long long c) {
    return ((c + (1ll << (kMirrorShift - 1))) >> kMirrorShift) << kMirrorShift;
}
__device__ inline int mirror_coord(long long xq, long long cq, const Inst& I, int a, const View& v) {
    long long d = minimg_q(xq - mirror_ref(cq), I.boxq[a], I.periodic[a]);
    long long r = (d + (1ll << (kMirrorShift - 1))) >> kMirrorShift;
    if (r > 2147483647ll || r < -2147483647ll) { flag_inst(v, I, kStatusMirrorRange); r = 0; }
    return (int)r;
}

// Cell radius R_k = max_i |x_i - c_k| over the cell (all types), equal to
// the FP64 definition: FP32 from the exact mirror (error < 1e-6 sigma) finds
// the candidates within this band of the maximum, FP64 decides among them.
constexpr float kBandR = 1e-5f;

// Gather of the cell-sorted state, one thread per new slot p: the particle
// of old slot perm[p] moves with its state, type and id, learns its new cell
// (the E-step's result for the old slot) and gets its exact mirror relative
// to that cell's centroid.  Every load and the mirror come before the first
// store: as far as the compiler knows the stores may alias the sources, and
// interleaved they would serialise the loads' latencies.
__global__ void __launch_bounds__(256) k_gather_particles(View v, View o, const int* __restrict__ perm,
                                                          const int* __restrict__ cell_new,
                                                          long long* __restrict__ xref) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const size_t N = v.N;
    const int so = perm[p];
    const int k = cell_new[so];
    long long x[3], vq[3], nq[3], wq[3];
    for (int a = 0; a < 3; a++) {
        x[a] = o.xq[a * N + so];
        vq[a] = o.vq[a * N + so];
        nq[a] = o.nq[a * N + so];
        wq[a] = o.wq[a * N + so];
    }
    const unsigned char t = o.type[so];
    const unsigned id = o.id[so];
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    int4 m;
    m.x = mirror_coord(x[0], v.cq[k], I, 0, v);
    m.y = mirror_coord(x[1], v.cq[(size_t)v.Ktot + k], I, 1, v);
    m.z = mirror_coord(x[2], v.cq[(size_t)2 * v.Ktot + k], I, 2, v);
    const int q0 = I.p0 + (int)id;
    m.w = t | (v.bptr[q0] < v.bptr[q0 + 1] ? kMirrorBonded : 0);
    float4 no;
    no.x = ll_to_float(nq[0]) * (float)kGridInv;
    no.y = ll_to_float(nq[1]) * (float)kGridInv;
    no.z = ll_to_float(nq[2]) * (float)kGridInv;
    no.w = __int_as_float(p);
    for (int a = 0; a < 3; a++) {
        v.xq[a * N + p] = x[a];
        v.vq[a * N + p] = vq[a];
        v.nq[a * N + p] = nq[a];
        v.wq[a * N + p] = wq[a];
        if (xref) xref[a * N + p] = x[a];
    }
    v.type[p] = t;
    v.id[p] = id;
    v.cell[p] = k;
    v.slot_of_id[q0] = p;
    v.mq[p] = m;
    v.mo[p] = no;
}

// Bitonic sort of 32 * NE records over a warp, slot lane + 32 u held in
// r[u] (records of r beyond NE untouched); slots at a distance >= 32 are
// exchanged inside a lane.
template <int NE>
__device__ inline void warp_bitonic_u32(unsigned (&r)[4], int lane) {
#pragma unroll
    for (int size = 2; size <= 32 * NE; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int du = stride >> 5;
#pragma unroll
                for (int u = 0; u < NE; u++) {
                    if (u & du) continue;
                    const bool up = ((lane + 32 * u) & size) == 0;
                    const unsigned x = r[u], y = r[u + du];
                    r[u] = up ? min(x, y) : max(x, y);
                    r[u + du] = up ? max(x, y) : min(x, y);
                }
            } else {
#pragma unroll
                for (int u = 0; u < NE; u++) {
                    const int e = lane + 32 * u;
                    const unsigned o = __shfl_xor_sync(0xffffffffu, r[u], stride);
                    const bool up = (e & size) == 0;
                    const bool lower = (e & stride) == 0;
                    r[u] = (lower == up) ? min(r[u], o) : max(r[u], o);
                }
            }
        }
    }
}

// Per-cell quantities read back from the gathered mirrors: one warp per cell
// computes the squared cell radius R_k^2 = max |x - c_k|^2 (FP32 with the
// FP64 definition inside a band; left in R for k_cell_radius), the pair
// kernel's cell normal (mean bilayer director, unit; +z without one) and, in
// each tile of 128 particles, every particle's rank along the tile's longer
// tangent extent.  rmax_bits: each instance's largest R_k^2 (bit pattern).
// Launched with 256 threads (8 warps, one cell each).
__global__ void __launch_bounds__(256, 6) k_cell_props(View v, unsigned long long* __restrict__ rmax_bits /* [B] */) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= v.Ktot) return;
    const int b = find_inst(v.inst_k0, v.B, k);
    const Inst& I = v.inst[b];
    const int s = v.cell_start[k], e = v.cell_start[k + 1];
    const size_t N = v.N;
    const long long ck[3] = {v.cq[k], v.cq[(size_t)v.Ktot + k], v.cq[(size_t)2 * v.Ktot + k]};
    float mx = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
    for (int p = s + lane; p < e; p += 32) {
        const int4 m = v.mq[p];
        const float4 no = v.mo[p];
        const float dx = m.x * kMirrorUnit, dy = m.y * kMirrorUnit, dz = m.z * kMirrorUnit;
        mx = fmaxf(mx, sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))));
        if (bilayer(m.w & 0xff)) { nx += no.x; ny += no.y; nz += no.z; }
    }
    for (int off = 16; off; off >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        nx += __shfl_xor_sync(0xffffffffu, nx, off);
        ny += __shfl_xor_sync(0xffffffffu, ny, off);
        nz += __shfl_xor_sync(0xffffffffu, nz, off);
    }
    // radius: FP64 definition for the particles within the band of the FP32 max
    double best = 0.0;
    for (int p = s + lane; p < e; p += 32) {
        const int4 m = v.mq[p];
        const float dx = m.x * kMirrorUnit, dy = m.y * kMirrorUnit, dz = m.z * kMirrorUnit;
        const float d = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        if (d >= mx - kBandR) {
            const double d2 = dist2_grid_d(v.xq[p], v.xq[N + p], v.xq[2 * N + p], ck[0], ck[1], ck[2], I);
            best = fmax(best, d2);
        }
    }
    // the max over the lanes on the bit patterns (a non-negative double's
    // bits order like its value): integer operations, not the FP64 pipe
    unsigned long long bb = (unsigned long long)__double_as_longlong(best);
    for (int off = 16; off; off >>= 1) bb = max(bb, (unsigned long long)__shfl_xor_sync(0xffffffffu, bb, off));
    best = __longlong_as_double((long long)bb);
    // the squared radius for now (k_cell_radius takes the square roots, one
    // cell per thread), and each instance's largest square
    if (lane == 0) {
        v.R[k] = best;
        atomicMax(&rmax_bits[b], bb);
    }
    // pair-kernel frame
    const float nn = sqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
    if (nn > 1e-3f) { nx /= nn; ny /= nn; nz /= nn; }
    else { nx = 0.f; ny = 0.f; nz = 1.f; }
    if (lane == 0) v.cnorm[k] = make_float4(nx, ny, nz, 0.f);
    const Frame F = tangent_frame(nx, ny, nz);
    // pair-kernel groups: ranks inside each tile of 128 particles
    for (int t0 = s; t0 < e; t0 += 128) {
        const int nt = min(128, e - t0);
        float ya[4], yb[4];
        float lo_a = 3.0e38f, hi_a = -3.0e38f, lo_b = 3.0e38f, hi_b = -3.0e38f;
        for (int u = 0; u < 4; u++) {
            const int t = lane + 32 * u;
            ya[u] = 0.f; yb[u] = 0.f;
            if (t < nt) {
                const int4 m = v.mq[t0 + t];
                float c;
                F.apply(m.x * kMirrorUnit, m.y * kMirrorUnit, m.z * kMirrorUnit, ya[u], yb[u], c);
                lo_a = fminf(lo_a, ya[u]); hi_a = fmaxf(hi_a, ya[u]);
                lo_b = fminf(lo_b, yb[u]); hi_b = fmaxf(hi_b, yb[u]);
            }
        }
        for (int off = 16; off; off >>= 1) {
            lo_a = fminf(lo_a, __shfl_xor_sync(0xffffffffu, lo_a, off));
            hi_a = fmaxf(hi_a, __shfl_xor_sync(0xffffffffu, hi_a, off));
            lo_b = fminf(lo_b, __shfl_xor_sync(0xffffffffu, lo_b, off));
            hi_b = fmaxf(hi_b, __shfl_xor_sync(0xffffffffu, hi_b, off));
        }
        const bool use_a = (hi_a - lo_a) >= (hi_b - lo_b);
        // 32-bit records: the key quantised to 24 bits over the tile's
        // extent (monotone), the tile index in the low 7 bits (equal keys
        // go by index); the rank of a particle is the slot its record ends
        // in after a warp bitonic sort
        const float klo = use_a ? lo_a : lo_b, kext = use_a ? hi_a - lo_a : hi_b - lo_b;
        const float ksc = kext > 0.f ? 16777215.0f / kext : 0.f;
        unsigned r[4];
        for (int u = 0; u < 4; u++) {
            const int t = lane + 32 * u;
            const float y = use_a ? ya[u] : yb[u];
            r[u] = (t < nt) ? (min(16777215u, (unsigned)((y - klo) * ksc)) << 7) | (unsigned)t : 0xffffffffu;
        }
        if (nt <= 64) warp_bitonic_u32<2>(r, lane);
        else warp_bitonic_u32<4>(r, lane);
        for (int u = 0; u < 4; u++) {
            if (r[u] == 0xffffffffu) continue;
            const int t = (int)(r[u] & 127u), q = lane + 32 * u;
            v.grank[t0 + t] = (unsigned char)q;
            v.mqr[t0 + q] = v.mq[t0 + t];
            v.mor[t0 + q] = v.mo[t0 + t];
        }
        __syncwarp();
    }
}


// Mirrors of the current order (after integration without a rebuild),
// written where the pair kernel reads them: slot p of its cell's tile of 128
// goes to the tile's position grank[p].
__global__ void k_mirrors(View v) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    size_t N = v.N;
    int c = v.cell[p];
    int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    int4 m;
    m.x = mirror_coord(v.xq[p], v.cq[c], I, 0, v);
    m.y = mirror_coord(v.xq[N + p], v.cq[(size_t)v.Ktot + c], I, 1, v);
    m.z = mirror_coord(v.xq[2 * N + p], v.cq[(size_t)2 * v.Ktot + c], I, 2, v);
    const unsigned id = v.id[p];
    m.w = v.type[p] | (v.bptr[I.p0 + id] < v.bptr[I.p0 + id + 1] ? kMirrorBonded : 0);
    float4 no;
    no.x = ll_to_float(v.nq[p]) * (float)kGridInv;
    no.y = ll_to_float(v.nq[N + p]) * (float)kGridInv;
    no.z = ll_to_float(v.nq[2 * N + p]) * (float)kGridInv;
    no.w = __int_as_float(p);
    const int cs = v.cell_start[c];
    const int q = cs + ((p - cs) & ~127) + (int)v.grank[p];
    v.mqr[q] = m;
    v.mor[q] = no;
}

// Cell radii R_k = sqrt(R_k^2) from k_cell_props and their FP32 copies, one
// thread per cell: an FP64 instruction occupies the FP64 pipe for a whole
// warp, so 32 cells share each square root instead of one.
__global__ void k_cell_radius(View v) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= v.Ktot) return;
    const double R = __dsqrt_rn(v.R[k]);
    v.R[k] = R;
    v.Rf[k] = (float)R;
}

// ============================================================== neighbouring cells
// nbr(k) = { j : |c_k - c_j| < ((R_k + R_j) + r_s + 2 skin)(1 + 1e-12) },
// evaluated exactly as the FP64 definition for candidates within a band of
// the threshold, and by an FP32 test with margin elsewhere.
constexpr float kBandA = 2e-3f;

// exact neighbouring-cell test of (k, j), FP32 with a margin outside the
// band and the definition's FP64 operations inside it
__device__ inline bool adj_test(const View& v, const Inst& I, int k, int j, double Rk, float Rkf, float df,
                                long long cx, long long cy, long long cz, float tailf) {
    // FP32 prefilter: radii rounded to FP32 differ from the definition's
    // FP64 sum by far less than the band
    const float tf = (Rkf + v.Rf[j]) + tailf;
    if (df < tf - kBandA) return true;
    if (df > tf + kBandA) return false;
    const double d = __dsqrt_rn(dist2_grid_d(cx, cy, cz, v.cq[j], v.cq[(size_t)v.Ktot + j], v.cq[(size_t)2 * v.Ktot + j], I));
    // same operation order as the definition: ((Rk + Rj) + rs) + (skin + skin)
    double tt = __dadd_rn(__dadd_rn(__dadd_rn(Rk, v.R[j]), I.rs), __dadd_rn(I.skin, I.skin));
    tt = __dmul_rn(tt, 1.0 + 1e-12);
    return d < tt;
}

// Neighbouring cells, one warp per cell: the lanes share the grid cells of
// the cube around the cell's own grid cell that the reach
// R_k + R_max + r_s + 2 skin can touch, test every centroid there with the
// exact rule, collect the row in shared memory and sort it.  A membrane
// whose proteins have a cell set of their own searches that set's grid too,
// so that its rows hold the neighbouring cells of both sets.  Rows longer than
// kAdjRow are flagged (kStatusAdjOverflow) and truncated. Each entry gets
// the pair kernel's staging descriptor (particle range, exact centroid
// offset at 2^-26 sigma) in the same fixed-stride row.
__global__ void __launch_bounds__(256, 6) k_adj_warp(View v, const unsigned long long* __restrict__ rmax_bits, int* __restrict__ count,
                           float* __restrict__ rho_out, int* __restrict__ pad /* [Ktot][kAdjRow] */) {
    __shared__ int row[8][kAdjRow];
    __shared__ int rown[8];
    const int wb = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= v.Ktot) return;
    const int b = find_inst(v.inst_k0, v.B, k);
    const Inst& I = v.inst[b];
    const double Rk = v.R[k];
    const float Rkf = v.Rf[k];
    const long long cx = v.cq[k], cy = v.cq[(size_t)v.Ktot + k], cz = v.cq[(size_t)2 * v.Ktot + k];
    // the cell's scalars in FP32 (every lane of the warp computes them, and
    // an FP64 operation costs a full warp's turn on the FP64 pipe): they only
    // set the FP32 prefilter and the search reach, whose band kBandA is far
    // wider than their rounding
    const float tailf = I.rsf + 2.0f * I.skinf;
    if (lane == 0) rown[wb] = 0;
    __syncwarp();
    auto reach_of = [&](float Rmaxf) { return ((Rkf + Rmaxf) + tailf) + kBandA; };
    // the largest radius of the set from its largest square (FP32: it only
    // sets the reach)
    auto rmax_of = [&](int s) { return sqrtf((float)__longlong_as_double((long long)rmax_bits[s])); };
    const float reach_own = reach_of(rmax_of(b));
    float rho = reach_own - kBandA;
    // the centroids of one set through its own grid G: every centroid within
    // the reach R_k + R_max(G) + r_s + 2 skin is tested with the exact rule;
    // own: the set of cell k, whose nearest non-neighbour bounds the
    // E-step's certificate (the other set's cells join the row only)
    auto scan = [&](const Inst& G, float Rmaxf, bool own) {
        const float reach = reach_of(Rmaxf);
        float p[3];
        int g[3];
        g[0] = grid_coord(cx, G, 0, p[0]);
        g[1] = grid_coord(cy, G, 1, p[1]);
        g[2] = grid_coord(cz, G, 2, p[2]);
        // cube radius: the first shell beyond which nothing is within reach
        int R = 0;
        for (;; R++) {
            bool ex;
            const float lb = shell_bound(p, g, R, G, ex);
            if (ex || lb > reach) break;
        }
        int lo[3], ext[3];
        bool full[3];
        for (int a = 0; a < 3; a++) {
            int l, h;
            full[a] = false;
            if (G.periodic[a]) {
                if (2 * R + 1 >= G.gdim[a]) { l = 0; h = G.gdim[a] - 1; full[a] = true; }
                else { l = g[a] - R; h = g[a] + R; }
            } else {
                l = max(0, g[a] - R);
                h = min(G.gdim[a] - 1, g[a] + R);
            }
            lo[a] = l;
            ext[a] = h - l + 1;
        }
        const float reach2 = reach * reach;
        // one lane per (y, z) row of the cube: the row's grid cells are
        // contiguous along x, and so are their centroids in grid order (one
        // or two segments when a periodic x range wraps)
        auto axis_gap = [&](int a, int u) {
            if (full[a]) return 0.f;
            const float cl = (!G.periodic[a] && u == 0) ? -3.0e38f : u * G.gh[a];
            const float ch = (!G.periodic[a] && u == G.gdim[a] - 1) ? 3.0e38f : (u + 1) * G.gh[a];
            return fmaxf(fmaxf(cl - p[a], p[a] - ch), 0.f);
        };
        const int rows = ext[1] * ext[2];
        for (int t = lane; t < rows; t += 32) {
            const int y = lo[1] + t % ext[1], z = lo[2] + t / ext[1];
            const float gy = axis_gap(1, y), gz = axis_gap(2, z);
            if (fmaf(gy, gy, gz * gz) > reach2) continue;      // the whole row is beyond the reach
            const int w1 = G.periodic[1] ? wrap_idx(y, G.gdim[1]) : y;
            const int w2 = G.periodic[2] ? wrap_idx(z, G.gdim[2]) : z;
            const long long rowbase = G.g0 + ((long long)w2 * G.gdim[1] + w1) * G.gdim[0];
            int xa[2], xb[2], nseg = 1;
            xa[0] = lo[0];
            xb[0] = lo[0] + ext[0] - 1;
            if (G.periodic[0] && !full[0]) {
                const int a0 = wrap_idx(xa[0], G.gdim[0]), b0 = wrap_idx(xb[0], G.gdim[0]);
                if (a0 <= b0) { xa[0] = a0; xb[0] = b0; }
                else { xa[0] = a0; xb[0] = G.gdim[0] - 1; xa[1] = 0; xb[1] = b0; nseg = 2; }
            }
            for (int sg = 0; sg < nseg; sg++) {
                const int q1 = v.gstart[rowbase + xb[sg] + 1];
                for (int q = v.gstart[rowbase + xa[sg]]; q < q1; q++) {
                    const float4 c = v.gcf[q];
                    const int j = __float_as_int(c.w);
                    const float dx = axis_dist(p[0], c.x, G, 0), dy = axis_dist(p[1], c.y, G, 1),
                                dz = axis_dist(p[2], c.z, G, 2);
                    const float df = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    if (adj_test(v, I, k, j, Rk, Rkf, df, cx, cy, cz, tailf)) {
                        const int at = atomicAdd(&rown[wb], 1);
                        if (at < kAdjRow) row[wb][at] = j;
                    } else if (own) {
                        rho = fminf(rho, df);
                    }
                }
            }
        }
    };
    scan(I, rmax_of(b), true);
    if (I.partner >= 0) scan(v.inst[I.partner], rmax_of(I.partner), false);
    for (int off = 16; off; off >>= 1) rho = fminf(rho, __shfl_xor_sync(0xffffffffu, rho, off));
    __syncwarp();
    int n = rown[wb];
    if (n > kAdjRow) {
        if (lane == 0) flag_inst(v, I, kStatusAdjOverflow);
        n = kAdjRow;
    }
    // ascending row: every entry goes to its rank (entries are distinct)
    int val[2], rk[2] = {0, 0};
    for (int u = 0; u < 2; u++) val[u] = (lane + 32 * u < n) ? row[wb][lane + 32 * u] : 0;
    for (int s2 = 0; s2 < n; s2++) {
        const int o = row[wb][s2];
        rk[0] += o < val[0];
        rk[1] += o < val[1];
    }
    for (int u = 0; u < 2; u++) {
        if (lane + 32 * u >= n) continue;
        const int j = val[u];
        pad[(size_t)k * kAdjRow + rk[u]] = j;
        // exact offset between the mirrors' reference points (multiples of
        // 2^-26 sigma; on a periodic axis less the image)
        const long long dx = minimg_q(mirror_ref(v.cq[j]) - mirror_ref(cx), I.boxq[0], I.periodic[0]);
        const long long dy = minimg_q(mirror_ref(v.cq[(size_t)v.Ktot + j]) - mirror_ref(cy), I.boxq[1], I.periodic[1]);
        const long long dz = minimg_q(mirror_ref(v.cq[(size_t)2 * v.Ktot + j]) - mirror_ref(cz), I.boxq[2], I.periodic[2]);
        AdjDesc d;
        d.start = v.cell_start[j];
        d.cnt = v.cell_start[j + 1] - d.start;
        d.ox = (int)(unsigned)(unsigned long long)((dx + (1ll << (kMirrorShift - 1))) >> kMirrorShift);
        d.oy = (int)(unsigned)(unsigned long long)((dy + (1ll << (kMirrorShift - 1))) >> kMirrorShift);
        d.oz = (int)(unsigned)(unsigned long long)((dz + (1ll << (kMirrorShift - 1))) >> kMirrorShift);
        d.cell = j;
        v.adjd[(size_t)k * kAdjRow + rk[u]] = d;
    }
    if (lane == 0) {
        count[k] = n;
        rho_out[k] = rho;
    }
}

// CSR rows from the fixed-stride rows (for the getters).
__global__ void k_adj_csr(View v, const int* __restrict__ pad) {
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= v.Ktot) return;
    const int a0 = v.adj_ptr[k], n = v.adj_ptr[k + 1] - a0;
    for (int t = lane; t < n && a0 + t < v.adj_cap; t += 32) v.adj[a0 + t] = pad[(size_t)k * kAdjRow + t];
}

// ============================================================== host side
static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

void Ensemble::build_grid() {
    View v = view();
    CK(cudaMemsetAsync(d_gcount, 0, sizeof(int) * (Gtot + 1), stream));
    k_grid_count<<<nblk(Ktot, 256), 256, 0, stream>>>(v, d_gcount, d_gidx);
    launches++;
    CK(cudaGetLastError());
    scan_exclusive(d_gcount, d_gstart, Gtot + 1);
    CK(cudaMemsetAsync(d_gcount, 0, sizeof(int) * (Gtot + 1), stream));
    k_grid_fill<<<nblk(Ktot, 256), 256, 0, stream>>>(v, d_gidx, d_gcount, d_cf);
    launches++;
    CK(cudaGetLastError());
}

void Ensemble::mstep_iter(const int* cell_of, int iter, unsigned* dmax) {
    View v = view();
    k_mstep_accum<<<nblk(N, 256), 256, 0, stream>>>(v, cell_of, d_S, d_cnt);
    launches++;
    CK(cudaGetLastError());
    if (dmax) CK(cudaMemsetAsync(dmax, 0, sizeof(unsigned) * B, stream));
    k_mstep_finish<<<nblk(Ktot, 256), 256, 0, stream>>>(v, d_S, d_cnt, iter, dmax, dmax ? d_cmove : nullptr);
    launches++;
    CK(cudaGetLastError());
}

void Ensemble::mirrors() {
    k_mirrors<<<nblk(N, 256), 256, 0, stream>>>(view());
    launches++;
    CK(cudaGetLastError());
}

// Skin trigger: has any particle moved more than the skin since the last
// rebuild?  FP32 estimate with a margin that errs towards rebuilding (a
// rebuild never changes the forces, only where they are found).
__global__ void k_displacement(View v, const long long* __restrict__ xref, unsigned* __restrict__ flag) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    size_t N = v.N;
    float d2 = 0.f;
    for (int a = 0; a < 3; a++) {
        float d = ll_to_float(minimg_q(v.xq[a * N + p] - xref[a * N + p], I.boxq[a], I.periodic[a])) * (float)kGridInv;
        d2 = fmaf(d, d, d2);
    }
    float s = I.skinf * (1.0f - 1e-5f);
    if (d2 > s * s) atomicOr(flag, 1u);
}

bool Ensemble::displacement_exceeds_skin() {
    CK(cudaMemsetAsync(d_cnt + Ktot, 0, sizeof(int), stream));
    k_displacement<<<nblk(N, 256), 256, 0, stream>>>(view(), d_xref, (unsigned*)(d_cnt + Ktot));
    launches++;
    CK(cudaGetLastError());
    unsigned f = 0;
    CK(cudaMemcpyAsync(&f, d_cnt + Ktot, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    return f != 0;
}

void Ensemble::estep(int* cell_out, float* lbound) {
    k_estep_warp<<<nblk(N, 128), 128, 0, stream>>>(view(), cell_out, lbound, nullptr, nullptr);
    launches++;
    CK(cudaGetLastError());
}

void Ensemble::estep_bounded(int* cell) {
    CK(cudaMemsetAsync(d_fbcount, 0, sizeof(int), stream));
    CK(cudaMemsetAsync(d_gmove, 0, sizeof(unsigned) * Gtot, stream));
    k_grid_move<<<nblk(Ktot, 256), 256, 0, stream>>>(view(), d_gidx, d_cmove, d_gmove);
    k_estep_bound<<<nblk(N, 256), 256, 0, stream>>>(view(), cell, d_lbound, d_cf, d_dmax, d_gmove, d_cell_tmp,
                                                    d_fbcount);
    k_estep_warp<<<nblk(N, 128), 128, 0, stream>>>(view(), cell, d_lbound, d_cell_tmp, d_fbcount);
    launches += 2;
    CK(cudaGetLastError());
}

void Ensemble::morton_relabel() {
    View v = view();
    if (!bbox_ready_) {
        // bbox init: min = +inf, max = -inf
        k_fill_bbox<<<1, 64, 0, stream>>>(d_bbox, B);
        launches++;
        k_bbox<<<nblk(Ktot, 256), 256, 0, stream>>>(v, d_bbox);
        launches++;
    }
    bbox_ready_ = false;
    k_morton_keys<<<nblk(Ktot, 256), 256, 0, stream>>>(v, d_bbox, d_keys);
    launches++;
    int ntiles = nblk(Ktot, kTile);
    k_tile_sort<<<ntiles, kTile, 0, stream>>>(v, d_keys, (SortRec*)d_sortrec);
    launches++;
    CK(cudaMemcpyAsync(d_cq_tmp, d_cq, sizeof(long long) * 3 * Ktot, cudaMemcpyDeviceToDevice, stream));
    k_rank_scatter<<<nblk((long long)ntiles * kTile, 256), 256, 0, stream>>>(v, (const SortRec*)d_sortrec, ntiles, d_cq_tmp,
                                                                            d_new_of_old);
    launches++;
    CK(cudaGetLastError());
}

void Ensemble::finish_cells() {
    View v = view();
    morton_relabel();
    build_grid();
    if (prev_adj_valid_) {
        CK(cudaMemsetAsync(d_fbcount, 0, sizeof(int), stream));
        k_cand_rows<<<nblk((long long)Ktot * kAdjRow, 256), 256, 0, stream>>>(d_adjcount, Ktot, d_adjpad, d_new_of_old, d_cf,
                                                                          d_candrows);
        k_estep_rows<<<nblk(N, 128), 128, 0, stream>>>(v, d_cell, d_adjcount, d_candrows, d_rho, d_new_of_old, d_dmax,
                                                      d_cell_new, d_cell_tmp, d_fbcount);
        k_estep_list<<<152 * 4, 128, 0, stream>>>(v, d_cell_tmp, d_fbcount, d_cell_new);
        launches += 3;
        CK(cudaGetLastError());
    } else {
        estep(d_cell_new, nullptr);
    }
    // stable counting sort
    CK(cudaMemsetAsync(d_cnt, 0, sizeof(int) * (Ktot + 1), stream));
    k_hist<<<nblk(N, 256), 256, 0, stream>>>(N, d_cell_new, d_cnt);
    launches++;
    scan_exclusive(d_cnt, d_cell_start, Ktot + 1);
    CK(cudaMemsetAsync(d_cnt, 0, sizeof(int) * (Ktot + 1), stream));
    k_scatter<<<nblk(N, 256), 256, 0, stream>>>(N, d_cell_new, d_cell_start, d_cnt, d_perm);
    launches++;
    k_segsort_warp<<<nblk((long long)Ktot * 32, 256), 256, 0, stream>>>(Ktot, d_cell_start, d_perm);
    // larger cells (rare) from lists, so that no launch scans every cell or particle
    CK(cudaMemsetAsync(d_seglist_n, 0, sizeof(int) * 2, stream));
    k_seglist<<<nblk(Ktot, 256), 256, 0, stream>>>(Ktot, d_cell_start, d_seglist, d_seglist + Ktot, d_seglist_n);
    k_segsort_list<<<152, 256, 0, stream>>>(d_cell_start, d_seglist, d_seglist_n, d_perm);
    k_segrank_list<<<152, 256, 0, stream>>>(d_cell_start, d_seglist + Ktot, d_seglist_n, d_perm, d_cell_tmp);
    launches += 4;
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(d_cnt, 0, sizeof(int) * (Ktot + 1), stream));
    // gather into the second buffer set, then swap
    swap_state();
    View nv = view();
    View ov = view_alt();
    CK(cudaMemsetAsync(d_rmax, 0, sizeof(unsigned long long) * B, stream));
    k_gather_particles<<<nblk(N, 256), 256, 0, stream>>>(nv, ov, d_perm, d_cell_new, d_xref);
    k_cell_props<<<nblk((long long)Ktot * 32, 256), 256, 0, stream>>>(nv, d_rmax);
    k_cell_radius<<<nblk(Ktot, 256), 256, 0, stream>>>(nv);
    launches += 3;
    CK(cudaGetLastError());
    // neighbouring cells
    k_adj_warp<<<nblk((long long)Ktot * 32, 256), 256, 0, stream>>>(nv, d_rmax, d_adjcount, d_rho, d_adjpad);
    launches++;
    CK(cudaGetLastError());
    prev_adj_valid_ = true;
    csr_valid_ = false;
    cells_valid = true;
    forces_valid = false;
    list_valid = false;
    n_rebuilds++;
}

void Ensemble::adjacency_csr() {
    if (csr_valid_ || !cells_valid) return;
    CK(cudaMemsetAsync(d_adjcount + Ktot, 0, sizeof(int), stream));
    scan_exclusive(d_adjcount, d_adj_ptr, Ktot + 1);
    k_adj_csr<<<nblk((long long)Ktot * 32, 256), 256, 0, stream>>>(view(), d_adjpad);
    launches++;
    CK(cudaGetLastError());
    csr_valid_ = true;
}

void Ensemble::rebuild(bool sums_ready) {
    // M-step on the cell-sorted particles, fused with the centroid bounding box
    k_fill_bbox<<<1, 64, 0, stream>>>(d_bbox, B);
    launches++;
    CK(cudaMemsetAsync(d_dmax, 0, sizeof(unsigned) * B, stream));
    if (sums_ready) k_mstep_apply<<<nblk(Ktot, 256), 256, 0, stream>>>(view(), d_msum, d_mcnt, d_bbox, d_dmax);
    else k_mstep_sorted<<<nblk(Ktot, 8), 256, 0, stream>>>(view(), d_bbox, d_dmax);
    launches++;
    CK(cudaGetLastError());
    bbox_ready_ = true;
    finish_cells();
}

}  // namespace orbc
