// Internal definitions shared by the CUDA translation units of liborbc.
//
// Number formats (chosen for GB300, where FP64 arithmetic and every
// conversion to or from a 64-bit type run at ~1-2 results/clock/SM against
// 128 FP32 FMAs):
//   - state (x, v, director n, angular velocity w): int64 on a 2^-40 grid,
//     so every value is an exact double and updates are exact integer adds;
//   - forces and torques: int64 at 2^-32 (eps/sigma, eps), accumulated from
//     FP32 pair terms through two exact int32 partial sums per component;
//   - pair-kernel mirror: int32 position relative to the particle's own
//     centroid at 2^-26 sigma, plus a float4 director;
//   - FP64 only where a discrete decision must equal the FP64 definition
//     (nearest centroid, cell radius, neighbouring cells, cutoff inclusion)
//     and only for the rare candidates inside a rounding band.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace orbc {

constexpr int kGridShift = 40;                       // state: 2^-40
constexpr double kGrid = 1099511627776.0;            // 2^40
constexpr double kGridInv = 9.094947017729282e-13;   // 2^-40
constexpr int kMirrorShift = 14;                     // mirror = state >> 14 -> 2^-26 sigma
constexpr float kMirrorUnit = 1.4901161193847656e-08f;  // 2^-26
constexpr double kForceUnit = 2.3283064365386963e-10;   // force/torque/energy fixed point 2^-32
constexpr float kMagic = 12582912.0f;                // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
constexpr int kMaxBondsPerParticle = 8;
constexpr int kLipid = 0;
constexpr int kBand3 = 3;
constexpr int kGlycophorin = 4;
constexpr int kMaxType = 4;
// flag in a mirror's type word (above the type byte): the particle has bonds
constexpr int kMirrorBonded = 0x100;
// Half-width (sigma) of the band around a cutoff inside which the FP32
// distance test defers to the exact FP64 decision.
constexpr float kCutBand = 1e-6f;

// Bilayer particles (lipids and the membrane proteins band-3 and
// glycophorin) carry a director and meet each other through the lipid
// potential with the constants of their species pair; junctions and
// spectrin beads are the cytoskeleton.
__host__ __device__ inline bool bilayer(int t) { return t == kLipid || t >= kBand3; }
// species index of a bilayer type: lipid 0, band-3 1, glycophorin 2
__host__ __device__ inline int species(int t) { return t < kBand3 ? 0 : t - 2; }
// Largest magnitude of one pair, bond or constraint term (force or torque
// component, eps/sigma or eps; a volume term in sigma^3): 2^24, so that a
// particle's 2^-32 fixed-point sum of a few hundred terms stays inside int64.
constexpr float kMaxTerm = 16777216.0f;

// ---------------------------------------------------------------- per-instance descriptor
struct Inst {
    // ranges in the packed arrays
    int p0, n;          // particles
    int k0, K;          // cells
    long long g0;       // grid cells
    int gdim[3];
    int nlip;
    long long gorg[3];  // grid origin on the 2^-40 grid
    float gh[3], ginv[3];  // grid edge per axis and its inverse (sigma)
    // box
    double box[3];
    long long boxq[3];  // box on the 2^-40 grid
    float boxf[3];
    int periodic[3];
    // potential
    float eps, rmin, rc, mu, s0, eps_wca, sig_wca, sig_pp;
    int zeta;
    double eps_d, rmin_d, rc_d, mu_d, s0_d, eps_wca_d, sig_wca_d, sig_pp_d;
    double rc2_ll, rc2_wca, rc2_pp;   // FP64 squared type-pair cutoffs (inclusion decision)
    double rs, skin;            // search cutoff and skin
    float rc2f_ll, rc2f_wca, rc2f_pp, rsf, skinf;
    float aw, eps2z_aw;         // (pi/2)/(rc - rmin) and eps 2 zeta aw
    // integrator (host-computed constants)
    float h_m, h_i;             // dt/2/m, dt/2/I
    float hdt;                  // dt/2
    float ct_m1, st, cr_m1, sr; // exp(-g dt) - 1 and noise amplitudes
    double h_m_d, h_i_d, hdt_d, ct_m1_d, st_d, cr_m1_d, sr_d;
    // the same, scaled by powers of two for FP64 increments in grid units
    // (state as integer-valued doubles): h_m 2^8 and h_i 2^8 (force and
    // torque at 2^-32 to a grid increment at 2^-40), st 2^40 and sr 2^40,
    // and dt/4 2^-40 (half the Cayley rotation vector from w in grid units)
    double hm8_d, hi8_d, st40_d, sr40_d, ca_d;
    // h_m 2^8 and dt/2 as exact integer fixed point, m 2^-s (m < 2^54): the
    // translational kick and the drifts multiply the int64 state by them
    // exactly and round once
    unsigned long long hm8_m, hdt_m;
    int hm8_s, hdt_s;
    // the Ornstein-Uhlenbeck update of v, round(ct_m1 v + stn xi), as the
    // exact sum of two integer products (ctm1_m 2^-ctm1_s, stn_m 2^-stn_s,
    // signed) when the two scales are close enough for a 128-bit sum
    // (ou_int), else in FP64
    long long ctm1_m, stn_m;
    int ctm1_s, stn_s, ou_int;
    // st and sr 2^40 times the noise's scale sqrt(12) 2^-33 (multiplying the
    // noise's exact integer part)
    double stn_d, srn_d;
    double mass, inertia;
    unsigned long long seed;
    unsigned instance;
    int rebuild_every;
    int n_lloyd;        // k-means rounds at initialisation
    // harmonic volume constraint (off when vol_on == 0): k_V, V0, the area
    // per lipid a, a/3 and the reference point on the 2^-40 grid
    int vol_on;
    double kv, v0, avol, a3;
    long long xcq[3];
    // separate cell sets of one membrane: the batch index of the other set
    // (-1: none; its cells join this set's neighbour rows), the offset of
    // this set's ids in the membrane (Philox counters, pair dumps), and
    // whether every particle is a centroid member (else only the lipids)
    int partner, id_base, all_members;
    // bilayer species pairs, index 3 s_i + s_j (lipid, band-3, glycophorin):
    // the lipid potential's well depth and cutoff of each pair (the
    // lipid-lipid entry is eps and rc), the FP32 constants (eps, aw,
    // eps 2 zeta aw), the squared FP64 cutoff and the FP32 band of the
    // inclusion decision; mm_rcp the FP32 cutoff of each pair and mm_rcf[s]
    // the largest one of species s.
    // has_mp: the instance holds band-3 or glycophorin particles;
    // bonded_bilayer: some bilayer particle has a bond (an anchor), so a
    // bilayer-cytoskeleton pair may be excluded from the WCA term.
    int has_mp, bonded_bilayer;
    float mm_eps[9], mm_aw[9], mm_e2za[9], mm_lo[9], mm_hi[9], mm_rcf[3], mm_rcp[9];
    double mm_eps_d[9], mm_rc_d[9], mm_rc2[9];
};

// ---------------------------------------------------------------- packed device arrays
// What the pair kernel needs to stage neighbouring cell l of cell k: its
// particle range and the exact offset c_l - c_k (minimum image) at the mirror
// resolution 2^-26 sigma, as wrap-around int32.
// Longest row of neighbouring cells; rows are stored at this fixed stride.
constexpr int kAdjRow = 64;

struct AdjDesc {
    int start, cnt;
    int ox, oy, oz;
    int cell;
};

struct View {
    int B;                      // instances
    int N, Ktot;
    long long Gtot;
    const Inst* inst;           // [B]
    const int* inst_p0;         // [B+1] particle offsets
    const int* inst_k0;         // [B+1] cell offsets
    // state (storage order, sorted by cell)
    long long *xq, *vq, *nq, *wq;   // [3][N] each (axis-major)
    unsigned char* type;
    unsigned* id;
    int* cell;                      // global cell of each slot
    int* slot_of_id;                // [N] indexed by p0 + id
    // forces (fixed point 2^-32)
    long long *F, *T;               // [3][N]
    long long* Fbig;                // [6][N] wide per-pair contributions (normally zero)
    // mirrors for the pair kernel
    int4* mq;                       // x - c at 2^-26 sigma, w = type | kMirrorBonded (has bonds)
    float4* mo;                     // director, w = slot (int bits)
    int4* mqr;                      // the same two, each tile of 128 particles of a cell
    float4* mor;                    // in the order of the pair kernel's group ranks
    float4* cnorm;                  // [Ktot] unit normal of each cell (mean lipid director)
    unsigned char* grank;           // [N] rank of each particle in its 128-particle tile along
                                    //     the tile's longer tangent extent (pair-kernel groups)
    // cells
    long long* cq;                  // [3][Ktot] centroids on the 2^-40 grid
    int* cell_start;                // [Ktot+1]
    double* R;                      // [Ktot] cell radius
    float* Rf;                      // [Ktot] the same rounded to FP32 (the neighbour rule's prefilter)
    int* adj_ptr;                   // [Ktot+1]
    int* adj;                       // [adj_cap]
    struct AdjDesc* adjd;           // [Ktot][kAdjRow] staging descriptors, row k ascending by cell
    const int* adjn;                // [Ktot] row lengths
    long long adj_cap;
    // centroid search grid
    int* gstart;                    // [Gtot+1]
    int* gcent;                     // [Ktot] centroid ids in grid order
    float4* gcf;                    // [Ktot] centroid xyz rel. to grid origin, w = id bits
    // bonds: CSR by (p0 + id)
    int* bptr;                      // [N+1]
    int* bpartner;                  // partner id (instance-local), ascending per particle
    // bonds as a flat list (each once): ends as p0 + id, instance, constants
    int nbond;
    const int2* bij;
    const int* binst;
    const float2* bkf;              // (r0, kb)
    const double2* bkd;
    // status word written by kernels (bit flags, see kStatus*), and one per
    // instance for the flags that belong to one instance (nullable)
    unsigned* status;
    unsigned* istatus;              // [B]
    // bounded waits: polls before a staging barrier gives up, and bytes a
    // barrier expects beyond those issued (0; a test sets it to make the
    // wait run out while every copy still lands)
    unsigned wait_polls;
    unsigned extra_tx;
    // [B][2] sum of (x - c).n over the lipids (the enclosed volume is a/3
    // times it): sums of the 2^-24 sigma floors and of the 2^-48 remainders
    // of its terms (volume constraint)
    long long* vol;
};

enum : unsigned {
    kStatusNaN = 1u,
    kStatusCellOverflow = 2u,
    kStatusAdjOverflow = 4u,
    kStatusMirrorRange = 8u,
    kStatusPairForceRange = 16u,
    kStatusTimeout = 32u,
    kStatusGridRange = 64u,
    kStatusListOverflow = 128u,   // more listed pairs than the neighbour lists and their overflow hold
};
// Flags raised by the data of one instance (its state, forces or cells);
// the others (a wait that timed out, the shared overflow list) concern the
// whole launch.
constexpr unsigned kStatusPerInstance =
    kStatusNaN | kStatusAdjOverflow | kStatusMirrorRange | kStatusPairForceRange | kStatusGridRange;

// ---------------------------------------------------------------- small helpers
__host__ __device__ inline long long floor_div_ll(long long a, long long b) {   // b > 0
    long long q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}
__host__ __device__ inline long long floor_mod_ll(long long a, long long b) { return a - b * floor_div_ll(a, b); }


// Minimum image on the 2^-40 grid: d - L * round(d / L), ties rounding up.
__device__ inline long long minimg_q(long long d, long long L, int per) {
    if (!per) return d;
    // FP32 estimate of round(d/L), then exact correction with integer compares
    long long k = (long long)rintf((float)d / (float)L);
    long long r = d - k * L;
    while (2 * r >= L) { r -= L; }
    while (2 * r < -L) { r += L; }
    return r;
}

// Exact double of a grid value.
__device__ inline double grid_to_double(long long q) { return __ll2double_rn(q) * kGridInv; }

// FP64 minimum image as the definition states it: d - L * rint(d / L).
__device__ inline double minimg_d(double d, double L, int per) {
    if (!per) return d;
    double q = __ddiv_rn(d, L);
    double r = rint(q);
    double p = __dmul_rn(L, r);
    return __dsub_rn(d, p);
}

// Squared distance ((dx*dx + dy*dy) + dz*dz) between two grid points, FP64
// without contraction, minimum image with the FP64 box.
__device__ inline double dist2_grid_d(long long ax, long long ay, long long az, long long bx, long long by,
                                      long long bz, const Inst& I) {
    // both coordinates are below 2^52 grid units, so each converts exactly
    // and their FP64 difference is exact: the int64 difference converted
    // once is the same double (three conversions instead of six and no
    // subtraction on the FP64 pipe)
    double dx = minimg_d(grid_to_double(ax - bx), I.box[0], I.periodic[0]);
    double dy = minimg_d(grid_to_double(ay - by), I.box[1], I.periodic[1]);
    double dz = minimg_d(grid_to_double(az - bz), I.box[2], I.periodic[2]);
    double s = __dmul_rn(dx, dx);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    return s;
}

// int64 -> float without a 64-bit conversion: hi * 2^32 + lo.
__device__ inline float ll_to_float(long long v) {
    int hi = (int)(v >> 32);
    unsigned lo = (unsigned)(v & 0xffffffffull);
    return fmaf((float)hi, 4294967296.0f, (float)lo);
}

// ---------------------------------------------------------------- exact fixed-point accumulation
// A per-pair FP32 value f contributes round(f * 2^32) to an int64 sum.  With
// h = round(f * 2^12) and l = round((f * 2^12 - h) * 2^20) (both exact FP32
// operations via the 1.5*2^23 magic constant, valid for |f| < 1024),
// round(f 2^32) = h 2^20 + l.  The raw float bits of the magic sums are added
// as int32 and the magic offset removed at the end, so each component costs
// four FP32 operations and two integer adds; integer sums make the result
// independent of summation order.
struct SplitAcc {
    int h, l;
    __device__ inline void zero() { h = 0; l = 0; }
    __device__ inline void add(float f) {
        float t = fmaf(f, 4096.0f, kMagic);
        float hf = t - kMagic;
        float r = fmaf(f, 4096.0f, -hf);
        float u = fmaf(r, 1048576.0f, kMagic);
        h += __float_as_int(t);
        l += __float_as_int(u);
    }
    __device__ inline long long finish(int count) const {
        int hh = h - count * kMagicBits;
        int ll = l - count * kMagicBits;
        return ((long long)hh << 20) + (long long)ll;
    }
};

// Round a float to the 2^-40 grid as int64 (exact FP32 splitting, |v| < 2^11).
__device__ inline long long float_to_grid(float v) {
    // v * 2^40 = h * 2^20 + l  with h = round(v * 2^20), |v * 2^20| < 2^22 required -> |v| < 4
    // for larger increments fall back to a split at 2^-8
    if (fabsf(v) < 3.9f) {
        float t = fmaf(v, 1048576.0f, kMagic);
        float hf = t - kMagic;
        float r = fmaf(v, 1048576.0f, -hf);
        float u = fmaf(r, 1048576.0f, kMagic);
        int h = __float_as_int(t) - kMagicBits;
        int l = __float_as_int(u) - kMagicBits;
        return ((long long)h << 20) + (long long)l;
    }
    // |v| < 2^11: h = round(v * 2^8), r scaled by 2^16 twice
    float t = fmaf(v, 256.0f, kMagic);
    float hf = t - kMagic;
    float r = fmaf(v, 256.0f, -hf);               // |r| <= 0.5, exact
    float t2 = fmaf(r, 65536.0f, kMagic);
    float hf2 = t2 - kMagic;
    float r2 = fmaf(r, 65536.0f, -hf2);
    float u = fmaf(r2, 65536.0f, kMagic);
    long long h = __float_as_int(t) - kMagicBits;
    long long m = __float_as_int(t2) - kMagicBits;
    long long l = __float_as_int(u) - kMagicBits;
    return (h << 32) + (m << 16) + l;
}

// Round a double to the 2^-40 grid (FP64 path only).
__device__ inline long long double_to_grid(double v) { return __double2ll_rn(v * kGrid); }

// ---------------------------------------------------------------- Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror & Shaw (SC'11).
__device__ inline uint4 philox4x32_10(uint4 c, uint2 k) {
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        uint4 n;
        n.x = hi1 ^ c.y ^ k.x;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k.y;
        n.w = lo0;
        c = n;
        k.x += W0;
        k.y += W1;
    }
    return c;
}

// Unit-variance uniform noise from a 32-bit word: sqrt(12) ((w + 1/2) 2^-32 - 1/2).
__device__ inline float noise_f(unsigned w) {
    float s = (float)(int)(w ^ 0x80000000u);            // w - 2^31
    return 3.46410161513775f * fmaf(s, 2.3283064365386963e-10f, 1.16415321826934814e-10f);
}
__device__ inline double noise_d(unsigned w) {
    double u = (__uint2double_rn(w) + 0.5) * 2.3283064365386963e-10;
    return 3.4641016151377544 * (u - 0.5);
}

__device__ inline int find_inst(const int* off, int B, int x) {   // off[B+1], returns b with off[b] <= x < off[b+1]
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Orthonormal tangent frame (rows e1, e2, n) of a unit normal n: e1 is n
// crossed with the coordinate axis least aligned with n.
struct Frame {
    float r[9];
    __device__ inline void apply(float x, float y, float z, float& a, float& b, float& c) const {
        a = fmaf(r[0], x, fmaf(r[1], y, r[2] * z));
        b = fmaf(r[3], x, fmaf(r[4], y, r[5] * z));
        c = fmaf(r[6], x, fmaf(r[7], y, r[8] * z));
    }
};

__device__ inline Frame tangent_frame(float nx, float ny, float nz) {
    const float ax = fabsf(nx), ay = fabsf(ny), az = fabsf(nz);
    float ux, uy, uz;
    if (ax <= ay && ax <= az) { ux = 0.f; uy = nz; uz = -ny; }
    else if (ay <= az) { ux = -nz; uy = 0.f; uz = nx; }
    else { ux = ny; uy = -nx; uz = 0.f; }
    const float un = sqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
    ux /= un; uy /= un; uz /= un;
    Frame f;
    f.r[0] = ux; f.r[1] = uy; f.r[2] = uz;
    f.r[3] = ny * uz - nz * uy; f.r[4] = nz * ux - nx * uz; f.r[5] = nx * uy - ny * ux;
    f.r[6] = nx; f.r[7] = ny; f.r[8] = nz;
    return f;
}

// Volume constraint: the sum D of (x - c).n over the bilayer is kept as two
// integer sums, of the terms' floors at 2^-24 sigma and of their remainders
// at 2^-48; the enclosed volume is (a/3) D.
constexpr double kVolUnit = 16777216.0;                 // 2^24: fixed point of (x - c).n, 2^-24 sigma
constexpr double kVolUnitInv = 5.9604644775390625e-08;  // 2^-24
constexpr double kVolFineInv = 3.552713678800501e-15;   // 2^-48: the remainders' unit
__host__ __device__ inline double volume_of(long long hi, long long lo) {
    return (double)hi * kVolUnitInv + (double)lo * kVolFineInv;
}

// A particle that moves its cell's centroid (the M-step): the bilayer's
// (lipids and membrane proteins), or every particle of a protein cell set.
__host__ __device__ inline bool centroid_member(const Inst& I, unsigned char type) {
    return I.all_members || bilayer(type);
}

// Raises status bits for the launch and for the instance I (a reference
// into v.inst).
__device__ inline void flag_inst(const View& v, const Inst& I, unsigned bits) {
    atomicOr(v.status, bits);
    if (v.istatus) atomicOr(v.istatus + (&I - v.inst), bits);
}

}  // namespace orbc
