// Device side of the time stepping: the B-A-O-A update of one particle
// from its force and torque, shared by the integrator's own launches and by
// the pair evaluation that runs the next step's update in its epilogue.
// ("Software Overview": force and torque, then update of position and
// orientation.  Reading: BAOAB Langevin, Leimkuhler & Matthews 2013,
// translational for every particle and rotational for lipids, with Cayley
// rotations of the director and uniform unit-variance noise from
// Philox4x32-10 keyed by (seed, instance; id, step, substream).)
#pragma once

#include "ensemble.cuh"

namespace orbc {

template <typename T> struct Num;
template <> struct Num<float> {
    static __device__ float st(long long q) { return ll_to_float(q) * (float)kGridInv; }
    static __device__ float frc(long long q) { return ll_to_float(q) * (float)kForceUnit; }
    static __device__ long long grid(float x) { return float_to_grid(x); }
    static __device__ float noise(unsigned w) { return noise_f(w); }
};
template <> struct Num<double> {
    static __device__ double st(long long q) { return grid_to_double(q); }
    static __device__ double frc(long long q) { return __ll2double_rn(q) * kForceUnit; }
    static __device__ long long grid(double x) { return double_to_grid(x); }
    // sqrt(12) ((w + 1/2) 2^-32 - 1/2) = sqrt(12) 2^-33 (2 (w - 2^31) + 1): the
    // integer is exact and the product is rounded once, as in the definition
    static __device__ double noise(unsigned w) {
        const long long s = 2 * (long long)(int)(w ^ 0x80000000u) + 1;   // |s| < 2^32, exact
        return (3.4641016151377544 * 1.16415321826934814453125e-10) * (double)s;
    }
};

template <typename T> struct Consts;
template <> struct Consts<float> {
    float hm, hi, hdt, ctm1, st, crm1, sr;
    __device__ Consts(const Inst& I) : hm(I.h_m), hi(I.h_i), hdt(I.hdt), ctm1(I.ct_m1), st(I.st), crm1(I.cr_m1), sr(I.sr) {}
};
template <> struct Consts<double> {
    double hm, hi, hdt, ctm1, st, crm1, sr;
    __device__ Consts(const Inst& I)
        : hm(I.h_m_d), hi(I.h_i_d), hdt(I.hdt_d), ctm1(I.ct_m1_d), st(I.st_d), crm1(I.cr_m1_d), sr(I.sr_d) {}
};

// Cayley rotation of the director by the rotation vector h w:
// a = h w / 2, n' = n + 2/(1 + |a|^2) (a x n + a x (a x n)); the increment is
// added to the grid value.
template <typename T>
__device__ inline void cayley(long long nq[3], const long long wq[3], T h) {
    using V = Num<T>;
    T n0 = V::st(nq[0]), n1 = V::st(nq[1]), n2 = V::st(nq[2]);
    T a0 = (T)0.5 * h * V::st(wq[0]), a1 = (T)0.5 * h * V::st(wq[1]), a2 = (T)0.5 * h * V::st(wq[2]);
    T aa = a0 * a0 + a1 * a1 + a2 * a2;
    T k = (T)2 / ((T)1 + aa);
    T b0 = a1 * n2 - a2 * n1, b1 = a2 * n0 - a0 * n2, b2 = a0 * n1 - a1 * n0;      // a x n
    T c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;      // a x (a x n)
    nq[0] += V::grid(k * (b0 + c0));
    nq[1] += V::grid(k * (b1 + c1));
    nq[2] += V::grid(k * (b2 + c2));
}

// |n_q|^2 - 2^80 for a director on the 2^-40 grid, exact in 128-bit integer
// arithmetic (the excess of its squared length over unit length in units of
// 2^-80); 0 when it is far from unit length (|excess| >= 2^63, not reached
// in practice: the correction is then skipped).
__device__ inline long long norm2_excess(const long long nq[3]) {
    unsigned long long H = 0, L = 0;
    for (int a = 0; a < 3; a++) {
        unsigned long long u = (unsigned long long)(nq[a] < 0 ? -nq[a] : nq[a]);
        unsigned long long lo = u * u, hi = __umul64hi(u, u);
        unsigned long long L2 = L + lo;
        H += hi + (L2 < L ? 1ull : 0ull);
        L = L2;
    }
    const long long hd = (long long)H - (1ll << 16);     // multiples of 2^64
    const long long D = (long long)L;
    // exact when the 128-bit excess fits in int64
    if (hd == 0 && D >= 0) return D;
    if (hd == -1 && D < 0) return D;
    return 0;
}

// Unit-norm correction n <- n (1 - delta/2), delta = |n|^2 - 1, first order
// (|delta| stays at the rounding level, ~1e-9).
__device__ inline void renormalise(long long nq[3], float) {
    const long long D = norm2_excess(nq);
    if (D == 0) return;
    float delta = ll_to_float(D) * 8.271806125530277e-25f;   // 2^-80
    for (int a = 0; a < 3; a++) nq[a] -= float_to_grid(Num<float>::st(nq[a]) * 0.5f * delta);
}
__device__ inline void renormalise(long long nq[3], double) {
    double n0 = grid_to_double(nq[0]), n1 = grid_to_double(nq[1]), n2 = grid_to_double(nq[2]);
    double delta = (n0 * n0 + n1 * n1 + n2 * n2) - 1.0;
    nq[0] -= double_to_grid(n0 * 0.5 * delta);
    nq[1] -= double_to_grid(n1 * 0.5 * delta);
    nq[2] -= double_to_grid(n2 * 0.5 * delta);
}

// Half kick of v and w with the force F and torque Tq (2^-32 fixed point;
// the torque projected perpendicular to n); reps = 2 applies the same
// rounded increments twice (the final B of the previous step and this step's
// B share their forces).
template <typename T>
__device__ inline void kick(long long vq[3], long long wq[3], const long long nq[3], bool lipid, const Consts<T>& C,
                            int reps, const long long F[3], const long long Tq[3]) {
    using V = Num<T>;
    for (int a = 0; a < 3; a++) vq[a] += reps * V::grid(C.hm * V::frc(F[a]));
    if (lipid) {
        T t0 = V::frc(Tq[0]), t1 = V::frc(Tq[1]), t2 = V::frc(Tq[2]);
        T n0 = V::st(nq[0]), n1 = V::st(nq[1]), n2 = V::st(nq[2]);
        T tn = t0 * n0 + t1 * n1 + t2 * n2;
        wq[0] += reps * V::grid(C.hi * (t0 - tn * n0));
        wq[1] += reps * V::grid(C.hi * (t1 - tn * n1));
        wq[2] += reps * V::grid(C.hi * (t2 - tn * n2));
    }
}

// The M-step's sums for the rebuild that follows (the "Spatial Searching
// Algorithm" update of each centroid from its lipids at the new positions):
// member i of cell k (a lipid, or any particle of a protein cell set) adds
// minimg(x_i - c_k) on the 2^-40 grid, exactly.  The
// lanes of a warp that share a cell add up a 24-bit low part and the high
// part separately in 32 bits, exact while |x_i - c_k| < 1024 sigma (the
// mirrors already flag anything beyond 32 sigma); one lane per cell adds the
// int64 totals.
__device__ inline void mstep_sums(const View& v, const Inst& I, int p, bool member, const long long* xq,
                                  long long* __restrict__ msum, int* __restrict__ mcnt, unsigned mask) {
    const int k = v.cell[p];
    const size_t K = v.Ktot;
    long long d[3] = {0, 0, 0};
    if (member)
        for (int a = 0; a < 3; a++) d[a] = minimg_q(xq[a] - v.cq[a * K + k], I.boxq[a], I.periodic[a]);
    const unsigned grp = __match_any_sync(mask, k);
    const unsigned n = __reduce_add_sync(grp, member ? 1u : 0u);
    long long tot[3];
    for (int a = 0; a < 3; a++) {
        const unsigned lo = __reduce_add_sync(grp, (unsigned)(d[a] & 0xffffff));
        const int hi = (int)__reduce_add_sync(grp, (unsigned)(int)(d[a] >> 24));
        tot[a] = (long long)hi * 16777216ll + (long long)lo;
    }
    if ((int)(threadIdx.x & 31) == __ffs(grp) - 1 && n > 0) {
        for (int a = 0; a < 3; a++) atomicAdd((unsigned long long*)&msum[a * K + k], (unsigned long long)tot[a]);
        atomicAdd(&mcnt[k], (int)n);
    }
}

// One particle's B A O A (after the final B of the previous step when
// FUSED) with its force F and torque Tq, from the state of v into the state
// arrays of o (o = v: in place; copy_static: o also receives type and id);
// msum: the M-step's sums for the rebuild that follows, taken over the
// lanes of mask.
template <typename T, bool FUSED>
__device__ inline void baoa_body(const View& v, const View& o, int p, const long long F[3], const long long Tq[3],
                                 const long long* __restrict__ steps, long long* __restrict__ msum,
                                 int* __restrict__ mcnt, unsigned mask, bool copy_static) {
    using V = Num<T>;
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    const Consts<T> C(I);
    const size_t N = v.N;
    const unsigned char type = v.type[p];
    const bool lipid = bilayer(type);
    long long xq[3], vq[3], nq[3] = {0, 0, 0}, wq[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) { xq[a] = v.xq[a * N + p]; vq[a] = v.vq[a * N + p]; }
    if (lipid) for (int a = 0; a < 3; a++) { nq[a] = v.nq[a * N + p]; wq[a] = v.wq[a * N + p]; }
    // (final B of the previous step), B
    kick<T>(vq, wq, nq, lipid, C, FUSED ? 2 : 1, F, Tq);
    // A
    T vd[3];
    for (int a = 0; a < 3; a++) {
        vd[a] = V::st(vq[a]);
        xq[a] += V::grid(C.hdt * vd[a]);
    }
    if (lipid) cayley<T>(nq, wq, C.hdt);
    // O
    const unsigned id = (unsigned)I.id_base + v.id[p];   // the id in the membrane
    const unsigned long long step = (unsigned long long)steps[b] + (FUSED ? 1ull : 0ull);
    const uint2 key = make_uint2((unsigned)I.seed, (unsigned)(I.seed >> 32) ^ I.instance);
    uint4 w0 = philox4x32_10(make_uint4(id, (unsigned)step, (unsigned)(step >> 32), 0u), key);
    T xi[3] = { V::noise(w0.x), V::noise(w0.y), V::noise(w0.z) };
    for (int a = 0; a < 3; a++) vq[a] += V::grid(C.ctm1 * vd[a] + C.st * xi[a]);
    if (lipid) {
        uint4 w1 = philox4x32_10(make_uint4(id, (unsigned)step, (unsigned)(step >> 32), 1u), key);
        T r0 = V::noise(w1.x), r1 = V::noise(w1.y), r2 = V::noise(w1.z);
        T n0 = V::st(nq[0]), n1 = V::st(nq[1]), n2 = V::st(nq[2]);
        T rn = r0 * n0 + r1 * n1 + r2 * n2;
        wq[0] += V::grid(C.crm1 * V::st(wq[0]) + C.sr * (r0 - rn * n0));
        wq[1] += V::grid(C.crm1 * V::st(wq[1]) + C.sr * (r1 - rn * n1));
        wq[2] += V::grid(C.crm1 * V::st(wq[2]) + C.sr * (r2 - rn * n2));
    }
    // A
    for (int a = 0; a < 3; a++) xq[a] += V::grid(C.hdt * V::st(vq[a]));
    if (lipid) {
        cayley<T>(nq, wq, C.hdt);
        renormalise(nq, (T)0);
    }
    for (int a = 0; a < 3; a++) { o.xq[a * N + p] = xq[a]; o.vq[a * N + p] = vq[a]; }
    // in place a protein's (zero) director and angular velocity need no
    // store; into the other buffer, whose slot held another particle, they do
    if (lipid || copy_static) for (int a = 0; a < 3; a++) { o.nq[a * N + p] = nq[a]; o.wq[a * N + p] = wq[a]; }
    if (copy_static) { o.type[p] = type; o.id[p] = v.id[p]; }
    if (msum) mstep_sums(v, I, p, centroid_member(I, type), xq, msum, mcnt, mask);
}

// ---------------------------------------------------------------- FP64 increments in grid units
// GB300 runs FP64 arithmetic and int64 <-> FP64 conversions at a few
// operations per clock per SM, so the FP64 B-A-O-A holds every state value
// as an integer-valued double in grid units (exact below 2^53) and folds the
// 2^40 and 2^-32 scale factors into host-computed constants: the same
// roundings as the computation in sigma units (power-of-two scaling commutes
// with rounding), about half the FP64 operations.  Values that do not change
// between phases are converted once.
__device__ inline double gd(long long q) { return __ll2double_rn(q); }
__device__ inline long long rg(double x) { return __double2ll_rn(x); }

// round(q m 2^-s) to the nearest integer, ties to even, from the exact
// 128-bit product (1 <= s <= 127, |q| m < 2^(64 + s)): the same rounding as
// __double2ll_rn of the exact product, so a kick or drift computed this way
// rounds once where the FP64 product would round to 53 bits first; integer
// pipes only.
__device__ inline long long mul_round(long long q, unsigned long long m, int s) {
    const unsigned long long a = (unsigned long long)(q < 0 ? -q : q);
    const unsigned long long lo = a * m, hi = __umul64hi(a, m);
    unsigned long long r;
    bool up;
    if (s < 64) {
        r = (hi << (64 - s)) | (lo >> s);
        const unsigned long long rem = lo & ((1ull << s) - 1ull), half = 1ull << (s - 1);
        up = rem > half || (rem == half && (r & 1ull));
    } else if (s == 64) {
        r = hi;
        up = lo > (1ull << 63) || (lo == (1ull << 63) && (r & 1ull));
    } else {
        const int t = s - 64;
        r = hi >> t;
        const unsigned long long rem = hi & ((1ull << t) - 1ull), half = 1ull << (t - 1);
        up = rem > half || (rem == half && (lo != 0 || (r & 1ull)));
    }
    r += up ? 1ull : 0ull;
    return q < 0 ? -(long long)r : (long long)r;
}

// Half kick(s): v += round(h_m 2^8 F), w += round(h_i 2^8 (T - (T.n) n)) in
// grid units, with N the director in grid units.
__device__ inline void kick_grid(long long vq[3], long long wq[3], const double N[3], bool lipid, const Inst& I,
                                 int reps, const long long F[3], const long long Tq[3]) {
    for (int a = 0; a < 3; a++) vq[a] += reps * mul_round(F[a], I.hm8_m, I.hm8_s);
    if (lipid) {
        const double T0 = gd(Tq[0]), T1 = gd(Tq[1]), T2 = gd(Tq[2]);
        const double u = (T0 * N[0] + T1 * N[1] + T2 * N[2]) * 8.271806125530277e-25;   // (T.N) 2^-80
        wq[0] += reps * rg(I.hi8_d * (T0 - u * N[0]));
        wq[1] += reps * rg(I.hi8_d * (T1 - u * N[1]));
        wq[2] += reps * rg(I.hi8_d * (T2 - u * N[2]));
    }
}

// Cayley increment of the director in grid units: a = (dt/4 2^-40) W,
// B = a x N, delta = round(2/(1 + |a|^2) (B + a x B)).  The angular
// velocity stays perpendicular to the director (the kicks and the noise are
// projected onto the plane normal to it, and each rotation turns the
// director about it), so a x B = a (a.N) - |a|^2 N = -|a|^2 N up to rounding.
// The factor 2/(1 + |a|^2): for |a|^2 <= 2^-14 (every rotation of a few
// degrees or less per half step) the alternating series
// 2 (1 - aa + aa^2 - aa^3), whose truncation error 2 aa^4 / (1 + aa) is
// below 2^-55 relative, i.e. within the FP64 rounding of the quotient, in
// three fused multiply-adds instead of a division; larger |a|^2 divide.
__device__ inline double cayley_factor(double aa) {
    if (aa <= 6.103515625e-05) return fma(aa, fma(aa, fma(-2.0, aa, 2.0), -2.0), 2.0);
    return 2.0 / (1.0 + aa);
}
__device__ inline void cayley_grid(const double N[3], const double W[3], const Inst& I, long long d[3]) {
    const double a0 = I.ca_d * W[0], a1 = I.ca_d * W[1], a2 = I.ca_d * W[2];
    const double aa = a0 * a0 + a1 * a1 + a2 * a2;
    const double k = cayley_factor(aa);
    const double b0 = a1 * N[2] - a2 * N[1], b1 = a2 * N[0] - a0 * N[2], b2 = a0 * N[1] - a1 * N[0];
    d[0] = rg(k * fma(-aa, N[0], b0));
    d[1] = rg(k * fma(-aa, N[1], b1));
    d[2] = rg(k * fma(-aa, N[2], b2));
}

// round(a ma 2^-sa + b mb 2^-sb) to the nearest integer, ties to even, from
// the exact 128-bit sum of the two products, aligned to the larger scale
// (the host keeps the alignment inside 128 bits: ou_int); integer pipes.
__device__ inline long long mul2_round(long long a, long long ma, int sa, long long b, long long mb, int sb) {
    __int128 pa = (__int128)a * ma, pb = (__int128)b * mb;
    int s = sa;
    // (shifts on the two's-complement bits)
    if (sb > sa) { pa = (__int128)((unsigned __int128)pa << (sb - sa)); s = sb; }
    else if (sa > sb) pb = (__int128)((unsigned __int128)pb << (sa - sb));
    const __int128 t = pa + pb;
    const bool neg = t < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-t) : (unsigned __int128)t;
    unsigned __int128 r = u >> s;
    const unsigned __int128 rem = u - (r << s), half = (unsigned __int128)1 << (s - 1);
    if (rem > half || (rem == half && (r & 1))) r++;
    return neg ? -(long long)r : (long long)r;
}

// The noise's integer part 2 (w - 2^31) + 1 (exact); the factor
// sqrt(12) 2^-33 is folded into the host constants stn_d and srn_d.
__device__ inline double noise_int(unsigned w) {
    return (double)(2 * (long long)(int)(w ^ 0x80000000u) + 1);
}

// The same with FP64 increments in grid units.
template <bool FUSED>
__device__ inline void baoa_d_body(const View& v, const View& o, int p, const long long F[3], const long long Tq[3],
                                   const long long* __restrict__ steps, long long* __restrict__ msum,
                                   int* __restrict__ mcnt, unsigned mask, bool copy_static) {
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    const size_t N = v.N;
    const unsigned char type = v.type[p];
    const bool lipid = bilayer(type);
    long long xq[3], vq[3], nq[3] = {0, 0, 0}, wq[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) { xq[a] = v.xq[a * N + p]; vq[a] = v.vq[a * N + p]; }
    if (lipid) for (int a = 0; a < 3; a++) { nq[a] = v.nq[a * N + p]; wq[a] = v.wq[a * N + p]; }
    double Nd[3] = {0.0, 0.0, 0.0};
    if (lipid) for (int a = 0; a < 3; a++) Nd[a] = gd(nq[a]);
    // (final B of the previous step), B
    kick_grid(vq, wq, Nd, lipid, I, FUSED ? 2 : 1, F, Tq);
    // A
    double Wd[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; a++) xq[a] += mul_round(vq[a], I.hdt_m, I.hdt_s);
    if (lipid) {
        for (int a = 0; a < 3; a++) Wd[a] = gd(wq[a]);
        long long d[3];
        cayley_grid(Nd, Wd, I, d);
        for (int a = 0; a < 3; a++) { nq[a] += d[a]; Nd[a] = gd(nq[a]); }
    }
    // O
    const unsigned id = (unsigned)I.id_base + v.id[p];   // the id in the membrane
    const unsigned long long step = (unsigned long long)steps[b] + (FUSED ? 1ull : 0ull);
    const uint2 key = make_uint2((unsigned)I.seed, (unsigned)(I.seed >> 32) ^ I.instance);
    const uint4 w0 = philox4x32_10(make_uint4(id, (unsigned)step, (unsigned)(step >> 32), 0u), key);
    const unsigned wv[3] = {w0.x, w0.y, w0.z};
    for (int a = 0; a < 3; a++) {
        const long long sn = 2 * (long long)(int)(wv[a] ^ 0x80000000u) + 1;   // the noise's exact integer
        vq[a] += I.ou_int ? mul2_round(vq[a], I.ctm1_m, I.ctm1_s, sn, I.stn_m, I.stn_s)
                          : rg(fma(I.ct_m1_d, gd(vq[a]), I.stn_d * (double)sn));
    }
    if (lipid) {
        const uint4 w1 = philox4x32_10(make_uint4(id, (unsigned)step, (unsigned)(step >> 32), 1u), key);
        // the noise scaled by sr first: its projection is linear
        const double r0 = I.srn_d * noise_int(w1.x), r1 = I.srn_d * noise_int(w1.y), r2 = I.srn_d * noise_int(w1.z);
        const double u = (r0 * Nd[0] + r1 * Nd[1] + r2 * Nd[2]) * 8.271806125530277e-25;   // (r.N) 2^-80
        const double rp[3] = {r0 - u * Nd[0], r1 - u * Nd[1], r2 - u * Nd[2]};
        for (int a = 0; a < 3; a++) {
            const long long d = rg(fma(I.cr_m1_d, Wd[a], rp[a]));
            wq[a] += d;
            Wd[a] = gd(wq[a]);
        }
    }
    // A
    for (int a = 0; a < 3; a++) xq[a] += mul_round(vq[a], I.hdt_m, I.hdt_s);
    if (lipid) {
        long long d[3];
        cayley_grid(Nd, Wd, I, d);
        for (int a = 0; a < 3; a++) { nq[a] += d[a]; Nd[a] = gd(nq[a]); }
        // unit-norm correction n <- n (1 - delta/2), delta = |n|^2 - 1, with
        // |N|^2 - 2^80 exact in 128-bit integer arithmetic (integer pipes)
        // and delta/2 = that 2^-81, one conversion and one product
        const double hdelta = gd(norm2_excess(nq)) * 4.1359030627651384e-25;   // 2^-81
        for (int a = 0; a < 3; a++) nq[a] -= rg(Nd[a] * hdelta);
    }
    for (int a = 0; a < 3; a++) { o.xq[a * N + p] = xq[a]; o.vq[a * N + p] = vq[a]; }
    // in place a protein's (zero) director and angular velocity need no
    // store; into the other buffer, whose slot held another particle, they do
    if (lipid || copy_static) for (int a = 0; a < 3; a++) { o.nq[a * N + p] = nq[a]; o.wq[a * N + p] = wq[a]; }
    if (copy_static) { o.type[p] = type; o.id[p] = v.id[p]; }
    if (msum) mstep_sums(v, I, p, centroid_member(I, type), xq, msum, mcnt, mask);
}

// Counts the previous step after a fused launch read the counters.
__global__ void k_step_advance(long long* __restrict__ steps, int B);

}  // namespace orbc
