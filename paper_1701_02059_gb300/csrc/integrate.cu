// Time stepping ("Software Overview": force and torque, then update of
// position and orientation).  Reading: BAOAB Langevin (Leimkuhler & Matthews
// 2013), translational for every particle and rotational for lipids, with
// Cayley rotations of the director and uniform unit-variance noise from
// Philox4x32-10 keyed by (seed, instance; id, step, substream).
//
// State is int64 on the 2^-40 grid; every update is an increment computed in
// FP64 (FP32 for ORBC_F32_FORCE_F32_STEP) and rounded onto the grid, so
// accumulation is exact integer arithmetic.
#include "ensemble.cuh"

#include <cstring>

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

// Unit-norm correction n <- n (1 - delta/2), delta = |n|^2 - 1, first order
// (|delta| stays at the rounding level, ~1e-9).
__device__ inline void renormalise(long long nq[3], float) {
    // exact |n_q|^2 - 2^80 in 128-bit integer arithmetic
    unsigned long long H = 0, L = 0;
    for (int a = 0; a < 3; a++) {
        unsigned long long u = (unsigned long long)(nq[a] < 0 ? -nq[a] : nq[a]);
        unsigned long long lo = u * u, hi = __umul64hi(u, u);
        unsigned long long L2 = L + lo;
        H += hi + (L2 < L ? 1ull : 0ull);
        L = L2;
    }
    long long hd = (long long)H - (1ll << 16);     // multiples of 2^64
    if (hd != 0 && hd != -1) return;               // far from unit length: leave (not reached in practice)
    long long D = (long long)L;                    // exact when |D| < 2^63
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

// Half kick of v and w with the current force and torque (torque projected
// perpendicular to n); reps = 2 applies the same rounded increments twice
// (the final B of the previous step and this step's B share their forces).
template <typename T>
__device__ inline void kick(long long vq[3], long long wq[3], const long long nq[3], const View& v, int p, bool lipid,
                            const Consts<T>& C, int reps = 1) {
    using V = Num<T>;
    const size_t N = v.N;
    for (int a = 0; a < 3; a++) vq[a] += reps * V::grid(C.hm * V::frc(v.F[a * N + p]));
    if (lipid) {
        T t0 = V::frc(v.T[p]), t1 = V::frc(v.T[N + p]), t2 = V::frc(v.T[2 * N + p]);
        T n0 = V::st(nq[0]), n1 = V::st(nq[1]), n2 = V::st(nq[2]);
        T tn = t0 * n0 + t1 * n1 + t2 * n2;
        wq[0] += reps * V::grid(C.hi * (t0 - tn * n0));
        wq[1] += reps * V::grid(C.hi * (t1 - tn * n1));
        wq[2] += reps * V::grid(C.hi * (t2 - tn * n2));
    }
}

// B A O A of one step (the final B follows the force evaluation).  FUSED:
// first the final B of the previous step, whose forces are the same, then
// this step's B A O A: the same two rounded updates as separate launches,
// without a second pass over memory.  The previous step is then not yet
// counted in steps[], so this step's index is steps[b] + 1.
// The M-step's sums for the rebuild that follows (the "Spatial Searching
// Algorithm" update of each centroid from its lipids at the new positions):
// member i of cell k (a lipid, or any particle of a protein cell set) adds
// minimg(x_i - c_k) on the 2^-40 grid, exactly.  The
// lanes of a warp that share a cell add up a 24-bit low part and the high
// part separately in 32 bits, exact while |x_i - c_k| < 1024 sigma (the
// mirrors already flag anything beyond 32 sigma); one lane per cell adds the
// int64 totals.
__device__ inline void mstep_sums(const View& v, const Inst& I, int p, bool member, const long long* xq,
                                  long long* __restrict__ msum, int* __restrict__ mcnt) {
    const int k = v.cell[p];
    const size_t K = v.Ktot;
    long long d[3] = {0, 0, 0};
    if (member)
        for (int a = 0; a < 3; a++) d[a] = minimg_q(xq[a] - v.cq[a * K + k], I.boxq[a], I.periodic[a]);
    const unsigned grp = __match_any_sync(__activemask(), k);
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

template <typename T, bool FUSED>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 4) k_baoa(View v, const long long* __restrict__ steps,
                                                 long long* __restrict__ msum, int* __restrict__ mcnt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    using V = Num<T>;
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    const Consts<T> C(I);
    const size_t N = v.N;
    const bool lipid = v.type[p] == kLipid;
    long long xq[3], vq[3], nq[3] = {0, 0, 0}, wq[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) { xq[a] = v.xq[a * N + p]; vq[a] = v.vq[a * N + p]; }
    if (lipid) for (int a = 0; a < 3; a++) { nq[a] = v.nq[a * N + p]; wq[a] = v.wq[a * N + p]; }
    // (final B of the previous step), B
    kick<T>(vq, wq, nq, v, p, lipid, C, FUSED ? 2 : 1);
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
    for (int a = 0; a < 3; a++) { v.xq[a * N + p] = xq[a]; v.vq[a * N + p] = vq[a]; }
    if (lipid) for (int a = 0; a < 3; a++) { v.nq[a * N + p] = nq[a]; v.wq[a * N + p] = wq[a]; }
    if (msum) mstep_sums(v, I, p, centroid_member(I, v.type[p]), xq, msum, mcnt);
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

// Half kick(s): v += round(h_m 2^8 F), w += round(h_i 2^8 (T - (T.n) n)) in
// grid units, with N the director in grid units.
__device__ inline void kick_grid(long long vq[3], long long wq[3], const double N[3], const View& v, int p,
                                 bool lipid, const Inst& I, int reps) {
    const size_t NN = v.N;
    for (int a = 0; a < 3; a++) vq[a] += reps * rg(I.hm8_d * gd(v.F[a * NN + p]));
    if (lipid) {
        const double T0 = gd(v.T[p]), T1 = gd(v.T[NN + p]), T2 = gd(v.T[2 * NN + p]);
        const double u = (T0 * N[0] + T1 * N[1] + T2 * N[2]) * 8.271806125530277e-25;   // (T.N) 2^-80
        wq[0] += reps * rg(I.hi8_d * (T0 - u * N[0]));
        wq[1] += reps * rg(I.hi8_d * (T1 - u * N[1]));
        wq[2] += reps * rg(I.hi8_d * (T2 - u * N[2]));
    }
}

// Cayley increment of the director in grid units: a = (dt/4 2^-40) W,
// B = a x N, C = a x B, delta = round(2/(1 + |a|^2) (B + C)).
__device__ inline void cayley_grid(const double N[3], const double W[3], const Inst& I, long long d[3]) {
    const double a0 = I.ca_d * W[0], a1 = I.ca_d * W[1], a2 = I.ca_d * W[2];
    const double aa = a0 * a0 + a1 * a1 + a2 * a2;
    const double k = 2.0 / (1.0 + aa);
    const double b0 = a1 * N[2] - a2 * N[1], b1 = a2 * N[0] - a0 * N[2], b2 = a0 * N[1] - a1 * N[0];
    const double c0 = a1 * b2 - a2 * b1, c1 = a2 * b0 - a0 * b2, c2 = a0 * b1 - a1 * b0;
    d[0] = rg(k * (b0 + c0));
    d[1] = rg(k * (b1 + c1));
    d[2] = rg(k * (b2 + c2));
}

// Noise in grid-unit form: sqrt(12) 2^-33 (2 (w - 2^31) + 1), exact integer,
// one rounding.
__device__ inline double noise_grid(unsigned w) {
    const long long s = 2 * (long long)(int)(w ^ 0x80000000u) + 1;
    return (3.4641016151377544 * 1.16415321826934814453125e-10) * (double)s;
}

template <bool FUSED>
__global__ void __launch_bounds__(256, 2) k_baoa_d(View v, const long long* __restrict__ steps,
                                                   long long* __restrict__ msum, int* __restrict__ mcnt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    const size_t N = v.N;
    const bool lipid = v.type[p] == kLipid;
    long long xq[3], vq[3], nq[3] = {0, 0, 0}, wq[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) { xq[a] = v.xq[a * N + p]; vq[a] = v.vq[a * N + p]; }
    if (lipid) for (int a = 0; a < 3; a++) { nq[a] = v.nq[a * N + p]; wq[a] = v.wq[a * N + p]; }
    double Nd[3] = {0.0, 0.0, 0.0};
    if (lipid) for (int a = 0; a < 3; a++) Nd[a] = gd(nq[a]);
    // (final B of the previous step), B
    kick_grid(vq, wq, Nd, v, p, lipid, I, FUSED ? 2 : 1);
    // A
    double Vd[3], Wd[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; a++) {
        Vd[a] = gd(vq[a]);
        xq[a] += rg(I.hdt_d * Vd[a]);
    }
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
    const double xi[3] = {noise_grid(w0.x), noise_grid(w0.y), noise_grid(w0.z)};
    for (int a = 0; a < 3; a++) {
        const long long d = rg(I.ct_m1_d * Vd[a] + I.st40_d * xi[a]);
        vq[a] += d;
        Vd[a] = gd(vq[a]);
    }
    if (lipid) {
        const uint4 w1 = philox4x32_10(make_uint4(id, (unsigned)step, (unsigned)(step >> 32), 1u), key);
        const double r0 = noise_grid(w1.x), r1 = noise_grid(w1.y), r2 = noise_grid(w1.z);
        const double u = (r0 * Nd[0] + r1 * Nd[1] + r2 * Nd[2]) * 8.271806125530277e-25;   // (r.N) 2^-80
        const double rp[3] = {r0 - u * Nd[0], r1 - u * Nd[1], r2 - u * Nd[2]};
        for (int a = 0; a < 3; a++) {
            const long long d = rg(I.cr_m1_d * Wd[a] + I.sr40_d * rp[a]);
            wq[a] += d;
            Wd[a] = gd(wq[a]);
        }
    }
    // A
    for (int a = 0; a < 3; a++) xq[a] += rg(I.hdt_d * Vd[a]);
    if (lipid) {
        long long d[3];
        cayley_grid(Nd, Wd, I, d);
        for (int a = 0; a < 3; a++) { nq[a] += d[a]; Nd[a] = gd(nq[a]); }
        // unit-norm correction n <- n (1 - delta/2), delta = |n|^2 - 1
        const double delta = (Nd[0] * Nd[0] + Nd[1] * Nd[1] + Nd[2] * Nd[2]) * 8.271806125530277e-25 - 1.0;
        for (int a = 0; a < 3; a++) nq[a] -= rg(Nd[a] * 0.5 * delta);
    }
    for (int a = 0; a < 3; a++) { v.xq[a * N + p] = xq[a]; v.vq[a * N + p] = vq[a]; }
    if (lipid) for (int a = 0; a < 3; a++) { v.nq[a * N + p] = nq[a]; v.wq[a * N + p] = wq[a]; }
    if (msum) mstep_sums(v, I, p, centroid_member(I, v.type[p]), xq, msum, mcnt);
}

__global__ void k_kick_d(View v, long long* __restrict__ steps) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    const size_t N = v.N;
    const bool lipid = v.type[p] == kLipid;
    long long vq[3], wq[3] = {0, 0, 0};
    double Nd[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; a++) vq[a] = v.vq[a * N + p];
    if (lipid) for (int a = 0; a < 3; a++) { Nd[a] = gd(v.nq[a * N + p]); wq[a] = v.wq[a * N + p]; }
    kick_grid(vq, wq, Nd, v, p, lipid, I, 1);
    for (int a = 0; a < 3; a++) v.vq[a * N + p] = vq[a];
    if (lipid) for (int a = 0; a < 3; a++) v.wq[a * N + p] = wq[a];
    if (p == I.p0) steps[b] += 1;
}

// Counts the previous step after a fused launch read the counters.
__global__ void k_step_advance(long long* __restrict__ steps, int B) {
    for (int b = threadIdx.x; b < B; b += blockDim.x) steps[b] += 1;
}

// Final B of the step; advances the step counter of every instance.
template <typename T>
__global__ void k_kick(View v, long long* __restrict__ steps) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    const Consts<T> C(I);
    const size_t N = v.N;
    const bool lipid = v.type[p] == kLipid;
    long long vq[3], nq[3] = {0, 0, 0}, wq[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) vq[a] = v.vq[a * N + p];
    if (lipid) for (int a = 0; a < 3; a++) { nq[a] = v.nq[a * N + p]; wq[a] = v.wq[a * N + p]; }
    kick<T>(vq, wq, nq, v, p, lipid, C);
    for (int a = 0; a < 3; a++) v.vq[a * N + p] = vq[a];
    if (lipid) for (int a = 0; a < 3; a++) v.wq[a * N + p] = wq[a];
    if (p == I.p0) steps[b] += 1;
}

// Kinetic energies K_trans = sum m v^2 / 2, K_rot = sum_lipids I w^2 / 2,
// per particle in FP64, summed exactly as 2^-32 fixed point.
__global__ void k_kinetic(View v, long long* __restrict__ energy) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    long long kt = 0, kr = 0;
    int b = -1;
    if (p < v.N) {
        b = find_inst(v.inst_p0, v.B, p);
        const Inst& I = v.inst[b];
        const size_t N = v.N;
        double s = 0.0, r = 0.0;
        for (int a = 0; a < 3; a++) { double x = grid_to_double(v.vq[a * N + p]); s += x * x; }
        kt = __double2ll_rn(0.5 * I.mass * s * 4294967296.0);
        if (v.type[p] == kLipid) {
            for (int a = 0; a < 3; a++) { double x = grid_to_double(v.wq[a * N + p]); r += x * x; }
            kr = __double2ll_rn(0.5 * I.inertia * r * 4294967296.0);
        }
    }
    // warp-aggregate per instance
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    long long st = 0, sr = 0;
    unsigned m = grp;
    while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        st += __shfl_sync(grp, kt, src);
        sr += __shfl_sync(grp, kr, src);
    }
    if (b >= 0 && (int)(threadIdx.x & 31) == __ffs(grp) - 1) {
        atomicAdd((unsigned long long*)&energy[b * 8 + 2], (unsigned long long)st);
        atomicAdd((unsigned long long*)&energy[b * 8 + 3], (unsigned long long)sr);
    }
}

// Velocity quench ("Initial structure generation": the generated system is
// optimised by velocity quenching to remove collisions between particles;
// the paper names no scheme, the reading is quick-min with rotations): with
// the current force, v += dt F/m, then v is replaced by its component along
// F (zero when it points against F) and scaled down so that |dt v| <=
// max_move; x += dt v.  Lipids likewise with w, the torque's part normal to
// the director and max_turn, the director turned by the Cayley map of dt w.
// FP64 increments rounded onto the grid.
__global__ void k_quench(View v, double dt, double max_move, double max_turn) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    using V = Num<double>;
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    const size_t N = v.N;
    double F[3], u[3];
    for (int a = 0; a < 3; a++) {
        F[a] = V::frc(v.F[a * N + p]);
        u[a] = V::st(v.vq[a * N + p]) + dt * F[a] / I.mass;
    }
    const double vf = u[0] * F[0] + u[1] * F[1] + u[2] * F[2], ff = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    for (int a = 0; a < 3; a++) u[a] = (vf > 0.0 && ff > 0.0) ? (vf / ff) * F[a] : 0.0;
    const double mv = dt * sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (mv > max_move)
        for (int a = 0; a < 3; a++) u[a] *= max_move / mv;
    for (int a = 0; a < 3; a++) {
        v.xq[a * N + p] += V::grid(dt * u[a]);
        v.vq[a * N + p] = V::grid(u[a]);
    }
    if (v.type[p] != kLipid) return;
    long long nq[3], wq[3];
    double n[3], t[3], w[3];
    for (int a = 0; a < 3; a++) {
        nq[a] = v.nq[a * N + p];
        n[a] = V::st(nq[a]);
        t[a] = V::frc(v.T[a * N + p]);
    }
    const double tn = t[0] * n[0] + t[1] * n[1] + t[2] * n[2];
    for (int a = 0; a < 3; a++) {
        t[a] -= tn * n[a];
        w[a] = V::st(v.wq[a * N + p]) + dt * t[a] / I.inertia;
    }
    const double wt = w[0] * t[0] + w[1] * t[1] + w[2] * t[2], tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; a++) w[a] = (wt > 0.0 && tt > 0.0) ? (wt / tt) * t[a] : 0.0;
    const double mw = dt * sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (mw > max_turn)
        for (int a = 0; a < 3; a++) w[a] *= max_turn / mw;
    for (int a = 0; a < 3; a++) wq[a] = V::grid(w[a]);
    cayley<double>(nq, wq, dt);
    renormalise(nq, 0.0);
    for (int a = 0; a < 3; a++) { v.nq[a * N + p] = nq[a]; v.wq[a * N + p] = wq[a]; }
}

// Largest |F| over the particles, as the bits of a positive double.
__global__ void k_fmax(View v, unsigned long long* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    double f = 0.0;
    if (p < v.N) {
        const size_t N = v.N;
        double s = 0.0;
        for (int a = 0; a < 3; a++) { const double x = Num<double>::frc(v.F[a * N + p]); s += x * x; }
        f = sqrt(s);
    }
    for (int off = 16; off; off >>= 1) f = fmax(f, __shfl_xor_sync(0xffffffffu, f, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(f));
}

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

void Ensemble::launch_integrate_first(bool fused, bool msums) {
    long long* ms = msums ? d_msum : nullptr;
    int* mc = msums ? d_mcnt : nullptr;
    if (step_f32()) {
        if (fused) k_baoa<float, true><<<nblk(N, 256), 256, 0, stream>>>(view(), d_step, ms, mc);
        else k_baoa<float, false><<<nblk(N, 256), 256, 0, stream>>>(view(), d_step, ms, mc);
    } else {
        if (fused) k_baoa_d<true><<<nblk(N, 256), 256, 0, stream>>>(view(), d_step, ms, mc);
        else k_baoa_d<false><<<nblk(N, 256), 256, 0, stream>>>(view(), d_step, ms, mc);
    }
    launches++;
    if (fused) {
        k_step_advance<<<1, 64, 0, stream>>>(d_step, B);
        launches++;
    }
    CK(cudaGetLastError());
}

void Ensemble::launch_kick(bool energies) {
    if (step_f32()) k_kick<float><<<nblk(N, 256), 256, 0, stream>>>(view(), d_step);
    else k_kick_d<<<nblk(N, 256), 256, 0, stream>>>(view(), d_step);
    launches++;
    CK(cudaGetLastError());
    (void)energies;
}

double Ensemble::quench(int nsteps, double dt, double max_move, double max_turn) {
    if (!cells_valid) throw StateError("cells not initialised");
    if (!forces_valid) launch_pairs(false, false);
    for (int s = 0; s < nsteps; s++) {
        k_quench<<<nblk(N, 256), 256, 0, stream>>>(view(), dt, max_move, max_turn);
        launches++;
        CK(cudaGetLastError());
        rebuild(false);
        launch_pairs(false, false);
    }
    forces_valid = true;
    // velocities and angular velocities zero at the end
    CK(cudaMemsetAsync(d_state[cur_][1], 0, sizeof(long long) * 3 * (size_t)N, stream));
    CK(cudaMemsetAsync(d_state[cur_][3], 0, sizeof(long long) * 3 * (size_t)N, stream));
    unsigned long long* d = nullptr;
    CK(cudaMallocAsync(&d, sizeof(unsigned long long), stream));
    CK(cudaMemsetAsync(d, 0, sizeof(unsigned long long), stream));
    k_fmax<<<nblk(N, 256), 256, 0, stream>>>(view(), d);
    launches++;
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, stream));
    CK(cudaFreeAsync(d, stream));
    CK(cudaStreamSynchronize(stream));
    double fm;
    std::memcpy(&fm, &bits, sizeof(fm));
    return fm;
}

void Ensemble::launch_kinetic() {
    k_kinetic<<<nblk(N, 256), 256, 0, stream>>>(view(), d_energy);
    launches++;
    CK(cudaGetLastError());
}

}  // namespace orbc
