// Pair and bond forces through the Voronoi cells (arXiv 1701.02059, "Force
// Evaluation"): the quad loop over cell v_i, its neighbouring cells v_j, the
// particles of v_i and the particles of v_j, with the lipid cells reused at
// the wider search cutoff for protein pairs and the bond list for linked
// proteins.
//
// GPU design (one CTA of 4 warps per cell):
//   1. the mirrors of every neighbouring cell (contiguous after the sort) are
//      staged in shared memory by 1-D bulk async copies (TMA) completing on
//      an mbarrier, then moved into the cell's own frame: an exact int32
//      offset (wrap-around arithmetic) and an FP32 copy rotated into the
//      cell's tangent frame (normal = mean lipid director) for filtering;
//   2. the cell's particles are split into compact groups of <= 32 along
//      their longer tangent extent; each group's warps cull the staged
//      particles against the group's bounding box (r_s + band) into a
//      candidate list, then every lane tests the same candidate at once
//      (broadcast reads) against its own particle, appending hits to a
//      per-lane queue in shared memory;
//   3. queued pairs are evaluated with the exact integer displacement
//      (2^-26 sigma), the type-pair cutoff decided in FP64 inside a 1e-6 sigma
//      band, and the FP32 (or FP64) potential; force and torque on i are
//      accumulated exactly in split integers, so the sum does not depend on
//      the order or on how candidates are split across warps;
//   4. every pair is computed from both sides (no atomics to other cells, as
//      the paper does across patch boundaries); bonds of i are added in the
//      epilogue.
#include "integrator.cuh"

#include <mutex>

namespace orbc {

constexpr int kPairThreads = 128;
constexpr int kStageCap = 624;     // staged particles per pass
constexpr int kQCap = 32;          // queued hits per lane before a flush
constexpr int kMaxNbr = 32;        // neighbouring cells per pass (one per lane of the set-up warp)
constexpr float kFilterBand = 1e-4f;

// ---------------------------------------------------------------- pair terms
// Lipid pair (see the header of orbc.h for the potential).  d = x_j - x_i.
// Returns U; adds force on i and torque on i.
template <typename T, typename IC>
__device__ inline T lipid_terms(const IC& I, T dx, T dy, T dz, T r2, T nix, T niy, T niz, T njx, T njy, T njz,
                                T& fx, T& fy, T& fz, T& tx, T& ty, T& tz, T* tj);

__device__ inline float taylor_cos(float x) {
    // Maclaurin series of cos through x^14 on [0, pi/2]; truncation < 1e-9
    float x2 = x * x;
    float p = -1.1470745597729725e-11f;
    p = fmaf(p, x2, 2.08767569878681e-09f);
    p = fmaf(p, x2, -2.755731922398589e-07f);
    p = fmaf(p, x2, 2.48015873015873e-05f);
    p = fmaf(p, x2, -0.001388888888888889f);
    p = fmaf(p, x2, 0.041666666666666664f);
    p = fmaf(p, x2, -0.5f);
    return fmaf(p, x2, 1.0f);
}
__device__ inline float taylor_sin(float x) {
    // Maclaurin series of sin through x^15 on [0, pi/2]; truncation < 1e-10
    float x2 = x * x;
    float p = -7.647163731819816e-13f;
    p = fmaf(p, x2, 1.6059043836821613e-10f);
    p = fmaf(p, x2, -2.505210838544172e-08f);
    p = fmaf(p, x2, 2.7557319223985893e-06f);
    p = fmaf(p, x2, -0.0001984126984126984f);
    p = fmaf(p, x2, 0.008333333333333333f);
    p = fmaf(p, x2, -0.16666666666666666f);
    return x * fmaf(p, x2, 1.0f);
}

// FP32 lipid pair; Z > 0 fixes zeta at compile time (Z = 0: runtime zeta).
// S0: the spontaneous-curvature term is present (sin theta0 != 0); without
// it the terms in s0 drop out of a, w and the torque.
template <int Z, bool S0 = true, typename IC = Inst>
__device__ inline float lipid_terms_f(const IC& I, float dx, float dy, float dz, float r2, float nix, float niy,
                                      float niz, float njx, float njy, float njz, float& fx, float& fy, float& fz,
                                      float& tx, float& ty, float& tz, float* tj = nullptr) {
    const float rinv = rsqrtf(r2);
    const float r = r2 * rinv;
    // rh = r_ij / r = -(d) / r
    const float hx = -dx * rinv, hy = -dy * rinv, hz = -dz * rinv;
    const float s0 = I.s0;
    const float nin = fmaf(nix, njx, fmaf(niy, njy, niz * njz));
    const float nir = fmaf(nix, hx, fmaf(niy, hy, niz * hz));
    const float njr = fmaf(njx, hx, fmaf(njy, hy, njz * hz));
    const float a = S0 ? fmaf(s0, njr - nir, fmaf(-nir, njr, nin)) - s0 * s0 : fmaf(-nir, njr, nin);
    const float phi = fmaf(I.mu, a - 1.0f, 1.0f);
    float f, fp, g, gp;
    if (r < I.rmin) {
        const float q = I.rmin * rinv;
        const float q2 = q * q, q4 = q2 * q2;
        f = fmaf(I.eps, q4 - 2.0f * q2, I.eps);
        fp = 4.0f * I.eps * rinv * (q2 - q4);
        g = -I.eps;
        gp = 0.0f;
    } else {
        const float th = I.aw * (r - I.rmin);
        const float c = taylor_cos(th), sn = taylor_sin(th);
        // c^(2 zeta - 1) by binary powering from the low bits: the general
        // path forms the same products in the same order as the zeta = 4
        // one, so an instance gives the same bits in a batch that mixes
        // exponents (which takes the general path) as alone
        float cp;
        if (Z == 4) {
            const float c2 = c * c, c4 = c2 * c2;
            cp = (c * c2) * c4;
        } else {
            cp = 1.0f;
            float bp = c;
            for (int e = 2 * I.zeta - 1; e > 0; e >>= 1) {
                if (e & 1) cp *= bp;
                bp *= bp;
            }
        }
        f = 0.0f;
        fp = 0.0f;
        g = -I.eps * cp * c;
        gp = I.eps2z_aw * cp * sn;
    }
    const float U = fmaf(g, phi, f);
    float wx = fmaf(-njr, nix, -nir * njx), wy = fmaf(-njr, niy, -nir * njy), wz = fmaf(-njr, niz, -nir * njz);
    if (S0) {
        wx = fmaf(s0, njx - nix, wx);
        wy = fmaf(s0, njy - niy, wy);
        wz = fmaf(s0, njz - niz, wz);
    }
    const float wr = fmaf(wx, hx, fmaf(wy, hy, wz * hz));
    const float radial = fmaf(gp, phi, fp);
    const float gm = g * I.mu;
    const float gmr = gm * rinv;
    fx += -radial * hx - gmr * fmaf(-wr, hx, wx);
    fy += -radial * hy - gmr * fmaf(-wr, hy, wy);
    fz += -radial * hz - gmr * fmaf(-wr, hz, wz);
    // da/dn_i = n_j - (n_j.rh + s0) rh ; tau_i = -g mu (n_i x da/dn_i)
    const float js = S0 ? njr + s0 : njr;
    const float gx = fmaf(-js, hx, njx), gy = fmaf(-js, hy, njy), gz = fmaf(-js, hz, njz);
    tx += -gm * (niy * gz - niz * gy);
    ty += -gm * (niz * gx - nix * gz);
    tz += -gm * (nix * gy - niy * gx);
    if (tj) {
        // da/dn_j = n_i - (n_i.rh - s0) rh ; tau_j = -g mu (n_j x da/dn_j)
        const float is = nir - s0;
        const float ux = fmaf(-is, hx, nix), uy = fmaf(-is, hy, niy), uz = fmaf(-is, hz, niz);
        tj[0] = -gm * (njy * uz - njz * uy);
        tj[1] = -gm * (njz * ux - njx * uz);
        tj[2] = -gm * (njx * uy - njy * ux);
    }
    return U;
}

template <typename T, typename IC>
__device__ inline T lipid_terms(const IC& I, T dx, T dy, T dz, T r2, T nix, T niy, T niz, T njx, T njy, T njz,
                                T& fx, T& fy, T& fz, T& tx, T& ty, T& tz, T* tj) {
    static_assert(sizeof(T) == 8, "the FP32 terms are lipid_terms_f");
    double r = sqrt(r2);
    double hx = -dx / r, hy = -dy / r, hz = -dz / r;
    double s0 = I.s0_d;
    double nin = nix * njx + niy * njy + niz * njz;
    double nir = nix * hx + niy * hy + niz * hz;
    double njr = njx * hx + njy * hy + njz * hz;
    double a = nin - nir * njr + s0 * (njr - nir) - s0 * s0;
    double phi = 1.0 + I.mu_d * (a - 1.0);
    double f, fp, g, gp;
    if (r < I.rmin_d) {
        double q = I.rmin_d / r;
        double q2 = q * q, q4 = q2 * q2;
        f = I.eps_d * (q4 - 2.0 * q2) + I.eps_d;
        fp = I.eps_d * (-4.0 * q4 / r + 4.0 * q2 / r);
        g = -I.eps_d;
        gp = 0.0;
    } else {
        double w = 1.5707963267948966 / (I.rc_d - I.rmin_d);
        double th = w * (r - I.rmin_d);
        double c, sn;
        sincos(th, &sn, &c);
        double cp = 1.0;
        for (int k = 0; k < 2 * I.zeta - 1; k++) cp *= c;
        f = 0.0;
        fp = 0.0;
        g = -I.eps_d * cp * c;
        gp = I.eps_d * (double)(2 * I.zeta) * cp * sn * w;
    }
    double U = f + g * phi;
    double wx = -njr * nix - nir * njx + s0 * (njx - nix);
    double wy = -njr * niy - nir * njy + s0 * (njy - niy);
    double wz = -njr * niz - nir * njz + s0 * (njz - niz);
    double wr = wx * hx + wy * hy + wz * hz;
    double radial = fp + gp * phi;
    double gm = g * I.mu_d;
    fx += -radial * hx - gm * (wx - wr * hx) / r;
    fy += -radial * hy - gm * (wy - wr * hy) / r;
    fz += -radial * hz - gm * (wz - wr * hz) / r;
    double js = njr + s0;
    double gx = njx - js * hx, gy = njy - js * hy, gz = njz - js * hz;
    tx += -gm * (niy * gz - niz * gy);
    ty += -gm * (niz * gx - nix * gz);
    tz += -gm * (nix * gy - niy * gx);
    if (tj) {
        double is = nir - s0;
        double ux = nix - is * hx, uy = niy - is * hy, uz = niz - is * hz;
        tj[0] = -gm * (njy * uz - njz * uy);
        tj[1] = -gm * (njz * ux - njx * uz);
        tj[2] = -gm * (njx * uy - njy * ux);
    }
    return U;
}

// WCA; d = x_j - x_i; adds the force on i.  pp: protein-protein size.
template <typename T>
__device__ inline T wca_terms(const Inst& I, bool pp, T dx, T dy, T dz, T r2, T& fx, T& fy, T& fz) {
    T sig = (sizeof(T) == 4) ? (T)(pp ? I.sig_pp : I.sig_wca) : (T)(pp ? I.sig_pp_d : I.sig_wca_d);
    T e = (sizeof(T) == 4) ? (T)I.eps_wca : (T)I.eps_wca_d;
    T s2 = sig * sig / r2;
    T s6 = s2 * s2 * s2;
    T s12 = s6 * s6;
    T fr = (T)4 * e * ((T)12 * s12 - (T)6 * s6) / r2;
    fx -= fr * dx;
    fy -= fr * dy;
    fz -= fr * dz;
    return (T)4 * e * (s12 - s6) + e;
}

// ---------------------------------------------------------------- accumulators
template <typename T> struct Acc;
template <> struct Acc<float> {
    // fast path: split int32 sums (|component sum| < 1000); wider values go
    // to an int64 side array with atomics (exact, rare)
    SplitAcc f[3], t[3];
    int nf, nt;
    bool used_big;
    __device__ void zero() { for (int a = 0; a < 3; a++) { f[a].zero(); t[a].zero(); } nf = 0; nt = 0; used_big = false; }
    __device__ void add3(const View& v, int p, SplitAcc* s, int& n, int c0, float x, float y, float z) {
        const float mag = fabsf(x) + fabsf(y) + fabsf(z);
        if (mag < 1000.0f) { s[0].add(x); s[1].add(y); s[2].add(z); n++; return; }
        // NaN, infinite, or a term beyond the range the 2^-32 fixed-point
        // sums hold (|component| < 2^31 after a few hundred terms)
        if (!(mag < kMaxTerm))
            flag_inst(v, v.inst[find_inst(v.inst_p0, v.B, p)], (mag == mag) ? kStatusPairForceRange : kStatusNaN);
        const size_t N = v.N;
        atomicAdd((unsigned long long*)&v.Fbig[(size_t)c0 * N + p], (unsigned long long)__float2ll_rn(x * 4294967296.0f));
        atomicAdd((unsigned long long*)&v.Fbig[(size_t)(c0 + 1) * N + p], (unsigned long long)__float2ll_rn(y * 4294967296.0f));
        atomicAdd((unsigned long long*)&v.Fbig[(size_t)(c0 + 2) * N + p], (unsigned long long)__float2ll_rn(z * 4294967296.0f));
        used_big = true;
    }
    __device__ void add_pair(const View& v, int p, float fx, float fy, float fz, float tx, float ty, float tz) {
        add3(v, p, f, nf, 0, fx, fy, fz);
        add3(v, p, t, nt, 3, tx, ty, tz);
    }
    __device__ void add_bond(const View& v, int p, float fx, float fy, float fz) { add3(v, p, f, nf, 0, fx, fy, fz); }
};
template <> struct Acc<double> {
    long long f[3], t[3];
    int np, nb;
    __device__ void zero() { for (int a = 0; a < 3; a++) { f[a] = 0; t[a] = 0; } np = 0; nb = 0; }
    __device__ static long long q(double v) { return __double2ll_rn(v * 4294967296.0); }
    __device__ void add_pair(const View& v, int p, double fx, double fy, double fz, double tx, double ty, double tz) {
        const double mag = fabs(fx) + fabs(fy) + fabs(fz) + fabs(tx) + fabs(ty) + fabs(tz);
        if (!(mag < (double)kMaxTerm))
            flag_inst(v, v.inst[find_inst(v.inst_p0, v.B, p)], (mag == mag) ? kStatusPairForceRange : kStatusNaN);
        f[0] += q(fx); f[1] += q(fy); f[2] += q(fz); t[0] += q(tx); t[1] += q(ty); t[2] += q(tz); np++;
    }
    __device__ void add_bond(const View&, int, double fx, double fy, double fz) { f[0] += q(fx); f[1] += q(fy); f[2] += q(fz); nb++; }
    __device__ long long F(int a) const { return f[a]; }
    __device__ long long Tq(int a) const { return t[a]; }
};

// exact FP64 inclusion decision for a pair inside the cutoff band; m: the
// bilayer species pair (cls 0)
__device__ inline bool exact_inside(const View& v, const Inst& I, int pi, int pj, int cls, int m = 0) {
    size_t N = v.N;
    double d2 = dist2_grid_d(v.xq[pj], v.xq[N + pj], v.xq[2 * N + pj], v.xq[pi], v.xq[N + pi], v.xq[2 * N + pi], I);
    return d2 < (cls == 0 ? I.mm_rc2[m] : (cls == 1 ? I.rc2_wca : I.rc2_pp));
}

// Pair class of two types: 0 two bilayer particles (the lipid potential), 1
// a bilayer particle and a cytoskeleton protein, 2 two cytoskeleton proteins
// (both WCA); m: the bilayer species pair 3 s_i + s_j of class 0.
__device__ inline int pair_class(int ti, int tj, int& m) {
    const bool bi = bilayer(ti), bj = bilayer(tj);
    m = (bi && bj) ? 3 * species(ti) + species(tj) : 0;
    return (bi && bj) ? 0 : ((bi || bj) ? 1 : 2);
}

// The lipid potential's constants of one bilayer species pair, in the field
// names of Inst (FP32 and FP64), for the pair-term functions.
struct LipK {
    float eps, rmin, mu, s0, aw, eps2z_aw;
    int zeta;
    double eps_d, rmin_d, rc_d, mu_d, s0_d;
    __device__ LipK(const Inst& I, int m)
        : eps(I.mm_eps[m]), rmin(I.rmin), mu(I.mu), s0(I.s0), aw(I.mm_aw[m]), eps2z_aw(I.mm_e2za[m]), zeta(I.zeta),
          eps_d(I.mm_eps_d[m]), rmin_d(I.rmin_d), rc_d(I.mm_rc_d[m]), mu_d(I.mu_d), s0_d(I.s0_d) {}
};

// 1-2 and 1-3 bonded pairs carry no excluded-volume term (bonded directly,
// or sharing a bond partner).  Ids are local to i's instance I; slot pj
// outside I (the partner cell set of a membrane, which no bond reaches) is
// never excluded.
__device__ inline bool is_excluded(const View& v, const Inst& I, unsigned idi, unsigned idj, int pj) {
    if ((unsigned)(pj - I.p0) >= (unsigned)I.n) return false;
    const int s = v.bptr[I.p0 + idi], e = v.bptr[I.p0 + idi + 1];
    const int s2 = v.bptr[I.p0 + idj], e2 = v.bptr[I.p0 + idj + 1];
    for (int q = s; q < e; q++) {
        const int c = v.bpartner[q];
        if ((unsigned)c == idj) return true;
        for (int w = s2; w < e2; w++)
            if (v.bpartner[w] == c) return true;
    }
    return false;
}

// ---------------------------------------------------------------- TMA helpers
__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ inline void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ inline void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ inline bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `polls` polls (2^22 by default: with the
// back-off, well over a second), records a timeout in the status word and
// returns false.
__device__ inline bool mbar_wait_bounded(unsigned long long* bar, unsigned phase, unsigned* status,
                                         unsigned polls) {
    for (unsigned it = 0; it < polls; it++) {
        if (mbar_try_wait(bar, phase)) return true;
        if (it > 64) __nanosleep(256);
    }
    atomicOr(status, kStatusTimeout);
    return false;
}

// ---------------------------------------------------------------- the kernel
struct NbrInfo {
    int base;       // first staged index
    int cnt;
    int start;      // global slot of the first particle
    int ox, oy, oz; // exact offset c_l - c_k at 2^-26 sigma (wrap-around int32)
};

template <typename T, bool S0, typename IC = Inst>
__device__ inline T lipid_dispatch(const IC& I, T dx, T dy, T dz, T r2, T nix, T niy, T niz, T njx, T njy, T njz,
                                   T& fx, T& fy, T& fz, T& tx, T& ty, T& tz, int zc, T* tj) {
    if constexpr (sizeof(T) == 4) {
        if (zc == 4)
            return lipid_terms_f<4, S0, IC>(I, dx, dy, dz, r2, nix, niy, niz, njx, njy, njz, fx, fy, fz, tx, ty, tz, tj);
        return lipid_terms_f<0, true, IC>(I, dx, dy, dz, r2, nix, niy, niz, njx, njy, njz, fx, fy, fz, tx, ty, tz, tj);
    } else {
        return lipid_terms<double, IC>(I, dx, dy, dz, r2, nix, niy, niz, njx, njy, njz, fx, fy, fz, tx, ty, tz, tj);
    }
}


// S0: some instance has a spontaneous-curvature term (s0 != 0).
template <typename T, bool ENERGY, bool DUMP, int Z, bool S0>
__global__ void __launch_bounds__(kPairThreads, 5) k_pairs(View v, long long* __restrict__ energy /* [B][8] */,
                                                            unsigned* __restrict__ dump,
                                                            unsigned long long* __restrict__ dump_count,
                                                            long long dump_cap) {
    // sy: staged mirrors, after staging in the cell-k frame (exact int32,
    //     2^-26 sigma), w = type
    // sY: the same particles in FP32, rotated into the tangent frame
    // so: directors, w = global slot
    __shared__ alignas(16) int4 sy[kStageCap];
    __shared__ alignas(16) float4 sY[kStageCap];
    __shared__ alignas(16) float4 so[kStageCap];
    __shared__ alignas(16) unsigned short cand[kPairThreads / 32][kStageCap];   // per-warp candidate list
    __shared__ unsigned short qbuf[kPairThreads / 32][kQCap][32];   // per-lane hit queues
    __shared__ NbrInfo nb[kMaxNbr];
    __shared__ unsigned long long bar;
    __shared__ int s_nstage, s_next, s_next_off, s_self, s_self_lo, s_self_hi, s_total;

    const int k = blockIdx.x;
    const int b = find_inst(v.inst_k0, v.B, k);
    const Inst& I = v.inst[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cs = v.cell_start[k], ce = v.cell_start[k + 1];
    // the cell's neighbour row (fixed stride; rows longer than kAdjRow are
    // flagged by the adjacency pass)
    const AdjDesc* __restrict__ row = v.adjd + (size_t)k * kAdjRow;
    const int a0 = 0;
    const int a1 = min(v.adjn[k], kAdjRow);
    const float rs_b = I.rsf + kFilterBand;
    const float rs2f = rs_b * rs_b;
    const float rcl = sqrtf(I.rc2f_ll), rcw = sqrtf(I.rc2f_wca), rcp = sqrtf(I.rc2f_pp);
    const float ll_lo = (rcl - kCutBand) * (rcl - kCutBand), ll_hi = (rcl + kCutBand) * (rcl + kCutBand);
    const float w_lo = (rcw - kCutBand) * (rcw - kCutBand), w_hi = (rcw + kCutBand) * (rcw + kCutBand);
    const float p_lo = (rcp - kCutBand) * (rcp - kCutBand), p_hi = (rcp + kCutBand) * (rcp + kCutBand);
    const size_t N = v.N;
    const int zc = (Z > 0) ? Z : I.zeta;
    unsigned phase = 0;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();

    for (int it0 = cs; it0 < ce; it0 += kPairThreads) {
        const int nti = min(kPairThreads, ce - it0);            // particles of this i-tile
        const int groups = (nti + 31) >> 5;                     // compact groups of <= 32
        const int nsplit = (groups == 1) ? 4 : (groups == 2 ? 2 : 1);
        const int igrp = warp % groups;
        const int jsplit = warp / groups;
        const bool wactive = jsplit < nsplit;
        const int gs = (nti + groups - 1) / groups;             // balanced group size

        // staging of one pass (warp 0): neighbour descriptors, bulk copies
        auto issue = [&](const int na, const int na_off) {
                if (warp == 0) {
                    // one lane per neighbouring cell: counts, offsets, staging slots
                    const int nn = na + lane;
                    const bool has = nn < a1;
                    int l = 0, st = 0, c = 0;
                    AdjDesc d;
                    if (has) {
                        d = row[nn];
                        l = d.cell;
                        st = d.start;
                        c = d.cnt;
                        if (lane == 0) { st += na_off; c -= na_off; }
                    }
                    int incl = c;
                    for (int off = 1; off < 32; off <<= 1) {
                        const int t = __shfl_up_sync(0xffffffffu, incl, off);
                        if (lane >= off) incl += t;
                    }
                    const int excl = incl - c;
                    const bool fits = has && incl <= kStageCap;
                    const bool part = has && excl < kStageCap && incl > kStageCap;
                    const unsigned fm = __ballot_sync(0xffffffffu, fits), pm = __ballot_sync(0xffffffffu, part);
                    const int m = __popc(fm) + (pm ? 1 : 0);
                    const bool staged = fits || part;
                    const int take = part ? kStageCap - excl : c;
                    if (staged) {
                        NbrInfo inf;
                        inf.base = excl; inf.cnt = take; inf.start = st;
                        inf.ox = d.ox; inf.oy = d.oy; inf.oz = d.oz;
                        nb[lane] = inf;
                    }
                    const unsigned selfm = __ballot_sync(0xffffffffu, staged && l == k);
                    const int total = __shfl_sync(0xffffffffu, excl + take, max(m - 1, 0));
                    // where the next pass starts: after the last fully staged
                    // neighbour, or inside the partially staged one
                    int nxt = na + __popc(fm), nxo = 0;
                    if (pm) {
                        const int p = __ffs(pm) - 1;
                        const int ex_p = __shfl_sync(0xffffffffu, excl, p);
                        nxt = na + p;
                        nxo = (p == 0 ? na_off : 0) + (kStageCap - ex_p);
                    }
                    // staged range of the own cell, and where its first particle would sit
                    int slo = -1, shi = -1, sb = 0;
                    {
                        const int p = selfm ? __ffs(selfm) - 1 : 0;
                        const int ex_p = __shfl_sync(0xffffffffu, excl, p);
                        const int tk_p = __shfl_sync(0xffffffffu, take, p);
                        if (selfm) {
                            slo = ex_p;
                            shi = ex_p + tk_p;
                            sb = ex_p - ((p == 0) ? na_off : 0);
                        }
                    }
                    if (lane == 0) {
                        s_nstage = m;
                        s_total = m > 0 ? total : 0;
                        s_next = nxt;
                        s_next_off = nxo;
                        s_self = sb; s_self_lo = slo; s_self_hi = shi;
                    }
                    if (m > 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        if (lane == 0) mbar_expect_tx(&bar, (unsigned)total * 32u + v.extra_tx);
                        __syncwarp();
                        if (staged && take > 0) {
                            bulk_g2s(&sy[excl], v.mqr + st, take * 16u, &bar);
                            bulk_g2s(&so[excl], v.mor + st, take * 16u, &bar);
                        }
                    }
                }
        };
        // the first pass's copies are in flight during the tile set-up
        if (a0 < a1) issue(a0, 0);

        // ---- tangent frame of the cell; the mirrors of each tile of 128 are
        //      stored in the order of their rank along the tile's longer
        //      tangent extent (prepared with the cell radii), so that the
        //      group of rank range [g gs, (g + 1) gs) is compact
        const float4 cn = v.cnorm[k];
        const Frame F = tangent_frame(cn.x, cn.y, cn.z);

        // ---- this lane's particle: rank r of the tile, slot pi
        const int r = igrp * gs + lane;
        const bool ivalid = wactive && lane < gs && r < nti;
        int ti = 0, pi = -1;
        int4 qi = make_int4(0, 0, 0, 0);
        float4 oi = make_float4(0, 0, 0, 0);
        float yix = 0.f, yiy = 0.f, yiz = 0.f;
        unsigned idi = 0;
        if (ivalid) {
            qi = v.mqr[it0 + r];
            oi = v.mor[it0 + r];
            pi = __float_as_int(oi.w);
            ti = qi.w & 0xff;
            F.apply(qi.x * kMirrorUnit, qi.y * kMirrorUnit, qi.z * kMirrorUnit, yix, yiy, yiz);
            if (DUMP) idi = (unsigned)I.id_base + v.id[pi];
        }
        // a lane without a particle sits far away: it passes no distance test
        if (!ivalid) { yix = 1.0e18f; yiy = 1.0e18f; yiz = 1.0e18f; }
        // group bounding box in the tangent frame, widened by the search radius
        float blo[3] = {ivalid ? yix : 3.0e38f, ivalid ? yiy : 3.0e38f, ivalid ? yiz : 3.0e38f};
        float bhi[3] = {ivalid ? yix : -3.0e38f, ivalid ? yiy : -3.0e38f, ivalid ? yiz : -3.0e38f};
        for (int a = 0; a < 3; a++)
            for (int off = 16; off; off >>= 1) {
                blo[a] = fminf(blo[a], __shfl_xor_sync(0xffffffffu, blo[a], off));
                bhi[a] = fmaxf(bhi[a], __shfl_xor_sync(0xffffffffu, bhi[a], off));
            }
        Acc<T> acc;
        acc.zero();
        double up = 0, vir = 0;     // per-particle energy and virial partials, FP64 in every mode

        // passes over chunks of neighbouring cells (a cell larger than the
        // stage is split across passes)
        bool first_pass = true;
        for (int na = a0, na_off = 0; na < a1;) {
            if (!first_pass) {
                __syncthreads();
                issue(na, na_off);
            }
            first_pass = false;
            __syncthreads();
            const int m = s_nstage;
            const int total = s_total;
            const int next = s_next, next_off = s_next_off;
            if (m == 0) { na = next; na_off = next_off; continue; }
            const int sself = s_self, sslo = s_self_lo, sshi = s_self_hi;
            int selfj = (sslo >= 0 && ivalid) ? sself + (it0 + r - cs) : -1;
            if (selfj < sslo || selfj >= sshi) selfj = -1;
            bool ok = mbar_wait_bounded(&bar, phase, v.status, v.wait_polls);
            if (__syncthreads_or(!ok)) {
                // give the copies in flight a second bounded wait, then leave
                if (ok == false) mbar_wait_bounded(&bar, phase, v.status, v.wait_polls);
                return;
            }
            phase ^= 1u;

            // ---- staged particles into the cell-k frame (exact) and the
            //      tangent frame (FP32)
            for (int q = 0; q < m; q++) {
                const NbrInfo inf = nb[q];
                for (int j = inf.base + tid; j < inf.base + inf.cnt; j += kPairThreads) {
                    int4 rj = sy[j];
                    rj.x = (int)((unsigned)rj.x + (unsigned)inf.ox);
                    rj.y = (int)((unsigned)rj.y + (unsigned)inf.oy);
                    rj.z = (int)((unsigned)rj.z + (unsigned)inf.oz);
                    sy[j] = rj;
                    float4 y;
                    F.apply(rj.x * kMirrorUnit, rj.y * kMirrorUnit, rj.z * kMirrorUnit, y.x, y.y, y.z);
                    y.w = 0.f;
                    sY[j] = y;
                }
            }
            __syncthreads();

            if (wactive) {
                // ---- candidates: staged particles within r_s (+ band) of the
                //      group's box; the warps of a group take every nsplit-th
                //      staged particle, so that their shares of the candidates
                //      and hits stay even (whole chunks per warp left them
                //      waiting on each other at the next barrier)
                int cnt = 0;
                for (int c0 = 0; c0 < total; c0 += nsplit * 32) {
                    const int j = c0 + lane * nsplit + jsplit;
                    bool in = false;
                    if (j < total) {
                        const float4 y = sY[j];
                        const float ex = fmaxf(fmaxf(blo[0] - y.x, y.x - bhi[0]), 0.f);
                        const float ey = fmaxf(fmaxf(blo[1] - y.y, y.y - bhi[1]), 0.f);
                        const float ez = fmaxf(fmaxf(blo[2] - y.z, y.z - bhi[2]), 0.f);
                        in = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < rs2f;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, in);
                    if (in) cand[warp][cnt + __popc(bal & ((1u << lane) - 1u))] = (unsigned short)j;
                    cnt += __popc(bal);
                }
                __syncwarp();

                int qn = 0;
                auto flush = [&]() {
                    int qmax = qn;
                    for (int off = 16; off; off >>= 1) qmax = max(qmax, __shfl_xor_sync(0xffffffffu, qmax, off));
                    for (int t = 0; t < qmax; t++) {
                        if (t >= qn) continue;
                        const int j = (int)qbuf[warp][t][lane];
                        const int4 mj = sy[j];
                        const float4 oj = so[j];
                        const int pj = __float_as_int(oj.w);
                        const int tj = mj.w & 0xff;
                        int m;
                        const int cls = pair_class(ti, tj, m);
                        const bool ll = cls == 0;
                        const int dxq = (int)((unsigned)mj.x - (unsigned)qi.x);
                        const int dyq = (int)((unsigned)mj.y - (unsigned)qi.y);
                        const int dzq = (int)((unsigned)mj.z - (unsigned)qi.z);
                        const float dxf = (float)dxq * kMirrorUnit, dyf = (float)dyq * kMirrorUnit,
                                    dzf = (float)dzq * kMirrorUnit;
                        const float r2f = fmaf(dxf, dxf, fmaf(dyf, dyf, dzf * dzf));
                        const float lo = cls == 0 ? (I.has_mp ? I.mm_lo[m] : ll_lo) : (cls == 1 ? w_lo : p_lo);
                        const float hi = cls == 0 ? (I.has_mp ? I.mm_hi[m] : ll_hi) : (cls == 1 ? w_hi : p_hi);
                        if (r2f >= hi) continue;
                        bool in = r2f < lo;
                        if (!in) in = exact_inside(v, I, pi, pj, cls, m);
                        if (in && cls != 0 && is_excluded(v, I, v.id[pi], v.id[pj], pj)) in = false;
                        if (!in) continue;
                        T fx = 0, fy = 0, fz = 0, tx = 0, ty = 0, tz = 0, U;
                        T dx, dy, dz, r2;
                        if constexpr (sizeof(T) == 4) {
                            dx = dxf; dy = dyf; dz = dzf; r2 = r2f;
                        } else {
                            dx = grid_to_double(minimg_q(v.xq[pj] - v.xq[pi], I.boxq[0], I.periodic[0]));
                            dy = grid_to_double(minimg_q(v.xq[N + pj] - v.xq[N + pi], I.boxq[1], I.periodic[1]));
                            dz = grid_to_double(minimg_q(v.xq[2 * N + pj] - v.xq[2 * N + pi], I.boxq[2], I.periodic[2]));
                            r2 = dx * dx + dy * dy + dz * dz;
                        }
                        if (ll) {
                            T nix, niy, niz, njx, njy, njz;
                            if constexpr (sizeof(T) == 4) {
                                nix = oi.x; niy = oi.y; niz = oi.z; njx = oj.x; njy = oj.y; njz = oj.z;
                            } else {
                                nix = grid_to_double(v.nq[pi]); niy = grid_to_double(v.nq[N + pi]);
                                niz = grid_to_double(v.nq[2 * N + pi]);
                                njx = grid_to_double(v.nq[pj]); njy = grid_to_double(v.nq[N + pj]);
                                njz = grid_to_double(v.nq[2 * N + pj]);
                            }
                            if (I.has_mp)
                                U = lipid_dispatch<T, S0, LipK>(LipK(I, m), dx, dy, dz, r2, nix, niy, niz, njx, njy, njz,
                                                                fx, fy, fz, tx, ty, tz, zc, (T*)nullptr);
                            else
                                U = lipid_dispatch<T, S0>(I, dx, dy, dz, r2, nix, niy, niz, njx, njy, njz, fx, fy, fz, tx,
                                                          ty, tz, zc, (T*)nullptr);
                        } else {
                            U = wca_terms<T>(I, cls == 2, dx, dy, dz, r2, fx, fy, fz);
                        }
                        acc.add_pair(v, pi, fx, fy, fz, tx, ty, tz);
                        if (ENERGY) {
                            up += 0.5 * (double)U;
                            vir += -0.5 * ((double)dx * (double)fx + (double)dy * (double)fy + (double)dz * (double)fz);
                        }
                        if (DUMP) {
                            const unsigned idj =
                                (unsigned)v.inst[find_inst(v.inst_p0, v.B, pj)].id_base + v.id[pj];
                            if (idi < idj) {
                                unsigned long long slot = atomicAdd(dump_count, 1ull);
                                if ((long long)slot < dump_cap) { dump[2 * slot] = idi; dump[2 * slot + 1] = idj; }
                            }
                        }
                    }
                    qn = 0;
                    __syncwarp();
                };
                // ---- every lane tests the same candidate (broadcast reads)
                static_assert(kStageCap % 8 == 0, "candidate lists are read 8 at a time");
                for (int c = 0; c < cnt; c += 8) {
                    if (__any_sync(0xffffffffu, qn > kQCap - 8)) flush();
                    const uint4 c8 = *reinterpret_cast<const uint4*>(&cand[warp][c]);   // 8 indices, broadcast
                    const unsigned cw[4] = {c8.x, c8.y, c8.z, c8.w};
#pragma unroll
                    for (int u = 0; u < 8; u++) {
                        if (c + u < cnt) {
                            const int j = (int)((cw[u >> 1] >> (16 * (u & 1))) & 0xffffu);
                            const float4 y = sY[j];
                            const float ex = y.x - yix, ey = y.y - yiy, ez = y.z - yiz;
                            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                            if (d2 < rs2f && j != selfj) { qbuf[warp][qn][lane] = (unsigned short)j; qn++; }
                        }
                    }
                }
                flush();
            }
            na = next;
            na_off = next_off;
        }

        // combine the warps of a group (exact integer sums) and write; rows
        // are indexed by the rank r.  The red rows of the later splits
        // ((nsplit - 1) x nti <= 96 rows of 56 bytes) fit in sY, which no
        // warp reads any more.
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
            // the warps of a group hold partial sums of the same particles:
            // the later splits hand theirs over by plain stores, split 0 adds
            // them and writes the particle
            static_assert(3 * 32 * 14 * sizeof(int) <= kStageCap * sizeof(float4), "split rows must fit in sY");
            int (*red)[14] = reinterpret_cast<int (*)[14]>(&sY[0]);
            if (ivalid && jsplit > 0) {
                int* d = red[(jsplit - 1) * nti + r];
                d[0] = acc.f[0].h; d[1] = acc.f[0].l; d[2] = acc.f[1].h; d[3] = acc.f[1].l;
                d[4] = acc.f[2].h; d[5] = acc.f[2].l; d[6] = acc.t[0].h; d[7] = acc.t[0].l;
                d[8] = acc.t[1].h; d[9] = acc.t[1].l; d[10] = acc.t[2].h; d[11] = acc.t[2].l;
                d[12] = acc.nf; d[13] = acc.nt;
            }
            const bool any_big = __syncthreads_or(ivalid && acc.used_big);
            if (ivalid && jsplit == 0) {
                int sm[14] = {acc.f[0].h, acc.f[0].l, acc.f[1].h, acc.f[1].l, acc.f[2].h, acc.f[2].l,
                              acc.t[0].h, acc.t[0].l, acc.t[1].h, acc.t[1].l, acc.t[2].h, acc.t[2].l, acc.nf, acc.nt};
                for (int q = 1; q < nsplit; q++) {
                    const int* d = red[(q - 1) * nti + r];
#pragma unroll
                    for (int c = 0; c < 14; c++) sm[c] += d[c];
                }
                const int p = pi;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    SplitAcc f; f.h = sm[2 * a]; f.l = sm[2 * a + 1];
                    SplitAcc t; t.h = sm[6 + 2 * a]; t.l = sm[6 + 2 * a + 1];
                    long long fb = 0, tb = 0;
                    if (any_big) {
                        fb = __ldcg(&v.Fbig[(size_t)a * N + p]);
                        tb = __ldcg(&v.Fbig[(size_t)(3 + a) * N + p]);
                        v.Fbig[(size_t)a * N + p] = 0; v.Fbig[(size_t)(3 + a) * N + p] = 0;
                    }
                    v.F[a * N + p] = f.finish(sm[12]) + fb;
                    v.T[a * N + p] = t.finish(sm[13]) + tb;
                }
            }
        } else {
            long long (*red64)[6] = reinterpret_cast<long long (*)[6]>(&sY[0]);
            for (int q = tid; q < kPairThreads * 6; q += kPairThreads) (&red64[0][0])[q] = 0;
            __syncthreads();
            if (ivalid)
                for (int a = 0; a < 3; a++) {
                    atomicAdd((unsigned long long*)&red64[r][a], (unsigned long long)acc.F(a));
                    atomicAdd((unsigned long long*)&red64[r][3 + a], (unsigned long long)acc.Tq(a));
                }
            __syncthreads();
            if (tid < nti) {
                const int p = __float_as_int(v.mor[it0 + tid].w);   // slot of rank tid
                for (int a = 0; a < 3; a++) { v.F[a * N + p] = red64[tid][a]; v.T[a * N + p] = red64[tid][3 + a]; }
            }
        }
        if (ENERGY) {
            // per-particle energies to fixed point, exact integer sums per instance
            long long eu = 0, ew = 0;
            if (ivalid) {
                eu = __double2ll_rn(up * 4294967296.0);
                ew = __double2ll_rn(vir * 4294967296.0);
            }
            for (int off = 16; off; off >>= 1) {
                eu += __shfl_xor_sync(0xffffffffu, eu, off);
                ew += __shfl_xor_sync(0xffffffffu, ew, off);
            }
            if (lane == 0) {
                atomicAdd((unsigned long long*)&energy[b * 8 + 0], (unsigned long long)eu);
                atomicAdd((unsigned long long*)&energy[b * 8 + 4], (unsigned long long)ew);
            }
        }
        __syncthreads();
    }
}

// ================================================================ split pair path
// The quad loop in two launches: a per-cell search that lists, for every
// particle, the staged particles of its neighbouring cells within its
// type-pair cutoff (+ two skins + a rounding band), and an evaluation with
// one thread per particle over its list, which takes the exact inclusion
// decision and the pair terms.  The search keeps only what the filter needs
// (no evaluation, queues or combine), so it runs with more resident warps;
// the evaluation has no barriers and full lanes.  Forces are the same exact
// integer sums as in the one-launch kernel, whatever order the list holds.
//
// List entry: (row << 26) | q, where q indexes the rank-ordered mirrors and
// row is the neighbouring cell's place in the row of the particle's cell,
// whose exact offset c_l - c_k the search writes to rowoff.  Lists hold
// kListCap entries per particle (t-major: entry t of particle q at t N + q);
// further entries go to an overflow list evaluated with integer atomics.
constexpr int kSearchStage = 768;
constexpr int kListCap = 32;
constexpr int kRowShift = 26;

struct SNbr {
    int base, cnt, start, row;
    int ox, oy, oz;
};

// Eight CTAs per SM (the shared-memory limit): 0.833 against 0.863 ms at seven.
// MP (band-3 or glycophorin in the batch): the staged particles carry three
// partner classes (lipid 0, cytoskeleton 1, bilayer protein 2) and each
// particle culls them at its own cutoff for that class, so that a lipid's
// list is not widened to the cutoff of its widest protein pair.
template <bool MP>
__global__ void __launch_bounds__(kPairThreads, 8)
    k_pair_search(View v, int* __restrict__ nlist, int* __restrict__ ncnt, int cap, int2* __restrict__ ovf,
                  int* __restrict__ novf, int ovf_cap, int4* __restrict__ rowoff) {
    // sY: staged mirrors (int4 by the bulk copy), then in the tangent frame
    //     (FP32), w = 0 for a bilayer particle and 1 for a cytoskeleton protein
    // sQ: the list entry of each staged particle
    // cand: per warp, the byte offsets (16 j) in sY of the culled candidates
    __shared__ alignas(16) float4 sY[kSearchStage];
    __shared__ int sQ[kSearchStage];
    __shared__ alignas(16) unsigned short cand[kPairThreads / 32][kSearchStage];
    // each lane's own particle's position in its warp's candidate list (the
    // self pair is removed once per 32 candidates instead of per test)
    __shared__ unsigned short spos[kPairThreads / 32][32];
    __shared__ SNbr nb[kMaxNbr];
    __shared__ int s_cnt[kPairThreads];
    __shared__ unsigned long long bar;
    __shared__ int s_nstage, s_next, s_next_off, s_self, s_self_lo, s_self_hi, s_total;

    const int k = blockIdx.x;
    const int b = find_inst(v.inst_k0, v.B, k);
    const Inst& I = v.inst[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cs = v.cell_start[k], ce = v.cell_start[k + 1];
    const AdjDesc* __restrict__ row = v.adjd + (size_t)k * kAdjRow;
    const int a1 = min(v.adjn[k], kAdjRow);
    const size_t N = v.N;
    const float sk = 2.0f * I.skinf + kFilterBand;
    const float rsb = I.rsf + sk, rs2f = rsb * rsb;
    const float cw = sqrtf(I.rc2f_wca) + sk, cp = sqrtf(I.rc2f_pp) + sk;
    unsigned phase = 0;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();

    for (int it0 = cs; it0 < ce; it0 += kPairThreads) {
        const int nti = min(kPairThreads, ce - it0);
        const int groups = (nti + 31) >> 5;
        const int nsplit = (groups == 1) ? 4 : (groups == 2 ? 2 : 1);
        const int igrp = warp % groups;
        const int jsplit = warp / groups;
        const bool wactive = jsplit < nsplit;
        const int gs = (nti + groups - 1) / groups;
        s_cnt[tid] = 0;

        auto issue = [&](const int na, const int na_off) {
            if (warp == 0) {
                const int nn = na + lane;
                const bool has = nn < a1;
                int l = 0, st = 0, c = 0;
                AdjDesc d;
                if (has) {
                    d = row[nn];
                    l = d.cell;
                    st = d.start;
                    c = d.cnt;
                    // each row's exact offset, written where the row is first
                    // staged (lane 0 of a pass that continues a split row
                    // was written in the pass before)
                    if (it0 == cs && !(lane == 0 && na_off > 0))
                        rowoff[(size_t)k * kAdjRow + nn] = make_int4(d.ox, d.oy, d.oz, 0);
                    if (lane == 0) { st += na_off; c -= na_off; }
                }
                int incl = c;
                for (int off = 1; off < 32; off <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, off);
                    if (lane >= off) incl += t;
                }
                const int excl = incl - c;
                const bool fits = has && incl <= kSearchStage;
                const bool part = has && excl < kSearchStage && incl > kSearchStage;
                const unsigned fm = __ballot_sync(0xffffffffu, fits), pm = __ballot_sync(0xffffffffu, part);
                const int m = __popc(fm) + (pm ? 1 : 0);
                const bool staged = fits || part;
                const int take = part ? kSearchStage - excl : c;
                if (staged) {
                    SNbr inf;
                    inf.base = excl; inf.cnt = take; inf.start = st; inf.row = nn;
                    inf.ox = d.ox; inf.oy = d.oy; inf.oz = d.oz;
                    nb[lane] = inf;
                }
                const unsigned selfm = __ballot_sync(0xffffffffu, staged && l == k);
                const int total = __shfl_sync(0xffffffffu, excl + take, max(m - 1, 0));
                int nxt = na + __popc(fm), nxo = 0;
                if (pm) {
                    const int p = __ffs(pm) - 1;
                    const int ex_p = __shfl_sync(0xffffffffu, excl, p);
                    nxt = na + p;
                    nxo = (p == 0 ? na_off : 0) + (kSearchStage - ex_p);
                }
                int slo = -1, shi = -1, sb = 0;
                {
                    const int p = selfm ? __ffs(selfm) - 1 : 0;
                    const int ex_p = __shfl_sync(0xffffffffu, excl, p);
                    const int tk_p = __shfl_sync(0xffffffffu, take, p);
                    if (selfm) {
                        slo = ex_p;
                        shi = ex_p + tk_p;
                        sb = ex_p - ((p == 0) ? na_off : 0);
                    }
                }
                if (lane == 0) {
                    s_nstage = m;
                    s_total = m > 0 ? total : 0;
                    s_next = nxt;
                    s_next_off = nxo;
                    s_self = sb; s_self_lo = slo; s_self_hi = shi;
                }
                if (m > 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    if (lane == 0) mbar_expect_tx(&bar, (unsigned)total * 16u + v.extra_tx);
                    __syncwarp();
                    if (staged && take > 0) bulk_g2s(&sY[excl], v.mqr + st, take * 16u, &bar);
                }
            }
        };
        if (0 < a1) issue(0, 0);

        const float4 cn = v.cnorm[k];
        const Frame F = tangent_frame(cn.x, cn.y, cn.z);
        const int r = igrp * gs + lane;
        const bool ivalid = wactive && lane < gs && r < nti;
        int ti = 0;
        float yix = 1.0e18f, yiy = 1.0e18f, yiz = 1.0e18f;
        if (ivalid) {
            const int4 qi = v.mqr[it0 + r];
            ti = qi.w & 0xff;
            F.apply(qi.x * kMirrorUnit, qi.y * kMirrorUnit, qi.z * kMirrorUnit, yix, yiy, yiz);
        }
        // squared search radius for a bilayer and for a cytoskeleton partner
        // (for a bilayer particle the widest cutoff of its species; with MP
        // the lipid partners' and the bilayer proteins' apart)
        const bool bi = bilayer(ti);
        const int si = species(ti);
        const float cl = (MP ? I.mm_rcp[3 * si] : I.mm_rcf[si]) + sk;
        const float cutL = bi ? cl * cl : cw * cw;
        const float cutP = bi ? cw * cw : cp * cp;
        const float cutD = cutP - cutL;
        // MP: the cutoff of a partner of class c in {0, 1, 2} as
        // cutL + c (qa + c qb), through cutP at c = 1 and cutM at c = 2
        float qa = cutD, qb = 0.f;
        if (MP) {
            const float cm = fmaxf(I.mm_rcp[3 * si + 1], I.mm_rcp[3 * si + 2]) + sk;
            const float cutM = bi ? cm * cm : cw * cw;
            qb = 0.5f * (cutM - cutL) - cutD;
            qa = cutD - qb;
        }
        // the group box's cull radius: the search cutoff, or for a group
        // without bilayer particles (a protein cell) the larger of its two
        // cutoffs
        const bool glip = __any_sync(0xffffffffu, ivalid && bi);
        const float rcull2 = glip ? rs2f : fmaxf(cw, cp) * fmaxf(cw, cp);
        float blo[3] = {ivalid ? yix : 3.0e38f, ivalid ? yiy : 3.0e38f, ivalid ? yiz : 3.0e38f};
        float bhi[3] = {ivalid ? yix : -3.0e38f, ivalid ? yiy : -3.0e38f, ivalid ? yiz : -3.0e38f};
        for (int a = 0; a < 3; a++)
            for (int off = 16; off; off >>= 1) {
                blo[a] = fminf(blo[a], __shfl_xor_sync(0xffffffffu, blo[a], off));
                bhi[a] = fmaxf(bhi[a], __shfl_xor_sync(0xffffffffu, bhi[a], off));
            }
        const int qi_idx = it0 + r;

        bool first_pass = true;
        for (int na = 0, na_off = 0; na < a1;) {
            if (!first_pass) {
                __syncthreads();
                issue(na, na_off);
            }
            first_pass = false;
            __syncthreads();
            const int m = s_nstage;
            const int total = s_total;
            const int next = s_next, next_off = s_next_off;
            if (m == 0) { na = next; na_off = next_off; continue; }
            const int sself = s_self, sslo = s_self_lo, sshi = s_self_hi;
            int selfj = (sslo >= 0 && ivalid) ? sself + (it0 + r - cs) : -1;
            if (selfj < sslo || selfj >= sshi) selfj = -1;
            bool ok = mbar_wait_bounded(&bar, phase, v.status, v.wait_polls);
            if (__syncthreads_or(!ok)) {
                if (ok == false) mbar_wait_bounded(&bar, phase, v.status, v.wait_polls);
                return;
            }
            phase ^= 1u;
            // staged particles into the cell's frame (exact) and the tangent
            // frame (FP32), with their list entries
            for (int q = 0; q < m; q++) {
                const SNbr inf = nb[q];
                for (int j = inf.base + tid; j < inf.base + inf.cnt; j += kPairThreads) {
                    const int4 rj = reinterpret_cast<const int4*>(sY)[j];
                    const int x = (int)((unsigned)rj.x + (unsigned)inf.ox);
                    const int y = (int)((unsigned)rj.y + (unsigned)inf.oy);
                    const int z = (int)((unsigned)rj.z + (unsigned)inf.oz);
                    float4 w;
                    F.apply(x * kMirrorUnit, y * kMirrorUnit, z * kMirrorUnit, w.x, w.y, w.z);
                    const int tj = rj.w & 0xff;
                    w.w = MP ? (tj == kLipid ? 0.0f : (bilayer(tj) ? 2.0f : 1.0f)) : (bilayer(tj) ? 0.0f : 1.0f);
                    sY[j] = w;
                    sQ[j] = (inf.row << kRowShift) | (inf.start + (j - inf.base));
                }
            }
            __syncthreads();

            if (wactive) {
                int cnt = 0;
                spos[warp][lane] = 0xffffu;
                __syncwarp();
                // staged index of lane 0's own particle (own cell, this pass)
                const int self0 = sself + (it0 + igrp * gs - cs);
                for (int c0 = 0; c0 < total; c0 += nsplit * 32) {
                    const int j = c0 + lane * nsplit + jsplit;
                    bool in = false;
                    if (j < total) {
                        const float4 y = sY[j];
                        const float ex = fmaxf(fmaxf(blo[0] - y.x, y.x - bhi[0]), 0.f);
                        const float ey = fmaxf(fmaxf(blo[1] - y.y, y.y - bhi[1]), 0.f);
                        const float ez = fmaxf(fmaxf(blo[2] - y.z, y.z - bhi[2]), 0.f);
                        in = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < rcull2;
                    }
                    const unsigned bal = __ballot_sync(0xffffffffu, in);
                    if (in) {
                        const int at = cnt + __popc(bal & ((1u << lane) - 1u));
                        cand[warp][at] = (unsigned short)(j << 4);   // byte offset of sY[j]
                        // the own particle of lane t of this group
                        const int t = j - self0;
                        if (sslo >= 0 && j >= sslo && j < sshi && t >= 0 && t < gs) spos[warp][t] = (unsigned short)at;
                    }
                    cnt += __popc(bal);
                }
                // pad to a multiple of 32 with a valid staged index
                if (cnt + lane < ((cnt + 31) & ~31)) cand[warp][cnt + lane] = 0;
                __syncwarp();
                const int sp = selfj >= 0 ? (int)spos[warp][lane] : -1;   // 0xffff: not in this warp's list
                // every lane tests the same 32 candidates (broadcast reads)
                // into a bit mask, then writes its hits; the padding of the
                // candidate list past cnt is never read as a hit
                static_assert(kSearchStage % 32 == 0, "candidate lists are read 32 at a time");
                static_assert(kSearchStage * 16 <= 65536, "candidate byte offsets fit 16 bits");
                for (int c0 = 0; c0 < cnt; c0 += 32) {
                    unsigned hits = 0u;
#pragma unroll
                    for (int h = 0; h < 4; h++) {
                        const uint4 c8 = *reinterpret_cast<const uint4*>(&cand[warp][c0 + 8 * h]);
                        const unsigned cw8[4] = {c8.x, c8.y, c8.z, c8.w};
#pragma unroll
                        for (int u = 0; u < 8; u++) {
                            const unsigned off = (cw8[u >> 1] >> (16 * (u & 1))) & 0xffffu;
                            const float4 y = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(sY) + off);
                            const float ex = y.x - yix, ey = y.y - yiy, ez = y.z - yiz;
                            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                            const float cut = MP ? fmaf(y.w, fmaf(y.w, qb, qa), cutL) : fmaf(y.w, cutD, cutL);
                            if (d2 < cut) hits |= 1u << (8 * h + u);
                        }
                    }
                    if (cnt - c0 < 32) hits &= (1u << (cnt - c0)) - 1u;
                    if ((unsigned)(sp - c0) < 32u) hits &= ~(1u << (sp - c0));
                    while (hits) {
                        const int u = __ffs(hits) - 1;
                        hits &= hits - 1u;
                        const int e = sQ[cand[warp][c0 + u] >> 4];
                        const int pos = atomicAdd(&s_cnt[r], 1);
                        if (pos < cap) {
                            nlist[(size_t)pos * N + qi_idx] = e;
                        } else {
                            const int o = atomicAdd(novf, 1);
                            if (o < ovf_cap) ovf[o] = make_int2(qi_idx, e);
                            else atomicOr(v.status, kStatusListOverflow);
                        }
                    }
                }
            }
            na = next;
            na_off = next_off;
        }
        __syncthreads();
        if (tid < nti) ncnt[it0 + tid] = s_cnt[tid];
        __syncthreads();
    }
}

// One listed pair: exact integer displacement (2^-26 sigma), the type-pair
// cutoff decided in FP32 outside a 1e-6 sigma band and in FP64 inside it,
// bonded exclusions, then the FP32 pair terms.  Returns false when the pair
// does not interact.
template <int Z, bool S0>
__device__ inline bool listed_pair(const View& v, const Inst& I, int zc, int pi, int ti, int4 qi, float4 oi, int4 mj,
                                   float4 oj, int4 o, float ll_lo, float ll_hi, float w_lo, float w_hi, float p_lo,
                                   float p_hi, float& fx, float& fy, float& fz, float& tx, float& ty, float& tz) {
    const int pj = __float_as_int(oj.w);
    const int tj = mj.w & 0xff;
    int m;
    const int cls = pair_class(ti, tj, m);
    const bool ll = cls == 0;
    const int dxq = (int)((unsigned)mj.x + (unsigned)o.x - (unsigned)qi.x);
    const int dyq = (int)((unsigned)mj.y + (unsigned)o.y - (unsigned)qi.y);
    const int dzq = (int)((unsigned)mj.z + (unsigned)o.z - (unsigned)qi.z);
    const float dx = (float)dxq * kMirrorUnit, dy = (float)dyq * kMirrorUnit, dz = (float)dzq * kMirrorUnit;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float lo = cls == 0 ? (I.has_mp ? I.mm_lo[m] : ll_lo) : (cls == 1 ? w_lo : p_lo);
    const float hi = cls == 0 ? (I.has_mp ? I.mm_hi[m] : ll_hi) : (cls == 1 ? w_hi : p_hi);
    if (r2 >= hi) return false;
    bool in = r2 < lo;
    if (!in) in = exact_inside(v, I, pi, pj, cls, m);
    if (in && cls != 0 && is_excluded(v, I, v.id[pi], v.id[pj], pj)) in = false;
    if (!in) return false;
    if (ll && I.has_mp)
        lipid_dispatch<float, S0, LipK>(LipK(I, m), dx, dy, dz, r2, oi.x, oi.y, oi.z, oj.x, oj.y, oj.z, fx, fy, fz, tx,
                                        ty, tz, zc, (float*)nullptr);
    else if (ll)
        lipid_dispatch<float, S0>(I, dx, dy, dz, r2, oi.x, oi.y, oi.z, oj.x, oj.y, oj.z, fx, fy, fz, tx, ty, tz, zc,
                                  (float*)nullptr);
    else
        wca_terms<float>(I, cls == 2, dx, dy, dz, r2, fx, fy, fz);
    return true;
}

// The FP32 constants of the pair terms, held in registers by the evaluation.
struct PairC {
    float eps, rmin, mu, s0, aw, eps2z_aw, eps_wca, sig_wca, sig_pp;
    int zeta;
    float ll_lo, ll_hi, w_lo, w_hi, p_lo, p_hi;   // squared cutoffs -+ the FP64 decision band
    __device__ explicit PairC(const Inst& I)
        : eps(I.eps), rmin(I.rmin), mu(I.mu), s0(I.s0), aw(I.aw), eps2z_aw(I.eps2z_aw), eps_wca(I.eps_wca),
          sig_wca(I.sig_wca), sig_pp(I.sig_pp), zeta(I.zeta) {
        const float rcl = sqrtf(I.rc2f_ll), rcw = sqrtf(I.rc2f_wca), rcp = sqrtf(I.rc2f_pp);
        ll_lo = (rcl - kCutBand) * (rcl - kCutBand); ll_hi = (rcl + kCutBand) * (rcl + kCutBand);
        w_lo = (rcw - kCutBand) * (rcw - kCutBand); w_hi = (rcw + kCutBand) * (rcw + kCutBand);
        p_lo = (rcp - kCutBand) * (rcp - kCutBand); p_hi = (rcp + kCutBand) * (rcp + kCutBand);
    }
};

// One particle's list (the thread of rank q): the listed particles' mirrors
// read from global memory (L1/L2), the constants of the pair terms in
// registers, the force and torque summed as exact split integers; terms of
// 1000 or more go to the int64 side array (big = true).
// MP: the batch holds band-3 or glycophorin, whose pairs take the constants
// of their bilayer species pair (the lipid-only instantiation tests the
// lipid type alone).
template <int Z, bool S0, bool MP = false>
__device__ __forceinline__ void eval_list(const View& v, int q, const int* __restrict__ nlist,
                                          const int* __restrict__ ncnt, int cap, const int4* __restrict__ rowoff,
                                          SplitAcc af[3], SplitAcc at[3], int& nterm, bool& big, int& pi_out) {
    const size_t N = v.N;
    const int4 qi = v.mqr[q];
    const float4 oi = v.mor[q];
    const int pi = __float_as_int(oi.w);
    pi_out = pi;
    const int ti = qi.w & 0xff;
    const int k = v.cell[pi];
    const int b = find_inst(v.inst_p0, v.B, pi);
    const Inst& I = v.inst[b];
    const PairC C(I);
    const int zc = (Z > 0) ? Z : C.zeta;
    const int4* __restrict__ ro = rowoff + (size_t)k * kAdjRow;
    const int n = min(ncnt[q], cap);
    // a particle without bonds has no excluded pair: its list skips the test
    // (the lipid-only instantiation runs only when no bilayer particle has a
    // bond, so that only pairs of cytoskeleton proteins can be excluded)
    const bool ibond = (qi.w & kMirrorBonded) != 0;
    for (int a = 0; a < 3; a++) { af[a].zero(); at[a].zero(); }
    nterm = 0;
    big = false;
    // the next list entry is in flight while a pair is evaluated; the
    // mirrors are read through the read-only data path
    int e_next = n > 0 ? __ldcs(nlist + q) : 0;
    for (int t = 0; t < n; t++) {
        const int e = e_next;
        if (t + 1 < n) e_next = __ldcs(nlist + (size_t)(t + 1) * N + q);
        const int qj = e & ((1 << kRowShift) - 1);
        const int4 o = __ldg(ro + ((unsigned)e >> kRowShift));
        const int4 mj = __ldg(v.mqr + qj);
        const float4 oj = __ldg(v.mor + qj);
        const int tj = mj.w & 0xff;
        int m = 0;
        int cls;
        if constexpr (MP) {
            cls = pair_class(ti, tj, m);
        } else {
            const bool l2 = (ti == kLipid) && (tj == kLipid);
            cls = l2 ? 0 : ((ti == kLipid || tj == kLipid) ? 1 : 2);
        }
        const bool ll = cls == 0;
        const int dxq = (int)((unsigned)mj.x + (unsigned)o.x - (unsigned)qi.x);
        const int dyq = (int)((unsigned)mj.y + (unsigned)o.y - (unsigned)qi.y);
        const int dzq = (int)((unsigned)mj.z + (unsigned)o.z - (unsigned)qi.z);
        const float dx = (float)dxq * kMirrorUnit, dy = (float)dyq * kMirrorUnit, dz = (float)dzq * kMirrorUnit;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        // (a lipid pair, m = 0, keeps the constants held in registers)
        const bool tab = MP && m != 0;
        const float lo = cls == 0 ? (tab ? I.mm_lo[m] : C.ll_lo) : (cls == 1 ? C.w_lo : C.p_lo);
        const float hi = cls == 0 ? (tab ? I.mm_hi[m] : C.ll_hi) : (cls == 1 ? C.w_hi : C.p_hi);
        if (r2 >= hi) continue;
        if (!(r2 < lo) && !exact_inside(v, I, pi, __float_as_int(oj.w), cls, m)) continue;
        if ((MP ? (cls != 0 && ibond) : cls == 2) &&
            is_excluded(v, I, v.id[pi], v.id[__float_as_int(oj.w)], __float_as_int(oj.w)))
            continue;
        float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (ll && MP) {
            // one code path for every species pair (lanes with different
            // pairs stay converged): the pair's constants picked first
            PairC Cm = C;
            if (tab) {
                Cm.eps = I.mm_eps[m];
                Cm.aw = I.mm_aw[m];
                Cm.eps2z_aw = I.mm_e2za[m];
            }
            if (zc == 4)
                lipid_terms_f<4, S0>(Cm, dx, dy, dz, r2, oi.x, oi.y, oi.z, oj.x, oj.y, oj.z, f[0], f[1], f[2], f[3],
                                     f[4], f[5]);
            else
                lipid_terms_f<0, true>(Cm, dx, dy, dz, r2, oi.x, oi.y, oi.z, oj.x, oj.y, oj.z, f[0], f[1], f[2],
                                       f[3], f[4], f[5]);
        } else if (ll) {
            if (zc == 4)
                lipid_terms_f<4, S0>(C, dx, dy, dz, r2, oi.x, oi.y, oi.z, oj.x, oj.y, oj.z, f[0], f[1], f[2], f[3],
                                     f[4], f[5]);
            else
                lipid_terms_f<0, true>(C, dx, dy, dz, r2, oi.x, oi.y, oi.z, oj.x, oj.y, oj.z, f[0], f[1], f[2], f[3],
                                       f[4], f[5]);
        } else {
            const float sig = cls == 2 ? C.sig_pp : C.sig_wca;
            const float s2 = sig * sig / r2;
            const float s6 = s2 * s2 * s2;
            const float s12 = s6 * s6;
            const float fr = 4.0f * C.eps_wca * (12.0f * s12 - 6.0f * s6) / r2;
            f[0] = -fr * dx; f[1] = -fr * dy; f[2] = -fr * dz;
        }
        const float mag = fabsf(f[0]) + fabsf(f[1]) + fabsf(f[2]) + fabsf(f[3]) + fabsf(f[4]) + fabsf(f[5]);
        if (mag < 1000.0f) {
            for (int a = 0; a < 3; a++) { af[a].add(f[a]); at[a].add(f[3 + a]); }
            nterm++;
        } else {
            // terms of 1000 or more go to the int64 side array (exact, rare)
            if (!(mag < kMaxTerm)) flag_inst(v, I, (mag == mag) ? kStatusPairForceRange : kStatusNaN);
            for (int a = 0; a < 6; a++)
                atomicAdd((unsigned long long*)&v.Fbig[(size_t)a * N + pi],
                          (unsigned long long)__float2ll_rn(f[a] * 4294967296.0f));
            big = true;
        }
    }
}

// Evaluation: one thread per particle (rank order) over its list (see
// eval_list).  (Measured on the 4M cell: evaluating from mirrors staged in
// shared memory per cell, with each list split over two or four threads,
// took 1.31 ms against 1.06 ms for this kernel.)
// Compiled for 5 and 7 CTAs per SM (the autotuner's second dimension):
// seven (72 registers, a few spilled) hide more of the gathers' latency than
// five without spills, 0.785 against 0.857 ms on the 4M cell.
// MP: the batch holds band-3 or glycophorin (eval_list).
template <int Z, bool S0, int MINB, bool MP = false>
__global__ void __launch_bounds__(128, MINB)
    k_pair_eval(View v, const int* __restrict__ nlist, const int* __restrict__ ncnt, int cap,
                const int4* __restrict__ rowoff) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= v.N) return;
    const size_t N = v.N;
    SplitAcc af[3], at[3];
    int nterm, pi;
    bool big;
    eval_list<Z, S0, MP>(v, q, nlist, ncnt, cap, rowoff, af, at, nterm, big, pi);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long fb = 0, tb = 0;
        if (big) {
            fb = __ldcg(&v.Fbig[(size_t)a * N + pi]);
            tb = __ldcg(&v.Fbig[(size_t)(3 + a) * N + pi]);
            v.Fbig[(size_t)a * N + pi] = 0;
            v.Fbig[(size_t)(3 + a) * N + pi] = 0;
        }
        v.F[a * N + pi] = af[a].finish(nterm) + fb;
        v.T[a * N + pi] = at[a].finish(nterm) + tb;
    }
}

// The evaluation of one step with the next step's update in its epilogue:
// each particle's force and torque are complete once its own list is done
// (the bonds, the listed pairs beyond the lists' capacity and the large
// terms were added beforehand to the side array, flagged per particle; the
// volume constraint's pressure is added here), and its B-A-O-A update (with
// the final B of this step) needs nothing else, so the FP64 update of one
// warp overlaps the FP32 pair terms of the others.  The updated state goes
// to the other state buffer (o): the exact inclusion decisions of the other
// threads still read this step's positions.  D: FP64 increments.
template <int Z, bool S0, bool D>
__global__ void __launch_bounds__(128, 4)
    k_pair_eval_step(View v, View o, const int* __restrict__ nlist, const int* __restrict__ ncnt, int cap,
                     const int4* __restrict__ rowoff, unsigned char* __restrict__ sflag,
                     const long long* __restrict__ steps, long long* __restrict__ msum, int* __restrict__ mcnt) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned live = __ballot_sync(0xffffffffu, q < v.N);
    if (q >= v.N) return;
    const size_t N = v.N;
    SplitAcc af[3], at[3];
    int nterm, pi;
    bool big;
    eval_list<Z, S0>(v, q, nlist, ncnt, cap, rowoff, af, at, nterm, big, pi);
    const bool side = big || sflag[pi];
    long long F[3], Tq[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        long long fb = 0, tb = 0;
        if (side) {
            fb = __ldcg(&v.Fbig[(size_t)a * N + pi]);
            tb = __ldcg(&v.Fbig[(size_t)(3 + a) * N + pi]);
            v.Fbig[(size_t)a * N + pi] = 0;
            v.Fbig[(size_t)(3 + a) * N + pi] = 0;
        }
        F[a] = af[a].finish(nterm) + fb;
        Tq[a] = at[a].finish(nterm) + tb;
    }
    if (side) sflag[pi] = 0;
    const Inst& I = v.inst[find_inst(v.inst_p0, v.B, pi)];
    if (I.vol_on && bilayer(v.type[pi])) {
        // the volume constraint's pressure on the lipid's area element, as
        // the constraint's own launch computes it
        const double V = I.a3 * volume_of(__ldg(&v.vol[2 * (&I - v.inst)]), __ldg(&v.vol[2 * (&I - v.inst) + 1]));
        const float pa = (float)(-I.kv * (V - I.v0) * I.avol);
        for (int a = 0; a < 3; a++) {
            const float f = pa * (ll_to_float(v.nq[a * N + pi]) * (float)kGridInv);
            if (!(fabsf(f) < kMaxTerm)) flag_inst(v, I, f == f ? kStatusPairForceRange : kStatusNaN);
            else F[a] += __float2ll_rn(f * 4294967296.0f);
        }
    }
    for (int a = 0; a < 3; a++) { v.F[a * N + pi] = F[a]; v.T[a * N + pi] = Tq[a]; }
    __syncwarp(live);
    if (D) baoa_d_body<true>(v, o, pi, F, Tq, steps, msum, mcnt, live, true);
    else baoa_body<float, true>(v, o, pi, F, Tq, steps, msum, mcnt, live, true);
}

// Listed pairs beyond kListCap: the same terms, added to F and T by 64-bit
// integer atomics (each term rounded to 2^-32 exactly as the split sums do,
// so the totals are the same integers).
// sflag (nullable): add to the side array instead, and flag the particle
// (the evaluation with the update in its epilogue collects it).
template <int Z, bool S0>
__global__ void k_pair_overflow(View v, const int2* __restrict__ ovf, const int* __restrict__ novf, int ovf_cap,
                                const int4* __restrict__ rowoff, unsigned char* __restrict__ sflag) {
    const int n = min(*novf, ovf_cap);
    const size_t N = v.N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const int2 pr = ovf[x];
        const int q = pr.x, e = pr.y;
        const int4 qi = v.mqr[q];
        const float4 oi = v.mor[q];
        const int pi = __float_as_int(oi.w);
        const int ti = qi.w & 0xff;
        const int k = v.cell[pi];
        const int b = find_inst(v.inst_p0, v.B, pi);
        const Inst& I = v.inst[b];
        const int zc = (Z > 0) ? Z : I.zeta;
        const float rcl = sqrtf(I.rc2f_ll), rcw = sqrtf(I.rc2f_wca), rcp = sqrtf(I.rc2f_pp);
        const int qj = e & ((1 << kRowShift) - 1);
        const int4 o = rowoff[(size_t)k * kAdjRow + ((unsigned)e >> kRowShift)];
        float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (!listed_pair<Z, S0>(v, I, zc, pi, ti, qi, oi, v.mqr[qj], v.mor[qj], o, (rcl - kCutBand) * (rcl - kCutBand),
                                (rcl + kCutBand) * (rcl + kCutBand), (rcw - kCutBand) * (rcw - kCutBand),
                                (rcw + kCutBand) * (rcw + kCutBand), (rcp - kCutBand) * (rcp - kCutBand),
                                (rcp + kCutBand) * (rcp + kCutBand), f[0], f[1], f[2], f[3], f[4], f[5]))
            continue;
        const float mag = fabsf(f[0]) + fabsf(f[1]) + fabsf(f[2]) + fabsf(f[3]) + fabsf(f[4]) + fabsf(f[5]);
        if (!(mag < kMaxTerm)) flag_inst(v, I, (mag == mag) ? kStatusPairForceRange : kStatusNaN);
        long long* const Ft = sflag ? v.Fbig : v.F;
        long long* const Tt = sflag ? v.Fbig + 3 * N : v.T;
        for (int a = 0; a < 3; a++) {
            atomicAdd((unsigned long long*)&Ft[a * N + pi], (unsigned long long)__float2ll_rn(f[a] * 4294967296.0f));
            atomicAdd((unsigned long long*)&Tt[a * N + pi], (unsigned long long)__float2ll_rn(f[3 + a] * 4294967296.0f));
        }
        if (sflag) sflag[pi] = 1;
    }
}

// Harmonic bonds ("Force Evaluation": a list of bonds between proteins is
// maintained): one thread per bond, after the pair kernel wrote F.  The bond
// force is rounded to the 2^-32 grid once and added to both ends with
// opposite signs by 64-bit integer atomics: integer sums do not depend on
// the order, and the result equals evaluating the bond from each end.
// sflag (nullable): add to the side array instead, and flag both ends.
template <typename T, bool ENERGY>
__global__ void k_bonds(View v, long long* __restrict__ energy /* [B][8] */, unsigned char* __restrict__ sflag) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    int b = -1;
    long long eb = 0, ew = 0;
    if (q < v.nbond) {
        b = v.binst[q];
        const Inst& I = v.inst[b];
        const size_t N = v.N;
        const int2 e = v.bij[q];
        const int pi = v.slot_of_id[e.x], pj = v.slot_of_id[e.y];
        const long long ddx = minimg_q(v.xq[pj] - v.xq[pi], I.boxq[0], I.periodic[0]);
        const long long ddy = minimg_q(v.xq[N + pj] - v.xq[N + pi], I.boxq[1], I.periodic[1]);
        const long long ddz = minimg_q(v.xq[2 * N + pj] - v.xq[2 * N + pi], I.boxq[2], I.periodic[2]);
        T dx, dy, dz, r0, kb;
        if constexpr (sizeof(T) == 4) {
            dx = ll_to_float(ddx) * (float)kGridInv; dy = ll_to_float(ddy) * (float)kGridInv;
            dz = ll_to_float(ddz) * (float)kGridInv;
            const float2 kf = v.bkf[q];
            r0 = kf.x; kb = kf.y;
        } else {
            dx = grid_to_double(ddx); dy = grid_to_double(ddy); dz = grid_to_double(ddz);
            const double2 kd = v.bkd[q];
            r0 = kd.x; kb = kd.y;
        }
        const T r = sqrt(dx * dx + dy * dy + dz * dz);
        const T dr = r - r0;
        const T c = kb * dr / r;
        const T g[3] = {c * dx, c * dy, c * dz};     // force on the first end
        for (int a = 0; a < 3; a++) {
            long long f;
            if constexpr (sizeof(T) == 4) f = __float2ll_rn(g[a] * 4294967296.0f);
            else f = __double2ll_rn(g[a] * 4294967296.0);
            if (!(fabs(g[a]) < (T)kMaxTerm)) flag_inst(v, I, (g[a] == g[a]) ? kStatusPairForceRange : kStatusNaN);
            long long* const Ft = sflag ? v.Fbig : v.F;
            atomicAdd((unsigned long long*)&Ft[a * N + pi], (unsigned long long)f);
            atomicAdd((unsigned long long*)&Ft[a * N + pj], (unsigned long long)(-f));
        }
        if (sflag) { sflag[pi] = 1; sflag[pj] = 1; }
        if (ENERGY) {
            // energy and virial partials in FP64 from the exact displacement
            const double ex = grid_to_double(ddx), ey = grid_to_double(ddy), ez = grid_to_double(ddz);
            const double r2d = ex * ex + ey * ey + ez * ez;
            const double rd = sqrt(r2d);
            const double r0d = (double)r0, kbd = (double)kb;
            const double drd = rd - r0d;
            eb = __double2ll_rn(0.5 * kbd * drd * drd * 4294967296.0);
            ew = __double2ll_rn(-(kbd * drd * rd) * 4294967296.0);
        }
    }
    if (ENERGY) {
        // warp-aggregate per instance, then one atomic per instance and warp
        const unsigned grp = __match_any_sync(0xffffffffu, b);
        long long sb = 0, sw = 0;
        unsigned m = grp;
        while (m) {
            const int src = __ffs(m) - 1;
            m &= m - 1;
            sb += __shfl_sync(grp, eb, src);
            sw += __shfl_sync(grp, ew, src);
        }
        if (b >= 0 && (int)(threadIdx.x & 31) == __ffs(grp) - 1) {
            atomicAdd((unsigned long long*)&energy[b * 8 + 1], (unsigned long long)sb);
            atomicAdd((unsigned long long*)&energy[b * 8 + 4], (unsigned long long)sw);
        }
    }
}

// The pair kernel runs five CTAs per SM only with the whole unified L1 /
// shared memory given to shared memory; ask for that once per process.
template <typename Kern> static void prefer_shared(Kern k) {
    CK(cudaFuncSetAttribute((const void*)k, cudaFuncAttributePreferredSharedMemoryCarveout,
                            (int)cudaSharedmemCarveoutMaxShared));
}
static void prefer_shared_all() {
    static std::once_flag once;
    std::call_once(once, [] {
        prefer_shared(k_pairs<float, false, true, 0, true>);
        prefer_shared(k_pairs<float, true, false, 4, true>);
        prefer_shared(k_pairs<float, true, false, 4, false>);
        prefer_shared(k_pairs<float, true, false, 0, true>);
        prefer_shared(k_pairs<float, false, false, 4, true>);
        prefer_shared(k_pairs<float, false, false, 4, false>);
        prefer_shared(k_pairs<float, false, false, 0, true>);
        prefer_shared(k_pairs<double, false, true, 0, true>);
        prefer_shared(k_pairs<double, true, false, 0, true>);
        prefer_shared(k_pairs<double, false, false, 0, true>);
    });
}

void Ensemble::alloc_lists() {
    list_cap = kListCap;
    ovf_cap = std::max(N / 4, 4096);
    d_nlist = alloc<int>((size_t)list_cap * N);
    d_ncnt = alloc<int>(N);
    d_novf = alloc<int2>(ovf_cap);
    d_novf_n = alloc<int>(1);
    d_rowoff = alloc<int4>(adj_cap);
    d_sflag = alloc<unsigned char>(N);
    list_valid = false;
}

void Ensemble::launch_pairs(bool energies, bool dump) {
    View v = view();
    if (energies) CK(cudaMemsetAsync(d_energy, 0, sizeof(long long) * 8 * B, stream));
    bool z4 = true, s0z = true;
    for (auto& I : inst_h) { z4 = z4 && I.zeta == 4; s0z = s0z && I.s0_d == 0.0; }
    const dim3 g(Ktot), t(kPairThreads);
    prefer_shared_all();
    if (!force_f64() && !energies && !dump) {
        // split path: neighbour lists (once per cell reorder), evaluation,
        // listed pairs beyond the lists' capacity
        if (!list_valid) {
            tic("pair_search");
            CK(cudaMemsetAsync(d_novf_n, 0, sizeof(int), stream));
            if (any_mp())
                k_pair_search<true><<<g, t, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_novf, d_novf_n, ovf_cap, d_rowoff);
            else
                k_pair_search<false><<<g, t, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_novf, d_novf_n, ovf_cap, d_rowoff);
            launches++;
            CK(cudaGetLastError());
            toc();
            list_valid = true;
        }
        tic("pairs");
        const int ng = (int)((N + 127) / 128);
        // the batch's launch shape: the choice of its largest instance
        int ctas = prm_h[0].eval_ctas, nmax = -1;
        for (int b = 0; b < B; b++)
            if (inst_h[b].n > nmax) { nmax = inst_h[b].n; ctas = prm_h[b].eval_ctas; }
#define ORBC_EVAL(Z, S)                                                                                    \
    do {                                                                                                   \
        if (ctas == 5) k_pair_eval<Z, S, 5><<<ng, 128, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_rowoff); \
        else k_pair_eval<Z, S, 7><<<ng, 128, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_rowoff);          \
    } while (0)
        if (any_mp()) {
            // band-3 or glycophorin present (or a bonded bilayer particle):
            // the evaluation with the bilayer species pairs' constants
            if (z4 && s0z) {
                if (ctas == 5) k_pair_eval<4, false, 5, true><<<ng, 128, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_rowoff);
                else k_pair_eval<4, false, 7, true><<<ng, 128, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_rowoff);
            } else {
                if (ctas == 5) k_pair_eval<0, true, 5, true><<<ng, 128, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_rowoff);
                else k_pair_eval<0, true, 7, true><<<ng, 128, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_rowoff);
            }
            k_pair_overflow<0, true><<<152, 128, 0, stream>>>(v, d_novf, d_novf_n, ovf_cap, d_rowoff, nullptr);
        } else if (z4 && s0z) {
            ORBC_EVAL(4, false);
            k_pair_overflow<4, false><<<152, 128, 0, stream>>>(v, d_novf, d_novf_n, ovf_cap, d_rowoff, nullptr);
        } else if (z4) {
            ORBC_EVAL(4, true);
            k_pair_overflow<4, true><<<152, 128, 0, stream>>>(v, d_novf, d_novf_n, ovf_cap, d_rowoff, nullptr);
        } else {
            ORBC_EVAL(0, true);
            k_pair_overflow<0, true><<<152, 128, 0, stream>>>(v, d_novf, d_novf_n, ovf_cap, d_rowoff, nullptr);
        }
#undef ORBC_EVAL
        launches += 2;
        CK(cudaGetLastError());
        toc();
    } else {
    tic("pairs");
    if (!force_f64()) {
        if (dump) k_pairs<float, false, true, 0, true><<<g, t, 0, stream>>>(v, d_energy, d_dump, d_dump_count, dump_cap);
        else if (energies && z4 && s0z) k_pairs<float, true, false, 4, false><<<g, t, 0, stream>>>(v, d_energy, nullptr, nullptr, 0);
        else if (energies && z4) k_pairs<float, true, false, 4, true><<<g, t, 0, stream>>>(v, d_energy, nullptr, nullptr, 0);
        else if (energies) k_pairs<float, true, false, 0, true><<<g, t, 0, stream>>>(v, d_energy, nullptr, nullptr, 0);
        else if (z4 && s0z) k_pairs<float, false, false, 4, false><<<g, t, 0, stream>>>(v, d_energy, nullptr, nullptr, 0);
        else if (z4) k_pairs<float, false, false, 4, true><<<g, t, 0, stream>>>(v, d_energy, nullptr, nullptr, 0);
        else k_pairs<float, false, false, 0, true><<<g, t, 0, stream>>>(v, d_energy, nullptr, nullptr, 0);
    } else {
        if (dump) k_pairs<double, false, true, 0, true><<<g, t, 0, stream>>>(v, d_energy, d_dump, d_dump_count, dump_cap);
        else if (energies) k_pairs<double, true, false, 0, true><<<g, t, 0, stream>>>(v, d_energy, nullptr, nullptr, 0);
        else k_pairs<double, false, false, 0, true><<<g, t, 0, stream>>>(v, d_energy, nullptr, nullptr, 0);
    }
    launches++;
    toc();
    }
    tic("bonds");
    const int nb = (int)((std::max(nbond, 1) + 255) / 256);
    if (!force_f64()) {
        if (energies) k_bonds<float, true><<<nb, 256, 0, stream>>>(v, d_energy, nullptr);
        else k_bonds<float, false><<<nb, 256, 0, stream>>>(v, d_energy, nullptr);
    } else {
        if (energies) k_bonds<double, true><<<nb, 256, 0, stream>>>(v, d_energy, nullptr);
        else k_bonds<double, false><<<nb, 256, 0, stream>>>(v, d_energy, nullptr);
    }
    launches++;
    CK(cudaGetLastError());
    toc();
    if (!dump) launch_volume(energies);
}

void Ensemble::launch_pairs_step(bool msums) {
    View v = view();
    bool z4 = true, s0z = true;
    for (auto& I : inst_h) { z4 = z4 && I.zeta == 4; s0z = s0z && I.s0_d == 0.0; }
    prefer_shared_all();
    if (!list_valid) {
        tic("pair_search");
        CK(cudaMemsetAsync(d_novf_n, 0, sizeof(int), stream));
        k_pair_search<false><<<Ktot, kPairThreads, 0, stream>>>(v, d_nlist, d_ncnt, list_cap, d_novf, d_novf_n, ovf_cap,
                                                                d_rowoff);
        launches++;
        CK(cudaGetLastError());
        toc();
        list_valid = true;
    }
    tic("pairs_step");
    // what the epilogue cannot compute from a particle's own list goes to
    // the side array first: bonds, listed pairs beyond the lists' capacity;
    // then the constrained volume
    const int nb = (int)((std::max(nbond, 1) + 255) / 256);
    k_bonds<float, false><<<nb, 256, 0, stream>>>(v, d_energy, d_sflag);
    if (z4 && s0z) k_pair_overflow<4, false><<<152, 128, 0, stream>>>(v, d_novf, d_novf_n, ovf_cap, d_rowoff, d_sflag);
    else if (z4) k_pair_overflow<4, true><<<152, 128, 0, stream>>>(v, d_novf, d_novf_n, ovf_cap, d_rowoff, d_sflag);
    else k_pair_overflow<0, true><<<152, 128, 0, stream>>>(v, d_novf, d_novf_n, ovf_cap, d_rowoff, d_sflag);
    launches += 2;
    launch_volume_sum();
    long long* ms = msums ? d_msum : nullptr;
    int* mc = msums ? d_mcnt : nullptr;
    const View o = view_alt();
    const int ng = (int)((N + 127) / 128);
    const bool d = !step_f32();
#define ORBC_EVAL_STEP(Z, S, D) \
    k_pair_eval_step<Z, S, D><<<ng, 128, 0, stream>>>(v, o, d_nlist, d_ncnt, list_cap, d_rowoff, d_sflag, d_step, ms, mc)
    if (z4 && s0z) { if (d) ORBC_EVAL_STEP(4, false, true); else ORBC_EVAL_STEP(4, false, false); }
    else if (z4) { if (d) ORBC_EVAL_STEP(4, true, true); else ORBC_EVAL_STEP(4, true, false); }
    else { if (d) ORBC_EVAL_STEP(0, true, true); else ORBC_EVAL_STEP(0, true, false); }
#undef ORBC_EVAL_STEP
    launches++;
    CK(cudaGetLastError());
    toc();
    swap_state();
    k_step_advance<<<1, 64, 0, stream>>>(d_step, B);
    launches++;
    CK(cudaGetLastError());
    forces_valid = false;   // F and T belong to the positions before the update
}

}  // namespace orbc
