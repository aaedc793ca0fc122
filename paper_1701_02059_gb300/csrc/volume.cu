// Harmonic volume constraint and the upper-rim height map of the membrane
// fluctuation measurement ("Validation and Benchmark", the whole-cell run).
//
// Volume: V = sum over lipids of (a/3) (x_i - c) . n_i (the divergence
// theorem with each lipid's director as its surface normal), U_V =
// k_V (V - V0)^2 / 2, acting as the uniform pressure P = -k_V (V - V0) on
// each lipid's area element: F_i += P a n_i, no torque (a uniform pressure
// has no moment about the element's centre).  Two launches after the pair
// and bond forces: the sum D of (x - c).n (each term split into its 2^-24
// sigma floor and the remainder at 2^-48, two integer sums by atomics, so D
// does not depend on the order; V = (a/3) D in FP64), then the per-lipid
// force rounded to the 2^-32 force grid and added in place.  (x - c).n and the force are FP32 in the
// FP32-force modes and FP64 when every force is FP64.  Both launches touch
// each lipid once and are bound by HBM bandwidth: 49 bytes per lipid for
// the sum (type, x, n), 73 for the force (type, n, F read and written).
//
// Height map: the lipids above z_min inside an annulus about a vertical
// axis, binned on an (x, y) grid; every decision in FP64 with correctly
// rounded operations on the exact state, z summed exactly as two integer
// halves of its 2^-40 grid value.
#include "ensemble.cuh"

namespace orbc {

constexpr int kVolThreads = 256;

template <typename T> __device__ inline T to_sigma(long long q);
template <> __device__ inline float to_sigma<float>(long long q) { return ll_to_float(q) * (float)kGridInv; }
template <> __device__ inline double to_sigma<double>(long long q) { return grid_to_double(q); }

__device__ inline void add2(long long* out, long long h, long long l) {
    if (h) atomicAdd((unsigned long long*)&out[0], (unsigned long long)h);
    if (l) atomicAdd((unsigned long long*)&out[1], (unsigned long long)l);
}

// Sum of per-thread partials into out[2 b], out[2 b + 1]: one butterfly and
// one atomic pair per warp when the warp holds one instance, else per lane.
__device__ inline void warp_flush(long long h, long long l, int b, long long* out) {
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    if (grp == 0xffffffffu) {
        for (int o = 16; o > 0; o >>= 1) {
            h += __shfl_xor_sync(0xffffffffu, h, o);
            l += __shfl_xor_sync(0xffffffffu, l, o);
        }
        if ((threadIdx.x & 31) == 0 && b >= 0) add2(out + 2 * b, h, l);
    } else if (b >= 0) {
        add2(out + 2 * b, h, l);
    }
}

// One lipid's (x - c).n split exactly into its floor at 2^-24 sigma and the
// remainder rounded at 2^-48 (integer sums of both do not depend on the
// order; they wrap harmlessly in int64 as long as the final sum stays below
// 2^39 sigma).  In FP32 the scaled value is an integer already when
// |(x - c).n| >= 1, and the remainder is exact in both precisions.
__device__ inline void split_term(float dn, long long& th, long long& tl) {
    const float s = dn * 16777216.0f, fl = floorf(s);
    th = __float2ll_rn(fl);
    tl = __float2ll_rn((s - fl) * 16777216.0f);
}
__device__ inline void split_term(double dn, long long& th, long long& tl) {
    const double s = dn * kVolUnit, fl = floor(s);
    th = __double2ll_rn(fl);
    tl = __double2ll_rn((s - fl) * kVolUnit);
}

// D = sum over lipids of (x - c).n per instance; V = (a/3) D.  b_only < 0:
// every instance with the constraint on, with its own centre; b_only >= 0:
// that instance alone with the centre given (the volume query, summed into
// out[0..1]).
template <typename T>
__global__ void __launch_bounds__(kVolThreads) k_volume_sum(View v, int b_only, long long xc0, long long xc1,
                                                            long long xc2, long long* __restrict__ out) {
    const size_t N = v.N;
    const int stride = gridDim.x * blockDim.x;
    int cur = -1;
    long long acc_h = 0, acc_l = 0;
    // the loop runs the same number of rounds in every lane of a warp, so
    // that the warp-wide flush below sees all 32 lanes
    const int rounds = (int)((N + stride - 1) / stride);
    for (int r = 0; r < rounds; r++) {
        const int p = r * stride + blockIdx.x * blockDim.x + threadIdx.x;
        int b = -1;
        long long th = 0, tl = 0;
        if (p < (int)N && bilayer(v.type[p])) {
            const int bi = find_inst(v.inst_p0, v.B, p);
            const Inst& I = v.inst[bi];
            if (b_only >= 0 ? bi == b_only : I.vol_on != 0) {
                const long long c[3] = {b_only >= 0 ? xc0 : I.xcq[0], b_only >= 0 ? xc1 : I.xcq[1],
                                        b_only >= 0 ? xc2 : I.xcq[2]};
                T dn = 0;
                for (int a = 0; a < 3; a++)
                    dn += to_sigma<T>(v.xq[a * N + p] - c[a]) * to_sigma<T>(v.nq[a * N + p]);
                if (!(fabs(dn) < (T)kMaxTerm)) flag_inst(v, I, dn == dn ? kStatusPairForceRange : kStatusNaN);
                else split_term(dn, th, tl);
                b = b_only >= 0 ? 0 : bi;
            }
        }
        // flush when this lane's instance changes
        if (b >= 0 && b != cur) {
            if (cur >= 0) add2(out + 2 * cur, acc_h, acc_l);
            cur = b;
            acc_h = 0;
            acc_l = 0;
        }
        acc_h += th;
        acc_l += tl;
    }
    warp_flush(acc_h, acc_l, cur, out);
}

// Constraint forces, added to F in place; with ENERGY the constraint energy
// joins the bond energy.
template <typename T, bool ENERGY>
__global__ void __launch_bounds__(kVolThreads) k_volume_apply(View v, const long long* __restrict__ vol,
                                                              long long* __restrict__ energy /* [B][8] */) {
    const size_t N = v.N;
    const int stride = gridDim.x * blockDim.x;
    int bc = -1;
    T pa = 0;                                      // P a of instance bc
    bool on = false;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < (int)N; p += stride) {
        if (!bilayer(v.type[p])) continue;
        const int b = find_inst(v.inst_p0, v.B, p);
        const Inst& I = v.inst[b];
        if (b != bc) {
            bc = b;
            on = I.vol_on != 0;
            const double V = I.a3 * volume_of(__ldg(&vol[2 * b]), __ldg(&vol[2 * b + 1]));
            pa = (T)(-I.kv * (V - I.v0) * I.avol);
        }
        if (!on) continue;
        for (int a = 0; a < 3; a++) {
            const T f = pa * to_sigma<T>(v.nq[a * N + p]);
            if (!(fabs(f) < (T)kMaxTerm)) {
                flag_inst(v, I, f == f ? kStatusPairForceRange : kStatusNaN);
                continue;
            }
            long long fq;
            if constexpr (sizeof(T) == 4) fq = __float2ll_rn(f * 4294967296.0f);
            else fq = __double2ll_rn(f * 4294967296.0);
            v.F[a * N + p] += fq;
        }
    }
    if (ENERGY && blockIdx.x == 0) {
        for (int b = threadIdx.x; b < v.B; b += blockDim.x) {
            const Inst& I = v.inst[b];
            if (!I.vol_on) continue;
            const double dV = I.a3 * volume_of(vol[2 * b], vol[2 * b + 1]) - I.v0;
            const double u = 0.5 * I.kv * dV * dV;
            if (!(u < 1073741824.0)) {          // 2^30: the 2^-32 sum stays inside int64
                flag_inst(v, I, u == u ? kStatusPairForceRange : kStatusNaN);
                continue;
            }
            atomicAdd((unsigned long long*)&energy[b * 8 + 1], (unsigned long long)__double2ll_rn(u * 4294967296.0));
        }
    }
}

static int volume_grid(int N) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int need = (N + kVolThreads - 1) / kVolThreads;
    return std::max(1, std::min(need, sms * 8));
}

void Ensemble::launch_volume_sum() {
    if (!vol_any) return;
    CK(cudaMemsetAsync(d_vol, 0, sizeof(long long) * 2 * B, stream));
    if (force_f64()) k_volume_sum<double><<<volume_grid(N), kVolThreads, 0, stream>>>(view(), -1, 0, 0, 0, d_vol);
    else k_volume_sum<float><<<volume_grid(N), kVolThreads, 0, stream>>>(view(), -1, 0, 0, 0, d_vol);
    launches++;
    CK(cudaGetLastError());
}

void Ensemble::launch_volume(bool energies) {
    if (!vol_any) return;
    View v = view();
    const int g = volume_grid(N);
    tic("volume");
    CK(cudaMemsetAsync(d_vol, 0, sizeof(long long) * 2 * B, stream));
    if (force_f64()) {
        k_volume_sum<double><<<g, kVolThreads, 0, stream>>>(v, -1, 0, 0, 0, d_vol);
        if (energies) k_volume_apply<double, true><<<g, kVolThreads, 0, stream>>>(v, d_vol, d_energy);
        else k_volume_apply<double, false><<<g, kVolThreads, 0, stream>>>(v, d_vol, d_energy);
    } else {
        k_volume_sum<float><<<g, kVolThreads, 0, stream>>>(v, -1, 0, 0, 0, d_vol);
        if (energies) k_volume_apply<float, true><<<g, kVolThreads, 0, stream>>>(v, d_vol, d_energy);
        else k_volume_apply<float, false><<<g, kVolThreads, 0, stream>>>(v, d_vol, d_energy);
    }
    launches += 2;
    CK(cudaGetLastError());
    toc();
}

void Ensemble::set_volume(int b, double kv, double v0, double area, const double xc[3]) {
    Inst& I = inst_h[b];
    I.vol_on = kv > 0.0;
    I.kv = kv;
    I.v0 = v0;
    I.avol = area;
    I.a3 = area / 3.0;
    for (int a = 0; a < 3; a++) I.xcq[a] = llrint(xc[a] * kGrid);
    CK(cudaMemcpyAsync(d_inst + b, &I, sizeof(Inst), cudaMemcpyHostToDevice, stream));
    CK(cudaStreamSynchronize(stream));
    bool any = false;
    for (const Inst& J : inst_h) any = any || J.vol_on;
    if (any != vol_any) {
        // the captured step holds the volume launches or not
        for (int q = 0; q < 2; q++)
            if (graph_[q]) { cudaGraphExecDestroy(graph_[q]); graph_[q] = nullptr; }
    }
    vol_any = any;
    forces_valid = false;
}

double Ensemble::volume(int b, double area, const double xc[3]) {
    View v = view();
    long long* d = nullptr;
    CK(cudaMallocAsync(&d, sizeof(long long) * 2, stream));
    long long h[2] = {0, 0};
    try {
        CK(cudaMemsetAsync(d, 0, sizeof(long long) * 2, stream));
        k_volume_sum<double><<<volume_grid(N), kVolThreads, 0, stream>>>(
            v, b, llrint(xc[0] * kGrid), llrint(xc[1] * kGrid), llrint(xc[2] * kGrid), d);
        launches++;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(h, d, sizeof(long long) * 2, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
    } catch (...) {
        cudaFreeAsync(d, stream);
        throw;
    }
    CK(cudaFreeAsync(d, stream));
    return area / 3.0 * volume_of(h[0], h[1]);
}

// ---------------------------------------------------------------- height map
struct HeightArgs {
    double x0, y0, dx, dy, z_min, ax, ay, rho_in, rho_out;
    int nx, ny, b;
};

constexpr int kHeightSharedBins = 1024;

// Per bin: z summed as (z >> 24) and (z & (2^24 - 1)) in two int64 (exact
// for any count below 2^39), and the count.  Bins of up to 1024 collect in
// shared memory first.
__global__ void __launch_bounds__(kVolThreads) k_height_map(View v, HeightArgs A, long long* __restrict__ hi,
                                                            long long* __restrict__ lo,
                                                            unsigned long long* __restrict__ cnt) {
    __shared__ long long s_hi[kHeightSharedBins], s_lo[kHeightSharedBins];
    __shared__ unsigned long long s_cnt[kHeightSharedBins];
    const int nb = A.nx * A.ny;
    const bool shared_bins = nb <= kHeightSharedBins;
    if (shared_bins) {
        for (int q = threadIdx.x; q < nb; q += blockDim.x) { s_hi[q] = 0; s_lo[q] = 0; s_cnt[q] = 0; }
        __syncthreads();
    }
    const size_t N = v.N;
    const int p_lo = v.inst_p0[A.b], p_hi = v.inst_p0[A.b + 1];
    for (int p = p_lo + blockIdx.x * blockDim.x + threadIdx.x; p < p_hi; p += gridDim.x * blockDim.x) {
        if (!bilayer(v.type[p])) continue;
        const long long zq = v.xq[2 * N + p];
        const double x = grid_to_double(v.xq[p]), y = grid_to_double(v.xq[N + p]), z = grid_to_double(zq);
        if (!(z > A.z_min)) continue;
        const double rx = __dsub_rn(x, A.ax), ry = __dsub_rn(y, A.ay);
        const double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(rx, rx), __dmul_rn(ry, ry)));
        if (!(rho >= A.rho_in && rho < A.rho_out)) continue;
        const double fx = floor(__ddiv_rn(__dsub_rn(x, A.x0), A.dx));
        const double fy = floor(__ddiv_rn(__dsub_rn(y, A.y0), A.dy));
        if (!(fx >= 0.0 && fy >= 0.0 && fx < (double)A.nx && fy < (double)A.ny)) continue;
        const int q = (int)fy * A.nx + (int)fx;
        const long long h = zq >> 24, l = zq & 0xFFFFFFll;
        if (shared_bins) {
            atomicAdd((unsigned long long*)&s_hi[q], (unsigned long long)h);
            atomicAdd((unsigned long long*)&s_lo[q], (unsigned long long)l);
            atomicAdd(&s_cnt[q], 1ull);
        } else {
            atomicAdd((unsigned long long*)&hi[q], (unsigned long long)h);
            atomicAdd((unsigned long long*)&lo[q], (unsigned long long)l);
            atomicAdd(&cnt[q], 1ull);
        }
    }
    if (shared_bins) {
        __syncthreads();
        for (int q = threadIdx.x; q < nb; q += blockDim.x) {
            if (!s_cnt[q]) continue;
            atomicAdd((unsigned long long*)&hi[q], (unsigned long long)s_hi[q]);
            atomicAdd((unsigned long long*)&lo[q], (unsigned long long)s_lo[q]);
            atomicAdd(&cnt[q], s_cnt[q]);
        }
    }
}

void Ensemble::height_map(int b, double x0, double y0, double dx, double dy, int nx, int ny, double z_min,
                          const double axis[2], double rho_in, double rho_out, double* h, int* count) {
    const size_t nb = (size_t)nx * ny;
    HeightArgs A{x0, y0, dx, dy, z_min, axis[0], axis[1], rho_in, rho_out, nx, ny, b};
    long long* d = nullptr;
    CK(cudaMallocAsync(&d, sizeof(long long) * 3 * nb, stream));
    std::vector<long long> hl(3 * nb);
    try {
        CK(cudaMemsetAsync(d, 0, sizeof(long long) * 3 * nb, stream));
        View v = view();
        const int n = inst_h[b].n;
        int dev = 0, sms = 152;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int g = std::max(1, std::min((n + kVolThreads - 1) / kVolThreads, sms * 4));
        k_height_map<<<g, kVolThreads, 0, stream>>>(v, A, d, d + nb, (unsigned long long*)(d + 2 * nb));
        launches++;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hl.data(), d, sizeof(long long) * 3 * nb, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
    } catch (...) {
        cudaFreeAsync(d, stream);
        throw;
    }
    CK(cudaFreeAsync(d, stream));
    for (size_t q = 0; q < nb; q++) {
        const long long c = hl[2 * nb + q];
        count[q] = (int)c;
        if (!c) { h[q] = 0.0; continue; }
        // exact sum hi 2^24 + lo on the 2^-40 grid, one rounding to double
        const __int128 s = (__int128)hl[q] * 16777216 + (__int128)hl[nb + q];
        h[q] = (double)s * kGridInv / (double)c;
    }
}

}  // namespace orbc
