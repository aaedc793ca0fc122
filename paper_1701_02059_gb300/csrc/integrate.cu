// Time stepping ("Software Overview": force and torque, then update of
// position and orientation).  Reading: BAOAB Langevin (Leimkuhler & Matthews
// 2013), translational for every particle and rotational for lipids, with
// Cayley rotations of the director and uniform unit-variance noise from
// Philox4x32-10 keyed by (seed, instance; id, step, substream).
//
// State is int64 on the 2^-40 grid; every update is an increment computed in
// FP64 (FP32 for ORBC_F32_FORCE_F32_STEP) and rounded onto the grid, so
// accumulation is exact integer arithmetic.
#include "integrator.cuh"

#include <cstring>

namespace orbc {

// B A O A of one step (the final B follows the force evaluation).  FUSED:
// first the final B of the previous step, whose forces are the same, then
// this step's B A O A: the same two rounded updates as separate launches,
// without a second pass over memory.  The previous step is then not yet
// counted in steps[], so this step's index is steps[b] + 1.
template <typename T, bool FUSED>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 2 : 4) k_baoa(View v, const long long* __restrict__ steps,
                                                 long long* __restrict__ msum, int* __restrict__ mcnt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const size_t N = v.N;
    long long F[3], Tq[3];
    for (int a = 0; a < 3; a++) { F[a] = v.F[a * N + p]; Tq[a] = v.T[a * N + p]; }
    baoa_body<T, FUSED>(v, v, p, F, Tq, steps, msum, mcnt, __activemask(), false);
}

template <bool FUSED>
__global__ void __launch_bounds__(256, 3) k_baoa_d(View v, const long long* __restrict__ steps,
                                                   long long* __restrict__ msum, int* __restrict__ mcnt) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const size_t N = v.N;
    long long F[3], Tq[3];
    for (int a = 0; a < 3; a++) { F[a] = v.F[a * N + p]; Tq[a] = v.T[a * N + p]; }
    baoa_d_body<FUSED>(v, v, p, F, Tq, steps, msum, mcnt, __activemask(), false);
}

__global__ void k_kick_d(View v, long long* __restrict__ steps) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_inst(v.inst_p0, v.B, p);
    const Inst& I = v.inst[b];
    const size_t N = v.N;
    const bool lipid = bilayer(v.type[p]);
    long long vq[3], wq[3] = {0, 0, 0};
    double Nd[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; a++) vq[a] = v.vq[a * N + p];
    if (lipid) for (int a = 0; a < 3; a++) { Nd[a] = gd(v.nq[a * N + p]); wq[a] = v.wq[a * N + p]; }
    long long F[3], Tq[3];
    for (int a = 0; a < 3; a++) { F[a] = v.F[a * N + p]; Tq[a] = v.T[a * N + p]; }
    kick_grid(vq, wq, Nd, lipid, I, 1, F, Tq);
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
    const bool lipid = bilayer(v.type[p]);
    long long vq[3], nq[3] = {0, 0, 0}, wq[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++) vq[a] = v.vq[a * N + p];
    if (lipid) for (int a = 0; a < 3; a++) { nq[a] = v.nq[a * N + p]; wq[a] = v.wq[a * N + p]; }
    long long F[3], Tq[3];
    for (int a = 0; a < 3; a++) { F[a] = v.F[a * N + p]; Tq[a] = v.T[a * N + p]; }
    kick<T>(vq, wq, nq, lipid, C, 1, F, Tq);
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
        if (bilayer(v.type[p])) {
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
    if (!bilayer(v.type[p])) return;
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
