// Host orchestration of the hot path and the C ABI declared in orbc.h.
#include "abi_common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <exception>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>

#include "../../include/orbc.h"

namespace orbc {

// ============================================================== Ensemble basics
// Device memory comes from the stream-ordered pool, which keeps freed blocks
// for reuse (batches are re-packed while the arena runs); the pool is trimmed
// when a system or an arena is destroyed.
static void keep_pool_memory() {
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { cudaGetLastError(); return; }
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev] = true;
}

void trim_pool() {
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess)
        cudaMemPoolTrimTo(pool, 0);
    cudaGetLastError();
}

Ensemble::Ensemble(cudaStream_t s) : stream(s) { keep_pool_memory(); }

Ensemble::~Ensemble() { free_all(); }

void Ensemble::free_all() {
    for (int q = 0; q < 2; q++)
        if (graph_[q]) { cudaGraphExecDestroy(graph_[q]); graph_[q] = nullptr; }
    for (void* p : allocs_) cudaFreeAsync(p, stream);
    allocs_.clear();
    bytes_ = 0;
    for (int* p : scan_tmp_) if (p) cudaFreeAsync(p, stream);
    scan_tmp_.clear();
    scan_tmp_n_.clear();
    if (ev0_) { cudaEventDestroy(ev0_); ev0_ = nullptr; }
    if (ev1_) { cudaEventDestroy(ev1_); ev1_ = nullptr; }
    d_dump = nullptr;
    d_dump_count = nullptr;
    dump_cap = 0;
}

template <typename T>
T* Ensemble::alloc(size_t count) {
    void* p = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw CudaError(cudaErrorMemoryAllocation, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    allocs_.push_back(p);
    bytes_ += bytes;
    CK(cudaMemsetAsync(p, 0, bytes, stream));
    return (T*)p;
}

View Ensemble::view() {
    View v;
    v.B = B; v.N = N; v.Ktot = Ktot; v.Gtot = Gtot;
    v.inst = d_inst; v.inst_p0 = d_p0; v.inst_k0 = d_k0;
    v.xq = d_state[cur_][0]; v.vq = d_state[cur_][1]; v.nq = d_state[cur_][2]; v.wq = d_state[cur_][3];
    v.type = d_type[cur_]; v.id = d_id[cur_];
    v.cell = d_cell; v.slot_of_id = d_slot_of_id;
    v.F = d_F; v.T = d_T; v.Fbig = d_Fbig;
    v.mq = d_mq; v.mo = d_mo; v.mqr = d_mqr; v.mor = d_mor; v.cnorm = d_cnorm; v.grank = d_grank;
    v.cq = d_cq; v.cell_start = d_cell_start; v.R = d_R; v.Rf = d_Rf; v.adj_ptr = d_adj_ptr; v.adj = d_adj; v.adj_cap = adj_cap; v.adjd = d_adjd;
    v.adjn = d_adjcount;
    v.gstart = d_gstart; v.gcent = d_gcent; v.gcf = d_gcf;
    v.bptr = d_bptr; v.bpartner = d_bpartner;
    v.nbond = nbond; v.bij = d_bij; v.binst = d_binst; v.bkf = d_bkf; v.bkd = d_bkd;
    v.status = d_status;
    v.istatus = d_istatus;
    v.wait_polls = wait_polls;
    v.extra_tx = extra_tx;
    v.vol = d_vol;
    return v;
}

View Ensemble::view_alt() {
    cur_ ^= 1;
    View v = view();
    cur_ ^= 1;
    return v;
}

void Ensemble::swap_state() { cur_ ^= 1; }

void Ensemble::sync() { CK(cudaStreamSynchronize(stream)); }

// Per-instance flags of the launches since the last clear.
std::vector<unsigned> Ensemble::read_instance_status(bool clear) {
    std::vector<unsigned> s(B, 0u);
    CK(cudaMemcpyAsync(s.data(), d_istatus, sizeof(unsigned) * B, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (clear) CK(cudaMemsetAsync(d_istatus, 0, sizeof(unsigned) * B, stream));
    return s;
}

unsigned Ensemble::read_status(bool clear) {
    unsigned s = 0;
    CK(cudaMemcpyAsync(&s, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    // a flagged launch may have left the neighbour lists partial
    if (s) list_valid = false;
    if (clear && s) CK(cudaMemsetAsync(d_status, 0, sizeof(unsigned), stream));
    return s;
}

// ---------------------------------------------------------------- timing
struct PendingTime { std::string name; cudaEvent_t a, b; };
static thread_local std::vector<PendingTime> g_pending;

void Ensemble::tic(const char* name) {
    if (!timing) return;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(cudaEventRecord(a, stream));
    g_pending.push_back({name, a, b});
    open_ = name;
}

void Ensemble::toc() {
    if (!timing || g_pending.empty()) return;
    CK(cudaEventRecord(g_pending.back().b, stream));
    open_ = nullptr;
}

static void collect_times(std::vector<Ensemble::TimedKernel>& out) {
    for (auto& p : g_pending) {
        float ms = 0;
        if (cudaEventSynchronize(p.b) == cudaSuccess) cudaEventElapsedTime(&ms, p.a, p.b);
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
        auto it = std::find_if(out.begin(), out.end(), [&](const Ensemble::TimedKernel& t) { return t.name == p.name; });
        if (it == out.end()) { out.push_back({p.name, 0.0, 0}); it = out.end() - 1; }
        it->ms += ms;
        it->launches += 1;
    }
    g_pending.clear();
}

// ---------------------------------------------------------------- set-up
static Inst make_inst(const Params& P) {
    Inst I;
    std::memset(&I, 0, sizeof(I));
    const double two_sixth = 1.122462048309373;
    I.eps = (float)P.eps; I.rmin = (float)(two_sixth * P.sigma); I.rc = (float)P.rc_lipid; I.mu = (float)P.mu;
    I.s0 = (float)P.sin_theta0; I.eps_wca = (float)P.eps_wca; I.sig_wca = (float)P.sigma_wca; I.zeta = P.zeta;
    I.sig_pp = (float)P.sigma_wca_pp; I.sig_pp_d = P.sigma_wca_pp;
    I.eps_d = P.eps; I.rmin_d = two_sixth * P.sigma; I.rc_d = P.rc_lipid; I.mu_d = P.mu; I.s0_d = P.sin_theta0;
    I.eps_wca_d = P.eps_wca; I.sig_wca_d = P.sigma_wca;
    const double rcw = two_sixth * P.sigma_wca, rcp = two_sixth * P.sigma_wca_pp;
    I.rc2_ll = P.rc_lipid * P.rc_lipid;
    I.rc2_wca = rcw * rcw;
    I.rc2_pp = rcp * rcp;
    I.rc2f_ll = (float)I.rc2_ll;
    I.rc2f_wca = (float)I.rc2_wca;
    I.rc2f_pp = (float)I.rc2_pp;
    I.rs = std::max(P.rc_lipid, std::max(rcw, rcp));
    I.rsf = (float)I.rs;
    I.aw = (float)(1.5707963267948966 / (P.rc_lipid - two_sixth * P.sigma));
    I.eps2z_aw = (float)(P.eps * 2.0 * P.zeta * (1.5707963267948966 / (P.rc_lipid - two_sixth * P.sigma)));
    I.skin = P.skin;
    I.skinf = (float)P.skin;
    for (int a = 0; a < 3; a++) {
        I.periodic[a] = P.periodic[a];
        I.box[a] = P.periodic[a] ? P.box[a] : 0.0;
        I.boxq[a] = P.periodic[a] ? llrint(P.box[a] * kGrid) : 0;
        I.boxf[a] = (float)I.box[a];
    }
    const double h = 0.5 * P.dt;
    I.h_m_d = h / P.mass; I.h_i_d = h / P.inertia; I.hdt_d = h;
    const double ct = std::exp(-P.gamma_t * P.dt), cr = std::exp(-P.gamma_r * P.dt);
    I.ct_m1_d = std::expm1(-P.gamma_t * P.dt);
    I.cr_m1_d = std::expm1(-P.gamma_r * P.dt);
    I.st_d = std::sqrt(std::max(0.0, (1.0 - ct * ct) * P.kT / P.mass));
    I.sr_d = std::sqrt(std::max(0.0, (1.0 - cr * cr) * P.kT / P.inertia));
    I.hm8_d = std::ldexp(I.h_m_d, 8); I.hi8_d = std::ldexp(I.h_i_d, 8);
    // the double as an integer times a power of two (exact): x = f 2^e,
    // f in [1/2, 1), m = f 2^53, s = 53 - e
    auto fix = [](double x, unsigned long long& m, int& s) {
        int e = 0;
        const double f = std::frexp(x, &e);
        m = (unsigned long long)std::ldexp(f, 53);
        s = 53 - e;
        if (!(x > 0) || s < 1 || s > 127) { m = 0; s = 1; }   // not reached for valid dt, mass
    };
    fix(I.hm8_d, I.hm8_m, I.hm8_s);
    fix(I.hdt_d, I.hdt_m, I.hdt_s);
    I.st40_d = std::ldexp(I.st_d, 40); I.sr40_d = std::ldexp(I.sr_d, 40); I.ca_d = std::ldexp(0.5 * h, -40);
    const double noise_scale = 3.4641016151377544 * 1.16415321826934814453125e-10;   // sqrt(12) 2^-33
    I.stn_d = I.st40_d * noise_scale;
    I.srn_d = I.sr40_d * noise_scale;
    // signed: ct_m1 = expm1(-gamma dt) <= 0; a zero constant takes the other's
    // scale (its product vanishes)
    auto fix_s = [&](double x, long long& m, int& s) {
        unsigned long long u = 0;
        fix(std::fabs(x), u, s);
        m = x < 0 ? -(long long)u : (long long)u;
    };
    fix_s(I.ct_m1_d, I.ctm1_m, I.ctm1_s);
    fix_s(I.stn_d, I.stn_m, I.stn_s);
    if (I.ctm1_m == 0) I.ctm1_s = I.stn_s;
    if (I.stn_m == 0) I.stn_s = I.ctm1_s;
    // the 128-bit sum holds |v| < 2^52 grid units times a 53-bit mantissa
    // shifted by up to 21 bits, or a 33-bit noise integer times one shifted
    // by up to 40
    I.ou_int = (I.stn_s <= I.ctm1_s) ? (I.ctm1_s - I.stn_s <= 40) : (I.stn_s - I.ctm1_s <= 21);
    I.h_m = (float)I.h_m_d; I.h_i = (float)I.h_i_d; I.hdt = (float)I.hdt_d;
    I.ct_m1 = (float)I.ct_m1_d; I.cr_m1 = (float)I.cr_m1_d; I.st = (float)I.st_d; I.sr = (float)I.sr_d;
    I.mass = P.mass; I.inertia = P.inertia;
    I.seed = P.seed; I.instance = P.instance;
    I.rebuild_every = P.rebuild_every;
    I.n_lloyd = P.n_lloyd_init;
    // bilayer species pairs: the lipid-lipid entry and every entry left at 0
    // take eps and rc_lipid, so their constants equal the lipid pair's
    for (int q = 0; q < 9; q++) {
        const double e = (q > 0 && P.eps_mem[q] > 0) ? P.eps_mem[q] : P.eps;
        const double rc = (q > 0 && P.rc_mem[q] > 0) ? P.rc_mem[q] : P.rc_lipid;
        const double w = 1.5707963267948966 / (rc - two_sixth * P.sigma);
        I.mm_eps_d[q] = e;
        I.mm_rc_d[q] = rc;
        I.mm_rc2[q] = rc * rc;
        I.mm_eps[q] = (float)e;
        I.mm_aw[q] = (float)w;
        I.mm_e2za[q] = (float)(e * 2.0 * P.zeta * w);
        const float rcf = std::sqrt((float)I.mm_rc2[q]);
        I.mm_rcp[q] = rcf;
        I.mm_lo[q] = (rcf - kCutBand) * (rcf - kCutBand);
        I.mm_hi[q] = (rcf + kCutBand) * (rcf + kCutBand);
        I.rs = std::max(I.rs, rc);
    }
    I.rsf = (float)I.rs;
    for (int a = 0; a < 3; a++)
        I.mm_rcf[a] = std::sqrt(std::max((float)I.mm_rc2[3 * a], std::max((float)I.mm_rc2[3 * a + 1], (float)I.mm_rc2[3 * a + 2])));
    return I;
}

// Every array whose size follows from B, N and Ktot (not the grid).
void Ensemble::alloc_core(const std::vector<int>& p0, const std::vector<int>& k0, bool any_skin) {
    d_inst = alloc<Inst>(B);
    d_p0 = alloc<int>(B + 1);
    d_k0 = alloc<int>(B + 1);
    CK(cudaMemcpyAsync(d_p0, p0.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_k0, k0.data(), sizeof(int) * (B + 1), cudaMemcpyHostToDevice, stream));
    for (int s = 0; s < 2; s++) {
        for (int q = 0; q < 4; q++) d_state[s][q] = alloc<long long>((size_t)3 * N);
        d_type[s] = alloc<unsigned char>(N);
        d_id[s] = alloc<unsigned>(N);
    }
    cur_ = 0;
    d_cell = alloc<int>(N);
    d_slot_of_id = alloc<int>(N);
    d_F = alloc<long long>((size_t)3 * N);
    d_T = alloc<long long>((size_t)3 * N);
    d_Fbig = alloc<long long>((size_t)6 * N);
    d_mq = alloc<int4>(N);
    d_mo = alloc<float4>(N);
    d_mqr = alloc<int4>(N);
    d_mor = alloc<float4>(N);
    d_cq = alloc<long long>((size_t)3 * Ktot);
    d_cq_tmp = alloc<long long>((size_t)3 * Ktot);
    d_cell_start = alloc<int>(Ktot + 1);
    d_R = alloc<double>(Ktot);
    d_Rf = alloc<float>(Ktot);
    d_adj_ptr = alloc<int>(Ktot + 1);
    d_adjcount = alloc<int>(Ktot + 1);
    adj_cap = (long long)Ktot * 64;
    d_adj = alloc<int>(adj_cap);
    d_gcent = alloc<int>(Ktot);
    d_gcf = alloc<float4>(Ktot);
    d_gidx = alloc<int>(Ktot);
    d_status = alloc<unsigned>(1);
    d_istatus = alloc<unsigned>(B);
    d_S = alloc<long long>((size_t)3 * Ktot);
    d_msum = alloc<long long>((size_t)3 * Ktot);   // zeroed by alloc, re-zeroed by each use
    d_mcnt = alloc<int>(Ktot);
    d_cnt = alloc<int>(Ktot + 1);
    d_bbox = alloc<long long>((size_t)6 * B);
    d_keys = alloc<unsigned long long>(Ktot);
    d_sortrec = alloc<unsigned char>((size_t)16 * ((Ktot + 1023) / 1024) * 1024);
    d_new_of_old = alloc<int>(Ktot);
    d_cell_new = alloc<int>(N);
    d_perm = alloc<int>(N);
    d_cell_tmp = alloc<int>(N);
    d_rmax = alloc<unsigned long long>(B);
    d_rho = alloc<float>(Ktot);
    d_lbound = alloc<float>(N);
    d_cmove = alloc<float>(Ktot);
    d_cf = alloc<float4>(Ktot);
    d_cnorm = alloc<float4>(Ktot);
    d_grank = alloc<unsigned char>(N);
    d_dmax = alloc<unsigned>(B);
    d_fbcount = alloc<int>(1);
    d_adjpad = alloc<int>((size_t)Ktot * 64);
    d_seglist = alloc<int>((size_t)2 * Ktot);
    d_seglist_n = alloc<int>(2);
    d_adjd = alloc<AdjDesc>(adj_cap);
    d_candrows = alloc<float4>(adj_cap);
    alloc_lists();
    prev_adj_valid_ = false;
    csr_valid_ = false;
    d_energy = alloc<long long>((size_t)8 * B);
    d_vol = alloc<long long>((size_t)2 * B);
    vol_any = false;
    for (const Inst& I : inst_h) vol_any = vol_any || I.vol_on;
    d_step = alloc<long long>(B);
    CK(cudaMemcpyAsync(d_step, step_h.data(), sizeof(long long) * B, cudaMemcpyHostToDevice, stream));
    d_xref = any_skin ? alloc<long long>((size_t)3 * N) : nullptr;
}

// Bond CSR by (p0 + id), both directions; r0 and kb per entry in FP32 and FP64.
// [n][3] to axis-major [3][n].
__global__ void k_aos_to_soa(const long long* __restrict__ aos, int n, long long* __restrict__ soa) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < 3; a++) soa[(size_t)a * n + i] = aos[(size_t)3 * i + a];
}

// Bond partner lists on the device, keyed by p0 + id: counts, scan, fill,
// then each (short) list sorted so the order does not depend on the atomics.
__global__ void k_bond_count(int nbond, const int2* __restrict__ bij, int* __restrict__ cnt,
                             unsigned* __restrict__ status) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nbond; q += gridDim.x * blockDim.x) {
        const int2 e = bij[q];
        const int ci = atomicAdd(&cnt[e.x], 1), cj = atomicAdd(&cnt[e.y], 1);
        if (ci >= kMaxBondsPerParticle || cj >= kMaxBondsPerParticle) atomicOr(status, 1u);
    }
}

__global__ void k_bond_fill(int nbond, const int2* __restrict__ bij, const int* __restrict__ binst,
                            const int* __restrict__ p0, const int* __restrict__ bptr, int* __restrict__ fill,
                            int* __restrict__ partner) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nbond; q += gridDim.x * blockDim.x) {
        const int2 e = bij[q];
        const int base = p0[binst[q]];
        partner[bptr[e.x] + atomicAdd(&fill[e.x], 1)] = e.y - base;
        partner[bptr[e.y] + atomicAdd(&fill[e.y], 1)] = e.x - base;
    }
}

__global__ void k_bond_sort(int N, const int* __restrict__ bptr, int* __restrict__ partner) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int s = bptr[i], e = bptr[i + 1];
    for (int x = s + 1; x < e; x++) {
        const int t = partner[x];
        int y = x - 1;
        while (y >= s && partner[y] > t) { partner[y + 1] = partner[y]; y--; }
        partner[y + 1] = t;
    }
}

void Ensemble::upload_bonds(const std::vector<BondSpec>& bl, const std::vector<int>& p0) {
    // the bonds once each (for the bond kernel), keys p0 + id
    nbond = 0;
    for (int b = 0; b < B; b++) nbond += (int)bl[b].r0->size();
    std::vector<int2> bij(std::max(nbond, 1));
    std::vector<int> binst(std::max(nbond, 1));
    std::vector<float2> bkf(std::max(nbond, 1));
    std::vector<double2> bkd(std::max(nbond, 1));
    for (int b = 0, q0 = 0; b < B; b++) {
        const int nb = (int)bl[b].r0->size();
        for (int q = 0; q < nb; q++) {
            bij[q0 + q] = make_int2(p0[b] + (*bl[b].bonds)[2 * q], p0[b] + (*bl[b].bonds)[2 * q + 1]);
            binst[q0 + q] = b;
            bkf[q0 + q] = make_float2((float)(*bl[b].r0)[q], (float)(*bl[b].kb)[q]);
            bkd[q0 + q] = make_double2((*bl[b].r0)[q], (*bl[b].kb)[q]);
        }
        q0 += nb;
    }
    d_bij = alloc<int2>(std::max(nbond, 1));
    d_binst = alloc<int>(std::max(nbond, 1));
    d_bkf = alloc<float2>(std::max(nbond, 1));
    d_bkd = alloc<double2>(std::max(nbond, 1));
    if (nbond > 0) {
        CK(cudaMemcpyAsync(d_bij, bij.data(), sizeof(int2) * nbond, cudaMemcpyHostToDevice, stream));
        CK(cudaMemcpyAsync(d_binst, binst.data(), sizeof(int) * nbond, cudaMemcpyHostToDevice, stream));
        CK(cudaMemcpyAsync(d_bkf, bkf.data(), sizeof(float2) * nbond, cudaMemcpyHostToDevice, stream));
        CK(cudaMemcpyAsync(d_bkd, bkd.data(), sizeof(double2) * nbond, cudaMemcpyHostToDevice, stream));
    }
    // partner lists (CSR by p0 + id) for the exclusions of the pair kernel
    d_bptr = alloc<int>(N + 1);
    d_bpartner = alloc<int>(std::max(2 * nbond, 1));
    int* cnt = alloc<int>(N + 1);    // zeroed
    int* fill = alloc<int>(N);
    unsigned* flag = alloc<unsigned>(1);
    if (nbond > 0) {
        k_bond_count<<<152 * 8, 256, 0, stream>>>(nbond, d_bij, cnt, flag);
        launches++;
    }
    scan_exclusive(cnt, d_bptr, N + 1);
    if (nbond > 0) {
        k_bond_fill<<<152 * 8, 256, 0, stream>>>(nbond, d_bij, d_binst, d_p0, d_bptr, fill, d_bpartner);
        k_bond_sort<<<(N + 255) / 256, 256, 0, stream>>>(N, d_bptr, d_bpartner);
        launches += 2;
    }
    CK(cudaGetLastError());
    unsigned over = 0;
    CK(cudaMemcpyAsync(&over, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));   // the host vectors die here
    if (over) throw ArgError("more than 8 bonds on one particle");
}

void Ensemble::setup(const std::vector<const HostInstance*>& list) {
    free_all();
    B = (int)list.size();
    if (B < 1) throw ArgError("no instance");
    precision = list[0]->prm.precision;
    N = 0; Ktot = 0;
    inst_h.assign(B, Inst());
    prm_h.clear();
    std::vector<int> p0(B + 1, 0), k0(B + 1, 0);
    for (int b = 0; b < B; b++) {
        const HostInstance& h = *list[b];
        if (h.prm.precision != precision) throw ArgError("all instances of a batch need the same precision");
        inst_h[b] = make_inst(h.prm);
        inst_h[b].p0 = N; inst_h[b].n = h.n;
        inst_h[b].k0 = Ktot; inst_h[b].K = h.prm.n_centroids;
        inst_h[b].partner = h.partner;
        inst_h[b].id_base = h.id_base;
        inst_h[b].all_members = h.all_members;
        // centroid members: the bilayer particles, or every particle of a
        // protein cell set
        inst_h[b].nlip = h.all_members ? h.n : (int)std::count_if(h.type.begin(), h.type.end(), bilayer);
        inst_h[b].has_mp = std::any_of(h.type.begin(), h.type.end(), [](unsigned char t) { return t >= kBand3; });
        if (!h.r0.empty()) {
            std::vector<unsigned char> bil((size_t)h.n);
            for (int i = 0; i < h.n; i++) bil[h.id[i]] = bilayer(h.type[i]);
            for (size_t q = 0; q < h.r0.size() && !inst_h[b].bonded_bilayer; q++)
                inst_h[b].bonded_bilayer = bil[(size_t)h.bonds[2 * q]] || bil[(size_t)h.bonds[2 * q + 1]];
        }
        inst_h[b].vol_on = h.vol_kv > 0.0;
        inst_h[b].kv = h.vol_kv;
        inst_h[b].v0 = h.vol_v0;
        inst_h[b].avol = h.vol_area;
        inst_h[b].a3 = h.vol_area / 3.0;
        for (int a = 0; a < 3; a++) inst_h[b].xcq[a] = llrint(h.vol_xc[a] * kGrid);
        prm_h.push_back(h.prm);
        N += h.n;
        Ktot += h.prm.n_centroids;
        p0[b + 1] = N;
        k0[b + 1] = Ktot;
    }
    step_h.assign(B, 0);
    for (int b = 0; b < B; b++) step_h[b] = list[b]->step0;
    bool any_skin = false;
    for (const HostInstance* hp : list) any_skin |= (hp->prm.rebuild_every > 1);
    alloc_core(p0, k0, any_skin);

    // state: the host's [n][3] arrays are copied as they are and made
    // axis-major on the device
    std::vector<unsigned char> ty(N);
    std::vector<unsigned> ids(N);
    std::vector<int> slot(N);
    const GridVec HostInstance::*fields[4] = {&HostInstance::xq, &HostInstance::vq, &HostInstance::nq,
                                              &HostInstance::wq};
    {
        long long* aos = nullptr;
        CK(cudaMallocAsync(&aos, sizeof(long long) * 3 * (size_t)N, stream));
        for (int q = 0; q < 4; q++) {
            for (int b = 0; b < B; b++) {
                const GridVec& src = (*list[b]).*fields[q];
                CK(cudaMemcpyAsync(aos + (size_t)3 * p0[b], src.data(), sizeof(long long) * 3 * (size_t)list[b]->n,
                                   cudaMemcpyHostToDevice, stream));
            }
            k_aos_to_soa<<<(N + 255) / 256, 256, 0, stream>>>(aos, N, d_state[0][q]);
            launches++;
        }
        CK(cudaGetLastError());
        CK(cudaFreeAsync(aos, stream));
    }
    for (int b = 0; b < B; b++) {
        const HostInstance& h = *list[b];
        const int pb = p0[b];
        parallel_for(h.n, [&](long long i0, long long i1) {   // ids are a permutation: no write conflicts
            for (long long i = i0; i < i1; i++) {
                ty[pb + i] = h.type[i];
                ids[pb + i] = h.id[i];
                slot[pb + h.id[i]] = pb + (int)i;
            }
        });
    }
    CK(cudaMemcpyAsync(d_type[0], ty.data(), N, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_id[0], ids.data(), sizeof(unsigned) * N, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_slot_of_id, slot.data(), sizeof(int) * N, cudaMemcpyHostToDevice, stream));

    // bonds
    std::vector<BondSpec> bl(B);
    for (int b = 0; b < B; b++) bl[b] = BondSpec{&list[b]->bonds, &list[b]->r0, &list[b]->kb};
    upload_bonds(bl, p0);

    // initial centroids (host) and the centroid-grid geometry of each instance
    std::vector<long long> c0((size_t)3 * Ktot);
    Gtot = 0;
    for (int b = 0; b < B; b++) {
        const HostInstance& h = *list[b];
        Inst& I = inst_h[b];
        const int K = I.K;
        std::vector<long long> c((size_t)3 * K);
        if (!h.centroids.empty()) {
            for (int q = 0; q < 3 * K; q++) c[q] = llrint(h.centroids[q] * kGrid);
        } else {
            // members (lipids, or every particle of a protein cell set) in
            // id order, centroid k = member floor(k M / K)
            std::vector<int> by_id(h.n);
            parallel_for(h.n, [&](long long i0, long long i1) {
                for (long long i = i0; i < i1; i++) by_id[h.id[i]] = (int)i;
            });
            // the member slots in id order: counts per chunk of ids, then
            // fill (one chunk per 64k ids, at most 64: a small instance runs
            // inline instead of paying for host threads)
            const int nch = (int)std::min<long long>(64, std::max<long long>(1, (long long)h.n >> 16));
            const long long per = ((long long)h.n + nch - 1) / nch;
            std::vector<long long> cnt(nch + 1, 0);
            parallel_for(nch, [&](long long c0, long long c1) {
                for (long long ch = c0; ch < c1; ch++)
                    for (long long idv = ch * per; idv < std::min<long long>(h.n, (ch + 1) * per); idv++)
                        cnt[ch + 1] += h.all_members || bilayer(h.type[by_id[idv]]);
            }, 1);
            for (int ch = 0; ch < nch; ch++) cnt[ch + 1] += cnt[ch];
            std::vector<int> lip((size_t)cnt[nch]);
            parallel_for(nch, [&](long long c0, long long c1) {
                for (long long ch = c0; ch < c1; ch++) {
                    long long o = cnt[ch];
                    for (long long idv = ch * per; idv < std::min<long long>(h.n, (ch + 1) * per); idv++)
                        if (h.all_members || bilayer(h.type[by_id[idv]])) lip[(size_t)o++] = by_id[idv];
                }
            }, 1);
            if ((int)lip.size() < K)
                throw ArgError(h.all_members ? "more protein centroids than proteins" : "more centroids than lipids");
            for (int k = 0; k < K; k++) {
                int s = lip[(size_t)((long long)k * (long long)lip.size() / K)];
                for (int a = 0; a < 3; a++) c[(size_t)3 * k + a] = h.xq[(size_t)3 * s + a];
            }
        }
        for (int k = 0; k < K; k++)
            for (int a = 0; a < 3; a++)
                if (I.periodic[a]) c[(size_t)3 * k + a] = floor_mod_ll(c[(size_t)3 * k + a], I.boxq[a]);
        for (int k = 0; k < K; k++)
            for (int a = 0; a < 3; a++) c0[(size_t)a * Ktot + I.k0 + k] = c[(size_t)3 * k + a];
        // grid: edge ~ centroid spacing on a membrane of this many lipids (a
        // protein cell set spreads its K centroids over its partner's
        // membrane: the lipid count measures the area)
        const int area_n = (I.all_members && I.partner >= 0) ? inst_h[I.partner].nlip : I.nlip;
        double hgrid = h.prm.grid_h > 0 ? h.prm.grid_h : std::sqrt(1.0863 * std::max(area_n, 1) / (double)K);
        hgrid = std::max(hgrid, 1.0);
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = 1e300; hi[a] = -1e300;
            for (int k = 0; k < K; k++) {
                double x = c[(size_t)3 * k + a] * kGridInv;
                lo[a] = std::min(lo[a], x);
                hi[a] = std::max(hi[a], x);
            }
        }
        for (int tries = 0;; tries++) {
            long long G = 1;
            for (int a = 0; a < 3; a++) {
                if (I.periodic[a]) {
                    I.gdim[a] = std::max(1, (int)std::floor(I.box[a] / hgrid));
                    I.gh[a] = (float)(I.box[a] / I.gdim[a]);
                    I.gorg[a] = 0;
                } else {
                    double o = lo[a] - hgrid;
                    I.gdim[a] = std::max(1, (int)std::ceil((hi[a] - lo[a] + 2 * hgrid) / hgrid));
                    I.gh[a] = (float)hgrid;
                    I.gorg[a] = llrint(o * kGrid);
                }
                I.ginv[a] = 1.0f / I.gh[a];
                G *= I.gdim[a];
            }
            if (G <= (1ll << 24) || tries > 20) break;
            hgrid *= 1.25;
        }
        I.g0 = Gtot;
        Gtot += (long long)I.gdim[0] * I.gdim[1] * I.gdim[2];
    }
    d_gstart = alloc<int>(Gtot + 1);
    d_gmove = alloc<unsigned>(Gtot);
    d_gcount = alloc<int>(Gtot + 1);
    CK(cudaMemcpyAsync(d_cq, c0.data(), sizeof(long long) * 3 * Ktot, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(d_inst, inst_h.data(), sizeof(Inst) * B, cudaMemcpyHostToDevice, stream));
    // warm the scan scratch for the largest size used later
    scan_exclusive(d_gcount, d_gstart, Gtot + 1);
    scan_exclusive(d_cnt, d_cell_start, Ktot + 1);
    CK(cudaStreamSynchronize(stream));
    n_lloyd_.clear();
    for (const HostInstance* hp : list) n_lloyd_.push_back(hp->prm.n_lloyd_init);
    cells_valid = false;
    forces_valid = false;
}

void Ensemble::setup(const HostInstance& h) { setup(std::vector<const HostInstance*>{&h}); }

void Ensemble::init_cells() {
    int iters = 0;
    for (int x : n_lloyd_) iters = std::max(iters, x);
    for (int it = 0; it < iters; it++) {
        tic("grid");
        build_grid();
        toc();
        // the first round searches every particle and records a lower bound
        // on its second-nearest centroid; later rounds search only the
        // particles whose bound no longer certifies their centroid
        tic("estep");
        if (it == 0) estep(d_cell, d_lbound);
        else estep_bounded(d_cell);
        toc();
        tic("mstep");
        mstep_iter(d_cell, it, d_dmax);
        toc();
    }
    finish_cells();
    unsigned st = read_status(true);
    if (st) throw StateError("cell initialisation flagged status " + std::to_string(st));
    collect_times(kernel_times);
}

void Ensemble::compute_forces(bool energies) {
    if (!cells_valid) throw StateError("cells not initialised");
    launch_pairs(energies, false);
    if (energies) launch_kinetic();
    forces_valid = true;
}

void Ensemble::energies(std::vector<double>& out) {
    std::vector<long long> e((size_t)8 * B);
    CK(cudaMemcpyAsync(e.data(), d_energy, sizeof(long long) * 8 * B, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    out.assign((size_t)5 * B, 0.0);
    for (int b = 0; b < B; b++)
        for (int q = 0; q < 5; q++) out[(size_t)5 * b + q] = (double)e[(size_t)8 * b + q] * kForceUnit;
}

void Ensemble::integrate(int nsteps) {
    if (!cells_valid) throw StateError("cells not initialised");
    if (!forces_valid) launch_pairs(false, false);
    // with FP32 forces, each step's force launch also runs the next step's
    // B-A-O-A (the last step's forces are evaluated alone, before the final B)
    // (the fused evaluation has no instantiation for bilayer species pairs
    // or bonded bilayer particles)
    const bool fuse = fuse_steps && !force_f64() && !any_mp();
    for (int s = 0; s < nsteps; s++) {
        step_body(s > 0, fuse && s > 0, fuse && s + 1 < nsteps);
        for (auto& x : step_h) x++;
    }
    if (nsteps > 0) {
        tic("integrate_kick");
        launch_kick(false);
        toc();
    }
    forces_valid = true;
    collect_times(kernel_times);
}

// One time step without its final B: B-A-O-A (after the previous step's
// final B when fused), cell rebuild (or mirrors), forces.
void Ensemble::step_body(bool fused, bool baoa_done, bool eval_step) {
    // rebuilding every step: the B-A-O-A launch also sums the M-step's
    // per-cell displacements of the centroid members
    const int re = prm_h[0].rebuild_every;
    const bool every = re <= 1 && !d_xref;
    if (!baoa_done) {
        tic("integrate_baoa");
        launch_integrate_first(fused, every);
        toc();
    }
    bool due = (re <= 1) || ((step_h[0] + 1) % re == 0);
    if (!due && d_xref) due = displacement_exceeds_skin();
    if (due) {
        tic("rebuild");
        rebuild(every);
        toc();
    } else {
        tic("mirrors");
        mirrors();
        toc();
    }
    if (eval_step) launch_pairs_step(every);
    else launch_pairs(false, false);
}

// ---------------------------------------------------------------- getters
// Host copies in id order: converted on the device (k_to_id_order), then one
// copy per array.
void Ensemble::get_state(int b, double* pos, double* vel, double* ori, double* angvel, long long* step) {
    const Inst& I = inst_h[b];
    double* tmp = nullptr;
    CK(cudaMallocAsync(&tmp, sizeof(double) * 3 * (size_t)std::max(I.n, 1), stream));
    double* outs[4] = {pos, vel, ori, angvel};
    try {
        for (int q = 0; q < 4; q++) {
            if (!outs[q]) continue;
            to_id_order(b, d_state[cur_][q], kGridInv, tmp);
            CK(cudaMemcpyAsync(outs[q], tmp, sizeof(double) * 3 * (size_t)I.n, cudaMemcpyDeviceToHost, stream));
        }
        if (step) CK(cudaMemcpyAsync(step, d_step + b, sizeof(long long), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
    } catch (...) {
        cudaFreeAsync(tmp, stream);
        throw;
    }
    CK(cudaFreeAsync(tmp, stream));
}

void Ensemble::get_forces(int b, double* f, double* t) {
    const Inst& I = inst_h[b];
    double* tmp = nullptr;
    CK(cudaMallocAsync(&tmp, sizeof(double) * 3 * (size_t)std::max(I.n, 1), stream));
    long long* src[2] = {d_F, d_T};
    double* outs[2] = {f, t};
    try {
        for (int q = 0; q < 2; q++) {
            if (!outs[q]) continue;
            to_id_order(b, src[q], kForceUnit, tmp);
            CK(cudaMemcpyAsync(outs[q], tmp, sizeof(double) * 3 * (size_t)I.n, cudaMemcpyDeviceToHost, stream));
        }
        CK(cudaStreamSynchronize(stream));
    } catch (...) {
        cudaFreeAsync(tmp, stream);
        throw;
    }
    CK(cudaFreeAsync(tmp, stream));
}

void Ensemble::get_cells(int b, int* cell_of_id, unsigned* slot_ids, double* centroids, int* cell_start,
                         double* radius, int* adj_ptr, int* adj) {
    adjacency_csr();
    const Inst& I = inst_h[b];
    const int n = I.n, K = I.K;
    std::vector<unsigned> ids(n);
    std::vector<int> cl(n);
    CK(cudaMemcpyAsync(ids.data(), d_id[cur_] + I.p0, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(cl.data(), d_cell + I.p0, sizeof(int) * n, cudaMemcpyDeviceToHost, stream));
    std::vector<int> cs(K + 1), ap(K + 1);
    CK(cudaMemcpyAsync(cs.data(), d_cell_start + I.k0, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(ap.data(), d_adj_ptr + I.k0, sizeof(int) * (K + 1), cudaMemcpyDeviceToHost, stream));
    std::vector<double> R(K);
    CK(cudaMemcpyAsync(R.data(), d_R + I.k0, sizeof(double) * K, cudaMemcpyDeviceToHost, stream));
    std::vector<long long> c((size_t)3 * K);
    for (int a = 0; a < 3; a++)
        CK(cudaMemcpyAsync(c.data() + (size_t)a * K, d_cq + (size_t)a * Ktot + I.k0, sizeof(long long) * K,
                           cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    for (int i = 0; i < n; i++) {
        if (cell_of_id) cell_of_id[ids[i]] = cl[i] - I.k0;
        if (slot_ids) slot_ids[i] = ids[i];
    }
    if (centroids)
        for (int k = 0; k < K; k++)
            for (int a = 0; a < 3; a++) centroids[(size_t)3 * k + a] = (double)c[(size_t)a * K + k] * kGridInv;
    if (cell_start) for (int k = 0; k <= K; k++) cell_start[k] = cs[k] - I.p0;
    if (radius) std::copy(R.begin(), R.end(), radius);
    if (adj_ptr) for (int k = 0; k <= K; k++) adj_ptr[k] = ap[k] - ap[0];
    if (adj) {
        long long L = ap[K] - ap[0];
        std::vector<int> a((size_t)std::max(L, 1ll));
        if (L > 0)
            CK(cudaMemcpyAsync(a.data(), d_adj + ap[0], sizeof(int) * L, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (long long q = 0; q < L; q++) adj[q] = a[q] - I.k0;
    }
}

// The cells of every instance of the batch as one list (global cell
// numbers, ids offset by each instance's id_base): a membrane with separate
// protein cells, or a single instance.
void Ensemble::get_cells_all(int* cell_of_id, unsigned* slot_ids, double* centroids, int* cell_start, double* radius,
                             int* adj_ptr, int* adj) {
    adjacency_csr();
    std::vector<unsigned> ids(N);
    std::vector<int> cl(N);
    CK(cudaMemcpyAsync(ids.data(), d_id[cur_], sizeof(unsigned) * N, cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(cl.data(), d_cell, sizeof(int) * N, cudaMemcpyDeviceToHost, stream));
    std::vector<int> cs(Ktot + 1), ap(Ktot + 1);
    CK(cudaMemcpyAsync(cs.data(), d_cell_start, sizeof(int) * (Ktot + 1), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(ap.data(), d_adj_ptr, sizeof(int) * (Ktot + 1), cudaMemcpyDeviceToHost, stream));
    std::vector<double> R(Ktot);
    CK(cudaMemcpyAsync(R.data(), d_R, sizeof(double) * Ktot, cudaMemcpyDeviceToHost, stream));
    std::vector<long long> c((size_t)3 * Ktot);
    CK(cudaMemcpyAsync(c.data(), d_cq, sizeof(long long) * 3 * Ktot, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    for (int b = 0; b < B; b++)
        for (int i = inst_h[b].p0; i < inst_h[b].p0 + inst_h[b].n; i++) ids[i] += (unsigned)inst_h[b].id_base;
    for (int i = 0; i < N; i++) {
        if (cell_of_id) cell_of_id[ids[i]] = cl[i];
        if (slot_ids) slot_ids[i] = ids[i];
    }
    if (centroids)
        for (int k = 0; k < Ktot; k++)
            for (int a = 0; a < 3; a++) centroids[(size_t)3 * k + a] = (double)c[(size_t)a * Ktot + k] * kGridInv;
    if (cell_start) std::copy(cs.begin(), cs.end(), cell_start);
    if (radius) std::copy(R.begin(), R.end(), radius);
    if (adj_ptr) for (int k = 0; k <= Ktot; k++) adj_ptr[k] = ap[k] - ap[0];
    if (adj) {
        const long long L = ap[Ktot] - ap[0];
        if (L > 0) CK(cudaMemcpyAsync(adj, d_adj + ap[0], sizeof(int) * L, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
    }
}

long long Ensemble::adjacency_len_all() {
    adjacency_csr();
    int ap[2];
    CK(cudaMemcpyAsync(&ap[0], d_adj_ptr, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(&ap[1], d_adj_ptr + Ktot, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    return ap[1] - ap[0];
}

long long Ensemble::adjacency_len(int b) {
    adjacency_csr();
    const Inst& I = inst_h[b];
    int ap[2];
    CK(cudaMemcpyAsync(&ap[0], d_adj_ptr + I.k0, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaMemcpyAsync(&ap[1], d_adj_ptr + I.k0 + I.K, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    return ap[1] - ap[0];
}

long long Ensemble::dump_pairs(int b, long long cap, unsigned* pairs) {
    if (!cells_valid) throw StateError("cells not initialised");
    if (B != 1 && !(B == 2 && inst_h[0].partner == 1))
        throw ArgError("pair dump is available for single-membrane systems");
    (void)b;
    // cap == 0 or no output: count only
    long long want = pairs ? cap : 0;
    if (!d_dump_count) d_dump_count = alloc<unsigned long long>(1);
    if (want > dump_cap) {
        d_dump = alloc<unsigned>((size_t)2 * want);
        dump_cap = want;
    }
    long long saved = dump_cap;
    if (want == 0) dump_cap = 0;
    CK(cudaMemsetAsync(d_dump_count, 0, sizeof(unsigned long long), stream));
    launch_pairs(false, true);
    dump_cap = saved;
    unsigned long long cnt = 0;
    CK(cudaMemcpyAsync(&cnt, d_dump_count, sizeof(cnt), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (want == 0) return (long long)cnt;
    long long n = (long long)std::min<unsigned long long>(cnt, (unsigned long long)want);
    std::vector<unsigned> h((size_t)2 * std::max(n, 1ll));
    if (n > 0) CK(cudaMemcpyAsync(h.data(), d_dump, sizeof(unsigned) * 2 * n, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    std::vector<std::pair<unsigned, unsigned>> v((size_t)n);
    for (long long q = 0; q < n; q++) v[q] = {h[2 * q], h[2 * q + 1]};
    std::sort(v.begin(), v.end());
    for (long long q = 0; q < n; q++) { pairs[2 * q] = v[q].first; pairs[2 * q + 1] = v[q].second; }
    return (long long)cnt;
}

// Per-slot int64 fixed-point arrays of instance b to FP64 [n][3] in id order.
__global__ void k_to_id_order(const unsigned* __restrict__ id, const long long* __restrict__ q, size_t N, int p0, int n,
                              double unit, double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int p = p0 + t;
    const unsigned i = id[p];
    for (int a = 0; a < 3; a++) out[(size_t)3 * i + a] = __ll2double_rn(q[(size_t)a * N + p]) * unit;
}

void Ensemble::to_id_order(int b, const long long* q, double unit, double* out) {
    const Inst& I = inst_h[b];
    k_to_id_order<<<(I.n + 255) / 256, 256, 0, stream>>>(d_id[cur_], q, (size_t)N, I.p0, I.n, unit, out);
    launches++;
    CK(cudaGetLastError());
}

void Ensemble::get_state_device(int b, double* pos, double* vel, double* ori, double* angvel) {
    double* outs[4] = {pos, vel, ori, angvel};
    for (int q = 0; q < 4; q++)
        if (outs[q]) to_id_order(b, d_state[cur_][q], kGridInv, outs[q]);
    CK(cudaStreamSynchronize(stream));
}

void Ensemble::get_forces_device(int b, double* f, double* t) {
    if (f) to_id_order(b, d_F, kForceUnit, f);
    if (t) to_id_order(b, d_T, kForceUnit, t);
    CK(cudaStreamSynchronize(stream));
}

}  // namespace orbc

// ============================================================== C ABI
using namespace orbc;

struct orbc_system {
    Params prm;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Ensemble* ens = nullptr;
    HostInstance host;
    HostInstance parts[2];     // the lipid and protein cell sets while they are set up
    bool have_particles = false;
    bool dirty = false;        // the host copy is newer than the device (set-up pending)
    bool host_stale = false;   // the device has stepped past the host copy
    std::string err;
};

static void pull_state(orbc_system* s);

// Separate protein cells: the membrane runs as two instances of one batch,
// its lipids (the lipid cell set) and its proteins (the protein cell set),
// each the other's partner: their neighbour rows hold the cells of both
// sets, and the proteins' ids, Philox counters and pair dumps are offset by
// N_L.  Type-major ids keep every particle's id.
static void split_sets(const HostInstance& h, HostInstance& L, HostInstance& P) {
    const int n = h.n;
    const int nl = (int)std::count_if(h.type.begin(), h.type.end(), bilayer);
    for (int i = 0; i < n; i++)
        if (bilayer(h.type[i]) != ((int)h.id[i] < nl))
            throw ArgError("separate protein cells need type-major ids (the bilayer holds ids 0..N_L-1)");
    if (nl < 1 || nl == n) throw ArgError("separate protein cells need a bilayer and cytoskeleton proteins");
    L = HostInstance();
    P = HostInstance();
    L.prm = h.prm;
    L.prm.n_protein_centroids = 0;
    P.prm = h.prm;
    P.prm.n_centroids = h.prm.n_protein_centroids;
    P.prm.n_protein_centroids = 0;
    L.n = nl;
    P.n = n - nl;
    HostInstance* to[2] = {&L, &P};
    for (HostInstance* t : to) {
        t->xq.resize((size_t)3 * t->n); t->vq.resize((size_t)3 * t->n);
        t->nq.resize((size_t)3 * t->n); t->wq.resize((size_t)3 * t->n);
        t->type.reserve(t->n); t->id.reserve(t->n);
    }
    int o[2] = {0, 0};
    for (int i = 0; i < n; i++) {
        const int w = bilayer(h.type[i]) ? 0 : 1;
        HostInstance& t = *to[w];
        for (int a = 0; a < 3; a++) {
            t.xq[(size_t)3 * o[w] + a] = h.xq[(size_t)3 * i + a];
            t.vq[(size_t)3 * o[w] + a] = h.vq[(size_t)3 * i + a];
            t.nq[(size_t)3 * o[w] + a] = h.nq[(size_t)3 * i + a];
            t.wq[(size_t)3 * o[w] + a] = h.wq[(size_t)3 * i + a];
        }
        t.type.push_back(h.type[i]);
        t.id.push_back(w ? h.id[i] - (unsigned)nl : h.id[i]);
        o[w]++;
    }
    for (size_t q = 0; q < h.r0.size(); q++) {
        const int a = h.bonds[2 * q], b = h.bonds[2 * q + 1];
        if (a < nl || b < nl)
            throw ArgError("with separate protein cells every bond joins two cytoskeleton proteins (no anchors)");
        P.bonds.push_back(a - nl);
        P.bonds.push_back(b - nl);
        P.r0.push_back(h.r0[q]);
        P.kb.push_back(h.kb[q]);
    }
    if (!h.centroids.empty()) {
        const size_t kl = (size_t)3 * h.prm.n_centroids;
        L.centroids.assign(h.centroids.begin(), h.centroids.begin() + kl);
        P.centroids.assign(h.centroids.begin() + kl, h.centroids.end());
    }
    L.step0 = P.step0 = h.step0;
    L.vol_kv = h.vol_kv; L.vol_v0 = h.vol_v0; L.vol_area = h.vol_area;
    for (int a = 0; a < 3; a++) L.vol_xc[a] = h.vol_xc[a];
    L.partner = 1; P.partner = 0;
    P.id_base = nl;
    P.all_members = 1;
}

// The device set-up runs once, when a call first needs the device after the
// particles or bonds changed.
static void sync_device(orbc_system* s) {
    if (!s->dirty) return;
    if (s->prm.n_protein_centroids > 0) {
        split_sets(s->host, s->parts[0], s->parts[1]);
        s->ens->setup(std::vector<const HostInstance*>{&s->parts[0], &s->parts[1]});
        s->parts[0] = HostInstance();
        s->parts[1] = HostInstance();
    } else {
        s->ens->setup(s->host);
    }
    s->dirty = false;
}

// The handle's membrane from every instance of its batch, in id order (each
// instance's ids start at its id_base).
static void sys_get_state(orbc_system* s, double* pos, double* vel, double* ori, double* angvel, long long* step) {
    Ensemble& e = *s->ens;
    for (int b = 0; b < e.B; b++) {
        const size_t o = (size_t)3 * e.inst_h[b].id_base;
        e.get_state(b, pos ? pos + o : nullptr, vel ? vel + o : nullptr, ori ? ori + o : nullptr,
                    angvel ? angvel + o : nullptr, b == 0 ? step : nullptr);
    }
}

// Current device state back into the host copy (exact: grid values), so a
// re-setup keeps the trajectory.
static void pull_state(orbc_system* s) {
    HostInstance& h = s->host;
    const int n = h.n;
    std::vector<double> pos((size_t)3 * n), vel((size_t)3 * n), ori((size_t)3 * n), w((size_t)3 * n);
    long long step = 0;
    sys_get_state(s, pos.data(), vel.data(), ori.data(), w.data(), &step);
    std::vector<unsigned> ids(n);
    for (int i = 0; i < n; i++) ids[i] = (unsigned)i;
    std::vector<unsigned char> ty(n);
    for (int i = 0; i < n; i++) ty[h.id[i]] = h.type[i];
    parallel_for((long long)3 * n, [&](long long q0, long long q1) {
        for (long long q = q0; q < q1; q++) {
            h.xq[q] = llrint(pos[q] * kGrid);
            h.vq[q] = llrint(vel[q] * kGrid);
            h.nq[q] = llrint(ori[q] * kGrid);
            h.wq[q] = llrint(w[q] * kGrid);
        }
    });
    h.id = ids;
    h.type = ty;
    h.step0 = step;
}

static int fail(orbc_system* s, int code, const std::string& what) {
    if (s) s->err = what;
    return code;
}

template <typename F>
static int guarded(orbc_system* s, F&& f) {
    return guarded_call(s ? &s->err : nullptr, std::forward<F>(f));
}

Params orbc::to_params(const orbc_params* p) {
    Params P;
    P.eps = p->eps; P.sigma = p->sigma; P.rc_lipid = p->rc_lipid; P.mu = p->mu; P.sin_theta0 = p->sin_theta0;
    P.zeta = p->zeta; P.eps_wca = p->eps_wca; P.sigma_wca = p->sigma_wca; P.sigma_wca_pp = p->sigma_wca_pp;
    P.dt = p->dt; P.kT = p->kT; P.gamma_t = p->gamma_t; P.gamma_r = p->gamma_r; P.mass = p->mass; P.inertia = p->inertia;
    for (int a = 0; a < 3; a++) { P.box[a] = p->box[a]; P.periodic[a] = p->periodic[a] ? 1 : 0; }
    P.n_centroids = p->n_centroids; P.n_lloyd_init = p->n_lloyd_init; P.rebuild_every = p->rebuild_every;
    P.skin = p->skin; P.grid_h = p->grid_h; P.seed = p->seed; P.instance = p->instance;
    P.precision = (int)p->precision;
    P.n_protein_centroids = p->n_protein_centroids;
    P.eval_ctas = p->eval_ctas == 0 ? 7 : p->eval_ctas;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) { P.eps_mem[3 * a + b] = p->eps_mem[a][b]; P.rc_mem[3 * a + b] = p->rc_mem[a][b]; }
    return P;
}

void orbc::check_params(const Params& P) {
    auto fin = [](double x) { return std::isfinite(x); };
    if (!(fin(P.eps) && fin(P.sigma) && P.sigma > 0 && fin(P.rc_lipid) && P.rc_lipid > 1.122462048309373 * P.sigma))
        throw ArgError("invalid lipid potential parameters (need rc_lipid > 2^(1/6) sigma)");
    if (P.zeta < 1 || P.zeta > 16) throw ArgError("zeta must be in 1..16");
    if (!(fin(P.eps_wca) && fin(P.sigma_wca) && P.sigma_wca > 0 && fin(P.sigma_wca_pp) && P.sigma_wca_pp > 0))
        throw ArgError("invalid WCA parameters");
    if (!(P.dt > 0 && fin(P.dt) && P.mass > 0 && P.inertia > 0 && P.kT >= 0 && P.gamma_t >= 0 && P.gamma_r >= 0))
        throw ArgError("invalid integrator parameters");
    for (int a = 0; a < 3; a++)
        if (P.periodic[a] && !(P.box[a] > 0 && P.box[a] < 4096)) throw ArgError("periodic axis needs 0 < box < 4096");
    if (P.n_centroids < 1) throw ArgError("n_centroids must be >= 1");
    if (P.n_lloyd_init < 0) throw ArgError("n_lloyd_init must be >= 0");
    if (P.rebuild_every < 1) throw ArgError("rebuild_every must be >= 1");
    if (P.rebuild_every > 1 && !(P.skin > 0)) throw ArgError("rebuild_every > 1 needs a positive skin");
    if (!(P.skin >= 0 && fin(P.skin)) || !(P.grid_h >= 0 && fin(P.grid_h))) throw ArgError("invalid skin or grid_h");
    if (P.precision < 0 || P.precision > 2) throw ArgError("unknown precision");
    if (P.n_protein_centroids < 0) throw ArgError("n_protein_centroids must be >= 0");
    if (P.eval_ctas != 5 && P.eval_ctas != 7) throw ArgError("eval_ctas must be 0, 5 or 7");
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            const double e = P.eps_mem[3 * a + b], rc = P.rc_mem[3 * a + b];
            if (!(fin(e) && e >= 0 && fin(rc) && rc >= 0))
                throw ArgError("bilayer species table: entries must be finite and >= 0");
            if (e != P.eps_mem[3 * b + a] || rc != P.rc_mem[3 * b + a])
                throw ArgError("bilayer species table must be symmetric");
            if (rc > 0 && !(rc > 1.122462048309373 * P.sigma && rc < 64.0))
                throw ArgError("bilayer species cutoff must lie in (2^(1/6) sigma, 64 sigma)");
        }
    if (P.eps_mem[0] != 0 || P.rc_mem[0] != 0)
        throw ArgError("the lipid-lipid entry of the species table is eps and rc_lipid (leave it 0)");
}


void orbc::parallel_for(long long n, const std::function<void(long long, long long)>& f, long long grain) {
    if (n <= 0) return;
    grain = std::max(1ll, grain);
    const long long nt = std::min<long long>({16, std::max(1u, std::thread::hardware_concurrency()), (n + grain - 1) / grain});
    if (nt <= 1) { f(0, n); return; }
    std::vector<std::thread> th;
    std::vector<std::exception_ptr> err((size_t)nt);
    const long long chunk = (n + nt - 1) / nt;
    for (long long t = 0; t < nt; t++)
        th.emplace_back([&, t] {
            try {
                const long long b = t * chunk, e = std::min(n, b + chunk);
                if (b < e) f(b, e);
            } catch (...) {
                err[(size_t)t] = std::current_exception();
            }
        });
    for (auto& x : th) x.join();
    for (auto& e : err)
        if (e) std::rethrow_exception(e);
}

HostInstance orbc::host_instance(const Params& prm, int n, const double* pos, const double* vel, const double* ori,
                                 const double* angvel, const unsigned char* type, const unsigned* id) {
    if (n < 1 || !pos || !vel || !ori || !angvel || !type || !id) throw ArgError("null pointer or n < 1");
    HostInstance h;
    h.prm = prm;
    h.n = n;
    // sized without zero-filling: every entry is written below
    h.xq.resize((size_t)3 * n); h.vq.resize((size_t)3 * n); h.nq.resize((size_t)3 * n); h.wq.resize((size_t)3 * n);
    h.type.assign(type, type + n);
    h.id.assign(id, id + n);
    // ids a permutation of 0..n-1 (each marked once), types known
    std::unique_ptr<std::atomic<unsigned char>[]> seen(new std::atomic<unsigned char>[n]);
    parallel_for(n, [&](long long i0, long long i1) {
        for (long long i = i0; i < i1; i++) seen[i].store(0, std::memory_order_relaxed);
    });
    parallel_for(n, [&](long long i0, long long i1) {
        for (long long i = i0; i < i1; i++) {
            if (id[i] >= (unsigned)n || seen[id[i]].exchange(1, std::memory_order_relaxed))
                throw ArgError("ids must be a permutation of 0..n-1");
            if (type[i] > kMaxType) throw ArgError("unknown particle type");
        }
    });
    parallel_for(n, [&](long long i0, long long i1) {
        for (long long i = i0; i < i1; i++) {
            for (int a = 0; a < 3; a++) {
                double x = pos[3 * i + a], v = vel[3 * i + a];
                if (!std::isfinite(x) || !std::isfinite(v)) throw ArgError("non-finite position or velocity");
                if (std::fabs(x) >= 4096.0) throw ArgError("|position| must be < 4096 sigma");
                if (std::fabs(v) >= 1e6) throw ArgError("|velocity| too large");
                h.xq[(size_t)3 * i + a] = llrint(x * kGrid);
                h.vq[(size_t)3 * i + a] = llrint(v * kGrid);
            }
            if (bilayer(type[i])) {
                double o[3], w[3];
                for (int a = 0; a < 3; a++) { o[a] = ori[3 * i + a]; w[a] = angvel[3 * i + a]; }
                for (int a = 0; a < 3; a++)
                    if (!std::isfinite(o[a]) || !std::isfinite(w[a])) throw ArgError("non-finite orientation");
                double nn = std::sqrt(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
                if (std::fabs(nn - 1.0) > 1e-6) throw ArgError("lipid orientation must be a unit vector");
                for (int a = 0; a < 3; a++) {
                    h.nq[(size_t)3 * i + a] = llrint(o[a] * kGrid);
                    h.wq[(size_t)3 * i + a] = llrint(w[a] * kGrid);
                }
            } else {
                for (int a = 0; a < 3; a++) { h.nq[(size_t)3 * i + a] = 0; h.wq[(size_t)3 * i + a] = 0; }
            }
        }
    });
    return h;
}

void orbc::host_bonds(HostInstance& h, int nb, const int* ij, const double* r0, const double* kb) {
    if (nb < 0 || (nb > 0 && (!ij || !r0 || !kb))) throw ArgError("invalid bond arrays");
    for (int q = 0; q < nb; q++) {
        if (ij[2 * q] < 0 || ij[2 * q] >= h.n || ij[2 * q + 1] < 0 || ij[2 * q + 1] >= h.n || ij[2 * q] == ij[2 * q + 1])
            throw ArgError("bond id out of range");
        if (!(r0[q] >= 0 && std::isfinite(r0[q]) && kb[q] >= 0 && std::isfinite(kb[q])))
            throw ArgError("invalid bond constants");
    }
    h.bonds.assign(ij, ij + 2 * (size_t)nb);
    h.r0.assign(r0, r0 + nb);
    h.kb.assign(kb, kb + nb);
}

int orbc::status_code(unsigned st) {
    if (st & kStatusTimeout) return ORBC_E_TIMEOUT;
    if (st & (kStatusNaN | kStatusPairForceRange)) return ORBC_E_NAN;
    return ORBC_E_STATE;
}

extern "C" {

void orbc_default_params(orbc_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->eps = 1.0; p->sigma = 1.0; p->rc_lipid = 2.6; p->mu = 3.0; p->sin_theta0 = 0.0; p->zeta = 4;
    p->eps_wca = 1.0; p->sigma_wca = 1.0; p->sigma_wca_pp = 0.5;
    p->dt = 0.01; p->kT = 0.2; p->gamma_t = 1.0; p->gamma_r = 1.0; p->mass = 1.0; p->inertia = 1.0;
    p->n_centroids = 64; p->n_lloyd_init = 10; p->rebuild_every = 1; p->skin = 0.0; p->grid_h = 0.0;
    p->seed = 0; p->instance = 0; p->precision = ORBC_F32_FORCE_F64_STATE;
    p->n_protein_centroids = 0;
    p->eval_ctas = 0;
}

int orbc_create(const orbc_params* params, void* cuda_stream, orbc_system** out) {
    if (!params || !out) return ORBC_E_ARG;
    *out = nullptr;
    orbc_system* s = new (std::nothrow) orbc_system();
    if (!s) return ORBC_E_NOMEM;
    int rc = guarded(s, [&] {
        s->prm = to_params(params);
        check_params(s->prm);
        if (cuda_stream) s->stream = (cudaStream_t)cuda_stream;
        else { CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)); s->own_stream = true; }
        s->ens = new Ensemble(s->stream);
    });
    if (rc != ORBC_OK) {
        delete s;
        return rc;
    }
    *out = s;
    return ORBC_OK;
}

int orbc_set_particles(orbc_system* s, int n, const double* pos, const double* vel, const double* ori,
                       const double* angvel, const unsigned char* type, const unsigned* id) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        HostInstance h = host_instance(s->prm, n, pos, vel, ori, angvel, type, id);
        // the volume constraint belongs to the handle, not to the particles
        h.vol_kv = s->host.vol_kv;
        h.vol_v0 = s->host.vol_v0;
        h.vol_area = s->host.vol_area;
        for (int a = 0; a < 3; a++) h.vol_xc[a] = s->host.vol_xc[a];
        s->host = std::move(h);
        s->have_particles = true;
        s->dirty = true;
        s->host_stale = false;
    });
}

int orbc_set_bonds(orbc_system* s, int nb, const int* ij, const double* r0, const double* kb) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        if (!s->have_particles) throw StateError("set particles before bonds");
        if (s->host_stale) pull_state(s);
        host_bonds(s->host, nb, ij, r0, kb);
        s->dirty = true;
        s->host_stale = false;
    });
}

int orbc_init_cells(orbc_system* s, const double* centroids) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        if (!s->have_particles) throw StateError("no particles");
        if (s->host_stale) pull_state(s);
        const int K = s->prm.n_centroids + s->prm.n_protein_centroids;
        if (centroids) {
            for (int q = 0; q < 3 * K; q++)
                if (!std::isfinite(centroids[q]) || std::fabs(centroids[q]) >= 4096.0) throw ArgError("invalid centroid");
            s->host.centroids.assign(centroids, centroids + 3 * (size_t)K);
        } else {
            s->host.centroids.clear();
        }
        s->dirty = true;
        sync_device(s);
        s->host_stale = false;
        s->ens->init_cells();
    });
}

int orbc_rebuild_cells(orbc_system* s) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        sync_device(s);
        if (!s->ens->cells_valid) throw StateError("cells not initialised");
        s->ens->rebuild();
        unsigned st = s->ens->read_status(true);
        if (st) throw StateError("rebuild flagged status " + std::to_string(st));
    });
}

int orbc_compute_forces(orbc_system* s, double* energies_out) {
    if (!s) return ORBC_E_ARG;
    unsigned st = 0;
    int rc = guarded(s, [&] {
        sync_device(s);
        s->ens->compute_forces(energies_out != nullptr);
        st = s->ens->read_status(true);
        if (st) s->ens->forces_valid = false;
        if (!st && energies_out) {
            std::vector<double> e;
            s->ens->energies(e);
            // the membrane's totals over the instances of its batch
            for (int q = 0; q < 5; q++) {
                energies_out[q] = 0.0;
                for (int b = 0; b < s->ens->B; b++) energies_out[q] += e[(size_t)5 * b + q];
            }
        }
    });
    if (rc == ORBC_OK && st) return fail(s, status_code(st), "device status " + std::to_string(st));
    return rc;
}

int orbc_integrate(orbc_system* s, int nsteps) {
    if (!s) return ORBC_E_ARG;
    if (nsteps < 0) return fail(s, ORBC_E_ARG, "nsteps < 0");
    unsigned st = 0;
    int rc = guarded(s, [&] {
        sync_device(s);
        s->host_stale = true;
        s->ens->integrate(nsteps);
        st = s->ens->read_status(true);
        if (st) s->ens->forces_valid = false;
    });
    if (rc == ORBC_OK && st) return fail(s, status_code(st), "device status " + std::to_string(st));
    return rc;
}

int orbc_get_state(orbc_system* s, double* pos, double* vel, double* ori, double* angvel, long long* step) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        if (!s->have_particles) throw StateError("no particles");
        sync_device(s);
        sys_get_state(s, pos, vel, ori, angvel, step);
    });
}

int orbc_set_particles_device(orbc_system* s, int n, const double* pos, const double* vel, const double* ori,
                              const double* angvel, const unsigned char* type, const unsigned* id) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        if (n < 1 || !pos || !vel || !ori || !angvel || !type || !id) throw ArgError("null pointer or n < 1");
        std::vector<double> hp((size_t)3 * n), hv((size_t)3 * n), ho((size_t)3 * n), hw((size_t)3 * n);
        std::vector<unsigned char> ht(n);
        std::vector<unsigned> hi(n);
        const double* src[4] = {pos, vel, ori, angvel};
        double* dst[4] = {hp.data(), hv.data(), ho.data(), hw.data()};
        for (int q = 0; q < 4; q++)
            CK(cudaMemcpyAsync(dst[q], src[q], sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaMemcpyAsync(ht.data(), type, (size_t)n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaMemcpyAsync(hi.data(), id, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        s->host = host_instance(s->prm, n, hp.data(), hv.data(), ho.data(), hw.data(), ht.data(), hi.data());
        s->have_particles = true;
        s->dirty = true;
        s->host_stale = false;
    });
}

int orbc_get_state_device(orbc_system* s, double* pos, double* vel, double* ori, double* angvel) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        if (!s->have_particles) throw StateError("no particles");
        sync_device(s);
        for (int b = 0; b < s->ens->B; b++) {
            const size_t o = (size_t)3 * s->ens->inst_h[b].id_base;
            s->ens->get_state_device(b, pos ? pos + o : nullptr, vel ? vel + o : nullptr, ori ? ori + o : nullptr,
                                     angvel ? angvel + o : nullptr);
        }
    });
}

int orbc_get_forces_device(orbc_system* s, double* force, double* torque) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        sync_device(s);
        if (!s->ens->forces_valid) throw StateError("forces not computed");
        for (int b = 0; b < s->ens->B; b++) {
            const size_t o = (size_t)3 * s->ens->inst_h[b].id_base;
            s->ens->get_forces_device(b, force ? force + o : nullptr, torque ? torque + o : nullptr);
        }
    });
}

int orbc_get_forces(orbc_system* s, double* force, double* torque) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        sync_device(s);
        if (!s->ens->forces_valid) throw StateError("forces not computed");
        for (int b = 0; b < s->ens->B; b++) {
            const size_t o = (size_t)3 * s->ens->inst_h[b].id_base;
            s->ens->get_forces(b, force ? force + o : nullptr, torque ? torque + o : nullptr);
        }
    });
}

int orbc_get_cells(orbc_system* s, int* cell_of_id, unsigned* slot_ids, double* centroids, int* cell_start,
                   double* radius, int* adj_ptr, int* adj) {
    if (!s) return ORBC_E_ARG;
    return guarded(s, [&] {
        sync_device(s);
        if (!s->ens->cells_valid) throw StateError("cells not initialised");
        s->ens->get_cells_all(cell_of_id, slot_ids, centroids, cell_start, radius, adj_ptr, adj);
    });
}

int orbc_get_adjacency_len(orbc_system* s, long long* len) {
    if (!s || !len) return ORBC_E_ARG;
    return guarded(s, [&] {
        sync_device(s);
        if (!s->ens->cells_valid) throw StateError("cells not initialised");
        *len = s->ens->adjacency_len_all();
    });
}

int orbc_dump_pairs(orbc_system* s, long long cap, unsigned* pairs, long long* npairs) {
    if (!s || !npairs || cap < 0) return ORBC_E_ARG;
    return guarded(s, [&] {
        sync_device(s);
        *npairs = s->ens->dump_pairs(0, cap, pairs);
    });
}

void orbc_default_mesh_params(orbc_mesh_params* mp) {
    if (!mp) return;
    std::memset(mp, 0, sizeof(*mp));
    mp->spacing = 1.12; mp->slack = 1.03; mp->kb = 100.0; mp->offset = 1.0; mp->d_min = 0.8; mp->d_ll = 0.2;
    mp->beads = 4; mp->seed = 0;
    mp->band3_fraction = 0.0; mp->kb_anchor = 50.0; mp->glycophorin = 0; mp->band3_edges = 0;
}

int orbc_quench(orbc_system* s, int nsteps, double dt, double max_move, double max_turn, double* fmax_out) {
    if (!s) return ORBC_E_ARG;
    if (nsteps < 0 || !(dt > 0) || !(max_move > 0) || !(max_turn > 0)) return fail(s, ORBC_E_ARG, "invalid quench");
    unsigned st = 0;
    double fm = 0.0;
    int rc = guarded(s, [&] {
        sync_device(s);
        if (!s->ens->cells_valid) throw StateError("cells not initialised");
        s->host_stale = true;
        fm = s->ens->quench(nsteps, dt, max_move, max_turn);
        st = s->ens->read_status(true);
        if (st) s->ens->forces_valid = false;
    });
    if (rc == ORBC_OK && st) return fail(s, status_code(st), "device status " + std::to_string(st));
    if (rc == ORBC_OK && fmax_out) *fmax_out = fm;
    return rc;
}

int orbc_set_volume_constraint(orbc_system* s, double kv, double v0, double area_per_lipid, const double* center) {
    if (!s) return ORBC_E_ARG;
    if (!center || !(kv >= 0) || !std::isfinite(kv) || !std::isfinite(v0) || !std::isfinite(area_per_lipid) ||
        !std::isfinite(center[0]) || !std::isfinite(center[1]) || !std::isfinite(center[2]))
        return fail(s, ORBC_E_ARG, "invalid volume constraint");
    if (kv > 0 && !(area_per_lipid > 0)) return fail(s, ORBC_E_ARG, "volume constraint needs a positive area per lipid");
    if (kv > 0 && (s->prm.periodic[0] || s->prm.periodic[1] || s->prm.periodic[2]))
        return fail(s, ORBC_E_ARG, "volume constraint needs a non-periodic box");
    for (int a = 0; a < 3; a++)
        if (!(std::fabs(center[a]) < 4096.0)) return fail(s, ORBC_E_ARG, "volume centre out of range");
    return guarded(s, [&] {
        HostInstance& h = s->host;
        h.vol_kv = kv;
        h.vol_v0 = v0;
        h.vol_area = area_per_lipid;
        for (int a = 0; a < 3; a++) h.vol_xc[a] = center[a];
        if (s->have_particles && !s->dirty) s->ens->set_volume(0, kv, v0, area_per_lipid, center);
    });
}

int orbc_get_volume(orbc_system* s, double area_per_lipid, const double* center, double* volume_out) {
    if (!s) return ORBC_E_ARG;
    if (!center || !volume_out || !std::isfinite(area_per_lipid)) return fail(s, ORBC_E_ARG, "invalid volume query");
    for (int a = 0; a < 3; a++)
        if (!(std::fabs(center[a]) < 4096.0)) return fail(s, ORBC_E_ARG, "volume centre out of range");
    if (!s->have_particles) return fail(s, ORBC_E_STATE, "no particles");
    double V = 0.0;
    unsigned st = 0;
    int rc = guarded(s, [&] {
        sync_device(s);
        V = s->ens->volume(0, area_per_lipid, center);
        st = s->ens->read_status(true);
    });
    if (rc == ORBC_OK && st) return fail(s, status_code(st), "device status " + std::to_string(st));
    if (rc == ORBC_OK) *volume_out = V;
    return rc;
}

int orbc_height_map(orbc_system* s, double x0, double y0, double dx, double dy, int nx, int ny, double z_min,
                    const double* axis, double rho_in, double rho_out, double* h_out, int* count_out) {
    if (!s) return ORBC_E_ARG;
    auto fin = [](double x) { return std::isfinite(x); };
    if (!axis || !h_out || !count_out || nx < 1 || ny < 1 || (long long)nx * ny > (1ll << 24) || !(dx > 0) ||
        !(dy > 0) || !fin(x0) || !fin(y0) || !fin(dx) || !fin(dy) || !fin(z_min) || !fin(axis[0]) || !fin(axis[1]) ||
        std::isnan(rho_in) || std::isnan(rho_out))
        return fail(s, ORBC_E_ARG, "invalid height map");
    if (!s->have_particles) return fail(s, ORBC_E_STATE, "no particles");
    return guarded(s, [&] {
        sync_device(s);
        s->ens->height_map(0, x0, y0, dx, dy, nx, ny, z_min, axis, rho_in, rho_out, h_out, count_out);
    });
}

int orbc_set_step_fusion(orbc_system* s, int on) {
    if (!s) return ORBC_E_ARG;
    s->ens->fuse_steps = on != 0;
    return ORBC_OK;
}

int orbc_set_wait_test(orbc_system* s, unsigned extra_tx_bytes, unsigned max_polls) {
    if (!s || max_polls < 1 || max_polls > (1u << 22) || extra_tx_bytes > 4096 || (extra_tx_bytes % 16) != 0)
        return ORBC_E_ARG;
    s->ens->extra_tx = extra_tx_bytes;
    s->ens->wait_polls = max_polls;
    return ORBC_OK;
}

int orbc_set_timing(orbc_system* s, int on) {
    if (!s) return ORBC_E_ARG;
    s->ens->timing = on != 0;
    s->ens->reset_times();
    return ORBC_OK;
}

int orbc_get_kernel_times(orbc_system* s, char* names_csv, int names_cap, float* ms, int cap, int* count) {
    if (!s || !count) return ORBC_E_ARG;
    auto& t = s->ens->kernel_times;
    *count = (int)t.size();
    std::string names;
    for (size_t q = 0; q < t.size(); q++) {
        if (q) names += ",";
        names += t[q].name + ":" + std::to_string(t[q].launches);
        if (ms && (int)q < cap) ms[q] = (float)t[q].ms;
    }
    if (names_csv && names_cap > 0) {
        std::strncpy(names_csv, names.c_str(), (size_t)names_cap - 1);
        names_csv[names_cap - 1] = 0;
    }
    return ORBC_OK;
}

int orbc_get_launch_count(orbc_system* s, long long* count) {
    if (!s || !count) return ORBC_E_ARG;
    *count = s->ens->launches;
    return ORBC_OK;
}

const char* orbc_last_error(const orbc_system* s) { return s ? s->err.c_str() : "null handle"; }

void orbc_destroy(orbc_system* s) {
    if (!s) return;
    if (s->ens) {
        cudaStreamSynchronize(s->stream);
        delete s->ens;
        cudaStreamSynchronize(s->stream);
        trim_pool();
    }
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
