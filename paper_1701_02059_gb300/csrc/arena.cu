// Batched arena: many independent membranes of uneven size resident on the
// device at once, packed into one set of arrays so that every phase of the
// time step (B-A-O-A, cell rebuild, forces, B) is one launch over all of
// them; the step loop is replayed from a CUDA graph.  Instances are admitted
// against an HBM budget while others run (continuous batching) and leave the
// batch when they have taken their steps.  Each instance is initialised
// exactly as a plain system is (k-means clustering, initial forces), and the
// batch only concatenates per-instance work, so an instance's trajectory is
// bit-identical alone and in any mix.
#include "abi_common.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <memory>
#include <mutex>
#include <system_error>
#include <thread>

namespace orbc {

// ---------------------------------------------------------------- snapshots
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

void Snapshot::allocate(int n_, int K_, cudaStream_t st) {
    release();
    stream = st;
    n = n_;
    K = K_;
    const size_t s_state = align256(sizeof(long long) * 3 * (size_t)n);
    const size_t s_u8 = align256((size_t)n);
    const size_t s_i32 = align256(sizeof(int) * (size_t)n);
    const size_t s_cs = align256(sizeof(int) * ((size_t)K + 1));
    const size_t s_cq = align256(sizeof(long long) * 3 * (size_t)K);
    bytes = 6 * s_state + s_u8 + 2 * s_i32 + s_cs + s_cq;
    if (cudaMallocAsync(&block, bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        block = nullptr;
        throw CudaError(cudaErrorMemoryAllocation, "snapshot allocation failed");
    }
    char* p = (char*)block;
    for (int q = 0; q < 4; q++) { state[q] = (long long*)p; p += s_state; }
    F = (long long*)p; p += s_state;
    T = (long long*)p; p += s_state;
    type = (unsigned char*)p; p += s_u8;
    id = (unsigned*)p; p += s_i32;
    cell = (int*)p; p += s_i32;
    cell_start = (int*)p; p += s_cs;
    cq = (long long*)p;
}

void Snapshot::release() {
    if (block) cudaFreeAsync(block, stream);
    block = nullptr;
    bytes = 0;
}

__global__ void k_offset(int* __restrict__ a, long long n, int delta) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] += delta;
}

__global__ void k_slot_of_id(View v) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= v.N) return;
    const int b = find_inst(v.inst_p0, v.B, p);
    v.slot_of_id[v.inst[b].p0 + (int)v.id[p]] = p;
}

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// defined with the plain system's getters: int64 fixed point of a slot range
// to FP64 [n][3] in id order
__global__ void k_to_id_order(const unsigned* __restrict__ id, const long long* __restrict__ q, size_t N, int p0, int n,
                              double unit, double* __restrict__ out);

static void d2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
}

void Ensemble::export_instance(int b, Snapshot& s) {
    if (!cells_valid || !forces_valid) throw StateError("instance has no cell list or forces to carry");
    const Inst& I = inst_h[b];
    const int n = I.n, K = I.K;
    s.allocate(n, K, stream);
    s.inst = I;
    s.prm = prm_h[b];
    s.step = step_h[b];
    for (int q = 0; q < 4; q++)
        for (int a = 0; a < 3; a++)
            d2d(s.state[q] + (size_t)a * n, d_state[cur_][q] + (size_t)a * N + I.p0, sizeof(long long) * n, stream);
    for (int a = 0; a < 3; a++) {
        d2d(s.F + (size_t)a * n, d_F + (size_t)a * N + I.p0, sizeof(long long) * n, stream);
        d2d(s.T + (size_t)a * n, d_T + (size_t)a * N + I.p0, sizeof(long long) * n, stream);
        d2d(s.cq + (size_t)a * K, d_cq + (size_t)a * Ktot + I.k0, sizeof(long long) * K, stream);
    }
    d2d(s.type, d_type[cur_] + I.p0, (size_t)n, stream);
    d2d(s.id, d_id[cur_] + I.p0, sizeof(unsigned) * n, stream);
    d2d(s.cell, d_cell + I.p0, sizeof(int) * n, stream);
    d2d(s.cell_start, d_cell_start + I.k0, sizeof(int) * (K + 1), stream);
    k_offset<<<nblk(n, 256), 256, 0, stream>>>(s.cell, n, -I.k0);
    k_offset<<<nblk(K + 1, 256), 256, 0, stream>>>(s.cell_start, K + 1, -I.p0);
    launches += 2;
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(stream));
}

void Ensemble::setup_from(const std::vector<const Snapshot*>& list) {
    free_all();
    B = (int)list.size();
    if (B < 1) throw ArgError("no instance");
    precision = list[0]->prm.precision;
    N = 0;
    Ktot = 0;
    inst_h.assign(B, Inst());
    prm_h.clear();
    step_h.assign(B, 0);
    std::vector<int> p0(B + 1, 0), k0(B + 1, 0);
    for (int b = 0; b < B; b++) {
        const Snapshot& s = *list[b];
        if (s.prm.precision != precision) throw ArgError("all instances of a batch need the same precision");
        if (s.prm.rebuild_every != 1) throw ArgError("carried instances must rebuild every step");
        inst_h[b] = s.inst;
        inst_h[b].p0 = N;
        inst_h[b].k0 = Ktot;
        prm_h.push_back(s.prm);
        step_h[b] = s.step;
        N += s.n;
        Ktot += s.K;
        p0[b + 1] = N;
        k0[b + 1] = Ktot;
    }
    alloc_core(p0, k0, false);
    Gtot = 0;
    for (int b = 0; b < B; b++) {
        inst_h[b].g0 = Gtot;
        Gtot += (long long)inst_h[b].gdim[0] * inst_h[b].gdim[1] * inst_h[b].gdim[2];
    }
    d_gstart = alloc<int>(Gtot + 1);
    d_gcount = alloc<int>(Gtot + 1);
    CK(cudaMemcpyAsync(d_inst, inst_h.data(), sizeof(Inst) * B, cudaMemcpyHostToDevice, stream));
    for (int b = 0; b < B; b++) {
        const Snapshot& s = *list[b];
        const int n = s.n, K = s.K;
        for (int q = 0; q < 4; q++)
            for (int a = 0; a < 3; a++)
                d2d(d_state[0][q] + (size_t)a * N + p0[b], s.state[q] + (size_t)a * n, sizeof(long long) * n, stream);
        for (int a = 0; a < 3; a++) {
            d2d(d_F + (size_t)a * N + p0[b], s.F + (size_t)a * n, sizeof(long long) * n, stream);
            d2d(d_T + (size_t)a * N + p0[b], s.T + (size_t)a * n, sizeof(long long) * n, stream);
            d2d(d_cq + (size_t)a * Ktot + k0[b], s.cq + (size_t)a * K, sizeof(long long) * K, stream);
        }
        d2d(d_type[0] + p0[b], s.type, (size_t)n, stream);
        d2d(d_id[0] + p0[b], s.id, sizeof(unsigned) * n, stream);
        d2d(d_cell + p0[b], s.cell, sizeof(int) * n, stream);
        k_offset<<<nblk(n, 256), 256, 0, stream>>>(d_cell + p0[b], n, k0[b]);
        // instance b's K + 1 offsets; the last one equals the next instance's first
        d2d(d_cell_start + k0[b], s.cell_start, sizeof(int) * (K + 1), stream);
        k_offset<<<nblk(K + 1, 256), 256, 0, stream>>>(d_cell_start + k0[b], K + 1, p0[b]);
        launches += 2;
    }
    k_slot_of_id<<<nblk(N, 256), 256, 0, stream>>>(view());
    launches++;
    CK(cudaGetLastError());
    std::vector<BondSpec> bl(B);
    for (int b = 0; b < B; b++) bl[b] = BondSpec{&list[b]->bonds, &list[b]->r0, &list[b]->kb};
    upload_bonds(bl, p0);
    // warm the scan scratch (outputs into arrays the next rebuild rewrites)
    scan_exclusive(d_gcount, d_gstart, Gtot + 1);
    scan_exclusive(d_cnt, d_adj_ptr, Ktot + 1);
    CK(cudaStreamSynchronize(stream));
    n_lloyd_.assign(B, 0);
    // the next step starts from the carried forces and ownership; its rebuild
    // recomputes the mirrors, radii and neighbouring cells
    cells_valid = true;
    forces_valid = true;
    list_valid = false;
}

// ---------------------------------------------------------------- graphs
void Ensemble::integrate_graph(int nsteps) {
    if (!cells_valid) throw StateError("cells not initialised");
    const bool eager = timing || d_xref != nullptr || prm_h[0].rebuild_every != 1;
    if (eager) {
        integrate(nsteps);
        return;
    }
    if (!forces_valid) {
        launch_pairs(false, false);
        forces_valid = true;
    }
    if (nsteps <= 0) return;
    // the first step runs eagerly (unfused; after a set-up it also seeds the
    // E-step from the grid search); the fused steps are graph replays
    step_body(false);
    for (auto& x : step_h) x++;
    for (int s = 1; s < nsteps; s++) {
        const int p = cur_;
        if (!graph_[p]) {
            const long long l0 = launches, r0 = n_rebuilds;
            cudaGraph_t g = nullptr;
            CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
            try {
                step_body(true);
            } catch (...) {
                cudaStreamEndCapture(stream, &g);
                if (g) cudaGraphDestroy(g);
                cur_ = p;
                throw;
            }
            CK(cudaStreamEndCapture(stream, &g));
            cudaError_t e = cudaGraphInstantiate(&graph_[p], g, 0);
            cudaGraphDestroy(g);
            CK(e);
            // capturing ran no kernel: restore the host-side state it advanced
            graph_launches_ = launches - l0;
            launches = l0;
            n_rebuilds = r0;
            cur_ = p;
        }
        CK(cudaGraphLaunch(graph_[p], stream));
        cur_ = p ^ 1;   // the step's gather swapped the state buffers
        launches += graph_launches_;
        n_rebuilds++;
        for (auto& x : step_h) x++;
    }
    launch_kick(false);
    forces_valid = true;
}

// ---------------------------------------------------------------- arena
struct ArenaSlot {
    // kFailed: the instance's own data raised a device flag (non-finite or
    // out-of-range forces, a particle beyond its cell's mirror range, ...);
    // it left the batch, the others continue
    enum { kFree = 0, kPending = 1, kResident = 2, kDone = 3, kFailed = 4 };
    int state = kFree;
    unsigned status = 0;     // the flags that failed it
    long long target = 0, done = 0;
    size_t bytes = 0;       // packed arrays of a batch of one + one snapshot
    long long n = 0;
    std::vector<int> bonds;  // host copy of the bond list (ids local to the instance)
    std::vector<double> r0, kb;
    std::unique_ptr<Snapshot> snap;   // carried state while pending or finished
};

// Device bytes that the set-up of one instance in a batch of one allocates
// whatever its geometry: per particle the state in two buffers (192),
// types and ids (10), cell and slot maps (8), forces, torques and the wide
// side array (96), mirrors (64), sort scratch, bounds and ranks (17) and the
// neighbour lists (132); per cell the neighbour rows at their fixed stride
// of 64 (4,096) and the per-cell arrays (258).  A lower bound of
// Ensemble::bytes_allocated(): the centroid grid, the bond lists and
// allocation rounding come on top.
static size_t instance_bytes_lower_bound(const HostInstance& h) {
    const size_t n = (size_t)h.n, K = (size_t)std::max(h.prm.n_centroids, 1);
    return n * 519 + K * 4354;
}

class Arena {
public:
    Arena(size_t budget, int precision, cudaStream_t st, bool own) :
        budget_(budget), precision_(precision), stream_(st), own_stream_(own) {
        CK(cudaGetDevice(&device_));
    }
    ~Arena() {
        batch_.reset();
        slots_.clear();
        cudaStreamSynchronize(stream_);
        trim_pool();
        if (own_stream_) cudaStreamDestroy(stream_);
    }

    size_t reserved() const {
        size_t s = 0;
        for (auto& x : slots_) if (x.state != ArenaSlot::kFree) s += x.bytes;
        return s;
    }

    static CudaError over_budget() { return CudaError(cudaErrorMemoryAllocation, "over the HBM budget"); }

    // Set-up, k-means initialisation and first forces of one instance on
    // stream st, carried out to a snapshot (a batch of one initialises the
    // instance exactly as a plain system does).  fits(b) is called with the
    // set-up's allocation once it is known and throws when that is over the
    // budget; *bytes receives the set-up's and the snapshot's bytes.
    template <typename Fits>
    std::unique_ptr<Snapshot> prepare(HostInstance& h, cudaStream_t st, size_t* bytes, Fits&& fits) {
        auto snap = std::make_unique<Snapshot>();
        Ensemble e(st);
        e.setup(h);
        *bytes = e.bytes_allocated();
        fits(*bytes);
        e.init_cells();
        e.compute_forces(false);
        const unsigned status = e.read_status(true);
        if (status) throw StateError("instance initialisation flagged status " + std::to_string(status));
        e.export_instance(0, *snap);
        *bytes += snap->bytes;
        return snap;
    }

    int commit(HostInstance& h, long long nsteps, std::unique_ptr<Snapshot> snap, size_t bytes) {
        int slot = -1;
        for (int i = 0; i < (int)slots_.size(); i++)
            if (slots_[i].state == ArenaSlot::kFree) { slot = i; break; }
        if (slot < 0) { slots_.emplace_back(); slot = (int)slots_.size() - 1; }
        ArenaSlot& S = slots_[slot];
        S.state = ArenaSlot::kPending;
        S.target = nsteps;
        S.done = 0;
        S.bytes = bytes;
        S.n = h.n;
        S.snap = std::move(snap);
        S.bonds = std::move(h.bonds);
        S.r0 = std::move(h.r0);
        S.kb = std::move(h.kb);
        dirty_ = true;
        return slot;
    }

    // Checks of an admission that need neither the device nor the budget.
    void precheck(const HostInstance& h, long long nsteps) const {
        if (nsteps < 1) throw ArgError("nsteps must be >= 1");
        if (h.prm.precision != precision_) throw ArgError("instance precision differs from the arena's");
        if (h.prm.rebuild_every != 1) throw ArgError("arena instances rebuild their cells every step");
        if (h.prm.n_centroids > (int)h.n) throw ArgError("more centroids than particles");
    }

    int admit(HostInstance& h, long long nsteps) {
        precheck(h, nsteps);
        // refuse from the sizes alone, before any device allocation, when the
        // arrays every set-up allocates already exceed the budget (the same
        // test as after the set-up, on a lower bound of its bytes); the exact
        // check follows the set-up
        const size_t lb = instance_bytes_lower_bound(h);
        if (reserved() + lb + lb / 2 > budget_) throw over_budget();
        size_t bytes = 0;
        auto snap = prepare(h, stream_, &bytes, [&](size_t b) {
            if (reserved() + b + b / 2 > budget_) throw over_budget();
        });
        if (reserved() + bytes > budget_) throw over_budget();
        return commit(h, nsteps, std::move(snap), bytes);
    }

    // Admits requests 0..count-1 in order with up to `threads` set-ups under
    // way at once, each on a stream of its own.  make(k) builds request k's
    // host instance (validation and quantisation, also in the workers).  The
    // budget tests are admit()'s, taken in request order: a set-up starts
    // when the committed instances, the set-ups under way and its own lower
    // bound fit, waits while set-ups ahead of it may still free room, and is
    // refused once none is ahead; a later request never takes room an
    // earlier one needs.  Stops at the first request that fails: returns its
    // index (count when all were admitted) with its code and message, and
    // discards the set-ups of the requests after it.
    template <typename Make>
    int admit_many(int count, int threads, Make&& make, const long long* nsteps, int* slots, int* code,
                   std::string* msg) {
        struct Cancelled {};
        std::mutex mu;
        std::condition_variable cv;
        std::vector<size_t> held(count, 0);   // reservation of each set-up under way
        int next = 0, gate = 0, committed = 0, failed = count;
        *code = ORBC_OK;
        // bytes held by the set-ups under way ahead of request k
        auto ahead = [&](int k) {
            size_t s = 0;
            for (int j = committed; j < k; j++) s += held[j];
            return s;
        };
        // waits until the committed instances, the set-ups ahead of k and
        // need fit; refuses once every request ahead of k is committed
        auto wait_for_room = [&](std::unique_lock<std::mutex>& lk, int k, size_t need) {
            for (;;) {
                if (failed < k) throw Cancelled{};
                if (reserved() + ahead(k) + need <= budget_) return;
                if (committed == k) throw over_budget();
                cv.wait(lk);
            }
        };
        // spawned workers make the arena's device current; the calling
        // thread keeps its own current device, as every other arena call does
        auto worker = [&](bool spawned) {
            cudaStream_t st = nullptr;
            if ((spawned && cudaSetDevice(device_) != cudaSuccess) ||
                cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                std::lock_guard<std::mutex> lk(mu);
                // a request this worker would have taken fails with the
                // CUDA error; others already taken finish
                if (next < count && next < failed) {
                    failed = next;
                    *code = ORBC_E_CUDA;
                    *msg = "could not create an admission stream";
                }
                cv.notify_all();
                return;
            }
            for (;;) {
                int k;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    if (next >= failed) break;   // failed <= count
                    k = next++;
                }
                std::string err;
                const int rc = guarded_call(&err, [&] {
                    try {
                        HostInstance h = make(k);
                        precheck(h, nsteps[k]);
                        const size_t lb = instance_bytes_lower_bound(h);
                        {
                            std::unique_lock<std::mutex> lk(mu);
                            cv.wait(lk, [&] { return gate == k || failed < k; });
                            try {
                                wait_for_room(lk, k, lb + lb / 2);
                            } catch (...) {
                                gate = k + 1;
                                cv.notify_all();
                                throw;
                            }
                            held[k] = lb + lb / 2;
                            gate = k + 1;
                            cv.notify_all();
                        }
                        size_t bytes = 0;
                        auto snap = prepare(h, st, &bytes, [&](size_t b) {
                            std::unique_lock<std::mutex> lk(mu);
                            wait_for_room(lk, k, b + b / 2);
                            held[k] = b + b / 2;
                        });
                        std::unique_lock<std::mutex> lk(mu);
                        cv.wait(lk, [&] { return committed == k || failed < k; });
                        if (failed < k) throw Cancelled{};
                        held[k] = 0;
                        if (reserved() + bytes > budget_) throw over_budget();
                        snap->stream = stream_;   // released later on the arena's stream
                        slots[k] = commit(h, nsteps[k], std::move(snap), bytes);
                        committed = k + 1;
                        cv.notify_all();
                    } catch (const Cancelled&) {
                    }
                });
                std::lock_guard<std::mutex> lk(mu);
                held[k] = 0;
                if (rc != ORBC_OK && k < failed) {
                    failed = k;
                    *code = rc;
                    *msg = err;
                }
                if (gate == k && rc != ORBC_OK) gate = k + 1;
                cv.notify_all();
            }
            cudaStreamSynchronize(st);
            cudaStreamDestroy(st);
        };
        threads = std::max(1, std::min(threads, count));
        std::vector<std::thread> pool;
        try {
            for (int t = 1; t < threads; t++) pool.emplace_back(worker, true);
        } catch (const std::system_error&) {
            // fewer workers: the ones started and this thread take every request
        }
        worker(false);
        for (auto& t : pool) t.join();
        return std::min(failed, committed);
    }

    // Steps every resident instance by min(max_steps, fewest steps left).
    int run(int max_steps, bool graphs) {
        if (max_steps < 1) throw ArgError("max_steps must be >= 1");
        const auto t0 = std::chrono::steady_clock::now();
        if (dirty_) {
            repack();
            repacks_++;
        }
        const auto t1 = std::chrono::steady_clock::now();
        repack_s_ += std::chrono::duration<double>(t1 - t0).count();
        if (!batch_) return 0;
        long long s = max_steps;
        for (int slot : batch_slot_) s = std::min(s, slots_[slot].target - slots_[slot].done);
        if (graphs) batch_->integrate_graph((int)s);
        else batch_->integrate((int)s);
        const unsigned st = batch_->read_status(true);
        if (st) {
            // flags that belong to single instances fail those instances
            // only: they leave the batch at the next re-pack and the others,
            // which never read another instance's data, have advanced
            // exactly as alone; anything else fails the whole call
            const std::vector<unsigned> ist = batch_->read_instance_status(true);
            bool attributed = false;
            for (unsigned x : ist) attributed |= (x != 0u);
            if ((st & ~kStatusPerInstance) || !attributed) {
                last_status_ = st;
                throw StateError("device status " + std::to_string(st));
            }
            for (int b = 0; b < (int)batch_slot_.size(); b++)
                if (ist[b]) {
                    ArenaSlot& S = slots_[batch_slot_[b]];
                    S.state = ArenaSlot::kFailed;
                    S.status = ist[b];
                    dirty_ = true;
                }
        }
        for (int b = 0; b < (int)batch_slot_.size(); b++) {
            ArenaSlot& S = slots_[batch_slot_[b]];
            if (S.state == ArenaSlot::kFailed) continue;
            S.done += s;
            if (S.done >= S.target) {
                S.snap = std::make_unique<Snapshot>();
                batch_->export_instance(b, *S.snap);
                S.state = ArenaSlot::kDone;
                dirty_ = true;
            }
        }
        step_s_ += std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
        steps_ += s;
        return (int)s;
    }

    void stats(double* repack_s, double* step_s, long long* repacks, long long* steps) const {
        if (repack_s) *repack_s = repack_s_;
        if (step_s) *step_s = step_s_;
        if (repacks) *repacks = repacks_;
        if (steps) *steps = steps_;
    }

    void poll(int* out, int cap, int* ndone) const {
        int k = 0;
        for (int i = 0; i < (int)slots_.size(); i++)
            if (slots_[i].state == ArenaSlot::kDone || slots_[i].state == ArenaSlot::kFailed) {
                if (out && k < cap) out[k] = i;
                k++;
            }
        *ndone = k;
    }

    void retire(int slot, double* pos, double* vel, double* ori, double* angvel, long long* step) {
        if (slot >= 0 && slot < (int)slots_.size() && slots_[slot].state == ArenaSlot::kFailed) {
            // a failed instance has no state to copy out: free its slot and
            // report its flags
            ArenaSlot& S = slots_[slot];
            const unsigned st = S.status;
            S.snap.reset();
            S.state = ArenaSlot::kFree;
            S.bytes = 0;
            S.status = 0;
            last_status_ = st;
            throw StateError("instance failed with device status " + std::to_string(st));
        }
        if (slot < 0 || slot >= (int)slots_.size() || slots_[slot].state != ArenaSlot::kDone)
            throw ArgError("slot is not finished");
        ArenaSlot& S = slots_[slot];
        const Snapshot& s = *S.snap;
        const int n = s.n;
        // to FP64 in id order on the device, then one copy per array
        double* outs[4] = {pos, vel, ori, angvel};
        double* tmp = nullptr;
        CK(cudaMallocAsync(&tmp, sizeof(double) * 12 * (size_t)std::max(n, 1), stream_));
        try {
            for (int q = 0; q < 4; q++) {
                if (!outs[q]) continue;
                double* t = tmp + (size_t)3 * q * n;
                k_to_id_order<<<nblk(n, 256), 256, 0, stream_>>>(s.id, s.state[q], (size_t)n, 0, n, kGridInv, t);
                launches_++;
                CK(cudaGetLastError());
                CK(cudaMemcpyAsync(outs[q], t, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, stream_));
            }
            CK(cudaStreamSynchronize(stream_));
        } catch (...) {
            cudaFreeAsync(tmp, stream_);
            throw;
        }
        CK(cudaFreeAsync(tmp, stream_));
        if (step) *step = s.step;
        S.snap.reset();
        S.state = ArenaSlot::kFree;
        S.bytes = 0;
    }

    void info(int* resident, int* pending, int* done, long long* particles, unsigned long long* bytes) const {
        int r = 0, p = 0, d = 0;
        long long np = 0;
        for (auto& x : slots_) {
            if (x.state == ArenaSlot::kResident) { r++; np += x.n; }
            if (x.state == ArenaSlot::kPending) p++;
            if (x.state == ArenaSlot::kDone || x.state == ArenaSlot::kFailed) d++;
        }
        if (resident) *resident = r;
        if (pending) *pending = p;
        if (done) *done = d;
        if (particles) *particles = np;
        if (bytes) *bytes = (unsigned long long)reserved();
    }

    // HBM bytes a slot holds against the budget (-1: no such slot).
    long long slot_bytes(int slot) const {
        if (slot < 0 || slot >= (int)slots_.size()) return -1;
        return slots_[slot].state == ArenaSlot::kFree ? 0 : (long long)slots_[slot].bytes;
    }

    long long launches() const { return launches_ + (batch_ ? batch_->launches : 0); }
    unsigned last_status_ = 0;
    std::string err;

private:
    // New batch = unfinished resident instances (carried) + pending ones.
    void repack() {
        std::vector<int> members;
        if (batch_) {
            for (int b = 0; b < (int)batch_slot_.size(); b++) {
                ArenaSlot& S = slots_[batch_slot_[b]];
                if (S.state != ArenaSlot::kResident) continue;
                S.snap = std::make_unique<Snapshot>();
                batch_->export_instance(b, *S.snap);
                members.push_back(batch_slot_[b]);
            }
            launches_ += batch_->launches;
            batch_.reset();
        }
        for (int i = 0; i < (int)slots_.size(); i++)
            if (slots_[i].state == ArenaSlot::kPending) members.push_back(i);
        batch_slot_.clear();
        dirty_ = false;
        if (members.empty()) return;
        std::vector<const Snapshot*> list;
        for (int i : members) {
            Snapshot* sp = slots_[i].snap.get();
            sp->bonds = slots_[i].bonds;
            sp->r0 = slots_[i].r0;
            sp->kb = slots_[i].kb;
            list.push_back(sp);
        }
        auto e = std::make_unique<Ensemble>(stream_);
        e->setup_from(list);
        for (int i : members) {
            slots_[i].state = ArenaSlot::kResident;
            slots_[i].snap.reset();   // the batch holds the state now
        }
        batch_ = std::move(e);
        batch_slot_ = members;
    }

    size_t budget_;
    int precision_;
    cudaStream_t stream_;
    bool own_stream_;
    int device_ = 0;
    std::unique_ptr<Ensemble> batch_;
    std::vector<int> batch_slot_;
    std::vector<ArenaSlot> slots_;
    bool dirty_ = false;
    long long launches_ = 0;
    double repack_s_ = 0.0, step_s_ = 0.0;    // host wall time inside re-packing / stepping
    long long repacks_ = 0, steps_ = 0;
};

}  // namespace orbc

// ============================================================== C ABI
using namespace orbc;

struct orbc_arena {
    Arena* a = nullptr;
    std::string err;
};

extern "C" {

int orbc_arena_create(unsigned long long hbm_budget_bytes, orbc_precision precision, void* cuda_stream,
                      orbc_arena** out) {
    if (!out) return ORBC_E_ARG;
    *out = nullptr;
    if (hbm_budget_bytes == 0 || (precision != ORBC_F32_FORCE_F64_STATE && precision != ORBC_F64_ALL &&
                                  precision != ORBC_F32_FORCE_F32_STEP))
        return ORBC_E_ARG;
    orbc_arena* h = new (std::nothrow) orbc_arena();
    if (!h) return ORBC_E_NOMEM;
    int rc = guarded_call(&h->err, [&] {
        cudaStream_t st = (cudaStream_t)cuda_stream;
        bool own = false;
        if (!st) {
            CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            own = true;
        }
        h->a = new Arena((size_t)hbm_budget_bytes, (int)precision, st, own);
    });
    if (rc != ORBC_OK) {
        delete h;
        return rc;
    }
    *out = h;
    return ORBC_OK;
}

int orbc_arena_admit(orbc_arena* h, const orbc_params* params, int n, const double* pos, const double* vel,
                     const double* ori, const double* angvel, const unsigned char* type, const unsigned* id, int nb,
                     const int* ij, const double* r0, const double* kb, long long nsteps, int* slot) {
    if (!h || !params || !slot) return ORBC_E_ARG;
    *slot = -1;
    return guarded_call(&h->err, [&] {
        Params P = to_params(params);
        check_params(P);
        if (P.n_protein_centroids > 0) throw ArgError("the arena takes no separate protein cells");
        HostInstance inst = host_instance(P, n, pos, vel, ori, angvel, type, id);
        host_bonds(inst, nb, ij, r0, kb);
        *slot = h->a->admit(inst, nsteps);
    });
}

int orbc_arena_admit_many(orbc_arena* h, const orbc_arena_request* req, int count, int threads, int* slots,
                          int* admitted) {
    if (!h || count < 0 || (count > 0 && (!req || !slots)) || !admitted) return ORBC_E_ARG;
    *admitted = 0;
    for (int k = 0; k < count; k++) slots[k] = -1;
    if (count == 0) return ORBC_OK;
    std::vector<long long> nsteps(count);
    for (int k = 0; k < count; k++) nsteps[k] = req[k].nsteps;
    int code = ORBC_OK;
    std::string msg;
    const int rc = guarded_call(&h->err, [&] {
        *admitted = h->a->admit_many(
            count, threads <= 0 ? 8 : std::min(threads, 16),
            [&](int k) {
                const orbc_arena_request& r = req[k];
                if (!r.params) throw ArgError("request without parameters");
                Params P = to_params(r.params);
                check_params(P);
                if (P.n_protein_centroids > 0) throw ArgError("the arena takes no separate protein cells");
                HostInstance inst = host_instance(P, r.n, r.pos, r.vel, r.ori, r.angvel, r.type, r.id);
                host_bonds(inst, r.nb, r.ij, r.r0, r.kb);
                return inst;
            },
            nsteps.data(), slots, &code, &msg);
    });
    if (rc != ORBC_OK) return rc;
    if (code != ORBC_OK) h->err = "request " + std::to_string(*admitted) + ": " + msg;
    return code;
}

int orbc_arena_run(orbc_arena* h, int max_steps, int use_graphs, int* steps_done) {
    if (!h) return ORBC_E_ARG;
    if (steps_done) *steps_done = 0;
    h->a->last_status_ = 0;
    int rc = guarded_call(&h->err, [&] {
        int s = h->a->run(max_steps, use_graphs != 0);
        if (steps_done) *steps_done = s;
    });
    if (rc == ORBC_E_STATE && h->a->last_status_) return status_code(h->a->last_status_);
    return rc;
}

int orbc_arena_poll(orbc_arena* h, int* done_slots, int cap, int* ndone) {
    if (!h || !ndone || cap < 0 || (cap > 0 && !done_slots)) return ORBC_E_ARG;
    h->a->poll(done_slots, cap, ndone);
    return ORBC_OK;
}

int orbc_arena_retire(orbc_arena* h, int slot, double* pos, double* vel, double* ori, double* angvel,
                      long long* step) {
    if (!h) return ORBC_E_ARG;
    h->a->last_status_ = 0;
    int rc = guarded_call(&h->err, [&] { h->a->retire(slot, pos, vel, ori, angvel, step); });
    if (rc == ORBC_E_STATE && h->a->last_status_) return status_code(h->a->last_status_);
    return rc;
}

int orbc_arena_info(const orbc_arena* h, int* resident, int* pending, int* done, long long* particles,
                    unsigned long long* bytes_reserved) {
    if (!h) return ORBC_E_ARG;
    h->a->info(resident, pending, done, particles, bytes_reserved);
    return ORBC_OK;
}

int orbc_arena_slot_bytes(const orbc_arena* h, int slot, unsigned long long* bytes) {
    if (!h || !bytes) return ORBC_E_ARG;
    const long long b = h->a->slot_bytes(slot);
    if (b < 0) return ORBC_E_ARG;
    *bytes = (unsigned long long)b;
    return ORBC_OK;
}

long long orbc_arena_launch_count(const orbc_arena* h) { return h ? h->a->launches() : -1; }

int orbc_arena_stats(const orbc_arena* h, double* repack_s, double* step_s, long long* repacks, long long* steps) {
    if (!h) return ORBC_E_ARG;
    h->a->stats(repack_s, step_s, repacks, steps);
    return ORBC_OK;
}

const char* orbc_arena_last_error(const orbc_arena* h) { return h ? h->err.c_str() : "null handle"; }

void orbc_arena_destroy(orbc_arena* h) {
    if (!h) return;
    delete h->a;
    delete h;
}

}  // extern "C"
