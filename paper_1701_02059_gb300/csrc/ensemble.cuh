// Host-side owner of a packed batch of instances (one or many membranes)
// and the launchers of every kernel of the hot path.  The plain C-ABI
// system is a batch of one; the batched arena packs many instances into the
// same arrays so every phase is one launch over all of them.
#pragma once
#include "orbc_internal.cuh"

#include <stdexcept>
#include <string>
#include <vector>

namespace orbc {

struct CudaError : std::runtime_error {
    cudaError_t code;
    CudaError(cudaError_t c, const std::string& what) : std::runtime_error(what), code(c) {}
};

#define CK(x)                                                                                                   \
    do {                                                                                                        \
        cudaError_t e_ = (x);                                                                                   \
        if (e_ != cudaSuccess)                                                                                  \
            throw ::orbc::CudaError(e_, std::string(cudaGetErrorString(e_)) + " at " + __FILE__ + ":" +         \
                                            std::to_string(__LINE__) + " (" #x ")");                            \
    } while (0)

struct ArgError : std::runtime_error {
    explicit ArgError(const std::string& w) : std::runtime_error(w) {}
};
struct StateError : std::runtime_error {
    explicit StateError(const std::string& w) : std::runtime_error(w) {}
};

// Physical and run parameters of one instance (mirrors orbc_params).
struct Params {
    double eps = 1, sigma = 1, rc_lipid = 2.6, mu = 3, sin_theta0 = 0;
    int zeta = 4;
    double eps_wca = 1, sigma_wca = 1, sigma_wca_pp = 0.5;
    double dt = 0.01, kT = 0.2, gamma_t = 1, gamma_r = 1, mass = 1, inertia = 1;
    double box[3] = {0, 0, 0};
    int periodic[3] = {0, 0, 0};
    int n_centroids = 64, n_lloyd_init = 10, rebuild_every = 1;
    double skin = 0, grid_h = 0;
    unsigned long long seed = 0;
    unsigned instance = 0;
    int precision = 0;   // 0 = FP32 forces, FP64 increments; 1 = FP64 everywhere; 2 = FP32 forces and increments
    int n_protein_centroids = 0;   // > 0: the proteins get a cell set of their own
    int eval_ctas = 7;             // pair evaluation launched for 5 or 7 CTAs per SM
    // bilayer species pairs [3 s_i + s_j] (lipid, band-3, glycophorin): the
    // lipid potential's well depth and cutoff, 0 = the lipid-lipid value
    double eps_mem[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, rc_mem[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

// One instance as given by the caller (host memory, id order not required).
// Allocator that leaves scalars uninitialised on resize: large host arrays
// that are filled right after they are sized.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
    template <typename U>
    struct rebind { using other = NoInitAlloc<U>; };
    NoInitAlloc() = default;
    template <typename U>
    NoInitAlloc(const NoInitAlloc<U>&) {}
    template <typename U>
    void construct(U* p) noexcept { ::new ((void*)p) U; }
    template <typename U, typename... A>
    void construct(U* p, A&&... a) { ::new ((void*)p) U(std::forward<A>(a)...); }
};
using GridVec = std::vector<long long, NoInitAlloc<long long>>;

struct HostInstance {
    Params prm;
    int n = 0;
    GridVec xq, vq, nq, wq;                  // [n][3] on the 2^-40 grid
    std::vector<unsigned char> type;
    std::vector<unsigned> id;
    std::vector<int> bonds;                  // [nb][2] ids
    std::vector<double> r0, kb;
    std::vector<double> centroids;           // optional initial centroids [K][3]
    long long step0 = 0;                     // steps already taken
    // harmonic volume constraint (kv = 0: off)
    double vol_kv = 0.0, vol_v0 = 0.0, vol_area = 0.0, vol_xc[3] = {0.0, 0.0, 0.0};
    // one cell set of a membrane split into lipid and protein cell sets:
    // the batch index of the other set (-1: none), the ids' offset in the
    // membrane, and whether every particle (not only the lipids) moves the
    // centroids
    int partner = -1, id_base = 0, all_members = 0;
};

// Bond list of one instance (ids local to the instance).
struct BondSpec {
    const std::vector<int>* bonds;
    const std::vector<double>* r0;
    const std::vector<double>* kb;
};

// One instance's carried state in device buffers of its own: what a packed
// batch needs to continue the instance bit for bit after it is re-packed
// (state, forces, centroids, cell ownership in the cell-sorted order).
struct Snapshot {
    Inst inst;                                // descriptor (p0, k0, g0 of the batch it came from)
    Params prm;
    int n = 0, K = 0;
    long long step = 0;
    std::vector<int> bonds;                   // host copy of the bond list
    std::vector<double> r0, kb;
    long long* state[4] = {nullptr, nullptr, nullptr, nullptr};   // x, v, n, w: [3][n]
    unsigned char* type = nullptr;
    unsigned* id = nullptr;
    int* cell = nullptr;                      // [n], local cell index
    int* cell_start = nullptr;                // [K + 1], local offsets
    long long* cq = nullptr;                  // [3][K]
    long long* F = nullptr;                   // [3][n]
    long long* T = nullptr;                   // [3][n]
    void* block = nullptr;                    // one device allocation holding all of the above
    size_t bytes = 0;
    cudaStream_t stream = nullptr;            // allocation and release are stream-ordered
    void allocate(int n_, int K_, cudaStream_t st);
    void release();
    ~Snapshot() { release(); }
};

// Releases the stream-ordered pool's cached blocks (after a system or arena
// is destroyed).
void trim_pool();

class Ensemble {
public:
    explicit Ensemble(cudaStream_t s);
    ~Ensemble();
    Ensemble(const Ensemble&) = delete;
    Ensemble& operator=(const Ensemble&) = delete;

    // set-up: particles and bonds of every instance; allocates everything
    void setup(const std::vector<const HostInstance*>& list);
    void setup(const HostInstance& h);
    // set-up from carried instances: continues each where it stopped
    void setup_from(const std::vector<const Snapshot*>& list);
    void export_instance(int b, Snapshot& s);
    size_t bytes_allocated() const { return bytes_; }
    // one step captured as a CUDA graph per state-buffer parity, replayed
    void integrate_graph(int nsteps);
    void init_cells();                       // seeding + Lloyd + reorder
    // one EM update + reorder; sums_ready: the B-A-O-A launch before it
    // already summed each cell's lipid displacements (d_msum, d_mcnt)
    void rebuild(bool sums_ready = false);
    void compute_forces(bool energies);
    void integrate(int nsteps);
    // velocity quench; returns the largest |F| at the end
    double quench(int nsteps, double dt, double max_move, double max_turn);
    void energies(std::vector<double>& out); // [B][5] after compute_forces(true)
    // volume constraint of instance b (kv = 0: off); forces become stale
    void set_volume(int b, double kv, double v0, double area, const double xc[3]);
    // enclosed volume of instance b for the given area per lipid and centre
    double volume(int b, double area, const double xc[3]);
    // upper-rim height map of instance b (host outputs of nx * ny)
    void height_map(int b, double x0, double y0, double dx, double dy, int nx, int ny, double z_min,
                    const double axis[2], double rho_in, double rho_out, double* h, int* count);

    // host copies (instance b, id order)
    void get_state(int b, double* pos, double* vel, double* ori, double* angvel, long long* step);
    void get_forces(int b, double* f, double* t);
    void get_state_device(int b, double* pos, double* vel, double* ori, double* angvel);
    // per-slot int64 array q of instance b to FP64 [n][3] in id order (device)
    void to_id_order(int b, const long long* q, double unit, double* out);
    void get_forces_device(int b, double* f, double* t);
    void get_cells(int b, int* cell_of_id, unsigned* slot_ids, double* centroids, int* cell_start, double* radius,
                   int* adj_ptr, int* adj);
    long long adjacency_len(int b);
    // every instance of the batch as one list (global cell numbers, ids offset by id_base)
    void get_cells_all(int* cell_of_id, unsigned* slot_ids, double* centroids, int* cell_start, double* radius,
                       int* adj_ptr, int* adj);
    long long adjacency_len_all();
    // the neighbour rows as CSR (adj_ptr, adj), built on demand for the getters
    void adjacency_csr();
    long long dump_pairs(int b, long long cap, unsigned* pairs);
    unsigned read_status(bool clear);
    std::vector<unsigned> read_instance_status(bool clear);
    void sync();

    // timing of individual kernels (CUDA events on the stream)
    bool timing = false;
    struct TimedKernel { std::string name; double ms = 0; int launches = 0; };
    std::vector<TimedKernel> kernel_times;
    void reset_times() { kernel_times.clear(); }

    int B = 0, N = 0, Ktot = 0;
    long long Gtot = 0;
    bool cells_valid = false, forces_valid = false;
    long long n_rebuilds = 0;
    long long launches = 0;               // kernels launched by this ensemble
    std::vector<Inst> inst_h;
    std::vector<Params> prm_h;
    std::vector<long long> step_h;
    cudaStream_t stream;
    int precision = 0;
    // pair and bond terms in FP64 (ORBC_F64_ALL), integrator increments in
    // FP32 (ORBC_F32_FORCE_F32_STEP)
    bool force_f64() const { return precision == 1; }
    bool step_f32() const { return precision == 2; }
    // the pair evaluation with bilayer species pairs and exclusions of
    // bilayer-cytoskeleton pairs: some instance holds band-3 or glycophorin,
    // or a bilayer particle with a bond
    bool any_mp() const {
        for (const Inst& I : inst_h)
            if (I.has_mp || I.bonded_bilayer) return true;
        return false;
    }

    View view();
    View view_alt();
    void swap_state();
    void scan_exclusive(const int* in, int* out, long long n);

    // phases
    void build_grid();
    void mstep(const int* cell_of) { mstep_iter(cell_of, -1); }
    // iter < 0: every instance updates; dmax (nullable): largest centroid move per instance
    void mstep_iter(const int* cell_of, int iter, unsigned* dmax = nullptr);
    bool displacement_exceeds_skin();
    void launch_kinetic();
    void estep(int* cell_out, float* lbound);       // grid search; lbound: second-nearest bounds
    void estep_bounded(int* cell);                  // k-means rounds after the first (bounds in d_lbound)
    void morton_relabel();
    void finish_cells();
    void launch_pairs(bool energies, bool dump);
    // the forces of the current positions with the next step's B-A-O-A (after
    // this step's final B) in the evaluation's epilogue; the new state lands
    // in the other buffer, which becomes current; msums: the epilogue takes
    // the M-step's sums for the next rebuild
    void launch_pairs_step(bool msums);
    void launch_volume_sum();                // D of every constrained instance into d_vol
    bool fuse_steps = false;                 // run each step's B-A-O-A in the previous step's force launch
    void launch_volume(bool energies);       // after the pair and bond forces
    void alloc_lists();
    void launch_integrate_first(bool fused, bool msums = false);
    void launch_kick(bool energies);
    void mirrors();

    // timing helpers
    struct Timer;
    void tic(const char* name);
    void toc();

private:
    void free_all();
    void alloc_core(const std::vector<int>& p0, const std::vector<int>& k0, bool any_skin);
    void upload_bonds(const std::vector<BondSpec>& bl, const std::vector<int>& p0);
    // fused: the previous step's final B is still due; baoa_done: this step's
    // B-A-O-A already ran in the previous step's force launch; eval_step: the
    // force launch also runs the next step's B-A-O-A
    void step_body(bool fused, bool baoa_done = false, bool eval_step = false);
    size_t bytes_ = 0;
    cudaGraphExec_t graph_[2] = {nullptr, nullptr};
    long long graph_launches_ = 0;
    template <typename T> T* alloc(size_t count);
    std::vector<void*> allocs_;
    int cur_ = 0;
    bool bbox_ready_ = false;   // set by the fused M-step of a rebuild
    bool csr_valid_ = false;        // d_adj_ptr / d_adj hold the current rows as CSR
    bool prev_adj_valid_ = false;   // the cell list of the previous rebuild can seed the E-step
    // timing state
    cudaEvent_t ev0_ = nullptr, ev1_ = nullptr;
    const char* open_ = nullptr;

public:
    // device arrays (see View for meanings)
    Inst* d_inst = nullptr;
    int *d_p0 = nullptr, *d_k0 = nullptr;
    long long* d_state[2][4] = {{nullptr}};
    unsigned char* d_type[2] = {nullptr, nullptr};
    unsigned* d_id[2] = {nullptr, nullptr};
    int* d_cell = nullptr;
    int* d_slot_of_id = nullptr;
    long long *d_F = nullptr, *d_T = nullptr, *d_Fbig = nullptr;
    int4* d_mq = nullptr;
    float4* d_mo = nullptr;
    int4* d_mqr = nullptr;     // mirrors in group-rank order (read by the pair kernel)
    float4* d_mor = nullptr;
    long long *d_cq = nullptr, *d_cq_tmp = nullptr;
    int* d_cell_start = nullptr;
    double* d_R = nullptr;
    float* d_Rf = nullptr;
    int *d_adj_ptr = nullptr, *d_adj = nullptr, *d_adjcount = nullptr;
    long long adj_cap = 0;
    int *d_gstart = nullptr, *d_gcount = nullptr, *d_gcent = nullptr, *d_gidx = nullptr;
    float4* d_gcf = nullptr;
    int *d_bptr = nullptr, *d_bpartner = nullptr;
    int nbond = 0;
    int2* d_bij = nullptr;
    int* d_binst = nullptr;
    float2* d_bkf = nullptr;
    double2* d_bkd = nullptr;
    unsigned wait_polls = 1u << 22;          // bounded staging waits (see View)
    unsigned extra_tx = 0;
    unsigned* d_status = nullptr;
    unsigned* d_istatus = nullptr;           // [B] flags raised by one instance's data
    long long* d_S = nullptr;
    long long* d_msum = nullptr;   // [3][Ktot] M-step sums from the B-A-O-A launch (zero between uses)
    int* d_mcnt = nullptr;         // [Ktot] lipids per cell, same
    int* d_cnt = nullptr;
    long long* d_bbox = nullptr;
    unsigned long long* d_keys = nullptr;
    void* d_sortrec = nullptr;
    int* d_new_of_old = nullptr;
    int *d_cell_new = nullptr, *d_perm = nullptr, *d_cell_tmp = nullptr;
    unsigned long long* d_rmax = nullptr;
    float* d_rho = nullptr;                  // [Ktot] distance to the nearest non-neighbour centroid
    float* d_lbound = nullptr;
    float* d_cmove = nullptr;                // [Ktot] k-means: move of each centroid in the last M-step
    unsigned* d_gmove = nullptr;             // [Gtot] k-means: largest move of the centroids in a grid cell               // [N] k-means: lower bound on the second-nearest centroid
    float4* d_cf = nullptr;                  // [Ktot] FP32 centroids by cell
    float4* d_cnorm = nullptr;               // [Ktot] cell normals (pair-kernel frames)
    unsigned char* d_grank = nullptr;        // [N] pair-kernel group ranks
    unsigned* d_dmax = nullptr;              // [B] largest centroid move of the last M-step (float bits)
    int* d_fbcount = nullptr;                // particles the certified E-step left to the grid search
    int* d_adjpad = nullptr;                 // [Ktot][64] neighbouring-cell rows before compaction
    int* d_seglist = nullptr;                // [2][Ktot] cells for the block sort / the rank sort
    int* d_seglist_n = nullptr;              // [2] their counts
    AdjDesc* d_adjd = nullptr;               // [adj_cap] staging descriptors of the rows
    float4* d_candrows = nullptr;            // [adj_cap] previous rows renumbered, with centroids (E-step)
    // neighbour lists of the split pair path (valid until the next reorder)
    int* d_nlist = nullptr;                  // [list_cap][N] entries (row << 26 | q), t-major
    int* d_ncnt = nullptr;                   // [N] listed pairs per particle (rank order)
    int2* d_novf = nullptr;                  // [ovf_cap] (q, entry) beyond list_cap
    int* d_novf_n = nullptr;                 // their count
    unsigned char* d_sflag = nullptr;        // [N] side-array contributions pending for the particle
    int4* d_rowoff = nullptr;                // [adj_cap] exact offset c_l - c_k of each row entry
    int list_cap = 0, ovf_cap = 0;
    bool list_valid = false;
    long long* d_xref = nullptr;
    long long* d_energy = nullptr;           // [B][8] fixed-point sums
    long long* d_vol = nullptr;              // [B][2] sum of (x - c).n (floors at 2^-24, remainders at 2^-48)
    bool vol_any = false;                    // some instance has the volume constraint on
    long long* d_step = nullptr;             // [B]
    unsigned* d_dump = nullptr;
    unsigned long long* d_dump_count = nullptr;
    long long dump_cap = 0;
    std::vector<int> n_lloyd_;
    std::vector<int*> scan_tmp_;
    std::vector<long long> scan_tmp_n_;
};

}  // namespace orbc
