/*
 * orbc.h -- C ABI of the GB300-native Voronoi-cell-list CGMD hot path of
 * OpenRBC (Tang, Lu, Li, Evangelinos, Grinberg, Sachdeva & Karniadakis,
 * arXiv 1701.02059).
 *
 * The calls follow the paper's statement of the problem: set up a system,
 * build the adaptive Voronoi cell list, evaluate forces and torques, and
 * advance positions and orientations ("Software Overview": time-stepping
 * loop of force and torque followed by the update of position and
 * orientation; "Spatial Searching Algorithm": group particles into adaptive
 * clusters, compute interactions between neighbouring clusters, update the
 * cluster composition, repeat).
 *
 * Conventions shared by every entry point:
 *   - Every call returns an orbc_status; no C++ exception crosses the ABI.
 *   - Pointers named host_* or documented as host pointers are read or
 *     written synchronously and stay owned by the caller.  The library owns
 *     every device allocation it makes and frees it in orbc_destroy /
 *     orbc_arena_destroy.
 *   - Arrays of 3-vectors are row-major [n][3] doubles.  Getters write in
 *     particle-id order (ids are 0..n-1).
 *   - Units are reduced: sigma (length), epsilon (energy), tau (time).
 *   - The state is held on a fixed-point grid of 2^-40 (sigma, sigma/tau,
 *     1, 1/tau): inputs are rounded to it (round-half-even) and every value
 *     read back is an exact double.
 *   - A failed call leaves the handle usable unless it returns
 *     ORBC_E_STATE; orbc_last_error() describes the last failure.
 *   - Calls on one handle are not thread-safe; distinct handles are
 *     independent.  Work is issued on the stream given at creation and every
 *     call that returns data to the host synchronises that stream.
 */
#ifndef ORBC_H
#define ORBC_H

#include <stddef.h>

#if defined(__GNUC__)
#define ORBC_API __attribute__((visibility("default")))
#else
#define ORBC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ORBC_OK = 0,
    ORBC_E_ARG = -1,       /* invalid argument (null pointer, size, NaN, range) */
    ORBC_E_NOMEM = -2,     /* device allocation failed or HBM budget exceeded   */
    ORBC_E_CUDA = -3,      /* CUDA runtime error                                */
    ORBC_E_STATE = -4,     /* call out of order, or the device state is invalid */
    ORBC_E_NAN = -5,       /* non-finite force or state detected on the device, or a
                              pair/bond term of 2^24 eps/sigma or more (beyond the
                              range of the 2^-32 fixed-point force sums)          */
    ORBC_E_TIMEOUT = -6    /* a bounded device wait gave up                     */
} orbc_status;

/* Arithmetic of the time step.  In every mode the state (x, v, n, w) is held
 * as int64 on the 2^-40 grid and forces, torques and energies are summed as
 * exact 2^-32 fixed point, so sums do not depend on the order of the terms. */
typedef enum {
    ORBC_F32_FORCE_F64_STATE = 0,  /* FP32 pair/bond forces; FP64 integrator increments (angular kicks,
                                      Ornstein-Uhlenbeck update, Cayley map, renormalisation; the
                                      translational kick, the drifts and the velocity's Ornstein-Uhlenbeck
                                      update as exact integer products of the int64 state with the FP64
                                      constants, rounded once) and FP64
                                      per-particle energy/virial partials                               */
    ORBC_F64_ALL = 1,              /* FP64 pair/bond forces and FP64 integrator increments             */
    ORBC_F32_FORCE_F32_STEP = 2    /* FP32 pair/bond forces and FP32 integrator increments (rounded onto
                                      the same int64 grid): the narrowest, fastest variant             */
} orbc_precision;

/* Particle types of the two-component red-cell model ("Initial structure
 * generation"): lipids carry an orientation; junctions (actin) and spectrin
 * beads are point particles joined by bonds; band-3 and glycophorin are
 * proteins of the bilayer and carry an orientation like the lipids.  A
 * band-3 joined by a bond to the spectrin is immobile, one without a bond
 * mobile; glycophorin is joined to the junctions.  Lipids, band-3 and
 * glycophorin are the "bilayer" particles. */
enum { ORBC_LIPID = 0, ORBC_JUNCTION = 1, ORBC_SPECTRIN = 2, ORBC_BAND3 = 3, ORBC_GLYCOPHORIN = 4 };

/*
 * Model, integrator and cell-list parameters.  orbc_default_params() fills
 * the values used throughout this project.
 *
 * Pair potential (the paper cites the two-component CGMD model without its
 * formulas; these follow the one-particle-thick lipid model it builds on,
 * Yuan et al., PRE 82, 011905, 2010).  With r_ij = x_i - x_j, rh = r_ij/r:
 *   a = (n_i x rh).(n_j x rh) + s0 (n_j - n_i).rh - s0^2, phi = 1 + mu (a - 1)
 *   U = eps[(rmin/r)^4 - 2 (rmin/r)^2] + (1 - phi) eps      r < rmin
 *   U = -eps cos^(2 zeta)((pi/2)(r - rmin)/(rc - rmin)) phi  rmin <= r < rc
 * with rmin = 2^(1/6) sigma.  Two bilayer particles (lipid, band-3,
 * glycophorin) interact through this potential with the well depth
 * eps_mem[s_i][s_j] and cutoff rc_mem[s_i][s_j] of their species pair
 * (s = 0 lipid, 1 band-3, 2 glycophorin; an entry of 0 takes eps or
 * rc_lipid; the paper names the proteins but prints none of the cited
 * model's constants, so the table is the caller's).  Every other pair is
 * purely repulsive WCA, 4 eps_wca [(s/r)^12 - (s/r)^6] + eps_wca for
 * r < 2^(1/6) s, with s = sigma_wca for bilayer-cytoskeleton pairs and
 * s = sigma_wca_pp for pairs of cytoskeleton proteins; pairs that are bonded
 * or share a bond partner (1-2, 1-3) are excluded from the WCA term (a
 * spectrin chain's beads, an anchored protein and its anchor), never from
 * the bilayer potential ("Force Evaluation": protein interactions use the
 * lipid cells with a wider search cutoff).
 *
 * Integrator: BAOAB Langevin (translational for all particles, rotational
 * for the bilayer's with Cayley rotations of the director), noise from
 * Philox4x32-10 keyed by (seed, instance; particle id, step, substream).
 */
typedef struct {
    double eps, sigma, rc_lipid, mu, sin_theta0;   /* lipid-lipid potential               */
    int zeta;                                      /* cos^(2 zeta) tail exponent           */
    int pad0;
    double eps_wca, sigma_wca;                     /* lipid-protein excluded volume        */
    double sigma_wca_pp;                           /* protein-protein excluded-volume size */
    double dt, kT, gamma_t, gamma_r, mass, inertia;/* integrator                           */
    double box[3];                                 /* box lengths on periodic axes         */
    int periodic[3];                               /* 1 = periodic axis                    */
    int n_centroids;                               /* Voronoi cells                        */
    int n_lloyd_init;                              /* k-means rounds at initialisation     */
    int rebuild_every;                             /* rebuild cadence in steps (>= 1)      */
    double skin;                                   /* neighbour skin (sigma), 0 = none     */
    double grid_h;                                 /* centroid-search grid edge, 0 = auto  */
    unsigned long long seed;
    unsigned instance;                             /* Philox key word, per ensemble member */
    orbc_precision precision;
    int n_protein_centroids;                       /* > 0: a separate cell set for the     */
                                                   /* proteins (detached cytoskeleton)     */
    int eval_ctas;                                 /* pair evaluation CTAs per SM: 5 or 7, */
                                                   /* 0 = 7 (launch shape; results equal)  */
    double eps_mem[3][3];                          /* bilayer species pairs: well depth,   */
    double rc_mem[3][3];                           /* cutoff; symmetric, >= 0, 0 = eps or  */
                                                   /* rc_lipid; [0][0] must be 0           */
} orbc_params;

typedef struct orbc_system orbc_system;   /* opaque; owns its device memory */

/* Fills p with the project's defaults: eps = sigma = 1, rc = 2.6, mu = 3,
 * zeta = 4, sin_theta0 = 0, eps_wca = sigma_wca = 1, sigma_wca_pp = 0.5,
 * dt = 0.01, kT = 0.2,
 * gamma_t = gamma_r = 1, mass = inertia = 1, no periodic axis,
 * n_centroids = 64, n_lloyd_init = 10, rebuild_every = 1, skin = 0,
 * grid_h = 0, seed = 0, instance = 0, ORBC_F32_FORCE_F64_STATE,
 * n_protein_centroids = 0, eval_ctas = 0, eps_mem = rc_mem = 0 (every bilayer
 * species pair as the lipid pair).  Errors of the table (orbc_create):
 * ORBC_E_ARG for a negative, non-finite or asymmetric entry, a nonzero [0][0]
 * entry, or a cutoff outside (2^(1/6) sigma, 64 sigma).
 *
 * Separate protein cells ("Force Evaluation": a cell whose cytoskeleton is
 * partly or fully detached from the bilayer gets a separate set of Voronoi
 * cells for its proteins): with n_protein_centroids = K_P > 0, cells
 * 0..K_L-1 (K_L = n_centroids) cluster the bilayer (lipids, band-3,
 * glycophorin) and K_L..K_L+K_P-1 the cytoskeleton's proteins; each
 * particle belongs to the nearest centroid of its own set, each centroid is
 * the mean of its own members, each set is numbered along its own Morton
 * curve, and the neighbouring-cell rule runs over both sets together, so the
 * pair search finds every type pair.  The ids must then be type-major (the
 * bilayer holds ids 0..N_L-1) and every bond joins two cytoskeleton proteins
 * (a detached network has no anchors); the arena does not take such
 * systems.  With shared cells (K_P = 0) the centroids are the means of the
 * bilayer particles. */
ORBC_API void orbc_default_params(orbc_params* p);

/* Creates a handle.  cuda_stream is a cudaStream_t (NULL = the library's own
 * non-blocking stream).  The device is the current CUDA device.
 * Errors: ORBC_E_ARG for null pointers or invalid parameters (non-positive
 * dt or box on a periodic axis, n_centroids < 1, rebuild_every < 1, skin > 0
 * required when rebuild_every > 1), ORBC_E_CUDA. */
ORBC_API int orbc_create(const orbc_params* params, void* cuda_stream, orbc_system** out);

/* Copies n particles from host memory ("Initial structure generation": the
 * system's particles with their types).  pos, vel: [n][3]; ori, angvel:
 * [n][3], read for bilayer particles only (ori must be unit, angvel is
 * projected perpendicular to it); type: [n] (ORBC_LIPID .. ORBC_GLYCOPHORIN); id: [n],
 * a permutation of 0..n-1.  The arrays are validated and copied on the host;
 * the device set-up (allocation, upload, bond lists) runs at the first call
 * that needs the device, which then reports its errors (ORBC_E_NOMEM,
 * ORBC_E_CUDA, and the bond limit of orbc_set_bonds as ORBC_E_ARG).
 * Invalidates cells and forces.
 * Errors: ORBC_E_ARG (null pointer, n < 1, non-finite value, |x| >= 4096
 * sigma, unknown type, ids not a permutation), ORBC_E_NOMEM. */
ORBC_API int orbc_set_particles(orbc_system* s, int n, const double* pos, const double* vel, const double* ori,
                       const double* angvel, const unsigned char* type, const unsigned* id);

/* Harmonic bonds 1/2 kb (r - r0)^2 between particle ids ("Force
 * Evaluation": a list of bonds between proteins is maintained).  ij: [nb][2]
 * ids; r0, kb: [nb].  At most 8 bonds per particle (checked when the device
 * lists are built, see orbc_set_particles).  Call after orbc_set_particles;
 * after steps the stepped state is kept.  Errors: ORBC_E_ARG (ids out of
 * range, a particle bonded to itself, negative or non-finite constants),
 * ORBC_E_STATE (no particles), ORBC_E_NOMEM. */
ORBC_API int orbc_set_bonds(orbc_system* s, int nb, const int* ij, const double* r0, const double* kb);

/* Initial k-means clustering ("Spatial Searching Algorithm"): centroids
 * [n_centroids][3] from host memory, or NULL to seed them from the bilayer
 * particles in id order (centroid k = bilayer particle floor(k N_L / K));
 * then n_lloyd_init rounds of
 * nearest-centroid assignment and centroid update; then the two-level
 * reorder (centroids along a Morton curve, particles stably by cell) and the
 * neighbouring-cell lists.  Errors: ORBC_E_ARG (more centroids than bilayer particles),
 * ORBC_E_STATE (no particles, or a cell with more than 64 neighbouring cells:
 * each cell's row is held at a fixed stride of 64, which a membrane with
 * about 60 particles per cell fills to about 8; a particle cloud in 3-D or a
 * large skin can exceed it, and fewer, larger cells bring it back),
 * ORBC_E_NOMEM, ORBC_E_CUDA. */
ORBC_API int orbc_init_cells(orbc_system* s, const double* centroids);

/* One update of the Voronoi cells ("Spatial Searching Algorithm": online EM
 * update of centroid location and particle ownership, then the two-level
 * reorder): centroid M-step from the current ownership, Morton relabel,
 * exact nearest-centroid E-step, stable counting sort of the particles and
 * their state, cell radii and neighbouring-cell lists.
 * Errors: ORBC_E_STATE (cells not initialised, or a cell with more than 64
 * neighbouring cells, as for orbc_init_cells), ORBC_E_CUDA. */
ORBC_API int orbc_rebuild_cells(orbc_system* s);

/* Forces and torques on every particle through the quad loop over cells,
 * neighbouring cells and their particles, plus bonds ("Force Evaluation").
 * energies_out (host, nullable): [U_pair, U_bond, K_trans, K_rot, W] with W
 * the virial sum of r_ij . F_ij over pairs and bonds.
 * Errors: ORBC_E_STATE (cells not initialised), ORBC_E_NAN, ORBC_E_CUDA. */
ORBC_API int orbc_compute_forces(orbc_system* s, double* energies_out);

/* Advances nsteps BAOAB steps ("Software Overview": force and torque, then
 * position and orientation update), rebuilding the cells every
 * rebuild_every steps or when a particle has moved more than the skin.
 * Errors: ORBC_E_ARG (nsteps < 0), ORBC_E_STATE (cells not initialised, or a
 * rebuild found a cell with more than 64 neighbouring cells), ORBC_E_NAN,
 * ORBC_E_CUDA. */
ORBC_API int orbc_integrate(orbc_system* s, int nsteps);

/* Host copies of the state in id order; any pointer may be NULL.  step:
 * number of steps taken. */
ORBC_API int orbc_get_state(orbc_system* s, double* pos, double* vel, double* ori, double* angvel, long long* step);

/* Forces and torques of the last force evaluation, in id order. */
ORBC_API int orbc_get_forces(orbc_system* s, double* force, double* torque);

/* Device-pointer variants (for callers whose arrays live on the GPU, e.g.
 * torch tensors; all on the handle's stream, which the call synchronises).
 * orbc_get_state_device / orbc_get_forces_device write [n][3] FP64 arrays
 * in id order with a kernel (no host round trip); any pointer may be NULL.
 * orbc_set_particles_device takes the arrays of orbc_set_particles in device
 * memory; they are read back once for the host-side validation and set-up
 * (a set-up cost, not a per-step one).  Errors as the host variants. */
ORBC_API int orbc_set_particles_device(orbc_system* s, int n, const double* pos, const double* vel, const double* ori,
                                       const double* angvel, const unsigned char* type, const unsigned* id);
ORBC_API int orbc_get_state_device(orbc_system* s, double* pos, double* vel, double* ori, double* angvel);
ORBC_API int orbc_get_forces_device(orbc_system* s, double* force, double* torque);

/* Cell list: cell_of_id [n]; slot_ids [n] (id stored at each storage slot,
 * the particle reorder); centroids [K][3]; cell_start [K+1]; radius [K];
 * adj_ptr [K+1] and adj [adj_len] (neighbouring cells, ascending, CSR).
 * Any pointer may be NULL; orbc_get_adjacency_len gives adj_len. */
ORBC_API int orbc_get_cells(orbc_system* s, int* cell_of_id, unsigned* slot_ids, double* centroids, int* cell_start,
                   double* radius, int* adj_ptr, int* adj);
ORBC_API int orbc_get_adjacency_len(orbc_system* s, long long* len);

/* Debug: every interacting pair found by the quad loop, as (id_lo, id_hi),
 * sorted; writes up to cap pairs to host memory and the total to *npairs. */
ORBC_API int orbc_dump_pairs(orbc_system* s, long long cap, unsigned* pairs, long long* npairs);

/* Sizes and timing of the last call: per-kernel device times in ms of the
 * last orbc_integrate / orbc_compute_forces when timing is on. */
ORBC_API int orbc_set_timing(orbc_system* s, int on);
ORBC_API int orbc_get_kernel_times(orbc_system* s, char* names_csv, int names_cap, float* ms, int cap, int* count);

/* Stable counting sort of n items by cell id on device memory (the particle
 * level of the two-level reorder, "Spatial Searching Algorithm": particles
 * reordered by the Voronoi cell they belong to).  d_cell: [n] cell ids in
 * [0, K), device memory.  Writes d_perm: [n], d_perm[new] = old index, the
 * items of one cell in their input order; and d_cell_start: [K+1], the first
 * slot of every cell.  Work is ordered on cuda_stream (NULL = the legacy
 * default stream); scratch is taken with cudaMallocAsync on that stream and
 * released before the call returns, and the call synchronises the stream.
 * Cost: O(n) for cells of up to 2,048 items (warp and block sorts); a cell
 * of m > 2,048 items is ordered by ranking every item against the others,
 * O(m^2) work for that cell (a single cell of 10^5 items takes 10^10
 * comparisons, of 10^6 items 10^12: keep cells small).
 * Errors: ORBC_E_ARG (null pointer, n < 0, K < 1, a cell id outside
 * [0, K)), ORBC_E_NOMEM, ORBC_E_CUDA. */
ORBC_API int orbc_cell_sort(const int* d_cell, int n, int K, int* d_perm, int* d_cell_start, void* cuda_stream);

/* orbc_cell_sort for callers that cannot allocate device memory (a pool or
 * arena allocator that owns the device, a runtime that forbids cudaMalloc
 * after start-up).  The paper has no counterpart; this is a deployment
 * variant.  Same arguments, results and errors as orbc_cell_sort; it calls
 * no allocator.  Its scratch is one fixed array of about 4.7 MB in the
 * library's device memory, present on every device that loads the library
 * until the process exits, which bounds the sizes: n <= 1,048,576 and
 * K <= 65,536, larger requests return ORBC_E_NOMEM.  Every call made while
 * its stream is not capturing looks up the array's device address with the
 * current device (cudaGetSymbolAddress), so a device reset or a new context
 * between calls is followed; make the first call on each device before any
 * stream capture.  A call made while its stream is capturing does not look
 * the address up: it reuses the one found by the last call on that device
 * (ORBC_E_CUDA if there was none), which is stale if the context was reset
 * or replaced since.  Every call reuses the same array
 * and zeroes what must start at zero; calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * Synchronises the stream. */
ORBC_API int orbc_cell_sort_noalloc(const int* d_cell, int n, int K, int* d_perm, int* d_cell_start,
                                    void* cuda_stream);

/* Test of the bounded waits (no counterpart in the paper).  Every wait of a
 * kernel on its shared-memory staging barrier gives up after a number of
 * polls (2^22 by default, well over a second), records a timeout that the
 * call returns as ORBC_E_TIMEOUT, waits (bounded again) for its copies and
 * leaves the kernel.  extra_tx_bytes (a multiple of 16, at most 4096; 0 in
 * normal use) makes each staging barrier expect that many bytes more than
 * the copies bring, so every copy lands but the barrier never completes and
 * the wait runs out; max_polls (1 .. 2^22) sets the limit.  The pair kernels
 * of the handle's next calls use these settings; orbc_set_wait_test(s, 0,
 * 1 << 22) restores normal operation.  A call that timed out leaves the
 * forces of that call invalid and the handle usable.  Errors: ORBC_E_ARG. */
ORBC_API int orbc_set_wait_test(orbc_system* s, unsigned extra_tx_bytes, unsigned max_polls);

/* ------------------------------------------------------------------------
 * Initial structure ("Initial structure generation": a two-component system
 * generated from a triangular mesh -- actin/glycophorin particles on the
 * vertices, spectrin along the edges, lipids placed at random on each face by
 * uniform sampling of the triangle, a minimum inter-particle distance, then
 * a velocity quench that removes collisions).
 */
typedef struct {
    double spacing;             /* lipid spacing s: one lipid per (sqrt(3)/2) s^2 of face area      */
    double slack;               /* chain bond rest length = slack |J_b - J_a| / (beads + 1)          */
    double kb;                  /* chain bond constant                                               */
    double offset;              /* protein network this far inside the surface (along vertex normals) */
    double d_min;               /* lipid candidates closer than this to a protein particle dropped   */
    double d_ll;                /* ... and closer than this to an earlier lipid candidate            */
    int beads;                  /* spectrin particles per mesh edge (0 .. 64)                         */
    int pad0;
    unsigned long long seed;    /* Philox key of the face counts and samples                          */
    double band3_fraction;      /* share of the face samples that are mobile band-3 (0 .. 1)          */
    double kb_anchor;           /* anchor bond constant (glycophorin-junction, band-3-spectrin)       */
    int glycophorin;            /* 1: a glycophorin on every vertex, bonded to its junction          */
    int band3_edges;            /* 1: an immobile band-3 on every edge, bonded to its chain (beads>0) */
} orbc_mesh_params;

/* Fills mp with spacing 1.12, slack 1.03, kb 100, offset 1, d_min 0.8,
 * d_ll 0.2, beads 4, seed 0, band3_fraction 0, kb_anchor 50, glycophorin 0,
 * band3_edges 0. */
ORBC_API void orbc_default_mesh_params(orbc_mesh_params* mp);

/* Builds the particles and bonds of a membrane on a triangular mesh, on the
 * GPU: verts [nv][3], faces [nf][3] vertex indices wound counter-clockwise
 * seen from outside (host arrays, copied).  Face f holds floor(A_f / a) +
 * [u < frac(A_f / a)] lipid candidates (a = (sqrt(3)/2) spacing^2, u a
 * Philox4x32-10 variate at counter (f, 0, 0, 2)); candidate k of face f is
 * ((1 - sqrt r1) p_a + sqrt r1 (1 - r2) p_b) + sqrt r1 r2 p_c with r1, r2
 * from counter (f, k, 0, 3), its director the face's unit normal.  Junctions
 * sit at v - offset n_v (n_v the normalised exact sum of the vertex's face
 * cross products); each undirected edge carries `beads` spectrin particles
 * evenly spaced between its junctions, chained by harmonic bonds.  A
 * candidate closer than d_min to a protein particle or closer than d_ll to
 * an earlier candidate is dropped.  The bilayer's proteins: with
 * glycophorin = 1 a glycophorin sits on every vertex (director n_v), bonded
 * to its junction; with band3_edges = 1 an immobile band-3 sits at the
 * midpoint (a + b) / 2 of every edge (director the normalised sum of the two
 * vertices' normal sums), bonded to the chain's bead floor((beads - 1) / 2);
 * each anchor's rest length is its length at construction, its constant
 * kb_anchor; candidate k of face f is a mobile band-3 instead of a lipid when
 * word 2 at counter (f, k, 0, 3), as (w + 1/2) 2^-32, is below
 * band3_fraction.  Glycophorin and edge band-3 count as protein particles
 * for d_min.  Output (host, id order): the kept face samples (lipids and
 * mobile band-3), the glycophorin (vertex order), the edge band-3 (edge
 * order), then the junctions (vertex order), then the spectrin (edge
 * order): pos, ori [n][3] (ori zero for the cytoskeleton), type [n]; bonds
 * [nb][2] ids (the chains', then the anchors, glycophorin's first), r0,
 * kb [nb].  *n_out and *nb_out always receive the totals; the arrays are
 * written when cap >= n and bond_cap >= nb (pass 0 to query the sizes).
 * The result does not depend on the launch shape.  cuda_stream: as in
 * orbc_cell_sort; the call synchronises it and frees its scratch.
 * Errors: ORBC_E_ARG (null pointer, vertex index out of range, a degenerate
 * face, non-finite or |x| >= 4096 coordinates, invalid parameters (also
 * band3_fraction outside [0, 1], a negative kb_anchor, band3_edges with no
 * beads), or a nonzero capacity smaller than the totals), ORBC_E_NOMEM,
 * ORBC_E_CUDA. */
ORBC_API int orbc_mesh_build(const orbc_mesh_params* mp, int nv, const double* verts, int nf, const int* faces,
                             long long cap, double* pos, double* ori, unsigned char* type, long long* n_out,
                             long long bond_cap, int* bonds, double* r0, double* kb, long long* nb_out,
                             void* cuda_stream);

/* Velocity quench of the handle's system (after orbc_init_cells): nsteps
 * steps of v += dt F/m, v replaced by its component along F (zero when it
 * points against F) and limited to |dt v| <= max_move, x += dt v; for bilayer particles
 * the same with w, the torque's part normal to the director and max_turn,
 * the director turned by the Cayley map of dt w; cells rebuilt and forces
 * evaluated every step.  Velocities and angular velocities are zero at the
 * end and the step counter does not move.  fmax_out (nullable): the largest
 * |F| after the last step.  Errors: ORBC_E_ARG (nsteps < 0, non-positive dt
 * or limits), ORBC_E_STATE (cells not initialised), ORBC_E_NAN, ORBC_E_CUDA. */
ORBC_API int orbc_quench(orbc_system* s, int nsteps, double dt, double max_move, double max_turn, double* fmax_out);

/* Whether each step's force launch also runs the next step's B-A-O-A update
 * in its epilogue (on = 1; FP32-force modes; default 0, separate launches).
 * Every particle's update needs only its own force, so the update could
 * overlap the pair evaluation of the other particles; on GB300 the fused
 * launch is slower (its state loads, permuted within the cell tiles, wait
 * with few resident warps).  Both settings give the same trajectory bit for
 * bit.  Errors: ORBC_E_ARG (null handle). */
ORBC_API int orbc_set_step_fusion(orbc_system* s, int on);

/* Harmonic volume constraint on the handle's membrane ("Validation and
 * Benchmark": the whole-cell run holds its surface-to-volume ratio by a
 * harmonic volume constraint; the paper states no functional form, so the
 * enclosed volume is taken from the bilayer particles (lipids and membrane
 * proteins) by the divergence theorem with each one's director as its
 * surface normal):
 *   V = sum over the bilayer of (a / 3) (x_i - c) . n_i,   U_V = k_V (V - V0)^2 / 2,
 * a = area_per_lipid (sigma^2, the area per bilayer particle), c = center
 * (sigma, a fixed point inside the membrane).  U_V acts as the uniform
 * pressure P = -k_V (V - V0) on each area element: the force P a n_i and no torque (moving one element
 * by delta along its normal changes the enclosed volume by a delta; a
 * uniform pressure has no moment about the element).  U_V is added to the
 * bond energy (energies[1]) and nothing to the virial.  Each (x_i - c).n_i
 * is rounded to 2^-48 sigma before an exact integer sum, so V does not
 * depend on the order; (x_i - c).n_i is FP32 in the FP32-force modes and
 * FP64 otherwise (and in orbc_get_volume), the factor a/3 and the pressure
 * FP64, the force P a n_i FP32 or FP64 as the pair forces.  kv = 0 switches the
 * constraint off; the setting survives later orbc_set_particles calls.
 * Errors: ORBC_E_ARG (null center, kv < 0, non-finite values, a
 * non-positive area with kv > 0, a periodic axis with kv > 0), ORBC_E_CUDA. */
ORBC_API int orbc_set_volume_constraint(orbc_system* s, double kv, double v0, double area_per_lipid,
                                        const double* center);

/* The enclosed volume V of the current state (the sum above) for the given
 * area per lipid and center, whether or not the constraint acts.
 * Errors: ORBC_E_ARG (null pointer, non-finite values), ORBC_E_STATE (no
 * particles), ORBC_E_CUDA. */
ORBC_API int orbc_get_volume(orbc_system* s, double area_per_lipid, const double* center, double* volume_out);

/* Height map of the membrane's upper rim for the fluctuation measurement
 * ("Validation and Benchmark": the instantaneous vertical fluctuation
 * dh(x, y) along the upper rim of a cell held in place): the bilayer particles with
 * z > z_min whose distance rho from the vertical axis through (axis[0],
 * axis[1]) lies in [rho_in, rho_out) are binned on the grid
 * x in [x0 + i dx, x0 + (i + 1) dx), y in [y0 + j dy, ...), i < nx, j < ny;
 * h_out[j nx + i] = their mean z (0 for an empty bin), count_out[j nx + i]
 * their number (both host arrays of nx ny).  Every selection and bin index
 * is decided in FP64 from the exact state with correctly rounded operations;
 * z is summed exactly as an integer on the state grid.  dh over time is h
 * minus its time mean, bin by bin.  Errors: ORBC_E_ARG (null pointer,
 * nx or ny < 1, nx ny > 2^24, non-positive dx or dy, non-finite values),
 * ORBC_E_STATE (no particles), ORBC_E_CUDA. */
ORBC_API int orbc_height_map(orbc_system* s, double x0, double y0, double dx, double dy, int nx, int ny, double z_min,
                             const double* axis, double rho_in, double rho_out, double* h_out, int* count_out);

/* Number of CUDA kernels this handle has launched since creation. */
ORBC_API int orbc_get_launch_count(orbc_system* s, long long* count);

ORBC_API const char* orbc_last_error(const orbc_system* s);
ORBC_API void orbc_destroy(orbc_system* s);

/* Autotuner of the cell-tile shape and the pair evaluation's launch shape
 * (no counterpart in the paper, which fixes the cell count by hand): times
 * the real step ("Spatial Searching Algorithm" + "Force Evaluation":
 * initialisation, then `steps` timed steps) of a copy of the given system
 * for each particles-per-cell size (32, 45, 61, 80, 100) and each pair
 * evaluation occupancy (5 or 7 CTAs per SM, compiled instances of the
 * kernel), and writes the fastest centroid count to *n_centroids_out, its
 * CTAs per SM to *eval_ctas_out (nullable) and its ms per step to
 * *ms_per_step_out (nullable).  Arrays as in orbc_set_particles /
 * orbc_set_bonds (host, copied); params->n_centroids and ->eval_ctas are
 * ignored.  cache_path (nullable): a text file of "shape K ctas ms" lines; a
 * system of the same shape (counts, periodic box, precision, extent) is
 * answered from it without timing, and new results are appended.
 * Errors: ORBC_E_ARG, ORBC_E_NOMEM, ORBC_E_CUDA, ORBC_E_STATE. */
ORBC_API int orbc_autotune(const orbc_params* params, int n, const double* pos, const double* vel, const double* ori,
                           const double* angvel, const unsigned char* type, const unsigned* id, int nb, const int* ij,
                           const double* r0, const double* kb, int steps, const char* cache_path,
                           int* n_centroids_out, int* eval_ctas_out, double* ms_per_step_out);

/* ------------------------------------------------------------------------
 * Batched arena and continuous batching.  The paper runs one membrane per
 * process; these calls have no counterpart in it.  They keep many
 * independent instances resident on the device, packed into one set of
 * arrays, so each phase of the time step ("Software Overview", flow chart)
 * is one launch over all of them; the step loop is replayed from a CUDA
 * graph.  An instance is initialised exactly as orbc_init_cells +
 * orbc_compute_forces would, and its trajectory is bit-identical to the
 * plain system's whatever else shares the batch.
 *
 * Typical loop: admit instances (at any time, also while others run), call
 * orbc_arena_run repeatedly, poll for finished slots, retire them.
 */
typedef struct orbc_arena orbc_arena;   /* opaque; owns its device memory */

/* hbm_budget_bytes bounds the device memory reserved by admitted instances
 * (packed arrays plus one carried copy each, which a re-pack needs).  All
 * instances share one precision (any orbc_precision).  cuda_stream as in
 * orbc_create.
 * Errors: ORBC_E_ARG (budget 0, unknown precision, null out), ORBC_E_CUDA. */
ORBC_API int orbc_arena_create(unsigned long long hbm_budget_bytes, orbc_precision precision, void* cuda_stream,
                               orbc_arena** out);

/* Admits one instance that will take nsteps steps: the same host arrays as
 * orbc_set_particles and orbc_set_bonds (copied; the caller keeps them).
 * The instance is initialised on the device now (k-means clustering and
 * initial forces) and joins the batch at the next orbc_arena_run.  params
 * must have rebuild_every = 1 and the arena's precision.  *slot receives
 * the slot number used by poll and retire.
 * Errors: ORBC_E_NOMEM when the instance does not fit the remaining budget
 * (nothing is kept; admit again after retiring others), ORBC_E_ARG, ORBC_E_CUDA. */
ORBC_API int orbc_arena_admit(orbc_arena* a, const orbc_params* params, int n, const double* pos, const double* vel,
                              const double* ori, const double* angvel, const unsigned char* type, const unsigned* id,
                              int nb, const int* ij, const double* r0, const double* kb, long long nsteps, int* slot);

/* One request of orbc_arena_admit_many: orbc_arena_admit's arguments. */
typedef struct orbc_arena_request {
    const orbc_params* params;
    int n;
    const double* pos;
    const double* vel;
    const double* ori;
    const double* angvel;
    const unsigned char* type;
    const unsigned* id;
    int nb;
    const int* ij;
    const double* r0;
    const double* kb;
    long long nsteps;
} orbc_arena_request;

/* Admits req[0..count) in order, as orbc_arena_admit would one after the
 * other, with up to `threads` of them (<= 0: 8; at most 16) validated,
 * quantised and initialised at once on host threads of the library, each
 * with a CUDA stream of its own.  The budget test is orbc_arena_admit's,
 * taken in request order: a request's initialisation starts only when it
 * fits beside the admitted instances and the initialisations under way
 * ahead of it, and it is refused only when it does not fit once every
 * request ahead of it is admitted.  Stops at the first request that fails:
 * *admitted receives the number admitted (always a prefix of req), slots[k]
 * the slot of request k (-1 from *admitted on), and the return value is the
 * failing request's error (ORBC_OK when all were admitted); initialisations
 * of later requests already under way are discarded.  The caller keeps its
 * arrays; calls on one arena must not overlap.
 * Errors: ORBC_E_NOMEM (budget), ORBC_E_ARG (null req, slots or admitted,
 * count < 0, or a request's own argument errors), ORBC_E_STATE, ORBC_E_CUDA. */
ORBC_API int orbc_arena_admit_many(orbc_arena* a, const orbc_arena_request* req, int count, int threads, int* slots,
                                   int* admitted);

/* Re-packs the batch if instances were admitted or finished, then advances
 * every resident instance by s = min(max_steps, fewest steps any of them has
 * left) steps (use_graphs != 0: replay of a captured step).  Instances that
 * reach their step count leave the batch and become finished.  *steps_done
 * (nullable) receives s (0 when nothing is resident).
 * An instance whose own data raises a device flag during the call (non-
 * finite or out-of-range pair or bond terms, a particle beyond the mirror
 * range of its cell, a cell with more than 64 neighbouring cells) fails
 * alone: it is reported by orbc_arena_poll, leaves the batch, and
 * orbc_arena_retire returns its error; the other instances advance exactly
 * as they would alone and the call returns ORBC_OK.  Failures are detected
 * at the end of the call, so a failed instance may have stepped on garbage
 * for up to max_steps steps; a small max_steps narrows that.
 * Errors: ORBC_E_TIMEOUT and the shared neighbour-list overflow (ORBC_E_STATE)
 * fail the whole call; ORBC_E_ARG (max_steps < 1), ORBC_E_CUDA. */
ORBC_API int orbc_arena_run(orbc_arena* a, int max_steps, int use_graphs, int* steps_done);

/* Finished or failed slots: up to cap slot numbers into done_slots, their
 * count into *ndone.  Errors: ORBC_E_ARG. */
ORBC_API int orbc_arena_poll(orbc_arena* a, int* done_slots, int cap, int* ndone);

/* Copies a finished instance's state out in id order (pos, vel, ori, angvel:
 * [n][3], each nullable; step: nullable) and frees its slot and memory.  For
 * a failed slot it copies nothing, frees the slot and returns the failure
 * (ORBC_E_NAN for non-finite or out-of-range terms, ORBC_E_STATE otherwise).
 * Errors: ORBC_E_ARG (slot not finished), ORBC_E_CUDA. */
ORBC_API int orbc_arena_retire(orbc_arena* a, int slot, double* pos, double* vel, double* ori, double* angvel,
                               long long* step);

/* HBM bytes slot `slot` holds against the budget (its share of the batch
 * and, while it waits or has finished, its snapshot): 0 for a free slot.
 * Errors: ORBC_E_ARG (null handle or bytes, slot out of range). */
ORBC_API int orbc_arena_slot_bytes(const orbc_arena* a, int slot, unsigned long long* bytes);

/* Counts of resident, pending (admitted, not yet packed) and finished
 * instances, resident particles and reserved bytes; each output nullable. */
ORBC_API int orbc_arena_info(const orbc_arena* a, int* resident, int* pending, int* done, long long* particles,
                             unsigned long long* bytes_reserved);

/* Kernels the arena has launched so far (graph replays count each kernel). */
ORBC_API long long orbc_arena_launch_count(const orbc_arena* a);

/* Host wall time spent re-packing the batch and stepping it (including the
 * export of finished instances), the number of re-packs and of batched steps
 * so far; each output nullable.  Errors: ORBC_E_ARG. */
ORBC_API int orbc_arena_stats(const orbc_arena* a, double* repack_s, double* step_s, long long* repacks,
                              long long* steps);

/* Message of the last failed arena call ("" if none). */
ORBC_API const char* orbc_arena_last_error(const orbc_arena* a);

/* Frees the arena, its batch and every slot (NULL is ignored). */
ORBC_API void orbc_arena_destroy(orbc_arena* a);

#ifdef __cplusplus
}
#endif

#endif /* ORBC_H */
