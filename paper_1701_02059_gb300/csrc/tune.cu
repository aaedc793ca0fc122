// Autotuner of the cell-tile shape and of the pair evaluation's launch
// shape.  The tile is the number of particles per Voronoi cell (hence the
// number of centroids): a cell is the list search's CTA, which stages its
// neighbouring cells and searches its particles in groups of 32, and the
// rebuild's per-cell kernels work one warp per cell, so the cell size trades
// staging and search overheads against candidate counts.  The launch shape
// is the evaluation's occupancy, 5 or 7 CTAs per SM (compiled instances:
// more resident warps against a few spilled registers).  Every combination
// runs the real step (k-means initialisation, then timed steps) on a copy of
// the caller's system; the fastest is returned and, with a cache path,
// remembered for systems of the same shape.  The pair set does not depend on
// either choice, nor do the forces on the launch shape; with FP32 forces
// they do not depend on the cell size either (the mirrors' reference points
// are the centroids rounded to the mirror grid).
#include "abi_common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <fstream>
#include <mutex>
#include <sstream>

namespace orbc {

static const int kTileCandidates[] = {32, 45, 61, 80, 100};
static const int kEvalCtas[] = {5, 7};

// Shape of a system for the cache: particle, lipid, membrane-protein and bond
// counts, periodic axes and box, precision, and the extent of the particles
// (rounded).
static std::string tune_key(const HostInstance& h) {
    const int nl = (int)std::count(h.type.begin(), h.type.end(), (unsigned char)kLipid);
    const int nmp = (int)std::count_if(h.type.begin(), h.type.end(), [](unsigned char t) { return t >= kBand3; });
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < h.n; i++)
        for (int a = 0; a < 3; a++) {
            const double x = (double)h.xq[(size_t)3 * i + a] * kGridInv;
            lo[a] = std::min(lo[a], x);
            hi[a] = std::max(hi[a], x);
        }
    std::ostringstream k;
    k << "n=" << h.n << ",lipids=" << nl << ",bonds=" << h.r0.size() << ",prec=" << h.prm.precision;
    if (nmp) k << ",mp=" << nmp;
    for (int a = 0; a < 3; a++)
        k << ",p" << a << "=" << h.prm.periodic[a] << ":" << std::lround(h.prm.box[a]) << ":"
          << std::lround(hi[a] - lo[a]);
    return k.str();
}

static std::mutex g_tune_mu;

// "shape K ctas ms" lines (the last entry of a shape wins).
static bool cache_lookup(const char* path, const std::string& key, int& K, int& ctas, double& ms) {
    if (!path) return false;
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        std::istringstream ls(line);
        std::string k;
        int kk, cc;
        double m;
        if (ls >> k >> kk >> cc >> m && k == key && (cc == 5 || cc == 7)) { K = kk; ctas = cc; ms = m; found = true; }
    }
    return found;
}

static void cache_store(const char* path, const std::string& key, int K, int ctas, double ms) {
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    if (f) f << key << " " << K << " " << ctas << " " << ms << "\n";
}

// Milliseconds per step of h with K centroids and the evaluation at ctas
// CTAs per SM: initialisation and two warm-up steps untimed, then `steps`
// steps timed with events on the stream.
static double time_tile(const HostInstance& h, int K, int ctas, int steps, cudaStream_t st) {
    HostInstance c = h;
    c.prm.n_centroids = K;
    c.prm.eval_ctas = ctas;
    c.centroids.clear();
    Ensemble e(st);
    e.setup(c);
    e.init_cells();
    e.integrate(2);
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CK(cudaEventRecord(a, st));
    e.integrate(steps);
    CK(cudaEventRecord(b, st));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const unsigned status = e.read_status(true);
    if (status) throw StateError("trial with " + std::to_string(K) + " cells flagged status " + std::to_string(status));
    return (double)ms / steps;
}

}  // namespace orbc

using namespace orbc;

extern "C" int orbc_autotune(const orbc_params* params, int n, const double* pos, const double* vel, const double* ori,
                             const double* angvel, const unsigned char* type, const unsigned* id, int nb, const int* ij,
                             const double* r0, const double* kb, int steps, const char* cache_path,
                             int* n_centroids_out, int* eval_ctas_out, double* ms_per_step_out) {
    if (!params || !n_centroids_out || steps < 1) return ORBC_E_ARG;
    std::string err;
    return guarded_call(&err, [&] {
        Params P = to_params(params);
        check_params(P);
        if (P.n_protein_centroids > 0) throw ArgError("the autotuner takes no separate protein cells");
        HostInstance h = host_instance(P, n, pos, vel, ori, angvel, type, id);
        host_bonds(h, nb, ij, r0, kb);
        const std::string key = tune_key(h);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            int K = 0, ctas = 7;
            double ms = 0;
            if (cache_lookup(cache_path, key, K, ctas, ms)) {
                *n_centroids_out = K;
                if (eval_ctas_out) *eval_ctas_out = ctas;
                if (ms_per_step_out) *ms_per_step_out = ms;
                return;
            }
        }
        const int nl = (int)std::count_if(h.type.begin(), h.type.end(), bilayer);
        cudaStream_t st;
        CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        int bestK = -1, bestC = 7, lastK = -1;
        double best = 1e300;
        try {
            for (int ppc : kTileCandidates) {
                const int K = std::max(1, std::min(nl, (int)std::lround((double)n / ppc)));
                if (K == lastK) continue;        // small systems: sizes that round to the same count
                lastK = K;
                for (int ctas : kEvalCtas) {
                    const double ms = time_tile(h, K, ctas, steps, st);
                    if (ms < best) { best = ms; bestK = K; bestC = ctas; }
                }
            }
        } catch (...) {
            cudaStreamDestroy(st);
            throw;
        }
        cudaStreamDestroy(st);
        trim_pool();
        if (bestK < 1) throw ArgError("no lipid to seed a cell");
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            cache_store(cache_path, key, bestK, bestC, best);
        }
        *n_centroids_out = bestK;
        if (eval_ctas_out) *eval_ctas_out = bestC;
        if (ms_per_step_out) *ms_per_step_out = best;
    });
}
