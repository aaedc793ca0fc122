// Standalone stable counting sort of items by cell id on device pointers:
// the particle level of the two-level reorder (arXiv 1701.02059, "Spatial
// Searching Algorithm": particles reordered by the Voronoi cell they belong
// to).  Same kernels as the cell-list rebuild: histogram, exclusive scan,
// atomic scatter, then each cell's slot list sorted by old index (warp
// bitonic up to 128, block bitonic up to 2048, exact rank beyond).
#include "ensemble.cuh"

#include <mutex>

#include "../../include/orbc.h"

namespace orbc {

// kernels defined in cells.cu
__global__ void k_hist(int N, const int* __restrict__ cell, int* __restrict__ cnt);
__global__ void k_scatter(int N, const int* __restrict__ cell, const int* __restrict__ start, int* __restrict__ cursor,
                          int* __restrict__ tmp);
__global__ void k_segsort_warp(int Ktot, const int* __restrict__ start, int* __restrict__ tmp);
__global__ void k_segsort(int Ktot, const int* __restrict__ start, int* __restrict__ tmp, unsigned* status);
__global__ void k_segrank(int N, const int* __restrict__ cell, const int* __restrict__ start, const int* __restrict__ tmp,
                          int* __restrict__ out);
__global__ void k_segcopy(int N, const int* __restrict__ cell, const int* __restrict__ start, const int* __restrict__ src,
                          int* __restrict__ tmp);

// Exclusive scan of m counts by one block: each thread sums a contiguous
// chunk, the block scans the chunk totals, each thread writes its chunk.
__global__ void k_scan_single(const int* __restrict__ in, int* __restrict__ out, int m) {
    __shared__ int tot[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int chunk = (m + T - 1) / T;
    const int b = t * chunk, e = min(m, b + chunk);
    int s = 0;
    for (int q = b; q < e; q++) s += in[q];
    tot[t] = s;
    __syncthreads();
    for (int off = 1; off < T; off <<= 1) {
        int x = (t >= off) ? tot[t - off] : 0;
        __syncthreads();
        tot[t] += x;
        __syncthreads();
    }
    int run = tot[t] - s;
    for (int q = b; q < e; q++) {
        int x = in[q];
        out[q] = run;
        run += x;
    }
}

__global__ void k_check_cells(const int* __restrict__ cell, int n, int K, unsigned* __restrict__ bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (cell[i] < 0 || cell[i] >= K)) atomicOr(bad, 1u);
}

static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// scratch: counts [K+1], cursor [K+1], tmp [n], flag [1]
void cell_sort_run(const int* d_cell, int n, int K, int* d_perm, int* d_start, cudaStream_t st, int* counts,
                   int* cursor, int* tmp, unsigned* flag) {
    CK(cudaMemsetAsync(counts, 0, sizeof(int) * (K + 1), st));
    CK(cudaMemsetAsync(cursor, 0, sizeof(int) * (K + 1), st));
    k_hist<<<nblk(n, 256), 256, 0, st>>>(n, d_cell, counts);
    k_scan_single<<<1, 1024, 0, st>>>(counts, d_start, K + 1);
    k_scatter<<<nblk(n, 256), 256, 0, st>>>(n, d_cell, d_start, cursor, d_perm);
    k_segsort_warp<<<nblk((long long)K * 32, 256), 256, 0, st>>>(K, d_start, d_perm);
    k_segsort<<<std::min(K, 1024), 256, 0, st>>>(K, d_start, d_perm, flag);
    k_segrank<<<nblk(n, 256), 256, 0, st>>>(n, d_cell, d_start, d_perm, tmp);
    k_segcopy<<<nblk(n, 256), 256, 0, st>>>(n, d_cell, d_start, tmp, d_perm);
    CK(cudaGetLastError());
}

bool cell_sort_cells_valid(const int* d_cell, int n, int K, cudaStream_t st, unsigned* flag) {
    CK(cudaMemsetAsync(flag, 0, sizeof(unsigned), st));
    k_check_cells<<<nblk(n, 256), 256, 0, st>>>(d_cell, n, K, flag);
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return h == 0;
}

}  // namespace orbc

extern "C" int orbc_cell_sort(const int* d_cell, int n, int K, int* d_perm, int* d_cell_start, void* cuda_stream) {
    using namespace orbc;
    if (n < 0 || K < 1 || (n > 0 && (!d_cell || !d_perm)) || !d_cell_start) return ORBC_E_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    void* buf = nullptr;
    try {
        const size_t bytes = sizeof(int) * ((size_t)2 * (K + 1) + (size_t)n + 1);
        if (cudaMallocAsync(&buf, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return ORBC_E_NOMEM;
        }
        int* counts = (int*)buf;
        int* cursor = counts + (K + 1);
        int* tmp = cursor + (K + 1);
        unsigned* flag = (unsigned*)(tmp + n);
        int rc = ORBC_OK;
        if (n > 0 && !cell_sort_cells_valid(d_cell, n, K, st, flag)) rc = ORBC_E_ARG;
        else if (n > 0) cell_sort_run(d_cell, n, K, d_perm, d_cell_start, st, counts, cursor, tmp, flag);
        else CK(cudaMemsetAsync(d_cell_start, 0, sizeof(int) * (K + 1), st));
        CK(cudaFreeAsync(buf, st));
        CK(cudaStreamSynchronize(st));
        return rc;
    } catch (const std::exception&) {
        if (buf) cudaFreeAsync(buf, st);
        return ORBC_E_CUDA;
    }
}

// ---------------------------------------------------------------------------
// Variant for callers that cannot allocate device memory: code running under
// a pool or arena allocator that owns the whole device, or inside a runtime
// that forbids cudaMalloc after start-up.  Its scratch is a fixed array in
// the library's own device memory, present on every device that loads the
// library until the process exits.
namespace orbc {
constexpr int kStaticMaxItems = 1 << 20;   // n <= 1,048,576
constexpr int kStaticMaxCells = 1 << 16;   // K <= 65,536
constexpr size_t kStaticInts = 2 * ((size_t)kStaticMaxCells + 1) + (size_t)kStaticMaxItems + 64;
static __device__ __align__(256) int g_cell_sort_scratch[kStaticInts];   // ~4.7 MB per device

// Host code may not use g_cell_sort_scratch as a device address: its host
// name is only a stand-in.  The device address is looked up with the device
// current (cudaGetSymbolAddress) on every call made outside stream capture,
// so a context that was reset or replaced since the last call is picked up;
// inside a capture the lookup may not run, and the address found by the last
// call outside capture on the same device is used.
static std::mutex g_scratch_mu;
static int* g_scratch_addr[64] = {nullptr};

static int* static_scratch(int dev, cudaStream_t st) {
    if (dev < 0 || dev >= 64) return nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        int* p = nullptr;
        if (cudaGetSymbolAddress((void**)&p, g_cell_sort_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}
}  // namespace orbc

extern "C" int orbc_cell_sort_noalloc(const int* d_cell, int n, int K, int* d_perm, int* d_cell_start,
                                      void* cuda_stream) {
    using namespace orbc;
    if (n < 0 || K < 1 || (n > 0 && (!d_cell || !d_perm)) || !d_cell_start) return ORBC_E_ARG;
    if (n > kStaticMaxItems || K > kStaticMaxCells) return ORBC_E_NOMEM;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return ORBC_E_CUDA; }
    int* base = static_scratch(dev, st);
    if (!base) return ORBC_E_CUDA;
    try {
        int* counts = base;
        int* cursor = counts + (K + 1);
        int* tmp = cursor + (K + 1);
        unsigned* flag = (unsigned*)(tmp + n);
        if (n > 0 && !cell_sort_cells_valid(d_cell, n, K, st, flag)) return ORBC_E_ARG;
        if (n > 0) cell_sort_run(d_cell, n, K, d_perm, d_cell_start, st, counts, cursor, tmp, flag);
        else CK(cudaMemsetAsync(d_cell_start, 0, sizeof(int) * (K + 1), st));
        CK(cudaStreamSynchronize(st));
        return ORBC_OK;
    } catch (const std::exception&) {
        return ORBC_E_CUDA;
    }
}
