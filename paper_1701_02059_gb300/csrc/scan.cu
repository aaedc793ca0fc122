// Device-wide exclusive prefix sum of int32 counts (cell histograms, grid
// occupancy, neighbour counts): per-block scan of 1024 elements, recursive
// scan of the block totals, then a uniform add.
#include "ensemble.cuh"

namespace orbc {

constexpr int kScanBlock = 1024;   // 256 threads x 4 elements

__global__ void k_scan_block(const int* __restrict__ in, int* __restrict__ out, long long n, int* __restrict__ sums) {
    __shared__ int warp_tot[8];
    long long base = (long long)blockIdx.x * kScanBlock + threadIdx.x * 4;
    int v[4];
    for (int q = 0; q < 4; q++) v[q] = (base + q < n) ? in[base + q] : 0;
    int t = v[0] + v[1] + v[2] + v[3];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = t;
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = (lane < 8) ? warp_tot[lane] : 0;
        for (int off = 1; off < 8; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, off);
            if (lane >= off) s += y;
        }
        if (lane < 8) warp_tot[lane] = s;
    }
    __syncthreads();
    int excl = x - t + (w > 0 ? warp_tot[w - 1] : 0);
    for (int q = 0; q < 4; q++) {
        if (base + q < n) out[base + q] = excl;
        excl += v[q];
    }
    if (threadIdx.x == blockDim.x - 1 && sums) sums[blockIdx.x] = warp_tot[7];
}

__global__ void k_scan_add(int* __restrict__ out, long long n, const int* __restrict__ offs) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / kScanBlock];
}

void Ensemble::scan_exclusive(const int* in, int* out, long long n) {
    if (n <= 0) return;
    long long nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 1) {
        k_scan_block<<<1, 256, 0, stream>>>(in, out, n, nullptr);
        launches++;
        CK(cudaGetLastError());
        return;
    }
    // scratch per recursion level, grown on demand
    int level = 0;
    std::vector<std::pair<int*, long long>> lv;
    long long m = nb;
    while (true) {
        if ((int)scan_tmp_.size() <= level) { scan_tmp_.push_back(nullptr); scan_tmp_n_.push_back(0); }
        if (scan_tmp_n_[level] < 2 * m + 2) {
            // stream-ordered pool memory: no device-wide synchronisation, as
            // a plain allocation and free would have
            if (scan_tmp_[level]) CK(cudaFreeAsync(scan_tmp_[level], stream));
            CK(cudaMallocAsync(&scan_tmp_[level], sizeof(int) * (2 * m + 2), stream));
            scan_tmp_n_[level] = 2 * m + 2;
        }
        lv.push_back({scan_tmp_[level], m});
        if (m <= kScanBlock) break;
        m = (m + kScanBlock - 1) / kScanBlock;
        level++;
    }
    // up: block scans producing sums at each level
    k_scan_block<<<(int)nb, 256, 0, stream>>>(in, out, n, lv[0].first);
    launches++;
    for (size_t l = 0; l + 1 < lv.size(); l++) {
        long long cnt = lv[l].second;
        int* sums = lv[l].first;
        int* scanned = lv[l].first + cnt + 1;
        long long nbl = (cnt + kScanBlock - 1) / kScanBlock;
        k_scan_block<<<(int)nbl, 256, 0, stream>>>(sums, scanned, cnt, lv[l + 1].first);
        launches++;
    }
    {
        size_t l = lv.size() - 1;
        long long cnt = lv[l].second;
        k_scan_block<<<1, 256, 0, stream>>>(lv[l].first, lv[l].first + cnt + 1, cnt, nullptr);
        launches++;
    }
    // down: add scanned offsets
    for (long long l = (long long)lv.size() - 2; l >= 0; l--) {
        long long cnt = lv[l].second;
        int* scanned = lv[l].first + cnt + 1;
        const int* offs = lv[l + 1].first + lv[l + 1].second + 1;
        k_scan_add<<<(int)((cnt + 255) / 256), 256, 0, stream>>>(scanned, cnt, offs);
        launches++;
    }
    k_scan_add<<<(int)((n + 255) / 256), 256, 0, stream>>>(out, n, lv[0].first + lv[0].second + 1);
    launches++;
    CK(cudaGetLastError());
}

}  // namespace orbc
