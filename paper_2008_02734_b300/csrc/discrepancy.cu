// Alignment discrepancy of two warping paths (Section 4.3, Results): for every
// cell (i, j) of path 1, the row error min |j - k| over the cells (i, k) of
// path 2 and the column error min |i - k| over its cells (k, j).
//
// A warping path never steps back, so its cells in row i are one run
// (i, rlo[i]) .. (i, rhi[i]) and its cells in column j one run clo[j] .. chi[j];
// a path from (0, 0) to (M-1, N-1) with unit steps visits every row and every
// column.  The row error of (i, j) is then max(0, rlo[i] - j, j - rhi[i]), and
// likewise for columns: one pass over path 2 records the runs (a cell is the
// first or last of its run when its neighbour in the path leaves the row or
// column), one pass over path 1 reads them.  Both passes check that their path
// is a warping path of the M x N problem before they touch the run arrays.
#include <algorithm>
#include <cstdint>

#include "dtw_common.cuh"
#include "dtw_kernels.h"

namespace dtwb {

namespace {

constexpr int kDiscThreads = 256;

// Is cell t of path P (K cells) a valid warping-path cell of the M x N problem:
// in range, the right endpoints, and a (0,1), (1,0) or (1,1) step from cell t-1?
__device__ __forceinline__ bool path_cell_ok(const int32_t* P, long long K, long long t, long long M, long long N,
                                             int& i, int& j) {
    i = P[2 * t];
    j = P[2 * t + 1];
    bool ok = i >= 0 && i < M && j >= 0 && j < N;
    if (t == 0) ok = ok && i == 0 && j == 0;
    if (t == K - 1) ok = ok && i == M - 1 && j == N - 1;
    if (t > 0) {
        const int di = i - P[2 * t - 2], dj = j - P[2 * t - 1];
        ok = ok && (di == 0 || di == 1) && (dj == 0 || dj == 1) && di + dj > 0;
    }
    return ok;
}

__global__ void __launch_bounds__(kDiscThreads)
    path_runs_kernel(const int32_t* __restrict__ P, long long K, long long M, long long N, int32_t* __restrict__ rlo,
                     int32_t* __restrict__ rhi, int32_t* __restrict__ clo, int32_t* __restrict__ chi,
                     int* __restrict__ status) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < K; t += (long long)gridDim.x * blockDim.x) {
        int i, j;
        if (!path_cell_ok(P, K, t, M, N, i, j)) {
            atomicOr(status, 2);
            continue;
        }
        if (t == 0 || P[2 * t - 2] != i) rlo[i] = j;
        if (t == K - 1 || P[2 * t + 2] != i) rhi[i] = j;
        if (t == 0 || P[2 * t - 1] != j) clo[j] = i;
        if (t == K - 1 || P[2 * t + 3] != j) chi[j] = i;
    }
}

__global__ void __launch_bounds__(kDiscThreads)
    discrepancy_kernel(const int32_t* __restrict__ P, long long K, long long M, long long N,
                       const int32_t* __restrict__ rlo, const int32_t* __restrict__ rhi,
                       const int32_t* __restrict__ clo, const int32_t* __restrict__ chi, int32_t* __restrict__ err,
                       int* __restrict__ status, int* __restrict__ max_err) {
    int local_max = 0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < K; t += (long long)gridDim.x * blockDim.x) {
        int i, j;
        if (!path_cell_ok(P, K, t, M, N, i, j)) {
            atomicOr(status, 1);
            err[t] = -1;
            err[K + t] = -1;
            continue;
        }
        const int re = max(0, max(rlo[i] - j, j - rhi[i]));
        const int ce = max(0, max(clo[j] - i, i - chi[j]));
        err[t] = re;
        err[K + t] = ce;
        local_max = max(local_max, max(re, ce));
    }
    local_max = __reduce_max_sync(0xffffffffu, (unsigned)local_max);
    if ((threadIdx.x & 31) == 0) atomicMax(max_err, local_max);
}

}  // namespace

size_t discrepancy_workspace_bytes(long long M, long long N) {
    return 256 + ((size_t)(2 * M + 2 * N) * sizeof(int32_t) + 255) / 256 * 256;
}

// P1, P2 and err on the device; ws holds discrepancy_workspace_bytes(M, N).
int path_discrepancy(const int32_t* P1, long long K1, const int32_t* P2, long long K2, long long M, long long N,
                     int32_t* err, int32_t* max_out, void* ws, int num_sms, cudaStream_t st) {
    int* status = static_cast<int*>(ws);  // [0] status bits, [1] max error
    int32_t* rlo = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + 256);
    int32_t* rhi = rlo + M;
    int32_t* clo = rhi + M;
    int32_t* chi = clo + N;
    if (cudaMemsetAsync(status, 0, 2 * sizeof(int), st) != cudaSuccess) return DTW_ECUDA;
    const long long cap = (long long)num_sms * 8;
    const unsigned g2 = (unsigned)std::max(1LL, std::min(cap, (K2 + kDiscThreads - 1) / kDiscThreads));
    const unsigned g1 = (unsigned)std::max(1LL, std::min(cap, (K1 + kDiscThreads - 1) / kDiscThreads));
    path_runs_kernel<<<g2, kDiscThreads, 0, st>>>(P2, K2, M, N, rlo, rhi, clo, chi, status);
    discrepancy_kernel<<<g1, kDiscThreads, 0, st>>>(P1, K1, M, N, rlo, rhi, clo, chi, err, status, status + 1);
    int h[2] = {0, 0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, status, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DTW_ECUDA;
    if (h[0]) return DTW_EINVAL;
    if (max_out) *max_out = h[1];
    return DTW_OK;
}

}  // namespace dtwb
