// The paper's own GPU form, kept as the comparator of the tiled path: Algorithm 1
// (DiagDTW) with one kernel launch per anti-diagonal and one thread per cell,
// three rotating diagonal buffers in global memory, FP64 frame costs and FP64
// accumulation, driven by Algorithm 2 on the host -- forward sweep to the
// central diagonals, backward sweep of the reversed series, F + B - C argmin over
// three central diagonals (Lemmas 1 and 2), depth-first recursion, and textbook
// DTW (Section 2.1) once a box side drops below m = 500 (Section 3.2).
//
// The frame cost is evaluated exactly like a CPU FP64 reference would
// (dimensions in order, separate multiply and add, correctly rounded sqrt).
#include <cmath>
#include <vector>

#include "dtw_common.cuh"
#include "dtw_kernels.h"

namespace dtwb {

namespace {

constexpr int kPlainBase = 500;  // the paper's recursion cutoff m

__device__ __forceinline__ double plain_cost(const PlainProblem& pb, long long i, long long j) {
    if (pb.kind == KIND_ABS) {
        const long long t = (long long)static_cast<const int32_t*>(pb.X)[i] -
                            (long long)static_cast<const int32_t*>(pb.Y)[j];
        return (double)(t < 0 ? -t : t);
    }
    const float* x = static_cast<const float*>(pb.X) + i * pb.d;
    const float* y = static_cast<const float*>(pb.Y) + j * pb.d;
    double s = 0.0;
    for (int k = 0; k < pb.d; ++k) {
        const double t = __dsub_rn((double)x[k], (double)y[k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return __dsqrt_rn(s);
}

struct PBox {
    long long i0, j0, Ms, Ns;
};

// One anti-diagonal k of the box, forward (rev = 0) or on the reversed series.
__global__ void plain_diag_kernel(PlainProblem pb, PBox bx, int rev, long long k, const double* dm2,
                                  const double* dm1, double* dk) {
    const long long alo = k - (bx.Ns - 1) > 0 ? k - (bx.Ns - 1) : 0;
    const long long ahi = k < bx.Ms - 1 ? k : bx.Ms - 1;
    const long long a = alo + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (a > ahi) return;
    const long long b = k - a;
    const long long gi = rev ? bx.i0 + bx.Ms - 1 - a : bx.i0 + a;
    const long long gj = rev ? bx.j0 + bx.Ns - 1 - b : bx.j0 + b;
    const double c = plain_cost(pb, gi, gj);
    double best;
    if (k == 0) {
        best = 0.0;
    } else {
        best = __longlong_as_double(0x7ff0000000000000LL);
        if (a >= 1 && b >= 1) best = fmin(best, dm2[a - 1]);
        if (a >= 1) best = fmin(best, dm1[a - 1]);
        if (b >= 1) best = fmin(best, dm1[a]);
    }
    dk[a] = best + c;
}

// S = F + B - C over diagonals cd-1..cd+1; pairs (f0,b2), (f1,b1), (f2,b0).
__global__ void plain_pivot_kernel(PlainProblem pb, PBox bx, long long cd, const double* f0, const double* f1,
                                   const double* f2, const double* b0, const double* b1, const double* b2,
                                   double* out_best, long long* out_ab) {
    __shared__ double sv[32];
    __shared__ long long sk[32];
    double best = __longlong_as_double(0x7ff0000000000000LL);
    long long bestkey = -1;  // (t, a) packed as t * Ms + a: lowest diagonal, then lowest a
    const double* fd[3] = {f0, f1, f2};
    const double* bd[3] = {b2, b1, b0};
    for (int t = 0; t < 3; ++t) {
        const long long k = cd - 1 + t;
        const long long alo = k - (bx.Ns - 1) > 0 ? k - (bx.Ns - 1) : 0;
        const long long ahi = k < bx.Ms - 1 ? k : bx.Ms - 1;
        for (long long a = alo + threadIdx.x; a <= ahi; a += blockDim.x) {
            const double S = fd[t][a] + bd[t][bx.Ms - 1 - a] - plain_cost(pb, bx.i0 + a, bx.j0 + (k - a));
            const long long key = t * bx.Ms + a;
            if (S < best || (S == best && key < bestkey)) {
                best = S;
                bestkey = key;
            }
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_down_sync(kFull, best, o);
        const long long ok = __shfl_down_sync(kFull, bestkey, o);
        if (ok >= 0 && (ov < best || (ov == best && (bestkey < 0 || ok < bestkey)))) {
            best = ov;
            bestkey = ok;
        }
    }
    if (lane == 0) {
        sv[w] = best;
        sk[w] = bestkey;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            if (sk[i] >= 0 && (sv[i] < best || (sv[i] == best && (bestkey < 0 || sk[i] < bestkey)))) {
                best = sv[i];
                bestkey = sk[i];
            }
        }
        const long long t = bestkey / bx.Ms, a = bestkey % bx.Ms;
        out_best[0] = best;
        out_ab[0] = a;
        out_ab[1] = (cd - 1 + t) - a;
    }
}

// Textbook DTW on one box: anti-diagonal DP by one block, byte backpointers
// (first minimum in the order DIAG, UP, LEFT) in global memory, then a
// backtrace appending the box's cells at path[*len] (dropping the first cell
// when the path already holds the shared pivot).
__global__ void __launch_bounds__(1024) plain_base_kernel(PlainProblem pb, PBox bx, double* diag3, uint8_t* P,
                                                          int32_t* path, long long* len, double* cost) {
    const double INF = __longlong_as_double(0x7ff0000000000000LL);
    double* dm2 = diag3;
    double* dm1 = diag3 + bx.Ms;
    double* dk = diag3 + 2 * bx.Ms;
    const long long K = bx.Ms + bx.Ns - 1;
    for (long long k = 0; k < K; ++k) {
        const long long alo = k - (bx.Ns - 1) > 0 ? k - (bx.Ns - 1) : 0;
        const long long ahi = k < bx.Ms - 1 ? k : bx.Ms - 1;
        for (long long a = alo + threadIdx.x; a <= ahi; a += blockDim.x) {
            const long long b = k - a;
            const double c = plain_cost(pb, bx.i0 + a, bx.j0 + b);
            double best;
            uint8_t mv;
            if (k == 0) {
                best = 0.0;
                mv = 3;
            } else if (a == 0) {
                best = dm1[a];
                mv = 2;
            } else if (b == 0) {
                best = dm1[a - 1];
                mv = 1;
            } else {
                const double dg = dm2[a - 1], up = dm1[a - 1], lf = dm1[a];
                best = dg;
                mv = 0;
                if (up < best) {
                    best = up;
                    mv = 1;
                }
                if (lf < best) {
                    best = lf;
                    mv = 2;
                }
            }
            dk[a] = best + c;
            P[a * bx.Ns + b] = mv;
        }
        __syncthreads();
        double* t = dm2;
        dm2 = dm1;
        dm1 = dk;
        dk = t;
    }
    (void)INF;
    if (threadIdx.x == 0) {
        *cost = dm1[bx.Ms - 1];
        // backtrace into a reversed run at the end of the free path space, then copy
        long long a = bx.Ms - 1, b = bx.Ns - 1;
        const long long start = *len;
        const long long cap = bx.Ms + bx.Ns - 1;
        // count the box path first
        long long n = 0;
        {
            long long aa = a, bb = b;
            for (;;) {
                ++n;
                const uint8_t mv = P[aa * bx.Ns + bb];
                if (mv == 3 || n > cap) break;
                if (mv == 0) {
                    --aa;
                    --bb;
                } else if (mv == 1) {
                    --aa;
                } else {
                    --bb;
                }
            }
        }
        const long long skip = start > 0 ? 1 : 0;  // the first cell is the previous box's last
        long long pos = start + n - 1 - skip;
        for (long long c = 0; c < n - skip; ++c) {
            path[2 * pos] = (int32_t)(bx.i0 + a);
            path[2 * pos + 1] = (int32_t)(bx.j0 + b);
            --pos;
            const uint8_t mv = P[a * bx.Ns + b];
            if (mv == 0) {
                --a;
                --b;
            } else if (mv == 1) {
                --a;
            } else if (mv == 2) {
                --b;
            }
        }
        *len = start + n - skip;
    }
}

long long diag_len(const PBox& bx, long long k) {
    const long long alo = k - (bx.Ns - 1) > 0 ? k - (bx.Ns - 1) : 0;
    const long long ahi = k < bx.Ms - 1 ? k : bx.Ms - 1;
    return ahi >= alo ? ahi - alo + 1 : 0;
}

// Algorithm 1 on the device: diagonals 0..kstop, one launch each.  The three
// buffers rotate; on return o[0..2] point at diagonals kstop-2, kstop-1, kstop.
cudaError_t diagdtw(const PlainProblem& pb, const PBox& bx, int rev, long long kstop, double* bufs[3],
                    double* o[3], cudaStream_t st, long long* cells) {
    double *dm2 = bufs[0], *dm1 = bufs[1], *dk = bufs[2];
    for (long long k = 0; k <= kstop; ++k) {
        const long long n = diag_len(bx, k);
        plain_diag_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pb, bx, rev, k, dm2, dm1, dk);
        *cells += n;
        double* t = dm2;
        dm2 = dm1;
        dm1 = dk;
        dk = t;
    }
    o[0] = dk;
    o[1] = dm2;
    o[2] = dm1;
    return cudaGetLastError();
}

}  // namespace

size_t plain_workspace_bytes(int64_t M, int64_t N) {
    const int64_t mn = M < N ? M : N;
    const int64_t side = mn < kPlainBase ? mn : kPlainBase;
    // 6 diagonal buffers of M doubles, the base-case diagonals, byte pointers of
    // the largest base box (one side < 500, the other <= max(M, N)), and results
    return (size_t)(9 * M + 64) * sizeof(double) + (size_t)(side + 1) * (size_t)(M > N ? M : N) + 4096;
}

int plain_align(const PlainProblem& pb, int32_t* d_path, double* cost, int64_t* K, void* work, size_t work_bytes,
                cudaStream_t st, long long* cells) {
    const long long M = pb.M, N = pb.N;
    if (work_bytes < plain_workspace_bytes(M, N)) return DTW_ENOMEM;
    char* w = static_cast<char*>(work);
    double* fb[3];
    double* bb[3];
    for (int t = 0; t < 3; ++t) fb[t] = reinterpret_cast<double*>(w) + t * M;
    for (int t = 0; t < 3; ++t) bb[t] = reinterpret_cast<double*>(w) + (3 + t) * M;
    double* base3 = reinterpret_cast<double*>(w) + 6 * M;
    double* res_best = reinterpret_cast<double*>(w) + 9 * M;
    double* res_cost = res_best + 1;
    long long* res_ab = reinterpret_cast<long long*>(res_best + 8);
    long long* d_len = res_ab + 4;
    uint8_t* ptrs = reinterpret_cast<uint8_t*>(reinterpret_cast<double*>(w) + 9 * M + 64);
    cudaMemsetAsync(d_len, 0, sizeof(long long), st);

    *cells = 0;
    double root_cost = NAN;
    bool root = true;
    std::vector<PBox> stack;
    stack.push_back(PBox{0, 0, M, N});
    cudaError_t e = cudaSuccess;
    while (!stack.empty() && e == cudaSuccess) {
        const PBox bx = stack.back();
        stack.pop_back();
        if (bx.Ms < kPlainBase || bx.Ns < kPlainBase || bx.Ms <= 2 || bx.Ns <= 2) {
            plain_base_kernel<<<1, 1024, 0, st>>>(pb, bx, base3, ptrs, d_path, d_len, res_cost);
            *cells += bx.Ms * bx.Ns;
            if (root) {
                e = cudaMemcpyAsync(&root_cost, res_cost, sizeof(double), cudaMemcpyDeviceToHost, st);
                root = false;
            }
            if (e == cudaSuccess) e = cudaGetLastError();
            continue;
        }
        const long long Kd = bx.Ms + bx.Ns - 1;
        const long long cd = (Kd - 1) / 2;
        double* fo[3];
        double* bo[3];
        e = diagdtw(pb, bx, 0, cd + 1, fb, fo, st, cells);
        if (e == cudaSuccess) e = diagdtw(pb, bx, 1, Kd - 1 - (cd - 1), bb, bo, st, cells);
        if (e != cudaSuccess) break;
        plain_pivot_kernel<<<1, 1024, 0, st>>>(pb, bx, cd, fo[0], fo[1], fo[2], bo[0], bo[1], bo[2], res_best,
                                               res_ab);
        long long ab[2];
        double best;
        e = cudaMemcpyAsync(ab, res_ab, sizeof(ab), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&best, res_best, sizeof(best), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        if (root) {
            root_cost = best;
            root = false;
        }
        const long long pa = ab[0], pbb = ab[1];
        if (pa < 0 || pbb < 0 || pa >= bx.Ms || pbb >= bx.Ns) return DTW_EINTERNAL;
        // depth-first, left box first: push the right box, then the left
        stack.push_back(PBox{bx.i0 + pa, bx.j0 + pbb, bx.Ms - pa, bx.Ns - pbb});
        stack.push_back(PBox{bx.i0, bx.j0, pa + 1, pbb + 1});
    }
    if (e != cudaSuccess) return DTW_ECUDA;
    long long n = 0;
    e = cudaMemcpyAsync(&n, d_len, sizeof(n), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return DTW_ECUDA;
    *K = n;
    *cost = root_cost;
    return 0;
}

}  // namespace dtwb
