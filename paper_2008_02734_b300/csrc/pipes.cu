// Instruction-rate measurements for the per-cell roofline of the sweep: how
// many of each instruction the cell update is built from the GPU issues per
// second when nothing but that instruction is in flight.  The roofline the
// benchmark reports divides the algorithmic instruction count of a cell by
// such rates (the update D = C + min(diagonal, up, left) of the recurrence in
// Section 2.1, costed per cell).
//
// Every thread runs eight independent dependency chains of one instruction
// (enough to cover its latency at full occupancy: 64 warps per SM), so the
// measured rate is the pipe's issue rate.  Integer minimum chains take one
// operand that changes every iteration (one extra XOR per eight minima, which
// the count includes in its denominator only as the minima: a lower bound on
// the pipe) so that no compiler can fold an idempotent recurrence.
#include <cstdint>
#include <cuda_runtime.h>

#include "dtw_b300.h"

namespace dtwb {
namespace {

constexpr int kPipeThreads = 256;
constexpr int kPipeBlocksPerSM = 8;
constexpr int kChains = 8;

enum PipeOp { OP_MIN3 = 0, OP_SAD, OP_FFMA, OP_FFMA2, OP_SQRT, OP_DADD, OP_COUNT };

template <int OP>
__global__ void __launch_bounds__(kPipeThreads) pipe_kernel(int iters, int32_t a, int32_t b, float fa, float fb,
                                                            uint32_t* sink) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t out = 0;
    if constexpr (OP == OP_MIN3 || OP == OP_SAD) {
        int32_t x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = tid * 31 + k * 7 + a;
        for (int it = 0; it < iters; ++it) {
            const int32_t t = a ^ it;
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if constexpr (OP == OP_MIN3) x[k] = __vimin3_s32(x[k], t, b + k);
                else x[k] = (int32_t)__sad(x[k], a + k, (unsigned)x[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) out ^= (uint32_t)x[k];
    } else if constexpr (OP == OP_FFMA || OP == OP_SQRT) {
        float x[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fa + (float)(tid & 255) * 1e-3f + (float)k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if constexpr (OP == OP_FFMA) x[k] = __fmaf_rn(x[k], fa, fb);
                else x[k] = __fsqrt_rn(x[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) out ^= __float_as_uint(x[k]);
    } else if constexpr (OP == OP_FFMA2) {
        float2 x[kChains];
        const float2 m = make_float2(fa, fa), c = make_float2(fb, fb);
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = make_float2(fa + (float)k, fb + (float)(tid & 255));
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = __ffma2_rn(x[k], m, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) out ^= __float_as_uint(x[k].x) ^ __float_as_uint(x[k].y);
    } else {  // OP_DADD
        double x[kChains];
        const double da = (double)fa;
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = (double)fb + (double)(tid & 255) + (double)k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) x[k] = __dadd_rn(x[k], da);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) out ^= (uint32_t)__double2loint(x[k]);
    }
    sink[tid] = out;
}

template <int OP>
cudaError_t launch_pipe(int blocks, int iters, uint32_t* sink, cudaStream_t st) {
    pipe_kernel<OP><<<blocks, kPipeThreads, 0, st>>>(iters, 3, 1 << 20, 0.999f, 1e-3f, sink);
    return cudaGetLastError();
}

cudaError_t launch_op(int op, int blocks, int iters, uint32_t* sink, cudaStream_t st) {
    switch (op) {
        case OP_MIN3: return launch_pipe<OP_MIN3>(blocks, iters, sink, st);
        case OP_SAD: return launch_pipe<OP_SAD>(blocks, iters, sink, st);
        case OP_FFMA: return launch_pipe<OP_FFMA>(blocks, iters, sink, st);
        case OP_FFMA2: return launch_pipe<OP_FFMA2>(blocks, iters, sink, st);
        case OP_SQRT: return launch_pipe<OP_SQRT>(blocks, iters, sink, st);
        default: return launch_pipe<OP_DADD>(blocks, iters, sink, st);
    }
}

// Dependent-chain latency: one warp runs a single chain of kLatOps operations,
// each taking the previous one's result, and thread 0 stores the clock64 cycles
// the chain took.  Cycles per operation = the operation's latency on the chain
// of a recurrence (the integer and FP64 cell updates of the sweep sit on one).
constexpr int kLatOps = 2048;
enum LatOp { LAT_MIN3 = 0, LAT_SAD, LAT_FADD, LAT_DADD, LAT_SHFL, LAT_COUNT };

template <int OP>
__global__ void __launch_bounds__(32) latency_kernel(int32_t a, int32_t b, float fa, long long* cycles,
                                                     uint32_t* sink) {
    uint32_t out = 0;
    long long t0 = 0, t1 = 0;
    if constexpr (OP == LAT_MIN3 || OP == LAT_SAD || OP == LAT_SHFL) {
        int32_t x = a + (int32_t)threadIdx.x;
        t0 = clock64();
#pragma unroll 16
        for (int i = 0; i < kLatOps; ++i) {
            if constexpr (OP == LAT_MIN3) x = __vimin3_s32(x, b, a + i);
            else if constexpr (OP == LAT_SAD) x = (int32_t)__sad(a, b, (unsigned)x);
            else x = __shfl_up_sync(0xffffffffu, x, 1);
        }
        t1 = clock64();
        out = (uint32_t)x;
    } else if constexpr (OP == LAT_FADD) {
        float x = fa;
        t0 = clock64();
#pragma unroll 16
        for (int i = 0; i < kLatOps; ++i) x = __fadd_rn(x, fa);
        t1 = clock64();
        out = __float_as_uint(x);
    } else {  // LAT_DADD
        double x = (double)fa;
        const double da = (double)fa;
        t0 = clock64();
#pragma unroll 16
        for (int i = 0; i < kLatOps; ++i) x = __dadd_rn(x, da);
        t1 = clock64();
        out = (uint32_t)__double2loint(x);
    }
    sink[threadIdx.x] = out;
    if (threadIdx.x == 0) *cycles = t1 - t0;
}

template <int OP>
cudaError_t launch_lat(long long* cycles, uint32_t* sink, cudaStream_t st) {
    latency_kernel<OP><<<1, 32, 0, st>>>(5, 7, 1.0f, cycles, sink);
    return cudaGetLastError();
}

cudaError_t launch_latency(int op, long long* cycles, uint32_t* sink, cudaStream_t st) {
    switch (op) {
        case LAT_MIN3: return launch_lat<LAT_MIN3>(cycles, sink, st);
        case LAT_SAD: return launch_lat<LAT_SAD>(cycles, sink, st);
        case LAT_FADD: return launch_lat<LAT_FADD>(cycles, sink, st);
        case LAT_DADD: return launch_lat<LAT_DADD>(cycles, sink, st);
        default: return launch_lat<LAT_SHFL>(cycles, sink, st);
    }
}

}  // namespace
}  // namespace dtwb

// See include/dtw_b300.h.
extern "C" DTW_API int dtw_pipe_rates(double* rates_out, int32_t n) {
    using namespace dtwb;
    if (!rates_out || n < 1) return DTW_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DTW_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return DTW_ECUDA;
    const int blocks = sms * kPipeBlocksPerSM;
    uint32_t* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DTW_OK;
    if (cudaMalloc(&sink, sizeof(uint32_t) * (size_t)blocks * kPipeThreads) != cudaSuccess) return DTW_ENOMEM;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        rc = DTW_ECUDA;
    const int nops = n < (int)OP_COUNT ? n : (int)OP_COUNT;
    for (int op = 0; op < nops && rc == DTW_OK; ++op) {
        // about 10^10 instructions for the fast pipes, 2.5 10^8 for FP64 adds
        const int iters = op == OP_DADD ? 128 : (op == OP_SQRT ? 512 : 4096);
        float ms = 0.f;
        cudaError_t e = launch_op(op, blocks, iters / 8, sink, st);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = launch_op(op, blocks, iters, sink, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess || ms <= 0.f) {
            rc = DTW_ECUDA;
            break;
        }
        const double count = (double)blocks * kPipeThreads * (double)iters * kChains;
        rates_out[op] = count / (ms * 1e-3);
    }
    // entries OP_COUNT.. : dependent latencies in cycles (the sink's first words
    // hold the cycle count, the rest the chains' results)
    const int nlat = rc == DTW_OK && n > (int)OP_COUNT ? (n - (int)OP_COUNT < (int)LAT_COUNT ? n - (int)OP_COUNT
                                                                                           : (int)LAT_COUNT)
                                                       : 0;
    long long* cyc = reinterpret_cast<long long*>(sink);
    for (int op = 0; op < nlat && rc == DTW_OK; ++op) {
        long long h = 0;
        cudaError_t e = launch_latency(op, cyc, sink + 64, st);  // warm-up (instruction cache)
        if (e == cudaSuccess) e = launch_latency(op, cyc, sink + 64, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess || h <= 0) {
            rc = DTW_ECUDA;
            break;
        }
        rates_out[OP_COUNT + op] = (double)h / kLatOps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(sink);
    return rc == DTW_OK ? nops + nlat : rc;
}
