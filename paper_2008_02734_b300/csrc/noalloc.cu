// dtw_cost_noalloc: the whole-matrix cost sweep of dtw_cost, for callers that
// must not allocate device memory.
//
// Everything the sweep needs besides its inputs and its output -- the pair and
// box descriptors, the sweep descriptor and result, the control block, the
// integer range scratch and the boundary row between bands -- lives in one fixed
// device array defined in this file.  The array is part of the library's
// device image: every GPU that loads the library holds it until the process
// exits, and every call on a device reuses the same bytes.
#include <atomic>
#include <cmath>
#include <mutex>

#include "dtw_b300.h"
#include "dtw_common.cuh"
#include "dtw_kernels.h"

using namespace dtwb;

namespace {

constexpr long long kShortMax = DTW_NOALLOC_MAX_SHORT;  // max min(M, N)
constexpr long long kLongMax = DTW_NOALLOC_MAX_LONG;    // max max(M, N)
constexpr long long kPadCols = 64;                      // column padding of the widest kernel variant

constexpr size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// byte offsets inside the scratch array
constexpr size_t kOffPair = 0;
constexpr size_t kOffBox = kOffPair + up256(sizeof(PairDesc));
constexpr size_t kOffSweep = kOffBox + up256(sizeof(Box));
constexpr size_t kOffRes = kOffSweep + up256(sizeof(Sweep));
constexpr size_t kOffCtl = kOffRes + up256(sizeof(SweepRes));
constexpr size_t kOffMinMax = kOffCtl + up256(sizeof(LevelCtl));
constexpr size_t kOffClear = kOffMinMax + 128;  // 1: this call clears the boundary row first
constexpr long long kBufWords = 2 * (kShortMax + kPadCols);  // two epoch-stamped words per column
constexpr size_t kOffBuf = kOffMinMax + 256;
constexpr size_t kScratchBytes = kOffBuf + up256(8 * (size_t)kBufWords);
// Epochs one call may take: the plan gives each band of the sweep its own (a
// band has at least 32 rows), plus one.
constexpr uint32_t kCallEpochs = (uint32_t)(kLongMax / 32 + 2);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};  // device address of the scratch array, per device
int g_sms[kMaxDevices] = {};

// Writes the pair, the root box and a zeroed control block for this call (the
// previous call's contents are still there).  The boundary-word epoch counter
// is carried over, so that words left by earlier calls are never accepted.
// When the counter could wrap within this call (or a test sets it, ep_set >= 0),
// the epochs restart at 1 and the call first clears the boundary row: no word
// written before the restart can then bear an epoch the call expects.
__global__ void noalloc_init_kernel(const void* X, int M, const void* Y, int N, long long ep_set) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    PairDesc* pd = reinterpret_cast<PairDesc*>(g_noalloc_scratch + kOffPair);
    pd->X = X;
    pd->Y = Y;
    pd->M = M;
    pd->N = N;
    pd->row_off = 0;
    pd->flags = 0;
    pd->path = nullptr;
    Box* b = reinterpret_cast<Box*>(g_noalloc_scratch + kOffBox);
    b->pair = 0;
    b->i0 = 0;
    b->j0 = 0;
    b->H = M;
    b->W = N;
    b->flags = BOX_ROOT;
    b->known_i = -1;
    b->known_f = NAN;
    LevelCtl* c = reinterpret_cast<LevelCtl*>(g_noalloc_scratch + kOffCtl);
    uint32_t ep = ep_set >= 0 ? (uint32_t)ep_set : c->epoch_base;
    int* clear = reinterpret_cast<int*>(g_noalloc_scratch + kOffClear);
    *clear = 0;
    if (ep == 0 || ep > 0xFFFFFFFFu - kCallEpochs) {
        ep = 1;
        *clear = 1;
    }
    *c = LevelCtl{};
    c->epoch_base = ep;
    SweepRes* r = reinterpret_cast<SweepRes*>(g_noalloc_scratch + kOffRes);
    *r = SweepRes{};
}

// Zeroes the boundary row when the init kernel restarted the epochs (otherwise
// every thread returns at once).
__global__ void noalloc_clear_kernel() {
    if (*reinterpret_cast<const int*>(g_noalloc_scratch + kOffClear) == 0) return;
    unsigned long long* w = reinterpret_cast<unsigned long long*>(g_noalloc_scratch + kOffBuf);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < kBufWords;
         i += (long long)gridDim.x * blockDim.x)
        w[i] = 0ull;
}

bool on_device(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Once per device, with that device current: the scratch array's device address.
int setup(int dev, char** base, int* sms) {
    std::lock_guard<std::mutex> g(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return DTW_EINVAL;
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DTW_ECUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DTW_ECUDA;
        g_addr[dev] = p;
        g_sms[dev] = n;
    }
    *base = static_cast<char*>(g_addr[dev]);
    *sms = g_sms[dev];
    return DTW_OK;
}

std::mutex g_call_mu;  // the scratch is shared: one call at a time from the host
std::atomic<long long> g_ep_set{-1};  // test hook: the next call's first epoch

}  // namespace

namespace dtwb {
void noalloc_set_epoch(long long ep) { g_ep_set.store(ep); }
}  // namespace dtwb

extern "C" int dtw_cost_noalloc(const void* X, int64_t M, const void* Y, int64_t N, int32_t d, int32_t cost_kind,
                                double* cost_out, void* cuda_stream) {
    if (!X || !Y || !cost_out || M < 1 || N < 1 || d < 1) return DTW_EINVAL;
    if (cost_kind != DTW_EUCLID_F32 && cost_kind != DTW_ABS_I32) return DTW_EINVAL;
    if (cost_kind == DTW_ABS_I32 && d != 1) return DTW_EINVAL;
    const long long lo = M < N ? M : N, hi = M < N ? N : M;
    if (lo > kShortMax || hi > kLongMax) return DTW_ENOMEM;  // larger than the fixed scratch
    if (!on_device(X) || !on_device(Y)) return DTW_EINVAL;   // no staging: inputs must be on the device
    const int kind = cost_kind == DTW_ABS_I32 ? KIND_ABS : KIND_EUC;
    if (kind == KIND_EUC && (d == 12 || d == 64) && ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15))
        return DTW_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DTW_ECUDA;
    char* base = nullptr;
    int sms = 0;
    int rc = setup(dev, &base, &sms);
    if (rc) return rc;

    std::lock_guard<std::mutex> g(g_call_mu);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    PairDesc* pairs = reinterpret_cast<PairDesc*>(base + kOffPair);
    Box* box = reinterpret_cast<Box*>(base + kOffBox);
    Sweep* sweep = reinterpret_cast<Sweep*>(base + kOffSweep);
    SweepRes* res = reinterpret_cast<SweepRes*>(base + kOffRes);
    LevelCtl* ctl = reinterpret_cast<LevelCtl*>(base + kOffCtl);
    int32_t* minmax = reinterpret_cast<int32_t*>(base + kOffMinMax);

    noalloc_init_kernel<<<1, 32, 0, st>>>(X, (int)M, Y, (int)N, g_ep_set.exchange(-1));
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        noalloc_clear_kernel<<<sms, 256, 0, st>>>();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && kind == KIND_ABS) e = launch_int_range_check(pairs, 1, (int)hi, minmax, ctl, st);
    // the plan resets the band ticket and assigns this call's epochs
    PlanArgs pa{box, 1, pairs, MODE_COST, kind, 0, sweep_block_cols(kind, d), sweep_band_rows(kind, d),
                sweep_group_bands(kind), sweep, ctl,
                1, kBufWords, 0, nullptr, 0, false, nullptr};
    if (e == cudaSuccess) e = launch_plan(pa, st);
    SweepArgs sa{sweep, ctl, reinterpret_cast<unsigned long long*>(base + kOffBuf), nullptr, res, d, 1 << 22, -1};
    if (e == cudaSuccess) e = launch_sweep(kind, d, false, sa, sms, 0, st);
    SweepRes hr{};
    LevelCtl hc{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hr, res, sizeof(hr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        // kernels enqueued before the failure may still run on the shared array:
        // wait for them before another call may start
        cudaStreamSynchronize(st);
        cudaGetLastError();
        return DTW_ECUDA;
    }
    switch (hc.err) {
        case ERR_NONE: break;
        case ERR_TIMEOUT: return DTW_ETIMEOUT;
        case ERR_OVERFLOW: return DTW_EOVERFLOW;
        case ERR_CAPACITY: return DTW_ENOMEM;
        default: return DTW_EINTERNAL;
    }
    *cost_out = kind == KIND_ABS ? (double)hr.end_i : hr.end_f;
    return DTW_OK;
}
