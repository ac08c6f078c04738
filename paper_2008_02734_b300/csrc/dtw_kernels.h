// Launchers of the library's kernels (host side).  Internal header.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "dtw_b300.h"
#include "dtw_common.cuh"

namespace dtwb {

struct SplitArgs {
    const Box* boxes;
    int n_boxes;
    const PairDesc* pairs;
    PairRes* pres;
    int kind, d;
    int halo;
    const Sweep* sweeps;
    const SweepRes* res;
    const void* outpool;
    Box* next;
    Box* base;
    LevelCtl* ctl;
    long long base_area;
    int cap_next, cap_base;
    int* box_done;    // per-box count of finished work items
    void* partials;   // per work item: kSplitRowsMax partial row minima (16 B each) of its window
    int n_items;      // work items of the level (as planned); < 0: read ctl->n_items on the device
    int num_sms;
};
struct SweepArgs {
    const Sweep* sweeps;
    LevelCtl* ctl;
    unsigned long long* bufpool;  // boundary rows: 1 or 2 epoch-stamped words per column
    void* outpool;                // split rows (Acc), each sweep's frame order, laid out by out_index
    SweepRes* res;                // per-sweep last-cell results
    int d;
    int spin_limit;
    long long skip_ticket;  // test hook: this level band never publishes (-1: none)
    int32_t* best = nullptr;  // KIND_LOCAL: 4 int32 per level band (value, frame row, column, written)
    const int2* tmap = nullptr;  // ticket -> (sweep, band group), when the plan wrote it (ctl->tmap_on)
    // Fused split (prog non-null): bands holding split rows publish their
    // progress in prog (kProgWords per sweep), and blocks that find the ticket
    // queue empty run the level's split work items (split) while the sweeps end.
    int* prog = nullptr;
    SplitArgs split{};
    int sms = 0;     // SMs of the device (set by the launch)
    int ytight = 0;  // d = 64 FP32-cost kinds: the launch allocated the tight frame ring
};

// Sweep variants
// variant (integer kind): 0 R=4 (default), 1 R=2, 2 R=8 rows per lane; U=4 columns;
// 3 R=4 with fully unrolled steady groups (longer code: faster on long bands, slower
// where many blocks share an SM's instruction cache).
constexpr int kSweepVariants = 4;
int sweep_block_cols(int kind, int d, int variant = 0);  // U
int sweep_band_rows(int kind, int d, int variant = 0);   // 32*R
int sweep_group_bands(int kind);  // bands per ticket (compute warps per block)
// every ticket of the kind's sweep must hold bands of one sweep only (the BF16
// form's MMAs, the d = 64 FP32-cost kinds' tight frame ring): the plan pads each
// sweep's bands to whole groups
bool sweep_whole_groups(int kind, int d);
// max_blocks > 0 caps the grid (one block per ticket suffices); 0: a full persistent grid.
cudaError_t launch_sweep(int kind, int d, bool tags, const SweepArgs& A, int num_sms, long long max_blocks,
                         cudaStream_t st, int variant = 0);
// One-time launch setup of the variant (attributes, occupancy); must precede a stream capture.
cudaError_t sweep_prepare(int kind, int d, bool tags, int variant = 0);
// The sweep variant a call runs: the integer kinds keep `variant`; the d = 12
// Euclidean kinds take their throughput form (variant 1: more resident blocks,
// fewer registers) when the first level's tickets, about `tickets0`, outnumber
// the blocks the default form keeps resident; the d = 64 FP32-cost kinds take
// the tight frame ring (variant 1: two blocks per SM) when they are three times
// the SMs or more; other kinds variant 0.
int sweep_variant_for(int kind, int d, int variant, long long tickets0, int num_sms);

// Level planning modes
constexpr int MODE_ALIGN = 0;  // per box: two half sweeps, or one tagged sweep (BOX_TAG)
constexpr int MODE_COST = 2;   // one untagged forward sweep of the whole box, last cell only

struct PlanArgs {
    const Box* boxes;
    int n_boxes;  // < 0: the count the split kernel left in ctl->n_next
    const PairDesc* pairs;
    int mode;
    int kind;
    int halo;  // split rows each side of the middle row written by half sweeps
    int U, BR, G;  // columns per block, rows per band, bands per ticket
    Sweep* sweeps;
    LevelCtl* ctl;
    long long cap_sweeps, cap_buf, cap_out;
    int* box_done;  // per-box split completion counters (reset here; MODE_ALIGN)
    long long cap_items;
    bool reset_base;  // also empty the base list (its boxes have been finished)
    Box* copy_to;     // non-null: the planned boxes are also copied here (same index)
    int local = 0;    // KIND_LOCAL, MODE_COST: 1 forward sweep with the local floor,
                      // 2 sweep of the reversed box without it; frame rows along X
    int2* tmap = nullptr;      // non-null: write the ticket map (group-major ticket order)
    long long cap_tickets = 0; // its capacity; a level that needs more uses the plain order
    long long map_min = 0;     // levels with at most this many plain tickets skip the map (all
                               // their tickets run at once, so their order does not matter)
    int* prog = nullptr;       // non-null: reset the sweeps' split-row progress words (fused split)
    int nwin = 1;              // windows of split rows per box at most (odd; 1: one split row per box)
    bool whole_groups = false; // pad each sweep's bands to whole groups of G (sweep_whole_groups)
};
cudaError_t launch_plan(const PlanArgs& a, cudaStream_t st);

cudaError_t launch_split(const SplitArgs& a, cudaStream_t st);

struct BaseArgs {
    const Box* base;
    int n_base;  // < 0: read ctl->n_base on the device
    const PairDesc* pairs;
    PairRes* pres;
    int32_t* jlo;
    int32_t* jhi;
    LevelCtl* ctl;
    int kind, d;
};
// Largest box (cells) the base-case kernel accepts.
#ifndef DTW_BASE_AREA_MAX
#define DTW_BASE_AREA_MAX 32768
#endif
constexpr long long kBaseAreaMax = DTW_BASE_AREA_MAX;
cudaError_t launch_base(const BaseArgs& a, cudaStream_t st);

struct AssembleArgs {
    const PairDesc* pairs;
    int n_pairs;
    int max_M;
    PairRes* pres;
    int32_t* jlo;
    int32_t* jhi;
    int32_t* off;
    LevelCtl* ctl;
    const int* idx;  // pairs to assemble: idx[0..n_pairs) (null: pairs 0..n_pairs-1)
};
cudaError_t launch_assemble(const AssembleArgs& a, cudaStream_t st);
cudaError_t launch_fill_i32(int32_t* p, long long n, int32_t v, cudaStream_t st);
cudaError_t launch_offset_path(int32_t* p, long long K, int32_t da, int32_t db, cudaStream_t st);
// minmax: 4 int32 per pair of scratch (min X, max X, min Y, max Y).  pair_err
// (optional): per-pair flags set to 1 instead of failing the whole call.
cudaError_t launch_int_range_check(const PairDesc* pairs, int n_pairs, int max_len, int32_t* minmax, LevelCtl* ctl,
                                   cudaStream_t st, int32_t* pair_err = nullptr);
// Serving support: appends root boxes staged in `roots` (n of them) to the box
// list `cur` from index cur0 on, or to the base list when their area is at most
// base_area; and marks flags[pair] = 1 for every box of the current level.
cudaError_t launch_append_roots(const Box* roots, int n, Box* cur, int cur0, Box* base, int cap_base,
                                long long base_area, LevelCtl* ctl, cudaStream_t st);
cudaError_t launch_mark_pairs(const Box* boxes, const LevelCtl* ctl, int32_t* flags, cudaStream_t st);
// Graph-driven level loop: sets the loop's condition to "another level": boxes
// planned, no device error and fewer than max_levels levels so far.
cudaError_t launch_level_cond(LevelCtl* ctl, cudaGraphConditionalHandle h, int max_levels, cudaStream_t st);
// Graph-driven level loop, integer kinds: sets the two IF conditions of the
// level's sweep kernels from the plan's count of tagged boxes (h_plain: none,
// the kernel without tagged sweeps; h_tags: some).
cudaError_t launch_sweep_select(const LevelCtl* ctl, cudaGraphConditionalHandle h_plain,
                                cudaGraphConditionalHandle h_tags, cudaStream_t st);

// Windows of split rows per box at most (DTW_OPT_SPLIT_WINDOWS), as read by the
// serving engines and dtw_footprint (api.cu keeps it).
constexpr int kSplitWindowsDefault = 7;
int split_windows_option();
void set_split_windows_option(int windows);

// Serving engine (serve.cu): device memory its groups may take from now on.
void serve_set_budget(uint64_t bytes);
// dtw_cost_noalloc (noalloc.cu), test hook: the next call's first boundary-word epoch.
void noalloc_set_epoch(long long ep);

// The paper's plain form (plain.cu)
struct PlainProblem {
    const void* X;
    const void* Y;
    int64_t M, N;
    int d, kind;
};
// Runs the plain FP64 form on device-resident X, Y; writes the path (device,
// 2*(M+N-1) int32) and returns K or a negative status through *K.
int plain_align(const PlainProblem& pb, int32_t* d_path, double* cost, int64_t* K, void* work,
                size_t work_bytes, cudaStream_t st, long long* cells);
size_t plain_workspace_bytes(int64_t M, int64_t N);

// Alignment discrepancy of two warping paths (discrepancy.cu): P1, P2, err on
// the device; err gets 2*K1 int32 (row errors, then column errors).
size_t discrepancy_workspace_bytes(long long M, long long N);
int path_discrepancy(const int32_t* P1, long long K1, const int32_t* P2, long long K2, long long M, long long N,
                     int32_t* err, int32_t* max_out, void* ws, int num_sms, cudaStream_t st);

}  // namespace dtwb
