// Byte layout of a device workspace (internal header).  Every capacity is
// linear in the summed lengths S = sum(M+N) of the pairs it serves: the
// boundary state of the linear-memory recursion (Section 3.2).
#pragma once

#include <cstddef>

#include "dtw_common.cuh"
#include "dtw_kernels.h"

namespace dtwb {

inline size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t feat, pairs, pres, boxA, boxB, base, sweeps, sres, bufpool, outpool, boxdone, partials, minmax, jlo, jhi,
        off, path, ctl, tmap, prog, total;
    long long cap_box, cap_base, cap_sweeps, cap_buf, cap_out, cap_items, cap_tickets;
};

// Split rows per sweep: up to `windows` windows of split rows per box, each of
// `win_rows` rows (kSplitRowsMax for the integer and edit kinds, 1 otherwise),
// never more than kOutRowsMax rows in all.
inline int split_windows_of(int windows) {
    return windows < 1 ? 1 : (windows > kSplitWinMax ? kSplitWinMax : windows);
}
inline int split_out_rows(int windows, int win_rows) {
    const int r = split_windows_of(windows) * win_rows;
    return r < kOutRowsMax ? r : kOutRowsMax;
}

// Rows per window of split rows of a kind: 2 kSplitHalo + 1 for the integer
// kinds (a unique minimiser is looked for around each split row), 1 otherwise.
inline int split_win_rows(int kind) { return int_kind(kind) ? 2 * kSplitHalo + 1 : 1; }

inline Layout make_layout(int B, long long sumM, long long sumN, long long feat_bytes, long long path_pairs,
                          int windows = 1, int win_rows = kSplitRowsMax) {
    const int out_rows = split_out_rows(windows, win_rows);
    windows = split_windows_of(windows);
    Layout L{};
    const long long S = sumM + sumN;
    L.cap_box = S / 2 + B + 16;
    L.cap_base = S + B + 16;
    L.cap_sweeps = 2 * L.cap_box;
    // two 64-bit words per column per sweep (columns padded to 8)
    L.cap_buf = 4 * (S + 2 * L.cap_box) + 2 * L.cap_box * 16;
    // out rows: per sweep nout rows of its columns padded to whole blocks (<= 8
    // columns).  One window: nout <= win_rows and the sweeps' columns sum to at
    // most S + 2 cap_box.  The boxes with more windows (a cut side of 36 rows or
    // more, so fewer than S/34 of them) have at most out_rows rows and their
    // sweeps' columns (the boxes' shorter sides, twice) sum to less than 3S/2.
    L.cap_out = (long long)win_rows * (S + 2 * L.cap_box * 8) + (long long)(out_rows - win_rows) * (3 * S / 2 + 64);
    // split work items: per window of a box's split rows, its columns in chunks of
    // nw kSplitChunk (split_item_cols), so at most Q/kSplitChunk + nw items.  A box
    // with nw > 1 windows has a cut side of at least 9 nw rows (windows kWinGap
    // rows apart), and the boxes of a level have H + W <= 2S in all, so they hold
    // fewer than S/4 windows beyond their first ones.
    L.cap_items = S / kSplitChunk + S / 4 + L.cap_box + 16;
    // ticket map: band groups of a level (bands are at least 32 rows); a level
    // that needs more falls back to the plain ticket order
    L.cap_tickets = S / 32 + 4096;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o = align_up(o + bytes);
        return r;
    };
    L.feat = take((size_t)feat_bytes);
    L.pairs = take(sizeof(PairDesc) * B);
    L.pres = take(sizeof(PairRes) * B);
    L.boxA = take(sizeof(Box) * L.cap_box);
    L.boxB = take(sizeof(Box) * L.cap_box);
    L.base = take(sizeof(Box) * L.cap_base);
    L.sweeps = take(sizeof(Sweep) * L.cap_sweeps);
    L.sres = take(sizeof(SweepRes) * L.cap_sweeps);
    L.bufpool = take(8 * (size_t)L.cap_buf);
    L.outpool = take(8 * (size_t)L.cap_out);
    L.boxdone = take(4 * (size_t)L.cap_box);
    L.partials = take(16 * (size_t)kSplitRowsMax * (size_t)L.cap_items);
    L.minmax = take(16 * (size_t)B);
    L.jlo = take(4 * (size_t)sumM);
    L.jhi = take(4 * (size_t)sumM);
    L.off = take(4 * (size_t)sumM);
    L.path = take(8 * (size_t)path_pairs);
    L.ctl = take(sizeof(LevelCtl));
    L.tmap = take(8 * (size_t)L.cap_tickets);
    L.prog = take(4 * 4 * (size_t)L.cap_sweeps);  // split-row progress, four words per sweep (fused split)
    L.total = o;
    return L;
}


}  // namespace dtwb
