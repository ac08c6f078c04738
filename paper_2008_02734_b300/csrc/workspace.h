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

inline Layout make_layout(int B, long long sumM, long long sumN, long long feat_bytes, long long path_pairs) {
    Layout L{};
    const long long S = sumM + sumN;
    L.cap_box = S / 2 + B + 16;
    L.cap_base = S + B + 16;
    L.cap_sweeps = 2 * L.cap_box;
    // two 64-bit words per column per sweep (columns padded to 8)
    L.cap_buf = 4 * (S + 2 * L.cap_box) + 2 * L.cap_box * 16;
    // out rows: per sweep nout <= kSplitRowsMax rows of its columns padded to whole blocks (<= 8 columns)
    L.cap_out = kSplitRowsMax * (S + 2 * L.cap_box * 8);
    // split work items: column chunks of every box's split rows
    L.cap_items = S / kSplitChunk + L.cap_box + 16;
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
