// Layout of the device workspace of the chain kernel: `nslots` slots, each
// with its basis slab, matrix copies and FP64 vectors (see skr_common.h).
#pragma once

#include <stddef.h>

#include "skr_common.h"

namespace skr {

struct SlabLayout {
    size_t o_basis, o_A64, o_Aw, o_dinv, o_x, o_r, o_b, o_node, o_cols, total;
    bool cols;
};

// Column stride for vectors of n unknowns split over cs CTAs (rows per CTA
// rounded up to 8, the stride to 64 elements).
inline long long chain_ld(long long n, int cs) {
    const long long chunk = (((n + cs - 1) / cs) + 7) / 8 * 8;
    return ((chunk * cs) + 63) / 64 * 64;
}

// cols: room for the column indices of CSR input (7 ints per row and slot)
inline SlabLayout slab_layout(int nslots, long long ld, long long nodecap, size_t esz, bool cols = false) {
    SlabLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t r = o;
        o += (bytes + 255) / 256 * 256;
        return r;
    };
    L.o_basis = take((size_t)nslots * NCOLS * ld * esz);
    L.o_A64 = take((size_t)nslots * 7 * ld * 8);
    L.o_Aw = take((size_t)nslots * AW_SLOTS * ld * esz);
    L.o_dinv = take((size_t)nslots * ld * 8);
    L.o_x = take((size_t)nslots * ld * 8);
    L.o_r = take((size_t)nslots * ld * 8);
    L.o_b = take((size_t)nslots * ld * 8);
    L.o_node = take((size_t)nslots * nodecap * 8);
    L.cols = cols;
    L.o_cols = cols ? take((size_t)nslots * 7 * ld * 4) : 0;
    L.total = o;
    return L;
}

inline Workspace slab_bind(char *base, const SlabLayout &L, int nslots, long long ld, long long nodecap) {
    Workspace ws;
    ws.basis = base + L.o_basis;
    ws.A64 = reinterpret_cast<double *>(base + L.o_A64);
    ws.Aw = base + L.o_Aw;
    ws.dinv = reinterpret_cast<double *>(base + L.o_dinv);
    ws.x = reinterpret_cast<double *>(base + L.o_x);
    ws.r = reinterpret_cast<double *>(base + L.o_r);
    ws.b = reinterpret_cast<double *>(base + L.o_b);
    ws.anode = reinterpret_cast<double *>(base + L.o_node);
    ws.cols = L.cols ? reinterpret_cast<int *>(base + L.o_cols) : nullptr;
    ws.ld = ld;
    ws.nodecap = nodecap;
    ws.nslots = nslots;
    return ws;
}

}  // namespace skr
