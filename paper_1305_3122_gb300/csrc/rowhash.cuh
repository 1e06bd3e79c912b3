// rowhash.cuh -- the per-row hash tables of the generic pattern builds (tet.cu, p2.cu).
//
// A row's neighbour ids are merged in a shared-memory open-addressing table of TS slots (linear
// probing, -1 marks a free slot) owned by one warp; TS is larger than the row's number of distinct
// ids, so every probe ends.
#pragma once

#include <stdint.h>

__device__ __forceinline__ uint32_t fe_row_hash(int32_t id) { return (uint32_t)id * 0x9E3779B1u; }

template <int TS>
struct RowTableShift {
    static_assert(TS == 128 || TS == 4096, "table sizes");
    static constexpr int value = 32 - (TS == 128 ? 7 : 12);
};

// Slot of id (inserted if absent); *fresh tells whether this call inserted it. Callers keep the
// slot of each insertion, so no id is looked up again.
template <int TS>
__device__ __forceinline__ int tab_insert(int32_t* tab, int32_t id, bool* fresh) {
    int s = (int)(fe_row_hash(id) >> RowTableShift<TS>::value);
    for (int step = 0; step < TS; step++) {
        int32_t old = atomicCAS(&tab[s], -1, id);
        if (old == -1) { *fresh = true; return s; }
        if (old == id) { *fresh = false; return s; }
        s = (s + 1) & (TS - 1);
    }
    *fresh = false;
    return 0;    // not reached: the table is never full
}
