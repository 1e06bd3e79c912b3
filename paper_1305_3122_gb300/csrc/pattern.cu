// pattern.cu -- the structural half of sparse(Ig, Jg, Kg): CSR structure, triangle fans, map.
//
// The paper forms Ig = me([1 2 3 1 2 3 1 2 3], :) and Jg = me([1 1 1 2 2 2 3 3 3], :)
// (Section 6, the remark on forming them from me) and lets sparse() sort the 9*nme (row, col)
// keys and merge equal ones (Section 5). Here the keys are sorted by a two-level (most-significant-digit first)
// radix sort that exploits their shape: the row digit is a counting sort (each triangle drops
// its two other vertices into the bucket of each of its vertices), and the column digit is
// sorted inside each row bucket, which holds only 2*valence+1 keys. Unique keys give
// row_ptr / col_idx.
//
// For the row-owner assembly (rowasm.cu) the build also orders each vertex's triangles around
// it: triangle (i, j, l) is counter-clockwise, so in a manifold mesh the triangles around i form
// one chain in which each triangle's l is the next one's j ("fan"; closed for interior vertices,
// open on the boundary). A row whose triangles form one such chain with at most FAN_MAX
// triangles is "simple": it stores its neighbours n_0 .. n_{d-1} in fan order with their column
// positions, plus the last neighbour n_d (n_d = n_0 when closed). Any other row (higher valence,
// several chains, an edge shared by more than two triangles) is "general": it stores its
// (j, l) pairs sorted, and is assembled by a block-per-row kernel.
//
// On request the build also resolves every triangle's 9 keys to storage positions (the
// element-to-nnz map, FE_PATTERN_MAP) and, for FE_PATTERN_GATHER, the per-non-zero lists of
// contributions c = 9k + 3*jl + il in ascending order (seg_ptr, perm).
#include <string>

#include "internal.cuh"

static constexpr int FAST_DEG = 32;    // rows with more triangles are handled by one block each
static constexpr int BIG_BLOCK = 256;
static constexpr int FAN_MAX = FE_FAN_MAX;   // longest fan the simple-row path handles in registers

enum { KIND_CLOSED = 0, KIND_OPEN = 1, KIND_GENERAL = 2 };

// ------------------------------------------------------------------ row digit (counting sort)

// Bucket entries of triangle k: for its vertex a, the two other vertices in counter-clockwise
// order (and, for the staged gather, the triangle/local id 3k + a). The cursors start at the
// bucket starts, so each atomic returns the entry's final slot. One thread handles the three
// vertices of a triangle; its three atomics are independent and issued together. (This pass is
// bound by random L2 transactions: one atomic and one store per incidence.)
__global__ void k_fill_adj(const int32_t* __restrict__ me, int32_t nme, int32_t* __restrict__ cur,
                           int2* __restrict__ adj, int32_t* __restrict__ vel) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[3] = {me[k], me[nme + k], me[2 * (int64_t)nme + k]};
        int32_t slot[3];
#pragma unroll
        for (int a = 0; a < 3; a++) slot[a] = FE_IDX(atomicAdd(&cur[v[a]], 1), 3 * (int64_t)nme);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            adj[slot[a]] = make_int2(v[(a + 1) % 3], v[(a + 2) % 3]);
            if (vel) vel[slot[a]] = 3 * (int32_t)k + a;
        }
    }
}

// ------------------------------------------------------------------ column digit, general rows

__device__ __forceinline__ void isort32(int32_t* x, int n) {
    for (int i = 1; i < n; i++) {
        int32_t v = x[i];
        int j = i - 1;
        while (j >= 0 && x[j] > v) { x[j + 1] = x[j]; j--; }
        x[j + 1] = v;
    }
}

__device__ __forceinline__ void isort64(long long* x, int n) {
    for (int i = 1; i < n; i++) {
        long long v = x[i];
        int j = i - 1;
        while (j >= 0 && x[j] > v) { x[j + 1] = x[j]; j--; }
        x[j + 1] = v;
    }
}


// ------------------------------------------------------------------ fans (simple rows)

// A row's fan with exactly D triangles (D <= FAN_MAX): triangle e is (i, J[e], L[e]),
// counter-clockwise. The analysis is written for a compile-time bound D on the row's valence n:
// a warp whose rows share their valence dispatches on it (n == D, so no loop runs over unused
// slots); a warp of mixed valences runs every row with D = FAN_MAX, the n..D-1 slots holding
// distinct negative ids that match no vertex and no other slot.
template <int D>
struct Fan {
    int32_t J[D], L[D];
};

template <int D>
__device__ __forceinline__ void load_fan(const int2* __restrict__ adj, int32_t beg, int n, Fan<D>& f) {
#pragma unroll
    for (int e = 0; e < D; e++) {
        int2 p = e < n ? adj[beg + e] : make_int2(-1 - e, -1 - e);
        f.J[e] = p.x;
        f.L[e] = p.y;
    }
}

// Analyses the fan: returns KIND_CLOSED / KIND_OPEN for one chain through all D triangles with
// distinct j's and distinct l's, else KIND_GENERAL. start = first triangle of the chain (for a
// closed fan, the one with the smallest j, so the order does not depend on the bucket order).
template <int D>
__device__ __forceinline__ int fan_kind(const Fan<D>& f, int n, int& start) {
    int nstart = 0, dup = 0, minj = INT32_MAX, minj_e = 0;
    start = 0;
#pragma unroll
    for (int e = 0; e < D; e++) {
        bool is_l = false;
#pragma unroll
        for (int g = 0; g < D; g++) {
            is_l |= f.L[g] == f.J[e];
            if (g > e) dup |= (f.J[g] == f.J[e]) | (f.L[g] == f.L[e]);
        }
        if (!is_l) { nstart++; start = e; }                // an unused slot is its own l: never a start
        if (e < n && f.J[e] < minj) { minj = f.J[e]; minj_e = e; }
    }
    if (dup || nstart > 1) return KIND_GENERAL;
    if (nstart == 0) start = minj_e;
    // follow the chain: it must visit every triangle once before closing (or ending)
    int32_t jstart = 0, lcur = 0;
#pragma unroll
    for (int e = 0; e < D; e++)
        if (e == start) { jstart = f.J[e]; lcur = f.L[e]; }
#pragma unroll
    for (int s = 1; s < D; s++) {
        if (s >= n) break;
        bool found = false;
        int32_t lnext = 0;
#pragma unroll
        for (int e = 0; e < D; e++)
            if (f.J[e] == lcur) { found = true; lnext = f.L[e]; }
        if (!found || lcur == jstart) return KIND_GENERAL;   // chain broken, or closed before the end
        lcur = lnext;
    }
    if (nstart == 0) return lcur == jstart ? KIND_CLOSED : KIND_GENERAL;
    return KIND_OPEN;
}

// Column position of vertex x in the row of vertex i with fan f (kind closed/open, last
// neighbour lend): the number of row entries below x.
template <int D>
__device__ __forceinline__ int fan_pos(const Fan<D>& f, int n, int32_t i, int kind, int32_t lend, int32_t x) {
    int p = (i < x) + (kind == KIND_OPEN && lend < x);
#pragma unroll
    for (int e = 0; e < D; e++) p += (e < n) & (f.J[e] < x);
    return p;
}

// Fan records and header of a simple row (closed or open fan with chain start `start`):
// fan-ordered neighbours with their column positions inside the row (fan[beg + e] = (n_e,
// pos(n_e))) and the header (n_d, pos_self | pos_nd << 14 | kind << 28). None of it depends on
// the row's CSR offset.
template <int D>
__device__ __forceinline__ void simple_row_records(int32_t i, int32_t beg, int n, int kind, int start, const Fan<D>& f,
                                                   int2* __restrict__ fan, int2* __restrict__ hdr) {
    int32_t jcur = 0, lcur = 0;
#pragma unroll
    for (int e = 0; e < D; e++)
        if (e == start) { jcur = f.J[e]; lcur = f.L[e]; }
    // the last neighbour: follow the chain to its end
    int32_t lend = lcur;
#pragma unroll
    for (int s = 1; s < D; s++) {
        if (s >= n) break;
        int32_t nl = lend;
#pragma unroll
        for (int e = 0; e < D; e++)
            if (f.J[e] == lend) nl = f.L[e];
        lend = nl;
    }
    int pself = fan_pos(f, n, i, kind, lend, i);
    int pend = fan_pos(f, n, i, kind, lend, lend);
#pragma unroll
    for (int s = 0; s < D; s++) {
        if (s >= n) break;
        fan[beg + s] = make_int2(jcur, fan_pos(f, n, i, kind, lend, jcur));
        int32_t nl = lcur;
#pragma unroll
        for (int e = 0; e < D; e++)
            if (f.J[e] == lcur) nl = f.L[e];
        jcur = lcur;
        lcur = nl;
    }
    hdr[i] = make_int2(lend, pself | (pend << 14) | (kind << 28));
}

// A simple row of valence n <= D: returns its column count, or 0 if the fan is not simple (then
// nothing is written).
template <int D>
__device__ __forceinline__ int32_t simple_row(int32_t i, int32_t beg, int n, const int2* __restrict__ adj,
                                              int2* __restrict__ fan, int2* __restrict__ hdr) {
    Fan<D> f;
    load_fan<D>(adj, beg, n, f);
    int start;
    int kind = fan_kind<D>(f, n, start);
    if (kind == KIND_GENERAL) return 0;
    simple_row_records<D>(i, beg, n, kind, start, f, fan, hdr);
    return n + 1 + (kind == KIND_OPEN);
}

// Row analysis, once per row: the column count, and everything of the row that does not depend
// on its CSR offset. Simple rows (one fan of at most FAN_MAX triangles): d + 1 entries (closed) or
// d + 2 (open), fan records and header. Other rows are general: those of at most FAST_DEG
// triangles are listed for one warp each, longer ones for one block each (k_row_big).
__global__ void k_row_analyse(const int32_t* __restrict__ vptr, const int2* __restrict__ adj, int32_t nq,
                              int32_t* __restrict__ row_nnz, int2* __restrict__ fan, int2* __restrict__ hdr,
                              int32_t* __restrict__ big_list, int32_t* __restrict__ big_count,
                              int32_t* __restrict__ mid_list, int32_t* __restrict__ mid_count, int* __restrict__ too_big) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = (int32_t)r;
        int32_t beg = vptr[i], d = vptr[i + 1] - beg;
        if (d == 0) { row_nnz[i] = 0; hdr[i] = make_int2(-1, KIND_GENERAL << 28); continue; }
        if (d <= FAN_MAX) {
            int32_t cnt = 0;
            // the warp's rows of valence 1..FAN_MAX: one specialisation if they share their valence,
            // else the bounded form for all (not one specialisation after another)
            const unsigned here = __activemask();
            if (__match_any_sync(here, d) == here) {
                switch (d) {
                    case 1: cnt = simple_row<1>(i, beg, 1, adj, fan, hdr); break;
                    case 2: cnt = simple_row<2>(i, beg, 2, adj, fan, hdr); break;
                    case 3: cnt = simple_row<3>(i, beg, 3, adj, fan, hdr); break;
                    case 4: cnt = simple_row<4>(i, beg, 4, adj, fan, hdr); break;
                    case 5: cnt = simple_row<5>(i, beg, 5, adj, fan, hdr); break;
                    case 6: cnt = simple_row<6>(i, beg, 6, adj, fan, hdr); break;
                    case 7: cnt = simple_row<7>(i, beg, 7, adj, fan, hdr); break;
                    default: cnt = simple_row<8>(i, beg, 8, adj, fan, hdr); break;
                }
            } else {
                cnt = simple_row<FAN_MAX>(i, beg, d, adj, fan, hdr);
            }
            static_assert(FAN_MAX == 8, "the valence dispatch covers 1..8");
            if (cnt > 0) {
                row_nnz[i] = cnt;
                continue;
            }
        }
        hdr[i] = make_int2(-1, KIND_GENERAL << 28);
        if (d > FAST_DEG) {
            if (d > FE_MAX_VALENCE) { *too_big = 1; row_nnz[i] = 0; continue; }
            big_list[atomicAdd(big_count, 1)] = i;
            continue;
        }
        // a medium general row: one warp of k_row_big does it (a lane sorting it here would hold
        // up the other 31 rows of its warp)
        mid_list[atomicAdd(mid_count, 1)] = i;
    }
}

// col_idx of the simple rows, once the offsets are known, from their fan records and header
// (general rows are placed by k_row_big). The 32 rows of a warp own one contiguous range of
// col_idx: the warp places its entries in shared memory first and writes the range with coalesced
// stores, leaving out the ranges of its general rows (scattered 4-byte stores made this pass
// L1-bound); a range too long for the staging area is written directly.
constexpr int CF_BLOCK = 256;
constexpr int CF_STAGE = 32 * (FAN_MAX + 2);                    // entries per warp (simple rows)
constexpr int32_t CF_SKIP = -1;                                  // a staged entry placed by another kernel

__global__ void __launch_bounds__(CF_BLOCK) k_col_fill(const int32_t* __restrict__ vptr, const int2* __restrict__ adj,
                                                       int32_t nq, const int32_t* __restrict__ row_ptr,
                                                       const int2* __restrict__ fan, const int2* __restrict__ hdr,
                                                       int32_t* __restrict__ col_idx) {
    __shared__ int32_t stage[CF_BLOCK / 32][CF_STAGE];
    const int lane = threadIdx.x & 31;
    int32_t* st = stage[threadIdx.x >> 5];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // every lane of a warp runs the same number of iterations (the loop bound is rounded up to a
    // multiple of 32 rows), so the warp-wide operations below see all 32 lanes
    const int64_t nq32 = ((int64_t)nq + 31) / 32 * 32;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq32; r += stride) {
        const bool act = r < nq;
        const int32_t i = (int32_t)r;
        int2 h = act ? hdr[i] : make_int2(0, 0);
        const int kind = act ? (h.y >> 28) : KIND_CLOSED;
        int32_t o = 0, e = 0, beg = 0, d = 0;
        if (act) {
            o = row_ptr[i];
            e = row_ptr[i + 1];
            beg = vptr[i];
            d = vptr[i + 1] - beg;
        }
        const bool general = act && kind == KIND_GENERAL;
        // the warp's range [lo, hi): rows are consecutive, so it starts at lane 0's offset and ends
        // at the last active lane's end
        const unsigned active = __ballot_sync(0xffffffffu, act);
        const int last = active ? 31 - __clz(active) : 0;
        const int32_t lo = __shfl_sync(0xffffffffu, o, 0);
        const int32_t hi = __shfl_sync(0xffffffffu, e, last);
        const bool staged = active && hi - lo <= CF_STAGE;                   // warp-uniform
        auto put = [&](int32_t at, int32_t v) {
            at = o + FE_IDX(at - o, e - o);                  // a column position inside its row
            if (staged) st[at - lo] = v;
            else col_idx[at] = v;
        };
        if (act && !general) {
            put(o + (h.y & 0x3FFF), i);
            if (kind == KIND_OPEN) put(o + ((h.y >> 14) & 0x3FFF), h.x);
            for (int32_t s = 0; s < d; s++) {
                int2 f = fan[beg + s];
                put(o + f.y, f.x);
            }
        } else if (general && staged) {
            // a general row: k_row_big places its columns later, so its range is marked to be
            // left out of the warp's copy
            for (int32_t t = o; t < e; t++) st[t - lo] = CF_SKIP;
        }
        if (staged) {
            __syncwarp();
            for (int32_t p = lane; p < hi - lo; p += 32) {
                const int32_t v = st[p];
                if (v != CF_SKIP) col_idx[lo + p] = v;
            }
            __syncwarp();
        }
    }
}

// ------------------------------------------------------------------ high-valence rows

// A medium general row (not one fan of at most FAN_MAX triangles, at most FAST_DEG triangles),
// one warp. Its columns are i and the distinct vertices among the 2d others of its triangles (none
// of which is i). Those 2d ids, two to a lane (element lane + 32 s), are sorted by a bitonic
// network over 64 elements (padded with INT32_MAX); an element is a column if it differs from the
// one before it, and its place is the number of such elements before it, plus one if i is
// smaller. Count pass (row_ptr null): the column count, the (j, l) pairs in lexicographic order
// (ties by bucket position, so a repeated triangle keeps both copies) and the row's place in the
// general-row list. Fill pass: the columns.
static_assert(2 * FAST_DEG <= 64, "a medium row's ids must fit two to a lane");
__device__ __forceinline__ void mid_row(int lane, int32_t i, int32_t beg, int32_t d, const int2* __restrict__ adj,
                                        const int32_t* __restrict__ row_ptr, int32_t* __restrict__ row_nnz,
                                        int32_t* __restrict__ col_idx, int2* __restrict__ fan,
                                        int32_t* __restrict__ gen_list, int32_t* __restrict__ gen_count) {
    const int2 p = lane < d ? adj[beg + lane] : make_int2(INT32_MAX, INT32_MAX);
    int32_t a0 = p.x, a1 = p.y;            // elements lane (slot 0) and lane + 32 (slot 1)
    // (element 2t and 2t + 1 of the row are triangle t's two vertices; the network sorts any order)
#pragma unroll
    for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j == 32) {
                // the partner is the same lane's other slot; for k = 64 every pair ascends
                const int32_t lo = min(a0, a1), hi = max(a0, a1);
                a0 = lo;
                a1 = hi;
            } else {
                const int32_t o0 = __shfl_xor_sync(0xffffffffu, a0, j);
                const int32_t o1 = __shfl_xor_sync(0xffffffffu, a1, j);
                const bool lower = (lane & j) == 0;
                const bool up0 = (lane & k) == 0, up1 = ((lane + 32) & k) == 0;
                a0 = (up0 == lower) ? min(a0, o0) : max(a0, o0);
                a1 = (up1 == lower) ? min(a1, o1) : max(a1, o1);
            }
        }
    }
    // the element before each: lane - 1 of the same slot, or lane 31 of slot 0 for slot 1's lane 0
    const int32_t prev0 = __shfl_up_sync(0xffffffffu, a0, 1);
    int32_t prev1 = __shfl_up_sync(0xffffffffu, a1, 1);
    const int32_t last0 = __shfl_sync(0xffffffffu, a0, 31);
    if (lane == 0) prev1 = last0;
    const bool new0 = a0 != INT32_MAX && (lane == 0 || a0 != prev0);
    const bool new1 = a1 != INT32_MAX && a1 != prev1;
    const unsigned b0 = __ballot_sync(0xffffffffu, new0), b1 = __ballot_sync(0xffffffffu, new1);
    const int ndist = __popc(b0) + __popc(b1);
    if (!row_ptr) {
        if (lane == 0) {
            row_nnz[i] = ndist + 1;
            gen_list[atomicAdd(gen_count, 1)] = i;
        }
        const long long key = ((long long)p.x << 32) | (unsigned)p.y;
        int rank = 0;
        for (int t = 0; t < d; t++) {
            const long long k2 = __shfl_sync(0xffffffffu, key, t);
            rank += (k2 < key) || (k2 == key && t < lane);
        }
        if (lane < d) fan[beg + FE_IDX(rank, d)] = p;
        return;
    }
    const unsigned below = (1u << lane) - 1u;
    const int r0 = __popc(b0 & below), r1 = __popc(b0) + __popc(b1 & below);
    // i's place: the distinct neighbours below it
    const int ri = __popc(__ballot_sync(0xffffffffu, new0 && a0 < i)) + __popc(__ballot_sync(0xffffffffu, new1 && a1 < i));
    const int32_t o = row_ptr[i], u = row_ptr[i + 1] - o;
    (void)u;                                                     // bounds of the checked build
    if (new0) col_idx[o + FE_IDX(r0 + (i < a0), u)] = a0;
    if (new1) col_idx[o + FE_IDX(r1 + (i < a1), u)] = a1;
    if (lane == 0) col_idx[o + FE_IDX(ri, u)] = i;
}

// General rows by k_row_big: those of more than FAST_DEG triangles one block each (the 2d+1
// columns go to shared memory; pass 1 flags the first occurrence of each value, pass 2 places
// each first occurrence at its rank among the distinct values), then the medium ones one warp
// each (mid_row). Count pass (row_ptr null): the column counts, and for the medium rows their
// sorted pairs and general-row list places; fill pass: the columns.
__global__ void k_row_big(const int32_t* __restrict__ big_list, const int32_t* __restrict__ nbig,
                          const int32_t* __restrict__ vptr, const int32_t* __restrict__ abase, const int2* __restrict__ adj,
                          const int32_t* __restrict__ row_ptr, int32_t* __restrict__ row_nnz,
                          int32_t* __restrict__ col_idx, const int32_t* __restrict__ mid_list,
                          const int32_t* __restrict__ nmid, int2* __restrict__ fan, int32_t* __restrict__ gen_list,
                          int32_t* __restrict__ gen_count) {
    extern __shared__ int32_t sm[];
    __shared__ int cnt;
  for (int32_t b = blockIdx.x; b < *nbig; b += gridDim.x) {
    __syncthreads();
    int32_t i = big_list[b];
    int32_t beg = abase[i], d = vptr[i + 1] - vptr[i];
    int n = 2 * d + 1;
    unsigned char* first = reinterpret_cast<unsigned char*>(sm + n);
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        int32_t v;
        if (t == 0) v = i;
        else { int2 p = adj[beg + (t - 1) / 2]; v = ((t - 1) & 1) ? p.y : p.x; }
        sm[t] = v;
    }
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        int32_t v = sm[t];
        unsigned char f = 1;
        for (int u = 0; u < t; u++) if (sm[u] == v) { f = 0; break; }
        first[t] = f;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        if (!first[t]) continue;
        int32_t v = sm[t];
        int less = 0;
        for (int u = 0; u < n; u++) less += (first[u] && sm[u] < v);
        atomicAdd(&cnt, 1);
        if (col_idx) col_idx[row_ptr[i] + less] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0 && row_nnz) row_nnz[i] = cnt;
  }
  const int lane = threadIdx.x & 31;
  const int32_t warp = (int32_t)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int32_t nwarps = (int32_t)(((int64_t)gridDim.x * blockDim.x) >> 5);
  for (int32_t b = warp; b < *nmid; b += nwarps) {
    const int32_t i = mid_list[b];
    mid_row(lane, i, abase[i], vptr[i + 1] - vptr[i], adj, row_ptr, row_nnz, col_idx, fan, gen_list, gen_count);
  }
}

// (j, l) pairs of a high-valence row in lexicographic order (rank of each 64-bit key).
__global__ void k_row_big_pairs(const int32_t* __restrict__ big_list, const int32_t* __restrict__ nbig,
                                const int32_t* __restrict__ vptr, const int32_t* __restrict__ abase, const int2* __restrict__ adj,
                                int2* __restrict__ fan, int2* __restrict__ hdr, int32_t* __restrict__ gen_list,
                                int32_t* __restrict__ gen_count) {
    extern __shared__ long long sk[];
  for (int32_t b = blockIdx.x; b < *nbig; b += gridDim.x) {
    __syncthreads();
    int32_t i = big_list[b];
    int32_t beg = vptr[i], d = vptr[i + 1] - beg, abeg = abase[i];
    for (int s = threadIdx.x; s < d; s += blockDim.x) {
        int2 p = adj[abeg + s];
        sk[s] = ((long long)p.x << 32) | (unsigned)p.y;
    }
    if (threadIdx.x == 0) {
        hdr[i] = make_int2(-1, KIND_GENERAL << 28);
        gen_list[atomicAdd(gen_count, 1)] = i;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < d; s += blockDim.x) {
        long long v = sk[s];
        int rank = 0;
        for (int t = 0; t < d; t++) rank += sk[t] < v;
        fan[beg + rank] = make_int2((int32_t)(v >> 32), (int32_t)(v & 0xffffffffLL));
    }
  }
}

// ------------------------------------------------------------------ staged-gather lists

// Contribution keys of row i: (col << 32 | c) for each of the 3 local columns of each triangle
// containing i, where c = 9k + 3*b + a (a = local index of i, b = local index of the column).
__device__ __forceinline__ void contrib_key(int32_t i, int2 p, int32_t e, long long out[3]) {
    int32_t k = e / 3;
    int a = e - 3 * k;
    int a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;
    long long base = 9LL * k + a;
    out[0] = ((long long)i << 32) | (base + 3 * a);
    out[1] = ((long long)p.x << 32) | (base + 3 * a1);
    out[2] = ((long long)p.y << 32) | (base + 3 * a2);
}

// Per non-zero, its contributions in ascending c (perm, grouped by seg_ptr), and the row's
// triangle list sorted by triangle (vel), for rows with at most FAST_DEG triangles.
__global__ void k_row_perm(const int32_t* __restrict__ vptr, const int32_t* __restrict__ abase, const int2* __restrict__ adj,
                           int32_t* __restrict__ vel,
                           int32_t nq, const int32_t* __restrict__ row_ptr, int32_t* __restrict__ seg_ptr,
                           int32_t* __restrict__ perm, int64_t n9) {
    long long keys[3 * FAST_DEG];
    int32_t ev[FAST_DEG];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t i = (int32_t)r;
        int32_t beg = vptr[i], d = vptr[i + 1] - beg;
        if (d == 0 || d > FAST_DEG) continue;
        int n = 0;
        for (int32_t s = 0; s < d; s++) {
            ev[s] = vel[beg + s];
            contrib_key(i, adj[abase[i] + s], ev[s], keys + n);
            n += 3;
        }
        isort64(keys, n);
        int32_t o = row_ptr[i], u = row_ptr[i + 1] - o;
        (void)u;                                                 // bounds of the checked build
        int32_t cbase = 3 * beg;   // this row's contributions occupy perm[3*vptr[i] .. 3*vptr[i+1])
        int t = 0;
        for (int s = 0; s < n; s++) {
            if (s == 0 || (keys[s] >> 32) != (keys[s - 1] >> 32)) seg_ptr[o + FE_IDX(t++, u)] = cbase + s;
            perm[FE_IDX(cbase + s, n9)] = FE_IDX((int32_t)(keys[s] & 0xffffffffLL), n9);
        }
        isort32(ev, d);
        for (int32_t s = 0; s < d; s++) vel[beg + s] = ev[s];
    }
}

// The same for a high-valence row, one block per row: 3d keys in shared memory (distinct, since
// c is unique). Pass 1: each key's rank among all keys gives its perm slot, and a key heads its
// column's segment if no smaller key has the same column. Pass 2: each head's rank among the
// heads is its column's position in the row. The row's triangle list is reordered by rank too.
__global__ void k_row_big_perm(const int32_t* __restrict__ big_list, const int32_t* __restrict__ nbig,
                               const int32_t* __restrict__ vptr, const int32_t* __restrict__ abase, const int2* __restrict__ adj,
                               int32_t* __restrict__ vel, const int32_t* __restrict__ row_ptr,
                               int32_t* __restrict__ seg_ptr, int32_t* __restrict__ perm) {
    extern __shared__ long long smk[];
  for (int32_t b = blockIdx.x; b < *nbig; b += gridDim.x) {
    __syncthreads();
    int32_t i = big_list[b];
    int32_t beg = vptr[i], d = vptr[i + 1] - beg;
    int n = 3 * d;
    int32_t* rank = reinterpret_cast<int32_t*>(smk + n);
    int32_t* vsort = rank + n;
    unsigned char* head = reinterpret_cast<unsigned char*>(vsort + d);
    for (int s = threadIdx.x; s < d; s += blockDim.x) {
        long long k3[3];
        contrib_key(i, adj[abase[i] + s], vel[beg + s], k3);
        smk[3 * s] = k3[0];
        smk[3 * s + 1] = k3[1];
        smk[3 * s + 2] = k3[2];
    }
    __syncthreads();
    int32_t cbase = 3 * beg;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        long long v = smk[t];
        int r = 0;
        unsigned char h = 1;
        for (int u = 0; u < n; u++) {
            long long w = smk[u];
            r += w < v;
            if ((w >> 32) == (v >> 32) && w < v) h = 0;
        }
        rank[t] = r;
        head[t] = h;
        perm[cbase + r] = (int32_t)(v & 0xffffffffLL);
    }
    for (int s = threadIdx.x; s < d; s += blockDim.x) {
        int32_t v = vel[beg + s];
        int r = 0;
        for (int u = 0; u < d; u++) r += vel[beg + u] < v;
        vsort[r] = v;
    }
    __syncthreads();
    int32_t o = row_ptr[i];
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        if (!head[t]) continue;
        long long col = smk[t] >> 32;
        int cr = 0;
        for (int u = 0; u < n; u++) cr += (head[u] && (smk[u] >> 32) < col);
        seg_ptr[o + cr] = cbase + rank[t];
    }
    for (int s = threadIdx.x; s < d; s += blockDim.x) vel[beg + s] = vsort[s];
  }
}

// ------------------------------------------------------------------ element-to-nnz map

// map[9k + 3b + a] = position of (me[a][k], me[b][k]); staged through shared memory so the
// 9 entries of consecutive triangles leave as one contiguous, coalesced block.
static constexpr int MAP_BLOCK = 256;

__global__ void k_build_map(const int32_t* __restrict__ me, int32_t nme, const int32_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col_idx, int32_t* __restrict__ map, int* __restrict__ missing) {
    __shared__ int32_t tile[9 * MAP_BLOCK];
    for (int64_t k0 = (int64_t)blockIdx.x * MAP_BLOCK; k0 < nme; k0 += (int64_t)gridDim.x * MAP_BLOCK) {
        int64_t k = k0 + threadIdx.x;
        if (k < nme) {
            int32_t v[3] = {me[k], me[nme + k], me[2 * (int64_t)nme + k]};
            for (int a = 0; a < 3; a++) {
                int32_t lo0 = row_ptr[v[a]], hi0 = row_ptr[v[a] + 1];
                for (int b = 0; b < 3; b++) {
                    int32_t lo = lo0, hi = hi0;
                    while (lo < hi) {
                        int32_t mid = (lo + hi) >> 1;
                        if (col_idx[mid] < v[b]) lo = mid + 1; else hi = mid;
                    }
                    if (lo >= hi0 || col_idx[lo] != v[b]) { *missing = 1; lo = 0; }
                    tile[9 * threadIdx.x + 3 * b + a] = lo;
                }
            }
        }
        __syncthreads();
        int64_t n = nme - k0 < MAP_BLOCK ? nme - k0 : MAP_BLOCK;
        for (int t = threadIdx.x; t < 9 * n; t += MAP_BLOCK) map[9 * k0 + t] = tile[t];
        __syncthreads();
    }
}

// 2x2 block expansion (elasticity): scalar row i with degree g gives rows 2i, 2i+1 with
// row_ptr2[2i+a] = 4 row_ptr[i] + 2 a g and columns 2j, 2j+1 for each scalar column j.
__global__ void k_expand(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t nq,
                         int32_t* __restrict__ row_ptr2, int32_t* __restrict__ col_idx2) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t b = row_ptr[r], g = row_ptr[r + 1] - b;
        for (int a = 0; a < 2; a++) {
            int32_t o = 4 * b + 2 * a * g;
            row_ptr2[2 * r + a] = o;
            for (int32_t t = 0; t < g; t++) {
                int32_t j = col_idx[b + t];
                col_idx2[o + 2 * t] = 2 * j;
                col_idx2[o + 2 * t + 1] = 2 * j + 1;
            }
        }
        if (r == nq - 1) row_ptr2[2 * (int64_t)nq] = 4 * row_ptr[nq];
    }
}

// seg_ptr[nnz] = 9 nme, with nnz read on the device (row_ptr[nq])
__global__ void k_set_last(int32_t* seg_ptr, const int32_t* row_ptr, int32_t nq, int32_t v) { seg_ptr[row_ptr[nq]] = v; }

// ------------------------------------------------------------------ driver

extern "C" void fe_pattern_destroy(fe_pattern p) {
    if (!p) return;
    FeStreamScope scope(p->last_stream);
    fe_free(p->row_ptr); fe_free(p->col_idx); fe_free(p->map);
    fe_free(p->row_ptr2); fe_free(p->col_idx2);
    fe_free(p->seg_ptr); fe_free(p->perm); fe_free(p->vptr); fe_free(p->vel); fe_free(p->kg);
    fe_free(p->fan); fe_free(p->hdr); fe_free(p->gen_rows); fe_free(p->row_ptr_w);
    fe_free(p->col_idx_w);
    delete p;
}

namespace {
struct Temps {
    int32_t *row_nnz = nullptr, *big_list = nullptr, *mid_list = nullptr, *counters = nullptr, *cur = nullptr;
    int* flag = nullptr;                 // points into counters (counters[0..1], flags[2..3], [4] medium rows)
    int2* adj = nullptr;
    ~Temps() {
        fe_free(row_nnz); fe_free(big_list); fe_free(mid_list); fe_free(counters); fe_free(adj);
        fe_free(cur);
    }
};
}  // namespace

static constexpr int BIG_GRID = 152;   // blocks of the high-valence kernels (they loop over the list)
static constexpr int ROW_BIG_GRID = 4 * 152;   // k_row_big: its medium rows take one warp each

// One host synchronisation: after the last kernel that can raise a flag, to read nnz and the
// flags. The row counts, the high-valence list and nnz stay on the device until then; col_idx is
// allocated at its upper bound (each row has at most 2 d + 1 entries: 6 nme + nq in all).
static fe_status build(fe_mesh m, int dofs, int flags, cudaStream_t s, fe_pattern p) {
    const int32_t nq = m->nq, nme = m->nme;
    const int64_t n3 = 3 * (int64_t)nme;
    const bool gather = flags & FE_PATTERN_GATHER;
    const bool want_map = gather || (flags & FE_PATTERN_MAP);
    const int64_t cap = 6 * (int64_t)nme + nq;
    if (cap >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "6*nme + nq must be < 2^31");
    Temps t;
    fe_status st;
    // Arrays are allocated just before their first use, so that the host-side allocation calls
    // overlap the kernels already queued instead of delaying the first one.
    if ((st = fe_alloc_n(&p->vptr, (size_t)nq + 1, "vertex pointers"))) return st;
    if ((st = fe_alloc_n(&t.cur, (size_t)nq + 1, "bucket cursors"))) return st;
    // row digit: counting sort of the 3 nme incidences (the counts come with the mesh: its
    // validation took them)
    if ((st = fe_exclusive_scan(m->deg, p->vptr, nq, s, nullptr, 1, t.cur))) return st;   // cursors start at the bucket starts
    if ((st = fe_alloc_n(&t.adj, (size_t)n3, "row buckets"))) return st;
    if (gather && (st = fe_alloc_n(&p->vel, (size_t)n3, "vertex-to-triangle lists"))) return st;
    if (nme > 0) {
        { FE_PROF("k_fill_adj", s); k_fill_adj<<<fe_grid(nme, 256, 16), 256, 0, s>>>(m->me, nme, t.cur, t.adj, p->vel); }
        FE_LAUNCHED("k_fill_adj");
    }
    // column digit inside each row, unique, and the CSR offsets
    if ((st = fe_alloc_n(&t.row_nnz, (size_t)nq + 1, "row counts"))) return st;
    if ((st = fe_alloc_n(&t.big_list, (size_t)nq + 1, "high-valence rows"))) return st;
    if ((st = fe_alloc_n(&t.mid_list, (size_t)nq + 1, "medium general rows"))) return st;
    // counters: [0] high-valence rows, [1] general rows, [2] a valence over the limit, [3] a key
    // missing from the pattern, [4] medium general rows
    if ((st = fe_alloc_n(&t.counters, 8, "counters and flags"))) return st;
    t.flag = t.counters + 2;
    if ((st = fe_alloc_n(&p->row_ptr, (size_t)nq + 1, "row_ptr"))) return st;
    if ((st = fe_alloc_n(&p->col_idx, (size_t)cap, "col_idx"))) return st;
    if ((st = fe_alloc_n(&p->fan, (size_t)n3, "row fans"))) return st;
    if ((st = fe_alloc_n(&p->hdr, (size_t)nq, "row fan headers"))) return st;
    if ((st = fe_alloc_n(&p->gen_rows, (size_t)nq + 1, "general-row list"))) return st;
    if (gather) {
        if ((st = fe_alloc_n(&p->seg_ptr, (size_t)cap + 1, "seg_ptr"))) return st;
        if ((st = fe_alloc_n(&p->perm, 9 * (size_t)nme, "perm"))) return st;
    }
    if (want_map && (st = fe_alloc_n(&p->map, 9 * (size_t)nme, "element-to-nnz map"))) return st;
    const size_t big_smem = (2 * (size_t)FE_MAX_VALENCE + 1) * (sizeof(int32_t) + 1);

    // counts and offset-free records (one fan analysis per row), offsets (scan of the counts),
    // then col_idx of the rows with at most FAST_DEG triangles
    auto rows = [&]() -> fe_status {
        fe_status sa;
        if (nq > 0) {
            { FE_PROF("k_row_analyse", s); k_row_analyse<<<fe_grid(nq, 128, 16), 128, 0, s>>>(p->vptr, t.adj, nq, t.row_nnz, p->fan, p->hdr, t.big_list,
                                                                                             t.counters, t.mid_list, t.counters + 4, t.flag); }
            FE_LAUNCHED("k_row_analyse");
            { FE_PROF("k_row_big", s); k_row_big<<<ROW_BIG_GRID, BIG_BLOCK, big_smem, s>>>(t.big_list, t.counters, p->vptr, p->vptr, t.adj, nullptr, t.row_nnz, nullptr,
                                                                                   t.mid_list, t.counters + 4, p->fan, p->gen_rows, t.counters + 1); }
            FE_LAUNCHED("k_row_big (count)");
        }
        if ((sa = fe_exclusive_scan(t.row_nnz, p->row_ptr, nq, s, nullptr))) return sa;
        if (nq > 0) {
            { FE_PROF("k_col_fill", s); k_col_fill<<<fe_grid(nq, CF_BLOCK, 8), CF_BLOCK, 0, s>>>(p->vptr, t.adj, nq, p->row_ptr, p->fan, p->hdr, p->col_idx); }
            FE_LAUNCHED("k_col_fill");
        }
        return FE_OK;
    };
    // high-valence rows, staged-gather lists, map (all need the offsets)
    auto rows_rest = [&]() -> fe_status {
        if (nq > 0) {
            { FE_PROF("k_row_big", s); k_row_big<<<ROW_BIG_GRID, BIG_BLOCK, big_smem, s>>>(t.big_list, t.counters, p->vptr, p->vptr, t.adj, p->row_ptr, nullptr, p->col_idx,
                                                                                   t.mid_list, t.counters + 4, nullptr, nullptr, nullptr); }
            FE_LAUNCHED("k_row_big (fill)");
            size_t pair_smem = (size_t)FE_MAX_VALENCE * sizeof(long long);
            { FE_PROF("k_row_big_pairs", s); k_row_big_pairs<<<BIG_GRID, BIG_BLOCK, pair_smem, s>>>(t.big_list, t.counters, p->vptr, p->vptr, t.adj, p->fan, p->hdr,
                                                                                                       p->gen_rows, t.counters + 1); }
            FE_LAUNCHED("k_row_big_pairs");
            if (gather) {
                { FE_PROF("k_row_perm", s); k_row_perm<<<fe_grid(nq, 128), 128, 0, s>>>(p->vptr, p->vptr, t.adj, p->vel, nq, p->row_ptr, p->seg_ptr, p->perm, 9 * (int64_t)nme); }
                FE_LAUNCHED("k_row_perm");
                size_t sm = 3 * (size_t)FE_MAX_VALENCE * (sizeof(long long) + sizeof(int32_t) + 1) +
                            (size_t)FE_MAX_VALENCE * sizeof(int32_t);
                FE_CUDA(cudaFuncSetAttribute(k_row_big_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
                { FE_PROF("k_row_big_perm", s); k_row_big_perm<<<BIG_GRID, BIG_BLOCK, sm, s>>>(t.big_list, t.counters, p->vptr, p->vptr, t.adj, p->vel, p->row_ptr, p->seg_ptr, p->perm); }
                FE_LAUNCHED("k_row_big_perm");
            }
        }
        if (gather) {
            { FE_PROF("k_set_last", s); k_set_last<<<1, 1, 0, s>>>(p->seg_ptr, p->row_ptr, nq, (int32_t)(9 * (int64_t)nme)); }
            FE_LAUNCHED("k_set_last");
        }
        if (want_map && nme > 0) {
            { FE_PROF("k_build_map", s); k_build_map<<<fe_grid(nme, MAP_BLOCK), MAP_BLOCK, 0, s>>>(m->me, nme, p->row_ptr, p->col_idx, p->map, t.flag + 1); }
            FE_LAUNCHED("k_build_map");
        }
        return FE_OK;
    };
    // one host synchronisation: flags, the counts of the lists, nnz
    int host_c[4] = {0, 0, 0, 0};
    int32_t tot32 = 0;
    int32_t wends[2] = {0, 0};
    auto read_back = [&]() -> fe_status {
        FE_CUDA(cudaMemcpyAsync(host_c, t.counters, sizeof host_c, cudaMemcpyDeviceToHost, s));
        FE_CUDA(cudaMemcpyAsync(&tot32, p->row_ptr + nq, sizeof tot32, cudaMemcpyDeviceToHost, s));
        if (p->row1 >= 0) {                               // a row window's ends (fe_pattern_build_rows)
            FE_CUDA(cudaMemcpyAsync(&wends[0], p->row_ptr + p->row0, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            FE_CUDA(cudaMemcpyAsync(&wends[1], p->row_ptr + p->row1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        }
        FE_CUDA(cudaStreamSynchronize(s));
        return FE_OK;
    };
    FE_CUDA(cudaMemsetAsync(t.counters, 0, 8 * sizeof(int32_t), s));
    if ((st = rows())) return st;
    if ((st = rows_rest())) return st;
    if ((st = read_back())) return st;
    if (host_c[2])
        return fe_fail(FE_ERR_LIMIT, "a vertex belongs to more than FE_MAX_VALENCE=" + std::to_string(FE_MAX_VALENCE) + " triangles");
    if (host_c[3]) return fe_fail(FE_ERR_CUDA, "internal error: a triangle key is missing from the pattern");
    int32_t host_counts[2] = {host_c[0], host_c[1]};
    const int64_t tot = tot32;
    p->nnz_scalar = tot;
    p->n_gen = host_counts[1];
    p->n_rows = nq;
    p->nnz = tot;
    if (p->row1 >= 0) {
        p->base_w = wends[0];
        p->n_rows = p->row1 - p->row0;
        p->nnz = (int64_t)wends[1] - wends[0];
    }
    if (dofs == 2) {
        if (4 * tot >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "elasticity nnz exceeds int32");
        if ((st = fe_alloc_n(&p->row_ptr2, 2 * (size_t)nq + 1, "row_ptr (dofs=2)"))) return st;
        if ((st = fe_alloc_n(&p->col_idx2, 4 * (size_t)tot, "col_idx (dofs=2)"))) return st;
        if (nq > 0) {
            { FE_PROF("k_expand", s); k_expand<<<fe_grid(nq, 256), 256, 0, s>>>(p->row_ptr, p->col_idx, nq, p->row_ptr2, p->col_idx2); }
            FE_LAUNCHED("k_expand");
        } else {
            FE_CUDA(cudaMemsetAsync(p->row_ptr2, 0, sizeof(int32_t), s));
        }
        p->n_rows = 2 * (int64_t)nq;
        p->nnz = 4 * tot;
    }
    if (gather) {
        size_t kg = dofs == 2 ? 36 * (size_t)nme : 18 * (size_t)nme;
        if ((st = fe_alloc_n(&p->kg, kg, "element value staging"))) return st;
    }
    return FE_OK;
}

static fe_status pattern_new(fe_mesh m, int dofs, int flags, fe_stream stream, fe_pattern* out, int32_t row0 = 0,
                             int32_t row1 = -1) {
    fe_pattern p = new fe_pattern_s();
    p->row0 = row0;
    p->row1 = row1;
    p->dofs = dofs;
    p->flags = flags;
    p->nq = m->nq;
    p->nme = m->nme;
    p->topology_id = m->topology_id;
    p->last_stream = (cudaStream_t)stream;
    FeStreamScope scope((cudaStream_t)stream);
    fe_status st = build(m, dofs, flags, (cudaStream_t)stream, p);
    if (st) {
        cudaStreamSynchronize((cudaStream_t)stream);
        fe_pattern_destroy(p);
        return st;
    }
    *out = p;
    return FE_OK;
}

extern "C" fe_status fe_pattern_build(fe_mesh m, int dofs, int flags, fe_stream stream, fe_pattern* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!m) return fe_fail(FE_ERR_INVALID_ARG, "null mesh");
    if (m->part1 >= 0)
        return fe_fail(FE_ERR_INVALID_ARG, "a part (fe_mesh_create_part) builds row windows of its owned rows only "
                                           "(fe_pattern_build_part)");
    if (dofs != 1 && dofs != 2) return fe_fail(FE_ERR_INVALID_ARG, "dofs_per_vertex must be 1 or 2");
    if (flags & ~(FE_PATTERN_GATHER | FE_PATTERN_MAP)) return fe_fail(FE_ERR_INVALID_ARG, "unknown pattern flag");
    if (dofs == 2 && 36 * (int64_t)m->nme >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "36*nme must be < 2^31");
    if (9 * (int64_t)m->nme >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "9*nme must be < 2^31");
    return pattern_new(m, dofs, flags, stream, out);
}

fe_status fe_pattern_build_rows(fe_mesh m, int32_t row0, int32_t row1, fe_stream stream, fe_pattern* out) {
    *out = nullptr;
    if (9 * (int64_t)m->nme >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "9*nme must be < 2^31");
    return pattern_new(m, 1, FE_PATTERN_DEFAULT, stream, out, row0, row1);
}

extern "C" fe_status fe_pattern_info(fe_pattern p, int64_t* n_rows, int64_t* nnz, const int32_t** row_ptr,
                                     const int32_t** col_idx) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (n_rows) *n_rows = p->n_rows;
    if (nnz) *nnz = p->nnz;
    if (p->row1 >= 0) {                                   // a row window: its rows only
        if (row_ptr) *row_ptr = p->row_ptr_w;
        if (col_idx) *col_idx = p->col_idx_w ? p->col_idx_w : p->col_idx + p->base_w;
        return FE_OK;
    }
    if (row_ptr) *row_ptr = p->dofs == 2 ? p->row_ptr2 : p->row_ptr;
    if (col_idx) *col_idx = p->dofs == 2 ? p->col_idx2 : p->col_idx;
    return FE_OK;
}

extern "C" fe_status fe_pattern_map(fe_pattern p, const int32_t** map, int64_t* len) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (!p->map) return fe_fail(FE_ERR_INVALID_ARG, "pattern built without FE_PATTERN_MAP");
    if (map) *map = p->map;
    if (len) *len = 9 * (int64_t)p->nme;
    return FE_OK;
}
