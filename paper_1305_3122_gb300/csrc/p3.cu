// p3.cu -- P3 (cubic) triangles: dof numbering, CSR structure and the mass and stiffness.
//
// The paper states that its method extends to P_k elements and gives no formulas; this is k = 3.
// With the barycentric coordinates l0, l1, l2 of a triangle (the P1 functions, grad l_a as in
// Eq. 4), the ten local dofs are the vertices (l_a (3 l_a - 1)(3 l_a - 2) / 2), two nodes on each
// edge (a, b) of (0,1), (1,2), (2,0) (9/2 l_a l_b (3 l_a - 1), then 9/2 l_a l_b (3 l_b - 1)) and the
// centroid (27 l0 l1 l2). The element matrices follow from the integrals of products of these
// polynomials, which are |T| times rational constants:
//   M^e_ij = |T| C_ij,
//   S^e_ij = sum over the pairs (k, l) in {(0,1), (1,2), (2,0)} of W^{kl}_ij (e_k . e_l) / (2D),
// with D = 2|T| and e_k the edge opposite vertex k (Eq. 3). The second form uses
// grad l_k . grad l_l = e_k . e_l / D^2 and, since the gradients of l0 + l1 + l2 = 1 sum to zero,
// |grad l_k|^2 = -(the sum of the other two products with grad l_k): writing
// I^{kl}_ij = (1/|T|) int_T (d phi_i / d l_k)(d phi_j / d l_l), W^{kl} = I^{kl} + I^{lk} - I^{kk} - I^{ll}.
// C and W are computed once on the host from the basis polynomials (monomials of the barycentric
// coordinates, integrated with int_T l0^a l1^b l2^c = 2|T| a! b! c! / (a + b + c + 2)!) and kept
// in constant memory.
//
// Dofs: vertex i is dof i; edge e (numbered from the scalar pattern as for P2: edges.cuh) owns
// nq + 2e (its node nearer the smaller vertex id) and nq + 2e + 1; triangle k's bubble is
// nq + 2 nE + k. Pattern: the incidences (element k, local dof a) are bucketed by dof with a
// counting sort; one warp per row merges the ten dofs of each of the row's elements in a
// shared-memory hash table (rowhash.cuh), ranks the distinct ids (the sorted columns) and writes
// each incidence's ten in-row positions (the element-to-nnz map, row-major per element:
// map[100k + 10 il + jl]), made absolute once the offsets are known. Assembly: one thread per
// element in FP64 with 100 FP64 atomics; or, deterministic, the element matrices staged and one
// warp per row adding its incidences' element rows in ascending element order (the row pass lists
// each row's incidences in that order with their column positions), so that every non-zero sums its
// contributions in ascending element order, bit-identical from run to run.
#include <string>

#include "edges.cuh"
#include "rowhash.cuh"

namespace {

constexpr int P3_BLOCK = 256;
constexpr int P3_WARPS = 4;
constexpr int FAST_TS = 128, FAST_EMAX = 12;                  // 10 * 12 ids < 128 slots
constexpr int BIG_TS = 4096, BIG_EMAX = FE_P3_MAX_VALENCE;    // 10 * 400 ids < 4096 slots
static_assert(10 * FAST_EMAX < FAST_TS && 10 * BIG_EMAX < BIG_TS, "tables hold every id");
constexpr int RS_FAST = 10 * FAST_EMAX;                       // row-sum accumulators of a warp (fast rows)
constexpr int RS_SHORT = 16;                                  // row-sum accumulators of a thread (edge and bubble rows)
constexpr int RS_BLOCK = 128;

// Element dofs (edof[10k .. 10k+9]) and the dofs' element counts.
__global__ void k_p3_edof(const int32_t* __restrict__ me, int32_t nme, int32_t nq, const int32_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ col_idx, const int32_t* __restrict__ eoff,
                          const int32_t* __restrict__ dpos, int64_t ne, int32_t* __restrict__ edof,
                          int32_t* __restrict__ deg) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v[3] = {me[k], me[nme + k], me[2 * (int64_t)nme + k]};
        int32_t d[10];
#pragma unroll
        for (int a = 0; a < 3; a++) d[a] = v[a];
#pragma unroll
        for (int t = 0; t < 3; t++) {
            const int32_t a = v[t], b = v[t == 2 ? 0 : t + 1];
            const int32_t base = nq + 2 * edge_rank(row_ptr, col_idx, eoff, dpos, a, b);
            d[3 + 2 * t] = base + (a < b ? 0 : 1);                 // the node nearer a
            d[4 + 2 * t] = base + (a < b ? 1 : 0);                 // the node nearer b
        }
        d[9] = (int32_t)(nq + 2 * ne + k);
        int2* o = reinterpret_cast<int2*>(edof + 10 * k);
#pragma unroll
        for (int j = 0; j < 5; j++) o[j] = make_int2(d[2 * j], d[2 * j + 1]);
#pragma unroll
        for (int a = 0; a < 10; a++) atomicAdd(&deg[d[a]], 1);
    }
}

__global__ void k_p3_fill(const int32_t* __restrict__ edof, int32_t nme, int32_t* __restrict__ cur,
                          int32_t* __restrict__ inc) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 10; a++)
            inc[FE_IDX(atomicAdd(&cur[edof[10 * k + a]], 1), 10 * (int64_t)nme)] = 10 * (int32_t)k + a;
    }
}

template <int TS, int EMAX>
struct P3Smem {
    int32_t tab[TS];
    int32_t rnk[TS];
    int32_t uid[TS];
    int32_t uslot[TS];
    int32_t key[EMAX];
    int16_t xs[10 * EMAX];   // the slot of each incidence's ten ids
    int32_t ucount;
};

// Where the row pass puts the deterministic variant's lists (ikey null: no lists).
struct P3Lists {
    int32_t* ikey;       // [10 nme] each row's incidence keys 10k + a in ascending order, row r from vptr[r]
    int32_t* ipos;       // [10 nme][5] their ten in-row column positions, 16 bits each
    int32_t* long_rows;  // rows of more than RS_FAST columns (summed by k_p3_rowsum_long)
    int32_t* n_long;     // their number
};

// One row by one warp: its sorted distinct columns into tmp at 10 vptr[r] (each incidence brings
// at most ten), their count, and the ten relative positions of every incidence in map.
template <int TS, int EMAX>
__device__ void p3_row(int32_t r, int32_t beg, int32_t d, const int32_t* __restrict__ inc, const int32_t* __restrict__ edof,
                       P3Smem<TS, EMAX>& sm, int32_t* __restrict__ tmp, int32_t* __restrict__ cnt,
                       int32_t* __restrict__ map, const P3Lists& ls) {
    const int lane = threadIdx.x & 31;
    for (int s = lane; s < TS; s += 32) sm.tab[s] = -1;
    if (lane == 0) sm.ucount = 0;
    for (int t = lane; t < d; t += 32) sm.key[t] = inc[beg + t];
    __syncwarp();
    for (int x = lane; x < 10 * d; x += 32) {
        const int32_t id = edof[10 * (int64_t)(sm.key[x / 10] / 10) + x % 10];
        bool fresh;
        const int s = tab_insert<TS>(sm.tab, id, &fresh);
        sm.xs[x] = (int16_t)s;
        if (fresh) {
            const int p = atomicAdd(&sm.ucount, 1);
            sm.uid[p] = id;
            sm.uslot[p] = s;
        }
    }
    __syncwarp();
    const int u = sm.ucount;
    const int64_t tb = 10 * (int64_t)beg;
    for (int p = lane; p < u; p += 32) {
        const int32_t id = sm.uid[p];
        int rk = 0;
        for (int qq = 0; qq < u; qq++) rk += sm.uid[qq] < id;
        sm.rnk[sm.uslot[p]] = rk;
        tmp[tb + rk] = id;
    }
    __syncwarp();
    for (int t = lane; t < d; t += 32) {
        const int32_t kk = sm.key[t] / 10, a = sm.key[t] - 10 * kk;
        int32_t* mo = map + 100 * (int64_t)kk + 10 * a;
        int32_t o[10];
#pragma unroll
        for (int jl = 0; jl < 10; jl++) {
            o[jl] = sm.rnk[sm.xs[10 * t + jl]];              // the slot its insertion got
            mo[jl] = o[jl];
        }
        if (ls.ikey) {                                        // the incidence's place in element order
            int c0 = 0;
            for (int tt = 0; tt < d; tt++) c0 += sm.key[tt] < sm.key[t];
            ls.ikey[beg + c0] = sm.key[t];
            int32_t* po = ls.ipos + 5 * (int64_t)(beg + c0);
#pragma unroll
            for (int j = 0; j < 5; j++) po[j] = (int32_t)((unsigned)o[2 * j] | ((unsigned)o[2 * j + 1] << 16));
        }
    }
    if (lane == 0) {
        cnt[r] = u;
        if (ls.ikey && u > RS_FAST) ls.long_rows[atomicAdd(ls.n_long, 1)] = r;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(P3_WARPS * 32) k_p3_rows(const int32_t* __restrict__ vptr, const int32_t* __restrict__ inc,
                                                           const int32_t* __restrict__ edof, int32_t nrows,
                                                           int32_t* __restrict__ tmp, int32_t* __restrict__ cnt,
                                                           int32_t* __restrict__ map, int32_t* __restrict__ big_list,
                                                           int32_t* __restrict__ big_count, P3Lists ls) {
    __shared__ P3Smem<FAST_TS, FAST_EMAX> sm_all[P3_WARPS];
    P3Smem<FAST_TS, FAST_EMAX>& sm = sm_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    for (int64_t rr = (int64_t)blockIdx.x * P3_WARPS + (threadIdx.x >> 5); rr < nrows; rr += (int64_t)gridDim.x * P3_WARPS) {
        const int32_t r = (int32_t)rr, beg = vptr[r], d = vptr[r + 1] - beg;
        if (d <= 2) continue;                                    // k_p3_short_rows
        if (d > FAST_EMAX) {
            if (lane == 0) big_list[atomicAdd(big_count, 1)] = r;
            continue;
        }
        p3_row<FAST_TS, FAST_EMAX>(r, beg, d, inc, edof, sm, tmp, cnt, map, ls);
    }
}

// The rows of at most two elements (an edge's dofs in a manifold mesh, a bubble, an unused
// vertex), one thread each: the at most 20 ids sorted in registers (a fixed compare-exchange
// sequence: static indices only); the rank of a value is the number of distinct smaller ones.
__global__ void __launch_bounds__(P3_BLOCK) k_p3_short_rows(const int32_t* __restrict__ vptr, const int32_t* __restrict__ inc,
                                                            const int32_t* __restrict__ edof, int32_t nrows,
                                                            int32_t* __restrict__ tmp, int32_t* __restrict__ cnt,
                                                            int32_t* __restrict__ map, P3Lists ls) {
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < nrows; rr += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)rr, beg = vptr[r], d = vptr[r + 1] - beg;
        if (d > 2) continue;
        int32_t key[2] = {d > 0 ? inc[beg] : -1, d > 1 ? inc[beg + 1] : -1};
        if (key[1] >= 0 && key[1] < key[0]) {                   // ascending element order
            const int32_t x = key[0];
            key[0] = key[1];
            key[1] = x;
        }
        int32_t x[20];
#pragma unroll
        for (int t = 0; t < 2; t++)
#pragma unroll
            for (int j = 0; j < 10; j++) x[10 * t + j] = key[t] >= 0 ? edof[10 * (int64_t)(key[t] / 10) + j] : INT32_MAX;
#pragma unroll
        for (int i = 1; i < 20; i++)
#pragma unroll
            for (int j = i; j > 0; j--) {
                const int32_t lo = min(x[j - 1], x[j]), hi = max(x[j - 1], x[j]);
                x[j - 1] = lo;
                x[j] = hi;
            }
        const int64_t tb = 10 * (int64_t)beg;
        int u = 0;
#pragma unroll
        for (int i = 0; i < 20; i++) {
            const bool first = x[i] != INT32_MAX && (i == 0 || x[i] != x[i - 1]);
            if (first) tmp[tb + u] = x[i];
            u += first;
        }
        cnt[r] = u;
#pragma unroll
        for (int t = 0; t < 2; t++) {
            if (key[t] < 0) continue;
            const int32_t kk = key[t] / 10, a = key[t] - 10 * kk;
            const int32_t* e = edof + 10 * (int64_t)kk;
            int32_t* o = map + 100 * (int64_t)kk + 10 * a;
            unsigned sl[10];
#pragma unroll
            for (int jl = 0; jl < 10; jl++) {
                const int32_t v = e[jl];
                int rank = 0;
#pragma unroll
                for (int i = 0; i < 20; i++) rank += x[i] < v && (i == 0 || x[i] != x[i - 1]);
                o[jl] = rank;
                sl[jl] = (unsigned)rank;
            }
            if (ls.ikey) {                                       // key[] is in ascending order: place t
                ls.ikey[beg + t] = key[t];
                int32_t* po = ls.ipos + 5 * (int64_t)(beg + t);
#pragma unroll
                for (int j = 0; j < 5; j++) po[j] = (int32_t)(sl[2 * j] | (sl[2 * j + 1] << 16));
            }
        }
    }
}

// The rows of more than FAST_EMAX elements, one warp each (tables in dynamic shared memory).
__global__ void __launch_bounds__(32) k_p3_rows_big(const int32_t* __restrict__ vptr, const int32_t* __restrict__ inc,
                                                    const int32_t* __restrict__ edof, const int32_t* __restrict__ big_list,
                                                    const int32_t* __restrict__ big_count, int32_t* __restrict__ tmp,
                                                    int32_t* __restrict__ cnt, int32_t* __restrict__ map,
                                                    int* __restrict__ too_big, P3Lists ls) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P3Smem<BIG_TS, BIG_EMAX>& sm = *reinterpret_cast<P3Smem<BIG_TS, BIG_EMAX>*>(smem_raw);
    const int32_t n = *big_count;
    for (int32_t b = blockIdx.x; b < n; b += gridDim.x) {
        const int32_t r = big_list[b], beg = vptr[r], d = vptr[r + 1] - beg;
        if (d > BIG_EMAX) {
            if (threadIdx.x == 0) {
                *too_big = 1;
                cnt[r] = 0;
            }
            continue;
        }
        p3_row<BIG_TS, BIG_EMAX>(r, beg, d, inc, edof, sm, tmp, cnt, map, ls);
    }
}

// col_idx from the rows' sorted columns: a warp takes 32 consecutive rows and copies them one
// after another, its lanes over the row's entries (coalesced loads and stores).
__global__ void __launch_bounds__(P3_BLOCK) k_p3_cols(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                      int32_t ndof, const int32_t* __restrict__ tmp, int32_t* __restrict__ col_idx) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r0 = 32 * ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); r0 < ndof; r0 += 32 * warps) {
        const int64_t mine = r0 + lane;
        int32_t rb = 0, u = 0;
        int64_t tb = 0;
        if (mine < ndof) {
            rb = row_ptr[mine];
            u = row_ptr[mine + 1] - rb;
            tb = 10 * (int64_t)vptr[mine];
        }
        for (int j = 0; j < 32 && r0 + j < ndof; j++) {
            const int32_t b = __shfl_sync(0xffffffffu, rb, j), n = __shfl_sync(0xffffffffu, u, j);
            const int64_t t = __shfl_sync(0xffffffffu, tb, j);
            for (int c = lane; c < n; c += 32) col_idx[b + c] = tmp[t + c];
        }
    }
}

// The map's in-row positions made absolute: map[100k + 10 il + jl] += row_ptr[edof[k][il]].
__global__ void k_p3_map_base(const int32_t* __restrict__ edof, int32_t nme, const int32_t* __restrict__ row_ptr,
                              int32_t* __restrict__ map) {
    const int64_t n = 100 * (int64_t)nme;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = c / 100;
        const int il = (int)((c - 100 * k) / 10);
        map[c] += row_ptr[edof[10 * k + il]];
    }
}

// ------------------------------------------------------------------ element matrices

// C (mass, times |T|) and W (stiffness, per pair (0,1), (1,2), (2,0)): row-major 10 x 10.
__constant__ double c_p3_mass[100];
__constant__ double c_p3_w[3][100];

// One thread per element: the 100 entries, added with FP64 atomics through the map. The entries
// are formed one at a time from the three edge products (constant-memory tables, the same entry
// for the whole warp at a time), so no 10 x 10 matrix is held in registers.
template <int KIND>
__global__ void __launch_bounds__(P3_BLOCK) k_p3_atomic(const int32_t* __restrict__ me, int32_t nme, const double2* __restrict__ q,
                                                        const int32_t* __restrict__ map, double* __restrict__ val, int64_t nnz) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        const double2 p0 = q[me[k]], p1 = q[me[nme + k]], p2 = q[me[2 * (int64_t)nme + k]];
        const double ex[3] = {p1.x - p2.x, p2.x - p0.x, p0.x - p1.x};
        const double ey[3] = {p1.y - p2.y, p2.y - p0.y, p0.y - p1.y};
        const double D = ex[1] * ey[2] - ex[2] * ey[1];
        const double T = 0.5 * D, s = 0.5 / D;
        const double c01 = (ex[0] * ex[1] + ey[0] * ey[1]) * s, c12 = (ex[1] * ex[2] + ey[1] * ey[2]) * s,
                     c20 = (ex[2] * ex[0] + ey[2] * ey[0]) * s;
        const int32_t* mk = map + 100 * k;
#pragma unroll 10
        for (int t = 0; t < 100; t++) {
            const double v = KIND == FE_P3_MASS ? T * c_p3_mass[t]
                                                : c01 * c_p3_w[0][t] + c12 * c_p3_w[1][t] + c20 * c_p3_w[2][t];
            atomicAdd(&val[FE_IDX(mk[t], nnz)], v);
        }
    }
}

// The element matrices into the staging buffer, row-major per element (kg[100k + 10 il + jl]).
// Threads of a block take consecutive elements and write their 100 values through shared memory,
// so that the block's stores cover one contiguous range.
constexpr int STAGE_BLOCK = 64;

template <int KIND>
__global__ void __launch_bounds__(STAGE_BLOCK) k_p3_stage(const int32_t* __restrict__ me, int32_t nme, const double2* __restrict__ q,
                                                          double* __restrict__ kg) {
    __shared__ double tile[STAGE_BLOCK * 101];                // rows of 101: the threads' writes fall in different banks
    for (int64_t k0 = (int64_t)blockIdx.x * STAGE_BLOCK; k0 < nme; k0 += (int64_t)gridDim.x * STAGE_BLOCK) {
        const int64_t k = k0 + threadIdx.x;
        if (k < nme) {
            const double2 p0 = q[me[k]], p1 = q[me[nme + k]], p2 = q[me[2 * (int64_t)nme + k]];
            const double ex[3] = {p1.x - p2.x, p2.x - p0.x, p0.x - p1.x};
            const double ey[3] = {p1.y - p2.y, p2.y - p0.y, p0.y - p1.y};
            const double D = ex[1] * ey[2] - ex[2] * ey[1];
            const double T = 0.5 * D, s = 0.5 / D;
            const double c01 = (ex[0] * ex[1] + ey[0] * ey[1]) * s, c12 = (ex[1] * ex[2] + ey[1] * ey[2]) * s,
                         c20 = (ex[2] * ex[0] + ey[2] * ey[0]) * s;
#pragma unroll 10
            for (int t = 0; t < 100; t++)
                tile[threadIdx.x * 101 + t] = KIND == FE_P3_MASS ? T * c_p3_mass[t]
                                                                 : c01 * c_p3_w[0][t] + c12 * c_p3_w[1][t] + c20 * c_p3_w[2][t];
        }
        __syncthreads();
        const int n = (int)min((int64_t)STAGE_BLOCK, (int64_t)nme - k0);
        for (int c = threadIdx.x; c < 100 * n; c += STAGE_BLOCK) kg[100 * k0 + c] = tile[(c / 100) * 101 + c % 100];
        __syncthreads();
    }
}

// Row sums of the staged matrices, one warp per row: the row's incidences in ascending element
// order each add row a of element k (kg[100k + 10a ..], ten values, one per lane of lanes 0..9)
// into the row's accumulators in shared memory at the incidence's ten column positions (distinct,
// so the lanes never collide). Accumulators start at -0.0, so every sum equals its first
// contribution followed by the others in ascending element order, bit for bit. acc: this warp's
// accumulators (at least the row's column count).
__device__ __forceinline__ void p3_rowsum(int32_t r, const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                          const int32_t* __restrict__ ikey, const int32_t* __restrict__ ipos,
                                          const double* __restrict__ kg, double* __restrict__ val, double* acc,
                                          int64_t n10) {
    const int lane = threadIdx.x & 31;
    const int32_t rb = row_ptr[r], u = row_ptr[r + 1] - rb;
    const int32_t b0 = vptr[r], d = vptr[r + 1] - b0;
    for (int c = lane; c < u; c += 32) acc[c] = -0.0;
    __syncwarp();
    for (int32_t t = 0; t < d; t++) {
        if (lane < 10) {
            const int32_t key = FE_IDX(ikey[b0 + t], n10);
            const unsigned pw = (unsigned)ipos[5 * (int64_t)(b0 + t) + (lane >> 1)];
            const int pos = FE_IDX((int)((pw >> (16 * (lane & 1))) & 0xFFFFu), u);
            acc[pos] += kg[10 * (int64_t)key + lane];             // 100k + 10a + lane
        }
        __syncwarp();
    }
    for (int c = lane; c < u; c += 32) val[rb + c] = acc[c];
    __syncwarp();
}

__global__ void __launch_bounds__(P3_WARPS * 32) k_p3_rowsum(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                             int32_t ndof, const int32_t* __restrict__ ikey,
                                                             const int32_t* __restrict__ ipos, const double* __restrict__ kg,
                                                             double* __restrict__ val, int64_t n10) {
    __shared__ double acc_all[P3_WARPS][RS_FAST];
    double* acc = acc_all[threadIdx.x >> 5];
    for (int64_t rr = (int64_t)blockIdx.x * P3_WARPS + (threadIdx.x >> 5); rr < ndof; rr += (int64_t)gridDim.x * P3_WARPS) {
        const int32_t r = (int32_t)rr, u = row_ptr[r + 1] - row_ptr[r];
        if (u <= RS_SHORT || u > RS_FAST) continue;             // k_p3_rowsum_short, k_p3_rowsum_long
        p3_rowsum(r, vptr, row_ptr, ikey, ipos, kg, val, acc, n10);
    }
}

// The rows of at most RS_SHORT columns (an interior edge's two dofs: 16 columns, a bubble: 10),
// one thread each: accumulators in shared memory (column c of this thread's row at
// acc[c * RS_BLOCK]), the incidences' ten entries added in ascending element order, starting
// from -0.0 as in p3_rowsum, so the sums are the same bit for bit.
__global__ void __launch_bounds__(RS_BLOCK) k_p3_rowsum_short(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                              int32_t ndof, const int32_t* __restrict__ ikey,
                                                              const int32_t* __restrict__ ipos, const double* __restrict__ kg,
                                                              double* __restrict__ val, int64_t n10) {
    __shared__ double acc_all[RS_SHORT * RS_BLOCK];
    double* acc = acc_all + threadIdx.x;
    for (int64_t r = blockIdx.x * (int64_t)RS_BLOCK + threadIdx.x; r < ndof; r += (int64_t)gridDim.x * RS_BLOCK) {
        const int32_t rb = row_ptr[r], u = row_ptr[r + 1] - rb;
        if (u > RS_SHORT) continue;
        const int32_t b0 = vptr[r], d = vptr[r + 1] - b0;
        for (int c = 0; c < u; c++) acc[c * RS_BLOCK] = -0.0;
        for (int32_t t = 0; t < d; t++) {
            const int32_t key = FE_IDX(ikey[b0 + t], n10);
            const int32_t* pw = ipos + 5 * (int64_t)(b0 + t);
            const double2* e = reinterpret_cast<const double2*>(kg + 10 * (int64_t)key);   // 100k + 10a: 16-byte aligned
            double v[10];
            unsigned w[5];
#pragma unroll
            for (int j = 0; j < 5; j++) {
                const double2 x = e[j];
                v[2 * j] = x.x;
                v[2 * j + 1] = x.y;
                w[j] = (unsigned)pw[j];
            }
            // an incidence's ten columns are distinct: all ten accumulators are read before any
            // is written back
            double* pc[10];
            double y[10];
#pragma unroll
            for (int j = 0; j < 10; j++) pc[j] = acc + FE_IDX((int)((w[j >> 1] >> (16 * (j & 1))) & 0xFFFFu), u) * RS_BLOCK;
#pragma unroll
            for (int j = 0; j < 10; j++) y[j] = *pc[j];
#pragma unroll
            for (int j = 0; j < 10; j++) *pc[j] = y[j] + v[j];
        }
        for (int c = 0; c < u; c++) val[rb + c] = acc[c * RS_BLOCK];
    }
}

// The rows longer than RS_FAST columns (listed by the row pass), one warp each, accumulators in
// dynamic shared memory.
__global__ void __launch_bounds__(32) k_p3_rowsum_long(const int32_t* __restrict__ long_rows, int32_t n_long,
                                                       const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ ikey, const int32_t* __restrict__ ipos,
                                                       const double* __restrict__ kg, double* __restrict__ val, int64_t n10) {
    extern __shared__ double acc_long[];
    for (int32_t b = blockIdx.x; b < n_long; b += gridDim.x)
        p3_rowsum(long_rows[b], vptr, row_ptr, ikey, ipos, kg, val, acc_long, n10);
}

}  // namespace

// ------------------------------------------------------------------ host: element constants
//
// The basis functions as lists of terms coef * l0^a l1^b l2^c; products and derivatives term by
// term; integrals over T divided by |T| with 2 a! b! c! / (a + b + c + 2)!. Degrees stay below 7.

#include <mutex>
#include <vector>

namespace {

struct Term {
    double c;
    int e[3];
};
using Poly = std::vector<Term>;

double fact(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= i; return f; }

double integral_over_area(const Poly& p) {
    double s = 0.0;
    for (const Term& t : p) s += t.c * 2.0 * fact(t.e[0]) * fact(t.e[1]) * fact(t.e[2]) / fact(t.e[0] + t.e[1] + t.e[2] + 2);
    return s;
}

Poly times(const Poly& a, const Poly& b) {
    Poly out;
    for (const Term& x : a)
        for (const Term& y : b) out.push_back(Term{x.c * y.c, {x.e[0] + y.e[0], x.e[1] + y.e[1], x.e[2] + y.e[2]}});
    return out;
}

Poly d_dl(const Poly& a, int k) {
    Poly out;
    for (const Term& t : a)
        if (t.e[k] > 0) {
            Term u = t;
            u.c *= t.e[k];
            u.e[k] -= 1;
            out.push_back(u);
        }
    return out;
}

// the ten local basis functions (local dof order of the header)
std::vector<Poly> p3_basis() {
    std::vector<Poly> phi(10);
    for (int a = 0; a < 3; a++) {                             // l (3l - 1)(3l - 2)/2 = 9/2 l^3 - 9/2 l^2 + l
        Term t3{4.5, {0, 0, 0}}, t2{-4.5, {0, 0, 0}}, t1{1.0, {0, 0, 0}};
        t3.e[a] = 3; t2.e[a] = 2; t1.e[a] = 1;
        phi[a] = {t3, t2, t1};
    }
    for (int t = 0; t < 3; t++) {
        const int a = t, b = (t + 1) % 3;
        for (int side = 0; side < 2; side++) {                // 9/2 l_a l_b (3 l_n - 1), n = a then b
            const int n = side == 0 ? a : b;
            Term hi{13.5, {0, 0, 0}}, lo{-4.5, {0, 0, 0}};
            hi.e[a] += 1; hi.e[b] += 1; hi.e[n] += 1;
            lo.e[a] += 1; lo.e[b] += 1;
            phi[3 + 2 * t + side] = {hi, lo};
        }
    }
    phi[9] = {Term{27.0, {1, 1, 1}}};
    return phi;
}

struct P3Tables {
    double mass[100];
    double w[3][100];
};

P3Tables make_tables() {
    P3Tables tb;
    const std::vector<Poly> phi = p3_basis();
    std::vector<std::vector<Poly>> d(10, std::vector<Poly>(3));
    for (int i = 0; i < 10; i++)
        for (int k = 0; k < 3; k++) d[i][k] = d_dl(phi[i], k);
    const int pk[3] = {0, 1, 2}, pl[3] = {1, 2, 0};            // the pairs (0,1), (1,2), (2,0)
    for (int i = 0; i < 10; i++)
        for (int j = 0; j < 10; j++) {
            tb.mass[10 * i + j] = integral_over_area(times(phi[i], phi[j]));
            double I[3][3];
            for (int k = 0; k < 3; k++)
                for (int l = 0; l < 3; l++) I[k][l] = integral_over_area(times(d[i][k], d[j][l]));
            for (int p = 0; p < 3; p++) {
                const int k = pk[p], l = pl[p];
                tb.w[p][10 * i + j] = I[k][l] + I[l][k] - I[k][k] - I[l][l];
            }
        }
    return tb;
}

// The constant tables on the current device, once per device.
fe_status p3_tables_ready() {
    static std::mutex mu;
    static bool ready[64] = {};
    static P3Tables tb = make_tables();
    int dev = 0;
    FE_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fe_fail(FE_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[dev]) {
        FE_CUDA(cudaMemcpyToSymbol(c_p3_mass, tb.mass, sizeof tb.mass));
        FE_CUDA(cudaMemcpyToSymbol(c_p3_w, tb.w, sizeof tb.w));
        ready[dev] = true;
    }
    return FE_OK;
}

struct P3Temps {
    int32_t *ucnt = nullptr, *dpos = nullptr, *eoff = nullptr, *deg = nullptr, *vptr = nullptr, *cur = nullptr;
    int32_t *inc = nullptr, *cnt = nullptr, *tmp = nullptr, *big = nullptr, *counters = nullptr;
    ~P3Temps() {
        fe_free(ucnt); fe_free(dpos); fe_free(eoff); fe_free(deg); fe_free(vptr); fe_free(cur);
        fe_free(inc); fe_free(cnt); fe_free(tmp); fe_free(big); fe_free(counters);
    }
};

}  // namespace

extern "C" void fe_p3_pattern_destroy(fe_p3_pattern p) {
    if (!p) return;
    FeStreamScope scope(p->last_stream);
    fe_free(p->row_ptr); fe_free(p->col_idx); fe_free(p->map); fe_free(p->edof);
    fe_free(p->vptr); fe_free(p->ikey); fe_free(p->ipos); fe_free(p->kg); fe_free(p->long_rows);
    delete p;
}

extern "C" fe_status fe_p3_pattern_build(fe_mesh m, fe_pattern p1, int flags, fe_stream stream, fe_p3_pattern* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    fe_status st;
    if ((st = fe_check_pair(m, p1, 1))) return st;
    if (p1->row1 >= 0) return fe_fail(FE_ERR_INVALID_ARG, "the P3 pattern needs a whole-mesh scalar pattern, not a row window");
    const int32_t nq = m->nq, nme = m->nme;
    if (100 * (int64_t)nme >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "100*nme must be < 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    const bool gather = (flags & FE_PATTERN_GATHER) != 0;
    fe_p3_pattern p = new fe_p3_pattern_s();
    p->flags = gather ? FE_PATTERN_GATHER : 0;
    p->nq = nq;
    p->nme = nme;
    p->topology_id = m->topology_id;
    p->last_stream = s;
    P3Temps t;
    auto fail = [&](fe_status e) {
        cudaStreamSynchronize(s);
        fe_p3_pattern_destroy(p);
        return e;
    };
    // edges: rank of each entry right of the diagonal of the scalar pattern
    if ((st = fe_alloc_n(&t.ucnt, (size_t)nq + 1, "upper counts"))) return fail(st);
    if ((st = fe_alloc_n(&t.dpos, (size_t)nq + 1, "diagonal places"))) return fail(st);
    if ((st = fe_alloc_n(&t.eoff, (size_t)nq + 1, "edge offsets"))) return fail(st);
    if (nq > 0) {
        { FE_PROF("k_edge_upper", s); k_edge_upper<<<fe_grid(nq, P3_BLOCK), P3_BLOCK, 0, s>>>(p1->row_ptr, p1->col_idx, nq, t.ucnt, t.dpos); }
        FE_LAUNCHED("k_edge_upper");
    }
    int64_t ne = 0;
    if ((st = fe_exclusive_scan(t.ucnt, t.eoff, nq, s, &ne))) return fail(st);          // synchronises
    if ((int64_t)nq + 2 * ne + nme >= INT32_MAX) return fail(fe_fail(FE_ERR_LIMIT, "too many P3 dofs"));
    const int32_t ndof = (int32_t)(nq + 2 * ne + nme);
    p->ne = ne;
    p->ndof = ndof;
    // element dofs and the dofs' element counts
    if ((st = fe_alloc_n(&p->edof, 10 * (size_t)nme, "element dofs"))) return fail(st);
    if ((st = fe_alloc_n(&t.deg, (size_t)ndof + 1, "dof valences"))) return fail(st);
    if (cudaMemsetAsync(t.deg, 0, sizeof(int32_t) * ((size_t)ndof + 1), s) != cudaSuccess) return fail(fe_fail(FE_ERR_CUDA, "memset"));
    if (nme > 0) {
        { FE_PROF("k_p3_edof", s); k_p3_edof<<<fe_grid(nme, P3_BLOCK, 8), P3_BLOCK, 0, s>>>(m->me, nme, nq, p1->row_ptr, p1->col_idx, t.eoff, t.dpos, ne, p->edof, t.deg); }
        FE_LAUNCHED("k_p3_edof");
    }
    if ((st = fe_alloc_n(&t.vptr, (size_t)ndof + 1, "dof pointers"))) return fail(st);
    if ((st = fe_alloc_n(&t.cur, (size_t)ndof + 1, "bucket cursors"))) return fail(st);
    if ((st = fe_exclusive_scan(t.deg, t.vptr, ndof, s, nullptr, 1, t.cur))) return fail(st);
    if ((st = fe_alloc_n(&t.inc, 10 * (size_t)nme, "dof incidences"))) return fail(st);
    if (nme > 0) {
        { FE_PROF("k_p3_fill", s); k_p3_fill<<<fe_grid(nme, P3_BLOCK, 8), P3_BLOCK, 0, s>>>(p->edof, nme, t.cur, t.inc); }
        FE_LAUNCHED("k_p3_fill");
    }
    // rows
    if ((st = fe_alloc_n(&t.cnt, (size_t)ndof + 1, "row counts"))) return fail(st);
    if ((st = fe_alloc_n(&t.tmp, 100 * (size_t)nme + 1, "row columns"))) return fail(st);
    if ((st = fe_alloc_n(&t.big, (size_t)ndof + 1, "long rows"))) return fail(st);
    if ((st = fe_alloc_n(&t.counters, 4, "counters"))) return fail(st);
    if ((st = fe_alloc_n(&p->map, 100 * (size_t)nme, "element-to-nnz map"))) return fail(st);
    if (cudaMemsetAsync(t.counters, 0, 4 * sizeof(int32_t), s) != cudaSuccess) return fail(fe_fail(FE_ERR_CUDA, "memset"));
    if (gather) {
        if ((st = fe_alloc_n(&p->ikey, 10 * (size_t)nme, "row incidence keys"))) return fail(st);
        if ((st = fe_alloc_n(&p->ipos, 50 * (size_t)nme, "row incidence positions"))) return fail(st);
        if ((st = fe_alloc_n(&p->long_rows, (size_t)ndof + 1, "long rows"))) return fail(st);
    }
    const P3Lists ls{p->ikey, p->ipos, p->long_rows, t.counters + 2};
    if (ndof > 0) {
        { FE_PROF("k_p3_short_rows", s); k_p3_short_rows<<<fe_grid(ndof, P3_BLOCK, 8), P3_BLOCK, 0, s>>>(
              t.vptr, t.inc, p->edof, ndof, t.tmp, t.cnt, p->map, ls); }
        FE_LAUNCHED("k_p3_short_rows");
        { FE_PROF("k_p3_rows", s); k_p3_rows<<<fe_grid(((int64_t)ndof + P3_WARPS - 1) / P3_WARPS, 1, 12), P3_WARPS * 32, 0, s>>>(
              t.vptr, t.inc, p->edof, ndof, t.tmp, t.cnt, p->map, t.big, t.counters, ls); }
        FE_LAUNCHED("k_p3_rows");
        const size_t big_smem = sizeof(P3Smem<BIG_TS, BIG_EMAX>);
        FE_CUDA(cudaFuncSetAttribute(k_p3_rows_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem));
        { FE_PROF("k_p3_rows_big", s); k_p3_rows_big<<<fe_sm_count(), 32, big_smem, s>>>(t.vptr, t.inc, p->edof, t.big, t.counters,
                                                                                          t.tmp, t.cnt, p->map, t.counters + 1, ls); }
        FE_LAUNCHED("k_p3_rows_big");
    }
    if ((st = fe_alloc_n(&p->row_ptr, (size_t)ndof + 1, "row_ptr"))) return fail(st);
    int64_t nnz = 0;
    if ((st = fe_exclusive_scan(t.cnt, p->row_ptr, ndof, s, &nnz))) return fail(st);   // synchronises
    int flags_h[2] = {0, 0};                                    // a row above the valence limit, long rows
    if (cudaMemcpyAsync(flags_h, t.counters + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(fe_fail(FE_ERR_CUDA, "flag read-back"));
    const int too_big = flags_h[0];
    p->n_long = flags_h[1];
    if (too_big)
        return fail(fe_fail(FE_ERR_LIMIT, "a vertex belongs to more than FE_P3_MAX_VALENCE=" +
                                              std::to_string(FE_P3_MAX_VALENCE) + " triangles"));
    p->nnz = nnz;
    if ((st = fe_alloc_n(&p->col_idx, (size_t)nnz, "col_idx"))) return fail(st);
    if (ndof > 0) {
        { FE_PROF("k_p3_cols", s); k_p3_cols<<<fe_grid(ndof, P3_BLOCK, 8), P3_BLOCK, 0, s>>>(t.vptr, p->row_ptr, ndof, t.tmp, p->col_idx); }
        FE_LAUNCHED("k_p3_cols");
    }
    if (nme > 0) {
        { FE_PROF("k_p3_map_base", s); k_p3_map_base<<<fe_grid(100 * (int64_t)nme, P3_BLOCK), P3_BLOCK, 0, s>>>(p->edof, nme, p->row_ptr, p->map); }
        FE_LAUNCHED("k_p3_map_base");
    }
    if (gather) {
        if ((st = fe_alloc_n(&p->kg, 100 * (size_t)nme, "element value staging"))) return fail(st);
        p->vptr = t.vptr;                            // the row sums need the incidence offsets
        t.vptr = nullptr;
    }
    *out = p;
    return FE_OK;
}

extern "C" fe_status fe_p3_pattern_info(fe_p3_pattern p, int64_t* n_dofs, int64_t* nnz, const int32_t** row_ptr,
                                        const int32_t** col_idx) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (n_dofs) *n_dofs = p->ndof;
    if (nnz) *nnz = p->nnz;
    if (row_ptr) *row_ptr = p->row_ptr;
    if (col_idx) *col_idx = p->col_idx;
    return FE_OK;
}

extern "C" fe_status fe_p3_pattern_dofs(fe_p3_pattern p, const int32_t** edof, const int32_t** map, int64_t* n_edges) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (edof) *edof = p->edof;
    if (map) *map = p->map;
    if (n_edges) *n_edges = p->ne;
    return FE_OK;
}

extern "C" fe_status fe_p3_assemble(fe_mesh m, fe_p3_pattern p, int kind, int variant, double* values, int64_t cap,
                                    fe_stream stream) {
    FE_RANGE(__func__);
    if (!m || !p) return fe_fail(FE_ERR_INVALID_ARG, "null mesh or pattern");
    if (m->topology_id != p->topology_id) return fe_fail(FE_ERR_INVALID_ARG, "the pattern was built for another mesh");
    if (kind != FE_P3_MASS && kind != FE_P3_STIFF) return fe_fail(FE_ERR_INVALID_ARG, "unknown kind");
    if (variant != FE_VARIANT_ATOMIC && variant != FE_VARIANT_GATHER)
        return fe_fail(FE_ERR_INVALID_ARG, "P3 takes FE_VARIANT_ATOMIC or FE_VARIANT_GATHER");
    if (variant == FE_VARIANT_GATHER && !(p->flags & FE_PATTERN_GATHER))
        return fe_fail(FE_ERR_INVALID_ARG, "FE_VARIANT_GATHER needs a P3 pattern built with FE_PATTERN_GATHER");
    if (cap < p->nnz) return fe_fail(FE_ERR_BUFFER_TOO_SMALL, "cap is below nnz");
    if (!values && p->nnz > 0) return fe_fail(FE_ERR_INVALID_ARG, "values is null");
    fe_status st;
    if ((st = p3_tables_ready())) return st;
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    m->last_stream = s;
    p->last_stream = s;
    const int32_t nme = m->nme;
    if (variant == FE_VARIANT_ATOMIC) {
        if (p->nnz > 0) FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * p->nnz, s));
        if (nme == 0) return FE_OK;
        const unsigned g = fe_grid(nme, P3_BLOCK, 8);
        {
            FE_PROF("k_p3_atomic", s);
            if (kind == FE_P3_MASS) k_p3_atomic<FE_P3_MASS><<<g, P3_BLOCK, 0, s>>>(m->me, nme, m->q, p->map, values, p->nnz);
            else k_p3_atomic<FE_P3_STIFF><<<g, P3_BLOCK, 0, s>>>(m->me, nme, m->q, p->map, values, p->nnz);
        }
        FE_LAUNCHED("k_p3_atomic");
        return FE_OK;
    }
    if (nme == 0) return FE_OK;
    {
        const unsigned g = fe_grid(nme, STAGE_BLOCK, 16);
        FE_PROF("k_p3_stage", s);
        if (kind == FE_P3_MASS) k_p3_stage<FE_P3_MASS><<<g, STAGE_BLOCK, 0, s>>>(m->me, nme, m->q, p->kg);
        else k_p3_stage<FE_P3_STIFF><<<g, STAGE_BLOCK, 0, s>>>(m->me, nme, m->q, p->kg);
    }
    FE_LAUNCHED("k_p3_stage");
    const int32_t ndof = p->ndof;
    { FE_PROF("k_p3_rowsum_short", s); k_p3_rowsum_short<<<fe_grid(ndof, RS_BLOCK, 8), RS_BLOCK, 0, s>>>(
          p->vptr, p->row_ptr, ndof, p->ikey, p->ipos, p->kg, values, 10 * (int64_t)nme); }
    FE_LAUNCHED("k_p3_rowsum_short");
    { FE_PROF("k_p3_rowsum", s); k_p3_rowsum<<<fe_grid(((int64_t)ndof + P3_WARPS - 1) / P3_WARPS, 1, 12), P3_WARPS * 32, 0, s>>>(
          p->vptr, p->row_ptr, ndof, p->ikey, p->ipos, p->kg, values, 10 * (int64_t)nme); }
    FE_LAUNCHED("k_p3_rowsum");
    // rows of more than RS_FAST columns (vertices of more than 12 triangles): their accumulators in
    // dynamic shared memory, sized for the longest row any P3 pattern can have
    if (p->n_long > 0) {
        const size_t long_smem = sizeof(double) * 10 * (size_t)BIG_EMAX;
        FE_CUDA(cudaFuncSetAttribute(k_p3_rowsum_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)long_smem));
        { FE_PROF("k_p3_rowsum_long", s); k_p3_rowsum_long<<<(unsigned)min((int64_t)p->n_long, (int64_t)fe_sm_count() * 8), 32, long_smem, s>>>(
              p->long_rows, p->n_long, p->vptr, p->row_ptr, p->ikey, p->ipos, p->kg, values, 10 * (int64_t)nme); }
        FE_LAUNCHED("k_p3_rowsum_long");
    }
    return FE_OK;
}
