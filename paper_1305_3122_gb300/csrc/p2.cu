// p2.cu -- P2 (quadratic) triangles: dof numbering, CSR structure and the mass and stiffness.
//
// The paper states that its method extends to P_k elements and gives no formulas. The P2 element
// has the three vertex functions phi_a = l_a (2 l_a - 1) (local dofs 0, 1, 2) and the three edge
// functions 4 l0 l1, 4 l1 l2, 4 l2 l0 (local dofs 3, 4, 5: the midpoints of the edges (0,1), (1,2),
// (2,0)), with l_a the barycentric coordinates (the P1 functions) and G_kl = grad l_k . grad l_l
// (grad l_a as in Eq. (4)). Integrating the products with int_T l_i l_j = |T| (1 + delta_ij) / 12
// and friends gives, for vertices a != b, c the third vertex, and edges (a,b), (c,d):
//   M^e = |T|/180 [[6 -1 -1 0 -4 0] [-1 6 -1 0 0 -4] [-1 -1 6 -4 0 0]
//                  [0 0 -4 32 16 16] [-4 0 0 16 32 16] [0 -4 0 16 16 32]]
//   S_aa = |T| G_aa,  S_ab = -|T| G_ab / 3,
//   S(vertex a, edge (a,c)) = 4/3 |T| G_ac,  S(vertex a, the opposite edge) = 0,
//   S(edge (a,b), edge (c,d)) = 16 (G_ac I_bd + G_ad I_bc + G_bc I_ad + G_bd I_ac),  I_ij = |T| (1 + delta_ij) / 12.
//
// Dofs: vertex i is dof i; the edges follow, numbered in ascending order of (smaller vertex id,
// larger vertex id). Those are the entries above the diagonal of the scalar (P1) pattern in CSR
// order, so an edge's id is its rank among them: per row the number of entries right of the
// diagonal, a scan, and a binary search of the other vertex in the smaller vertex's row.
//
// Pattern: every element couples its six dofs. The incidences (element k, local dof a) are bucketed
// by dof with a counting sort; one warp per vertex row merges the dofs of the row's elements in a
// shared-memory hash table (rowhash.cuh), and one thread per edge row (at most two elements) sorts
// its at most 12 ids in registers; either ranks the distinct ids (the sorted columns) and writes
// each incidence's six in-row positions: the element-to-nnz map, row-major per element
// (map[36k + 6 il + jl]), made absolute once the offsets are known. Assembly: one thread per
// element, FP64, 36 FP64 atomics; or (the deterministic variant) the element matrices staged and
// one thread per row adding the row's incidences in ascending element order (the row passes also
// list each row's incidences in ascending element order with their column positions), so that every non-zero sums its
// contributions in ascending element order, bit-identical from run to run.
#include "internal.cuh"
#include "edges.cuh"
#include "rowhash.cuh"

namespace {

constexpr int P2_BLOCK = 256;
constexpr int P2_WARPS = 4;
constexpr int FAST_TS = 128, FAST_EMAX = 21;             // 6 * 21 ids < 128
constexpr int BIG_TS = 4096, BIG_EMAX = FE_P2_MAX_VALENCE;
static_assert(6 * FAST_EMAX < FAST_TS && 6 * BIG_EMAX < BIG_TS, "tables hold every id");
constexpr int RS_BLOCK = 128;                // row sums: one row per thread
constexpr int RS_VERTEX = 32;                // row sums: accumulators of a vertex row (1 + 3 d columns at valence d)
constexpr int RS_VERTEX_SHORT = 24;          // row sums: fewer accumulators when no vertex row is longer (8
                                             // resident blocks per SM instead of 6)
constexpr int RS_EDGE_MAX = 12;              // row sums: columns of an edge row in at most two triangles
constexpr int RS_LONG_MAX = 6 * BIG_EMAX;    // columns of the longest row

// Where the row passes put the deterministic variant's lists (rrec null: no lists).
struct P2Lists {
    int4* rrec;          // [6 nme]: each row's incidences in ascending element order, row r from vptr[r]:
                         // {key 6k + a, then the in-row positions of columns jl = 0..5, 16 bits each}
    int32_t* long_rows;  // rows with more columns than their thread's accumulators
    int32_t* n_long;     // their number, then 1 if a vertex row has more than RS_VERTEX_SHORT columns
    int32_t nq;
};

// edof[6k .. 6k+5]: the element's dofs; also counts each dof's elements.
__global__ void k_p2_edof(const int32_t* __restrict__ me, int32_t nme, int32_t nq, const int32_t* __restrict__ row_ptr,
                          const int32_t* __restrict__ col_idx, const int32_t* __restrict__ eoff,
                          const int32_t* __restrict__ dpos, int32_t* __restrict__ edof, int32_t* __restrict__ deg) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v0 = me[k], v1 = me[nme + k], v2 = me[2 * (int64_t)nme + k];
        int32_t d[6] = {v0, v1, v2, nq + edge_rank(row_ptr, col_idx, eoff, dpos, v0, v1),
                        nq + edge_rank(row_ptr, col_idx, eoff, dpos, v1, v2), nq + edge_rank(row_ptr, col_idx, eoff, dpos, v2, v0)};
        int2* o = reinterpret_cast<int2*>(edof + 6 * k);
        o[0] = make_int2(d[0], d[1]);
        o[1] = make_int2(d[2], d[3]);
        o[2] = make_int2(d[4], d[5]);
#pragma unroll
        for (int a = 0; a < 6; a++) atomicAdd(&deg[d[a]], 1);
    }
}

__global__ void k_p2_fill(const int32_t* __restrict__ edof, int32_t nme, int32_t* __restrict__ cur,
                          int32_t* __restrict__ inc) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 6; a++) inc[FE_IDX(atomicAdd(&cur[edof[6 * k + a]], 1), 6 * (int64_t)nme)] = 6 * (int32_t)k + a;
    }
}

template <int TS, int EMAX>
struct P2Smem {
    int32_t tab[TS];
    int32_t rnk[TS];
    int32_t uid[TS];
    int32_t uslot[TS];
    int32_t key[EMAX];
    int16_t xs[6 * EMAX];   // the slot of each incidence's six ids
    int32_t ucount;
};

// One row by one warp: sorted distinct columns into tmp at 6 vptr[r] (each incidence brings at
// most six), their count, and the six relative positions of every incidence in map.
template <int TS, int EMAX>
__device__ void p2_row(int32_t r, int32_t beg, int32_t d, const int32_t* __restrict__ inc, const int32_t* __restrict__ edof,
                       P2Smem<TS, EMAX>& sm, int32_t* __restrict__ tmp, int32_t* __restrict__ cnt,
                       int32_t* __restrict__ map, const P2Lists& ls) {
    const int lane = threadIdx.x & 31;
    for (int s = lane; s < TS; s += 32) sm.tab[s] = -1;
    if (lane == 0) sm.ucount = 0;
    for (int t = lane; t < d; t += 32) sm.key[t] = inc[beg + t];
    __syncwarp();
    for (int x = lane; x < 6 * d; x += 32) {
        const int32_t id = edof[6 * (int64_t)(sm.key[x / 6] / 6) + x % 6];
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
    const int64_t tb = 6 * (int64_t)beg;
    for (int p = lane; p < u; p += 32) {
        const int32_t id = sm.uid[p];
        int rk = 0;
        for (int qq = 0; qq < u; qq++) rk += sm.uid[qq] < id;
        sm.rnk[sm.uslot[p]] = rk;
        tmp[tb + rk] = id;
    }
    __syncwarp();
    for (int t = lane; t < d; t += 32) {
        const int32_t kk = sm.key[t] / 6, a = sm.key[t] - 6 * (sm.key[t] / 6);
        int32_t* mo = map + 36 * (int64_t)kk + 6 * a;
        int32_t o[6];
#pragma unroll
        for (int jl = 0; jl < 6; jl++) {
            o[jl] = sm.rnk[sm.xs[6 * t + jl]];          // the slot its insertion got
            mo[jl] = o[jl];
        }
        if (ls.rrec) {                                       // the incidence's place in element order
            int c0 = 0;
            for (int tt = 0; tt < d; tt++) c0 += sm.key[tt] < sm.key[t];
            ls.rrec[beg + c0] = make_int4(sm.key[t], (int)((unsigned)o[0] | ((unsigned)o[1] << 16)),
                                          (int)((unsigned)o[2] | ((unsigned)o[3] << 16)), (int)((unsigned)o[4] | ((unsigned)o[5] << 16)));
        }
    }
    if (lane == 0) {
        cnt[r] = u;
        // long: a vertex row longer than its thread's accumulators, or an edge row here (an edge in more
        // than two triangles: the edge-row sums handle at most two)
        if (ls.rrec && (r >= ls.nq || u > RS_VERTEX)) ls.long_rows[atomicAdd(ls.n_long, 1)] = r;
        if (ls.rrec && r < ls.nq && u > RS_VERTEX_SHORT) ls.n_long[1] = 1;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(P2_WARPS * 32) k_p2_rows(const int32_t* __restrict__ vptr, const int32_t* __restrict__ inc,
                                                           const int32_t* __restrict__ edof, int32_t nrows,
                                                           int32_t* __restrict__ tmp, int32_t* __restrict__ cnt,
                                                           int32_t* __restrict__ map, int32_t* __restrict__ big_list,
                                                           int32_t* __restrict__ big_count, P2Lists ls) {
    __shared__ P2Smem<FAST_TS, FAST_EMAX> sm_all[P2_WARPS];
    P2Smem<FAST_TS, FAST_EMAX>& sm = sm_all[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    for (int64_t rr = (int64_t)blockIdx.x * P2_WARPS + (threadIdx.x >> 5); rr < nrows; rr += (int64_t)gridDim.x * P2_WARPS) {
        const int32_t r = (int32_t)rr, beg = vptr[r], d = vptr[r + 1] - beg;
        if (d == 0) {
            if (lane == 0) cnt[r] = 0;
            continue;
        }
        if (d > FAST_EMAX) {
            if (lane == 0) big_list[atomicAdd(big_count, 1)] = r;
            continue;
        }
        p2_row<FAST_TS, FAST_EMAX>(r, beg, d, inc, edof, sm, tmp, cnt, map, ls);
    }
}

// Edge rows (dofs nq .. ndof - 1), one thread each: an edge lies in at most two triangles of a
// manifold mesh, so its row merges at most 12 ids, sorted in registers (a fixed compare-exchange
// sequence: static indices only); the rank of a value is the number of distinct smaller ones.
// Rows with more elements go to the long-row list.
__global__ void __launch_bounds__(P2_BLOCK) k_p2_edge_rows(const int32_t* __restrict__ vptr, const int32_t* __restrict__ inc,
                                                           const int32_t* __restrict__ edof, int32_t nq, int32_t ndof,
                                                           int32_t* __restrict__ tmp, int32_t* __restrict__ cnt,
                                                           int32_t* __restrict__ map, int32_t* __restrict__ big_list,
                                                           int32_t* __restrict__ big_count, P2Lists ls) {
    for (int64_t rr = nq + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < ndof; rr += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)rr, beg = vptr[r], d = vptr[r + 1] - beg;
        if (d > 2) {
            big_list[atomicAdd(big_count, 1)] = r;
            continue;
        }
        int32_t key[2] = {d > 0 ? inc[beg] : -1, d > 1 ? inc[beg + 1] : -1};
        int32_t x[12];
#pragma unroll
        for (int t = 0; t < 2; t++)
#pragma unroll
            for (int j = 0; j < 6; j++) x[6 * t + j] = key[t] >= 0 ? edof[6 * (int64_t)(key[t] / 6) + j] : INT32_MAX;
#pragma unroll
        for (int i = 1; i < 12; i++)
#pragma unroll
            for (int j = i; j > 0; j--) {
                const int32_t lo = min(x[j - 1], x[j]), hi = max(x[j - 1], x[j]);
                x[j - 1] = lo;
                x[j] = hi;
            }
        const int64_t tb = 6 * (int64_t)beg;
        int u = 0;
#pragma unroll
        for (int i = 0; i < 12; i++) {
            const bool first = x[i] != INT32_MAX && (i == 0 || x[i] != x[i - 1]);
            if (first) tmp[tb + u] = x[i];
            u += first;
        }
        cnt[r] = u;
#pragma unroll
        for (int t = 0; t < 2; t++) {
            if (key[t] < 0) continue;
            const int32_t kk = key[t] / 6, a = key[t] - 6 * kk;
            const int32_t* e = edof + 6 * (int64_t)kk;
            int32_t* o = map + 36 * (int64_t)kk + 6 * a;
            unsigned sl[6];
#pragma unroll
            for (int jl = 0; jl < 6; jl++) {
                const int32_t v = e[jl];
                int rank = 0;
#pragma unroll
                for (int i = 0; i < 12; i++) rank += x[i] < v && (i == 0 || x[i] != x[i - 1]);
                o[jl] = rank;
                sl[jl] = (unsigned)rank;
            }
            if (ls.rrec) {                                   // ascending element order (at most 12 columns: no long row)
                const int c0 = d > 1 && key[1 - t] < key[t];
                ls.rrec[beg + c0] = make_int4(key[t], (int)(sl[0] | (sl[1] << 16)), (int)(sl[2] | (sl[3] << 16)),
                                              (int)(sl[4] | (sl[5] << 16)));
            }
        }
    }
}

__global__ void __launch_bounds__(32) k_p2_rows_big(const int32_t* __restrict__ vptr, const int32_t* __restrict__ inc,
                                                    const int32_t* __restrict__ edof, const int32_t* __restrict__ big_list,
                                                    const int32_t* __restrict__ big_count, int32_t* __restrict__ tmp,
                                                    int32_t* __restrict__ cnt, int32_t* __restrict__ map,
                                                    int* __restrict__ too_big, P2Lists ls) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    P2Smem<BIG_TS, BIG_EMAX>& sm = *reinterpret_cast<P2Smem<BIG_TS, BIG_EMAX>*>(smem_raw);
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
        p2_row<BIG_TS, BIG_EMAX>(r, beg, d, inc, edof, sm, tmp, cnt, map, ls);
    }
}

// One thread per row (rows are short: many rows in flight hide the latency of each).
__global__ void __launch_bounds__(P2_BLOCK) k_p2_cols(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                      int32_t ndof, const int32_t* __restrict__ tmp, int32_t* __restrict__ col_idx) {
    for (int64_t rr = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; rr < ndof; rr += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)rr, rb = row_ptr[r], u = row_ptr[r + 1] - rb;
        const int64_t tb = 6 * (int64_t)vptr[r];
        for (int c = 0; c < u; c++) col_idx[rb + c] = tmp[tb + c];
    }
}

__global__ void k_p2_map_base(const int32_t* __restrict__ edof, int32_t nme, const int32_t* __restrict__ row_ptr,
                              int32_t* __restrict__ map) {
    const int64_t n = 36 * (int64_t)nme;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = c / 36;
        const int il = (int)((c - 36 * k) / 6);
        map[c] += row_ptr[edof[6 * k + il]];
    }
}

// ------------------------------------------------------------------ element matrices

template <int KIND>
__device__ __forceinline__ void p2_elem(double2 p0, double2 p1, double2 p2, double E[6][6]) {
    // e_a = the edge opposite vertex a (Eq. 3's u, v, w); D = 2|T|; grad l_a = (e_a,y, -e_a,x) / D
    const double ex[3] = {p1.x - p2.x, p2.x - p0.x, p0.x - p1.x};
    const double ey[3] = {p1.y - p2.y, p2.y - p0.y, p0.y - p1.y};
    const double D = ex[1] * ey[2] - ex[2] * ey[1];
    const double T = 0.5 * D;
    if (KIND == FE_P2_MASS) {
        const double m = T * (1.0 / 180.0);                  // constant reciprocals: no run-time division
        const double a = 6.0 * m, b = -m, c = -4.0 * m, d = 32.0 * m, e = 16.0 * m;
        const double tbl[6][6] = {{a, b, b, 0.0, c, 0.0}, {b, a, b, 0.0, 0.0, c}, {b, b, a, c, 0.0, 0.0},
                                  {0.0, 0.0, c, d, e, e}, {c, 0.0, 0.0, e, d, e}, {0.0, c, 0.0, e, e, d}};
#pragma unroll
        for (int i = 0; i < 6; i++)
#pragma unroll
            for (int j = 0; j < 6; j++) E[i][j] = tbl[i][j];
        return;
    }
    // T G_kl = T (e_k . e_l) / D^2 = (e_k . e_l) / (2 D)
    const double s = 0.5 / D;
    double G[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
        for (int l = k; l < 3; l++) {
            G[k][l] = (ex[k] * ex[l] + ey[k] * ey[l]) * s;
            G[l][k] = G[k][l];
        }
    const int ea[3] = {0, 1, 2}, eb[3] = {1, 2, 0};            // edge dof 3 + t joins vertices ea[t], eb[t]
    // vertices
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) E[a][b] = a == b ? G[a][a] : -G[a][b] * (1.0 / 3.0);
    // vertex - edge: 4/3 T G_ac for the edge (a, c), 0 for the opposite edge
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int t = 0; t < 3; t++) {
            double v = 0.0;
            if (ea[t] == a) v = 4.0 / 3.0 * G[a][eb[t]];
            else if (eb[t] == a) v = 4.0 / 3.0 * G[a][ea[t]];
            E[a][3 + t] = v;
            E[3 + t][a] = v;
        }
    // edge - edge: 16 (G_ac I_bd + G_ad I_bc + G_bc I_ad + G_bd I_ac), T I_ij = T (1 + delta_ij) / 12
#pragma unroll
    for (int t = 0; t < 3; t++)
#pragma unroll
        for (int u = t; u < 3; u++) {
            const int a = ea[t], b = eb[t], c = ea[u], d = eb[u];
            const double Ibd = (b == d ? 2.0 : 1.0) / 12.0, Ibc = (b == c ? 2.0 : 1.0) / 12.0;
            const double Iad = (a == d ? 2.0 : 1.0) / 12.0, Iac = (a == c ? 2.0 : 1.0) / 12.0;
            const double v = 16.0 * (G[a][c] * Ibd + G[a][d] * Ibc + G[b][c] * Iad + G[b][d] * Iac);
            E[3 + t][3 + u] = v;
            E[3 + u][3 + t] = v;
        }
}

template <int KIND>
__global__ void __launch_bounds__(P2_BLOCK) k_p2_atomic(const int32_t* __restrict__ me, int32_t nme, const double2* __restrict__ q,
                                                        const int32_t* __restrict__ map, double* __restrict__ val, int64_t nnz) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        double E[6][6];
        p2_elem<KIND>(q[me[k]], q[me[nme + k]], q[me[2 * (int64_t)nme + k]], E);
        const int32_t* mk = map + 36 * k;
#pragma unroll
        for (int il = 0; il < 6; il++)
#pragma unroll
            for (int jl = 0; jl < 6; jl++) atomicAdd(&val[FE_IDX(mk[6 * il + jl], nnz)], E[il][jl]);
    }
}

// The element matrices into the staging buffer, row-major per element (kg[36k + 6 il + jl]). The
// block's STAGE_BLOCK matrices go through shared memory (rows padded to 37 doubles, so the
// threads' writes fall in different banks) and leave as one contiguous range written with
// coalesced 16-byte stores; each thread writing its own 288 bytes directly would make every
// store instruction touch 32 different lines.
constexpr int STAGE_BLOCK = 128, STAGE_PAD = 37;

template <int KIND>
__global__ void __launch_bounds__(STAGE_BLOCK) k_p2_stage(const int32_t* __restrict__ me, int32_t nme, const double2* __restrict__ q,
                                                          double* __restrict__ kg) {
    __shared__ double tile[STAGE_BLOCK * STAGE_PAD];
    for (int64_t k0 = (int64_t)blockIdx.x * STAGE_BLOCK; k0 < nme; k0 += (int64_t)gridDim.x * STAGE_BLOCK) {
        const int64_t k = k0 + threadIdx.x;
        if (k < nme) {
            double E[6][6];
            p2_elem<KIND>(q[me[k]], q[me[nme + k]], q[me[2 * (int64_t)nme + k]], E);
#pragma unroll
            for (int il = 0; il < 6; il++)
#pragma unroll
                for (int jl = 0; jl < 6; jl++) tile[threadIdx.x * STAGE_PAD + 6 * il + jl] = E[il][jl];
        }
        __syncthreads();
        const int n = (int)min((int64_t)STAGE_BLOCK, (int64_t)nme - k0);
        double2* o = reinterpret_cast<double2*>(kg + 36 * k0);
        for (int c = threadIdx.x; c < 18 * n; c += STAGE_BLOCK) {       // 18 pairs per element
            const int e = c / 18, j = 2 * (c - 18 * e);
            o[c] = make_double2(tile[e * STAGE_PAD + j], tile[e * STAGE_PAD + j + 1]);
        }
        __syncthreads();
    }
}

// Row sums of the staged matrices for the rows [r0, r1), one row per thread: the row's incidences
// in ascending element order (records streamed from the row's list) each add row a of element k
// (kg[36k + 6a ..], 48 bytes) into the row's accumulators in shared memory at the record's six
// column positions. Accumulators start at -0.0, so every sum equals its first contribution
// followed by the others in ascending element order, bit for bit. Rows with more than RMAX
// columns are left to k_p2_rowsum_long.
template <int RMAX>
__global__ void __launch_bounds__(RS_BLOCK) k_p2_rowsum(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                        int32_t r0, int32_t r1, const int4* __restrict__ rrec,
                                                        const double* __restrict__ kg, double* __restrict__ val, int64_t n6) {
    __shared__ double acc[RMAX * RS_BLOCK];
    double* a = acc + threadIdx.x;                       // column c of this thread's row at a[c * RS_BLOCK]
    for (int64_t rr = r0 + blockIdx.x * (int64_t)RS_BLOCK + threadIdx.x; rr < r1; rr += (int64_t)gridDim.x * RS_BLOCK) {
        const int32_t rb = row_ptr[rr], u = row_ptr[rr + 1] - rb;
        if (u > RMAX) continue;
        const int32_t b0 = vptr[rr], d = vptr[rr + 1] - b0;
        for (int c = 0; c < u; c++) a[c * RS_BLOCK] = -0.0;
        int4 rec = d > 0 ? rrec[b0] : make_int4(0, 0, 0, 0);
        for (int32_t t = 0; t < d; t++) {
            const double2* e = reinterpret_cast<const double2*>(kg + 6 * (int64_t)FE_IDX(rec.x, n6));   // 36k + 6a
            double2 v[3];
#pragma unroll
            for (int j = 0; j < 3; j++) v[j] = e[j];
            const unsigned sl[3] = {(unsigned)rec.y, (unsigned)rec.z, (unsigned)rec.w};
            if (t + 1 < d) rec = rrec[b0 + t + 1];
            // an incidence's six columns are distinct: all six accumulators are read before any is
            // written back, so the six updates overlap instead of waiting on one another
            double* pc[6];
            double y[6];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                pc[2 * j] = a + FE_IDX(sl[j] & 0xFFFFu, u) * RS_BLOCK;
                pc[2 * j + 1] = a + FE_IDX(sl[j] >> 16, u) * RS_BLOCK;
            }
#pragma unroll
            for (int j = 0; j < 6; j++) y[j] = *pc[j];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                *pc[2 * j] = y[2 * j] + v[j].x;
                *pc[2 * j + 1] = y[2 * j + 1] + v[j].y;
            }
        }
        for (int c = 0; c < u; c++) val[rb + c] = a[c * RS_BLOCK];
    }
}

// Row sums of the edge rows in at most two triangles, one row per thread, in registers: column c
// takes the first incidence's entry at c, then adds the second's (ascending element order). The
// first value is taken as it is, which is bit for bit what adding it to -0.0 gives, so the sums
// equal those of k_p2_rowsum. Edge rows in more triangles are listed for k_p2_rowsum_long.
__global__ void __launch_bounds__(RS_BLOCK) k_p2_rowsum_edge(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                             int32_t r0, int32_t r1, const int4* __restrict__ rrec,
                                                             const double* __restrict__ kg, double* __restrict__ val) {
    for (int64_t rr = r0 + blockIdx.x * (int64_t)RS_BLOCK + threadIdx.x; rr < r1; rr += (int64_t)gridDim.x * RS_BLOCK) {
        const int32_t b0 = vptr[rr], d = vptr[rr + 1] - b0;
        if (d > 2) continue;
        const int32_t rb = row_ptr[rr], u = row_ptr[rr + 1] - rb;
        double v[2][6];
        unsigned sl[2][6];
#pragma unroll
        for (int t = 0; t < 2; t++) {
            const int4 rec = t < d ? rrec[b0 + t] : make_int4(0, -1, -1, -1);   // -1: no column
            if (t < d) {
                const double2* e = reinterpret_cast<const double2*>(kg + 6 * (int64_t)rec.x);
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const double2 x = e[j];
                    v[t][2 * j] = x.x;
                    v[t][2 * j + 1] = x.y;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 6; j++) v[t][j] = 0.0;
            }
            const unsigned w3[3] = {(unsigned)rec.y, (unsigned)rec.z, (unsigned)rec.w};
#pragma unroll
            for (int j = 0; j < 3; j++) {
                sl[t][2 * j] = w3[j] & 0xFFFFu;
                sl[t][2 * j + 1] = w3[j] >> 16;
            }
        }
#pragma unroll
        for (int c = 0; c < RS_EDGE_MAX; c++) {
            if (c >= u) break;
            double x0 = 0.0, x1 = 0.0;
            bool f0 = false, f1 = false;
#pragma unroll
            for (int j = 0; j < 6; j++) {
                if (sl[0][j] == (unsigned)c) { x0 = v[0][j]; f0 = true; }
                if (sl[1][j] == (unsigned)c) { x1 = v[1][j]; f1 = true; }
            }
            double a = f0 ? x0 : -0.0;
            if (f1) a = a + x1;
            val[rb + c] = a;
        }
    }
}

// The long rows, one warp each: lane l owns the columns c = l (mod 32) and adds their
// contributions in ascending element order (accumulators in dynamic shared memory, RS_LONG_MAX
// doubles at most).
__global__ void __launch_bounds__(32) k_p2_rowsum_long(const int32_t* __restrict__ long_rows, const int32_t* __restrict__ n_long,
                                                       const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                       const int4* __restrict__ rrec, const double* __restrict__ kg,
                                                       double* __restrict__ val) {
    extern __shared__ double accl[];
    const int lane = threadIdx.x;
    const int32_t n = *n_long;
    for (int32_t b = blockIdx.x; b < n; b += gridDim.x) {
        const int32_t r = long_rows[b];
        const int32_t rb = row_ptr[r], u = row_ptr[r + 1] - rb;
        const int32_t b0 = vptr[r], d = vptr[r + 1] - b0;
        for (int c = lane; c < u; c += 32) accl[c] = -0.0;
        __syncwarp();
        for (int32_t t = 0; t < d; t++) {
            const int4 rec = rrec[b0 + t];
            const int64_t base = 6 * (int64_t)rec.x;
            const unsigned c6[6] = {(unsigned)rec.y & 0xFFFFu, (unsigned)rec.y >> 16, (unsigned)rec.z & 0xFFFFu,
                                    (unsigned)rec.z >> 16, (unsigned)rec.w & 0xFFFFu, (unsigned)rec.w >> 16};
#pragma unroll
            for (int jl = 0; jl < 6; jl++)
                if ((int)(c6[jl] & 31u) == lane) accl[c6[jl]] += kg[base + jl];
        }
        __syncwarp();
        for (int c = lane; c < u; c += 32) val[rb + c] = accl[c];
        __syncwarp();
    }
}

}  // namespace

extern "C" void fe_p2_pattern_destroy(fe_p2_pattern p) {
    if (!p) return;
    FeStreamScope scope(p->last_stream);
    fe_free(p->row_ptr); fe_free(p->col_idx); fe_free(p->map); fe_free(p->edof);
    fe_free(p->vptr); fe_free(p->rrec); fe_free(p->long_rows); fe_free(p->n_long); fe_free(p->kg);
    delete p;
}

namespace {
struct P2Temps {
    int32_t *ucnt = nullptr, *dpos = nullptr, *eoff = nullptr, *deg = nullptr, *vptr = nullptr, *cur = nullptr;
    int32_t *inc = nullptr, *cnt = nullptr, *tmp = nullptr, *big = nullptr, *counters = nullptr;
    ~P2Temps() {
        fe_free(ucnt); fe_free(dpos); fe_free(eoff); fe_free(deg); fe_free(vptr); fe_free(cur);
        fe_free(inc); fe_free(cnt); fe_free(tmp); fe_free(big); fe_free(counters);
    }
};
}  // namespace

extern "C" fe_status fe_p2_pattern_build(fe_mesh m, fe_pattern p1, int flags, fe_stream stream, fe_p2_pattern* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    fe_status st;
    if ((st = fe_check_pair(m, p1, 1))) return st;
    if (p1->row1 >= 0) return fe_fail(FE_ERR_INVALID_ARG, "the P2 pattern needs a whole-mesh scalar pattern, not a row window");
    const int32_t nq = m->nq, nme = m->nme;
    if (36 * (int64_t)nme >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "36*nme must be < 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    const bool gather = (flags & FE_PATTERN_GATHER) != 0;
    fe_p2_pattern p = new fe_p2_pattern_s();
    p->flags = gather ? FE_PATTERN_GATHER : 0;
    p->nq = nq;
    p->nme = nme;
    p->topology_id = m->topology_id;
    p->last_stream = s;
    P2Temps t;
    auto fail = [&](fe_status e) {
        cudaStreamSynchronize(s);
        fe_p2_pattern_destroy(p);
        return e;
    };
    // edges: rank of each entry right of the diagonal of the scalar pattern
    if ((st = fe_alloc_n(&t.ucnt, (size_t)nq + 1, "upper counts"))) return fail(st);
    if ((st = fe_alloc_n(&t.dpos, (size_t)nq + 1, "diagonal places"))) return fail(st);
    if ((st = fe_alloc_n(&t.eoff, (size_t)nq + 1, "edge offsets"))) return fail(st);
    if (nq > 0) {
        { FE_PROF("k_edge_upper", s); k_edge_upper<<<fe_grid(nq, P2_BLOCK), P2_BLOCK, 0, s>>>(p1->row_ptr, p1->col_idx, nq, t.ucnt, t.dpos); }
        FE_LAUNCHED("k_edge_upper");
    }
    int64_t ne = 0;
    if ((st = fe_exclusive_scan(t.ucnt, t.eoff, nq, s, &ne))) return fail(st);          // synchronises
    if ((int64_t)nq + ne >= INT32_MAX) return fail(fe_fail(FE_ERR_LIMIT, "too many P2 dofs"));
    const int32_t ndof = (int32_t)(nq + ne);
    p->ne = ne;
    p->ndof = ndof;
    // element dofs and the dofs' element counts
    if ((st = fe_alloc_n(&p->edof, 6 * (size_t)nme, "element dofs"))) return fail(st);
    if ((st = fe_alloc_n(&t.deg, (size_t)ndof + 1, "dof valences"))) return fail(st);
    if (cudaMemsetAsync(t.deg, 0, sizeof(int32_t) * ((size_t)ndof + 1), s) != cudaSuccess) return fail(fe_fail(FE_ERR_CUDA, "memset"));
    if (nme > 0) {
        { FE_PROF("k_p2_edof", s); k_p2_edof<<<fe_grid(nme, P2_BLOCK, 16), P2_BLOCK, 0, s>>>(m->me, nme, nq, p1->row_ptr, p1->col_idx, t.eoff, t.dpos, p->edof, t.deg); }
        FE_LAUNCHED("k_p2_edof");
    }
    if ((st = fe_alloc_n(&t.vptr, (size_t)ndof + 1, "dof pointers"))) return fail(st);
    if ((st = fe_alloc_n(&t.cur, (size_t)ndof + 1, "bucket cursors"))) return fail(st);
    if ((st = fe_exclusive_scan(t.deg, t.vptr, ndof, s, nullptr, 1, t.cur))) return fail(st);
    if ((st = fe_alloc_n(&t.inc, 6 * (size_t)nme, "dof incidences"))) return fail(st);
    if (nme > 0) {
        { FE_PROF("k_p2_fill", s); k_p2_fill<<<fe_grid(nme, P2_BLOCK, 16), P2_BLOCK, 0, s>>>(p->edof, nme, t.cur, t.inc); }
        FE_LAUNCHED("k_p2_fill");
    }
    // rows
    if ((st = fe_alloc_n(&t.cnt, (size_t)ndof + 1, "row counts"))) return fail(st);
    if ((st = fe_alloc_n(&t.tmp, 36 * (size_t)nme + 1, "row columns"))) return fail(st);
    if ((st = fe_alloc_n(&t.big, (size_t)ndof + 1, "long rows"))) return fail(st);
    if ((st = fe_alloc_n(&t.counters, 4, "counters"))) return fail(st);
    if ((st = fe_alloc_n(&p->map, 36 * (size_t)nme, "element-to-nnz map"))) return fail(st);
    if (cudaMemsetAsync(t.counters, 0, 4 * sizeof(int32_t), s) != cudaSuccess) return fail(fe_fail(FE_ERR_CUDA, "memset"));
    if (gather) {
        if ((st = fe_alloc_n(&p->rrec, 6 * (size_t)nme, "row incidence records"))) return fail(st);
        if ((st = fe_alloc_n(&p->long_rows, (size_t)ndof + 1, "long rows"))) return fail(st);
        if ((st = fe_alloc_n(&p->n_long, 2, "long-row count and flag"))) return fail(st);
        if (cudaMemsetAsync(p->n_long, 0, 2 * sizeof(int32_t), s) != cudaSuccess) return fail(fe_fail(FE_ERR_CUDA, "memset"));
    }
    const P2Lists ls{p->rrec, p->long_rows, p->n_long, nq};
    if (ndof > 0) {
        if (nq > 0) {
            { FE_PROF("k_p2_rows", s); k_p2_rows<<<fe_grid(((int64_t)nq + P2_WARPS - 1) / P2_WARPS, 1, 12), P2_WARPS * 32, 0, s>>>(
                  t.vptr, t.inc, p->edof, nq, t.tmp, t.cnt, p->map, t.big, t.counters, ls); }
            FE_LAUNCHED("k_p2_rows");
        }
        if (ndof > nq) {
            { FE_PROF("k_p2_edge_rows", s); k_p2_edge_rows<<<fe_grid((int64_t)ndof - nq, P2_BLOCK, 8), P2_BLOCK, 0, s>>>(
                  t.vptr, t.inc, p->edof, nq, ndof, t.tmp, t.cnt, p->map, t.big, t.counters, ls); }
            FE_LAUNCHED("k_p2_edge_rows");
        }
        const size_t big_smem = sizeof(P2Smem<BIG_TS, BIG_EMAX>);
        FE_CUDA(cudaFuncSetAttribute(k_p2_rows_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem));
        { FE_PROF("k_p2_rows_big", s); k_p2_rows_big<<<fe_sm_count(), 32, big_smem, s>>>(t.vptr, t.inc, p->edof, t.big, t.counters,
                                                                                          t.tmp, t.cnt, p->map, t.counters + 1, ls); }
        FE_LAUNCHED("k_p2_rows_big");
    }
    if ((st = fe_alloc_n(&p->row_ptr, (size_t)ndof + 1, "row_ptr"))) return fail(st);
    int64_t nnz = 0;
    if ((st = fe_exclusive_scan(t.cnt, p->row_ptr, ndof, s, &nnz))) return fail(st);   // synchronises
    int too_big = 0;
    if (cudaMemcpyAsync(&too_big, t.counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (gather && cudaMemcpyAsync(p->n_long_host, p->n_long, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(fe_fail(FE_ERR_CUDA, "flag read-back"));
    if (too_big)
        return fail(fe_fail(FE_ERR_LIMIT, "a vertex belongs to more than FE_P2_MAX_VALENCE=" +
                                              std::to_string(FE_P2_MAX_VALENCE) + " triangles"));
    p->nnz = nnz;
    if ((st = fe_alloc_n(&p->col_idx, (size_t)nnz, "col_idx"))) return fail(st);
    if (ndof > 0) {
        { FE_PROF("k_p2_cols", s); k_p2_cols<<<fe_grid(ndof, P2_BLOCK, 8), P2_BLOCK, 0, s>>>(t.vptr, p->row_ptr, ndof, t.tmp, p->col_idx); }
        FE_LAUNCHED("k_p2_cols");
    }
    if (nme > 0) {
        { FE_PROF("k_p2_map_base", s); k_p2_map_base<<<fe_grid(36 * (int64_t)nme, P2_BLOCK), P2_BLOCK, 0, s>>>(p->edof, nme, p->row_ptr, p->map); }
        FE_LAUNCHED("k_p2_map_base");
    }
    if (gather) {
        if ((st = fe_alloc_n(&p->kg, 36 * (size_t)nme, "element value staging"))) return fail(st);
        p->vptr = t.vptr;                            // the row sums need the incidence offsets
        t.vptr = nullptr;
    }
    *out = p;
    return FE_OK;
}

extern "C" fe_status fe_p2_pattern_info(fe_p2_pattern p, int64_t* n_dofs, int64_t* nnz, const int32_t** row_ptr,
                                        const int32_t** col_idx) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (n_dofs) *n_dofs = p->ndof;
    if (nnz) *nnz = p->nnz;
    if (row_ptr) *row_ptr = p->row_ptr;
    if (col_idx) *col_idx = p->col_idx;
    return FE_OK;
}

extern "C" fe_status fe_p2_pattern_dofs(fe_p2_pattern p, const int32_t** edof, const int32_t** map, int64_t* n_edges) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (edof) *edof = p->edof;
    if (map) *map = p->map;
    if (n_edges) *n_edges = p->ne;
    return FE_OK;
}

extern "C" fe_status fe_p2_assemble(fe_mesh m, fe_p2_pattern p, int kind, int variant, double* values, int64_t cap,
                                    fe_stream stream) {
    FE_RANGE(__func__);
    if (!m || !p) return fe_fail(FE_ERR_INVALID_ARG, "null mesh or pattern");
    if (m->topology_id != p->topology_id) return fe_fail(FE_ERR_INVALID_ARG, "the pattern was built for another mesh");
    if (kind != FE_P2_MASS && kind != FE_P2_STIFF) return fe_fail(FE_ERR_INVALID_ARG, "unknown kind");
    if (variant != FE_VARIANT_ATOMIC && variant != FE_VARIANT_GATHER)
        return fe_fail(FE_ERR_INVALID_ARG, "P2 takes FE_VARIANT_ATOMIC or FE_VARIANT_GATHER");
    if (variant == FE_VARIANT_GATHER && !(p->flags & FE_PATTERN_GATHER))
        return fe_fail(FE_ERR_INVALID_ARG, "FE_VARIANT_GATHER needs a P2 pattern built with FE_PATTERN_GATHER");
    if (cap < p->nnz) return fe_fail(FE_ERR_BUFFER_TOO_SMALL, "cap is below nnz");
    if (!values && p->nnz > 0) return fe_fail(FE_ERR_INVALID_ARG, "values is null");
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    m->last_stream = s;
    p->last_stream = s;
    if (p->nnz == 0) return FE_OK;
    const int32_t nme = m->nme;
    if (variant == FE_VARIANT_GATHER) {
        if (nme > 0) {
            FE_PROF("k_p2_stage", s);
            const unsigned g = fe_grid(nme, STAGE_BLOCK, 4);
            if (kind == FE_P2_MASS) k_p2_stage<FE_P2_MASS><<<g, STAGE_BLOCK, 0, s>>>(m->me, nme, m->q, p->kg);
            else k_p2_stage<FE_P2_STIFF><<<g, STAGE_BLOCK, 0, s>>>(m->me, nme, m->q, p->kg);
        }
        FE_LAUNCHED("k_p2_stage");
        const int32_t nq = p->nq, ndof = p->ndof;
        if (nq > 0) {
            FE_PROF("k_p2_rowsum (vertex rows)", s);
            if (!p->n_long_host[1])
                k_p2_rowsum<RS_VERTEX_SHORT><<<fe_grid(nq, RS_BLOCK, 8), RS_BLOCK, 0, s>>>(p->vptr, p->row_ptr, 0, nq, p->rrec,
                                                                                         p->kg, values, 6 * (int64_t)nme);
            else
                k_p2_rowsum<RS_VERTEX><<<fe_grid(nq, RS_BLOCK, 8), RS_BLOCK, 0, s>>>(p->vptr, p->row_ptr, 0, nq, p->rrec, p->kg,
                                                                                   values, 6 * (int64_t)nme);
            FE_LAUNCHED("k_p2_rowsum (vertex rows)");
        }
        if (ndof > nq) {
            { FE_PROF("k_p2_rowsum_edge", s); k_p2_rowsum_edge<<<fe_grid((int64_t)ndof - nq, RS_BLOCK, 16), RS_BLOCK, 0, s>>>(
                  p->vptr, p->row_ptr, nq, ndof, p->rrec, p->kg, values); }
            FE_LAUNCHED("k_p2_rowsum (edge rows)");
        }
        if (p->n_long_host[0] > 0) {
            const size_t sm = (size_t)RS_LONG_MAX * sizeof(double);
            { FE_PROF("k_p2_rowsum_long", s); k_p2_rowsum_long<<<fe_sm_count() * 8, 32, sm, s>>>(
                  p->long_rows, p->n_long, p->vptr, p->row_ptr, p->rrec, p->kg, values); }
            FE_LAUNCHED("k_p2_rowsum_long");
        }
        return FE_OK;
    }
    FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (size_t)p->nnz, s));
    if (nme > 0) {
        FE_PROF("k_p2_atomic", s);
        const unsigned g = fe_grid(nme, P2_BLOCK, 8);
        if (kind == FE_P2_MASS) k_p2_atomic<FE_P2_MASS><<<g, P2_BLOCK, 0, s>>>(m->me, nme, m->q, p->map, values, p->nnz);
        else k_p2_atomic<FE_P2_STIFF><<<g, P2_BLOCK, 0, s>>>(m->me, nme, m->q, p->map, values, p->nnz);
    }
    FE_LAUNCHED("k_p2_atomic");
    return FE_OK;
}
