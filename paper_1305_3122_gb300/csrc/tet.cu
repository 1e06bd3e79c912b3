// tet.cu -- P1 tetrahedra (3-D): mesh handles, pattern build and the assembly of M, M^w and S.
//
// The paper states that its method extends to three dimensions and gives no formulas. The
// element matrices follow the standard P1 integrals on a tetrahedron K with vertices p0..p3:
// with edge vectors a = p1 - p0, b = p2 - p0, c = p3 - p0 and det = a . (b x c) = 6|K|, the
// barycentric gradients are grad(phi_1) = (b x c)/det, grad(phi_2) = (c x a)/det,
// grad(phi_3) = (a x b)/det, grad(phi_0) = -(their sum), and
//   M^e_ab   = |K|/20 (1 + delta_ab)
//   M^w_ab   = |K|/120 (2 W + 4 w_a) on the diagonal, |K|/120 (W + w_a + w_b) off it (W = sum w)
//   S^e_ab   = |K| grad(phi_a) . grad(phi_b) = (g_a . g_b) / (6 det), g = the unnormalised gradients.
//
// Pattern (the structural half of sparse()): a counting sort by vertex drops, for each
// tetrahedron k and each of its vertices a, the record (its three other vertices, 4k + a) into the
// bucket of vertex me[a][k]. One warp per row then inserts the row's neighbour ids into a
// shared-memory hash table (repeats merge; each insertion keeps the slot it got), ranks the distinct
// ids (their rank is the column's position in the sorted row), and writes, for every incidence,
// the in-row positions of its four columns: the element-to-nnz map, row-major per element
// (map[16k + 4 il + jl]), relative to the row start until the offsets are known. For the
// deterministic gather variant the warp also lists the row's incidences in ascending element order,
// each with the in-row positions of its four columns: row i has exactly (its valence) incidences,
// so its part of the list starts at vptr[i] before any offset is known. The assembly then stages
// the element matrices and sums each row from that list (row a of element k is the 32-byte sector
// at 16k + 4a of the staging buffer), so every non-zero adds its contributions in ascending
// element order.
#include "ff.cuh"
#include "internal.cuh"
#include "rowhash.cuh"

namespace {

constexpr int TET_BLOCK = 256;
constexpr int ROW_WARPS = 4;                 // warps per block in the row pass (fast rows)
constexpr int FAST_TS = 128;                 // hash-table slots per warp, fast rows (small, for occupancy)
constexpr int FAST_EMAX = 42;                // fast rows: at most 42 tetrahedra (3 * 42 + 1 ids < 128)
constexpr int BIG_TS = 4096;                 // one warp per block for rows up to FE_TET_MAX_VALENCE
constexpr int BIG_EMAX = FE_TET_MAX_VALENCE;
constexpr int RS_BLOCK = 128;                // row sums: threads per block, one row each
constexpr int RS_MAX = FE_TET_RS_MAX;        // row sums: longest row summed by one thread (longer: one warp)
constexpr int RS_SHORT = FE_TET_RS_SHORT;    // row sums: smaller accumulators when no row is longer (twice
                                             // the resident blocks and more L1: 1.30 against 2.80 ms at 128^3)
static_assert(3 * BIG_EMAX + 1 < BIG_TS, "the big-row table must hold every distinct id");
static_assert(3 * FAST_EMAX + 1 < FAST_TS, "the fast-row table must hold every distinct id");

enum { BAD_RANGE = 1, BAD_REPEAT = 2, BAD_ORIENT = 4 };

__global__ void k_tet_pack(const double* __restrict__ q, int32_t nq, double4_32a* __restrict__ q4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x)
        q4[i] = make_double4_32a(q[i], q[nq + i], q[2 * (int64_t)nq + i], 0.0);
}

// Sign of det[p1-p0 | p2-p0 | p3-p0] > 0, first from truncated-float coordinates: each float
// edge component is within delta = 2^-22 M + 2^-24 E of the exact one (M = largest |coordinate|,
// E = largest |edge component|), which moves the determinant by at most 16 delta (E + delta)^2
// (Hadamard's bound for each perturbed column), and the float evaluation errs by at most
// 4 * 2^-24 times the sum of the six |products| <= 6 E^3. When |det_f| exceeds both the sign is
// certain; otherwise (or out of the float range) the determinant is recomputed in FP64.
__device__ __forceinline__ bool tet_positive(double4_32a p0, double4_32a p1, double4_32a p2, double4_32a p3) {
    const float x0 = fe_trunc_float(p0.x), y0 = fe_trunc_float(p0.y), z0 = fe_trunc_float(p0.z);
    const float x1 = fe_trunc_float(p1.x), y1 = fe_trunc_float(p1.y), z1 = fe_trunc_float(p1.z);
    const float x2 = fe_trunc_float(p2.x), y2 = fe_trunc_float(p2.y), z2 = fe_trunc_float(p2.z);
    const float x3 = fe_trunc_float(p3.x), y3 = fe_trunc_float(p3.y), z3 = fe_trunc_float(p3.z);
    const float ax = x1 - x0, ay = y1 - y0, az = z1 - z0;
    const float bx = x2 - x0, by = y2 - y0, bz = z2 - z0;
    const float cx = x3 - x0, cy = y3 - y0, cz = z3 - z0;
    const float det = ax * (by * cz - bz * cy) - ay * (bx * cz - bz * cx) + az * (bx * cy - by * cx);
    float M = fmaxf(fmaxf(fmaxf(fabsf(x0), fabsf(y0)), fmaxf(fabsf(z0), fabsf(x1))),
                    fmaxf(fmaxf(fabsf(y1), fabsf(z1)), fmaxf(fabsf(x2), fabsf(y2))));
    M = fmaxf(M, fmaxf(fmaxf(fabsf(z2), fabsf(x3)), fmaxf(fabsf(y3), fabsf(z3))));
    float E = fmaxf(fmaxf(fmaxf(fabsf(ax), fabsf(ay)), fmaxf(fabsf(az), fabsf(bx))),
                    fmaxf(fmaxf(fabsf(by), fabsf(bz)), fmaxf(fabsf(cx), fabsf(cy))));
    E = fmaxf(E, fabsf(cz));
    const float delta = 2.4e-7f * M + 6.0e-8f * E;
    const float err = 2.9e-6f * E * E * E + 16.0f * delta * (E + delta) * (E + delta);
    if (fabsf(det) > err && E < 1e12f && E > 1e-10f && M < 1e30f) return det > 0.0f;
    const double dax = p1.x - p0.x, day = p1.y - p0.y, daz = p1.z - p0.z;
    const double dbx = p2.x - p0.x, dby = p2.y - p0.y, dbz = p2.z - p0.z;
    const double dcx = p3.x - p0.x, dcy = p3.y - p0.y, dcz = p3.z - p0.z;
    return dax * (dby * dcz - dbz * dcy) - day * (dbx * dcz - dbz * dcx) + daz * (dbx * dcy - dby * dcx) > 0.0;
}

// Range, repeats and orientation of every tetrahedron; counts each vertex's tetrahedra.
__global__ void k_tet_validate(const double4_32a* __restrict__ q, int32_t nq, const int32_t* __restrict__ me,
                               int32_t nme, int* __restrict__ word, int32_t* __restrict__ deg) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[4];
#pragma unroll
        for (int a = 0; a < 4; a++) v[a] = me[a * (int64_t)nme + k];
        int bad = 0;
        bool in = true;
#pragma unroll
        for (int a = 0; a < 4; a++) in &= v[a] >= 0 && v[a] < nq;
        if (!in) {
            bad = BAD_RANGE;
        } else {
#pragma unroll
            for (int a = 0; a < 4; a++) atomicAdd(&deg[v[a]], 1);
            if (v[0] == v[1] || v[0] == v[2] || v[0] == v[3] || v[1] == v[2] || v[1] == v[3] || v[2] == v[3])
                bad = BAD_REPEAT;
            else if (!tet_positive(q[v[0]], q[v[1]], q[v[2]], q[v[3]]))
                bad = BAD_ORIENT;
        }
        if (bad) {
            atomicOr(&word[0], bad);
            atomicMin(&word[bad == BAD_RANGE ? 1 : bad == BAD_REPEAT ? 2 : 3], (int)k);
        }
    }
}

// Bucket records: for tetrahedron k and vertex a, (v[a+1], v[a+2], v[a+3], 4k + a) (indices mod 4)
// into the bucket of v[a]; the cursors start at the bucket starts.
__global__ void k_tet_fill(const int32_t* __restrict__ me, int32_t nme, int32_t* __restrict__ cur,
                           int4* __restrict__ adj) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[4];
#pragma unroll
        for (int a = 0; a < 4; a++) v[a] = me[a * (int64_t)nme + k];
        int32_t slot[4];
#pragma unroll
        for (int a = 0; a < 4; a++) slot[a] = FE_IDX(atomicAdd(&cur[v[a]], 1), 4 * (int64_t)nme);
#pragma unroll
        for (int a = 0; a < 4; a++)
            adj[slot[a]] = make_int4(v[(a + 1) & 3], v[(a + 2) & 3], v[(a + 3) & 3], 4 * (int32_t)k + a);
    }
}

// Per-warp shared memory of the row pass for a table of TS slots and at most EMAX incidences.
template <int TS, int EMAX>
struct RowSmem {
    int32_t tab[TS];     // ids (-1: empty)
    int32_t rnk[TS];     // rank (column position) of each slot's id
    int32_t uid[TS];     // the distinct ids, in insertion order
    int32_t uslot[TS];   // their slots
    int4 e[EMAX];        // the row's bucket records
    int16_t xs[4 * EMAX];  // the slot of each incidence's four ids (the row's vertex, then x, y, z)
    int32_t ucount;
};

// Where the gather lists of the deterministic variant go.
struct RowLists {
    int32_t* inc;        // [4 nme]: the keys 4k + a of each row's incidences, ascending, row i from vptr[i]
    uint2* islot;        // [4 nme]: the in-row positions of their columns jl = 0..3, 16 bits each
    int32_t* long_rows;  // rows with more than RS_MAX columns
    int32_t* n_long;     // their number
    int32_t* any_over_short;  // set when a row has more than RS_SHORT columns
};

// One row by one warp: distinct columns (sorted, into tmp at 3 vptr[i] + i), their count, the
// relative map of every incidence, and (GATHER) the row's incidence list in ascending element
// order with the positions of their columns.
template <int TS, int EMAX, bool GATHER>
__device__ void tet_row(int32_t i, int32_t beg, int32_t d, const int4* __restrict__ adj, RowSmem<TS, EMAX>& sm,
                        int32_t* __restrict__ tmp, int32_t* __restrict__ cnt, int32_t* __restrict__ map,
                        const RowLists& rl) {
    const int lane = threadIdx.x & 31;
    for (int s = lane; s < TS; s += 32) {
        sm.tab[s] = -1;
    }
    if (lane == 0) sm.ucount = 0;
    for (int t = lane; t < d; t += 32) sm.e[t] = adj[beg + t];
    __syncwarp();
    // every incidence contributes the row's own vertex and its three other vertices
    for (int x = lane; x < 4 * d; x += 32) {
        const int4 r = sm.e[x >> 2];
        const int q = x & 3;
        const int32_t id = q == 0 ? i : q == 1 ? r.x : q == 2 ? r.y : r.z;
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
    const int64_t tb = 3 * (int64_t)beg + i;
    for (int p = lane; p < u; p += 32) {
        const int32_t id = sm.uid[p];
        int r = 0;
        for (int qq = 0; qq < u; qq++) r += sm.uid[qq] < id;
        sm.rnk[sm.uslot[p]] = r;
        tmp[tb + r] = id;
    }
    __syncwarp();
    // relative map: the four column positions of each incidence, one 16-byte store
    for (int t = lane; t < d; t += 32) {
        const int4 r = sm.e[t];
        const int a = r.w & 3;
        const int32_t k = r.w >> 2;
        const int ri = sm.rnk[sm.xs[4 * t]];
        const int rx = sm.rnk[sm.xs[4 * t + 1]];
        const int ry = sm.rnk[sm.xs[4 * t + 2]];
        const int rz = sm.rnk[sm.xs[4 * t + 3]];
        int o[4];
#pragma unroll
        for (int jl = 0; jl < 4; jl++) {
            const int off = (jl - a) & 3;     // 0: the row's vertex, 1..3: the record's x, y, z
            o[jl] = off == 0 ? ri : off == 1 ? rx : off == 2 ? ry : rz;
        }
        *reinterpret_cast<int4*>(map + 16 * (int64_t)k + 4 * a) = make_int4(o[0], o[1], o[2], o[3]);
        if (GATHER) {
            // the incidence's place in the row's ascending element order (the keys 4k + a of one
            // row are distinct)
            int c0 = 0;
            for (int tt = 0; tt < d; tt++) c0 += sm.e[tt].w < r.w;
            rl.inc[beg + c0] = r.w;
            rl.islot[beg + c0] = make_uint2((unsigned)o[0] | ((unsigned)o[1] << 16), (unsigned)o[2] | ((unsigned)o[3] << 16));
        }
    }
    if (lane == 0) {
        cnt[i] = u;
        if (GATHER && u > RS_MAX) rl.long_rows[atomicAdd(rl.n_long, 1)] = i;
        if (GATHER && u > RS_SHORT) *rl.any_over_short = 1;
    }
    __syncwarp();
}

// Rows with at most FAST_EMAX tetrahedra, one warp each; longer rows are listed for k_tet_rows_big.
template <bool GATHER>
__global__ void __launch_bounds__(ROW_WARPS * 32, 12) k_tet_rows(const int32_t* __restrict__ vptr, const int4* __restrict__ adj,
                                                            int32_t nq, int32_t* __restrict__ tmp, int32_t* __restrict__ cnt,
                                                            int32_t* __restrict__ map, RowLists rl, int32_t* __restrict__ big_list,
                                                            int32_t* __restrict__ big_count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowSmem<FAST_TS, FAST_EMAX>& sm = reinterpret_cast<RowSmem<FAST_TS, FAST_EMAX>*>(smem_raw)[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * ROW_WARPS;
    for (int64_t r = (int64_t)blockIdx.x * ROW_WARPS + (threadIdx.x >> 5); r < nq; r += nwarps) {
        const int32_t i = (int32_t)r;
        const int32_t beg = vptr[i], d = vptr[i + 1] - beg;
        if (d == 0) {
            if (lane == 0) cnt[i] = 0;
            continue;
        }
        if (d > FAST_EMAX) {
            if (lane == 0) big_list[atomicAdd(big_count, 1)] = i;
            continue;
        }
        tet_row<FAST_TS, FAST_EMAX, GATHER>(i, beg, d, adj, sm, tmp, cnt, map, rl);
    }
}

template <bool GATHER>
__global__ void __launch_bounds__(32) k_tet_rows_big(const int32_t* __restrict__ vptr, const int4* __restrict__ adj,
                                                     const int32_t* __restrict__ big_list,
                                                     const int32_t* __restrict__ big_count, int32_t* __restrict__ tmp,
                                                     int32_t* __restrict__ cnt, int32_t* __restrict__ map, RowLists rl,
                                                     int* __restrict__ too_big) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowSmem<BIG_TS, BIG_EMAX>& sm = *reinterpret_cast<RowSmem<BIG_TS, BIG_EMAX>*>(smem_raw);
    const int32_t n = *big_count;
    for (int32_t b = blockIdx.x; b < n; b += gridDim.x) {
        const int32_t i = big_list[b];
        const int32_t beg = vptr[i], d = vptr[i + 1] - beg;
        if (d > BIG_EMAX) {
            if (threadIdx.x == 0) {
                *too_big = 1;
                cnt[i] = 0;
            }
            continue;
        }
        tet_row<BIG_TS, BIG_EMAX, GATHER>(i, beg, d, adj, sm, tmp, cnt, map, rl);
    }
}

// Columns into their final places, one warp per row.
__global__ void __launch_bounds__(TET_BLOCK) k_tet_cols(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                        int32_t nq, const int32_t* __restrict__ tmp, int32_t* __restrict__ col_idx) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (TET_BLOCK / 32);
    for (int64_t r = (int64_t)blockIdx.x * (TET_BLOCK / 32) + (threadIdx.x >> 5); r < nq; r += nwarps) {
        const int32_t i = (int32_t)r;
        const int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb;
        const int64_t tb = 3 * (int64_t)vptr[i] + i;
        for (int c = lane; c < u; c += 32) col_idx[rb + c] = tmp[tb + c];
    }
}

// map[16k + 4 il + jl] += row_ptr[me[il][k]]: relative positions become absolute.
__global__ void k_tet_map_base(const int32_t* __restrict__ me, int32_t nme, const int32_t* __restrict__ row_ptr,
                               int32_t* __restrict__ map) {
    const int64_t n = 16 * (int64_t)nme;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = c >> 4;
        const int il = (int)(c >> 2) & 3;
        map[c] += row_ptr[me[il * (int64_t)nme + k]];
    }
}

// ------------------------------------------------------------------ element matrices

template <int KIND>
__device__ __forceinline__ void tet_elem(const double4_32a p[4], const double w[4], double E[4][4]) {
    const double ax = p[1].x - p[0].x, ay = p[1].y - p[0].y, az = p[1].z - p[0].z;
    const double bx = p[2].x - p[0].x, by = p[2].y - p[0].y, bz = p[2].z - p[0].z;
    const double cx = p[3].x - p[0].x, cy = p[3].y - p[0].y, cz = p[3].z - p[0].z;
    // unnormalised gradients g_1 = b x c, g_2 = c x a, g_3 = a x b
    double g[4][3];
    g[1][0] = by * cz - bz * cy; g[1][1] = bz * cx - bx * cz; g[1][2] = bx * cy - by * cx;
    g[2][0] = cy * az - cz * ay; g[2][1] = cz * ax - cx * az; g[2][2] = cx * ay - cy * ax;
    g[3][0] = ay * bz - az * by; g[3][1] = az * bx - ax * bz; g[3][2] = ax * by - ay * bx;
    const double det = ax * g[1][0] + ay * g[1][1] + az * g[1][2];   // a . (b x c) = 6|K|
    if (KIND == FE_TET_STIFF) {
        // The gradients and det stay in FP64 (exact to 2^-53, so no cancellation in a cross
        // product or in det is amplified); 1/(6 det), the ten dot products and their scaling run
        // in double-float on the FP32 pipes (ff.cuh), erring by a few units of 2^-48 of
        // |g_a| |g_b| / (6 det) each. That halves the FP64 instructions of an element (85 -> 46,
        // counting the ten conversions back). The twelve gradient components are scaled by a
        // common power of two 2^k that brings the largest to [1, 2) (their products then stay
        // far inside the float range whatever the mesh's size), and 2^-2k goes into 1/(6 det).
        // Every entry keeps its own dot product: deriving vertex 0's entries from the zero row
        // sums loses too much to cancellation on thin tetrahedra (2.7e-13 of the row maximum at
        // the centre of an 80-tetrahedron star).
#pragma unroll
        for (int t = 0; t < 3; t++) g[0][t] = -(g[1][t] + g[2][t] + g[3][t]);
        unsigned emax = 0;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int t = 0; t < 3; t++) emax = max(emax, fp64_biased_exponent(g[a][t]));
        const int k = ff_group_scale(emax);
        ff G[4][3];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int t = 0; t < 3; t++) G[a][t] = ff_from_double_scaled(g[a][t], k);
        // 2^-2k / (6 det): det scaled by 2^2k in the conversion (exact), the reciprocal in
        // double-float (about 46 bits)
        const ff D = ff_from_double_scaled(det, 2 * k);
        const bool ok = D.h != 0.0f;                  // zero: 2^2k det outside the double-float range
        const ff sf = ff_rcp_fast(ff_mulf(D, 6.0f));
        if (ok) {
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = a; b < 4; b++) {
                    const ff d = ff_add(ff_dot2(G[a][0], G[a][1], G[b][0], G[b][1]), ff_mul(G[a][2], G[b][2]));
                    const double v = ff_to_double(ff_mul(d, sf));
                    E[a][b] = v;
                    E[b][a] = v;
                }
        } else {                                      // outside the double-float range: all FP64
            const double sd = 1.0 / (6.0 * det);
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = a; b < 4; b++) {
                    const double v = (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]) * sd;
                    E[a][b] = v;
                    E[b][a] = v;
                }
        }
    } else if (KIND == FE_TET_MASS) {
        const double m = det / 120.0;                 // |K| / 20
        const double m2 = 2.0 * m;
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) E[a][b] = a == b ? m2 : m;
    } else {
        // the ten distinct entries: m (2W + 4 w_a) on the diagonal, m (W + w_a + w_b) off it
        // |K| / 120 by a constant reciprocal (no run-time division: the stage kernel of this kind is
        // bound by its FP64 instructions, 1.15 -> 1.01 ms at 128^3; the mass kind, bound by its stores,
        // measured slower that way and keeps its division)
        const double m = det * (1.0 / 720.0);
        const double mW = m * (w[0] + w[1] + w[2] + w[3]);
        double u[4];
#pragma unroll
        for (int a = 0; a < 4; a++) u[a] = m * w[a];
        const double mW2 = 2.0 * mW;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            E[a][a] = fma(4.0, u[a], mW2);
#pragma unroll
            for (int b = a + 1; b < 4; b++) {
                const double v = mW + u[a] + u[b];
                E[a][b] = v;
                E[b][a] = v;
            }
        }
    }
}

template <int KIND>
__device__ __forceinline__ void tet_load(const int32_t* __restrict__ me, int32_t nme, int64_t k, const double4_32a* __restrict__ q,
                                         const double* __restrict__ w, double4_32a p[4], double wl[4]) {
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int32_t v = me[a * (int64_t)nme + k];
        p[a] = q[v];
        wl[a] = KIND == FE_TET_WMASS ? w[v] : 0.0;
    }
}

template <int KIND>
__global__ void __launch_bounds__(TET_BLOCK) k_tet_atomic(const int32_t* __restrict__ me, int32_t nme, const double4_32a* __restrict__ q,
                                                          const double* __restrict__ w, const int32_t* __restrict__ map,
                                                          double* __restrict__ val, int64_t nnz) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        double4_32a p[4];
        double wl[4], E[4][4];
        tet_load<KIND>(me, nme, k, q, w, p, wl);
        tet_elem<KIND>(p, wl, E);
        const int4* m4 = reinterpret_cast<const int4*>(map + 16 * k);
#pragma unroll
        for (int il = 0; il < 4; il++) {
            const int4 m = m4[il];
            atomicAdd(&val[FE_IDX(m.x, nnz)], E[il][0]);
            atomicAdd(&val[FE_IDX(m.y, nnz)], E[il][1]);
            atomicAdd(&val[FE_IDX(m.z, nnz)], E[il][2]);
            atomicAdd(&val[FE_IDX(m.w, nnz)], E[il][3]);
        }
    }
}

template <int KIND>
__global__ void __launch_bounds__(TET_BLOCK) k_tet_stage(const int32_t* __restrict__ me, int32_t nme, const double4_32a* __restrict__ q,
                                                         const double* __restrict__ w, double* __restrict__ kg) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        double4_32a p[4];
        double wl[4], E[4][4];
        tet_load<KIND>(me, nme, k, q, w, p, wl);
        tet_elem<KIND>(p, wl, E);
        double2* o = reinterpret_cast<double2*>(kg + 16 * k);
#pragma unroll
        for (int il = 0; il < 4; il++) {
            o[2 * il] = make_double2(E[il][0], E[il][1]);
            o[2 * il + 1] = make_double2(E[il][2], E[il][3]);
        }
    }
}

// Row sums of the staged element matrices, one row per thread: the row's incidences in ascending
// element order each add row a of element k (the 32-byte sector at kg[16k + 4a]) to the row's
// accumulators in shared memory, at the in-row positions of the four columns. Accumulators start
// at -0.0, so every sum equals its first contribution followed by the others in ascending element
// order, bit for bit. Rows with more than RMAX columns are left to k_tet_rowsum_long. Four
// incidences are loaded before any is added (four random sectors in flight per thread), and the
// next four's keys and slots are loaded meanwhile.
template <int RMAX>
__global__ void __launch_bounds__(RS_BLOCK) k_tet_rowsum(const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                         int32_t nq, const int32_t* __restrict__ inc,
                                                         const uint2* __restrict__ islot, const double* __restrict__ kg,
                                                         double* __restrict__ val, int64_t n4) {
    __shared__ double acc[RMAX * RS_BLOCK];
    double* a = acc + threadIdx.x;                       // column c of this thread's row at a[c * RS_BLOCK]
    for (int64_t r = blockIdx.x * (int64_t)RS_BLOCK + threadIdx.x; r < nq; r += (int64_t)gridDim.x * RS_BLOCK) {
        const int32_t rb = row_ptr[r], u = row_ptr[r + 1] - rb;
        if (u > RMAX) continue;
        const int32_t b0 = vptr[r], d = vptr[r + 1] - b0;
        for (int c = 0; c < u; c++) a[c * RS_BLOCK] = -0.0;
        int32_t key[4];
        uint2 sl[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            key[j] = j < d ? inc[b0 + j] : 0;
            sl[j] = j < d ? islot[b0 + j] : make_uint2(0u, 0u);
        }
        for (int32_t t0 = 0; t0 < d; t0 += 4) {
            double2 v[4][2];
            uint2 cs[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                cs[j] = sl[j];
                if (t0 + j < d) {
                    const double2* e = reinterpret_cast<const double2*>(kg + 4 * (int64_t)FE_IDX(key[j], n4));
                    v[j][0] = e[0];
                    v[j][1] = e[1];
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int32_t tn = t0 + 4 + j;
                key[j] = tn < d ? inc[b0 + tn] : 0;
                sl[j] = tn < d ? islot[b0 + tn] : make_uint2(0u, 0u);
            }
            // an incidence's four columns are distinct: its four accumulators are read before any
            // is written back, so the four updates overlap instead of waiting on one another
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (t0 + j < d) {
                    double* p0 = a + FE_IDX(cs[j].x & 0xFFFFu, u) * RS_BLOCK;
                    double* p1 = a + FE_IDX(cs[j].x >> 16, u) * RS_BLOCK;
                    double* p2 = a + FE_IDX(cs[j].y & 0xFFFFu, u) * RS_BLOCK;
                    double* p3 = a + FE_IDX(cs[j].y >> 16, u) * RS_BLOCK;
                    const double y0 = *p0, y1 = *p1, y2 = *p2, y3 = *p3;
                    *p0 = y0 + v[j][0].x;
                    *p1 = y1 + v[j][0].y;
                    *p2 = y2 + v[j][1].x;
                    *p3 = y3 + v[j][1].y;
                }
            }
        }
        for (int c = 0; c < u; c++) val[rb + c] = a[c * RS_BLOCK];
    }
}

// The rows with more than RS_MAX columns, one warp each: lane l owns the columns c = l (mod 32)
// and adds their contributions in ascending element order (accumulators in dynamic shared
// memory, 3 FE_TET_MAX_VALENCE + 1 doubles at most).
__global__ void __launch_bounds__(32) k_tet_rowsum_long(const int32_t* __restrict__ long_rows, const int32_t* __restrict__ n_long,
                                                        const int32_t* __restrict__ vptr, const int32_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ inc, const uint2* __restrict__ islot,
                                                        const double* __restrict__ kg, double* __restrict__ val) {
    extern __shared__ double accl[];
    const int lane = threadIdx.x;
    const int32_t n = *n_long;
    for (int32_t b = blockIdx.x; b < n; b += gridDim.x) {
        const int32_t i = long_rows[b];
        const int32_t rb = row_ptr[i], u = row_ptr[i + 1] - rb;
        const int32_t b0 = vptr[i], d = vptr[i + 1] - b0;
        for (int c = lane; c < u; c += 32) accl[c] = -0.0;
        __syncwarp();
        for (int32_t t = 0; t < d; t++) {
            const int32_t key = inc[b0 + t];
            const uint2 sl = islot[b0 + t];
            const unsigned c4[4] = {sl.x & 0xFFFFu, sl.x >> 16, sl.y & 0xFFFFu, sl.y >> 16};
#pragma unroll
            for (int jl = 0; jl < 4; jl++)
                if ((int)(c4[jl] & 31u) == lane) accl[c4[jl]] += kg[4 * (int64_t)key + jl];
        }
        __syncwarp();
        for (int c = lane; c < u; c += 32) val[rb + c] = accl[c];
        __syncwarp();
    }
}

}  // namespace

// ------------------------------------------------------------------ handles

extern "C" void fe_tet_mesh_destroy(fe_tet_mesh m) {
    if (!m) return;
    FeStreamScope scope(m->last_stream);
    fe_free(m->q);
    if (m->me_owned) fe_free(m->me);
    fe_free(m->err);
    fe_free(m->deg);
    delete m;
}

extern "C" fe_status fe_tet_mesh_create(int32_t nq, int32_t nme, const double* q, const int32_t* me, int ptr_kind,
                                        fe_stream stream, fe_tet_mesh* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (nq < 0 || nme < 0) return fe_fail(FE_ERR_INVALID_ARG, "nq and nme must be >= 0");
    if ((nq > 0 && !q) || (nme > 0 && !me)) return fe_fail(FE_ERR_INVALID_ARG, "q or me is null");
    if (ptr_kind != FE_PTR_HOST && ptr_kind != FE_PTR_DEVICE && ptr_kind != FE_PTR_DEVICE_BORROW)
        return fe_fail(FE_ERR_INVALID_ARG, "bad ptr_kind");
    if (16 * (int64_t)nme >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "16*nme must be < 2^31");
    const bool borrow = ptr_kind == FE_PTR_DEVICE_BORROW;
    const cudaMemcpyKind dir = ptr_kind == FE_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    fe_tet_mesh m = new fe_tet_mesh_s();
    m->last_stream = s;
    m->nq = nq;
    m->nme = nme;
    m->topology_id = fe_next_topology_id();
    double* qtmp = nullptr;
    fe_status st = fe_alloc_n(&m->q, (size_t)nq, "tetrahedral mesh coordinates");
    if (!st) st = fe_alloc_n(&m->err, 4, "mesh error word");
    if (!st) st = fe_alloc_n(&m->deg, (size_t)nq + 1, "vertex valences");
    if (!st && borrow) {
        m->me = const_cast<int32_t*>(me);
        m->me_owned = false;
    } else if (!st) {
        st = fe_alloc_n(&m->me, 4 * (size_t)nme, "tetrahedral mesh connectivity");
        if (!st && nme > 0 && cudaMemcpyAsync(m->me, me, 16 * (size_t)nme, dir, s) != cudaSuccess)
            st = fe_fail(FE_ERR_CUDA, "copy of me");
    }
    const double* qd = q;
    if (!st && nq > 0 && ptr_kind == FE_PTR_HOST) {
        st = fe_alloc_n(&qtmp, 3 * (size_t)nq, "coordinate staging");
        if (!st && cudaMemcpyAsync(qtmp, q, 24 * (size_t)nq, cudaMemcpyHostToDevice, s) != cudaSuccess)
            st = fe_fail(FE_ERR_CUDA, "copy of q");
        qd = qtmp;
    }
    if (st) { fe_free(qtmp); fe_tet_mesh_destroy(m); return st; }
    int word[4];
    cudaError_t e = cudaSuccess;
    if (nq > 0) {
        { FE_PROF("k_tet_pack", s); k_tet_pack<<<fe_grid(nq, TET_BLOCK), TET_BLOCK, 0, s>>>(qd, nq, m->q); }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->err + 1, 0x7F, 3 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->deg, 0, sizeof(int32_t) * ((size_t)nq + 1), s);
    if (e == cudaSuccess && nme > 0) {
        { FE_PROF("k_tet_validate", s); k_tet_validate<<<fe_grid(nme, TET_BLOCK, 16), TET_BLOCK, 0, s>>>(m->q, nq, m->me, nme, m->err, m->deg); }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(word, m->err, sizeof word, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    fe_free(qtmp);
    if (e != cudaSuccess) { fe_tet_mesh_destroy(m); return fe_cuda_fail(e, "tetrahedral mesh validation"); }
    if (word[0] & BAD_RANGE) {
        fe_tet_mesh_destroy(m);
        return fe_fail(FE_ERR_INDEX_RANGE, "tetrahedron " + std::to_string(word[1]) + " has a vertex id outside [0, nq)");
    }
    if (word[0] & BAD_REPEAT) {
        fe_tet_mesh_destroy(m);
        return fe_fail(FE_ERR_DEGENERATE, "tetrahedron " + std::to_string(word[2]) + " repeats a vertex");
    }
    if (word[0] & BAD_ORIENT) {
        fe_tet_mesh_destroy(m);
        return fe_fail(FE_ERR_ORIENTATION, "tetrahedron " + std::to_string(word[3]) +
                                               " has det[p1-p0 | p2-p0 | p3-p0] <= 0");
    }
    *out = m;
    return FE_OK;
}

extern "C" void fe_tet_pattern_destroy(fe_tet_pattern p) {
    if (!p) return;
    FeStreamScope scope(p->last_stream);
    fe_free(p->row_ptr); fe_free(p->col_idx); fe_free(p->map);
    fe_free(p->vptr); fe_free(p->inc); fe_free(p->islot); fe_free(p->long_rows); fe_free(p->n_long); fe_free(p->kg);
    fe_free(p->row_ptr3); fe_free(p->col_idx3);
    delete p;
}

namespace {
struct TetTemps {
    int32_t *vptr = nullptr, *cur = nullptr, *cnt = nullptr, *tmp = nullptr;
    int32_t *big = nullptr, *counters = nullptr;
    int4* adj = nullptr;
    ~TetTemps() {
        fe_free(vptr); fe_free(cur); fe_free(cnt); fe_free(tmp);
        fe_free(big); fe_free(counters); fe_free(adj);
    }
};

template <bool GATHER>
fe_status tet_rows(const TetTemps& t, int32_t nq, fe_tet_pattern p, cudaStream_t s) {
    const RowLists rl{p->inc, p->islot, p->long_rows, p->n_long, p->n_long ? p->n_long + 1 : nullptr};
    const size_t fast_smem = ROW_WARPS * sizeof(RowSmem<FAST_TS, FAST_EMAX>);
    const size_t big_smem = sizeof(RowSmem<BIG_TS, BIG_EMAX>);
    FE_CUDA(cudaFuncSetAttribute(k_tet_rows<GATHER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fast_smem));
    FE_CUDA(cudaFuncSetAttribute(k_tet_rows_big<GATHER>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)big_smem));
    { FE_PROF("k_tet_rows", s); k_tet_rows<GATHER><<<fe_grid(((int64_t)nq + ROW_WARPS - 1) / ROW_WARPS, 1, 8), ROW_WARPS * 32, fast_smem, s>>>(
          t.vptr, t.adj, nq, t.tmp, t.cnt, p->map, rl, t.big, t.counters); }
    FE_LAUNCHED("k_tet_rows");
    { FE_PROF("k_tet_rows_big", s); k_tet_rows_big<GATHER><<<fe_sm_count(), 32, big_smem, s>>>(
          t.vptr, t.adj, t.big, t.counters, t.tmp, t.cnt, p->map, rl, t.counters + 1); }
    FE_LAUNCHED("k_tet_rows_big");
    return FE_OK;
}
}  // namespace

extern "C" fe_status fe_tet_pattern_build(fe_tet_mesh m, int flags, fe_stream stream, fe_tet_pattern* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!m) return fe_fail(FE_ERR_INVALID_ARG, "null mesh");
    const bool gather = (flags & FE_PATTERN_GATHER) != 0;
    const int32_t nq = m->nq, nme = m->nme;
    const int64_t n4 = 4 * (int64_t)nme;
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    fe_tet_pattern p = new fe_tet_pattern_s();
    p->flags = (gather ? FE_PATTERN_GATHER : 0) | (flags & FE_TET_PATTERN_ELAS);
    p->nq = nq;
    p->nme = nme;
    p->topology_id = m->topology_id;
    p->last_stream = s;
    m->last_stream = s;
    TetTemps t;
    auto fail = [&](fe_status st) {
        cudaStreamSynchronize(s);
        fe_tet_pattern_destroy(p);
        return st;
    };
    fe_status st;
    const int64_t tcap = 3 * n4 + nq;            // sum over rows of 3 d + 1
    if ((st = fe_alloc_n(&t.vptr, (size_t)nq + 1, "vertex pointers"))) return fail(st);
    if ((st = fe_alloc_n(&t.cur, (size_t)nq + 1, "bucket cursors"))) return fail(st);
    if ((st = fe_exclusive_scan(m->deg, t.vptr, nq, s, nullptr, 1, t.cur))) return fail(st);
    if ((st = fe_alloc_n(&t.adj, (size_t)n4, "row buckets"))) return fail(st);
    if (nme > 0) {
        { FE_PROF("k_tet_fill", s); k_tet_fill<<<fe_grid(nme, TET_BLOCK, 16), TET_BLOCK, 0, s>>>(m->me, nme, t.cur, t.adj); }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(fe_cuda_fail(e, "k_tet_fill"));
    }
    if ((st = fe_alloc_n(&t.cnt, (size_t)nq + 1, "row counts"))) return fail(st);
    if ((st = fe_alloc_n(&t.tmp, (size_t)tcap, "row columns"))) return fail(st);
    if ((st = fe_alloc_n(&t.big, (size_t)nq + 1, "long rows"))) return fail(st);
    if ((st = fe_alloc_n(&t.counters, 4, "counters"))) return fail(st);
    if ((st = fe_alloc_n(&p->map, 16 * (size_t)nme, "element-to-nnz map"))) return fail(st);
    if (gather) {
        if ((st = fe_alloc_n(&p->inc, (size_t)n4, "row incidence lists"))) return fail(st);
        if ((st = fe_alloc_n(&p->islot, (size_t)n4, "row incidence column slots"))) return fail(st);
        if ((st = fe_alloc_n(&p->long_rows, (size_t)nq + 1, "long rows"))) return fail(st);
        if ((st = fe_alloc_n(&p->n_long, 2, "long-row count and longest row"))) return fail(st);
        if (cudaMemsetAsync(p->n_long, 0, 2 * sizeof(int32_t), s) != cudaSuccess) return fail(fe_fail(FE_ERR_CUDA, "memset"));
    }
    if (cudaMemsetAsync(t.counters, 0, 4 * sizeof(int32_t), s) != cudaSuccess) return fail(fe_fail(FE_ERR_CUDA, "memset"));
    if (nq > 0) {
        st = gather ? tet_rows<true>(t, nq, p, s) : tet_rows<false>(t, nq, p, s);
        if (st) return fail(st);
    }
    if ((st = fe_alloc_n(&p->row_ptr, (size_t)nq + 1, "row_ptr"))) return fail(st);
    int64_t nnz = 0;
    if ((st = fe_exclusive_scan(t.cnt, p->row_ptr, nq, s, &nnz))) return fail(st);   // synchronises
    int too_big = 0;
    if (cudaMemcpyAsync(&too_big, t.counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (gather && cudaMemcpyAsync(p->n_long_host, p->n_long, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(fe_fail(FE_ERR_CUDA, "flag read-back"));
    if (too_big)
        return fail(fe_fail(FE_ERR_LIMIT, "a vertex belongs to more than FE_TET_MAX_VALENCE=" +
                                              std::to_string(FE_TET_MAX_VALENCE) + " tetrahedra"));
    p->nnz = nnz;
    if ((st = fe_alloc_n(&p->col_idx, (size_t)nnz, "col_idx"))) return fail(st);
    if (gather && (st = fe_alloc_n(&p->kg, 16 * (size_t)nme, "element value staging"))) return fail(st);
    if (nq > 0) {
        const unsigned g = fe_grid(((int64_t)nq + 7) / 8, 1, 8);
        { FE_PROF("k_tet_cols", s); k_tet_cols<<<g, TET_BLOCK, 0, s>>>(t.vptr, p->row_ptr, nq, t.tmp, p->col_idx); }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(fe_cuda_fail(e, "k_tet_cols"));
    }
    if (nme > 0) {
        { FE_PROF("k_tet_map_base", s); k_tet_map_base<<<fe_grid(16 * (int64_t)nme, TET_BLOCK), TET_BLOCK, 0, s>>>(m->me, nme, p->row_ptr, p->map); }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(fe_cuda_fail(e, "k_tet_map_base"));
    }
    if (gather) {                                // the row sums need the incidence offsets
        p->vptr = t.vptr;
        t.vptr = nullptr;
    }
    if ((flags & FE_TET_PATTERN_ELAS) && (st = fe_tet_elas_structure(p, s))) return fail(st);
    *out = p;
    return FE_OK;
}

extern "C" fe_status fe_tet_pattern_info(fe_tet_pattern p, int64_t* n_rows, int64_t* nnz, const int32_t** row_ptr,
                                         const int32_t** col_idx) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (n_rows) *n_rows = p->nq;
    if (nnz) *nnz = p->nnz;
    if (row_ptr) *row_ptr = p->row_ptr;
    if (col_idx) *col_idx = p->col_idx;
    return FE_OK;
}

extern "C" fe_status fe_tet_pattern_map(fe_tet_pattern p, const int32_t** map, int64_t* len) {
    if (!p) return fe_fail(FE_ERR_INVALID_ARG, "null pattern");
    if (map) *map = p->map;
    if (len) *len = 16 * (int64_t)p->nme;
    return FE_OK;
}

extern "C" fe_status fe_tet_assemble(fe_tet_mesh m, fe_tet_pattern p, int kind, const double* w, int variant,
                                     double* values, int64_t cap, fe_stream stream) {
    FE_RANGE(__func__);
    if (!m || !p) return fe_fail(FE_ERR_INVALID_ARG, "null mesh or pattern");
    if (m->topology_id != p->topology_id) return fe_fail(FE_ERR_INVALID_ARG, "the pattern was built for another mesh");
    if (kind != FE_TET_MASS && kind != FE_TET_WMASS && kind != FE_TET_STIFF) return fe_fail(FE_ERR_INVALID_ARG, "unknown kind");
    if (kind == FE_TET_WMASS && !w && m->nq > 0) return fe_fail(FE_ERR_INVALID_ARG, "w is null");
    if (variant != FE_VARIANT_ATOMIC && variant != FE_VARIANT_GATHER)
        return fe_fail(FE_ERR_INVALID_ARG, "tetrahedra take FE_VARIANT_ATOMIC or FE_VARIANT_GATHER");
    if (variant == FE_VARIANT_GATHER && !(p->flags & FE_PATTERN_GATHER))
        return fe_fail(FE_ERR_INVALID_ARG, "FE_VARIANT_GATHER needs a pattern built with FE_PATTERN_GATHER");
    if (cap < p->nnz) return fe_fail(FE_ERR_BUFFER_TOO_SMALL, "cap is below nnz");
    if (!values && p->nnz > 0) return fe_fail(FE_ERR_INVALID_ARG, "values is null");
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    m->last_stream = s;
    p->last_stream = s;
    const int32_t nme = m->nme;
    if (p->nnz == 0) return FE_OK;
    const unsigned g = fe_grid(nme, TET_BLOCK, 8);
    if (variant == FE_VARIANT_ATOMIC) {
        FE_CUDA(cudaMemsetAsync(values, 0, sizeof(double) * (size_t)p->nnz, s));
        if (nme > 0) {
            FE_PROF("k_tet_atomic", s);
            if (kind == FE_TET_MASS) k_tet_atomic<FE_TET_MASS><<<g, TET_BLOCK, 0, s>>>(m->me, nme, m->q, w, p->map, values, p->nnz);
            else if (kind == FE_TET_WMASS) k_tet_atomic<FE_TET_WMASS><<<g, TET_BLOCK, 0, s>>>(m->me, nme, m->q, w, p->map, values, p->nnz);
            else k_tet_atomic<FE_TET_STIFF><<<g, TET_BLOCK, 0, s>>>(m->me, nme, m->q, w, p->map, values, p->nnz);
        }
        FE_LAUNCHED("k_tet_atomic");
        return FE_OK;
    }
    if (nme > 0) {
        FE_PROF("k_tet_stage", s);
        if (kind == FE_TET_MASS) k_tet_stage<FE_TET_MASS><<<g, TET_BLOCK, 0, s>>>(m->me, nme, m->q, w, p->kg);
        else if (kind == FE_TET_WMASS) k_tet_stage<FE_TET_WMASS><<<g, TET_BLOCK, 0, s>>>(m->me, nme, m->q, w, p->kg);
        else k_tet_stage<FE_TET_STIFF><<<g, TET_BLOCK, 0, s>>>(m->me, nme, m->q, w, p->kg);
    }
    FE_LAUNCHED("k_tet_stage");
    {
        FE_PROF("k_tet_rowsum", s);
        if (!p->n_long_host[1])
            k_tet_rowsum<RS_SHORT><<<fe_grid(m->nq, RS_BLOCK, 16), RS_BLOCK, 0, s>>>(p->vptr, p->row_ptr, m->nq, p->inc, p->islot, p->kg, values, 4 * (int64_t)nme);
        else
            k_tet_rowsum<RS_MAX><<<fe_grid(m->nq, RS_BLOCK, 8), RS_BLOCK, 0, s>>>(p->vptr, p->row_ptr, m->nq, p->inc, p->islot, p->kg, values, 4 * (int64_t)nme);
    }
    FE_LAUNCHED("k_tet_rowsum");
    if (p->n_long_host[0] > 0) {
        const size_t sm = (3 * (size_t)FE_TET_MAX_VALENCE + 1) * sizeof(double);
        { FE_PROF("k_tet_rowsum_long", s); k_tet_rowsum_long<<<fe_sm_count() * 8, 32, sm, s>>>(p->long_rows, p->n_long, p->vptr, p->row_ptr, p->inc, p->islot, p->kg, values); }
        FE_LAUNCHED("k_tet_rowsum_long");
    }
    return FE_OK;
}
