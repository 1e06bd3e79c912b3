// partition.cu -- one mesh over several ranks by rows, with redundant halo triangles.
//
// Each row of the global matrix is summed from the triangles that contain its vertex (the
// structural sum of Sections 5-6), so a rank that owns the rows [row_begin, row_end) needs exactly
// the triangles with at least one vertex in that range. Triangles shared by two ranks' vertices
// are held, and their element matrices computed, by both ("halo" triangles), so assembly needs no
// exchange of values: each rank writes its own rows, in global column ids, and the ranks' row
// blocks concatenated are the whole matrix. Nothing here communicates; how ranks are launched
// and how their row blocks are collected is up to the caller.
//
//   fe_mesh_create_part    keeps the triangles of a global mesh that touch the owned rows
//                          (selected and compacted on the device, in ascending triangle order),
//                          checks every triangle that it keeps, and numbers the part's vertices
//                          locally (the rank of each global id among them), so that everything
//                          after it -- valences, the pattern, the vertex records -- is sized by
//                          the part, not by the global mesh.
//   fe_pattern_build_part  the CSR rows [row_begin, row_end) of a part or of a whole mesh; a
//                          part's window maps its columns back to global ids.
//
// The local numbering keeps the order of the global ids, so each row's columns and its triangle
// fan come out in the same order as in the whole mesh, and the row-owner assembly gives each row
// the same bits.
#include <string>

#include "internal.cuh"

namespace {

enum { PART_RANGE = 1, PART_REPEAT = 2, PART_ORIENT = 4 };

// Selection word: [0] OR of the problems, [1] the kept triangles, [2..4] the first bad triangle
// of each kind (global index).
enum { W_BITS = 0, W_KEPT = 1, W_FIRST = 2 };

// Triangles are taken in tiles of PT_TILE: thread t of tile b holds triangles
// b * PT_TILE + j * PT_BLOCK + t, j < PT_ITEMS (coalesced loads for each j).
constexpr int PT_BLOCK = 256, PT_ITEMS = 8, PT_TILE = PT_BLOCK * PT_ITEMS, PT_WARPS = PT_BLOCK / 32;

__device__ __forceinline__ bool ids_in(int32_t v0, int32_t v1, int32_t v2, int32_t nq) {
    return v0 >= 0 && v0 < nq && v1 >= 0 && v1 < nq && v2 >= 0 && v2 < nq;
}

__device__ __forceinline__ bool touches(int32_t v0, int32_t v1, int32_t v2, int32_t r0, int32_t r1) {
    return (v0 >= r0 && v0 < r1) || (v1 >= r0 && v1 < r1) || (v2 >= r0 && v2 < r1);
}

// A triangle is kept when its ids are in range and one of its vertices is owned. Per tile: the
// number of kept triangles (tile_cnt, and their total in word[W_KEPT]); used[v] = 1 for every
// vertex of a kept triangle and every owned vertex (used is zero on entry; threads that mark the
// same vertex write the same value). Every kept triangle is checked as in the mesh validation
// (distinct ids, counter-clockwise: D > 0 in FP64 from coordinate differences); a triangle with
// an id out of range anywhere is reported, kept or not.
__global__ void __launch_bounds__(PT_BLOCK) k_part_count(const int32_t* __restrict__ me, int32_t nme, int32_t nq,
                                                         const double* __restrict__ q, int32_t r0, int32_t r1,
                                                         int32_t* __restrict__ used, int32_t* __restrict__ tile_cnt,
                                                         int* __restrict__ word) {
    __shared__ int red[PT_WARPS];
    for (int64_t v = r0 + blockIdx.x * (int64_t)PT_BLOCK + threadIdx.x; v < r1; v += (int64_t)gridDim.x * PT_BLOCK)
        used[v] = 1;
    const int64_t base = (int64_t)blockIdx.x * PT_TILE;
    int32_t tri[PT_ITEMS][3];                         // all loads issued before any is used
#pragma unroll
    for (int j = 0; j < PT_ITEMS; j++) {
        const int64_t k = base + j * PT_BLOCK + threadIdx.x;
        tri[j][0] = tri[j][1] = tri[j][2] = 0;
        if (k < nme) {
            tri[j][0] = me[k];
            tri[j][1] = me[nme + k];
            tri[j][2] = me[2 * (int64_t)nme + k];
        }
    }
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < PT_ITEMS; j++) {
        const int64_t k = base + j * PT_BLOCK + threadIdx.x;
        if (k >= nme) break;
        const int32_t v0 = tri[j][0], v1 = tri[j][1], v2 = tri[j][2];
        const bool in = ids_in(v0, v1, v2, nq);
        const bool mine = touches(v0, v1, v2, r0, r1);
        int bad = 0;
        if (!in) bad = PART_RANGE;
        else if (mine && (v0 == v1 || v1 == v2 || v0 == v2)) bad = PART_REPEAT;
        else if (mine) {
            const double x0 = q[v0], y0 = q[nq + v0];
            const double vx = q[v2] - x0, vy = q[nq + v2] - y0;          // p2 - p0
            const double wx = x0 - q[v1], wy = y0 - q[nq + v1];          // p0 - p1
            if (!(vx * wy - wx * vy > 0.0)) bad = PART_ORIENT;
        }
        if (in && mine) {
            cnt++;
            used[v0] = 1;
            used[v1] = 1;
            used[v2] = 1;
        }
        if (bad) {
            atomicOr(&word[W_BITS], bad);
            atomicMin(&word[W_FIRST + (bad == PART_RANGE ? 0 : bad == PART_REPEAT ? 1 : 2)], (int)k);
        }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0 && base < nme) {
        int t = 0;
        for (int w = 0; w < PT_WARPS; w++) t += red[w];
        tile_cnt[blockIdx.x] = t;
        if (t) atomicAdd(&word[W_KEPT], t);
    }
}

// The kept triangles, in ascending order, into me_part [3][n_part], their vertices renumbered by
// loc (exclusive scan of used). A tile's first place is the sum of the counts of the tiles before
// it; inside the tile, kept triangles are ranked by ballots in the order (j, warp, lane), which is
// the order of their indices.
__global__ void __launch_bounds__(PT_BLOCK) k_part_place(const int32_t* __restrict__ me, int32_t nme, int32_t nq,
                                                         int32_t r0, int32_t r1, const int32_t* __restrict__ tile_cnt,
                                                         const int32_t* __restrict__ loc, int32_t n_part,
                                                         int32_t* __restrict__ me_part) {
    __shared__ int red[PT_WARPS];
    __shared__ int at0[PT_ITEMS * PT_WARPS];
    if (tile_cnt[blockIdx.x] == 0) return;            // most tiles of a spatially compact part
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int a = 0;
    for (int t = threadIdx.x; t < (int)blockIdx.x; t += PT_BLOCK) a += tile_cnt[t];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[wid] = a;
    const int64_t base = (int64_t)blockIdx.x * PT_TILE;
    int32_t v[PT_ITEMS][3];
    int pre[PT_ITEMS];
    bool kp[PT_ITEMS];
#pragma unroll
    for (int j = 0; j < PT_ITEMS; j++) {
        const int64_t k = base + j * PT_BLOCK + threadIdx.x;
        kp[j] = false;
        v[j][0] = v[j][1] = v[j][2] = 0;
        if (k < nme) {
            v[j][0] = me[k];
            v[j][1] = me[nme + k];
            v[j][2] = me[2 * (int64_t)nme + k];
            kp[j] = ids_in(v[j][0], v[j][1], v[j][2], nq) && touches(v[j][0], v[j][1], v[j][2], r0, r1);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, kp[j]);
        pre[j] = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) at0[j * PT_WARPS + wid] = __popc(bal);
    }
    __syncthreads();
    if (wid == 0) {                                   // exclusive scan of the 64 counts, two per lane
        static_assert(PT_ITEMS * PT_WARPS == 64, "two counts per lane");
        int off = lane < PT_WARPS ? red[lane] : 0;
        for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
        const int c0 = at0[2 * lane], c1 = at0[2 * lane + 1];
        int x = c0 + c1;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        const int ex = off + x - c0 - c1;
        at0[2 * lane] = ex;
        at0[2 * lane + 1] = ex + c0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PT_ITEMS; j++) {
        if (!kp[j]) continue;
        const int64_t at = at0[j * PT_WARPS + wid] + pre[j];
        me_part[at] = loc[v[j][0]];
        me_part[n_part + at] = loc[v[j][1]];
        me_part[2 * (int64_t)n_part + at] = loc[v[j][2]];
    }
}

// The part's vertices: l2g[loc[v]] = v and their points q2[loc[v]] = (x, y) for every used v.
__global__ void k_part_vertices(const double* __restrict__ q, int32_t nq, const int32_t* __restrict__ used,
                                const int32_t* __restrict__ loc, int32_t* __restrict__ l2g, double2* __restrict__ q2) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nq; v += (int64_t)gridDim.x * blockDim.x) {
        if (!used[v]) continue;
        const int32_t l = loc[v];
        l2g[l] = (int32_t)v;
        q2[l] = make_double2(q[v], q[nq + v]);
    }
}

// The window's offsets from 0: out[t] = row_ptr[r0 + t] - row_ptr[r0], t = 0 .. n.
__global__ void k_window_offsets(const int32_t* __restrict__ row_ptr, int32_t r0, int32_t n, int32_t* __restrict__ out) {
    const int32_t base = row_ptr[r0];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t <= n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = row_ptr[r0 + t] - base;
}

// A part's window columns in the global numbering: out[e] = l2g[col[e]].
__global__ void k_window_columns(const int32_t* __restrict__ col, int64_t nnz, const int32_t* __restrict__ l2g,
                                 int32_t* __restrict__ out) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = l2g[col[e]];
}

}  // namespace

extern "C" fe_status fe_mesh_create_part(int32_t nq, int32_t nme, const double* q, const int32_t* me, int ptr_kind,
                                         int32_t row_begin, int32_t row_end, fe_stream stream, fe_mesh* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (nq < 0 || nme < 0) return fe_fail(FE_ERR_INVALID_ARG, "nq and nme must be >= 0");
    if ((nq > 0 && !q) || (nme > 0 && !me)) return fe_fail(FE_ERR_INVALID_ARG, "q or me is null");
    if (ptr_kind == FE_PTR_DEVICE_BORROW) ptr_kind = FE_PTR_DEVICE;
    if (ptr_kind != FE_PTR_HOST && ptr_kind != FE_PTR_DEVICE) return fe_fail(FE_ERR_INVALID_ARG, "bad ptr_kind");
    if (row_begin < 0 || row_end < row_begin || row_end > nq)
        return fe_fail(FE_ERR_INVALID_ARG, "owned rows must satisfy 0 <= row_begin <= row_end <= nq");
    if ((int64_t)nme * 9 >= INT32_MAX) return fe_fail(FE_ERR_LIMIT, "9*nme must be < 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    const bool host = ptr_kind == FE_PTR_HOST;
    double* q_tmp = nullptr;
    int32_t *me_tmp = nullptr, *tile_cnt = nullptr, *used = nullptr, *loc = nullptr, *me_part = nullptr;
    int* word = nullptr;
    // frees are ordered on the stream after the kernels that read these arrays
    auto cleanup = [&]() {
        fe_free(q_tmp); fe_free(me_tmp); fe_free(tile_cnt); fe_free(used); fe_free(loc); fe_free(word);
    };
    fe_status st = FE_OK;
    const double* qd = q;
    const int32_t* med = me;
    if (host) {
        st = fe_alloc_n(&q_tmp, 2 * (size_t)nq, "coordinate staging");
        if (!st) st = fe_alloc_n(&me_tmp, 3 * (size_t)nme, "connectivity staging");
        cudaError_t ce = cudaSuccess;
        if (!st && nq > 0) ce = cudaMemcpyAsync(q_tmp, q, 2 * sizeof(double) * nq, cudaMemcpyHostToDevice, s);
        if (!st && ce == cudaSuccess && nme > 0)
            ce = cudaMemcpyAsync(me_tmp, me, 3 * sizeof(int32_t) * nme, cudaMemcpyHostToDevice, s);
        if (!st && ce != cudaSuccess) st = fe_cuda_fail(ce, "mesh upload");
        qd = q_tmp;
        med = me_tmp;
    }
    const int64_t ntiles = ((int64_t)nme + PT_TILE - 1) / PT_TILE;
    if (!st) st = fe_alloc_n(&tile_cnt, (size_t)ntiles + 1, "halo tile counts");
    if (!st) st = fe_alloc_n(&used, (size_t)nq + 1, "part vertex flags");
    if (!st) st = fe_alloc_n(&loc, (size_t)nq + 1, "local vertex ids");
    if (!st) st = fe_alloc_n(&word, 8, "selection word");
    if (st) { cleanup(); return st; }
    // 1. count the kept triangles per tile and mark the part's vertices; 2. number the vertices by
    // an exclusive scan (its total lands in loc[nq]); one read-back of the word, the vertex total
    // and loc[row_begin]; 3. place the kept triangles
    cudaError_t e = cudaMemsetAsync(word, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(word + W_FIRST, 0x7F, 3 * sizeof(int), s);
    if (e == cudaSuccess && nq > 0) e = cudaMemsetAsync(used, 0, sizeof(int32_t) * (size_t)nq, s);
    const int64_t owned = (int64_t)row_end - row_begin;
    const int64_t grid = ntiles > 0 ? ntiles : (owned > 0 ? 1 : 0);
    if (e == cudaSuccess && grid > 0) {
        { FE_PROF("k_part_count", s); k_part_count<<<(unsigned)grid, PT_BLOCK, 0, s>>>(med, nme, nq, qd, row_begin, row_end, used, tile_cnt, word); }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { cleanup(); return fe_cuda_fail(e, "halo selection"); }
    if (nq > 0 && (st = fe_exclusive_scan(used, loc, nq, s, nullptr))) { cleanup(); return st; }
    int host_word[5] = {0, 0, 0, 0, 0};
    int32_t n_loc = 0, loc0 = 0;
    e = cudaMemcpyAsync(host_word, word, sizeof host_word, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nq > 0) e = cudaMemcpyAsync(&n_loc, loc + nq, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && nq > 0) e = cudaMemcpyAsync(&loc0, loc + row_begin, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cleanup(); return fe_cuda_fail(e, "halo selection"); }
    if (host_word[W_BITS] & PART_RANGE) {
        cleanup();
        return fe_fail(FE_ERR_INDEX_RANGE, "triangle " + std::to_string(host_word[W_FIRST]) + " has a vertex id outside [0, nq)");
    }
    if (host_word[W_BITS] & PART_REPEAT) {
        cleanup();
        return fe_fail(FE_ERR_DEGENERATE, "triangle " + std::to_string(host_word[W_FIRST + 1]) + " repeats a vertex");
    }
    if (host_word[W_BITS] & PART_ORIENT) {
        cleanup();
        return fe_fail(FE_ERR_ORIENTATION, "triangle " + std::to_string(host_word[W_FIRST + 2]) +
                                               " has signed area <= 0 (must be counter-clockwise)");
    }
    const int32_t n_part = host_word[W_KEPT];
    // the part as a mesh of its own: its connectivity passes to the mesh, whose creation counts the
    // valences the pattern build needs (every id was checked above, so without a second check or
    // read-back); then its vertices' points and global ids
    if ((st = fe_alloc_n(&me_part, 3 * (size_t)n_part, "halo connectivity"))) { cleanup(); return st; }
    if (n_part > 0) {
        { FE_PROF("k_part_place", s); k_part_place<<<(unsigned)ntiles, PT_BLOCK, 0, s>>>(med, nme, nq, row_begin, row_end, tile_cnt, loc, n_part, me_part); }
        e = cudaGetLastError();
        if (e != cudaSuccess) { fe_free(me_part); cleanup(); return fe_cuda_fail(e, "halo compaction"); }
    }
    fe_mesh m = nullptr;
    if ((st = fe_mesh_create_topology(n_loc, n_part, me_part, s, &m, false))) { cleanup(); return st; }
    if ((st = fe_alloc_n(&m->l2g, (size_t)n_loc, "local-to-global vertex ids"))) { cleanup(); fe_mesh_destroy(m); return st; }
    if (n_loc > 0) {
        { FE_PROF("k_part_vertices", s); k_part_vertices<<<fe_grid(nq, 256), 256, 0, s>>>(qd, nq, used, loc, m->l2g, m->q); }
        e = cudaGetLastError();
        if (e != cudaSuccess) { cleanup(); fe_mesh_destroy(m); return fe_cuda_fail(e, "part vertices"); }
    }
    cleanup();
    m->part0 = row_begin;
    m->part1 = row_end;
    m->nq_global = nq;
    m->loc0 = loc0;
    *out = m;
    return FE_OK;
}

extern "C" fe_status fe_pattern_build_part(fe_mesh m, int32_t row_begin, int32_t row_end, fe_stream stream,
                                           fe_pattern* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (!m) return fe_fail(FE_ERR_INVALID_ARG, "null mesh");
    const bool part = m->part1 >= 0;
    const int32_t lo = part ? m->part0 : 0, hi = part ? m->part1 : m->nq;
    if (row_begin < lo || row_end < row_begin || row_end > hi)
        return fe_fail(FE_ERR_INVALID_ARG, "the row window must lie in [0, nq) and, for a part, in its owned rows");
    const int32_t n = row_end - row_begin;
    const int32_t r0 = part ? row_begin - m->part0 + m->loc0 : row_begin;      // the window in the mesh's ids
    fe_pattern p = nullptr;
    fe_status st = fe_pattern_build_rows(m, r0, r0 + n, stream, &p);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    st = fe_alloc_n(&p->row_ptr_w, (size_t)n + 1, "window offsets");
    if (!st) {
        { FE_PROF("k_window_offsets", s); k_window_offsets<<<fe_grid((int64_t)n + 1, 256), 256, 0, s>>>(p->row_ptr, r0, n, p->row_ptr_w); }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = fe_cuda_fail(e, "row window");
    }
    if (!st && part) {
        // the columns the caller sees carry global ids; the kernels keep reading the local ones
        st = fe_alloc_n(&p->col_idx_w, (size_t)p->nnz, "window columns");
        if (!st && p->nnz > 0) {
            { FE_PROF("k_window_columns", s); k_window_columns<<<fe_grid(p->nnz, 256), 256, 0, s>>>(p->col_idx + p->base_w, p->nnz, m->l2g, p->col_idx_w); }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = fe_cuda_fail(e, "window columns");
        }
    }
    if (st) {
        cudaStreamSynchronize(s);
        fe_pattern_destroy(p);
        return st;
    }
    *out = p;
    return FE_OK;
}
