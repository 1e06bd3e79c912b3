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

// keep[k] = 1 if triangle k has a vertex in [r0, r1); used[v] = 1 for every vertex of a kept
// triangle and every owned vertex (used is zero on entry; threads that mark the same vertex write
// the same value). Every kept triangle is checked as in the mesh validation (ids in range,
// distinct, counter-clockwise: D > 0 in FP64 from coordinate differences); word: [0] OR of the
// problems, [1..3] the first bad triangle of each kind (global index). A triangle with an id out
// of range anywhere is reported, kept or not.
__global__ void k_part_select(const int32_t* __restrict__ me, int32_t nme, int32_t nq, const double* __restrict__ q,
                              int32_t r0, int32_t r1, int32_t* __restrict__ keep, int32_t* __restrict__ used,
                              int* __restrict__ word) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < r1; v += stride) used[v] = 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += stride) {
        const int32_t v0 = me[k], v1 = me[nme + k], v2 = me[2 * (int64_t)nme + k];
        const bool in = v0 >= 0 && v0 < nq && v1 >= 0 && v1 < nq && v2 >= 0 && v2 < nq;
        const bool mine = (v0 >= r0 && v0 < r1) || (v1 >= r0 && v1 < r1) || (v2 >= r0 && v2 < r1);
        keep[k] = in && mine;
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
            used[v0] = 1;
            used[v1] = 1;
            used[v2] = 1;
        }
        if (bad) {
            atomicOr(&word[0], bad);
            atomicMin(&word[bad == PART_RANGE ? 1 : bad == PART_REPEAT ? 2 : 3], (int)k);
        }
    }
}

// The kept triangles, in ascending order, into me_part [3][n_part] (pos = exclusive scan of
// keep), their vertices renumbered by loc (exclusive scan of used).
__global__ void k_part_compact(const int32_t* __restrict__ me, int32_t nme, const int32_t* __restrict__ keep,
                               const int32_t* __restrict__ pos, const int32_t* __restrict__ loc, int32_t n_part,
                               int32_t* __restrict__ me_part) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nme; k += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[k]) continue;
        const int64_t at = pos[k];
        me_part[at] = loc[me[k]];
        me_part[n_part + at] = loc[me[nme + k]];
        me_part[2 * (int64_t)n_part + at] = loc[me[2 * (int64_t)nme + k]];
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
    int32_t *me_tmp = nullptr, *keep = nullptr, *pos = nullptr, *used = nullptr, *loc = nullptr, *me_part = nullptr;
    int* word = nullptr;
    // frees are ordered on the stream after the kernels that read these arrays
    auto cleanup = [&]() {
        fe_free(q_tmp); fe_free(me_tmp); fe_free(keep); fe_free(pos); fe_free(used); fe_free(loc); fe_free(word);
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
    if (!st) st = fe_alloc_n(&keep, (size_t)nme + 1, "halo flags");
    if (!st) st = fe_alloc_n(&pos, (size_t)nme + 1, "halo positions");
    if (!st) st = fe_alloc_n(&used, (size_t)nq + 1, "part vertex flags");
    if (!st) st = fe_alloc_n(&loc, (size_t)nq + 1, "local vertex ids");
    if (!st) st = fe_alloc_n(&word, 4, "selection word");
    if (st) { cleanup(); return st; }
    // 1. select the triangles and the vertices; 2. number both by exclusive scans (the totals land
    // in pos[nme] and loc[nq]); one read-back of the word, the two totals and loc[row_begin]
    cudaError_t e = cudaMemsetAsync(word, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(word + 1, 0x7F, 3 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(used, 0, sizeof(int32_t) * ((size_t)nq + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(pos, 0, sizeof(int32_t), s);      // the totals when nme or nq is 0
    if (e == cudaSuccess) e = cudaMemsetAsync(loc, 0, sizeof(int32_t), s);
    const int64_t sel_n = nme > row_end - row_begin ? (int64_t)nme : (int64_t)row_end - row_begin;
    if (e == cudaSuccess && sel_n > 0) {
        { FE_PROF("k_part_select", s); k_part_select<<<fe_grid(sel_n, 256), 256, 0, s>>>(med, nme, nq, qd, row_begin, row_end, keep, used, word); }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { cleanup(); return fe_cuda_fail(e, "halo selection"); }
    if (nme > 0 && (st = fe_exclusive_scan(keep, pos, nme, s, nullptr))) { cleanup(); return st; }
    if (nq > 0 && (st = fe_exclusive_scan(used, loc, nq, s, nullptr))) { cleanup(); return st; }
    int host_word[4] = {0, 0, 0, 0};
    int32_t n_part = 0, n_loc = 0, loc0 = 0;
    e = cudaMemcpyAsync(host_word, word, sizeof host_word, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n_part, pos + nme, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n_loc, loc + nq, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&loc0, loc + row_begin, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { cleanup(); return fe_cuda_fail(e, "halo selection"); }
    if (host_word[0] & PART_RANGE) {
        cleanup();
        return fe_fail(FE_ERR_INDEX_RANGE, "triangle " + std::to_string(host_word[1]) + " has a vertex id outside [0, nq)");
    }
    if (host_word[0] & PART_REPEAT) {
        cleanup();
        return fe_fail(FE_ERR_DEGENERATE, "triangle " + std::to_string(host_word[2]) + " repeats a vertex");
    }
    if (host_word[0] & PART_ORIENT) {
        cleanup();
        return fe_fail(FE_ERR_ORIENTATION, "triangle " + std::to_string(host_word[3]) +
                                               " has signed area <= 0 (must be counter-clockwise)");
    }
    // 3. the kept triangles with local ids; the part as a mesh of its own (its connectivity passes
    // to the mesh, whose creation counts the valences the pattern build needs: every id was
    // checked above, so without a second check or read-back); its vertices' points and global ids
    if ((st = fe_alloc_n(&me_part, 3 * (size_t)n_part, "halo connectivity"))) { cleanup(); return st; }
    if (n_part > 0) {
        { FE_PROF("k_part_compact", s); k_part_compact<<<fe_grid(nme, 256), 256, 0, s>>>(med, nme, keep, pos, loc, n_part, me_part); }
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
    fe_pattern p = nullptr;
    fe_status st = fe_pattern_build_rows(m, stream, &p);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    const int32_t n = row_end - row_begin;
    const int32_t r0 = part ? row_begin - m->part0 + m->loc0 : row_begin;      // the window in the mesh's ids
    st = fe_alloc_n(&p->row_ptr_w, (size_t)n + 1, "window offsets");
    int32_t ends[2] = {0, 0};
    if (!st) {
        { FE_PROF("k_window_offsets", s); k_window_offsets<<<fe_grid((int64_t)n + 1, 256), 256, 0, s>>>(p->row_ptr, r0, n, p->row_ptr_w); }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[0], p->row_ptr + r0, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], p->row_ptr + r0 + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = fe_cuda_fail(e, "row window");
    }
    const int64_t nnz = (int64_t)ends[1] - ends[0];
    if (!st && part) {
        // the columns the caller sees carry global ids; the kernels keep reading the local ones
        st = fe_alloc_n(&p->col_idx_w, (size_t)nnz, "window columns");
        if (!st && nnz > 0) {
            { FE_PROF("k_window_columns", s); k_window_columns<<<fe_grid(nnz, 256), 256, 0, s>>>(p->col_idx + ends[0], nnz, m->l2g, p->col_idx_w); }
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = fe_cuda_fail(e, "window columns");
        }
    }
    if (st) { fe_pattern_destroy(p); return st; }
    p->row0 = r0;
    p->row1 = r0 + n;
    p->base_w = ends[0];
    p->n_rows = n;
    p->nnz = nnz;
    *out = p;
    return FE_OK;
}
