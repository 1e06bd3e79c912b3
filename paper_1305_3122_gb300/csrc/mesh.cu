// mesh.cu -- mesh handles: device copies of q and me, and validation of every triangle.
//
// Section 2 of the paper describes a mesh by q (vertex coordinates) and me (connectivity).
// The library keeps q as (x, y) pairs so that a vertex gather is one 16-byte load, and me in
// the caller's [3][nme] layout (coalesced per local vertex).
#include <atomic>

#include "internal.cuh"

static std::atomic<uint64_t> g_topology_counter{1};

uint64_t fe_next_topology_id() { return g_topology_counter.fetch_add(1); }

// q [2][nq] (x row, y row) -> q2 [nq] (x, y)
__global__ void k_pack_coords(const double* __restrict__ q, int32_t nq, double2* __restrict__ q2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x)
        q2[i] = make_double2(q[i], q[nq + i]);
}

// A part's coordinates from the global array: q [2][nq_global] -> q2 [nq], q2[i] = point l2g[i]
__global__ void k_pack_coords_part(const double* __restrict__ q, int32_t nq_global, const int32_t* __restrict__ l2g,
                                   int32_t nq, double2* __restrict__ q2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = l2g[i];
        q2[i] = make_double2(q[g], q[nq_global + g]);
    }
}

// Validation word layout: [0] = OR of error bits, [1] = first bad triangle (min), per kind.
enum { BAD_RANGE = 1, BAD_REPEAT = 2, BAD_ORIENT = 4 };

// Validation passes (mode bits): the connectivity alone, and the orientation (which needs the
// coordinates; its pass assumes ids already checked).
enum { VAL_TOPOLOGY = 1, VAL_ORIENT = 2 };

// Sign of D = (p1 - p0) x (p2 - p0) > 0, first from truncated-float coordinates; the float result is
// trusted when it exceeds a bound on its error (coordinate truncation 2^-23 |p|, float rounding of
// the differences and products), otherwise D is recomputed in FP64 from edge vectors
// v = p2 - p0, w = p0 - p1 as the oracle does.
__device__ __forceinline__ bool tri_positive(double2 p0, double2 p1, double2 p2) {
    float x0 = fe_trunc_float(p0.x), y0 = fe_trunc_float(p0.y);
    float ax = fe_trunc_float(p1.x) - x0, ay = fe_trunc_float(p1.y) - y0;
    float bx = fe_trunc_float(p2.x) - x0, by = fe_trunc_float(p2.y) - y0;
    float Df = ax * by - ay * bx;
    float M = fmaxf(fmaxf(fmaxf(fabsf(x0), fabsf(y0)), fmaxf(fabsf(ax), fabsf(ay))), fmaxf(fabsf(bx), fabsf(by)));
    float err = 3.0e-6f * M * (fabsf(ax) + fabsf(ay) + fabsf(bx) + fabsf(by));   // > 2^-19 bound
    if (fabsf(Df) > err && M < 1e18f && M > 1e-18f) return Df > 0.0f;
    double vx = p2.x - p0.x, vy = p2.y - p0.y, wx = p0.x - p1.x, wy = p0.y - p1.y;
    return vx * wy - wx * vy > 0.0;
}

__device__ __forceinline__ void report(int* __restrict__ word, int bad, int64_t k) {
    if (bad) {
        atomicOr(&word[0], bad);
        atomicMin(&word[bad == BAD_RANGE ? 1 : bad == BAD_REPEAT ? 2 : 3], (int)k);
    }
}

// Every triangle: vertex ids in range, three distinct vertices, counter-clockwise (tri_positive).
// Also counts each vertex's triangles (the row digit of the pattern build's counting sort), so a
// pattern build can skip that pass. One thread takes two consecutive triangles: a vertex they share
// (mesh generators list neighbouring triangles together; the two triangles of a cell share two) is
// counted with one atomic and its coordinates are loaded once. Every triangle's checks and report
// are its own.
__global__ void k_validate(const double2* __restrict__ q, int32_t nq, const int32_t* __restrict__ me,
                           int32_t nme, int* __restrict__ word, int32_t* __restrict__ deg, int mode) {
    const int64_t npair = ((int64_t)nme + 1) / 2;
    for (int64_t pi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pi < npair; pi += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k0 = 2 * pi, k1 = k0 + 1;
        const bool has1 = k1 < nme;
        int32_t v[3], u[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            v[a] = me[a * (int64_t)nme + k0];
            u[a] = has1 ? me[a * (int64_t)nme + k1] : 0;
        }
        const bool in0 = v[0] >= 0 && v[0] < nq && v[1] >= 0 && v[1] < nq && v[2] >= 0 && v[2] < nq;
        const bool in1 = has1 && u[0] >= 0 && u[0] < nq && u[1] >= 0 && u[1] < nq && u[2] >= 0 && u[2] < nq;
        // m[b]: the vertex of the first triangle equal to u[b] (-1: none, or not both in range)
        int m[3] = {-1, -1, -1};
        if (in0 && in1) {
#pragma unroll
            for (int b = 0; b < 3; b++)
#pragma unroll
                for (int a = 2; a >= 0; a--)
                    if (u[b] == v[a]) m[b] = a;
        }
        if (mode & VAL_TOPOLOGY) {
            if (in0) {
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const int c = 1 + (m[0] == a) + (m[1] == a) + (m[2] == a);
                    atomicAdd(&deg[v[a]], c);
                }
            }
            if (in1) {
#pragma unroll
                for (int b = 0; b < 3; b++)
                    if (m[b] < 0) atomicAdd(&deg[u[b]], 1);
            }
        }
        const bool rep0 = v[0] == v[1] || v[1] == v[2] || v[0] == v[2];
        const bool rep1 = u[0] == u[1] || u[1] == u[2] || u[0] == u[2];
        int bad0 = 0, bad1 = 0;
        if (!in0) bad0 = (mode & VAL_TOPOLOGY) ? BAD_RANGE : 0;
        else if (rep0) bad0 = (mode & VAL_TOPOLOGY) ? BAD_REPEAT : 0;
        if (has1) {
            if (!in1) bad1 = (mode & VAL_TOPOLOGY) ? BAD_RANGE : 0;
            else if (rep1) bad1 = (mode & VAL_TOPOLOGY) ? BAD_REPEAT : 0;
        }
        if (mode & VAL_ORIENT) {
            double2 pv[3], pu[3];
            const bool o0 = in0 && !rep0, o1 = in1 && !rep1;
            if (o0 || (in0 && in1)) {
#pragma unroll
                for (int a = 0; a < 3; a++) pv[a] = q[v[a]];
            }
            if (o1) {
#pragma unroll
                for (int b = 0; b < 3; b++) {                     // conditional selects: no local memory
                    if (m[b] < 0) pu[b] = q[u[b]];
                    else pu[b] = m[b] == 0 ? pv[0] : (m[b] == 1 ? pv[1] : pv[2]);
                }
            }
            if (o0 && !tri_positive(pv[0], pv[1], pv[2])) bad0 = BAD_ORIENT;
            if (o1 && !tri_positive(pu[0], pu[1], pu[2])) bad1 = BAD_ORIENT;
        }
        report(word, bad0, k0);
        if (has1) report(word, bad1, k1);
    }
}

static fe_status copy_in(void* dst, const void* src, size_t bytes, int ptr_kind, cudaStream_t s) {
    if (bytes == 0) return FE_OK;
    FE_CUDA(cudaMemcpyAsync(dst, src, bytes,
                            ptr_kind == FE_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    return FE_OK;
}

// q [2][n] with n = nq, or for a part the global nq (the part gathers its vertices' points)
static fe_status set_coords(fe_mesh m, const double* q, int ptr_kind, cudaStream_t s) {
    if (m->nq == 0) return FE_OK;
    const bool part = m->part1 >= 0;
    const int32_t n = part ? m->nq_global : m->nq;
    const double* qd = q;
    double* tmp = nullptr;
    if (ptr_kind == FE_PTR_HOST) {
        fe_status st = fe_alloc_n(&tmp, 2 * (size_t)n, "coordinate staging");
        if (st) return st;
        st = copy_in(tmp, q, 2 * (size_t)n * sizeof(double), ptr_kind, s);
        if (st) { fe_free(tmp); return st; }
        qd = tmp;
    }
    if (part) { FE_PROF("k_pack_coords_part", s); k_pack_coords_part<<<fe_grid(m->nq, 256), 256, 0, s>>>(qd, n, m->l2g, m->nq, m->q); }
    else { FE_PROF("k_pack_coords", s); k_pack_coords<<<fe_grid(m->nq, 256), 256, 0, s>>>(qd, m->nq, m->q); }
    cudaError_t e = cudaGetLastError();
    if (tmp) {
        cudaError_t e2 = cudaStreamSynchronize(s);
        fe_free(tmp);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return fe_cuda_fail(e, "k_pack_coords");
    return FE_OK;
}

extern "C" void fe_mesh_destroy(fe_mesh m) {
    if (!m) return;
    FeStreamScope scope(m->last_stream);
    fe_free(m->q);
    if (m->me_owned) fe_free(m->me);
    fe_free(m->err);
    fe_free(m->deg);
    fe_free(m->l2g);
    delete m;
}

extern "C" fe_status fe_mesh_create(int32_t nq, int32_t nme, const double* q, const int32_t* me,
                                    int ptr_kind, fe_stream stream, fe_mesh* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (nq < 0 || nme < 0) return fe_fail(FE_ERR_INVALID_ARG, "nq and nme must be >= 0");
    if ((nq > 0 && !q) || (nme > 0 && !me)) return fe_fail(FE_ERR_INVALID_ARG, "q or me is null");
    if (ptr_kind != FE_PTR_HOST && ptr_kind != FE_PTR_DEVICE && ptr_kind != FE_PTR_DEVICE_BORROW)
        return fe_fail(FE_ERR_INVALID_ARG, "bad ptr_kind");
    const bool borrow = ptr_kind == FE_PTR_DEVICE_BORROW;
    if (borrow) ptr_kind = FE_PTR_DEVICE;
    if ((int64_t)nme * 9 >= INT32_MAX)
        return fe_fail(FE_ERR_LIMIT, "9*nme must be < 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    FeStreamScope scope(s);
    fe_mesh m = new fe_mesh_s();
    m->last_stream = s;
    m->nq = nq;
    m->nme = nme;
    m->topology_id = fe_next_topology_id();
    fe_status st = fe_alloc_n(&m->q, (size_t)nq, "mesh coordinates");
    if (borrow) {
        m->me = const_cast<int32_t*>(me);
        m->me_owned = false;
    } else {
        if (!st) st = fe_alloc_n(&m->me, 3 * (size_t)nme, "mesh connectivity");
        if (!st) st = copy_in(m->me, me, 3 * (size_t)nme * sizeof(int32_t), ptr_kind, s);
    }
    if (!st) st = fe_alloc_n(&m->err, 4, "mesh error word");
    if (!st) st = fe_alloc_n(&m->deg, (size_t)nq + 1, "vertex valences");
    if (!st) st = set_coords(m, q, ptr_kind, s);
    if (st) { fe_mesh_destroy(m); return st; }
    // error word: [0] = 0, [1..3] = 0x7F7F7F7F (above any triangle index: "none yet" for atomicMin)
    int word[4];
    cudaError_t e = cudaMemsetAsync(m->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->err + 1, 0x7F, 3 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->deg, 0, sizeof(int32_t) * ((size_t)nq + 1), s);
    if (e == cudaSuccess && nme > 0) {
        { FE_PROF("k_validate", s); k_validate<<<fe_grid(((int64_t)nme + 1) / 2, 256, 16), 256, 0, s>>>(m->q, nq, m->me, nme, m->err, m->deg, VAL_TOPOLOGY | VAL_ORIENT); }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(word, m->err, sizeof word, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, sizeof(int) * 4, s);
    if (e != cudaSuccess) { fe_mesh_destroy(m); return fe_cuda_fail(e, "mesh validation"); }
    if (word[0] & BAD_RANGE) {
        fe_mesh_destroy(m);
        return fe_fail(FE_ERR_INDEX_RANGE, "triangle " + std::to_string(word[1]) + " has a vertex id outside [0, nq)");
    }
    if (word[0] & BAD_REPEAT) {
        fe_mesh_destroy(m);
        return fe_fail(FE_ERR_DEGENERATE, "triangle " + std::to_string(word[2]) + " repeats a vertex");
    }
    if (word[0] & BAD_ORIENT) {
        fe_mesh_destroy(m);
        return fe_fail(FE_ERR_ORIENTATION, "triangle " + std::to_string(word[3]) +
                                               " has signed area <= 0 (must be counter-clockwise)");
    }
    *out = m;
    return FE_OK;
}

// ------------------------------------------------------------------ staged creation
//
// The one-shot host call (fe_assemble_stiff_wmass_host) uploads the connectivity first and builds
// the pattern while the coordinates are still on their way: the mesh is created from device
// connectivity (ownership passes to the mesh) and checked for range, repeats and valences, which
// is all the pattern build needs; fe_mesh_attach_coords then packs the coordinates and queues the
// orientation check, whose result fe_mesh_orientation_status reads from the validation word.

fe_status fe_mesh_create_topology(int32_t nq, int32_t nme, int32_t* me_dev, cudaStream_t s, fe_mesh* out,
                                 bool checked) {
    *out = nullptr;
    fe_mesh m = new fe_mesh_s();
    m->last_stream = s;
    m->nq = nq;
    m->nme = nme;
    m->topology_id = fe_next_topology_id();
    m->me = me_dev;
    m->me_owned = true;
    fe_status st = fe_alloc_n(&m->q, (size_t)nq, "mesh coordinates");
    if (!st) st = fe_alloc_n(&m->err, 4, "mesh error word");
    if (!st) st = fe_alloc_n(&m->deg, (size_t)nq + 1, "vertex valences");
    if (st) { fe_mesh_destroy(m); return st; }
    int word[4];
    cudaError_t e = cudaMemsetAsync(m->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->err + 1, 0x7F, 3 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->deg, 0, sizeof(int32_t) * ((size_t)nq + 1), s);
    if (e == cudaSuccess && nme > 0) {
        { FE_PROF("k_validate", s); k_validate<<<fe_grid(((int64_t)nme + 1) / 2, 256, 16), 256, 0, s>>>(m->q, nq, m->me, nme, m->err, m->deg, VAL_TOPOLOGY); }
        e = cudaGetLastError();
    }
    if (!checked) {
        if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, sizeof(int) * 4, s);
        if (e != cudaSuccess) { fe_mesh_destroy(m); return fe_cuda_fail(e, "valence count"); }
        *out = m;
        return FE_OK;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(word, m->err, sizeof word, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { fe_mesh_destroy(m); return fe_cuda_fail(e, "mesh validation"); }
    if (word[0] & BAD_RANGE) {
        fe_mesh_destroy(m);
        return fe_fail(FE_ERR_INDEX_RANGE, "triangle " + std::to_string(word[1]) + " has a vertex id outside [0, nq)");
    }
    if (word[0] & BAD_REPEAT) {
        fe_mesh_destroy(m);
        return fe_fail(FE_ERR_DEGENERATE, "triangle " + std::to_string(word[2]) + " repeats a vertex");
    }
    *out = m;
    return FE_OK;
}

fe_status fe_mesh_attach_coords(fe_mesh m, const double* q_dev, cudaStream_t s) {
    const int32_t nq = m->nq, nme = m->nme;
    if (nq > 0) { FE_PROF("k_pack_coords", s); k_pack_coords<<<fe_grid(nq, 256), 256, 0, s>>>(q_dev, nq, m->q); }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(m->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->err + 1, 0x7F, 3 * sizeof(int), s);
    if (e == cudaSuccess && nme > 0) {
        { FE_PROF("k_validate", s); k_validate<<<fe_grid(((int64_t)nme + 1) / 2, 256, 16), 256, 0, s>>>(m->q, nq, m->me, nme, m->err, m->deg, VAL_ORIENT); }
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fe_cuda_fail(e, "orientation check");
    return FE_OK;
}

fe_status fe_mesh_orientation_status(const int word[4]) {
    if (word[0] & BAD_ORIENT)
        return fe_fail(FE_ERR_ORIENTATION, "triangle " + std::to_string(word[3]) +
                                               " has signed area <= 0 (must be counter-clockwise)");
    return FE_OK;
}

extern "C" fe_status fe_mesh_set_coords(fe_mesh m, const double* q, int ptr_kind, fe_stream stream) {
    FE_RANGE(__func__);
    if (!m || (m->nq > 0 && !q)) return fe_fail(FE_ERR_INVALID_ARG, "null mesh or q");
    if (ptr_kind == FE_PTR_DEVICE_BORROW) ptr_kind = FE_PTR_DEVICE;
    if (ptr_kind != FE_PTR_HOST && ptr_kind != FE_PTR_DEVICE) return fe_fail(FE_ERR_INVALID_ARG, "bad ptr_kind");
    FeStreamScope scope((cudaStream_t)stream);
    m->last_stream = (cudaStream_t)stream;
    return set_coords(m, q, ptr_kind, (cudaStream_t)stream);
}

extern "C" fe_status fe_mesh_check(fe_mesh m, fe_stream stream) {
    FE_RANGE(__func__);
    if (!m) return fe_fail(FE_ERR_INVALID_ARG, "null mesh");
    cudaStream_t s = (cudaStream_t)stream;
    int word = 0;
    FE_CUDA(cudaMemcpyAsync(&word, m->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    FE_CUDA(cudaStreamSynchronize(s));
    FE_CUDA(cudaMemsetAsync(m->err, 0, sizeof(int), s));
    // a value out of the double-float range is reported first: it also makes areas look <= 0
    if (word & 2)
        return fe_fail(FE_ERR_LIMIT, "an edge-vector component or a weight is outside the double-float range "
                                     "(nonzero magnitudes must lie in [2^-74, 2^128))");
    if (word & 1) return fe_fail(FE_ERR_ORIENTATION, "an assembly call met a triangle with signed area <= 0");
    return FE_OK;
}

extern "C" fe_status fe_mesh_info(fe_mesh m, int32_t* nq, int32_t* nme) {
    if (!m) return fe_fail(FE_ERR_INVALID_ARG, "null mesh");
    if (nq) *nq = m->part1 >= 0 ? m->nq_global : m->nq;     // a part: the global id space
    if (nme) *nme = m->nme;
    return FE_OK;
}
