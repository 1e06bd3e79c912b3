// internal.cuh -- shared declarations of the CUDA library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <type_traits>

#include "../../include/feasm.h"

// ------------------------------------------------------------------------ handles

struct fe_mesh_s {
    int32_t nq = 0, nme = 0;
    double2* q = nullptr;       // [nq] (x, y) pairs: one 16-byte load per vertex gather
    int32_t* me = nullptr;      // [3][nme], the caller's layout
    bool me_owned = true;       // false: the caller's device array, used in place
    int32_t* deg = nullptr;     // [nq + 1] triangles per vertex (counted during validation)
    int* err = nullptr;         // device error word: bit 0 = a triangle with signed area <= 0,
                                // bit 1 = a value outside the double-float range (see ff.cuh)
    uint64_t topology_id = 0;   // identifies the connectivity (patterns remember it)
    int32_t part0 = 0, part1 = -1;        // a rank's share of a row partition: owned rows [part0, part1)
                                          // of the global numbering (part1 < 0: a whole mesh)
    // A part numbers its vertices locally: local id = rank of the global id among the part's
    // vertices (those of its triangles and its owned rows), so the order of ids is kept and the
    // owned rows are the contiguous local ids [loc0, loc0 + part1 - part0). nq, q, me and deg
    // are local; every id the calls take or return is global.
    int32_t* l2g = nullptr;               // [nq] global id of each local vertex (parts only)
    int32_t nq_global = 0;                // the global mesh's nq (parts only)
    int32_t loc0 = 0;                     // local id of the first owned row (parts only)
    cudaStream_t last_stream = nullptr;   // frees are ordered on the last stream that used the handle
};

struct fe_pattern_s {
    int dofs = 1;
    int flags = 0;
    int32_t nq = 0, nme = 0;
    uint64_t topology_id = 0;
    int64_t n_rows = 0, nnz = 0;          // of the returned (possibly block-expanded) matrix
    int64_t nnz_scalar = 0;
    // scalar pattern (always)
    int32_t* row_ptr = nullptr;           // [nq + 1]
    int32_t* col_idx = nullptr;           // [nnz_scalar]
    int32_t* map = nullptr;               // [9 nme]: map[9k + 3 jl + il] = position of (me[il][k], me[jl][k])
    // block-expanded pattern (dofs == 2)
    int32_t* row_ptr2 = nullptr;          // [2 nq + 1]
    int32_t* col_idx2 = nullptr;          // [4 nnz_scalar]
    // FE_PATTERN_GATHER
    int32_t* seg_ptr = nullptr;           // [nnz_scalar + 1] into perm
    int32_t* perm = nullptr;              // [9 nme] contribution ids c, grouped by non-zero, ascending c
    int32_t* vptr = nullptr;              // [nq + 1] vertex -> triangle lists
    int32_t* vel = nullptr;               // [3 nme] entries 3k + a (triangle k, local vertex a), ascending k
    double* kg = nullptr;                 // staging of element values: 2 x 9 nme (dofs 1) or 36 nme (dofs 2)
    // row-owner assembly (always)
    int2* fan = nullptr;                  // [3 nme] per vertex: simple rows, neighbours in fan order
                                          // (vertex, column position); general rows, sorted (j, l) pairs
    int2* hdr = nullptr;                  // [nq] simple rows: (last neighbour, pos_self | pos_last << 14 |
                                          // kind << 28), kind 0 closed / 1 open; kind 2 = general row
    int32_t* gen_rows = nullptr;          // general rows (assembled one block per row)
    int32_t n_gen = 0;
    // row window (fe_pattern_build_part): the pattern exposes rows [row0, row1) only; row1 < 0: all
    int32_t row0 = 0, row1 = -1;
    int32_t* row_ptr_w = nullptr;         // [row1 - row0 + 1] the window's offsets, from 0
    int64_t base_w = 0;                   // row_ptr[row0]: the window's first entry in the full arrays
    int32_t* col_idx_w = nullptr;         // a part's window: its column ids in the global numbering
    cudaStream_t last_stream = nullptr;
};

// longest triangle fan a simple row may have (rows with more go to the general path)
constexpr int FE_FAN_MAX = 8;

// Tetrahedral (3-D P1) meshes and patterns (tet.cu).
struct fe_tet_mesh_s {
    int32_t nq = 0, nme = 0;
    double4_32a* q = nullptr;   // [nq] (x, y, z, 0): one 32-byte record per vertex gather
    int32_t* me = nullptr;      // [4][nme], the caller's layout
    bool me_owned = true;
    int32_t* deg = nullptr;     // [nq + 1] tetrahedra per vertex (counted during validation)
    int* err = nullptr;         // [4] validation word
    uint64_t topology_id = 0;
    cudaStream_t last_stream = nullptr;
};

struct fe_tet_pattern_s {
    int flags = 0;
    int32_t nq = 0, nme = 0;
    uint64_t topology_id = 0;
    int64_t nnz = 0;
    int32_t* row_ptr = nullptr;           // [nq + 1]
    int32_t* col_idx = nullptr;           // [nnz]
    int32_t* map = nullptr;               // [16 nme]: map[16k + 4 il + jl] = position of (me[il][k], me[jl][k])
    // FE_PATTERN_GATHER: each row's incidences in ascending element order and the staging buffer
    int32_t* vptr = nullptr;              // [nq + 1] start of row i's incidences
    int32_t* inc = nullptr;               // [4 nme] keys 4k + a (row i = me[a][k]), ascending within a row
    uint2* islot = nullptr;               // [4 nme] in-row positions of columns jl = 0..3, 16 bits each
    int32_t* long_rows = nullptr;         // [nq + 1] rows with more columns than one thread sums
    int32_t* n_long = nullptr;            // [2] their number, and 1 if a row is longer than 16 (device)
    int32_t n_long_host[2] = {0, 0};
    double* kg = nullptr;                 // [16 nme] staged element values
    // FE_TET_PATTERN_ELAS: the 3-D elasticity structure (3 x 3 blocks of the scalar one)
    int32_t* row_ptr3 = nullptr;          // [3 nq + 1]
    int32_t* col_idx3 = nullptr;          // [9 nnz]
    cudaStream_t last_stream = nullptr;
};

// Row sums of the tetrahedral ordered variants: the longest row (in scalar columns) summed by one
// thread, and the smaller accumulator count used when no row is longer. The pattern build lists
// the rows above the first and flags any row above the second.
constexpr int FE_TET_RS_MAX = 32;
constexpr int FE_TET_RS_SHORT = 16;

// Expands a built scalar tetrahedral pattern into the 3-D elasticity structure (tetelas.cu).
fe_status fe_tet_elas_structure(fe_tet_pattern p, cudaStream_t s);

// P2 (quadratic) triangle patterns (p2.cu).
struct fe_p2_pattern_s {
    int32_t nq = 0, nme = 0;
    int64_t ne = 0;                       // edges (dofs nq .. nq + ne - 1)
    int32_t ndof = 0;
    uint64_t topology_id = 0;
    int64_t nnz = 0;
    int32_t* row_ptr = nullptr;           // [ndof + 1]
    int32_t* col_idx = nullptr;           // [nnz]
    int32_t* edof = nullptr;              // [nme][6] element dofs (vertices, then edges (0,1), (1,2), (2,0))
    int32_t* map = nullptr;               // [36 nme] map[36k + 6 il + jl] = position of (edof[k][il], edof[k][jl])
    // FE_PATTERN_GATHER: each row's incidences in ascending element order and the staging buffer
    int flags = 0;
    int32_t* vptr = nullptr;              // [ndof + 1] start of row r's incidences
    int4* rrec = nullptr;                 // [6 nme] {key 6k + a (row r = edof[k][a]), six 16-bit column positions},
                                          // ascending keys within a row
    int32_t* long_rows = nullptr;         // [ndof + 1] rows with more columns than one thread sums
    int32_t* n_long = nullptr;            // [2] their number, and 1 if a vertex row is longer than 24 (device)
    int32_t n_long_host[2] = {0, 0};
    double* kg = nullptr;                 // [36 nme] staged element values
    cudaStream_t last_stream = nullptr;
};

// P3 (cubic) triangle patterns (p3.cu).
struct fe_p3_pattern_s {
    int32_t nq = 0, nme = 0;
    int64_t ne = 0;                       // edges: dofs nq .. nq + 2 ne - 1, two per edge
    int32_t ndof = 0;                     // nq + 2 ne + nme (the bubbles last)
    uint64_t topology_id = 0;
    int64_t nnz = 0;
    int32_t* row_ptr = nullptr;           // [ndof + 1]
    int32_t* col_idx = nullptr;           // [nnz]
    int32_t* edof = nullptr;              // [nme][10] element dofs
    int32_t* map = nullptr;               // [100 nme] map[100k + 10 il + jl] = position of (edof[k][il], edof[k][jl])
    // FE_PATTERN_GATHER: each row's incidences in ascending element order and the staging buffer
    int flags = 0;
    int32_t* vptr = nullptr;              // [ndof + 1] start of row r's incidences
    int32_t* ikey = nullptr;              // [10 nme] keys 10k + a (row r = edof[k][a]), ascending within a row
    int32_t* ipos = nullptr;              // [10 nme][5] the incidence's ten in-row column positions, 16 bits each
    double* kg = nullptr;                 // [100 nme] staged element values, row-major per element
    int32_t* long_rows = nullptr;         // rows of more columns than one warp's fast accumulators
    int32_t n_long = 0;
    cudaStream_t last_stream = nullptr;
};

uint64_t fe_next_topology_id();

// Staged mesh creation for the one-shot host call (mesh.cu): the connectivity (device array,
// owned by the mesh afterwards) is checked for range, repeats and valences with one
// synchronisation (checked = false: valences only, for connectivity built by the library itself,
// with no synchronisation); fe_mesh_attach_coords packs device coordinates [2][nq] and queues the
// orientation check (no synchronisation); fe_mesh_orientation_status interprets the error word
// read back afterwards (4 ints).
fe_status fe_mesh_create_topology(int32_t nq, int32_t nme, int32_t* me_dev, cudaStream_t s, fe_mesh* out,
                                 bool checked = true);
fe_status fe_mesh_attach_coords(fe_mesh m, const double* q_dev, cudaStream_t s);
fe_status fe_mesh_orientation_status(const int word[4]);

// The scalar pattern of any mesh, a part included, without the map or gather lists, exposed as
// the row window [row0, row1) of the mesh's own ids (pattern.cu): n_rows, nnz and base_w are set
// from the same read-back as the rest of the build; fe_pattern_build_part adds the window's
// offsets (and, for a part, its global column ids).
fe_status fe_pattern_build_rows(fe_mesh m, int32_t row0, int32_t row1, fe_stream stream, fe_pattern* out);

// High float (top 24 significant bits, truncated) of a double, by bit operations: no FP64
// instruction. |result - x| < 2^-23 |x|; zero and subnormals give zero, magnitudes above the
// float range give +-inf.
__device__ __forceinline__ float fe_trunc_float(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    int e = (int)((hi >> 20) & 0x7FF) - 1023;
    if (e < -126) return 0.0f;
    if (e > 127) return __uint_as_float((hi & 0x80000000u) | 0x7F800000u);
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)(e + 127) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}


// Row-owner assembly of S and M for batches of meshes (rowasm.cu): per-mesh arrays, tiles of
// rows, and the list of general rows as (mesh, row).
struct fe_row_mesh {
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const int32_t* vptr;
    const int2* fan;
    const int2* hdr;
    const double2* q;
    int* err;
    int32_t nq;
    int64_t n_inc, nnz;      // fan records (3 nme) and stored entries (bounds-checked builds)
};
struct fe_row_tile {
    int32_t mesh, r0, r1;
};
int fe_row_batch_resident(int block);
void fe_row_batch_launch(const fe_row_mesh* desc, const fe_row_tile* tiles, int32_t ntiles, const int2* general,
                         int32_t ngeneral, double* const* S, double* const* M, int block, cudaStream_t s);

// row-owner assembly (rowasm.cu); kind bits: 1 = S, 2 = M^w, 4 = M
fe_status fe_row_scalar(int kind_bits, fe_mesh m, fe_pattern p, const double* w, double* out0, double* out1,
                        cudaStream_t s);
fe_status fe_row_elas(fe_mesh m, fe_pattern p, double lam, double mu, double* out, cudaStream_t s);

struct fe_batch_s;   // batch.cu

// ------------------------------------------------------------------------ errors

fe_status fe_fail(fe_status st, const std::string& msg);
fe_status fe_cuda_fail(cudaError_t e, const char* what);

#define FE_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t fe_e_ = (call);                                       \
        if (fe_e_ != cudaSuccess) return fe_cuda_fail(fe_e_, #call);      \
    } while (0)

#define FE_LAUNCHED(name)                                                 \
    do {                                                                  \
        cudaError_t fe_e_ = cudaGetLastError();                           \
        if (fe_e_ != cudaSuccess) return fe_cuda_fail(fe_e_, name);       \
    } while (0)

// Device memory comes from a library-owned stream-ordered pool (cudaMallocFromPoolAsync) that
// keeps freed blocks for reuse, so building and destroying handles does not synchronise the
// device. Allocations and frees are ordered on the stream of the innermost FeStreamScope.
struct FeStreamScope {
    explicit FeStreamScope(cudaStream_t s);
    ~FeStreamScope();
    cudaStream_t prev;
};

// Device allocation helpers; return FE_ERR_OOM with a message on failure.
fe_status fe_alloc(void** p, size_t bytes, const char* what);
template <typename T>
inline fe_status fe_alloc_n(T** p, size_t n, const char* what) {
    return fe_alloc(reinterpret_cast<void**>(p), n * sizeof(T) + (n == 0 ? sizeof(T) : 0), what);
}
void fe_free(void* p);

// ------------------------------------------------------------------------ bounds-checked builds
//
// Built with -DFEASM_BOUNDS_CHECK, FE_IDX(i, n) checks an index that the library derived itself
// (an element-to-nnz map entry, a permutation entry, a fan record, a bucket or incidence slot, an
// in-row column position) against the size n of the array it addresses. An index outside [0, n)
// is counted in this source file's device counter and replaced by 0, so the access stays inside
// the array and nothing traps; fe_debug_bounds reads and clears the counters of all files. In
// the ordinary build FE_IDX(i, n) is i and n is not evaluated.
#ifdef FEASM_BOUNDS_CHECK
void fe_oob_register(unsigned long long (*reader)(int reset));
namespace {
__device__ unsigned long long fe_oob_count = 0;
__device__ __forceinline__ int64_t fe_idx_check(int64_t i, int64_t n) {
    if (i < 0 || i >= n) {
        atomicAdd(&fe_oob_count, 1ull);
        return 0;
    }
    return i;
}
unsigned long long fe_oob_read(int reset) {
    unsigned long long h = 0;
    cudaMemcpyFromSymbol(&h, fe_oob_count, sizeof h);
    if (reset) {
        const unsigned long long z = 0;
        cudaMemcpyToSymbol(fe_oob_count, &z, sizeof z);
    }
    return h;
}
struct FeOobRegistrar {
    FeOobRegistrar() { fe_oob_register(&fe_oob_read); }
};
FeOobRegistrar fe_oob_registrar;
}  // namespace
#define FE_IDX(i, n) ((std::decay<decltype(i)>::type)fe_idx_check((int64_t)(i), (int64_t)(n)))
#else
#define FE_IDX(i, n) (i)
#endif

// ------------------------------------------------------------------------ launch shapes

// NVTX range over an entry point (named after the function), shown by Nsight tools; without a tool
// attached the push and pop return at once.
struct FeRange {
    explicit FeRange(const char* name) { nvtxRangePushA(name); }
    ~FeRange() { nvtxRangePop(); }
    FeRange(const FeRange&) = delete;
    FeRange& operator=(const FeRange&) = delete;
};
#define FE_RANGE(name) FeRange fe_range_(name)

int fe_sm_count();
inline unsigned fe_grid(int64_t n, int block, int per_sm = 8) {
    int64_t need = (n + block - 1) / block;
    int64_t cap = (int64_t)fe_sm_count() * per_sm;
    if (need < 1) need = 1;
    return (unsigned)(need < cap ? need : cap);
}

// ------------------------------------------------------------------------ scan

// Exclusive prefix sum of in[0..n) into out[0..n], out[n] = total. int32 in, int32 out.
// Returns FE_ERR_LIMIT if the total does not fit in int32. Synchronises only if total_out
// is not null (it then reads the total back).
// With round > 1 (a power of two) each input is first rounded up to a multiple of round.
fe_status fe_exclusive_scan(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s,
                            int64_t* total_out, int round = 1, int32_t* out2 = nullptr);

// ------------------------------------------------------------------------ checks shared by calls

fe_status fe_check_pair(fe_mesh mesh, fe_pattern pat, int dofs);

// ------------------------------------------------------------------------ kernel timing

// Scope guard: records a CUDA event pair around the launches in its scope when profiling is
// enabled (fe_profile_enable), attributed to `name` (a string literal).
class FeProf {
  public:
    FeProf(const char* name, cudaStream_t s);
    ~FeProf();
    FeProf(const FeProf&) = delete;
    FeProf& operator=(const FeProf&) = delete;

  private:
    const char* name_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr;
};

#define FE_PROF(name, stream) FeProf fe_prof_guard_(name, stream)
