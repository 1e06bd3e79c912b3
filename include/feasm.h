/*
 * feasm.h -- C ABI of the GB300 (sm_103a) P1 finite-element assembly library (libfeasm.so).
 *
 * The library computes, for a triangulation given by vertex coordinates q and connectivity me
 * (Section 2 of Cuvelier, Japhet, Scarella, "An efficient way to perform the assembly of finite
 * element matrices in Matlab and Octave", INRIA RR-8305), the global sparse matrices
 *   M   mass              (element matrix Eq. 1)
 *   M^w weighted mass     (element matrix Eq. 2, w given at the vertices)
 *   S   stiffness         (element matrix Eq. 3)
 *   K   plane elasticity  (element matrix |T| B^T C B of Section 7, Lame lambda, mu)
 * by summing every element's contributions into CSR storage, which is what the paper does with
 * sparse(Ig, Jg, Kg, n, n) (Sections 5-7). It also provides the adjoint of S and M^w with respect
 * to q and w, and a batched form for many meshes.
 *
 * Conventions shared by every call
 *   - Indices are 0-based (the paper is 1-based). Vertex ids and CSR indices are int32.
 *   - q is [2][nq] row-major FP64: q[i] is x_i, q[nq + i] is y_i (the paper's q(1,i), q(2,i)).
 *   - me is [3][nme] row-major int32: me[a*nme + k] is local vertex a of triangle k. Triangles
 *     must be counter-clockwise with three distinct vertices.
 *   - The area |T| is computed from the coordinates (half the cross product of two edge
 *     vectors); it is not an input. Signed area <= 0 is an orientation error.
 *   - Elasticity (dofs_per_vertex = 2) numbers the unknowns interleaved: vertex i owns rows
 *     2i (x-displacement) and 2i+1 (y-displacement); the paper's 2i-1, 2i in 1-based terms.
 *   - CSR output: row_ptr[n_rows+1], col_idx[nnz] strictly ascending inside each row. The
 *     pattern is structural: (i, j) is stored iff i and j share a triangle, so a value that
 *     sums to exactly 0.0 is still stored. All four matrices are symmetric, so these CSR arrays
 *     are also the CSC arrays the paper describes in Section 4.
 *   - Every call that takes a stream is stream-ordered and asynchronous, except where noted
 *     ("synchronises"). Device pointers must be device-resident (cudaMalloc / torch CUDA
 *     tensors) on the current device; FE_PTR_HOST inputs may be pageable or pinned host memory.
 *   - Errors are returned as fe_status; nothing traps on the device. fe_last_error() gives a
 *     human-readable message for the last failing call on the calling host thread.
 *   - Handles own the device memory they allocate; output value buffers belong to the caller.
 *   - Limits: nq < 2^31; 9*nme < 2^31 (36*nme < 2^31 for elasticity); nnz < 2^31; at most
 *     FE_MAX_VALENCE triangles around one vertex.
 */
#ifndef FEASM_H
#define FEASM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FE_OK = 0,
    FE_ERR_INVALID_ARG = 1,      /* null pointer, negative size, bad flag or kind, lambda+mu <= 0 */
    FE_ERR_INDEX_RANGE = 2,      /* a vertex id outside [0, nq) */
    FE_ERR_DEGENERATE = 3,       /* a triangle with a repeated vertex */
    FE_ERR_ORIENTATION = 4,      /* a triangle with signed area <= 0 (clockwise or flat) */
    FE_ERR_BUFFER_TOO_SMALL = 5, /* output capacity below the pattern's nnz */
    FE_ERR_OOM = 6,              /* a device allocation failed */
    FE_ERR_CUDA = 7,             /* a CUDA runtime call failed (message has the CUDA error) */
    FE_ERR_TIMEOUT = 8,          /* a bounded device-side wait ran out (none in this version) */
    FE_ERR_LIMIT = 9             /* a size limit above is exceeded */
} fe_status;

#define FE_MAX_VALENCE 4096

/* CUDA stream handle; identical to cudaStream_t (pass torch.cuda.Stream.cuda_stream). */
typedef struct CUstream_st* fe_stream;

typedef struct fe_mesh_s* fe_mesh;        /* owns device copies of q and me */
typedef struct fe_pattern_s* fe_pattern;  /* owns the CSR structure and element-to-nnz map */
typedef struct fe_batch_s* fe_batch;      /* a set of (mesh, pattern) assembled together */
typedef struct fe_tet_mesh_s* fe_tet_mesh;       /* tetrahedral mesh: device q [3][nq], me [4][nme] */
typedef struct fe_tet_pattern_s* fe_tet_pattern; /* CSR structure and map of a tetrahedral mesh */
typedef struct fe_p2_pattern_s* fe_p2_pattern;   /* P2 dofs, CSR structure and map of a triangle mesh */
typedef struct fe_p3_pattern_s* fe_p3_pattern;   /* P3 dofs, CSR structure and map of a triangle mesh */

/* Where the arrays passed to fe_mesh_create live. FE_PTR_DEVICE_BORROW: device memory, and the
 * mesh uses the caller's me in place instead of copying it (q is always packed into the mesh's
 * own array); the caller keeps me valid and unchanged until fe_mesh_destroy. */
enum { FE_PTR_HOST = 0, FE_PTR_DEVICE = 1, FE_PTR_DEVICE_BORROW = 2 };

/* Scatter variants of the assembly calls. */
enum {
    FE_VARIANT_ATOMIC = 0, /* element-parallel; FP64 atomicAdd into values (zeroed first).
                              Rounding of each sum depends on the order atomics land. */
    FE_VARIANT_GATHER = 1, /* deterministic: element matrices are staged in contribution order
                              c, then one thread per non-zero sums its contributions in
                              ascending c (the order of the paper's sparse() call).
                              Bit-identical from run to run. Needs FE_PATTERN_GATHER. */
    FE_VARIANT_ROW = 2     /* deterministic and atomic-free (the fast path): one thread per CSR
                              row walks the row's triangles in ascending order, computes the
                              row's entries of each element matrix in double-float arithmetic
                              (about 2^-45 of the row's largest entry from FP64) and writes each
                              value once. Bit-identical from run to run. Any pattern. */
};

/* Pattern build flags. */
enum {
    FE_PATTERN_DEFAULT = 0, /* CSR structure + the per-vertex triangle lists of FE_VARIANT_ROW */
    FE_PATTERN_GATHER = 1,  /* also the element-to-nnz map, the per-non-zero contribution lists
                               (seg_ptr, perm) and the staging buffer of FE_VARIANT_GATHER and
                               of the deterministic adjoint */
    FE_PATTERN_MAP = 2      /* also the element-to-nnz map (FE_VARIANT_ATOMIC, adjoint, atomic batches) */
};

/* ----------------------------------------------------------------------------- meshes ---- */

/* Creates a mesh from q ([2][nq] FP64) and me ([3][nme] int32), both host (FE_PTR_HOST) or
 * device (FE_PTR_DEVICE) memory; the library copies them (the caller keeps ownership of its
 * arrays), except me under FE_PTR_DEVICE_BORROW, which is used in place. Validates every triangle: ids in [0, nq) (else FE_ERR_INDEX_RANGE), three distinct
 * vertices (FE_ERR_DEGENERATE), signed area > 0 (FE_ERR_ORIENTATION). Synchronises the stream
 * once to read the validation result. nme = 0 is allowed (an empty mesh). Paper: Section 2
 * (mesh arrays q, me; areas derived, see the header comment). */
fe_status fe_mesh_create(int32_t nq, int32_t nme, const double* q, const int32_t* me,
                         int ptr_kind, fe_stream stream, fe_mesh* out);

/* Replaces the coordinates (same topology), e.g. for finite differences or moving meshes: q
 * [2][nq] (for a part, the global mesh's q, from which it takes its vertices' points).
 * Asynchronous for device arrays; does not re-validate orientation (assembly calls report it,
 * see fe_mesh_check). */
fe_status fe_mesh_set_coords(fe_mesh mesh, const double* q, int ptr_kind, fe_stream stream);
/* (ptr_kind: FE_PTR_HOST or FE_PTR_DEVICE; FE_PTR_DEVICE_BORROW is taken as FE_PTR_DEVICE.) */

/* Reads and clears the mesh's device-side error word, set by an assembly call that met a
 * triangle with signed area <= 0 after fe_mesh_set_coords (FE_ERR_ORIENTATION), or, for
 * FE_VARIANT_ROW, a nonzero edge-vector component or weight of magnitude outside
 * [2^-74, 2^128) (FE_ERR_LIMIT; such values are then taken as zero). Synchronises the stream. */
fe_status fe_mesh_check(fe_mesh mesh, fe_stream stream);

/* The mesh's vertex and triangle counts (a part: the global nq and the triangles it keeps). */
fe_status fe_mesh_info(fe_mesh mesh, int32_t* nq, int32_t* nme);
void fe_mesh_destroy(fe_mesh mesh);

/* -------------------------------------------------------------------------- patterns ---- */

/* Builds the CSR structure of the global matrix and the element-to-nnz map: for a scalar
 * pattern (dofs_per_vertex = 1) map[9k + 3*jl + il] is the position in col_idx of
 * (me[il][k], me[jl][k]) -- the paper's Ig/Jg arrays (Section 6, the remark on forming Ig and Jg from me)
 * resolved once into storage positions, with c = 9k + 3*jl + il the column-wise element order
 * of Section 5.
 * For dofs_per_vertex = 2 the pattern is the 2x2 block expansion of the scalar one
 * (the 6 x nme index array of Section 7.2). The structural half of sparse(): a counting sort of the
 * (row, col) keys on the row, then a sort of the columns inside each row, then unique.
 * flags: FE_PATTERN_DEFAULT, FE_PATTERN_MAP, FE_PATTERN_GATHER (or-ed). Synchronises the
 * stream once (to learn nnz). Handles release their memory on the
 * last stream they were used on (stream-ordered); work on other streams must be ordered by
 * the caller before destroying them. */
fe_status fe_pattern_build(fe_mesh mesh, int dofs_per_vertex, int flags, fe_stream stream,
                           fe_pattern* out);

/* Borrowed device pointers, valid until fe_pattern_destroy. */
fe_status fe_pattern_info(fe_pattern pattern, int64_t* n_rows, int64_t* nnz,
                          const int32_t** row_ptr, const int32_t** col_idx);

/* The scalar element-to-nnz map (device, 9*nme int32, layout above). For a dofs=2 pattern this
 * is the map of the underlying scalar pattern. FE_ERR_INVALID_ARG if the pattern was built
 * without FE_PATTERN_MAP or FE_PATTERN_GATHER. */
fe_status fe_pattern_map(fe_pattern pattern, const int32_t** map, int64_t* len);

void fe_pattern_destroy(fe_pattern pattern);

/* -------------------------------------------------------------------------- assembly ---- */

/* Each call writes the nnz values of one matrix into values[0 .. nnz) (device, FP64,
 * capacity cap >= nnz, else FE_ERR_BUFFER_TOO_SMALL), in the order of the pattern's col_idx.
 * mesh and pattern must belong together (same mesh topology; FE_ERR_INVALID_ARG otherwise). */

/* M, Eq. (1): M^e = |T|/12 [[2,1,1],[1,2,1],[1,1,2]]. Scalar pattern. */
fe_status fe_assemble_mass(fe_mesh mesh, fe_pattern pattern, int variant, double* values,
                           int64_t cap, fe_stream stream);

/* M^w, Eq. (2), with w[nq] (device FP64) the values of w at the vertices. Scalar pattern. */
fe_status fe_assemble_wmass(fe_mesh mesh, fe_pattern pattern, const double* w, int variant,
                            double* values, int64_t cap, fe_stream stream);

/* S, Eq. (3): S^e = Gram(u, v, w) / (4|T|), u = q2-q3, v = q3-q1, w = q1-q2. Scalar pattern. */
fe_status fe_assemble_stiff(fe_mesh mesh, fe_pattern pattern, int variant, double* values,
                            int64_t cap, fe_stream stream);

/* S and M^w together in one pass over the triangles (they share the scalar pattern). */
fe_status fe_assemble_stiff_wmass(fe_mesh mesh, fe_pattern pattern, const double* w,
                                  int variant, double* S_values, double* Mw_values, int64_t cap,
                                  fe_stream stream);

/* K, Section 7: K^e = |T| B^T C B with C = [[l+2m, l, 0], [l, l+2m, 0], [0, 0, m]].
 * Needs a dofs_per_vertex = 2 pattern; lambda + mu > 0 (Section 7) else FE_ERR_INVALID_ARG. */
fe_status fe_assemble_elas(fe_mesh mesh, fe_pattern pattern, double lambda, double mu,
                           int variant, double* values, int64_t cap, fe_stream stream);

/* End to end: S and M^w (FE_VARIANT_ROW) from host arrays q [2][nq], me [3][nme], w [nq] to host
 * CSR arrays row_ptr [nq + 1], col_idx, S, Mw [cap]. Creates and validates the mesh, builds the
 * pattern, assembles, and copies back, overlapping the copies with the work where the data allow
 * (me goes up first and is checked for range and repeats while q and w follow, and the pattern is
 * built during their upload; the orientation check follows; the col_idx download and the value
 * download of each of 8 row blocks overlap the assembly of the later blocks). Inputs should be
 * pinned host memory for the uploads to overlap the work, and output buffers pinned host
 * memory for the copies to overlap (pageable memory works, without overlap). *nnz gets the
 * number of stored entries; if cap < nnz the call returns FE_ERR_BUFFER_TOO_SMALL with *nnz set
 * and row_ptr unspecified (6 nme + nq always suffices). Errors of the mesh as for fe_mesh_create,
 * and of the values as for fe_mesh_check. Synchronises. Not in the paper (its Matlab call has no
 * device memory). */
fe_status fe_assemble_stiff_wmass_host(int32_t nq, int32_t nme, const double* q, const int32_t* me,
                                       const double* w, int32_t* row_ptr, int32_t* col_idx, double* S,
                                       double* Mw, int64_t cap, int64_t* nnz, fe_stream stream);

/* S and M^w as fe_assemble_stiff_wmass with FE_VARIANT_GATHER, for callers that must not have
 * device memory allocated during the call (frameworks that own all device memory through their
 * own pool and forbid hidden allocations, plug-ins loaded into such hosts, loops with hard
 * latency budgets where an allocation could stall). The
 * element values are staged in a fixed device array built into the library (18 MiB, resident on
 * every GPU that loads the library until the process exits) instead of the pattern's buffer;
 * the call performs no allocation of any kind. The paper has no counterpart.
 *   - nme <= FE_NOALLOC_MAX_TRIANGLES, else FE_ERR_LIMIT (nothing is launched).
 *   - The pattern must be built with FE_PATTERN_GATHER (FE_ERR_INVALID_ARG otherwise).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture.
 *   - All calls share the one array: calls whose work overlaps on the GPU (other streams, other
 *     host threads) race and give wrong values; order them on one stream. Each call overwrites
 *     every staged entry it reads, so nothing carries over from the previous call. */
#define FE_NOALLOC_MAX_TRIANGLES 131072
fe_status fe_assemble_stiff_wmass_noalloc(fe_mesh mesh, fe_pattern pattern, const double* w,
                                          double* S_values, double* Mw_values, int64_t cap,
                                          fe_stream stream);

/* ---------------------------------------------------------- row partitions ---- */

/* One mesh over several ranks (processes, GPUs) by rows, with no exchange of values: row i of
 * the global matrix is the structural sum (Sections 5-6) over the triangles that contain vertex
 * i, so a rank that owns the rows [row_begin, row_end) needs exactly the triangles with a vertex
 * in that range. Triangles with vertices of two ranks are held and computed by both (halo
 * triangles); each rank writes its own rows, with global column ids, and the ranks' row blocks
 * in rank order form the whole CSR matrix. Not in the paper (one Matlab process); the calls
 * communicate nothing, the caller launches the ranks and collects their blocks.
 *
 * fe_mesh_create_part: from the global mesh (q [2][nq], me [3][nme], host or device as for
 * fe_mesh_create), keeps the triangles touching [row_begin, row_end) in ascending order (the
 * selection and compaction run on the device) and the coordinates of their vertices. Inside the
 * library the part numbers its vertices locally, so its memory and the work of every later call
 * scale with the part, not with the global mesh; every id the calls take or return stays global:
 * fe_mesh_info reports the global nq and the kept triangle count, fe_mesh_set_coords takes the
 * global q [2][nq], weights w are indexed by global vertex id (nq entries), and row windows list
 * global column ids. Checks the kept triangles as fe_mesh_create does, reporting global triangle
 * indices, and any vertex id outside [0, nq) (FE_ERR_INDEX_RANGE); 0 <= row_begin <= row_end
 * <= nq (FE_ERR_INVALID_ARG). A part builds row windows of its owned rows only
 * (fe_pattern_build_part; fe_pattern_build on a part is FE_ERR_INVALID_ARG). Synchronises once.
 * Destroy with fe_mesh_destroy. */
fe_status fe_mesh_create_part(int32_t nq, int32_t nme, const double* q, const int32_t* me, int ptr_kind,
                              int32_t row_begin, int32_t row_end, fe_stream stream, fe_mesh* out);

/* The CSR rows [row_begin, row_end) of a part (within its owned rows) or of a whole mesh, as a
 * pattern of n_rows = row_end - row_begin rows whose row_ptr starts at 0 and whose col_idx holds
 * global column ids (fe_pattern_info). Scalar (dofs_per_vertex 1) and without the map or the
 * gather lists: it assembles with FE_VARIANT_ROW only (fe_assemble_mass, _wmass, _stiff,
 * _stiff_wmass), into outputs of capacity >= its nnz, each row's values bit-identical to the
 * whole mesh's row-owner assembly. Synchronises. */
fe_status fe_pattern_build_part(fe_mesh mesh, int32_t row_begin, int32_t row_end, fe_stream stream,
                                fe_pattern* out);

/* ---------------------------------------------------------- tetrahedra (3-D P1) ---- */

/* The paper states that its method extends to three dimensions without giving the formulas. These
 * calls assemble the P1 matrices of a tetrahedral mesh from the standard integrals on a
 * tetrahedron K with vertices p0..p3 (0-based local indices a, b, c):
 *   mass           M^e_ab = |K|/20 (1 + delta_ab)
 *   weighted mass  M^{e,[w]}_ab = |K|/120 sum_c kappa_abc w_c, kappa = 6 when a = b = c, 2 when
 *                  exactly two of a, b, c are equal, 1 when all differ (w at the vertices)
 *   stiffness      S^e_ab = |K| grad(phi_a) . grad(phi_b)
 * with |K| = det[p1-p0 | p2-p0 | p3-p0] / 6, which must be > 0. The global matrix is the
 * structural sum of the element matrices, as for triangles (every pair of vertices sharing a
 * tetrahedron is stored, zeros included; fe_csr_drop_zeros removes them). */
enum { FE_TET_MASS = 0, FE_TET_WMASS = 1, FE_TET_STIFF = 2 };

/* Most tetrahedra around one vertex (fe_tet_pattern_build returns FE_ERR_LIMIT above it). */
#define FE_TET_MAX_VALENCE 1024

/* Creates a tetrahedral mesh from q ([3][nq] FP64: x row, y row, z row) and me ([4][nme] int32,
 * 0-based), host or device memory as for fe_mesh_create (FE_PTR_DEVICE_BORROW uses me in place).
 * Validates every tetrahedron: ids in [0, nq) (FE_ERR_INDEX_RANGE), four distinct vertices
 * (FE_ERR_DEGENERATE), det[p1-p0 | p2-p0 | p3-p0] > 0 (FE_ERR_ORIENTATION). Synchronises once.
 * 16 nme must be < 2^31. */
fe_status fe_tet_mesh_create(int32_t nq, int32_t nme, const double* q, const int32_t* me, int ptr_kind,
                             fe_stream stream, fe_tet_mesh* out);
void fe_tet_mesh_destroy(fe_tet_mesh mesh);

/* CSR structure (columns ascending in each row) and the element-to-nnz map of a tetrahedral mesh.
 * flags: FE_PATTERN_GATHER adds what FE_VARIANT_GATHER needs: each row's incidences in ascending
 * element order with the in-row positions of their columns, and the staging buffer;
 * FE_TET_PATTERN_ELAS (below) adds the structure of the 3-D elasticity matrix. Other bits are
 * ignored; the map is always built. Synchronises once (nnz). */
fe_status fe_tet_pattern_build(fe_tet_mesh mesh, int flags, fe_stream stream, fe_tet_pattern* out);
fe_status fe_tet_pattern_info(fe_tet_pattern pattern, int64_t* n_rows, int64_t* nnz, const int32_t** row_ptr,
                              const int32_t** col_idx);
/* The map (device, 16 nme int32): map[16k + 4 il + jl] = position of (me[il][k], me[jl][k]). Note
 * the order: row-major per element (il before jl), unlike the column-wise scalar triangle map. */
fe_status fe_tet_pattern_map(fe_tet_pattern pattern, const int32_t** map, int64_t* len);
void fe_tet_pattern_destroy(fe_tet_pattern pattern);

/* Values of one matrix kind (FE_TET_MASS, FE_TET_WMASS with w[nq] device FP64, FE_TET_STIFF) on
 * the pattern's structure, into values[0 .. nnz) (device, capacity cap). variant: FE_VARIANT_ATOMIC
 * (FP64 atomicAdd after zeroing) or FE_VARIANT_GATHER (element values staged, then each row sums
 * its incidences' element rows, so that each non-zero adds its contributions in ascending element
 * order: bit-identical from run to run; needs a pattern built with FE_PATTERN_GATHER). Element
 * arithmetic in FP64. */
fe_status fe_tet_assemble(fe_tet_mesh mesh, fe_tet_pattern pattern, int kind, const double* w, int variant,
                          double* values, int64_t cap, fe_stream stream);

/* 3-D linear elasticity on tetrahedra: the plane elasticity of Section 7 carried to three
 * dimensions (the paper announces the 3-D extension without formulas). Small strains, an
 * isotropic material with constant Lame parameters lambda and mu; its material matrix must be
 * positive definite: mu > 0 and 3 lambda + 2 mu > 0, both finite (else FE_ERR_INVALID_ARG; the
 * plane case's condition lambda + mu > 0 is the 2-D form of the second). Dofs are interleaved:
 * vertex v owns rows 3v (x), 3v + 1 (y) and 3v + 2 (z). With g_a = grad(phi_a) and |K| as above,
 * and the Voigt strain vector (e_xx, e_yy, e_zz, 2 e_xy, 2 e_yz, 2 e_zx), the element matrix is
 * K^e = |K| B^T C B, that is
 *   K^e[3a + s][3b + t] = |K| (lambda g_a,s g_b,t + mu g_a,t g_b,s + mu [s = t] g_a . g_b).
 * Structure: each entry (i, j) of the scalar tetrahedral pattern becomes the 3 x 3 block of rows
 * 3i .. 3i + 2 and columns 3j .. 3j + 2. Row 3i + s starts at 9 row_ptr[i] + 3 s len_i, where
 * len_i = row_ptr[i + 1] - row_ptr[i], and its columns ascend (3j, 3j + 1, 3j + 2 for each scalar
 * column j). fe_tet_pattern_build makes it when its flags include FE_TET_PATTERN_ELAS; 9 nnz must
 * be < 2^31 (FE_ERR_LIMIT). */
#define FE_TET_PATTERN_ELAS 4

/* The structure above: n_rows = 3 nq, nnz = 9 times the scalar nnz, row_ptr [3 nq + 1] and
 * col_idx [nnz] (device memory owned by the pattern). FE_ERR_INVALID_ARG if the pattern was built
 * without FE_TET_PATTERN_ELAS. */
fe_status fe_tet_pattern_elas_info(fe_tet_pattern pattern, int64_t* n_rows, int64_t* nnz, const int32_t** row_ptr,
                                   const int32_t** col_idx);

/* Values of the 3-D elasticity matrix on that structure, into values[0 .. nnz) (device, capacity
 * cap >= nnz, else FE_ERR_BUFFER_TOO_SMALL), in the order of its col_idx. The pattern needs
 * FE_TET_PATTERN_ELAS (FE_ERR_INVALID_ARG otherwise). variant:
 *   FE_VARIANT_ATOMIC: values zeroed, then each tetrahedron adds its 144 entries by FP64 atomicAdd
 *                      (positions from the scalar map and row_ptr).
 *   FE_VARIANT_GATHER: the element matrices are staged (1152 bytes per tetrahedron, allocated for
 *                      the call), then each row sums its incidences' element rows in ascending
 *                      element order, so every value is bit-identical from run to run. Needs a
 *                      pattern built with FE_PATTERN_GATHER as well.
 * Element arithmetic in FP64. */
fe_status fe_tet_assemble_elas(fe_tet_mesh mesh, fe_tet_pattern pattern, double lambda, double mu, int variant,
                               double* values, int64_t cap, fe_stream stream);

/* ------------------------------------------------------- P2 triangles (quadratic) ---- */

/* The paper states that its method extends to P_k elements without giving the formulas. These
 * calls assemble the P2 mass and stiffness of a triangle mesh from the definitions: with the
 * barycentric coordinates l0, l1, l2 of a triangle (the P1 functions; grad l_a as in Eq. 4), the
 * local dofs are the vertex functions l_a (2 l_a - 1) (a = 0, 1, 2) and the edge functions
 * 4 l0 l1, 4 l1 l2, 4 l2 l0 (local dofs 3, 4, 5: the midpoints of edges (0,1), (1,2), (2,0));
 * M^e_ij = int_T phi_i phi_j and S^e_ij = int_T grad phi_i . grad phi_j.
 * Global dofs: vertex i is dof i; the nE edges are dofs nq .. nq + nE - 1, numbered in ascending
 * order of (smaller vertex id, larger vertex id). The structure is the structural sum, as for
 * P1. Assembly by FP64 element matrices, scattered by FP64 atomics (values zeroed first) or, for
 * FE_VARIANT_GATHER, staged and summed row by row in ascending element order. */
enum { FE_P2_MASS = 0, FE_P2_STIFF = 1 };

/* Most triangles around one vertex for a P2 pattern (FE_ERR_LIMIT above it). */
#define FE_P2_MAX_VALENCE 680

/* Dofs, CSR structure and element-to-nnz map from a mesh and its scalar (dofs = 1) pattern, whose
 * structure numbers the edges. flags: FE_PATTERN_GATHER adds what FE_VARIANT_GATHER needs (each
 * row's incidences in ascending element order and the staging buffer); other bits are ignored.
 * Synchronises (the edge count, nnz). */
fe_status fe_p2_pattern_build(fe_mesh mesh, fe_pattern scalar_pattern, int flags, fe_stream stream, fe_p2_pattern* out);
fe_status fe_p2_pattern_info(fe_p2_pattern pattern, int64_t* n_dofs, int64_t* nnz, const int32_t** row_ptr,
                             const int32_t** col_idx);
/* edof (device, [nme][6] int32): each triangle's dofs in local order; map (device, 36 nme):
 * map[36k + 6 il + jl] = position of (edof[k][il], edof[k][jl]); *n_edges = nE. */
fe_status fe_p2_pattern_dofs(fe_p2_pattern pattern, const int32_t** edof, const int32_t** map, int64_t* n_edges);
void fe_p2_pattern_destroy(fe_p2_pattern pattern);

/* Values of FE_P2_MASS or FE_P2_STIFF into values[0 .. nnz) (device, capacity cap). variant:
 * FE_VARIANT_ATOMIC (FP64 atomicAdd after zeroing) or FE_VARIANT_GATHER (element matrices staged,
 * then each row sums its incidences' element rows, so that each non-zero adds its contributions
 * in ascending element order: bit-identical from run to run; needs a pattern built with
 * FE_PATTERN_GATHER). */
fe_status fe_p2_assemble(fe_mesh mesh, fe_p2_pattern pattern, int kind, int variant, double* values, int64_t cap,
                         fe_stream stream);

/* ------------------------------------------------------------- P3 triangles (cubic) ---- */

/* The P_k extension for k = 3 (the paper announces P_k without formulas). Local dofs, with the
 * barycentric coordinates l0, l1, l2 of a triangle:
 *   0, 1, 2   the vertices, l_a (3 l_a - 1)(3 l_a - 2) / 2;
 *   3..8      two per edge, for the edges (0,1), (1,2), (2,0) in turn: on edge (a, b) the node at
 *             2/3 p_a + 1/3 p_b, 9/2 l_a l_b (3 l_a - 1), then the node at 1/3 p_a + 2/3 p_b,
 *             9/2 l_a l_b (3 l_b - 1);
 *   9         the centroid, 27 l0 l1 l2;
 * M^e_ij = int_T phi_i phi_j and S^e_ij = int_T grad phi_i . grad phi_j. Global dofs: vertex i
 * is dof i; edge e (the nE edges numbered as for P2) owns dofs nq + 2e (its node nearer the
 * smaller vertex id) and nq + 2e + 1; triangle k's bubble is dof nq + 2 nE + k. The structure is
 * the structural sum. Assembly by FP64 element matrices, scattered by FP64 atomics (values zeroed
 * first) or, for FE_VARIANT_GATHER, staged and summed row by row in ascending element order
 * (bit-identical from run to run). */
enum { FE_P3_MASS = 0, FE_P3_STIFF = 1 };

/* Most triangles around one vertex for a P3 pattern (FE_ERR_LIMIT above it). */
#define FE_P3_MAX_VALENCE 400

/* Dofs, CSR structure and element-to-nnz map from a mesh and its whole-mesh scalar (dofs = 1)
 * pattern, whose structure numbers the edges. flags: FE_PATTERN_GATHER adds what
 * FE_VARIANT_GATHER needs (each row's incidences in ascending element order with their column
 * positions, and the staging buffer); other bits are ignored. 100 nme < 2^31 (FE_ERR_LIMIT).
 * Synchronises (the edge count, nnz). */
fe_status fe_p3_pattern_build(fe_mesh mesh, fe_pattern scalar_pattern, int flags, fe_stream stream, fe_p3_pattern* out);
fe_status fe_p3_pattern_info(fe_p3_pattern pattern, int64_t* n_dofs, int64_t* nnz, const int32_t** row_ptr,
                             const int32_t** col_idx);
/* edof (device, [nme][10] int32): each triangle's dofs in local order; map (device, 100 nme):
 * map[100k + 10 il + jl] = position of (edof[k][il], edof[k][jl]); *n_edges = nE. */
fe_status fe_p3_pattern_dofs(fe_p3_pattern pattern, const int32_t** edof, const int32_t** map, int64_t* n_edges);
void fe_p3_pattern_destroy(fe_p3_pattern pattern);

/* Values of FE_P3_MASS or FE_P3_STIFF into values[0 .. nnz) (device, capacity cap). variant:
 * FE_VARIANT_ATOMIC or FE_VARIANT_GATHER (needs a pattern built with FE_PATTERN_GATHER). */
fe_status fe_p3_assemble(fe_mesh mesh, fe_p3_pattern pattern, int kind, int variant, double* values, int64_t cap,
                         fe_stream stream);

/* -------------------------------------------------------------------- zero dropping ---- */

/* Matlab's sparse() stores no zero (Section 5): an entry of K that is zero adds nothing and a
 * position whose sum is zero is not stored. The assembly calls keep every structural position
 * (one pattern then serves every matrix and every q); this call gives the value-dependent
 * result. It removes from a CSR matrix every entry whose value compares equal to 0.0 (+0 and -0)
 * and keeps the others in their order (NaN compares unequal to 0 and stays). For the symmetric
 * M, M^w, S and K the CSR arrays are also Matlab's CSC arrays.
 *   row_ptr [n_rows + 1], col_idx [row_ptr[n_rows]], values [row_ptr[n_rows]]: the input, device,
 *     for example a pattern's arrays (fe_pattern_info) and an assembled value array;
 *   row_ptr_out [n_rows + 1], col_idx_out [cap], values_out [cap]: device, caller-owned; they
 *     must not overlap the inputs (FE_ERR_INVALID_ARG if they start at the same address);
 *   *nnz_out (host): the number of entries kept.
 * 0 <= n_rows < 2^31. Synchronises once, to read the count. If cap is below the count the call
 * returns FE_ERR_BUFFER_TOO_SMALL with *nnz_out set and row_ptr_out written, and col_idx_out /
 * values_out untouched. */
fe_status fe_csr_drop_zeros(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx,
                            const double* values, int32_t* row_ptr_out, int32_t* col_idx_out,
                            double* values_out, int64_t cap, int64_t* nnz_out, fe_stream stream);

/* --------------------------------------------------------------------------- adjoint ---- */

/* Needs a pattern with the element-to-nnz map (FE_PATTERN_MAP or FE_PATTERN_GATHER).
 * Gradient of L = sum_p gS[p] * S.values[p] + sum_p gM[p] * Mw.values[p] with respect to the
 * coordinates and the vertex weights (not in the paper: the derivative of Eqs. 2-3 with the
 * area taken from the coordinates). gS, gM: device FP64 [nnz] on the scalar pattern (either
 * may be NULL for zero). Writes dq ([2][nq], same layout as q) and dw ([nq]); both are
 * overwritten, not accumulated. variant FE_VARIANT_ATOMIC scatters per-vertex sums with
 * atomics; FE_VARIANT_GATHER stages per-element terms and sums each vertex's triangles in
 * ascending triangle order (bit-identical run to run, needs FE_PATTERN_GATHER). */
fe_status fe_adjoint_stiff_wmass(fe_mesh mesh, fe_pattern pattern, const double* w,
                                 const double* gS, const double* gM, int variant, double* dq,
                                 double* dw, fe_stream stream);

/* --------------------------------------------------------------------------- batches ---- */

/* A batch assembles S and M (the mass matrix of Eq. 1) for n independent meshes in one
 * persistent kernel launch, replayed from a captured CUDA graph. meshes[m] / patterns[m] are
 * borrowed (they must outlive the batch); patterns are scalar. Two schemes:
 *   FE_VARIANT_ROW     row owners walk tiles of rows (tile = rows per tile); any pattern;
 *   FE_VARIANT_ATOMIC  threads walk tiles of triangles (tile = triangles per tile) and add with
 *                      FP64 atomics; needs every pattern built with FE_PATTERN_MAP.
 * The scheme, block size and tile size come from fe_batch_tune, fe_batch_configure, or the
 * defaults (FE_VARIANT_ROW, 256, 1024). Not in the paper. */
fe_status fe_batch_create(int32_t n, const fe_mesh* meshes, const fe_pattern* patterns,
                          fe_batch* out);

/* Times every candidate (scheme x block size x tile size) on this batch with the given
 * output buffers, keeps the fastest and recaptures the graph; writes the chosen block and tile
 * to *block and *tile if not NULL (the scheme: fe_batch_get_config). Synchronises. */
fe_status fe_batch_tune(fe_batch batch, double* const* S_values, double* const* M_values,
                        fe_stream stream, int32_t* block, int32_t* tile);

/* fe_batch_tune with a file cache of its choices, so that a later process (or a later batch of
 * the same shape) skips the timing. cache_path names a JSON file (NULL or "": the path in the
 * environment variable FEASM_TUNE_CACHE; neither set: plain fe_batch_tune). Each entry is keyed
 * by the device's name and SM count and by the batch's signature (a hash of every mesh's vertex,
 * triangle and non-zero counts, in order, and of whether all patterns carry the element map).
 * A cached choice is configured without timing (*from_cache = 1, if not NULL); otherwise the
 * candidates are timed as by fe_batch_tune and the choice is added to the file (written to a
 * temporary name and renamed over it; FE_ERR_INVALID_ARG if it cannot be written). The cache
 * belongs to the tuning call, not to batch creation, because timing needs the output buffers.
 * Not in the paper (its assembly has no launch parameters). Synchronises. */
fe_status fe_batch_tune_cached(fe_batch batch, const char* cache_path, double* const* S_values,
                               double* const* M_values, fe_stream stream, int32_t* block,
                               int32_t* tile, int32_t* from_cache);

/* Sets the scheme and launch shape explicitly: variant FE_VARIANT_ROW (block 64..256) or
 * FE_VARIANT_ATOMIC (block 64..1024), block a multiple of 32, tile >= 1. Synchronises the
 * device (the graph may be in flight) and recaptures the graph. */
fe_status fe_batch_configure(fe_batch batch, int32_t variant, int32_t block, int32_t tile);

/* fe_batch_configure with the current scheme. */
fe_status fe_batch_set_shape(fe_batch batch, int32_t block, int32_t tile);

/* The current scheme, block size and tile size (any pointer may be NULL). */
fe_status fe_batch_get_config(fe_batch batch, int32_t* variant, int32_t* block, int32_t* tile);

/* S_values[m], M_values[m]: device FP64 outputs of mesh m (capacity = that pattern's nnz).
 * Replays the batch's graph; a new set of output pointers is copied into the batch's device
 * pointer tables first (stream-ordered). */
fe_status fe_batch_assemble_stiff_mass(fe_batch batch, double* const* S_values,
                                       double* const* M_values, fe_stream stream);

/* The same work as n separate plain launches of the batch's scheme (per mesh: the row-owner
 * kernels, or one memset pair and one atomic kernel), for comparison with the batched launch. */
fe_status fe_batch_assemble_stiff_mass_plain(fe_batch batch, double* const* S_values,
                                             double* const* M_values, fe_stream stream);

void fe_batch_destroy(fe_batch batch);

/* --------------------------------------------------------------------- kernel timing ---- */

/* Opt-in timing of the library's own kernels (measurement support; not in the paper). While
 * on, every kernel launch is bracketed by two CUDA events recorded on its launch stream
 * (skipped while that stream is being captured into a graph). fe_profile_read resolves the
 * pending events (it waits for them) and returns per kernel name the summed device time in
 * milliseconds and the number of launches: names is a caller array of max_entries x 64 chars,
 * total_ms and launches have max_entries elements (any of the three may be NULL); *count gets
 * the number of distinct kernels seen, which may exceed max_entries. fe_profile_reset drops
 * all totals. Thread-safe; process-wide. */
fe_status fe_profile_enable(int on);
fe_status fe_profile_reset(void);
fe_status fe_profile_read(int32_t max_entries, char* names, double* total_ms, int64_t* launches,
                          int32_t* count);

/* FP64 issue rate of this GPU, measured (measurement support; not in the paper): independent
 * fused multiply-add chains on every SM, 8 blocks of 256 threads per SM, timed with CUDA events
 * on stream: the fastest of five launches after two warm-up ones. *instr_per_s gets the FP64
 * instructions (one per thread and FMA) per second. Synchronises the stream; takes about 0.1 s. */
fe_status fe_measure_fp64_rate(double* instr_per_s, fe_stream stream);

/* ----------------------------------------------------------------------- test hooks ---- */

/* Allocation-failure injection, for the tests of the error paths (not in the paper): after
 * fe_debug_fail_alloc(n) with n >= 1, the n-th device allocation the library makes from then on
 * fails as if the device were out of memory. The call that makes it returns FE_ERR_OOM, having
 * released everything it had allocated. Later allocations succeed again; n <= 0 switches the
 * injection off. Process-wide. fe_debug_pool_used returns the bytes currently allocated from the
 * library's device memory pool (the memory that meshes, patterns, batches and running calls
 * hold), so that a test can check that a failed call left nothing behind. */
void fe_debug_fail_alloc(int64_t n);

/* Bounds-checked builds. A library compiled with -DFEASM_BOUNDS_CHECK checks every index it
 * derives itself (element-to-nnz map entries, permutation and incidence entries, fan records,
 * bucket slots, in-row column positions) against the array it addresses, counts the ones out of
 * range and redirects those accesses to element 0 instead of trapping. *checked is 1 in such a
 * build (0 otherwise); *violations is the count since the last reset (always 0 in an ordinary
 * build); reset != 0 clears it. Synchronises the device. Not in the paper (a testing aid, in place
 * of a memory checker). */
fe_status fe_debug_bounds(int32_t* checked, int64_t* violations, int32_t reset);
fe_status fe_debug_pool_used(int64_t* bytes);

/* ---------------------------------------------------------------------------- status ---- */

const char* fe_status_string(fe_status status);
const char* fe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FEASM_H */
