// batch.cu -- many independent meshes assembled in one persistent launch under a CUDA graph.
//
// Not in the paper. A batch assembles the stiffness S (Eq. 3) and mass M (Eq. 1) of each of its
// meshes with one of two schemes:
//   FE_VARIANT_ROW     the row-owner fan computation (rowasm.cu) over a list of row tiles
//                      (mesh, first row, end row): every value written once, no zeroing, no map;
//                      general rows of all meshes are a second list, one block each;
//   FE_VARIANT_ATOMIC  a list of triangle tiles (mesh, first triangle, end triangle): a zeroing
//                      kernel, then each triangle's entries added with FP64 atomics through the
//                      element-to-nnz map.
// One persistent kernel (grid = SMs x resident blocks) walks its tile list round-robin. The
// launches are captured once in a CUDA graph and replayed; outputs are read from device pointer
// tables, so changing the output buffers only rewrites the tables. fe_batch_tune times every
// (scheme, block size, tile size) in a small grid and keeps the fastest.
#include <string.h>

#include <vector>

#include "internal.cuh"

struct MeshDesc {
    const double2* q;
    const int32_t* me;
    const int32_t* map;
    int32_t nme;
    int32_t nnz;
};

struct Tile {
    int32_t mesh, k0, k1;
};

struct fe_batch_s {
    int32_t n = 0;
    int variant = FE_VARIANT_ROW;
    bool has_map = true;                 // every pattern carries the element-to-nnz map
    fe_row_mesh* d_rdesc = nullptr;
    int2* d_gen = nullptr;               // general rows (mesh, row)
    int32_t ngen = 0;
    std::vector<fe_mesh> meshes;
    std::vector<fe_pattern> patterns;
    MeshDesc* d_desc = nullptr;
    double** d_S = nullptr;   // [n] output pointers
    double** d_M = nullptr;
    double** h_ptrs = nullptr;   // pinned staging: S pointers then M pointers
    std::vector<double*> cur_S, cur_M;
    Tile* d_tiles = nullptr;
    int32_t ntiles = 0;
    int32_t block = 256, tile = 1024;
    int64_t total_nnz = 0, total_nme = 0;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap_stream = nullptr;
};

// One warp per mesh-chunk: zero all outputs.
__global__ void k_batch_zero(const MeshDesc* __restrict__ desc, int32_t n, double* const* __restrict__ S,
                             double* const* __restrict__ M) {
    for (int32_t m = blockIdx.x; m < n; m += gridDim.x) {
        int32_t nnz = desc[m].nnz;
        double* s = S[m];
        double* mm = M[m];
        for (int32_t i = threadIdx.x; i < nnz; i += blockDim.x) {
            s[i] = 0.0;
            mm[i] = 0.0;
        }
    }
}

__device__ __forceinline__ void tri_stiff_mass(const double2* __restrict__ q, const int32_t* __restrict__ me,
                                               int32_t nme, int32_t k, const int32_t* __restrict__ mk,
                                               double* __restrict__ S, double* __restrict__ M, int32_t nnz) {
    int32_t v0 = me[k], v1 = me[nme + k], v2 = me[2 * nme + k];
    double2 p0 = q[v0], p1 = q[v1], p2 = q[v2];
    double ex[3] = {p1.x - p2.x, p2.x - p0.x, p0.x - p1.x};
    double ey[3] = {p1.y - p2.y, p2.y - p0.y, p0.y - p1.y};
    double D = ex[1] * ey[2] - ex[2] * ey[1];
    double inv = 1.0 / (2.0 * D);
    double dia = D / 12.0, off = D / 24.0;
#pragma unroll
    for (int b = 0; b < 3; b++)
#pragma unroll
        for (int a = 0; a < 3; a++) {
            int32_t p = FE_IDX(mk[3 * b + a], nnz);
            atomicAdd(&S[p], (ex[a] * ex[b] + ey[a] * ey[b]) * inv);
            atomicAdd(&M[p], a == b ? dia : off);
        }
}

__global__ void k_batch_asm(const MeshDesc* __restrict__ desc, const Tile* __restrict__ tiles, int32_t ntiles,
                            double* const* __restrict__ S, double* const* __restrict__ M) {
    for (int32_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        Tile tl = tiles[t];
        MeshDesc d = desc[tl.mesh];
        double* s = S[tl.mesh];
        double* mm = M[tl.mesh];
        for (int32_t k = tl.k0 + threadIdx.x; k < tl.k1; k += blockDim.x)
            tri_stiff_mass(d.q, d.me, d.nme, k, d.map + 9 * (int64_t)k, s, mm, d.nnz);
    }
}

// Plain form: one kernel per mesh.
__global__ void k_mesh_asm(MeshDesc d, double* __restrict__ S, double* __restrict__ M) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < d.nme; k += gridDim.x * blockDim.x)
        tri_stiff_mass(d.q, d.me, d.nme, k, d.map + 9 * (int64_t)k, S, M, d.nnz);
}

static void drop_graph(fe_batch b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

static int resident_blocks(int block) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_asm, block, 0);
    return per_sm > 0 ? per_sm : 1;
}

// Tiles of triangles (FE_VARIANT_ATOMIC) or of rows (FE_VARIANT_ROW), b->tile units each.
static fe_status make_tiles(fe_batch b) {
    std::vector<Tile> tiles;
    for (int32_t m = 0; m < b->n; m++) {
        int32_t units = b->variant == FE_VARIANT_ROW ? b->meshes[m]->nq : b->meshes[m]->nme;
        for (int32_t k = 0; k < units; k += b->tile) {
            int32_t e = k + b->tile < units ? k + b->tile : units;
            tiles.push_back({m, k, e});
        }
    }
    fe_free(b->d_tiles);
    b->d_tiles = nullptr;
    b->ntiles = (int32_t)tiles.size();
    fe_status st = fe_alloc_n(&b->d_tiles, tiles.size(), "batch tiles");
    if (st) return st;
    if (!tiles.empty()) FE_CUDA(cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice));
    return FE_OK;
}

static void launch_batch(fe_batch b, cudaStream_t s) {
    if (b->variant == FE_VARIANT_ROW) {
        static_assert(sizeof(Tile) == sizeof(fe_row_tile), "tile layouts must agree");
        fe_row_batch_launch(b->d_rdesc, reinterpret_cast<const fe_row_tile*>(b->d_tiles), b->ntiles, b->d_gen, b->ngen,
                            b->d_S, b->d_M, b->block, s);
        return;
    }
    unsigned zgrid = (unsigned)(b->n < 4 * fe_sm_count() ? (b->n > 0 ? b->n : 1) : 4 * fe_sm_count());
    { FE_PROF("k_batch_zero", s); k_batch_zero<<<zgrid, 256, 0, s>>>(b->d_desc, b->n, b->d_S, b->d_M); }
    int64_t want = (int64_t)fe_sm_count() * resident_blocks(b->block);
    unsigned grid = (unsigned)(b->ntiles < want ? (b->ntiles > 0 ? b->ntiles : 1) : want);
    { FE_PROF("k_batch_asm", s); k_batch_asm<<<grid, b->block, 0, s>>>(b->d_desc, b->d_tiles, b->ntiles, b->d_S, b->d_M); }
}

static fe_status capture(fe_batch b) {
    drop_graph(b);
    FE_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    launch_batch(b, b->cap_stream);
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (e != cudaSuccess) return fe_cuda_fail(e, "graph capture");
    FE_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
    return FE_OK;
}

// Copies the output pointer tables to the device if they changed (stream-ordered).
static fe_status set_outputs(fe_batch b, double* const* S, double* const* M, cudaStream_t s) {
    if (!S || !M) return fe_fail(FE_ERR_INVALID_ARG, "null output table");
    for (int32_t m = 0; m < b->n; m++)
        if ((!S[m] || !M[m]) && b->patterns[m]->nnz > 0) return fe_fail(FE_ERR_INVALID_ARG, "null output buffer in batch");
    bool same = !b->cur_S.empty();
    for (int32_t m = 0; same && m < b->n; m++) same = b->cur_S[m] == S[m] && b->cur_M[m] == M[m];
    if (same) return FE_OK;
    // the previous copy from the pinned staging area must be finished before it is rewritten
    FE_CUDA(cudaStreamSynchronize(s));
    b->cur_S.assign(S, S + b->n);
    b->cur_M.assign(M, M + b->n);
    memcpy(b->h_ptrs, S, sizeof(double*) * b->n);
    memcpy(b->h_ptrs + b->n, M, sizeof(double*) * b->n);
    FE_CUDA(cudaMemcpyAsync(b->d_S, b->h_ptrs, sizeof(double*) * 2 * b->n, cudaMemcpyHostToDevice, s));
    return FE_OK;
}

extern "C" void fe_batch_destroy(fe_batch b) {
    if (!b) return;
    cudaDeviceSynchronize();   // the graph may still be running on a caller's stream
    FeStreamScope scope(nullptr);
    drop_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    fe_free(b->d_desc);
    fe_free(b->d_rdesc);
    fe_free(b->d_gen);
    fe_free(b->d_S);
    fe_free(b->d_tiles);
    if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
    delete b;
}

extern "C" fe_status fe_batch_create(int32_t n, const fe_mesh* meshes, const fe_pattern* patterns, fe_batch* out) {
    FE_RANGE(__func__);
    if (!out) return fe_fail(FE_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (n < 0 || (n > 0 && (!meshes || !patterns))) return fe_fail(FE_ERR_INVALID_ARG, "bad mesh list");
    std::vector<MeshDesc> desc(n > 0 ? n : 1);
    std::vector<fe_row_mesh> rdesc(n > 0 ? n : 1);
    std::vector<int2> gen;
    FeStreamScope scope(nullptr);
    fe_batch b = new fe_batch_s();
    b->n = n;
    for (int32_t m = 0; m < n; m++) {
        fe_status st = fe_check_pair(meshes[m], patterns[m], 1);
        if (!st && patterns[m]->row1 >= 0) st = fe_fail(FE_ERR_INVALID_ARG, "batches take whole-mesh patterns, not row windows");
        if (st) { fe_batch_destroy(b); return st; }
        fe_mesh me = meshes[m];
        fe_pattern p = patterns[m];
        b->meshes.push_back(me);
        b->patterns.push_back(p);
        b->has_map = b->has_map && p->map != nullptr;
        desc[m] = {me->q, me->me, p->map, me->nme, (int32_t)p->nnz};
        rdesc[m] = {p->row_ptr, p->col_idx, p->vptr, p->fan, p->hdr, me->q, me->err, me->nq, 3 * (int64_t)me->nme,
                    p->nnz_scalar};
        if (p->n_gen > 0) {
            std::vector<int32_t> rows(p->n_gen);
            cudaError_t e = cudaMemcpy(rows.data(), p->gen_rows, sizeof(int32_t) * p->n_gen, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { fe_batch_destroy(b); return fe_cuda_fail(e, "batch general rows"); }
            for (int32_t r : rows) gen.push_back(make_int2(m, r));
        }
        b->total_nnz += p->nnz;
        b->total_nme += me->nme;
    }
    if (!b->has_map) b->variant = FE_VARIANT_ROW;
    b->ngen = (int32_t)gen.size();
    fe_status st = fe_alloc_n(&b->d_desc, desc.size(), "batch descriptors");
    if (!st) st = fe_alloc_n(&b->d_rdesc, rdesc.size(), "batch row descriptors");
    if (!st) st = fe_alloc_n(&b->d_gen, gen.size(), "batch general rows");
    if (!st) st = fe_alloc_n(&b->d_S, 2 * (size_t)(n > 0 ? n : 1), "batch output tables");
    if (st) { fe_batch_destroy(b); return st; }
    b->d_M = b->d_S + n;
    cudaError_t e = cudaMemcpy(b->d_desc, desc.data(), sizeof(MeshDesc) * desc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_rdesc, rdesc.data(), sizeof(fe_row_mesh) * rdesc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !gen.empty()) e = cudaMemcpy(b->d_gen, gen.data(), sizeof(int2) * gen.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_ptrs, sizeof(double*) * 2 * (n > 0 ? n : 1));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { fe_batch_destroy(b); return fe_cuda_fail(e, "batch setup"); }
    st = make_tiles(b);
    if (!st) st = capture(b);
    if (st) { fe_batch_destroy(b); return st; }
    *out = b;
    return FE_OK;
}

static int max_block(int variant) { return variant == FE_VARIANT_ROW ? 256 : 1024; }

extern "C" fe_status fe_batch_configure(fe_batch b, int32_t variant, int32_t block, int32_t tile) {
    if (!b) return fe_fail(FE_ERR_INVALID_ARG, "null batch");
    if (variant != FE_VARIANT_ROW && variant != FE_VARIANT_ATOMIC)
        return fe_fail(FE_ERR_INVALID_ARG, "batches support FE_VARIANT_ROW and FE_VARIANT_ATOMIC");
    if (variant == FE_VARIANT_ATOMIC && !b->has_map)
        return fe_fail(FE_ERR_INVALID_ARG, "FE_VARIANT_ATOMIC needs every pattern built with FE_PATTERN_MAP");
    if (block < 64 || block > max_block(variant) || block % 32 || tile < 1) return fe_fail(FE_ERR_INVALID_ARG, "bad batch shape");
    if (variant == b->variant && block == b->block && tile == b->tile) return FE_OK;
    FE_CUDA(cudaDeviceSynchronize());   // the graph may be in flight
    FeStreamScope scope(nullptr);
    b->variant = variant;
    b->block = block;
    b->tile = tile;
    fe_status st = make_tiles(b);
    if (!st) st = capture(b);
    return st;
}

extern "C" fe_status fe_batch_set_shape(fe_batch b, int32_t block, int32_t tile) {
    if (!b) return fe_fail(FE_ERR_INVALID_ARG, "null batch");
    return fe_batch_configure(b, b->variant, block, tile);
}

extern "C" fe_status fe_batch_get_config(fe_batch b, int32_t* variant, int32_t* block, int32_t* tile) {
    if (!b) return fe_fail(FE_ERR_INVALID_ARG, "null batch");
    if (variant) *variant = b->variant;
    if (block) *block = b->block;
    if (tile) *tile = b->tile;
    return FE_OK;
}

extern "C" fe_status fe_batch_assemble_stiff_mass(fe_batch b, double* const* S, double* const* M, fe_stream stream) {
    FE_RANGE(__func__);
    if (!b) return fe_fail(FE_ERR_INVALID_ARG, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    fe_status st = set_outputs(b, S, M, s);
    if (st) return st;
    if (b->n == 0) return FE_OK;
    FE_CUDA(cudaGraphLaunch(b->exec, s));
    return FE_OK;
}

extern "C" fe_status fe_batch_assemble_stiff_mass_plain(fe_batch b, double* const* S, double* const* M, fe_stream stream) {
    FE_RANGE(__func__);
    if (!b) return fe_fail(FE_ERR_INVALID_ARG, "null batch");
    if (!S || !M) return fe_fail(FE_ERR_INVALID_ARG, "null output table");
    cudaStream_t s = (cudaStream_t)stream;
    for (int32_t m = 0; m < b->n; m++) {
        fe_mesh me = b->meshes[m];
        fe_pattern p = b->patterns[m];
        if (b->variant == FE_VARIANT_ROW) {
            if (p->nnz > 0 && (!S[m] || !M[m])) return fe_fail(FE_ERR_INVALID_ARG, "null output buffer in batch");
            fe_status st = fe_row_scalar(1 | 4, me, p, nullptr, S[m], M[m], s);   // W_S | W_M
            if (st) return st;
            continue;
        }
        if (p->nnz > 0) {
            if (!S[m] || !M[m]) return fe_fail(FE_ERR_INVALID_ARG, "null output buffer in batch");
            FE_CUDA(cudaMemsetAsync(S[m], 0, sizeof(double) * p->nnz, s));
            FE_CUDA(cudaMemsetAsync(M[m], 0, sizeof(double) * p->nnz, s));
        }
        if (me->nme == 0) continue;
        MeshDesc d = {me->q, me->me, p->map, me->nme, (int32_t)p->nnz};
        { FE_PROF("k_mesh_asm", s); k_mesh_asm<<<fe_grid(me->nme, 256), 256, 0, s>>>(d, S[m], M[m]); }
        FE_LAUNCHED("k_mesh_asm");
    }
    return FE_OK;
}

extern "C" fe_status fe_batch_tune(fe_batch b, double* const* S, double* const* M, fe_stream stream, int32_t* block_out,
                                   int32_t* tile_out) {
    FE_RANGE(__func__);
    if (!b) return fe_fail(FE_ERR_INVALID_ARG, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    fe_status st = set_outputs(b, S, M, s);
    if (st) return st;
    FE_CUDA(cudaStreamSynchronize(s));
    FeStreamScope scope(nullptr);
    const int variants[] = {FE_VARIANT_ROW, FE_VARIANT_ATOMIC};
    const int blocks[] = {128, 256, 512};
    const int tiles[] = {256, 1024, 4096};
    cudaEvent_t e0, e1;
    FE_CUDA(cudaEventCreate(&e0));
    FE_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bv = b->variant, bb = b->block, bt = b->tile;
    for (int var : variants)
    for (int blk : blocks)
        for (int tl : tiles) {
            if (var == FE_VARIANT_ATOMIC && !b->has_map) continue;
            if (blk > max_block(var)) continue;
            b->variant = var;
            b->block = blk;
            b->tile = tl;
            if ((st = make_tiles(b))) break;
            for (int w = 0; w < 2; w++) launch_batch(b, s);
            cudaEventRecord(e0, s);
            for (int r = 0; r < 5; r++) launch_batch(b, s);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) { st = fe_cuda_fail(e, "batch tuning"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; bv = var; bb = blk; bt = tl; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    b->variant = bv;
    b->block = bb;
    b->tile = bt;
    if ((st = make_tiles(b))) return st;
    if ((st = capture(b))) return st;
    if (block_out) *block_out = bb;
    if (tile_out) *tile_out = bt;
    return FE_OK;
}

// ---------------------------------------------------------------- tuning cache
//
// fe_batch_tune_cached keeps each tuning result in a small JSON file: one object mapping a key to
// the chosen scheme and shape,
//   {
//   "<device>|sm<count>|n<meshes>|<signature>": {"variant": 2, "block": 256, "tile": 1024, "ms": 0.98},
//   ...
//   }
// The signature is a 64-bit FNV-1a hash of every mesh's vertex, triangle and non-zero counts and
// of whether all patterns carry the element map (what the candidates' times depend on). The file
// is read and rewritten whole (written to a temporary name, then renamed over the old file), one
// entry per line; the reader accepts the files this writer produces.

#include <stdio.h>
#include <stdlib.h>
#include <unistd.h>

#include <map>
#include <string>

namespace {

struct TuneChoice {
    int variant = 0, block = 0, tile = 0;
    double ms = 0.0;
};

uint64_t fnv1a(uint64_t h, uint64_t v) {
    for (int i = 0; i < 8; i++) {
        h ^= (v >> (8 * i)) & 0xFFu;
        h *= 0x100000001B3ull;
    }
    return h;
}

std::string tune_key(fe_batch b) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) prop.name[0] = 0, prop.multiProcessorCount = 0;
    uint64_t h = 0xCBF29CE484222325ull;
    h = fnv1a(h, (uint64_t)b->n);
    h = fnv1a(h, b->has_map ? 1u : 0u);
    for (int32_t m = 0; m < b->n; m++) {
        h = fnv1a(h, (uint64_t)(uint32_t)b->meshes[m]->nq);
        h = fnv1a(h, (uint64_t)(uint32_t)b->meshes[m]->nme);
        h = fnv1a(h, (uint64_t)b->patterns[m]->nnz);
    }
    std::string name(prop.name);
    for (char& c : name)
        if (c == '"' || c == '\\' || c == '|' || (unsigned char)c < 32) c = '_';
    char buf[64];
    snprintf(buf, sizeof buf, "|sm%d|n%d|%016llx", prop.multiProcessorCount, (int)b->n, (unsigned long long)h);
    return name + buf;
}

// Entries of a cache file ("" or unreadable: none).
std::map<std::string, TuneChoice> read_cache(const char* path) {
    std::map<std::string, TuneChoice> out;
    FILE* f = fopen(path, "r");
    if (!f) return out;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        char* q0 = strchr(line, '"');
        if (!q0) continue;
        char* q1 = strchr(q0 + 1, '"');
        if (!q1) continue;
        TuneChoice c;
        const char* v = strstr(q1, "\"variant\":");
        const char* bl = strstr(q1, "\"block\":");
        const char* t = strstr(q1, "\"tile\":");
        const char* ms = strstr(q1, "\"ms\":");
        if (!v || !bl || !t) continue;
        c.variant = atoi(v + 10);
        c.block = atoi(bl + 8);
        c.tile = atoi(t + 7);
        c.ms = ms ? atof(ms + 5) : 0.0;
        out[std::string(q0 + 1, q1)] = c;
    }
    fclose(f);
    return out;
}

bool write_cache(const char* path, const std::map<std::string, TuneChoice>& entries) {
    std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fputs("{\n", f);
    size_t k = 0;
    for (const auto& e : entries) {
        fprintf(f, "\"%s\": {\"variant\": %d, \"block\": %d, \"tile\": %d, \"ms\": %.6f}%s\n", e.first.c_str(),
                e.second.variant, e.second.block, e.second.tile, e.second.ms, ++k < entries.size() ? "," : "");
    }
    fputs("}\n", f);
    bool ok = fclose(f) == 0;
    if (ok) ok = rename(tmp.c_str(), path) == 0;
    if (!ok) remove(tmp.c_str());
    return ok;
}

}  // namespace

extern "C" fe_status fe_batch_tune_cached(fe_batch b, const char* cache_path, double* const* S, double* const* M,
                                          fe_stream stream, int32_t* block_out, int32_t* tile_out,
                                          int32_t* from_cache) {
    FE_RANGE(__func__);
    if (!b) return fe_fail(FE_ERR_INVALID_ARG, "null batch");
    if (from_cache) *from_cache = 0;
    const char* path = cache_path && cache_path[0] ? cache_path : getenv("FEASM_TUNE_CACHE");
    if (!path || !path[0]) return fe_batch_tune(b, S, M, stream, block_out, tile_out);
    const std::string key = tune_key(b);
    std::map<std::string, TuneChoice> entries = read_cache(path);
    auto it = entries.find(key);
    if (it != entries.end()) {
        const TuneChoice& c = it->second;
        const bool usable = (c.variant == FE_VARIANT_ROW || (c.variant == FE_VARIANT_ATOMIC && b->has_map)) &&
                            c.block >= 64 && c.block <= max_block(c.variant) && c.block % 32 == 0 && c.tile >= 1;
        if (usable) {
            fe_status st = set_outputs(b, S, M, (cudaStream_t)stream);
            if (!st) st = fe_batch_configure(b, c.variant, c.block, c.tile);
            if (st) return st;
            if (block_out) *block_out = c.block;
            if (tile_out) *tile_out = c.tile;
            if (from_cache) *from_cache = 1;
            return FE_OK;
        }
    }
    int32_t blk = 0, tl = 0;
    fe_status st = fe_batch_tune(b, S, M, stream, &blk, &tl);
    if (st) return st;
    // the chosen configuration's time, for the record (one more timed replay set)
    TuneChoice c;
    c.variant = b->variant;
    c.block = blk;
    c.tile = tl;
    {
        cudaStream_t s = (cudaStream_t)stream;
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < 5; r++) launch_batch(b, s);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) c.ms = ms / 5;
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
        }
    }
    entries = read_cache(path);                        // another process may have added entries meanwhile
    entries[key] = c;
    if (!write_cache(path, entries))
        return fe_fail(FE_ERR_INVALID_ARG, std::string("could not write the tuning cache ") + path);
    if (block_out) *block_out = blk;
    if (tile_out) *tile_out = tl;
    return FE_OK;
}
