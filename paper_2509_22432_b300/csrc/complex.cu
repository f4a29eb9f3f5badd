// flood_complex_faces: the triangles and edges of a set of tetrahedra and the
// facet incidence of every simplex, on the device.
//
// The discretised complex of §4.1 admits a simplex only after all of its faces,
// so the filtration needs every face of Del(L) and, per simplex, the rows of
// its facets. The host triangulation (§4) yields tetrahedra only; this builds
// the rest. Triangles are the four faces of the tetrahedra (face j drops vertex
// j), edges the three faces of the triangles. A face is owned by the lowest
// (parent row, j) that produces it: an open-addressing hash table keyed by the
// face's vertex ids keeps that minimum (atomicMin), an exclusive scan over the
// owner flags numbers the rows in owner order, and every (parent, j) reads its
// facet's row from the table. The output therefore does not depend on thread
// timing. Rows keep ascending vertex ids; their order is the owner order, not
// lexicographic.
#include "scan.cuh"

namespace flood {
namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kVertexBits = 21;  // three ids per 64-bit key

// splitmix64's output mix (Steele, Lea and Flood, 2014) spreads packed ids
// over the table.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

// Item i = (parent p, face j) of K-simplices given as (n, K+1) ascending rows;
// n_dev (if set) overrides n with a count computed on the device.
template <int K>
__global__ void k_face_insert(const int32_t* parents, int64_t n, const int32_t* n_dev, int32_t nv,
                              unsigned long long* keys, uint32_t* owner, int64_t mask, int32_t* slot_of,
                              uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    const int64_t cnt = n_dev ? *n_dev : n;
    if (i >= cnt * (K + 1)) {
        if (i < n * (K + 1)) slot_of[i] = -1;
        return;
    }
    const int64_t p = i / (K + 1);
    const int j = static_cast<int>(i - p * (K + 1));
    const int32_t* row = parents + p * (K + 1);
    int32_t v[K + 1];
    bool ok = true;
#pragma unroll
    for (int t = 0; t <= K; ++t) {
        v[t] = row[t];
        ok &= v[t] >= 0 && v[t] < nv && (t == 0 || v[t] > v[t - 1]);
    }
    slot_of[i] = -1;
    if (!ok) {
        if (j == 0) atomicOr(flags, FLAG_RANGE);
        return;
    }
    unsigned long long key = 0;
#pragma unroll
    for (int t = 0; t <= K; ++t)
        if (t != j) key = (key << kVertexBits) | static_cast<unsigned long long>(v[t]);
    int64_t h = static_cast<int64_t>(mix64(key) & static_cast<unsigned long long>(mask));
    for (int64_t probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(&keys[h], kEmptyKey, key);
        if (prev == kEmptyKey || prev == key) {
            atomicMin(&owner[h], static_cast<uint32_t>(i));
            slot_of[i] = static_cast<int32_t>(h);
            return;
        }
        h = (h + 1) & mask;
    }
    atomicOr(flags, FLAG_INTERNAL);  // table full: cannot happen at load <= 1/2
}

__global__ void k_face_owner_flags(const int32_t* slot_of, int64_t n_items, const uint32_t* owner,
                                   int32_t* is_owner) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n_items) return;
    const int32_t h = slot_of[i];
    is_owner[i] = (h >= 0 && owner[h] == static_cast<uint32_t>(i)) ? 1 : 0;
}

// Faces (K vertices each) written by their owners at row rows[owner]; every
// item writes its parent's facet column j.
template <int K>
__global__ void k_face_emit(const int32_t* parents, int64_t n_items, const int32_t* slot_of, const uint32_t* owner,
                            const int32_t* rows, int32_t* faces, int32_t* parent_facets) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n_items) return;
    const int32_t h = slot_of[i];
    if (h < 0) return;
    const uint32_t o = owner[h];
    const int32_t r = rows[o];
    parent_facets[i] = r;  // item i = p * (K+1) + j is exactly facets[p][j]
    if (o != static_cast<uint32_t>(i)) return;
    const int64_t p = i / (K + 1);
    const int j = static_cast<int>(i - p * (K + 1));
    int c = 0;
#pragma unroll
    for (int t = 0; t <= K; ++t)
        if (t != j) faces[int64_t(r) * K + c++] = parents[p * (K + 1) + t];
}

// Dropping vertex 0 of an edge (a, b) leaves b, dropping vertex 1 leaves a.
__global__ void k_edge_facets(const int32_t* edges, const int32_t* n_edges, int32_t* edge_facets) {
    const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (e >= *n_edges) return;
    edge_facets[2 * e] = edges[2 * e + 1];
    edge_facets[2 * e + 1] = edges[2 * e];
}

int64_t table_size(int64_t items) {
    int64_t cap = 1024;
    while (cap < 2 * items) cap <<= 1;
    return cap;
}

unsigned grid_of(int64_t n) { return static_cast<unsigned>(ceil_div(std::max<int64_t>(n, 1), 256)); }

// One level: faces of the K-simplices `parents` (count n, or *n_dev if set),
// into faces (capacity max_faces x K) and parent_facets (n x (K+1)); the face
// count lands in *n_faces_dev.
template <int K>
int face_level(const int32_t* parents, int64_t n, const int32_t* n_dev, int32_t nv, int64_t max_faces,
               int32_t* faces, int32_t* parent_facets, int32_t** n_faces_dev, uint32_t* flags, cudaStream_t s,
               Scratch& scr) {
    const int64_t items = n * (K + 1);
    const int64_t cap = table_size(max_faces);
    unsigned long long* keys;
    uint32_t* owner;
    int32_t *slot_of, *is_owner, *rows;
    int rc;
    if ((rc = scr.alloc(&keys, cap)) || (rc = scr.alloc(&owner, cap)) || (rc = scr.alloc(&slot_of, items)) ||
        (rc = scr.alloc(&is_owner, items)) || (rc = scr.alloc(&rows, items + 1)))
        return rc;
    FLOOD_CUDA(cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * cap, s));
    FLOOD_CUDA(cudaMemsetAsync(owner, 0xff, sizeof(uint32_t) * cap, s));
    k_face_insert<K><<<grid_of(items), 256, 0, s>>>(parents, n, n_dev, nv, keys, owner, cap - 1, slot_of, flags);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    k_face_owner_flags<<<grid_of(items), 256, 0, s>>>(slot_of, items, owner, is_owner);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    if ((rc = exclusive_scan(is_owner, rows, items, s, scr))) return rc;
    k_face_emit<K><<<grid_of(items), 256, 0, s>>>(parents, items, slot_of, owner, rows, faces, parent_facets);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    *n_faces_dev = rows + items;
    return FLOOD_OK;
}

}  // namespace
}  // namespace flood

using namespace flood;

extern "C" int flood_complex_faces(const int32_t* tets, int64_t n_tets, int32_t n_vertices, int32_t* triangles,
                                   int32_t* edges, int32_t* tet_facets, int32_t* triangle_facets,
                                   int32_t* edge_facets, int64_t* n_triangles, int64_t* n_edges, void* stream) {
    if (n_tets < 0 || n_tets > (int64_t(1) << 24) || n_vertices < 1 || n_vertices >= (1 << kVertexBits) ||
        !n_triangles || !n_edges ||
        (n_tets > 0 && (!tets || !triangles || !edges || !tet_facets || !triangle_facets))) {
        set_error("flood_complex_faces: NULL output or sizes out of range (n_tets <= 2^24, n_vertices < 2^21)");
        return FLOOD_EINVAL;
    }
    *n_triangles = 0;
    *n_edges = 0;
    if (n_tets == 0) return FLOOD_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch scr(s);
    uint32_t* flags;
    int rc;
    if ((rc = scr.alloc(&flags, 1))) return rc;
    FLOOD_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
    // at most 4 distinct triangles and 6 distinct edges per tetrahedron
    int32_t *n_tri_dev, *n_edge_dev;
    if ((rc = face_level<3>(tets, n_tets, nullptr, n_vertices, 4 * n_tets, triangles, tet_facets, &n_tri_dev, flags,
                            s, scr)))
        return rc;
    if ((rc = face_level<2>(triangles, 4 * n_tets, n_tri_dev, n_vertices, 6 * n_tets, edges, triangle_facets,
                            &n_edge_dev, flags, s, scr)))
        return rc;
    if (edge_facets) {
        k_edge_facets<<<grid_of(6 * n_tets), 256, 0, s>>>(edges, n_edge_dev, edge_facets);
        note_launch();
        FLOOD_CUDA(cudaGetLastError());
    }
    int32_t counts[2] = {0, 0};
    FLOOD_CUDA(cudaMemcpyAsync(&counts[0], n_tri_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    FLOOD_CUDA(cudaMemcpyAsync(&counts[1], n_edge_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    if ((rc = finish(s, flags, "flood_complex_faces"))) return rc;
    *n_triangles = counts[0];
    *n_edges = counts[1];
    return FLOOD_OK;
}
