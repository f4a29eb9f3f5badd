// flood_persistence: persistence pairs of the flood filtration, on the device (§2).
//
// The flood values make Del(L) a filtered complex; its persistence diagrams
// (§2) come from the Z/2 reduction of the boundary matrix with simplices in
// filtration order: by value, then dimension, then lexicographic vertex ids
// (faces before cofaces on ties). This file computes that pairing on the GPU.
//
//   1. order   per dimension, a bitonic sort of (value bits, vertex ids) gives
//              every simplex its position; keys are unique, so the sort is
//              deterministic;
//   2. reduce  by decreasing dimension (the twist order). The columns of
//              dimension k, boundaries as sorted lists of positions of
//              dimension k-1, are reduced in parallel rounds: every non-zero
//              column finds the earliest column with the same pivot (its
//              largest row), and every other column with that pivot adds it
//              (symmetric difference of the two lists). Adding an earlier
//              column to a later one is a step of the standard column
//              reduction, and every reduced matrix reached by such steps has
//              the same pivots, so the pairs equal those of the sequential
//              reduction. Rounds end when all pivots are distinct;
//   3. clear   a simplex that is the pivot of a reduced column of dimension
//              k+1 creates a class, so its own column would reduce to zero:
//              it is skipped in dimension k.
// The tetrahedra are reduced on the anti-transposed matrix instead (columns:
// the triangles in reverse order, entries: the tetrahedra that contain them,
// in reverse order), whose pairs are the same (the pairing of a filtration
// and of its coboundary matrix agree). Its columns have at most two entries
// in a triangulated region of space and reduce like a graph's edges, in few
// rounds; the boundary columns of the tetrahedra of a void would need a
// round per step of a chain as long as the void's tetrahedra.
// Columns live in one pool of int32 rows; a sum is written to fresh space
// (an atomic bump of the pool head), and a full pool is compacted into a
// larger one between rounds.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "scan.cuh"

namespace flood {
namespace {

constexpr int kThreads = 256;
constexpr int kRoundsPerCheck = 8;
constexpr int kMaxRounds = 1 << 20;

struct Key {
    unsigned long long hi, lo;
};

__device__ __forceinline__ bool key_less(const Key& a, const Key& b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// (value bits, v0, v1, v2, v3), 32 + 4 x 21 bits, most significant first.
// Values are non-negative, so their bit patterns order like the values.
__global__ void k_order_keys(int k, int64_t n, int64_t n_pad, const int32_t* simplices, const float* values,
                             Key* keys, int32_t* idx, uint32_t* flags) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n_pad) return;
    if (i >= n) {
        keys[i] = Key{~0ull, ~0ull};
        idx[i] = -1;
        return;
    }
    unsigned long long v[4] = {0, 0, 0, 0};
    for (int j = 0; j <= k; ++j) {
        const int32_t id = k == 0 ? static_cast<int32_t>(i) : simplices[i * (k + 1) + j];
        if (id < 0 || id >= (1 << 21)) atomicOr(flags, FLAG_RANGE);
        v[j] = static_cast<unsigned long long>(id) & 0x1fffffull;
    }
    const float f = values[i];
    if (!(f >= 0.0f) || isinf(f)) atomicOr(flags, FLAG_NONFINITE);
    const unsigned long long fb = f > 0.0f ? __float_as_uint(f) : 0u;  // -0 and +0 are the same value
    keys[i] = Key{(fb << 32) | (v[0] << 11) | (v[1] >> 10), ((v[1] & 1023ull) << 54) | (v[2] << 33) | (v[3] << 12)};
    idx[i] = static_cast<int32_t>(i);
}

// One compare-exchange stage of a bitonic sort (ascending) over n_pad = 2^p keys.
__global__ void k_bitonic(Key* keys, int32_t* idx, int64_t n_pad, int64_t j, int64_t kk) {
    const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (i >= n_pad) return;
    const int64_t l = i ^ j;
    if (l <= i) return;
    const bool up = (i & kk) == 0;
    const Key a = keys[i], b = keys[l];
    if (key_less(b, a) == up) {
        keys[i] = b;
        keys[l] = a;
        const int32_t t = idx[i];
        idx[i] = idx[l];
        idx[l] = t;
    }
}

__global__ void k_positions(const int32_t* order, int64_t n, int32_t* pos) {
    const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (p < n) pos[order[p]] = static_cast<int32_t>(p);
}

// Column c (position c of dimension k): the positions of its k+1 facets,
// ascending; empty if cleared (its simplex is the pivot of a higher column).
__global__ void k_init_columns(int k, int64_t n, const int32_t* order_k, const int32_t* simplices,
                               const int32_t* facets, const int32_t* pos_lower, int64_t n_lower,
                               const uint8_t* cleared, int32_t* pool, int32_t* off, int32_t* len, uint32_t* flags) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= n) return;
    const int32_t r = order_k[c];
    int32_t e[4] = {0, 0, 0, 0};
    for (int j = 0; j <= k; ++j) {
        // an edge's facets are its vertices; higher simplices list facet rows
        const int32_t t = k == 1 ? simplices[int64_t(r) * 2 + j] : facets[int64_t(r) * (k + 1) + j];
        if (t < 0 || t >= n_lower) {
            atomicOr(flags, FLAG_RANGE);
            e[j] = 0;
        } else {
            e[j] = pos_lower[t];
        }
    }
    for (int a = 1; a <= k; ++a)  // insertion sort of at most four entries
        for (int b = a; b > 0 && e[b - 1] > e[b]; --b) {
            const int32_t t = e[b];
            e[b] = e[b - 1];
            e[b - 1] = t;
        }
    off[c] = static_cast<int32_t>(c * (k + 1));
    for (int j = 0; j <= k; ++j) pool[c * (k + 1) + j] = e[j];
    len[c] = cleared && cleared[c] ? 0 : k + 1;
}

// Coboundary columns of the triangles (the anti-transposed boundary matrix of
// the tetrahedra): per triangle position, the reversed positions n3-1-p of
// the tetrahedra that contain it.
__global__ void k_count_cofaces(int64_t n3, const int32_t* facets3, const int32_t* pos2, int64_t n2, int32_t* cnt,
                                uint32_t* flags) {
    const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (t >= n3) return;
    for (int j = 0; j < 4; ++j) {
        const int32_t f = facets3[t * 4 + j];
        if (f < 0 || f >= n2) {
            atomicOr(flags, FLAG_RANGE);
            continue;
        }
        atomicAdd(&cnt[pos2[f]], 1);
    }
}

__global__ void k_fill_cofaces(int64_t n3, const int32_t* facets3, const int32_t* pos2, int64_t n2,
                               const int32_t* pos3, const int32_t* ptr, int32_t* fill, int32_t* entries) {
    const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (t >= n3) return;
    const int32_t rev = static_cast<int32_t>(n3 - 1 - pos3[t]);
    for (int j = 0; j < 4; ++j) {
        const int32_t f = facets3[t * 4 + j];
        if (f < 0 || f >= n2) continue;
        const int32_t p = pos2[f];
        entries[ptr[p] + atomicAdd(&fill[p], 1)] = rev;
    }
}

// Column c of the coboundary matrix is triangle position n2-1-c: its entries
// sorted in place (a triangle has few cofaces); cleared columns are empty.
__global__ void k_init_coface_columns(int64_t n2, const int32_t* ptr, int32_t* pool, int32_t* off, int32_t* len) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= n2) return;
    const int64_t p = n2 - 1 - c;
    const int32_t b = ptr[p], e = ptr[p + 1];
    for (int32_t a = b + 1; a < e; ++a)
        for (int32_t q = a; q > b && pool[q - 1] > pool[q]; --q) {
            const int32_t t = pool[q];
            pool[q] = pool[q - 1];
            pool[q - 1] = t;
        }
    off[c] = b;
    len[c] = e - b;
}

// Round r, first half: the earliest column holding each pivot. owner[row] =
// (r << 32) | (0xffffffff - column), so the latest round wins and, within a
// round, the smallest column.
__global__ void k_round_owner(int64_t n, const int32_t* pool, const int32_t* off, const int32_t* len,
                              unsigned long long* owner, uint32_t r, int64_t n_rows, uint32_t* flags) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= n || len[c] == 0) return;
    const int32_t low = pool[off[c] + len[c] - 1];
    if (FLOOD_OOB(low, n_rows, flags)) return;
    atomicMax(&owner[low], (static_cast<unsigned long long>(r) << 32) | (0xffffffffu - static_cast<uint32_t>(c)));
}

// Second half: every column whose pivot belongs to an earlier column adds
// that column (the earlier one is not changed in this round: it owns its
// pivot). flags[0]: a column changed; flags[1]: the pool was full (the
// column keeps its list for a later round).
__global__ void k_round_add(int64_t n, int32_t* pool, int64_t pool_cap, unsigned long long* head, int32_t* off,
                            int32_t* len, const unsigned long long* owner, uint32_t* flags) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= n) return;
    const int32_t la = len[c];
    if (la == 0) return;
    const int32_t* A = pool + off[c];
    const int32_t low = A[la - 1];
    const int64_t o = 0xffffffffu - static_cast<uint32_t>(owner[low]);
    if (o == c) return;
    const int32_t lb = len[o];
    const int32_t* B = pool + off[o];
    const unsigned long long at = atomicAdd(head, static_cast<unsigned long long>(la + lb));
    if (at + la + lb > static_cast<unsigned long long>(pool_cap)) {
        atomicOr(&flags[1], 1u);
        return;
    }
    int32_t* D = pool + at;
    int32_t i = 0, j = 0, m = 0;
    while (i < la && j < lb) {
        const int32_t x = A[i], y = B[j];
        if (x < y) {
            D[m++] = x;
            ++i;
        } else if (y < x) {
            D[m++] = y;
            ++j;
        } else {  // equal rows cancel (Z/2)
            ++i;
            ++j;
        }
    }
    while (i < la) D[m++] = A[i++];
    while (j < lb) D[m++] = B[j++];
    off[c] = static_cast<int32_t>(at);
    len[c] = m;
    flags[0] = 1u;
}

// Move every column to the front of a fresh pool (offsets from a scan of the lengths).
__global__ void k_compact(int64_t n, const int32_t* pool, const int32_t* off, const int32_t* len,
                          const int32_t* new_off, int32_t* new_pool) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= n) return;
    const int32_t* a = pool + off[c];
    int32_t* d = new_pool + new_off[c];
    for (int32_t i = 0; i < len[c]; ++i) d[i] = a[i];
}

// After the rounds: the pivot of each column (-1: zero column), which marks
// the lower simplex as cleared (a birth), and whether the column is a pair.
__global__ void k_pivots(int64_t n, const int32_t* pool, const int32_t* off, const int32_t* len, int32_t* low,
                         uint8_t* cleared_lower, int32_t* is_pair) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= n) return;
    const int32_t l = len[c] > 0 ? pool[off[c] + len[c] - 1] : -1;
    low[c] = l;
    is_pair[c] = l >= 0;
    if (l >= 0) cleared_lower[l] = 1;
}

__global__ void k_emit_pairs(int64_t n, const int32_t* low, const int32_t* at, const int32_t* order_lower,
                             const int32_t* order_k, int32_t* pairs) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= n || low[c] < 0) return;
    pairs[2 * int64_t(at[c])] = order_lower[low[c]];
    pairs[2 * int64_t(at[c]) + 1] = order_k[c];
}

// Essential classes of dimension d: positions that are not the pivot of a
// higher column (not cleared) and whose own column is zero (every vertex's is).
__global__ void k_essential_flags(int64_t n, const uint8_t* cleared, const int32_t* low_own, int32_t* flag) {
    const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (p >= n) return;
    flag[p] = !(cleared && cleared[p]) && (!low_own || low_own[p] < 0);
}

__global__ void k_emit_rows(int64_t n, const int32_t* flag, const int32_t* at, const int32_t* order, int32_t* out) {
    const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (p < n && flag[p]) out[at[p]] = order[p];
}

inline unsigned blocks_for(int64_t n) { return static_cast<unsigned>(std::max<int64_t>(1, ceil_div(n, kThreads))); }

int64_t pow2_at_least(int64_t n) {
    int64_t p = 1;
    while (p < n) p <<= 1;
    return p;
}

// Positions of dimension k: order[p] = row at position p, pos[row] = p.
int order_dimension(int k, int64_t n, const int32_t* simplices, const float* values, int32_t* order, int32_t* pos,
                    uint32_t* flags, cudaStream_t s, Scratch& scr) {
    if (n == 0) return FLOOD_OK;
    const int64_t n_pad = pow2_at_least(n);
    Key* keys;
    int32_t* idx;
    int rc;
    if ((rc = scr.alloc(&keys, n_pad)) || (rc = scr.alloc(&idx, n_pad))) return rc;
    k_order_keys<<<blocks_for(n_pad), kThreads, 0, s>>>(k, n, n_pad, simplices, values, keys, idx, flags);
    note_launch();
    int stages = 0;
    for (int64_t kk = 2; kk <= n_pad; kk <<= 1)
        for (int64_t j = kk >> 1; j > 0; j >>= 1) {
            k_bitonic<<<blocks_for(n_pad), kThreads, 0, s>>>(keys, idx, n_pad, j, kk);
            ++stages;
        }
    note_launch(stages);
    FLOOD_CUDA(cudaMemcpyAsync(order, idx, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
    k_positions<<<blocks_for(n), kThreads, 0, s>>>(order, n, pos);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

// Columns in one pool: column c is pool[off[c], off[c] + len[c]), ascending.
struct Columns {
    int32_t *pool = nullptr, *off = nullptr, *len = nullptr;
    int64_t n = 0, cap = 0, used = 0;
};

// Boundary columns of dimension k (rows: positions of dimension k-1), with
// the columns of `cleared` positions empty.
int facet_columns(int k, int64_t n, int64_t n_lower, const int32_t* order_k, const int32_t* simplices,
                  const int32_t* facets, const int32_t* pos_lower, const uint8_t* cleared, uint32_t* flags,
                  cudaStream_t s, Scratch& scr, Columns* C) {
    C->n = n;
    C->used = n * (k + 1);
    C->cap = C->used * 8 + (int64_t(1) << 20);
    int rc;
    if ((rc = scr.alloc(&C->pool, C->cap)) || (rc = scr.alloc(&C->off, n)) || (rc = scr.alloc(&C->len, n))) return rc;
    k_init_columns<<<blocks_for(n), kThreads, 0, s>>>(k, n, order_k, simplices, facets, pos_lower, n_lower, cleared,
                                                      C->pool, C->off, C->len, flags);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

// Coboundary columns of the triangles (rows: reversed tetrahedron positions).
int coface_columns(int64_t n2, int64_t n3, const int32_t* facets3, const int32_t* pos2, const int32_t* pos3,
                   uint32_t* flags, cudaStream_t s, Scratch& scr, Columns* C) {
    int32_t *cnt, *ptr;
    int rc;
    if ((rc = scr.alloc(&cnt, n2)) || (rc = scr.alloc(&ptr, n2 + 1))) return rc;
    FLOOD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n2, s));
    k_count_cofaces<<<blocks_for(n3), kThreads, 0, s>>>(n3, facets3, pos2, n2, cnt, flags);
    note_launch();
    if ((rc = exclusive_scan(cnt, ptr, n2, s, scr))) return rc;
    C->n = n2;
    C->used = 4 * n3;  // every tetrahedron lists each of its 4 facets once
    C->cap = C->used * 8 + (int64_t(1) << 20);
    if ((rc = scr.alloc(&C->pool, C->cap)) || (rc = scr.alloc(&C->off, n2)) || (rc = scr.alloc(&C->len, n2)))
        return rc;
    FLOOD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * n2, s));
    k_fill_cofaces<<<blocks_for(n3), kThreads, 0, s>>>(n3, facets3, pos2, n2, pos3, ptr, cnt, C->pool);
    k_init_coface_columns<<<blocks_for(n2), kThreads, 0, s>>>(n2, ptr, C->pool, C->off, C->len);
    note_launch(2);
    FLOOD_CUDA(cudaGetLastError());
    return FLOOD_OK;
}

// Reduce the columns (rows 0..n_rows-1) by parallel rounds; low[c] receives
// each column's final pivot (-1: zero column) and marked[row] = 1 for every
// pivot row. Synchronises `s` every few rounds.
int reduce_columns(Columns& C, int64_t n_rows, int32_t* low, uint8_t* marked, int32_t* is_pair,
                   int64_t* rounds_out, uint32_t* flags, cudaStream_t s, Scratch& scr) {
    const int64_t n = C.n;
    *rounds_out = 0;
    if (n == 0) return FLOOD_OK;
    unsigned long long *owner, *head;
    uint32_t* rflags;  // [0] changed in the last round, [1] pool full
    int rc;
    if ((rc = scr.alloc(&owner, std::max<int64_t>(n_rows, 1))) || (rc = scr.alloc(&head, 1)) ||
        (rc = scr.alloc(&rflags, 2)))
        return rc;
    FLOOD_CUDA(cudaMemsetAsync(owner, 0, sizeof(unsigned long long) * std::max<int64_t>(n_rows, 1), s));
    FLOOD_CUDA(cudaMemsetAsync(rflags, 0, 2 * sizeof(uint32_t), s));
    const unsigned long long used = static_cast<unsigned long long>(C.used);
    FLOOD_CUDA(cudaMemcpyAsync(head, &used, sizeof(used), cudaMemcpyHostToDevice, s));
    uint32_t r = 0;
    for (;;) {
        for (int i = 0; i < kRoundsPerCheck; ++i) {
            ++r;
            FLOOD_CUDA(cudaMemsetAsync(rflags, 0, sizeof(uint32_t), s));
            k_round_owner<<<blocks_for(n), kThreads, 0, s>>>(n, C.pool, C.off, C.len, owner, r, n_rows, flags);
            k_round_add<<<blocks_for(n), kThreads, 0, s>>>(n, C.pool, C.cap, head, C.off, C.len, owner, rflags);
            note_launch(2);
        }
        FLOOD_CUDA(cudaGetLastError());
        uint32_t h[2];
        FLOOD_CUDA(cudaMemcpyAsync(h, rflags, sizeof(h), cudaMemcpyDeviceToHost, s));
        FLOOD_CUDA(cudaStreamSynchronize(s));
        if (h[1]) {  // pool full: compact the live columns into a pool twice as large
            int32_t *new_off, *new_pool;
            if ((rc = scr.alloc(&new_off, n + 1))) return rc;
            if ((rc = exclusive_scan(C.len, new_off, n, s, scr))) return rc;
            int32_t h_live = 0;
            FLOOD_CUDA(cudaMemcpyAsync(&h_live, new_off + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            FLOOD_CUDA(cudaStreamSynchronize(s));
            const int64_t live = h_live;
            const int64_t new_cap = std::max<int64_t>(2 * C.cap, 4 * live + (int64_t(1) << 20));
            if (new_cap >= (int64_t(1) << 31)) {
                set_error("flood_persistence: reduced columns exceed 2^31 entries");
                return FLOOD_ECAPACITY;
            }
            if ((rc = scr.alloc(&new_pool, new_cap))) return rc;
            k_compact<<<blocks_for(n), kThreads, 0, s>>>(n, C.pool, C.off, C.len, new_off, new_pool);
            note_launch();
            FLOOD_CUDA(cudaMemcpyAsync(C.off, new_off, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
            const unsigned long long nh = static_cast<unsigned long long>(live);
            FLOOD_CUDA(cudaMemcpyAsync(head, &nh, sizeof(nh), cudaMemcpyHostToDevice, s));
            FLOOD_CUDA(cudaMemsetAsync(rflags, 0, 2 * sizeof(uint32_t), s));
            C.pool = new_pool;
            C.cap = new_cap;
            FLOOD_CUDA(cudaStreamSynchronize(s));  // the host values above are copied before they go out of scope
            continue;
        }
        if (!h[0]) break;  // the last round changed nothing: every pivot is distinct
        if (r >= kMaxRounds) {
            set_error("flood_persistence: the reduction did not settle within %d rounds", kMaxRounds);
            return FLOOD_EINTERNAL;
        }
    }
    k_pivots<<<blocks_for(n), kThreads, 0, s>>>(n, C.pool, C.off, C.len, low, marked, is_pair);
    note_launch();
    FLOOD_CUDA(cudaGetLastError());
    *rounds_out = r;
    return FLOOD_OK;
}

// Pairs of the coboundary reduction, per tetrahedron position: the
// triangle it kills (its column's partner), or nothing.
__global__ void k_coface_pairs(int64_t n2, int64_t n3, const int32_t* low, int32_t* tri_of_tet, uint8_t* cleared2) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= n2 || low[c] < 0) return;
    const int64_t p2 = n2 - 1 - c, p3 = n3 - 1 - low[c];
    tri_of_tet[p3] = static_cast<int32_t>(p2);
    cleared2[p2] = 1;  // a triangle whose class a tetrahedron kills is a birth: its own column is zero
}

__global__ void k_tet_pair_flags(int64_t n3, const int32_t* tri_of_tet, int32_t* low3, int32_t* is_pair) {
    const int64_t p = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (p >= n3) return;
    low3[p] = tri_of_tet[p];
    is_pair[p] = tri_of_tet[p] >= 0;
}

}  // namespace
}  // namespace flood

using namespace flood;

extern "C" int flood_persistence(const int32_t* const simplices[4], const int32_t* const facets[4],
                                 const int64_t n_simplices[4], const float* const values[4],
                                 int32_t* const pairs[3], int64_t n_pairs[3], int32_t* const essential[4],
                                 int64_t n_essential[4], int64_t rounds[4], void* stream) {
    if (!simplices || !facets || !n_simplices || !values || !pairs || !n_pairs || !essential || !n_essential) {
        set_error("flood_persistence: NULL argument");
        return FLOOD_EINVAL;
    }
    int64_t n[4];
    for (int k = 0; k < 4; ++k) {
        n[k] = n_simplices[k];
        if (n[k] < 0 || n[k] >= (int64_t(1) << 30) || (n[k] > 0 && (!values[k] || !essential[k]))) {
            set_error("flood_persistence: n_simplices[%d] out of range or values/essential[%d] NULL", k, k);
            return FLOOD_EINVAL;
        }
        if (k >= 1 && n[k] > 0 && (!simplices[k] || (k >= 2 && !facets[k]) || !pairs[k - 1] || n[k - 1] == 0)) {
            set_error("flood_persistence: dimension %d needs simplices, facets (k >= 2), pairs[%d] and dimension %d",
                      k, k - 1, k - 1);
            return FLOOD_EINVAL;
        }
    }
    if (n[0] >= (int64_t(1) << 21)) {
        set_error("flood_persistence: at most 2^21 - 1 vertices");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = pending_error(s)) return rc;
    Scratch scr(s);
    uint32_t* flags;
    int rc;
    if ((rc = scr.alloc(&flags, 1))) return rc;
    FLOOD_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
    int32_t *order[4], *pos[4], *low[4], *is_pair[4], *at[4];
    uint8_t* cleared[4];
    for (int k = 0; k < 4; ++k) {
        order[k] = pos[k] = low[k] = is_pair[k] = at[k] = nullptr;
        cleared[k] = nullptr;
        if (n[k] == 0) continue;
        if ((rc = scr.alloc(&order[k], n[k])) || (rc = scr.alloc(&pos[k], n[k])) || (rc = scr.alloc(&low[k], n[k])) ||
            (rc = scr.alloc(&is_pair[k], n[k])) || (rc = scr.alloc(&at[k], n[k] + 1)) ||
            (rc = scr.alloc(&cleared[k], n[k])))
            return rc;
        FLOOD_CUDA(cudaMemsetAsync(cleared[k], 0, n[k], s));
        if ((rc = order_dimension(k, n[k], simplices[k], values[k], order[k], pos[k], flags, s, scr))) return rc;
    }
    // an input error (ids, values) must not reach the reduction
    uint32_t h_flags = 0;
    FLOOD_CUDA(cudaMemcpyAsync(&h_flags, flags, sizeof(h_flags), cudaMemcpyDeviceToHost, s));
    FLOOD_CUDA(cudaStreamSynchronize(s));
    if (h_flags) return status_from_flags(h_flags, "flood_persistence");
    int64_t r[4] = {0, 0, 0, 0};
    // Tetrahedra: the pairs of the anti-transposed (coboundary) matrix equal
    // those of the boundary matrix, and its columns (the cofaces of each
    // triangle, at most two in a triangulation of a region of space) reduce
    // in few rounds, where the tetrahedra's boundary columns would need a
    // round per step of every long chain of additions.
    if (n[3] > 0) {
        Columns C;
        int32_t *clow, *cpair, *tri_of_tet;
        uint8_t* cmark;
        if ((rc = scr.alloc(&clow, n[2])) || (rc = scr.alloc(&cpair, n[2])) || (rc = scr.alloc(&tri_of_tet, n[3])) ||
            (rc = scr.alloc(&cmark, n[3])))
            return rc;
        FLOOD_CUDA(cudaMemsetAsync(tri_of_tet, 0xff, sizeof(int32_t) * n[3], s));
        if ((rc = coface_columns(n[2], n[3], facets[3], pos[2], pos[3], flags, s, scr, &C)) ||
            (rc = reduce_columns(C, n[3], clow, cmark, cpair, &r[3], flags, s, scr)))
            return rc;
        k_coface_pairs<<<blocks_for(n[2]), kThreads, 0, s>>>(n[2], n[3], clow, tri_of_tet, cleared[2]);
        k_tet_pair_flags<<<blocks_for(n[3]), kThreads, 0, s>>>(n[3], tri_of_tet, low[3], is_pair[3]);
        note_launch(2);
        FLOOD_CUDA(cudaGetLastError());
    }
    for (int k = 2; k >= 1; --k) {  // twist: higher dimensions first, their pivots cleared below
        if (n[k] == 0) continue;
        Columns C;
        if ((rc = facet_columns(k, n[k], n[k - 1], order[k], simplices[k], facets[k], pos[k - 1], cleared[k], flags, s,
                                scr, &C)) ||
            (rc = reduce_columns(C, n[k - 1], low[k], cleared[k - 1], is_pair[k], &r[k], flags, s, scr)))
            return rc;
    }
    // pairs (birth row of dimension k-1, death row of dimension k), in the deaths' filtration order
    for (int k = 1; k <= 3; ++k) {
        n_pairs[k - 1] = 0;
        if (n[k] == 0) continue;
        if ((rc = exclusive_scan(is_pair[k], at[k], n[k], s, scr))) return rc;
        int32_t cnt = 0;
        FLOOD_CUDA(cudaMemcpyAsync(&cnt, at[k] + n[k], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        k_emit_pairs<<<blocks_for(n[k]), kThreads, 0, s>>>(n[k], low[k], at[k], order[k - 1], order[k], pairs[k - 1]);
        note_launch();
        FLOOD_CUDA(cudaStreamSynchronize(s));
        n_pairs[k - 1] = cnt;
    }
    // essential classes per dimension, in filtration order
    for (int d = 0; d < 4; ++d) {
        n_essential[d] = 0;
        if (n[d] == 0) continue;
        int32_t* flag;
        if ((rc = scr.alloc(&flag, n[d]))) return rc;
        k_essential_flags<<<blocks_for(n[d]), kThreads, 0, s>>>(n[d], cleared[d], d >= 1 ? low[d] : nullptr, flag);
        note_launch();
        if ((rc = exclusive_scan(flag, at[d], n[d], s, scr))) return rc;
        int32_t cnt = 0;
        FLOOD_CUDA(cudaMemcpyAsync(&cnt, at[d] + n[d], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        k_emit_rows<<<blocks_for(n[d]), kThreads, 0, s>>>(n[d], flag, at[d], order[d], essential[d]);
        note_launch();
        FLOOD_CUDA(cudaStreamSynchronize(s));
        n_essential[d] = cnt;
    }
    if (rounds)
        for (int k = 0; k < 4; ++k) rounds[k] = r[k];
    return finish(s, flags, "flood_persistence");
}
