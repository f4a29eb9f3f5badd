// flood_filtration_masked: the paper's own evaluation of the flood values,
// re-implemented on this GPU as a comparator for the pruned path.
//
// §4.2 and App. A.1 evaluate, for every simplex sigma, the full barycentric
// grid P_sigma of Lemma 1 (faces included) against the points of X inside the
// masking ball B(c, sqrt(2) r) of Lemma 2 (c the midpoint of the longest
// edge, r the largest distance from c to a vertex; radius r for an edge), and
// take f(sigma) = max over samples of the minimum over masked points. Lemma 2
// (which needs L ⊂ X) makes the masked minimum exact. Nothing is pruned and
// no facet values are reused: every (sample, masked point) pair is evaluated.
// One CTA per simplex: the cell grid supplies the candidate rows of the
// ball's bounding box, the ball test (the mask) compacts them into a
// shared-memory tile, and the threads split (sample, point) pairs: each
// thread keeps register minima for its samples over its share of the tile's
// points, combined across threads in shared memory at the end.
#include "geometry.cuh"

namespace flood {
namespace {

constexpr int kMThreads = 256;
constexpr int kMTile = 1536;  // masked points staged per round (static shared memory < 48 KB)
constexpr int kMaxFull = 1024;  // full-grid samples per simplex held in shared memory
constexpr int kSlots = 4;       // samples per thread

struct MaskedArgs {
    int k;
    int64_t n;
    const int32_t* simplices;
    const float* L;
    int32_t n_L;
    const float* vbound;
    const uint8_t* comp;  // full-grid compositions (F, k+1), lexicographic
    int F;
    float m;
    const GridView* gp;  // device copy of the grid's view
    float* val;
    uint32_t* flags;
    unsigned long long* pairs;
};

__global__ void __launch_bounds__(kMThreads) k_masked(MaskedArgs a) {
    __shared__ float4 s_pts[kMTile];
    __shared__ float s_px[kMaxFull], s_py[kMaxFull], s_pz[kMaxFull];
    __shared__ uint32_t s_min[kMaxFull];
    __shared__ int s_cnt;
    __shared__ uint32_t s_max;
    const int tid = threadIdx.x;
    const int k = a.k, F = a.F;
    const GridView g = *a.gp;
    // (sample, point) split: nparts threads share each sample's points
    const int nparts = F >= kMThreads ? 1 : kMThreads / F;
    const int part = tid % nparts, s_first = tid / nparts, s_step = kMThreads / nparts;
    unsigned long long my_pairs = 0;
    for (int64_t w = blockIdx.x; w < a.n; w += gridDim.x) {
        const int32_t* ids = a.simplices + w * (k + 1);
        float V[4][3];
        bool ok = true, member = true;
        for (int j = 0; j <= k; ++j) {
            const int32_t v = ids[j];
            ok &= v >= 0 && v < a.n_L;
            if (v >= 0 && v < a.n_L) {
                member &= a.vbound[v] == 0.0f;  // Lemma 2 needs the vertices to be points of X
                V[j][0] = a.L[3 * v];
                V[j][1] = a.L[3 * v + 1];
                V[j][2] = a.L[3 * v + 2];
            }
        }
        if (!ok || !member) {
            if (tid == 0) {
                atomicOr(a.flags, ok ? FLAG_NOT_SUBSET : FLAG_RANGE);
                a.val[w] = __int_as_float(0x7fc00000);
            }
            continue;  // uniform across the CTA
        }
        // masking ball: midpoint of the longest edge, radius sqrt(2) max_i |c - v_i| (r for an edge)
        int ia = 0, ib = 1;
        float best = -1.0f;
        for (int i = 0; i <= k; ++i)
            for (int j = i + 1; j <= k; ++j) {
                const float dx = V[i][0] - V[j][0], dy = V[i][1] - V[j][1], dz = V[i][2] - V[j][2];
                const float d2 = dx * dx + dy * dy + dz * dz;
                if (d2 > best) {
                    best = d2;
                    ia = i;
                    ib = j;
                }
            }
        const float c[3] = {0.5f * (V[ia][0] + V[ib][0]), 0.5f * (V[ia][1] + V[ib][1]), 0.5f * (V[ia][2] + V[ib][2])};
        float r2 = 0.0f;
        for (int i = 0; i <= k; ++i) {
            const float dx = V[i][0] - c[0], dy = V[i][1] - c[1], dz = V[i][2] - c[2];
            r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
        }
        // ball radius with a relative margin: a slightly larger ball holds the
        // masked set, so the minimum is the same
        const float R2 = (k == 1 ? r2 : 2.0f * r2) * (1.0f + 1.0f / 1024.0f);
        const float R = sqrtf(R2);
        // samples of the full grid (faces included): p = sum_j (c_j / m) v_j
        for (int s = tid; s < F; s += kMThreads) {
            const uint8_t* cc = a.comp + s * (k + 1);
            float x = 0.0f, y = 0.0f, z = 0.0f;
            for (int j = 0; j <= k; ++j) {
                const float lam = __fdiv_rn(static_cast<float>(cc[j]), a.m);
                x = __fmaf_rn(lam, V[j][0], x);
                y = __fmaf_rn(lam, V[j][1], y);
                z = __fmaf_rn(lam, V[j][2], z);
            }
            s_px[s] = x;
            s_py[s] = y;
            s_pz[s] = z;
            s_min[s] = 0x7f800000u;  // +inf
        }
        __syncthreads();
        float mn[kSlots], qx[kSlots], qy[kSlots], qz[kSlots];  // this thread's samples, in registers
#pragma unroll
        for (int q = 0; q < kSlots; ++q) {
            const int sq = s_first + q * s_step;
            mn[q] = INFINITY;
            qx[q] = sq < F ? s_px[sq] : 0.0f;
            qy[q] = sq < F ? s_py[sq] : 0.0f;
            qz[q] = sq < F ? s_pz[sq] : 0.0f;
        }
        const float zero[3] = {0.0f, 0.0f, 0.0f};
        const CellBox b = cull_box(g, c, zero, zero, R);
        const int rows = b.n[1] * b.n[2];
        if (tid == 0) s_cnt = 0;
        __syncthreads();
        // Rows of the ball's box are walked in chunks of kMThreads candidates;
        // a chunk is staged only when the tile has room for all of it, so the
        // tile never overflows. Row state and counts are the same in every
        // thread (read after a barrier), so every barrier is reached by all.
        int r = 0;
        int32_t cur = 0, re = 0;
        if (rows > 0) box_row(g, b, 0, cur, re);
        bool more = rows > 0;
        int cnt = 0;
        for (;;) {
            while (more && cnt <= kMTile - kMThreads) {
                if (cur >= re) {
                    if (++r >= rows) {
                        more = false;
                        break;
                    }
                    box_row(g, b, r, cur, re);
                    continue;
                }
                const int32_t i = cur + tid;
                bool in = false;
                float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (i < re) {
                    x = g.pts[i];
                    const float dx = x.x - c[0], dy = x.y - c[1], dz = x.z - c[2];
                    in = dx * dx + dy * dy + dz * dz <= R2;  // the mask
                }
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                int base = 0;
                if ((tid & 31) == 0 && bal) base = atomicAdd(&s_cnt, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (in) s_pts[base + __popc(bal & ((1u << (tid & 31)) - 1u))] = x;
                cur += kMThreads;
                __syncthreads();
                cnt = s_cnt;
                __syncthreads();
            }
            // every thread: its samples against its share of the staged points
            for (int j = part; j < cnt; j += nparts) {
                const float4 x = s_pts[j];
#pragma unroll
                for (int q = 0; q < kSlots; ++q) {
                    const int s = s_first + q * s_step;
                    if (s < F) {
                        const float dx = __fsub_rn(x.x, qx[q]), dy = __fsub_rn(x.y, qy[q]), dz = __fsub_rn(x.z, qz[q]);
                        mn[q] = fminf(mn[q], __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz))));
                    }
                }
            }
            if (tid == 0) my_pairs += static_cast<unsigned long long>(cnt) * F;
            __syncthreads();
            if (tid == 0) s_cnt = 0;
            cnt = 0;
            __syncthreads();
            if (!more) break;
        }
#pragma unroll
        for (int q = 0; q < kSlots; ++q) {
            const int s = s_first + q * s_step;
            if (s < F && mn[q] < INFINITY) atomicMin(&s_min[s], __float_as_uint(mn[q]));
        }
        if (tid == 0) s_max = 0u;
        __syncthreads();
        for (int s = tid; s < F; s += kMThreads) atomicMax(&s_max, s_min[s]);
        __syncthreads();
        if (tid == 0) a.val[w] = __fsqrt_rn(__uint_as_float(s_max));
        __syncthreads();
    }
    if (tid == 0 && my_pairs) atomicAdd(a.pairs, my_pairs);
}

// |X ∩ B(c, rho)| per simplex, summed per dimension: the masking ball of
// Lemma 2 as k_masked builds it (c the midpoint of the longest edge, rho =
// sqrt(2) max_i |c - v_i|, or that maximum for an edge), without k_masked's
// safety margin. One warp per simplex walks the rows of the ball's cell box.
__global__ void k_ball_counts(int k, int64_t n, const int32_t* simplices, const float* L, int32_t n_L,
                              const GridView* gp, unsigned long long* count, uint32_t* flags) {
    const int64_t w = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const GridView g = *gp;
    const int32_t* ids = simplices + w * (k + 1);
    float V[4][3];
    for (int j = 0; j <= k; ++j) {
        const int32_t v = ids[j];
        if (v < 0 || v >= n_L) {
            if (lane == 0) atomicOr(flags, FLAG_RANGE);
            return;
        }
        V[j][0] = L[3 * v];
        V[j][1] = L[3 * v + 1];
        V[j][2] = L[3 * v + 2];
    }
    int ia = 0, ib = 1;
    float best = -1.0f;
    for (int i = 0; i <= k; ++i)
        for (int j = i + 1; j <= k; ++j) {
            const float dx = V[i][0] - V[j][0], dy = V[i][1] - V[j][1], dz = V[i][2] - V[j][2];
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 > best) {
                best = d2;
                ia = i;
                ib = j;
            }
        }
    const float c[3] = {0.5f * (V[ia][0] + V[ib][0]), 0.5f * (V[ia][1] + V[ib][1]), 0.5f * (V[ia][2] + V[ib][2])};
    float r2 = 0.0f;
    for (int i = 0; i <= k; ++i) {
        const float dx = V[i][0] - c[0], dy = V[i][1] - c[1], dz = V[i][2] - c[2];
        r2 = fmaxf(r2, dx * dx + dy * dy + dz * dz);
    }
    const float R2 = k == 1 ? r2 : 2.0f * r2;
    const float zero[3] = {0.0f, 0.0f, 0.0f};
    const CellBox b = cull_box(g, c, zero, zero, sqrtf(R2));
    const int rows = b.n[1] * b.n[2];
    unsigned long long cnt = 0;
    for (int r = 0; r < rows; ++r) {
        int32_t rb, re;
        box_row(g, b, r, rb, re);
        for (int32_t i = rb + lane; i < re; i += 32) {
            const float4 x = g.pts[i];
            const float dx = x.x - c[0], dy = x.y - c[1], dz = x.z - c[2];
            cnt += dx * dx + dy * dy + dz * dz <= R2;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0 && cnt) atomicAdd(count, cnt);
}

// Full grid of Lemma 1: compositions of m into k+1 parts >= 0, lexicographic.
std::vector<uint8_t> full_table(int m, int k) {
    std::vector<uint8_t> out;
    int c[4] = {0, 0, 0, 0};
    if (k == 1) {
        for (c[0] = 0; c[0] <= m; ++c[0]) out.insert(out.end(), {uint8_t(c[0]), uint8_t(m - c[0])});
    } else if (k == 2) {
        for (c[0] = 0; c[0] <= m; ++c[0])
            for (c[1] = 0; c[0] + c[1] <= m; ++c[1])
                out.insert(out.end(), {uint8_t(c[0]), uint8_t(c[1]), uint8_t(m - c[0] - c[1])});
    } else {
        for (c[0] = 0; c[0] <= m; ++c[0])
            for (c[1] = 0; c[0] + c[1] <= m; ++c[1])
                for (c[2] = 0; c[0] + c[1] + c[2] <= m; ++c[2])
                    out.insert(out.end(),
                               {uint8_t(c[0]), uint8_t(c[1]), uint8_t(c[2]), uint8_t(m - c[0] - c[1] - c[2])});
    }
    return out;
}

}  // namespace
}  // namespace flood

using namespace flood;

extern "C" int flood_filtration_masked(const flood_grid* grid, const float* L, int32_t n_landmarks,
                                       const int32_t* const simplices[4], const int64_t n_simplices[4], int32_t m,
                                       float* const values[4], int64_t* pairs_out, void* stream) {
    if (!grid || !L || n_landmarks < 1 || !simplices || !n_simplices || !values || m < 1) {
        set_error("flood_filtration_masked: NULL argument or m < 1");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = pending_error(s)) return rc;
    Scratch scr(s);
    uint32_t* flags;
    unsigned long long* pairs;
    float *vval, *vbound;
    int32_t* vsrc;
    int rc;
    if ((rc = scr.alloc(&flags, 1)) || (rc = scr.alloc(&pairs, 1)) || (rc = scr.alloc(&vval, n_landmarks)) ||
        (rc = scr.alloc(&vbound, n_landmarks)) || (rc = scr.alloc(&vsrc, 2 * int64_t(n_landmarks))))
        return rc;
    FLOOD_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
    FLOOD_CUDA(cudaMemsetAsync(pairs, 0, sizeof(unsigned long long), s));
    if ((rc = launch_vertices(L, n_landmarks, grid, vval, vsrc, vbound, flags, s))) return rc;
    if (values[0]) FLOOD_CUDA(cudaMemcpyAsync(values[0], vval, sizeof(float) * n_landmarks,
                                              cudaMemcpyDeviceToDevice, s));
    std::vector<uint8_t> tables[4];
    uint8_t* dcomp[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 1; k <= 3; ++k) {
        if (n_simplices[k] <= 0) continue;
        if (!simplices[k] || !values[k]) {
            set_error("flood_filtration_masked: simplices[%d] and values[%d] must be given", k, k);
            return FLOOD_EINVAL;
        }
        tables[k] = full_table(m, k);
        const int F = static_cast<int>(tables[k].size() / (k + 1));
        if (F > kMaxFull || F > kSlots * kMThreads) {
            set_error("flood_filtration_masked: %d full-grid samples per %d-simplex exceed %d", F, k, kMaxFull);
            return FLOOD_EINVAL;
        }
        if ((rc = scr.alloc(&dcomp[k], tables[k].size()))) return rc;
        FLOOD_CUDA(cudaMemcpyAsync(dcomp[k], tables[k].data(), tables[k].size(), cudaMemcpyHostToDevice, s));
        MaskedArgs a{};
        a.k = k;
        a.n = n_simplices[k];
        a.simplices = simplices[k];
        a.L = L;
        a.n_L = n_landmarks;
        a.vbound = vbound;
        a.comp = dcomp[k];
        a.F = F;
        a.m = static_cast<float>(m);
        a.gp = view_of(grid);
        a.val = values[k];
        a.flags = flags;
        a.pairs = pairs;
        const int64_t blocks = std::min<int64_t>(a.n, int64_t(device_sm_count()) * 8);
        k_masked<<<static_cast<unsigned>(blocks), kMThreads, 0, s>>>(a);
        note_launch();
        FLOOD_CUDA(cudaGetLastError());
    }
    unsigned long long h_pairs = 0;
    FLOOD_CUDA(cudaMemcpyAsync(&h_pairs, pairs, sizeof(h_pairs), cudaMemcpyDeviceToHost, s));
    if ((rc = finish(s, flags, "flood_filtration_masked"))) return rc;
    if (pairs_out) *pairs_out = static_cast<int64_t>(h_pairs);
    return FLOOD_OK;
}

extern "C" int flood_masking_ball_counts(const flood_grid* grid, const float* L, int32_t n_landmarks,
                                         const int32_t* const simplices[4], const int64_t n_simplices[4],
                                         int64_t counts_out[4], void* stream) {
    if (!grid || !L || n_landmarks < 1 || !simplices || !n_simplices || !counts_out) {
        set_error("flood_masking_ball_counts: NULL argument or n_landmarks < 1");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (int rc = pending_error(s)) return rc;
    Scratch scr(s);
    uint32_t* flags;
    unsigned long long* cnt;
    int rc;
    if ((rc = scr.alloc(&flags, 1)) || (rc = scr.alloc(&cnt, 4))) return rc;
    FLOOD_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
    FLOOD_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), s));
    for (int k = 1; k <= 3; ++k) {
        if (n_simplices[k] <= 0) continue;
        if (!simplices[k]) {
            set_error("flood_masking_ball_counts: simplices[%d] is NULL", k);
            return FLOOD_EINVAL;
        }
        const unsigned blocks = static_cast<unsigned>(ceil_div(n_simplices[k] * 32, 256));
        k_ball_counts<<<blocks, 256, 0, s>>>(k, n_simplices[k], simplices[k], L, n_landmarks, view_of(grid), cnt + k,
                                             flags);
        note_launch();
        FLOOD_CUDA(cudaGetLastError());
    }
    unsigned long long h[4] = {0, 0, 0, 0};
    FLOOD_CUDA(cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s));
    if ((rc = finish(s, flags, "flood_masking_ball_counts"))) return rc;
    for (int k = 0; k < 4; ++k) counts_out[k] = static_cast<int64_t>(h[k]);
    return FLOOD_OK;
}
