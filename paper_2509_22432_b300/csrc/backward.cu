// flood_filtration_backward: gradient of F = sum_sigma g_sigma f(sigma).
//
// Our derivation from the value definition of §4.1: f(sigma) = |p* - x*| with
// p* = sum_j lambda_j v_j the attaining sample of the attaining simplex tau
// (recorded by the forward call as src; a grid sample of Lemma 1, a point of
// a given set for flood_filtration_given, or a vertex itself) and x* its
// nearest point of X.
// One warp per simplex recomputes p* with the forward arithmetic, finds x*
// among the points of the cells within u_{p*} = min_j (|p* - v_j| + d(v_j, X))
// of p* (a bound on d(p*, X); d(v_j, X) = 0 for landmarks that are points of
// X), ties to the lowest row of X, and scatters
//     grad_X[x*]  += g (x* - p*) / f,    grad_L[v_j] += g lambda_j (p* - x*) / f.
#include <vector>

#include "geometry.cuh"

namespace flood {

namespace {

struct BwdArgs {
    int k;
    int64_t n;
    const float* grad;
    const int32_t* src;      // (n, 2)
    const int32_t* simp[4];  // simplices of every dimension (vertex rows)
    int64_t n_simp[4];
    const uint8_t* comp[4];  // interior composition tables (grid samples)
    const float* w[4];       // given sets: barycentric coordinates (n_k, I[k], k+1)
    int I[4];
    float m;
    const float* L;
    const float* vbound;     // per landmark: d(v, X) rounded up, 0 for a point of X
    int32_t n_L;
    const GridView* gp;      // device copy of the grid's view
    float* grad_X;
    float* grad_L;
    uint32_t* flags;
};

__global__ void __launch_bounds__(256) k_backward(BwdArgs a) {
    const int64_t w = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= a.n) return;
    const GridView g = *a.gp;
    const float gam = a.grad[w];
    if (gam == 0.0f) return;
    const int32_t s0 = a.src[2 * w], sample = a.src[2 * w + 1];
    const int dim = s0 >> 28;
    const int64_t tau = s0 & ((1 << 28) - 1);
    if (dim > 3 || tau >= a.n_simp[dim] || (dim > 0 && (sample < 0 || sample >= a.I[dim]))) {
        if (lane == 0) atomicOr(a.flags, FLAG_RANGE);
        return;
    }
    const int32_t vtx = static_cast<int32_t>(tau);
    const int32_t* ids = dim == 0 ? &vtx : a.simp[dim] + tau * (dim + 1);
    float vb[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    bool members = true;
    for (int j = 0; j <= dim; ++j) {
        if (ids[j] < 0 || ids[j] >= a.n_L) {
            if (lane == 0) atomicOr(a.flags, FLAG_RANGE);
            return;
        }
        vb[j] = a.vbound[ids[j]];
        members &= vb[j] == 0.0f;
    }
    if (dim == 0 && members) return;  // a vertex that is a point of X: f = 0, zero subgradient
    Simplex S;
    load_simplex(a.L, ids, dim, S);
    const uint8_t* comp = nullptr;
    const float* lam_w = nullptr;
    float px = 0.0f, py = 0.0f, pz = 0.0f;  // a vertex: p* = v
    if (dim == 0) {
    } else if (a.w[dim]) {
        lam_w = a.w[dim] + (tau * a.I[dim] + sample) * (dim + 1);
        sample_offset_lambda(S, lam_w, dim, px, py, pz);
    } else {
        comp = a.comp[dim] + sample * (dim + 1);
        sample_offset(S, comp, dim, a.m, px, py, pz);
    }
    const float u = members ? __fsqrt_ru(vertex_bound_sq(S, dim, px, py, pz))
                            : vertex_bound_general(S, dim, px, py, pz, vb);
    const float off[3] = {px, py, pz};
    const CellBox b = cull_box(g, S.v0, off, off, u);
    const int rows = b.n[1] * b.n[2];
    // nearest point: minimum of (d^2 bits << 32 | original row), with the
    // offset x* - p* kept by the lane that holds it
    unsigned long long best = ~0ull;
    float bx = 0.0f, by = 0.0f, bz = 0.0f;
    for (int r = 0; r < rows; ++r) {
        int32_t rb, re;
        box_row(g, b, r, rb, re);
        for (int32_t i = rb + lane; i < re; i += 32) {
            const float4 x = g.pts[i];
            const float dx = __fsub_rn(__fsub_rn(x.x, S.v0[0]), px);
            const float dy = __fsub_rn(__fsub_rn(x.y, S.v0[1]), py);
            const float dz = __fsub_rn(__fsub_rn(x.z, S.v0[2]), pz);
            const float d2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
            const unsigned long long key = (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) |
                                           static_cast<uint32_t>(__float_as_int(x.w));
            if (key < best) {
                best = key;
                bx = dx;
                by = dy;
                bz = dz;
            }
        }
    }
    unsigned long long all = best;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = shfl_xor_u64(all, o);
        all = y < all ? y : all;
    }
    if (all == ~0ull) {
        if (lane == 0) atomicOr(a.flags, FLAG_INTERNAL);
        return;
    }
    const int owner = __ffs(__ballot_sync(0xffffffffu, best == all)) - 1;
    bx = __shfl_sync(0xffffffffu, bx, owner);
    by = __shfl_sync(0xffffffffu, by, owner);
    bz = __shfl_sync(0xffffffffu, bz, owner);
    const float f = __fsqrt_rn(__uint_as_float(static_cast<uint32_t>(all >> 32)));
    if (!(f > 0.0f)) return;
    const float scale = gam / f;
    const int32_t xi = static_cast<int32_t>(all & 0xffffffffu);
    if (lane == 0 && !FLOOD_OOB(xi, g.n_pts, a.flags)) {
        atomicAdd(&a.grad_X[3 * int64_t(xi) + 0], scale * bx);
        atomicAdd(&a.grad_X[3 * int64_t(xi) + 1], scale * by);
        atomicAdd(&a.grad_X[3 * int64_t(xi) + 2], scale * bz);
    }
    if (lane <= dim) {
        float lam;
        if (dim == 0) {
            lam = 1.0f;
        } else if (lam_w) {  // d p / d v_0 = 1 - sum_{j>=1} lambda_j, d p / d v_j = lambda_j
            lam = lam_w[lane];
            if (lane == 0) {
                float t = 0.0f;
                for (int j = 1; j <= dim; ++j) t += lam_w[j];
                lam = 1.0f - t;
            }
        } else {
            lam = __fdiv_rn(static_cast<float>(comp[lane]), a.m);
        }
        const int32_t v = ids[lane];
        atomicAdd(&a.grad_L[3 * v + 0], -scale * lam * bx);
        atomicAdd(&a.grad_L[3 * v + 1], -scale * lam * by);
        atomicAdd(&a.grad_L[3 * v + 2], -scale * lam * bz);
    }
}

}  // namespace

}  // namespace flood

using namespace flood;

namespace {

// Grid samples (weights == nullptr, resolution m) or given sets.
int backward_impl(const flood_grid* grid, const float* L, int32_t n_landmarks, const int32_t* const simplices[4],
                  const int64_t n_simplices[4], int32_t m, const float* const weights[4],
                  const int32_t n_samples[4], const int32_t* const src[4], const float* const grad_values[4],
                  float* grad_X, float* grad_L, void* stream_) {
    if (!grid || !L || n_landmarks < 1 || !simplices || !n_simplices || !src || !grad_values || !grad_X ||
        !grad_L || m < 1 || m > FLOOD_MAX_M || (weights && !n_samples)) {
        set_error("flood_filtration_backward: NULL argument or m out of range");
        return FLOOD_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream_);
    if (int rc = pending_error(s)) return rc;
    Scratch scr(s);
    uint32_t* flags;
    int rc;
    if ((rc = scr.alloc(&flags, 1))) return rc;
    FLOOD_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), s));
    BwdArgs a{};
    a.m = static_cast<float>(m);
    a.L = L;
    a.n_L = n_landmarks;
    // vertex values' bounds d(v, X) (0 for points of X), as in the forward pass
    float *vval, *vbound;
    int32_t* vsrc;
    if ((rc = scr.alloc(&vval, n_landmarks)) || (rc = scr.alloc(&vbound, n_landmarks)) ||
        (rc = scr.alloc(&vsrc, 2 * int64_t(n_landmarks))))
        return rc;
    if ((rc = launch_vertices(L, n_landmarks, grid, vval, vsrc, vbound, flags, s))) return rc;
    a.vbound = vbound;
    a.n_simp[0] = n_landmarks;
    a.gp = view_of(grid);
    a.grad_X = grad_X;
    a.grad_L = grad_L;
    a.flags = flags;
    std::vector<uint8_t> tables[4];
    for (int k = 1; k <= 3; ++k) {
        a.n_simp[k] = n_simplices[k];
        a.simp[k] = simplices[k];
        if (n_simplices[k] <= 0) continue;
        if (!simplices[k]) {
            set_error("flood_filtration_backward: simplices[%d] is NULL", k);
            return FLOOD_EINVAL;
        }
        if (weights) {
            a.I[k] = n_samples[k];
            a.w[k] = weights[k];
            if (a.I[k] < 0 || a.I[k] > FLOOD_MAX_GIVEN_SAMPLES || (a.I[k] > 0 && !a.w[k])) {
                set_error("flood_filtration_given_backward: weights[%d] / n_samples[%d] invalid", k, k);
                return FLOOD_EINVAL;
            }
            continue;
        }
        tables[k] = interior_table(m, k);
        a.I[k] = static_cast<int>(tables[k].size() / (k + 1));
        if (a.I[k] > 0 && (rc = device_interior_table(m, k, tables[k], &a.comp[k]))) return rc;
    }
    for (int k = 0; k <= 3; ++k) {
        const int64_t nk = k == 0 ? n_landmarks : n_simplices[k];
        if (nk <= 0 || !grad_values[k]) continue;
        if (!src[k]) {
            set_error("flood_filtration_backward: src[%d] is NULL", k);
            return FLOOD_EINVAL;
        }
        a.k = k;
        a.n = nk;
        a.grad = grad_values[k];
        a.src = src[k];
        k_backward<<<static_cast<unsigned>(ceil_div(a.n * 32, 256)), 256, 0, s>>>(a); note_launch();
        FLOOD_CUDA(cudaGetLastError());
    }
    return finish(s, flags, "flood_filtration_backward");
}

}  // namespace

extern "C" int flood_filtration_backward(const flood_grid* grid, const float* L, int32_t n_landmarks,
                                         const int32_t* const simplices[4], const int64_t n_simplices[4], int32_t m,
                                         const int32_t* const src[4], const float* const grad_values[4],
                                         float* grad_X, float* grad_L, void* stream) {
    return backward_impl(grid, L, n_landmarks, simplices, n_simplices, m, nullptr, nullptr, src, grad_values,
                         grad_X, grad_L, stream);
}

extern "C" int flood_filtration_given_backward(const flood_grid* grid, const float* L, int32_t n_landmarks,
                                               const int32_t* const simplices[4], const int64_t n_simplices[4],
                                               const float* const weights[4], const int32_t n_samples[4],
                                               const int32_t* const src[4], const float* const grad_values[4],
                                               float* grad_X, float* grad_L, void* stream) {
    if (!weights || !n_samples) {
        set_error("flood_filtration_given_backward: weights and n_samples must be given");
        return FLOOD_EINVAL;
    }
    return backward_impl(grid, L, n_landmarks, simplices, n_simplices, 1, weights, n_samples, src, grad_values,
                         grad_X, grad_L, stream);
}
