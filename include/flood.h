/*
 * flood.h — C ABI of libflood, a B300 (sm_103a) implementation of the Flood
 * complex filtration (Graf, Pellizzoni, Uray, Huber, Kwitt: "The Flood
 * Complex — Large-Scale Persistent Homology on Millions of Points").
 *
 * Pipeline: farthest point sampling picks landmarks L ⊂ X (§3.2); the caller
 * triangulates L on the host (Del(L), §4); every simplex sigma of Del(L) gets
 *
 *     f(sigma) = max_{p in P_sigma} min_{x in X} |p - x|            (§4.1)
 *
 * over the barycentric grid P_sigma of resolution m (Lemma 1), faces included
 * (the discretised complex Flood_r(X,L,P) of §4.1 admits a simplex only once
 * all of its faces are flooded).
 *
 * General conventions
 *   - Every entry point returns a flood_status (0 = FLOOD_OK). No exception,
 *     abort or device trap crosses the ABI; device-side validation failures
 *     and bounded-wait timeouts come back as statuses. flood_last_error()
 *     returns a message for the calling thread's last non-OK status.
 *   - Pointers documented as "device" must point to memory of the current
 *     CUDA device; "host" pointers to ordinary host memory. Buffers are owned
 *     by the caller except the opaque flood_grid, which the library owns and
 *     frees in flood_grid_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *     enqueued on it. The hot-path calls (flood_fps, flood_fps_blocks,
 *     flood_build_grid, flood_filtration, flood_filtration_batch,
 *     flood_filtration_given) are asynchronous: they check their arguments on
 *     the host, enqueue, and return without waiting. Their device-side
 *     status (non-finite input, ids out of range, a bounded wait that gave
 *     up, ...) is copied back in stream order and reported by
 *     flood_check(stream), or by the next library call on the same stream
 *     once it has arrived. Other entry points synchronise the stream and
 *     report their own status (stated per function).
 *   - Coordinates are float32, row-major (n, 3). Vertex ids are int32 rows of
 *     L. Values are Euclidean distances (not squared), float32.
 *   - Scratch device memory is taken from the stream-ordered allocator
 *     (cudaMallocAsync) and returned before the call ends; failure gives
 *     FLOOD_ENOMEM.
 */
#ifndef FLOOD_H
#define FLOOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------
 * flood_check — wait for `stream` and report the device-side status of the
 * asynchronous calls enqueued on it since the last check: FLOOD_OK, or the
 * first error (flood_last_error() names the call). Check before destroying a
 * stream that asynchronous calls used.
 * ------------------------------------------------------------------------ */
int flood_check(void* stream);

typedef enum flood_status {
    FLOOD_OK = 0,
    FLOOD_EINVAL = -1,       /* bad argument or input (non-finite point, id out of range, L ⊄ X) */
    FLOOD_ENOMEM = -2,       /* device or host allocation failed */
    FLOOD_ECUDA = -3,        /* a CUDA runtime call failed */
    FLOOD_ETIMEOUT = -4,     /* a bounded device-side wait gave up */
    FLOOD_EDEGENERATE = -5,  /* FPS ran out of distinct points */
    FLOOD_ECAPACITY = -6,    /* request exceeds a configured capacity (serving admission) */
    FLOOD_EINTERNAL = -7     /* an internal consistency check failed */
} flood_status;

#define FLOOD_MAX_DIM 3      /* simplices of dimension 0..3 (ambient dimension 3) */
#define FLOOD_MAX_M 64       /* largest supported grid resolution m */
#define FLOOD_MAX_GIVEN_SAMPLES 65536 /* largest per-simplex set of flood_filtration_given */
#define FLOOD_ND_MAX_DIM 5   /* ambient dimensions 2..5 of the general-dimension path */

/* ------------------------------------------------------------------------
 * flood_fps — farthest point sampling (§3.2: greedy k-centre, a factor-2
 * approximation of the optimal covering radius; used for L in §5).
 *
 * l_0 = X[start]; for j >= 1, every point keeps d_i = min over picked l of
 * kappa(x_i, l), and l_j = argmax_i d_i, ties to the LOWEST index. kappa is
 * the squared distance in IEEE binary32 with each operation rounded
 * separately (no fused multiply-add):
 *     dx = x.x - l.x, ...;  kappa = ((dx*dx + dy*dy) + dz*dz).
 * This makes the picked indices bit-exact and reproducible.
 *
 *   X          device, (n_points, 3) float32, finite
 *   out_idx    device, int64[n_landmarks]: picked rows of X in pick order
 *   out_key    device, float32[n_landmarks] or NULL: d of each pick when it
 *              was picked (out_key[0] = +inf; out_key[j] is the squared
 *              covering radius of the first j picks)
 * Errors: FLOOD_EINVAL (sizes, start out of range) on return; through
 *         flood_check: FLOOD_EINVAL (non-finite X), FLOOD_EDEGENERATE (fewer
 *         than n_landmarks distinct points; out_idx holds the picks made so
 *         far), FLOOD_ETIMEOUT (grid exchange wait).
 * Asynchronous (see the conventions above).
 * ------------------------------------------------------------------------ */
int flood_fps(const float* X, int64_t n_points, int32_t n_landmarks, int64_t start,
              int64_t* out_idx, float* out_key, void* stream);

/* ------------------------------------------------------------------------
 * flood_fps_blocks — flood_fps with an explicit launch width.
 *
 * Same picks as flood_fps (bit-exact whatever the width). n_blocks is the
 * number of co-resident 1024-thread blocks (one per SM) the persistent FPS
 * launch may use:
 *   0   automatic (what flood_fps does): the fewest blocks whose registers
 *       hold every point (7,168 points per block, one block per SM, so up
 *       to 1,060,864 points on a 148-SM B300; one block needs no grid-wide
 *       exchange), else as many blocks as SMs (at most 160) with points
 *       streamed from memory;
 *   1   one block: leaves the other SMs to concurrent work (many small
 *       clouds at once); points stream from memory above 7,168;
 *   k   k blocks (clamped to the SM count and to 160).
 * Errors: as flood_fps; FLOOD_EINVAL also for n_blocks < 0.
 * ------------------------------------------------------------------------ */
int flood_fps_blocks(const float* X, int64_t n_points, int32_t n_landmarks, int64_t start,
                     int32_t n_blocks, int64_t* out_idx, float* out_key, void* stream);

/* Counters of the calling thread's last successful flood_fps (or
 * flood_fps_blocks / flood_fps_noalloc) call. Picks are made in rounds: one
 * grid-wide exchange per round selects one or more picks (all exact). */
typedef struct flood_fps_stats {
    int64_t picks;     /* landmarks (including the start point) */
    int64_t rounds;    /* grid-wide exchange rounds */
    int32_t blocks;    /* persistent blocks launched (one per SM) */
    int32_t resident;  /* 1: every point stayed in registers; 0: points streamed from memory */
} flood_fps_stats;

int flood_last_fps_stats(flood_fps_stats* out);

/* ------------------------------------------------------------------------
 * flood_fps_scratch_bytes — device scratch that flood_fps_blocks takes for
 * n_points points and launch width n_blocks (0 = automatic, as flood_fps).
 *
 * Host arithmetic (the launch width is clamped to the current device's SM
 * count; without a device one SM is assumed). The sum of the library's
 * 256-byte-aligned scratch pieces: control words, exchange
 * slots, the Morton-ordered point copy (16 B per point), the running minima
 * when the points do not all fit in registers (4 B per point), and the
 * Morton sort's codes, histogram, offsets and prefix-sum scratch.
 *   out_bytes  host int64 output
 * Errors: FLOOD_EINVAL (n_points out of range, n_blocks < 0, NULL output).
 * ------------------------------------------------------------------------ */
int flood_fps_scratch_bytes(int64_t n_points, int32_t n_blocks, int64_t* out_bytes);

/* ------------------------------------------------------------------------
 * flood_fps_wait_test — exercises the bounded wait of the FPS exchange.
 *
 * Test support, not part of the method: runs flood_fps_blocks on n_blocks
 * (>= 2) blocks with a grid exchange that also waits for `extra_blocks`
 * (>= 1, n_blocks + extra_blocks <= 160) blocks that are never launched, so
 * that every wait of the first round runs out after `poll_limit` polls
 * (each poll is one round of L2 loads, about a microsecond). The kernel then
 * raises its timeout flag and every block returns; nothing traps or hangs.
 *   X, n_points, n_landmarks, out_idx   as flood_fps (start = 0)
 * Returns FLOOD_ETIMEOUT when the wait ran out (the expected outcome); the
 * device context stays usable. Synchronises `stream`.
 * ------------------------------------------------------------------------ */
int flood_fps_wait_test(const float* X, int64_t n_points, int32_t n_landmarks, int32_t n_blocks,
                        int32_t extra_blocks, uint32_t poll_limit, int64_t* out_idx, void* stream);

/* ------------------------------------------------------------------------
 * flood_fps_noalloc — flood_fps without any device allocation.
 *
 * The paper has no counterpart: this is a deployment variant. It is for
 * callers that cannot allow a library to allocate device memory, such as a
 * host application whose own memory pool owns the device, a latency-critical
 * loop that forbids allocator calls after start-up, or a plugin whose host
 * framework forbids its extensions from allocating. It computes exactly what
 * flood_fps computes (same kernels, same bit-exact picks) but takes all of
 * its scratch from one fixed-size array compiled into the library (27 MiB of
 * device memory, held by every GPU that loads the library until the process
 * exits) and calls no allocating routine.
 *
 *   Arguments, outputs and errors as flood_fps, plus:
 *   n_points   at most 1,048,576 (2^20); larger inputs are rejected with
 *              FLOOD_ECAPACITY and nothing is launched. The fixed array holds
 *              flood_fps_scratch_bytes(2^20, 1) bytes, the largest need of
 *              any launch width at that size (points streamed from memory).
 * The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress (with that device current). All calls share the one
 * array: calls whose work
 * overlaps on the GPU (other streams, other threads) race and corrupt each
 * other's results, so serialise them. Synchronises `stream` before returning.
 * ------------------------------------------------------------------------ */
int flood_fps_noalloc(const float* X, int64_t n_points, int32_t n_landmarks, int64_t start,
                      int64_t* out_idx, float* out_key, void* stream);

/* ------------------------------------------------------------------------
 * flood_gather_rows — the landmark rows L = X[idx] (§3: the landmarks are the
 * FPS picks of X; the triangulation and the filtration take L).
 *
 *   X      device, (n_points, dim) float32 row-major
 *   idx    device int64[n_idx], each in [0, n_points) (e.g. flood_fps's out_idx)
 *   L      device float32 (n_idx, dim) output: L[r] = X[idx[r]] bit for bit
 *          (idx and L may be NULL when n_idx = 0)
 * Errors: FLOOD_EINVAL (arguments; 1 <= dim <= 8) on return; through
 * flood_check: FLOOD_EINVAL (an index out of range; its row is not written).
 * Asynchronous.
 * ------------------------------------------------------------------------ */
int flood_gather_rows(const float* X, int64_t n_points, int32_t dim, const int64_t* idx, int64_t n_idx,
                      float* L, void* stream);

/* ------------------------------------------------------------------------
 * flood_build_grid — uniform cell grid over X.
 *
 * Replaces the paper's axis-presort and masking matrix (§4.2, App. A.1) as
 * the spatial index from which each simplex gathers the candidate points
 * that Lemma 2 allows it to restrict to. Points are counting-sorted by the
 * linear id of their cell (x fastest), so every row of cells along x is one
 * contiguous range of the sorted array.
 *
 *   X          device, (n_points, 3) float32, finite; not retained
 *   cell_size  edge length h of the cubic cells; <= 0 picks a default from
 *              the bounding box and n_points. h is enlarged if the dense
 *              cell table would exceed 2^27 cells.
 *   out        receives a library-owned grid (free with flood_grid_destroy)
 * The bounding box, the cell size and the table dimensions are computed on
 * the device (no host readback); the cell table is allocated for
 * min(2^27, max(2^16, 4 n_points)) cells and the cell edge is enlarged on the
 * device until the box fits (results of the filtration do not depend on the
 * cell size). flood_grid_get_info waits for the build and reads them back.
 * Errors: FLOOD_EINVAL (arguments), FLOOD_ENOMEM, FLOOD_ECUDA on return;
 * through flood_check: FLOOD_EINVAL (non-finite X). Asynchronous.
 * ------------------------------------------------------------------------ */
typedef struct flood_grid flood_grid;

typedef struct flood_grid_info {
    int64_t n_points;
    int64_t n_cells;
    int32_t dims[3];         /* cells along x, y, z */
    float cell_size;
    float origin[3];         /* lower corner of cell (0,0,0) */
    float bbox_lo[3];
    float bbox_hi[3];
    int64_t device_bytes;    /* device memory held by the grid */
} flood_grid_info;

int flood_build_grid(const float* X, int64_t n_points, float cell_size,
                     flood_grid** out, void* stream);
/* Waits for the grid's build to finish, then fills *out. */
int flood_grid_get_info(const flood_grid* grid, flood_grid_info* out);
/* Waits for all device work, then frees the grid. */
void flood_grid_destroy(flood_grid* grid);

/* ------------------------------------------------------------------------
 * flood_filtration — flood values of every simplex of Del(L) (§4.1).
 *
 *     f(sigma) = max over the barycentric grid P_sigma (Lemma 1, faces
 *                included) of the distance to the nearest point of X,
 *
 * computed as max( own, f(facets) ) with `own` the maximum over the interior
 * samples (all parts c_i >= 1, lambda_i = c_i/m), since P_tau ⊂ P_sigma
 * (App. A.1). Dimensions run in increasing order; a sample whose bound
 * u_p = min_i (|p - v_i| + d(v_i, X)) (>= d(p, X); for v_i ∈ X this is the
 * step behind Lemma 2) does not exceed the facet maximum cannot change the
 * value and is skipped, and the nearest-point search of every other sample
 * stops as soon as it is exact or falls to the facet maximum. Values and
 * attaining samples equal those of the full max-min. Vertices get d(v, X):
 * 0 for landmarks that are points of X (the usual case, L = X[FPS picks]);
 * L need not be a subset of X (§3), at the cost of one exact nearest-point
 * search per landmark outside X.
 *
 *   grid         from flood_build_grid on X
 *   L            device, (n_landmarks, 3) float32, finite; rows equal (bit
 *                for bit) to rows of X are recognised as points of X
 *   simplices[k] device int32 (n_simplices[k], k+1): ascending vertex ids
 *                (rows of L). simplices[0] may be NULL (vertices = rows of L;
 *                n_simplices[0] must equal n_landmarks or 0).
 *   facets[k]    device int32 (n_simplices[k], k+1), k >= 2: column j is the
 *                row in simplices[k-1] of the facet without vertex j.
 *                facets[0] and facets[1] are ignored (the facets of an edge
 *                are its vertices).
 *   m            grid resolution, 1 <= m <= FLOOD_MAX_M (m+1 points per edge)
 *   values[k]    device float32 (n_simplices[k]) output; NULL skips output
 *                of that dimension (it is still computed if a higher
 *                dimension needs it)
 *   src[k]       device int32 (n_simplices[k], 2) output or NULL: the
 *                attaining sample, (dim << 28 | simplex row, interior sample
 *                rank in lexicographic order). Ties go to the lowest
 *                (dim, row, sample). Used by flood_filtration_backward.
 * Empty dimensions (n_simplices[k] == 0) are allowed. Results depend only on
 * (simplex, sample, point) arithmetic, so they are bitwise reproducible.
 * Errors: FLOOD_EINVAL (m, sizes, NULL arrays), FLOOD_ENOMEM, FLOOD_ECUDA on
 *         return; through flood_check: FLOOD_EINVAL (ids out of range,
 *         non-finite L), FLOOD_ETIMEOUT (bounded shared-memory copy waits).
 * Asynchronous; the work counters of flood_last_filtration_stats are read
 * back without waiting.
 * ------------------------------------------------------------------------ */
int flood_filtration(const flood_grid* grid, const float* L, int32_t n_landmarks,
                     const int32_t* const simplices[4], const int32_t* const facets[4],
                     const int64_t n_simplices[4], int32_t m,
                     float* const values[4], int32_t* const src[4], void* stream);

/* ------------------------------------------------------------------------
 * flood_filtration_batch — flood_filtration for several clouds at once.
 *
 * Same definition and results as flood_filtration, per job (bit for bit:
 * every value depends only on its own cloud). The clouds' sample groups share
 * one persistent flood kernel launch per dimension, so many small clouds keep
 * the GPU busy together. Jobs may use different grids, complexes and m.
 *   jobs    host array of n_jobs job descriptions (device pointers inside,
 *           with the meaning and layout of flood_filtration's arguments)
 * Errors as flood_filtration; a bad job fails the whole call before any
 * launch. Asynchronous.
 * ------------------------------------------------------------------------ */
typedef struct flood_filtration_job {
    const flood_grid* grid;
    const float* L;
    int32_t n_landmarks;
    int32_t m;
    const int32_t* simplices[4];
    const int32_t* facets[4];
    int64_t n_simplices[4];
    float* values[4];
    int32_t* src[4];
} flood_filtration_job;

int flood_filtration_batch(const flood_filtration_job* jobs, int32_t n_jobs, void* stream);
/* ------------------------------------------------------------------------
 * flood_filtration_given — flood values for caller-given point sets P_sigma.
 *
 * §4.1 allows any finite P_sigma ⊂ conv(sigma) (Theorem 2 bounds the
 * diagram error by the sets' Hausdorff distance to the simplices); one named
 * choice is a uniform random draw per simplex, whose Hausdorff distance
 * Lemma 4 bounds. The discretised complex Flood_r(X, L, P) takes sigma once
 * P_tau ⊂ X_r for every face tau of sigma, so
 *
 *     f(sigma) = max( max_{p in P_sigma} d(p, X),  max_{facets tau} f(tau) ),
 *
 * with f(v) = d(v, X) = 0 for a vertex (P_v = {v}, L ⊂ X required). The same
 * kernels as flood_filtration compute it, with the same exact pruning.
 *
 *   grid, L, simplices, facets, n_simplices, values, src
 *                as flood_filtration (src[k][i] = (dim << 28 | row, s): the
 *                attaining point is sample s of that simplex's set)
 *   weights[k]   device float32 (n_simplices[k], n_samples[k], k+1), k >= 1:
 *                barycentric coordinates (lambda_0..lambda_k) of each point
 *                of each simplex's own set, relative to its ascending vertex
 *                ids. The point is p = v_0 + sum_{j>=1} lambda_j (v_j - v_0);
 *                lambda_0 is not read (it is 1 - sum_{j>=1} lambda_j). Points
 *                should lie in conv(sigma) (lambda_j >= 0, sum <= 1) for the
 *                paper's guarantees; the values are computed as defined
 *                either way. weights[0] is ignored.
 *   n_samples[k] points per simplex of dimension k, 0..FLOOD_MAX_GIVEN_SAMPLES,
 *                with n_simplices[k] * n_samples[k] < 2^31; 0 leaves only the
 *                faces' maximum. n_samples[0] is ignored.
 * With lambda_j = fl32(c_j / m) for the interior compositions c of m in
 * lexicographic order, the results (values and src) are bit for bit those of
 * flood_filtration with that m.
 * Errors: as flood_filtration; FLOOD_EINVAL also for a NULL weights[k] that
 * is needed, n_samples out of range (on return), or a non-finite lambda_j
 * (j >= 1, through flood_check). Asynchronous.
 * ------------------------------------------------------------------------ */
int flood_filtration_given(const flood_grid* grid, const float* L, int32_t n_landmarks,
                           const int32_t* const simplices[4], const int32_t* const facets[4],
                           const int64_t n_simplices[4], const float* const weights[4],
                           const int32_t n_samples[4], float* const values[4], int32_t* const src[4],
                           void* stream);

/* Work counters of the calling thread's last flood_filtration(_batch/_given)
 * call; waits for that call's device work (meaningful when it succeeded). */
typedef struct flood_filtration_stats {
    int64_t simplices[4];        /* simplices per dimension */
    int64_t samples[4];          /* interior samples resolved (NN queries) per dimension */
    int64_t pairs[4];            /* (sample, candidate point) distance evaluations per dimension */
    int64_t work_items[4];       /* sample groups processed by the flood kernel per dimension */
    int64_t active_samples[4];   /* interior samples that could exceed their facet maximum */
    int64_t shells[4];           /* cell shells scanned by all sample groups */
    int64_t tiles[4];            /* shared-memory tiles of candidate points streamed */
    float flood_kernel_ms[4];    /* device time of the flood kernel per dimension (CUDA events on `stream`) */
} flood_filtration_stats;

int flood_last_filtration_stats(flood_filtration_stats* out);

/* ------------------------------------------------------------------------
 * flood_filtration_masked — the paper's own evaluation, as a comparator.
 *
 * §4.2 / App. A.1: every sample of the FULL grid P_sigma of Lemma 1 (faces
 * included) against every point of X inside the masking ball of Lemma 2
 * (centre: midpoint of the longest edge; radius sqrt(2) max_i |c - v_i|, or
 * that maximum for an edge), f(sigma) = max over samples of the minimum over
 * the masked points. No pruning and no reuse of facet values. The values
 * equal flood_filtration's up to FP32 rounding (the arithmetic differs: the
 * direct form |x - p|^2 here); it exists to time the paper's design on the
 * same GPU.
 *   grid, L, simplices, n_simplices, m   as flood_filtration; every landmark
 *                must be a point of X (Lemma 2 assumes L ⊂ X), else
 *                FLOOD_EINVAL; C(m+3, 3) <= 1024 full-grid samples (m <= 15)
 *   values[k]    device float32 (n_k) output, k = 0..3 (values[0] may be NULL)
 *   pairs_out    host int64 or NULL: (sample, masked point) pairs evaluated
 * Errors: FLOOD_EINVAL, FLOOD_ENOMEM, FLOOD_ECUDA. Synchronises `stream`.
 * ------------------------------------------------------------------------ */
int flood_filtration_masked(const flood_grid* grid, const float* L, int32_t n_landmarks,
                            const int32_t* const simplices[4], const int64_t n_simplices[4], int32_t m,
                            float* const values[4], int64_t* pairs_out, void* stream);
/* ------------------------------------------------------------------------
 * flood_masking_ball_counts — size of the paper's masked candidate sets.
 *
 * §4.2: Lemma 2 restricts the nearest-point search of a simplex to the
 * points of X in the ball B(c, sqrt(2) r) (c the midpoint of the longest
 * edge, r = max_i |c - v_i|; radius r for an edge). This counts them:
 *   counts_out[k] = sum over k-simplices of |X ∩ B|   (host int64[4];
 *                   counts_out[0] = 0)
 * so that sum_k C(m-1, k) counts_out[k] is the method's own work in
 * (interior sample, candidate point) pairs, and sum_k C(m+k, k) counts_out[k]
 * that of the paper's full-grid evaluation. The ball test runs in FP32
 * (points within rounding of the sphere may count either way).
 *   grid, L, simplices, n_simplices   as flood_filtration
 * Errors: FLOOD_EINVAL, FLOOD_ENOMEM, FLOOD_ECUDA. Synchronises `stream`.
 * ------------------------------------------------------------------------ */
int flood_masking_ball_counts(const flood_grid* grid, const float* L, int32_t n_landmarks,
                              const int32_t* const simplices[4], const int64_t n_simplices[4],
                              int64_t counts_out[4], void* stream);

/* ------------------------------------------------------------------------
 * flood_persistence — persistence pairs of the flood filtration (§2), on
 * the device.
 *
 * The values make the complex a filtration (every face's value <= its
 * cofaces'); §2's persistence diagrams pair the simplex that creates each
 * homology class with the one that kills it. Simplices are ordered by
 * (value, dimension, lexicographic vertex ids), faces before cofaces on ties,
 * and the Z/2 boundary matrix is reduced with clearing (twist), higher
 * dimensions first; the tetrahedra's pairs come from the anti-transposed
 * (coboundary) matrix, which has the same pairs. The reduction runs in
 * parallel rounds of left-to-right column additions; any reduced form
 * reached that way has the pivots of the sequential reduction, so the pairs
 * are those of the standard algorithm.
 *   simplices, facets, n_simplices   as flood_filtration (device; vertex ids
 *                    < 2^21; simplices[0] is ignored: vertex i is row i)
 *   values[k]        device float32 (n_k): the flood values (finite, >= 0)
 *   pairs[k]         device int32 capacity (n_{k+1}, 2), k = 0..2: (birth row
 *                    of dimension k, death row of dimension k+1) per finite
 *                    pair (zero-persistence pairs included), in the deaths'
 *                    filtration order; n_pairs[k] (host) receives the count
 *   essential[k]     device int32 capacity n_k, k = 0..3: rows of dimension
 *                    k whose class never dies, in filtration order;
 *                    n_essential[k] (host) receives the count
 *   rounds           host int64[4] or NULL: parallel rounds per dimension
 * The diagram dgm_k is {(values[k][b], values[k+1][d])} over pairs[k] with
 * d's value above b's, plus (values[k][e], inf) per essential row.
 * Errors: FLOOD_EINVAL (sizes, NULL arrays, ids out of range, a value that is
 * negative or not finite), FLOOD_ENOMEM, FLOOD_ECAPACITY (columns beyond
 * 2^31 entries), FLOOD_ECUDA. Synchronises `stream`.
 * ------------------------------------------------------------------------ */
int flood_persistence(const int32_t* const simplices[4], const int32_t* const facets[4],
                      const int64_t n_simplices[4], const float* const values[4], int32_t* const pairs[3],
                      int64_t n_pairs[3], int32_t* const essential[4], int64_t n_essential[4], int64_t rounds[4],
                      void* stream);

/* ------------------------------------------------------------------------
 * flood_fp32_peak_probe — measured FP32 FMA throughput (roofline helper).
 *
 * Not part of the method: the flood kernels are bound by the FP32 pipe when
 * they are dense, and this launches a kernel that does nothing but
 * independent FP32 fused multiply-adds (16 chains per thread, 8 blocks of
 * 256 threads per SM) so that the caller can time it with CUDA events on
 * `stream`. packed = 0 issues scalar FMAs, 1 packed pairs (two lanes' worth
 * per instruction, the form the flood kernels use).
 *   iterations  loop trips per thread, 1..2^30
 *   flops_out   host: floating-point operations the launch performs (2 per FMA)
 * Errors: FLOOD_EINVAL, FLOOD_ENOMEM, FLOOD_ECUDA. Does not synchronise.
 * ------------------------------------------------------------------------ */
int flood_fp32_peak_probe(int32_t packed, int64_t iterations, double* flops_out, void* stream);

/* ------------------------------------------------------------------------
 * flood_complex_faces — faces of Del(L) and facet incidence, on the device.
 *
 * The discretised complex of §4.1 admits a simplex only after all of its
 * faces, so the filtration needs every face of the triangulation (§4) and,
 * per simplex, the rows of its facets. Given the tetrahedra, this writes the
 * distinct triangles (faces of the tetrahedra) and edges (faces of the
 * triangles) and the facet columns, in the layout flood_filtration reads:
 * facets[k][i][j] is the row in the (k-1)-simplices of simplex i without its
 * vertex j. Row order: a face's row follows the first (parent row, j) that
 * produces it (j = the dropped vertex), which is deterministic; it is not
 * lexicographic. Vertex ids ascend within every row.
 *
 *   tets             device int32 (n_tets, 4): ascending vertex ids in
 *                    [0, n_vertices); also simplices[3] of the complex
 *   n_tets           0..2^24
 *   n_vertices       1..2^21 - 1 (n_landmarks)
 *   triangles        device int32 capacity (4 n_tets, 3): rows [0, *n_triangles)
 *   edges            device int32 capacity (6 n_tets, 2): rows [0, *n_edges)
 *   tet_facets       device int32 (n_tets, 4): facets[3]
 *   triangle_facets  device int32 capacity (4 n_tets, 3): facets[2]
 *   edge_facets      device int32 capacity (6 n_tets, 2) or NULL: facets[1]
 *                    (the other vertex: (b, a) for edge (a, b))
 *   n_triangles, n_edges   host outputs: the counts
 * Every triangle and edge of the input is produced, each exactly once.
 * Errors: FLOOD_EINVAL (sizes, NULL outputs, a row not ascending or out of
 * range), FLOOD_ENOMEM, FLOOD_ECUDA. Synchronises `stream` before returning.
 * ------------------------------------------------------------------------ */
int flood_complex_faces(const int32_t* tets, int64_t n_tets, int32_t n_vertices, int32_t* triangles,
                        int32_t* edges, int32_t* tet_facets, int32_t* triangle_facets, int32_t* edge_facets,
                        int64_t* n_triangles, int64_t* n_edges, void* stream);
/* ------------------------------------------------------------------------
 * flood_filtration_backward — gradient of F = sum_sigma g_sigma f(sigma).
 *
 * Our derivation from the value definition of §4.1: with p* = sum_j
 * lambda_j v_j the attaining sample (from src) and x* its nearest point of X
 * (recomputed over the attaining simplex's cull box, ties to the lowest row
 * of X), f = |p* - x*| and, if f > 0,
 *     grad_X[x*]  += g (x* - p*) / f,
 *     grad_L[v_j] += g lambda_j (p* - x*) / f;
 * a vertex (its own value, or attaining a coface's) is p* = v, lambda = 1;
 * f = 0 (vertices that are points of X, degenerate cases) contributes nothing.
 *
 *   grid, L, simplices, n_simplices, m   as passed to flood_filtration
 *   src[k]          device int32 (n_k, 2) from flood_filtration
 *   grad_values[k]  device float32 (n_k) upstream gradients, or NULL (zero);
 *                   k = 0 are the vertex values (n_landmarks)
 *   grad_X          device float32 (n_points, 3), accumulated into
 *   grad_L          device float32 (n_landmarks, 3), accumulated into
 * Accumulation uses atomics, so the summation order (last bits) may vary.
 * Errors: FLOOD_EINVAL, FLOOD_ENOMEM, FLOOD_ECUDA. Synchronises `stream`.
 * ------------------------------------------------------------------------ */
int flood_filtration_backward(const flood_grid* grid, const float* L, int32_t n_landmarks,
                              const int32_t* const simplices[4], const int64_t n_simplices[4],
                              int32_t m, const int32_t* const src[4],
                              const float* const grad_values[4],
                              float* grad_X, float* grad_L, void* stream);
/* ------------------------------------------------------------------------
 * flood_filtration_given_backward — flood_filtration_backward for the values
 * of flood_filtration_given.
 *
 * The attaining point p* = v_0 + sum_{j>=1} lambda_j (v_j - v_0) comes from
 * the set named by src; its derivative moves v_j (j >= 1) with weight
 * lambda_j and v_0 with weight 1 - sum_{j>=1} lambda_j:
 *     grad_X[x*] += g (x* - p*) / f,   grad_L[v_j] += g lambda_j (p* - x*) / f.
 *   weights, n_samples   as passed to flood_filtration_given
 *   other arguments      as flood_filtration_backward (no m)
 * Errors: FLOOD_EINVAL, FLOOD_ENOMEM, FLOOD_ECUDA. Synchronises `stream`.
 * ------------------------------------------------------------------------ */
int flood_filtration_given_backward(const flood_grid* grid, const float* L, int32_t n_landmarks,
                                    const int32_t* const simplices[4], const int64_t n_simplices[4],
                                    const float* const weights[4], const int32_t n_samples[4],
                                    const int32_t* const src[4], const float* const grad_values[4],
                                    float* grad_X, float* grad_L, void* stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of many point clouds on one GPU.
 *
 * Not in the paper, which runs one cloud at a time; this is the request
 * loop around the same computation. A submitted cloud is admitted when an
 * in-flight slot is free and its estimated device memory fits the budget
 * (FIFO); it then runs FPS and the grid build on its own stream, is
 * triangulated on the host by the caller's callback, and joins the next
 * batched filtration (flood_filtration_batch) with every other cloud that is
 * ready at that moment (two batch threads, each on its own stream, so one
 * batch's host work overlaps another's kernels). Requests arriving while others run are admitted as
 * slots and memory free up, and their work overlaps on the device. Each
 * result equals what the one-cloud path computes on that cloud, bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct flood_server flood_server;

/* Simplex lists returned by the triangulation callback (host memory, layout
 * of flood_filtration's simplices/facets). The arrays must stay valid until
 * the library calls release(user, owner), which it does after copying them. */
typedef struct flood_host_complex {
    int64_t n_simplices[4];
    const int32_t* simplices[4];
    const int32_t* facets[4];
    void* owner;
} flood_host_complex;

/* Triangulate the landmarks (host, (n, 3) float32). Returns 0 on success;
 * any other value fails that request only. Called from library threads.
 * The callback may fill only the tetrahedra (n_simplices[1] = n_simplices[2]
 * = 0, facets ignored); the library then builds the triangles, edges and
 * facet incidence on the device (flood_complex_faces) and reports the rows
 * it built in flood_result.simplices. This is the faster mode: the host then
 * only triangulates (the Python Server uses it by default). */
typedef int (*flood_triangulate_fn)(void* user, const float* landmarks, int32_t n_landmarks,
                                    flood_host_complex* out);
typedef void (*flood_release_fn)(void* user, void* owner);

typedef struct flood_serve_config {
    int64_t device_budget_bytes;    /* admission budget for in-flight clouds (> 0) */
    int32_t max_inflight;           /* clouds admitted at once (>= 1) */
    int32_t max_batch;              /* clouds per batched filtration (>= 1; 1 = per-cloud path) */
    int32_t gpu_workers;            /* host threads driving FPS + grid (>= 1) */
    int32_t triangulation_workers;  /* host threads calling triangulate (>= 1) */
    float landmark_fraction;        /* n_landmarks when a request passes 0: round(fraction * N), >= 4 */
    float cell_factor;              /* grid cell = cell_factor * FPS covering radius (> 0), or 0: the
                                       tuning table's factor for each request's bucket */
    flood_triangulate_fn triangulate;
    flood_release_fn release;       /* may be NULL */
    void* user;
} flood_serve_config;

typedef struct flood_result {
    int32_t status;                 /* FLOOD_OK or this request's error */
    int32_t n_landmarks;
    int64_t n_simplices[4];
    const float* values[4];         /* host, owned by the server until flood_serve_release */
    const int64_t* landmarks;       /* host, n_landmarks rows of X (FPS order) */
    double latency_ms;              /* submit -> values on the host */
    const int32_t* simplices[4];    /* host (n_k, k+1), k >= 1: the rows values[k] refer to
                                       (the callback's, or the device-built faces); [0] NULL */
} flood_result;

typedef struct flood_serve_stats_t {
    int64_t submitted, completed, failed, inflight;
    int64_t batches;                /* batched filtration calls */
    double mean_batch;              /* clouds per batched call */
    double clouds_per_s;            /* completed / (last completion - first submission) */
    double p50_ms, p99_ms, mean_ms; /* latency over completed requests */
    int64_t device_bytes_in_use;
    int64_t device_bytes_peak;
} flood_serve_stats_t;

/* Start the server's threads. Errors: FLOOD_EINVAL (config), FLOOD_ENOMEM. */
int flood_serve_create(const flood_serve_config* config, flood_server** out);
/* Queue a cloud (X_host: host (N, 3) float32, copied before returning).
 * n_landmarks = 0 uses the configured fraction; m is the grid resolution.
 * Errors: FLOOD_EINVAL; FLOOD_ECAPACITY if the cloud alone exceeds the budget. */
int flood_serve_submit(flood_server* server, const float* X_host, int64_t n_points, int32_t n_landmarks,
                       int32_t m, uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a result. FLOOD_ETIMEOUT if not
 * done yet; otherwise *out describes it (out->status is its own outcome). */
int flood_serve_poll(flood_server* server, uint64_t ticket, int32_t timeout_ms, flood_result* out);
/* Free a finished request's host result. */
int flood_serve_release(flood_server* server, uint64_t ticket);
int flood_serve_stats(flood_server* server, flood_serve_stats_t* out);
/* Stop the threads (waiting for in-flight work) and free everything. */
void flood_serve_destroy(flood_server* server);

/* ------------------------------------------------------------------------
 * Tuning table: launch parameters of the filtration per workload bucket.
 *
 * Not in the paper. Two parameters change the speed of a filtration but not
 * its results (values and sources are bitwise the same for every choice):
 *   cell_factor   grid cell edge as a multiple of the FPS covering radius
 *                 (sqrt of the last FPS key); used by the serving loop and by
 *                 callers that size flood_build_grid's cells from FPS;
 *   heavy_shells  sample groups whose bound allows at least this many shells
 *                 of cells are run one per CTA instead of one per warp
 *                 (flood_filtration and its variants look it up per call).
 * Entries are keyed by (SM count, round(log2 points), round(log2 landmarks),
 * m); a lookup returns the entry of the nearest bucket (distance |d log2
 * points| + |d log2 landmarks| + |d m| / 4) among entries for the current
 * device's SM count, else the defaults (0.5, 9). The paper_2509_22432_b300.tune
 * module measures entries and writes them to a file; FLOOD_TUNE_CACHE names
 * a file loaded at the first use of the table. The table is process-wide and
 * thread-safe.
 * File format: one entry per line, "sm_count log2_points log2_landmarks m
 * cell_factor heavy_shells"; '#' starts a comment line.
 * ------------------------------------------------------------------------ */
typedef struct flood_tuning {
    float cell_factor;
    int32_t heavy_shells;
    int32_t tuned;           /* 1: from a table entry; 0: defaults */
} flood_tuning;

typedef struct flood_tuning_entry {
    int32_t sm_count;        /* >= 1 */
    int32_t log2_points;     /* 0..40 */
    int32_t log2_landmarks;  /* 0..40 */
    int32_t m;               /* 1..FLOOD_MAX_M */
    float cell_factor;       /* (0, 64] */
    int32_t heavy_shells;    /* 1..63 */
} flood_tuning_entry;

/* Parameters for a workload (host output). Errors: FLOOD_EINVAL. */
int flood_tuning_lookup(int64_t n_points, int32_t n_landmarks, int32_t m, flood_tuning* out);
/* Add or replace the entry of e's bucket. Errors: FLOOD_EINVAL (out of range). */
int flood_tuning_set(const flood_tuning_entry* e);
/* Add or replace entries from a file; *n_loaded (nullable) receives how many.
 * Errors: FLOOD_EINVAL (unreadable file or bad line; entries before it stay). */
int flood_tuning_load(const char* path, int32_t* n_loaded);
/* Copy up to `capacity` entries to out (host); *n_entries receives the total. */
int flood_tuning_entries(flood_tuning_entry* out, int32_t capacity, int32_t* n_entries);
/* Remove every entry (lookups return the defaults until entries are added). */
int flood_tuning_clear(void);

/* ========================================================================
 * General ambient dimension d = 2..5 (§3 leaves d free; §5.3 scales it:
 * Fig. 4c, swisscheese-like clouds with |X| = 1M, |L| = 1k, d = 2..5).
 * Points are rows of a row-major (n, d) float32 array; simplices go up to
 * dimension d. Same conventions as the three-dimensional entry points:
 * caller-owned device buffers, asynchronous on `stream`, device-side errors
 * through flood_check (or the next call on the stream).
 * ======================================================================== */

/* ------------------------------------------------------------------------
 * flood_fps_nd — farthest point sampling in R^d (§3.2, greedy k-centre).
 *
 * The same rule as flood_fps: l_0 = X[start]; each later pick maximises the
 * distance to the picks so far, ties to the lowest index. The key is the
 * binary32 squared distance with the d squares summed left to right and
 * every subtraction, product and sum rounded on its own (no fused
 * multiply-add), so picks are bit-exact against any implementation of that
 * arithmetic. dim = 3 runs flood_fps (the same key and picks); dim = 2 runs
 * flood_fps on the points at z = 0 (the extra key term is an exact 0, so the
 * keys and picks are the two-dimensional ones bit for bit), with a scratch
 * copy of 12 * n_points bytes from the stream-ordered pool.
 *   X          device, (n_points, dim) float32 row-major, finite
 *   dim        2..FLOOD_ND_MAX_DIM
 *   out_idx    device int64[n_landmarks]: the picks, out_idx[0] = start
 *   out_key    device float32[n_landmarks] or NULL: squared distance of each
 *              pick when picked (out_key[0] = +inf)
 * Errors: FLOOD_EINVAL (sizes, dim, start), FLOOD_ENOMEM, FLOOD_ECUDA on
 * return; through flood_check: FLOOD_EINVAL (non-finite X),
 * FLOOD_EDEGENERATE (fewer than n_landmarks distinct points),
 * FLOOD_ETIMEOUT (a bounded wait of the pick exchange gave up).
 * ------------------------------------------------------------------------ */
int flood_fps_nd(const float* X, int64_t n_points, int32_t dim, int32_t n_landmarks, int64_t start,
                 int64_t* out_idx, float* out_key, void* stream);

/* ------------------------------------------------------------------------
 * flood_build_grid_nd — uniform cell grid of X in R^d (the masking
 * structure of §4.2 for any d).
 *
 * A dense row-major table of cubic cells of edge h over X's bounding box,
 * with X's points copied in cell order (library-owned; X may be freed
 * afterwards). cell_size <= 0 picks h for about six points per cell over the
 * axes X spans; the table holds at most min(2^25, max(2^12, 2 n_points))
 * cells and h is enlarged on the device until it fits. Results of
 * flood_filtration_nd do not depend on h.
 * Errors: FLOOD_EINVAL (arguments), FLOOD_ENOMEM, FLOOD_ECUDA on return;
 * through flood_check: FLOOD_EINVAL (non-finite X). Asynchronous.
 * ------------------------------------------------------------------------ */
typedef struct flood_grid_nd flood_grid_nd;

typedef struct flood_grid_nd_info {
    int64_t n_points;
    int64_t n_cells;
    int32_t dim;
    int32_t dims[FLOOD_ND_MAX_DIM];      /* cells per axis (axes >= dim: 0) */
    float cell_size;
    float bbox_lo[FLOOD_ND_MAX_DIM];     /* also the lower corner of cell 0 */
    float bbox_hi[FLOOD_ND_MAX_DIM];
    int64_t device_bytes;
} flood_grid_nd_info;

int flood_build_grid_nd(const float* X, int64_t n_points, int32_t dim, float cell_size,
                        flood_grid_nd** out, void* stream);
/* Waits for the build, then fills *out. */
int flood_grid_nd_get_info(const flood_grid_nd* grid, flood_grid_nd_info* out);
/* Waits for all device work, then frees the grid. */
void flood_grid_nd_destroy(flood_grid_nd* grid);

/* ------------------------------------------------------------------------
 * flood_filtration_nd — flood values of every simplex of Del(L) in R^d (§4.1).
 *
 * f(sigma) = max over Lemma 1's grid P_sigma (faces included) of the
 * distance to the nearest point of X, computed as in flood_filtration:
 * max(own, f(facets)) over dimensions 0..d in increasing order, `own` the
 * maximum over the interior samples (lambda_i = c_i/m, all c_i >= 1).
 * A sample's nearest-point search stops as soon as its distance is exact or
 * can no longer exceed max(f(facets), the simplex's running maximum); every
 * such decision uses bounds rounded toward the safe side, so the value is
 * that of the full search: max(f(facets), sqrt(max over interior samples of
 * min over X of the binary32 squared distance)), whatever the cell size.
 * Vertices get d(v, X) (0 for rows of L that are points of X).
 *
 *   grid         from flood_build_grid_nd on X (its dim is the dimension d)
 *   L            device, (n_landmarks, d) float32, finite
 *   simplices[k] device int32 (n_simplices[k], k+1) vertex ids (rows of L),
 *                k = 1..d; simplices[0] is ignored (vertices are L's rows;
 *                n_simplices[0] must be n_landmarks or 0)
 *   facets[k]    device int32 (n_simplices[k], k+1), k >= 2: column j is the
 *                row in simplices[k-1] of the facet without vertex j
 *   m            1..FLOOD_MAX_M
 *   values[k]    device float32 (n_simplices[k]) output, k = 0..d (values[0]:
 *                n_landmarks entries); NULL skips the output (the dimension
 *                is still computed for the ones above it)
 * Entries above d must have n_simplices[k] == 0.
 * Errors: FLOOD_EINVAL (arguments), FLOOD_ENOMEM, FLOOD_ECUDA on return;
 * through flood_check: FLOOD_EINVAL (ids out of range, non-finite L),
 * FLOOD_EINTERNAL (a consistency check). Asynchronous; the work counters of
 * flood_last_filtration_nd_stats are read back without waiting.
 * ------------------------------------------------------------------------ */
int flood_filtration_nd(const flood_grid_nd* grid, const float* L, int32_t n_landmarks,
                        const int32_t* const simplices[FLOOD_ND_MAX_DIM + 1],
                        const int32_t* const facets[FLOOD_ND_MAX_DIM + 1],
                        const int64_t n_simplices[FLOOD_ND_MAX_DIM + 1], int32_t m,
                        float* const values[FLOOD_ND_MAX_DIM + 1], void* stream);

/* Work counters of the calling thread's last flood_filtration_nd, per
 * dimension (waits for that call's stream). items: (simplex, interior
 * sample) pairs (vertices: one each); pruned: settled by the vertices'
 * nearest points alone; resolved: settled within the 3^d cells around the
 * sample; exact: nearest distance exact within those cells; fallback: handed
 * to the shell search; pairs / pairs_fallback: (sample, point) distances
 * evaluated in each pass; cells: cells whose points were read. */
typedef struct flood_nd_stats {
    int32_t dim;
    int64_t items[FLOOD_ND_MAX_DIM + 1];
    int64_t pruned[FLOOD_ND_MAX_DIM + 1];
    int64_t resolved[FLOOD_ND_MAX_DIM + 1];
    int64_t exact[FLOOD_ND_MAX_DIM + 1];
    int64_t fallback[FLOOD_ND_MAX_DIM + 1];
    int64_t pairs[FLOOD_ND_MAX_DIM + 1];
    int64_t pairs_fallback[FLOOD_ND_MAX_DIM + 1];
    int64_t cells[FLOOD_ND_MAX_DIM + 1];
} flood_nd_stats;

int flood_last_filtration_nd_stats(flood_nd_stats* out);

/* Message for the calling thread's last non-OK status ("" if none). */
const char* flood_last_error(void);

/* Library version, e.g. "0.1.0". */
const char* flood_version(void);

/* Number of CUDA kernels libflood has launched in this process so far. */
int64_t flood_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* FLOOD_H */
