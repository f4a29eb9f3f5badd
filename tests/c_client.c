/* A plain C client of libflood (no Python): FPS, grid and filtration of the
 * regular tetrahedron X = L = {(1,1,1), (1,-1,-1), (-1,1,-1), (-1,-1,1)} at
 * m = 4. Its centroid is a grid sample and the circumcentre, so the
 * tetrahedron's value is the circumradius a sqrt(6) / 4 = sqrt(3) (edge
 * a = 2 sqrt(2)); each edge's is a / 2 = sqrt(2) (its midpoint). A triangle's
 * interior samples at m = 4 lie a sqrt(3) / 4 < sqrt(2) from a vertex, so each
 * triangle takes its edges' value sqrt(2). Prints the values; exit 0 if they
 * match. */
#include <math.h>
#include <stdio.h>
#include <cuda_runtime.h>
#include "flood.h"

int main(void) {
    const float X[12] = {1, 1, 1, 1, -1, -1, -1, 1, -1, -1, -1, 1};
    const int32_t edges[12] = {0, 1, 0, 2, 0, 3, 1, 2, 1, 3, 2, 3};
    /* triangles (lexicographic) and their facets: column j = the edge without vertex j */
    const int32_t tris[12] = {0, 1, 2, 0, 1, 3, 0, 2, 3, 1, 2, 3};
    const int32_t tri_facets[12] = {3, 1, 0, 4, 2, 0, 5, 2, 1, 5, 4, 3};
    const int32_t tet[4] = {0, 1, 2, 3};
    const int32_t tet_facets[4] = {3, 2, 1, 0};
    float *dX, *dvals[4];
    int64_t* didx;
    int32_t *dsimp[4] = {0, 0, 0, 0}, *dfac[4] = {0, 0, 0, 0};
    const int64_t n[4] = {4, 6, 4, 1};
    if (cudaMalloc((void**)&dX, sizeof X) || cudaMalloc((void**)&didx, 4 * sizeof(int64_t))) return 2;
    cudaMemcpy(dX, X, sizeof X, cudaMemcpyHostToDevice);
    for (int k = 0; k < 4; ++k)
        if (cudaMalloc((void**)&dvals[k], n[k] * sizeof(float))) return 2;
    cudaMalloc((void**)&dsimp[1], sizeof edges);
    cudaMalloc((void**)&dsimp[2], sizeof tris);
    cudaMalloc((void**)&dsimp[3], sizeof tet);
    cudaMalloc((void**)&dfac[2], sizeof tri_facets);
    cudaMalloc((void**)&dfac[3], sizeof tet_facets);
    cudaMemcpy(dsimp[1], edges, sizeof edges, cudaMemcpyHostToDevice);
    cudaMemcpy(dsimp[2], tris, sizeof tris, cudaMemcpyHostToDevice);
    cudaMemcpy(dsimp[3], tet, sizeof tet, cudaMemcpyHostToDevice);
    cudaMemcpy(dfac[2], tri_facets, sizeof tri_facets, cudaMemcpyHostToDevice);
    cudaMemcpy(dfac[3], tet_facets, sizeof tet_facets, cudaMemcpyHostToDevice);

    int64_t idx[4];
    if (flood_fps(dX, 4, 4, 0, didx, NULL, NULL) != FLOOD_OK) { printf("fps: %s\n", flood_last_error()); return 1; }
    cudaMemcpy(idx, didx, sizeof idx, cudaMemcpyDeviceToHost);
    flood_grid* grid = NULL;
    if (flood_build_grid(dX, 4, 0.0f, &grid, NULL) != FLOOD_OK) { printf("grid: %s\n", flood_last_error()); return 1; }
    const int32_t* simp[4] = {NULL, dsimp[1], dsimp[2], dsimp[3]};
    const int32_t* fac[4] = {NULL, NULL, dfac[2], dfac[3]};
    float* vals[4] = {dvals[0], dvals[1], dvals[2], dvals[3]};
    /* L = X (the landmarks are the points themselves, in their original order) */
    if (flood_filtration(grid, dX, 4, simp, fac, n, 4, vals, NULL, NULL) != FLOOD_OK) {
        printf("filtration: %s\n", flood_last_error());
        return 1;
    }
    /* the calls above are asynchronous: their device-side status arrives here */
    if (flood_check(NULL) != FLOOD_OK) {
        printf("check: %s\n", flood_last_error());
        return 1;
    }
    float v[4][6];
    for (int k = 0; k < 4; ++k) cudaMemcpy(v[k], dvals[k], n[k] * sizeof(float), cudaMemcpyDeviceToHost);
    flood_grid_destroy(grid);
    int ok = idx[0] == 0;
    for (int i = 0; i < 4; ++i) ok &= v[0][i] == 0.0f;
    for (int i = 0; i < 6; ++i) ok &= fabsf(v[1][i] - sqrtf(2.0f)) <= 1e-5f;
    for (int i = 0; i < 4; ++i) ok &= fabsf(v[2][i] - sqrtf(2.0f)) <= 1e-5f;
    ok &= fabsf(v[3][0] - sqrtf(3.0f)) <= 1e-5f;
    printf("edge %.7f triangle %.7f tetrahedron %.7f (sqrt 3 = %.7f) %s\n", v[1][0], v[2][0], v[3][0], sqrtf(3.0f),
           ok ? "ok" : "MISMATCH");
    return ok ? 0 : 1;
}
