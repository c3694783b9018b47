/*
 * lbm_c_client.c -- a plain C caller of the library's C-ABI (include/lbm.h), with no Python
 * and no PyTorch: it owns its device workspace (cudaMalloc) and stream, sets a Taylor-Green
 * field, advances it, and prints the conservation sums and a few moments.  The test suite
 * builds it with gcc against liblbm_gb300.so and compares its output with the Python path.
 *
 * usage: lbm_c_client <n> <steps>      (D3Q19, K = 3, tau = 0.6, FP32 storage, n^3 cells)
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "lbm.h"

static int check(lbm_status s, const char *what) {
    if (s != LBM_OK) {
        fprintf(stderr, "%s: %s (%s)\n", what, lbm_status_string(s), lbm_last_error());
        return 1;
    }
    return 0;
}

int main(int argc, char **argv) {
    const int n = argc > 1 ? atoi(argv[1]) : 24;
    const int steps = argc > 2 ? atoi(argv[2]) : 50;
    const int64_t dims[3] = {n, n, n};
    const long long C = (long long)n * n * n;
    const double PI = 3.14159265358979323846, u0 = 0.05, T0 = 1.0 / 3.0, k = 2.0 * PI / n;

    /* Taylor-Green fields: u = u0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0),
       rho = 1 + p / T0, p = u0^2 / 16 (cos 2kx + cos 2ky)(cos 2kz + 2) */
    double *rho = malloc(sizeof(double) * C), *u = malloc(sizeof(double) * 3 * C);
    if (!rho || !u) return 2;
    for (int z = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                const long long c = x + (long long)n * (y + (long long)n * z);
                const double X = k * x, Y = k * y, Z = k * z;
                rho[c] = 1.0 + u0 * u0 / 16.0 * (cos(2 * X) + cos(2 * Y)) * (cos(2 * Z) + 2.0) / T0;
                u[c] = u0 * sin(X) * cos(Y) * cos(Z);
                u[C + c] = -u0 * cos(X) * sin(Y) * cos(Z);
                u[2 * C + c] = 0.0;
            }

    const size_t ws_bytes = lbm_workspace_bytes(LBM_D3Q19, dims, LBM_STORE_F32);
    void *ws = NULL;
    cudaStream_t stream;
    if (ws_bytes == 0 || cudaMalloc(&ws, ws_bytes) != cudaSuccess || cudaStreamCreate(&stream) != cudaSuccess) {
        fprintf(stderr, "device set-up failed\n");
        return 2;
    }
    lbm_solver *s = NULL;
    if (check(lbm_create(LBM_D3Q19, dims, 0.6, 3, LBM_STORE_F32, 1.0, ws, ws_bytes, stream, &s), "create")) return 1;
    if (check(lbm_set_fields(s, rho, u, LBM_MEM_HOST), "set_fields")) return 1;
    if (check(lbm_step(s, steps), "step")) return 1;
    double cons[4];
    if (check(lbm_conservation(s, cons), "conservation")) return 1;
    if (check(lbm_get_moments(s, rho, u, LBM_MEM_HOST), "get_moments")) return 1;
    int64_t t = 0;
    if (check(lbm_time(s, &t), "time")) return 1;
    printf("t %lld\n", (long long)t);
    printf("conservation %.17g %.17g %.17g %.17g\n", cons[0], cons[1], cons[2], cons[3]);
    const long long probe[3] = {0, C / 3 + 5, C - 1};
    for (int q = 0; q < 3; ++q) {
        const long long c = probe[q];
        printf("cell %lld %.17g %.17g %.17g %.17g\n", c, rho[c], u[c], u[C + c], u[2 * C + c]);
    }
    if (check(lbm_destroy(s), "destroy")) return 1;
    cudaStreamDestroy(stream);
    cudaFree(ws);
    free(rho);
    free(u);
    return 0;
}
